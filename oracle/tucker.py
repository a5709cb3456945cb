"""Tucker-compressed basis in FP64 ("A Compression Scheme for Maxwell Basis").

Test infrastructure (see the package header).

Each basis column reshaped onto the (n1, n2, n3) voxel grid (raster order, mode
1 slowest) forms, over the q columns, a 4-way tensor T (n1, n2, n3, q).  The
factors U1, U2, U3 are shared by all columns and the fourth mode is left
uncompressed, so T ~ G x1 U1 x2 U2 x3 U3 with a core G (r1, r2, r3, q) (Eqs. 19-20;
the paper's reduced factors are read as n_k x r_k).  The k-mode product is the
contraction C_ijk = sum_p A_pjk B_ip written under Eq. 19.

HOSVD: U_k = leading left singular vectors of the mode-k unfolding; the core is
T x1 U1^H x2 U2^H x3 U3^H.  Truncation to accuracy eps keeps, per mode, the
fewest singular values whose discarded energy is at most eps^2 ||T||^2 / 3, so
that ||T - T~|| <= eps ||T|| (Eq. 21).
"""

import numpy as np


def mode_product(A, B, mode):
    """A x_mode B: contract axis ``mode`` of A with the second index of B."""
    out = np.tensordot(A, B, axes=([mode], [1]))  # contracted axis moved to the end
    return np.moveaxis(out, -1, mode)


def hosvd(T, ranks=None, eps=None):
    """Return (core, [U1, U2, U3]) for a (n1, n2, n3, q) tensor."""
    T = np.asarray(T, dtype=np.complex128)
    norm2 = np.sum(np.abs(T) ** 2)
    factors = []
    for mode in range(3):
        unf = np.moveaxis(T, mode, 0).reshape(T.shape[mode], -1)
        Uk, sk, _ = np.linalg.svd(unf, full_matrices=False)
        if ranks is not None:
            r = int(ranks[mode])
        elif eps is not None:
            tail = np.cumsum((sk ** 2)[::-1])[::-1]  # tail[i] = sum_{j >= i} s_j^2
            budget = eps ** 2 * norm2 / 3.0
            r = int(np.argmax(np.append(tail, 0.0) <= budget))
            r = max(r, 1)
        else:
            r = unf.shape[0]
        factors.append(Uk[:, :r])
    core = T
    for mode in range(3):
        core = mode_product(core, factors[mode].conj().T, mode)
    return core, factors


def tucker_full(core, factors):
    """Rebuild the (n1, n2, n3, q) tensor from core and factors."""
    T = core
    for mode in range(3):
        T = mode_product(T, factors[mode], mode)
    return T


class TuckerBasis:
    """Basis U in C^{N x q} held as a Tucker core and factors."""

    def __init__(self, core, factors):
        self.core = np.asarray(core, dtype=np.complex128)
        self.factors = [np.asarray(f, dtype=np.complex128) for f in factors]
        self.n = tuple(f.shape[0] for f in self.factors)
        self.r = tuple(f.shape[1] for f in self.factors)
        self.q = self.core.shape[3]
        self.N = int(np.prod(self.n))

    def expand(self, alpha):
        """s_k = (G x4 alpha_k^T) x1 U1 x2 U2 x3 U3, flattened; returns (C, N)."""
        alpha = np.atleast_2d(alpha)
        out = np.empty((alpha.shape[0], self.N), dtype=np.complex128)
        for c in range(alpha.shape[0]):
            gk = np.tensordot(self.core, alpha[c], axes=([3], [0]))  # (r1, r2, r3)
            for mode in range(3):
                gk = mode_product(gk, self.factors[mode], mode)
            out[c] = gk.ravel()
        return out

    def adjoint_expand(self, V):
        """U^H v_k for every row of V (C, N); returns (C, q)."""
        V = np.atleast_2d(V)
        out = np.empty((V.shape[0], self.q), dtype=np.complex128)
        for c in range(V.shape[0]):
            t = V[c].reshape(self.n)
            for mode in range(3):
                t = mode_product(t, self.factors[mode].conj().T, mode)
            out[c] = np.tensordot(self.core.conj(), t, axes=([0, 1, 2], [0, 1, 2]))
        return out

    def dense(self):
        return tucker_full(self.core, self.factors).reshape(self.N, self.q)
