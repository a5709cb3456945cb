"""The Maxwell-parameterised bilinear encoding operator, FP64.

Test infrastructure (see the package header).

Notation: p in C^N the image, alpha in C^{C x q} the coil coefficients (row k
is alpha_k), U in C^{N x q} the basis, s_k = U alpha_k the coil maps,
F_s the sampling operator (any object with ``fwd``/``adj`` on (..., N) and
(..., M) arrays, see ``fourier`` and ``nufft``).  Every function is the plain
definition; nothing is fused or reordered.
"""

import numpy as np


def expand(U, alpha):
    """s_k = U alpha_k for every coil (Eq. 5); returns (C, N).

    ``U`` is a dense (N, q) array or an object with ``expand`` (the Tucker
    basis of ``oracle.tucker``).
    """
    if hasattr(U, "expand"):
        return U.expand(alpha)
    return np.asarray(alpha) @ np.asarray(U).T


def expand_adjoint(U, v):
    """U^H v_k for every row of v (C, N); returns (C, q)."""
    if hasattr(U, "adjoint_expand"):
        return U.adjoint_expand(v)
    return np.asarray(v) @ np.asarray(U).conj()


def forward(Fs, U, alpha, p):
    """G(p, alpha_1..alpha_C) = [F_s(U alpha_k (.) p)]_k (Eq. 5); returns (C, M)."""
    s = expand(U, alpha)
    return Fs.fwd(s * np.asarray(p)[None, :])


def forward_maps(Fs, s, p):
    """G(p, s_1..s_C) = [F_s(s_k (.) p)]_k with explicit maps (Eq. 3)."""
    return Fs.fwd(np.asarray(s) * np.asarray(p)[None, :])


def adjoint(Fs, U, alpha, y):
    """SENSE adjoint S^H F^H y = sum_k conj(s_k) (.) F_s^H y_k (Eq. 1); returns (N,)."""
    s = expand(U, alpha)
    return np.sum(s.conj() * Fs.adj(y), axis=0)


def jacobian(Fs, U, alpha, p, dp, dalpha):
    """J(p, alpha)[dp; dalpha] = [F_s(U alpha_k (.) dp + p (.) U dalpha_k)]_k (Eq. 7)."""
    s = expand(U, alpha)
    ds = expand(U, dalpha)
    p = np.asarray(p)
    return Fs.fwd(s * np.asarray(dp)[None, :] + p[None, :] * ds)


def jacobian_adjoint(Fs, U, alpha, p, r):
    """J^H r (the display after Eq. 7), with ^H on a vector inside (.) read as
    element-wise complex conjugation.

    Returns (dp, dalpha): dp = sum_k conj(U alpha_k) (.) F_s^H r_k  (N,)
                          dalpha_k = U^H (conj(p) (.) F_s^H r_k)   (C, q)
    """
    s = expand(U, alpha)
    w = Fs.adj(r)
    dp = np.sum(s.conj() * w, axis=0)
    v = np.asarray(p).conj()[None, :] * w
    dalpha = expand_adjoint(U, v)
    return dp, dalpha


# --- several sets of maps (Discussion, "Forward Model Extensions") ----------
#
# The signal equation with M sets of maps adds bilinear terms:
#   y_k = F_s( sum_m (U alpha_{m,k}) (.) p_m ),
# alphas (M, C, q), ps (M, N).  M = 1 is the model above.


def forward_multi(Fs, U, alphas, ps):
    """y_k = F_s(sum_m U alpha_{m,k} (.) p_m); returns (C, M_samples)."""
    v = sum(expand(U, a) * np.asarray(p)[None, :] for a, p in zip(alphas, ps))
    return Fs.fwd(v)


def adjoint_multi(Fs, U, alphas, y):
    """The adjoint in the images: [sum_k conj(U alpha_{m,k}) (.) F_s^H y_k]_m; returns (M, N)."""
    w = Fs.adj(y)
    return np.stack([np.sum(expand(U, a).conj() * w, axis=0) for a in alphas])


def jacobian_multi(Fs, U, alphas, ps, dps, dalphas):
    """J[dp; dalpha] = [F_s(sum_m U alpha_{m,k} (.) dp_m + p_m (.) U dalpha_{m,k})]_k."""
    v = sum(expand(U, a) * np.asarray(dp)[None, :] + np.asarray(p)[None, :] * expand(U, da)
            for a, p, dp, da in zip(alphas, ps, dps, dalphas))
    return Fs.fwd(v)


def jacobian_adjoint_multi(Fs, U, alphas, ps, r):
    """J^H r for M sets of maps: dp_m = sum_k conj(U alpha_{m,k}) (.) F_s^H r_k,
    dalpha_{m,k} = U^H (conj(p_m) (.) F_s^H r_k); returns ((M, N), (M, C, q))."""
    w = Fs.adj(r)
    dps = np.stack([np.sum(expand(U, a).conj() * w, axis=0) for a in alphas])
    dalphas = np.stack([expand_adjoint(U, np.asarray(p).conj()[None, :] * w) for p in ps])
    return dps, dalphas
