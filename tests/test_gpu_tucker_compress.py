"""GPU Tucker compression of a dense basis ("A Compression Scheme for Maxwell
Basis", Eqs. 19-21) and the GPU Maxwell basis of a 3D volume, against the FP64
oracle.

Compression: the same complex64 tensor goes to both sides.  Checked: the
ranks (the GPU may raise r3 by up to 3 so that r1 r2 r3 is a multiple of 4),
the error of the GPU's Tucker basis against T within its own bound and within
eps (Eq. 21), the bound within 1e-6 of the oracle's (FP64 eigenvalue tails) and
the compressed tensor within 1e-5 of the oracle's (relative to ||T||) at equal
ranks, and exact recovery of a tensor of exactly low multilinear rank.
"""

import numpy as np
import pytest
import torch

import workloads as w
from oracle import basis as ob, tucker as ot

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    import paper_2008_09042_gb300 as mp

    return mp


@pytest.fixture(scope="module")
def ctx(mp):
    return mp.Context(0)


def _sin_theta(U, Uref):
    Uo = np.linalg.qr(U)[0]
    return float(np.linalg.norm(Uo - Uref @ (Uref.conj().T @ Uo), 2))


def _expand_all(mp, ctx, B, q):
    """The q basis columns of a (Tucker) basis: the expansion of the identity."""
    eye = torch.eye(q, dtype=torch.complex64, device="cuda")
    return mp.basis_expand(ctx, B, eye).cpu().numpy().astype(np.complex128)  # (q, N)


def _maxwell_3d(shape, q, n_sites, L, seed):
    om = w.random_excitations(6 * n_sites, L, seed=seed)
    U, sv, src = ob.build_maxwell_basis_3d(*shape, q, n_sites=n_sites, omega=om)
    return U, sv, src, om


def test_maxwell_basis_3d_matches_oracle(ctx, mp):
    shape, q = (8, 12, 16), 24
    U_ref, sv_ref, src, om = _maxwell_3d(shape, q, 12, 60, seed=21)
    U, sv = mp.maxwell_basis_3d(ctx, shape, q, src, om)
    ctx.synchronize()
    U = U.cpu().numpy().astype(np.complex128).T
    assert np.max(np.abs(sv - sv_ref[:sv.size])) <= 1e-10 * sv_ref[0]
    for qq in (8, 16, 24):
        assert sv_ref[qq - 1] > 1.05 * sv_ref[qq]
        assert _sin_theta(U[:, :qq], U_ref[:, :qq]) < 1e-5


@pytest.mark.parametrize("shape,q,eps", [((12, 16, 20), 24, 1e-4), ((16, 24, 8), 32, 1e-3), ((20, 12, 16), 16, 1e-5)])
def test_compress_matches_oracle_hosvd(ctx, mp, shape, q, eps):
    U, _, _, _ = _maxwell_3d(shape, q, 16, 96, seed=31 + q)
    T = U.T.astype(np.complex64)  # (q, N): [q][n1][n2][n3]
    Tt = T.astype(np.complex128).T.reshape(*shape, q)
    core_ref, fac_ref = ot.hosvd(Tt, eps=eps)
    r_ref = [f.shape[1] for f in fac_ref]
    norm2 = np.sum(np.abs(Tt) ** 2)
    tails = 0.0
    for mode in range(3):
        unf = np.moveaxis(Tt, mode, 0).reshape(shape[mode], -1)
        s = np.linalg.svd(unf, compute_uv=False)
        tails += np.sum(s[r_ref[mode]:] ** 2)
    bound_ref = np.sqrt(tails / norm2)
    B = mp.tucker_compress(ctx, torch.from_numpy(T).cuda(), shape, eps)
    ctx.synchronize()
    r = list(B.ranks)
    assert r[0] == r_ref[0] and r[1] == r_ref[1] and r_ref[2] <= r[2] <= r_ref[2] + 3
    assert (r[0] * r[1] * r[2]) % 4 == 0
    assert B.bound <= eps
    if r == r_ref:
        assert abs(B.bound - bound_ref) <= 1e-6
    That = _expand_all(mp, ctx, B, q)  # (q, N): the GPU's Tucker basis, column by column
    Tn = np.linalg.norm(T)
    err = np.linalg.norm(That - T.astype(np.complex128)) / Tn
    assert err <= B.bound + 1e-6  # FP32 core and factors on top of the truncation
    # at equal ranks both sides project T onto the same mode subspaces: the two
    # compressed tensors agree to single precision (a factor subspace off by d
    # moves the result by about d times T's energy at the truncation boundary)
    T_ref = ot.tucker_full(core_ref, fac_ref).reshape(-1, q).T
    if r == r_ref:
        assert np.linalg.norm(That - T_ref) / Tn < 1e-5
    else:
        assert np.linalg.norm(That - T_ref) / Tn < 2 * eps


def test_compress_recovers_exact_low_rank(ctx, mp):
    shape, ranks, q = (16, 20, 24), (4, 6, 5), 12
    core, fac = w.smooth_tucker_basis(shape, ranks, q, seed=41)
    T = ot.tucker_full(core, fac).reshape(-1, q).T.astype(np.complex64)  # (q, N)
    B = mp.tucker_compress(ctx, torch.from_numpy(T).cuda(), shape, 1e-4)
    ctx.synchronize()
    assert B.ranks[0] == 4 and B.ranks[1] == 6 and 5 <= B.ranks[2] <= 8
    That = _expand_all(mp, ctx, B, q)
    assert np.linalg.norm(That - T) / np.linalg.norm(T) < 1e-5


def test_compress_rejects_bad_arguments(ctx, mp):
    T = torch.zeros((4, 8 * 8 * 6), dtype=torch.complex64, device="cuda")
    with pytest.raises(mp.MpiError):
        mp.tucker_compress(ctx, T, (8, 8, 6), 0.0)  # eps must be > 0
    with pytest.raises(mp.MpiError):
        mp.tucker_compress(ctx, torch.zeros((4, 300 * 4 * 2), dtype=torch.complex64, device="cuda"), (300, 4, 2))
