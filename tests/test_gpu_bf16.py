"""GPU parity of the BF16 tensor-core expansion path (tcgen05) against the FP64 oracle.

The BF16 path rounds the basis and coefficients to BF16 and accumulates in
FP32; operator outputs must stay within relative L2 5e-3 of the FP64 oracle
(the FP32 operator tolerance is 1e-5).
"""

import numpy as np
import pytest
import torch

import workloads as w
from oracle import fourier, nufft, operator as op

pytestmark = pytest.mark.gpu
TOL = 5e-3


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def c64(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, dtype=np.complex64))).cuda()


def f64(t):
    return t.detach().cpu().numpy().astype(np.complex128)


@pytest.fixture(scope="module")
def mp():
    import paper_2008_09042_gb300 as mp

    return mp


@pytest.fixture(scope="module")
def ctx(mp):
    return mp.Context(0)


def test_bf16_expand_small_single_tile(ctx, mp):
    n, C, q = 16, 4, 32  # N = 256: two 128-pixel tiles, one 64-wide K chunk, MMA N = 16
    U = w.smooth_orthonormal_basis(n, n, q, seed=1).astype(np.complex64).astype(np.complex128)
    a = w.random_coefficients(C, q, seed=2).astype(np.complex64).astype(np.complex128)
    B = mp.Basis(ctx, U.T)
    s = f64(mp.basis_expand(ctx, B, c64(a), prec="bf16"))
    ctx.synchronize()
    assert rel(s, op.expand(U, a)) < TOL


@pytest.mark.parametrize("N,C,q", [(4000, 3, 20), (65536, 16, 128), (8192, 32, 96), (4096, 12, 160)])
def test_bf16_expand_shapes(ctx, mp, N, C, q):
    # ragged last pixel tile (N = 4000), padded K (2q not a multiple of 64), odd coil counts
    rng = np.random.default_rng(N + C)
    U = np.linalg.qr(rng.normal(size=(N, q)) + 1j * rng.normal(size=(N, q)))[0]
    U = U.astype(np.complex64).astype(np.complex128)
    a = w.random_coefficients(C, q, seed=3).astype(np.complex64).astype(np.complex128)
    B = mp.Basis(ctx, U.T)
    s = f64(mp.basis_expand(ctx, B, c64(a), prec="bf16"))
    ctx.synchronize()
    assert rel(s, op.expand(U, a)) < TOL


@pytest.mark.parametrize("shape,C,q", [((64, 64), 4, 32), ((256, 256), 16, 128), ((128, 192), 32, 64)])
def test_bf16_operator_matches_oracle(ctx, mp, shape, C, q):
    U = w.smooth_orthonormal_basis(shape[0], shape[1], q, seed=4).astype(np.complex64).astype(np.complex128)
    mask = w.poisson_disc_mask(shape[0], shape[1], 4, calib=(12, 12), seed=5)
    idx = w.mask_to_indices(mask)
    Fs = fourier.CartesianSampling(shape, idx)
    N = shape[0] * shape[1]
    a = w.random_coefficients(C, q, seed=6).astype(np.complex64).astype(np.complex128)
    p = w.random_image(N, seed=7).astype(np.complex64).astype(np.complex128)
    dp = w.random_image(N, seed=8).astype(np.complex64).astype(np.complex128)
    da = w.random_coefficients(C, q, seed=9).astype(np.complex64).astype(np.complex128)
    r = w.random_coefficients(C, idx.size, seed=10, decay=False).astype(np.complex64).astype(np.complex128)
    plan = mp.Plan(ctx, shape, sample_idx=idx)
    B = mp.Basis(ctx, U.T)
    ag, pg = c64(a), c64(p)
    assert rel(f64(mp.forward(ctx, plan, B, ag, pg, prec="bf16")), op.forward(Fs, U, a, p)) < TOL
    assert rel(f64(mp.adjoint(ctx, plan, B, ag, c64(r), prec="bf16")), op.adjoint(Fs, U, a, r)) < TOL
    assert rel(f64(mp.jacobian(ctx, plan, B, ag, pg, c64(dp), c64(da), prec="bf16")),
               op.jacobian(Fs, U, a, p, dp, da)) < TOL
    gp, ga = mp.jacobian_adjoint(ctx, plan, B, ag, pg, c64(r), prec="bf16")
    rp, ra = op.jacobian_adjoint(Fs, U, a, p, r)
    assert rel(f64(gp), rp) < TOL and rel(f64(ga), ra) < TOL
    ctx.synchronize()  # raises if a bounded wait ran out


def test_bf16_radial(ctx, mp):
    n, C, q = 64, 3, 16
    k = w.golden_angle_radial(16, 128).astype(np.float32)
    U = w.smooth_orthonormal_basis(n, n, q, seed=11).astype(np.complex64).astype(np.complex128)
    a = w.random_coefficients(C, q, seed=12).astype(np.complex64).astype(np.complex128)
    p = w.random_image(n * n, seed=13).astype(np.complex64).astype(np.complex128)
    plan = mp.Plan(ctx, (n, n), traj=k)
    B = mp.Basis(ctx, U.T)
    kb = nufft.KBGriddingNUFFT((n, n), k.astype(np.float64))
    y = f64(mp.forward(ctx, plan, B, c64(a), c64(p), prec="bf16"))
    assert rel(y, op.forward(kb, U, a, p)) < TOL
