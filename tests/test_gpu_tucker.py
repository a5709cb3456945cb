"""GPU parity of the Tucker-factored (3D) operator path against the FP64 oracle
("A Compression Scheme for Maxwell Basis", Eqs. 19-21)."""

import numpy as np
import pytest
import torch

import workloads as w
from oracle import fourier, operator as op, tucker

pytestmark = pytest.mark.gpu


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


def _tucker(dims, ranks, q, seed):
    core, fac = w.smooth_tucker_basis(dims, ranks, q, seed=seed)
    core = core.astype(np.complex64).astype(np.complex128)
    fac = [f.astype(np.complex64).astype(np.complex128) for f in fac]
    return core, fac


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("bf16", 5e-3)])
def test_tucker_operator_small(ctx, mp, prec, tol):
    dims, ranks, q, C = (16, 32, 48), (4, 6, 8), 12, 3
    core, fac = _tucker(dims, ranks, q, seed=1)
    tb = tucker.TuckerBasis(core, fac)
    mask = w.poisson_disc_mask_3d(*dims, R=3, calib=(6, 6), seed=2)
    idx = w.mask_to_indices(mask)
    Fs = fourier.CartesianSampling(dims, idx)
    N = int(np.prod(dims))
    a = w.random_coefficients(C, q, seed=3).astype(np.complex64).astype(np.complex128)
    p = w.random_image(N, seed=4).astype(np.complex64).astype(np.complex128)
    dp = w.random_image(N, seed=5).astype(np.complex64).astype(np.complex128)
    da = w.random_coefficients(C, q, seed=6).astype(np.complex64).astype(np.complex128)
    r = w.random_coefficients(C, idx.size, seed=7, decay=False).astype(np.complex64).astype(np.complex128)
    plan = mp.Plan(ctx, dims, sample_idx=idx)
    B = mp.TuckerBasis(ctx, core, fac)
    ag, pg = c64(a), c64(p)
    assert rel(f64(mp.basis_expand(ctx, B, ag, prec=prec)), op.expand(tb, a)) < tol
    assert rel(f64(mp.forward(ctx, plan, B, ag, pg, prec=prec)), op.forward(Fs, tb, a, p)) < tol
    assert rel(f64(mp.adjoint(ctx, plan, B, ag, c64(r), prec=prec)), op.adjoint(Fs, tb, a, r)) < tol
    assert rel(f64(mp.jacobian(ctx, plan, B, ag, pg, c64(dp), c64(da), prec=prec)),
               op.jacobian(Fs, tb, a, p, dp, da)) < tol
    gp, ga = mp.jacobian_adjoint(ctx, plan, B, ag, pg, c64(r), prec=prec)
    rp, ra = op.jacobian_adjoint(Fs, tb, a, p, r)
    assert rel(f64(gp), rp) < tol and rel(f64(ga), ra) < tol
    ctx.synchronize()


def test_tucker_full_size_maps_and_adjointness(ctx, mp):
    # the 128 x 128 x 96 volume, ranks (32, 40, 40), q = 256 Tucker basis
    dims, ranks, q = (96, 128, 128), (32, 40, 40), 256
    core, fac = _tucker(dims, ranks, q, seed=8)
    tb = tucker.TuckerBasis(core, fac)
    B = mp.TuckerBasis(ctx, core, fac)
    C = 2
    a = w.random_coefficients(C, q, seed=9).astype(np.complex64).astype(np.complex128)
    s = f64(mp.basis_expand(ctx, B, c64(a)))
    ref = op.expand(tb, a)
    assert rel(s, ref) < 1e-5
    # operator adjointness at full size with 32 coils (a property that holds at any size)
    C = 32
    mask = w.poisson_disc_mask_3d(*dims, R=8, calib=(24, 24), seed=10)
    idx = w.mask_to_indices(mask)
    assert idx.size == 128 * round(96 * 128 / 8)
    plan = mp.Plan(ctx, dims, sample_idx=idx)
    N = int(np.prod(dims))
    a = c64(w.random_coefficients(C, q, seed=11))
    p = c64(w.random_image(N, seed=12))
    r = c64(w.random_coefficients(C, idx.size, seed=13, decay=False))
    y = mp.forward(ctx, plan, B, a, p)
    x = mp.adjoint(ctx, plan, B, a, r)
    lhs = torch.vdot(y.flatten().to(torch.complex128), r.flatten().to(torch.complex128)).item()
    rhs = torch.vdot(p.to(torch.complex128), x.to(torch.complex128)).item()
    assert abs(lhs - rhs) / abs(lhs) < 1e-5
    ctx.synchronize()


@pytest.mark.parametrize("dims,ranks,prec", [
    ((64, 32, 64), (16, 8, 8), "fp32"),     # n1 = 64, r1 < 32 (zero-padded K)
    ((64, 32, 64), (32, 12, 10), "bf16"),
    ((96, 16, 64), (24, 8, 8), "fp32"),
    ((128, 16, 64), (32, 8, 8), "bf16"),    # n1 = 128: BF16 only on the fused kernel
    ((128, 16, 64), (32, 8, 8), "fp32"),    # ... FP32 takes the unfused passes
])
def test_tucker_fused_x1_shapes(ctx, mp, dims, ranks, prec):
    # forward and adjoint through the x1 kernel fused with the point-wise step and
    # the DFT along z (forward) or the sum over coils (adjoint), every coil count
    # path, against the oracle
    tol = 1e-5 if prec == "fp32" else 5e-3
    q, C = 20, 5
    core, fac = _tucker(dims, ranks, q, seed=21)
    tb = tucker.TuckerBasis(core, fac)
    idx = w.mask_to_indices(w.poisson_disc_mask_3d(*dims, R=4, calib=(8, 8), seed=22))
    Fs = fourier.CartesianSampling(dims, idx)
    N = int(np.prod(dims))
    a = w.random_coefficients(C, q, seed=23).astype(np.complex64).astype(np.complex128)
    p = w.random_image(N, seed=24).astype(np.complex64).astype(np.complex128)
    r = w.random_coefficients(C, idx.size, seed=25, decay=False).astype(np.complex64).astype(np.complex128)
    plan = mp.Plan(ctx, dims, sample_idx=idx)
    B = mp.TuckerBasis(ctx, core, fac)
    for rep in range(2):  # a second call reuses the cached operand tensor map
        assert rel(f64(mp.forward(ctx, plan, B, c64(a), c64(p), prec=prec)), op.forward(Fs, tb, a, p)) < tol
        assert rel(f64(mp.adjoint(ctx, plan, B, c64(a), c64(r), prec=prec)), op.adjoint(Fs, tb, a, r)) < tol
    ctx.synchronize()
