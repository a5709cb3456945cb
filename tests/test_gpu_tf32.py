"""GPU parity of the FP32 expansion on the tensor cores (3xTF32) against the FP64 oracle.

MPI_PREC_FP32 runs the basis expansion as three TF32 products of the split
operands (hi*hi + hi*lo + lo*hi), accumulated in FP32, wherever the coefficient
operand fits the kernel's shared-memory budget, and on the CUDA cores otherwise;
MPI_PREC_FP32_SIMT always takes the CUDA-core kernel.  Both must meet the FP32
operator tolerance, relative L2 <= 1e-5 against the oracle.
"""

import numpy as np
import pytest
import torch

import workloads as w
from oracle import fourier, operator as op

pytestmark = pytest.mark.gpu
TOL = 1e-5


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


def _basis(N, q, seed):
    rng = np.random.default_rng(seed)
    U = np.linalg.qr(rng.normal(size=(N, q)) + 1j * rng.normal(size=(N, q)))[0]
    return U.astype(np.complex64).astype(np.complex128)


# ragged last pixel tile (N = 4000, 23260, 38396), K padded to the 32-element
# chunk (2q = 40, 192, 320), one to eight K chunks, coefficient rows from 16 to
# 64; more tiles than CTAs, with a short (N = 23260) and a long (N = 38396) last
# wave on 152 SMs.
@pytest.mark.parametrize("N,C,q", [(256, 4, 32), (4000, 3, 20), (65536, 16, 128), (8192, 32, 96), (4096, 12, 160),
                                   (23260, 5, 40), (38396, 4, 24)])
def test_tf32_expand_shapes(ctx, mp, N, C, q):
    U = _basis(N, q, N + C)
    a = w.random_coefficients(C, q, seed=3).astype(np.complex64).astype(np.complex128)
    B = mp.Basis(ctx, U.T)
    ref = op.expand(U, a)
    assert mp.expand_path(ctx, B, C, "fp32") == "tf32x3"
    assert mp.expand_path(ctx, B, C, "fp32_simt") == "ffma"
    l0 = ctx.launches()
    s_tc = f64(mp.basis_expand(ctx, B, c64(a), prec="fp32"))
    l1 = ctx.launches()
    s_simt = f64(mp.basis_expand(ctx, B, c64(a), prec="fp32_simt"))
    ctx.synchronize()
    assert l1 - l0 == 1  # the coefficient operand is built inside the expansion kernel
    assert rel(s_tc, ref) < TOL
    assert rel(s_simt, ref) < TOL
    assert rel(s_tc, s_simt) < 5e-6


def test_tf32_coil_groups_for_wide_coefficients(ctx, mp):
    # 2C = 300 coefficient rows exceed one MMA's N: the coils run in groups on
    # the tensor cores, and the result is the same expansion
    N, C, q = 2048, 150, 24
    U = _basis(N, q, 5)
    a = w.random_coefficients(C, q, seed=6).astype(np.complex64).astype(np.complex128)
    B = mp.Basis(ctx, U.T)
    assert mp.expand_path(ctx, B, C, "fp32") == "tf32x3"
    l0 = ctx.launches()
    s = f64(mp.basis_expand(ctx, B, c64(a), prec="fp32"))
    assert ctx.launches() - l0 == 1  # the groups are grid rows of one launch
    ctx.synchronize()
    assert rel(s, op.expand(U, a)) < TOL


@pytest.mark.parametrize("prec", ["fp32", "fp32_simt"])
@pytest.mark.parametrize("shape,C,q", [((64, 64), 4, 32), ((256, 256), 16, 128), ((128, 192), 32, 64)])
def test_fp32_operator_family_matches_oracle(ctx, mp, prec, shape, C, q):
    # forward, adjoint, Jacobian (coefficient rows doubled) and Jacobian-adjoint;
    # at C = 32 the Jacobian's stacked [hi; lo] rows (256) leave no room for a
    # double-buffered accumulator, so that one call runs in two coil groups
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
    if prec == "fp32":
        assert mp.expand_path(ctx, B, C, prec) == "tf32x3"
        assert mp.expand_path(ctx, B, C, prec, jacobian=True) == "tf32x3"  # C = 32 runs in coil groups
    ag, pg = c64(a), c64(p)
    assert rel(f64(mp.forward(ctx, plan, B, ag, pg, prec=prec)), op.forward(Fs, U, a, p)) < TOL
    assert rel(f64(mp.adjoint(ctx, plan, B, ag, c64(r), prec=prec)), op.adjoint(Fs, U, a, r)) < TOL
    assert rel(f64(mp.jacobian(ctx, plan, B, ag, pg, c64(dp), c64(da), prec=prec)),
               op.jacobian(Fs, U, a, p, dp, da)) < TOL
    gp, ga = mp.jacobian_adjoint(ctx, plan, B, ag, pg, c64(r), prec=prec)
    rp, ra = op.jacobian_adjoint(Fs, U, a, p, r)
    assert rel(f64(gp), rp) < TOL and rel(f64(ga), ra) < TOL
    ctx.synchronize()  # raises if a bounded wait ran out


def test_tf32_reading_probe_and_cuda_core_route(mp):
    # The 3xTF32 kernels pass each raw FP32 tile as hi(x) and add lo(x) = x - hi(x)
    # separately, which is exact only if the tensor core reads an FP32 operand of
    # kind::tf32 by truncation to 19 bits.  The context measures that reading when
    # it is made; any other reading sends FP32 work to the CUDA-core kernels.  Here
    # the reading is checked, then the route taken with the 3xTF32 kernels switched
    # off is held to the same FP32 tolerance, dense and Tucker, every operator.
    from oracle import tucker

    ctx = mp.Context(0)
    assert ctx.tf32_reading() == "truncate"
    n, C, q = 64, 4, 24
    U = _basis(n * n, q, 5)
    idx = w.mask_to_indices(w.vd_lines_mask(n, n, 3, 16, seed=2))
    Fs = fourier.CartesianSampling((n, n), idx)
    plan = mp.Plan(ctx, (n, n), sample_idx=idx)
    B = mp.Basis(ctx, U.T)
    a2 = w.random_coefficients(C, q, seed=3).astype(np.complex64).astype(np.complex128)
    p2 = w.random_image(n * n, seed=4).astype(np.complex64).astype(np.complex128)
    y_ref = op.forward(Fs, U, a2, p2)
    assert mp.expand_path(ctx, B, C) == "tf32x3"
    ctx.set_tf32x3(False)
    assert mp.expand_path(ctx, B, C) == "ffma"
    ctx.profile(True)
    ctx.profile_read(reset=True)

    def four_operators(plan, B, Fs, basis_ref, a, p, N, M, Cn, qn):
        dp = w.random_image(N, seed=5).astype(np.complex64).astype(np.complex128)
        da = w.random_coefficients(Cn, qn, seed=6).astype(np.complex64).astype(np.complex128)
        r = w.random_coefficients(Cn, M, seed=7, decay=False).astype(np.complex64).astype(np.complex128)
        ag, pg = c64(a), c64(p)
        assert rel(f64(mp.forward(ctx, plan, B, ag, pg)), op.forward(Fs, basis_ref, a, p)) < TOL
        assert rel(f64(mp.adjoint(ctx, plan, B, ag, c64(r))), op.adjoint(Fs, basis_ref, a, r)) < TOL
        assert rel(f64(mp.jacobian(ctx, plan, B, ag, pg, c64(dp), c64(da))),
                   op.jacobian(Fs, basis_ref, a, p, dp, da)) < TOL
        gp, ga = mp.jacobian_adjoint(ctx, plan, B, ag, pg, c64(r))
        rp, ra = op.jacobian_adjoint(Fs, basis_ref, a, p, r)
        assert rel(f64(gp), rp) < TOL and rel(f64(ga), ra) < TOL

    four_operators(plan, B, Fs, U, a2, p2, n * n, idx.size, C, q)

    dims, ranks, qt, Ct = (16, 32, 48), (4, 6, 8), 12, 3
    core, fac = w.smooth_tucker_basis(dims, ranks, qt, seed=1)
    core = core.astype(np.complex64).astype(np.complex128)
    fac = [f.astype(np.complex64).astype(np.complex128) for f in fac]
    idx3 = w.mask_to_indices(w.poisson_disc_mask_3d(*dims, R=3, calib=(6, 6), seed=2))
    N3 = int(np.prod(dims))
    a3 = w.random_coefficients(Ct, qt, seed=3).astype(np.complex64).astype(np.complex128)
    p3 = w.random_image(N3, seed=4).astype(np.complex64).astype(np.complex128)
    four_operators(mp.Plan(ctx, dims, sample_idx=idx3), mp.TuckerBasis(ctx, core, fac),
                   fourier.CartesianSampling(dims, idx3), tucker.TuckerBasis(core, fac), a3, p3, N3, idx3.size,
                   Ct, qt)
    ctx.synchronize()
    _, kernels = ctx.profile_read(kernels=True)
    assert kernels and not any("tf32" in k or "k_uh_tc" in k for k in kernels), sorted(kernels)
    ctx.profile(False)
    # back on: the tensor-core route again, same result
    ctx.set_tf32x3(True)
    assert mp.expand_path(ctx, B, C) == "tf32x3"
    assert rel(f64(mp.forward(ctx, plan, B, c64(a2), c64(p2))), y_ref) < TOL
    ctx.synchronize()
