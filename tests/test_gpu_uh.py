"""GPU parity of the Jacobian adjoint's coefficient block on the tensor cores.

dalpha_c = U^H (conj(p) F_s^H r_c) (the Jacobian-adjoint display after Eq. 7)
runs as a split-K GEMM over the pixels: 3xTF32 for FP32, BF16 operands for
BF16, with a fixed-order reduction of the partial tiles.  The shapes cover two
M blocks of basis indices (q > 128), coil counts padded to 8 and split into
groups of 64, and pixel counts that end in a partial ring stage.  FP32 is held
to relative L2 <= 1e-5 against the FP64 oracle, BF16 to 5e-3.
"""

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


def _case(shape, C, q, seed):
    N = shape[0] * shape[1]
    rng = np.random.default_rng(seed)
    U = np.linalg.qr(rng.normal(size=(N, q)) + 1j * rng.normal(size=(N, q)))[0]
    U = U.astype(np.complex64).astype(np.complex128)
    mask = w.poisson_disc_mask(shape[0], shape[1], 3, calib=(12, 12), seed=seed + 1)
    idx = w.mask_to_indices(mask)
    a = w.random_coefficients(C, q, seed=seed + 2).astype(np.complex64).astype(np.complex128)
    p = w.random_image(N, seed=seed + 3).astype(np.complex64).astype(np.complex128)
    r = w.random_coefficients(C, idx.size, seed=seed + 4, decay=False).astype(np.complex64).astype(np.complex128)
    return U, idx, a, p, r


# q = 160 and 256 take two M blocks; C = 9 and 1 pad to 16 and 8 coil rows;
# C = 70 runs as coil groups of 64 and 6.  (Cartesian pixel counts are
# multiples of 256, so whole stages; the Tucker case below ends in a partial one.)
SHAPES = [((48, 64), 9, 160), ((96, 96), 1, 256), ((128, 128), 70, 24), ((256, 256), 16, 128), ((64, 64), 4, 32)]


@pytest.mark.parametrize("shape,C,q", SHAPES)
def test_coefficient_block_matches_oracle(ctx, mp, shape, C, q):
    U, idx, a, p, r = _case(shape, C, q, 100 + C + q)
    Fs = fourier.CartesianSampling(shape, idx)
    plan = mp.Plan(ctx, shape, sample_idx=idx)
    B = mp.Basis(ctx, U.T)
    rp, ra = op.jacobian_adjoint(Fs, U, a, p, r)
    res = {}
    for prec in ("fp32", "fp32_simt", "bf16"):
        gp, ga = mp.jacobian_adjoint(ctx, plan, B, c64(a), c64(p), c64(r), prec=prec)
        res[prec] = (f64(gp), f64(ga))
    ctx.synchronize()  # raises if a bounded wait ran out
    assert rel(res["fp32"][1], ra) < 1e-5
    assert rel(res["fp32"][0], rp) < 1e-5
    assert rel(res["fp32_simt"][1], ra) < 1e-5  # the CUDA-core contraction
    assert rel(res["fp32"][1], res["fp32_simt"][1]) < 5e-6
    assert rel(res["bf16"][1], ra) < 5e-3


@pytest.mark.parametrize("prec,name", [("fp32", "k_uh_tc<tf32x3>"), ("bf16", "k_uh_tc<bf16>")])
def test_coefficient_block_launches_and_is_reproducible(ctx, mp, prec, name):
    shape, C, q = (128, 96), 12, 64
    U, idx, a, p, r = _case(shape, C, q, 7)
    plan = mp.Plan(ctx, shape, sample_idx=idx)
    B = mp.Basis(ctx, U.T)
    ag, pg, rg = c64(a), c64(p), c64(r)
    mp.jacobian_adjoint(ctx, plan, B, ag, pg, rg, prec=prec)
    ctx.synchronize()
    ctx.profile(True)
    ctx.profile_read(reset=True)
    _, ga1 = mp.jacobian_adjoint(ctx, plan, B, ag, pg, rg, prec=prec)
    ctx.synchronize()
    _, kernels = ctx.profile_read(reset=True, kernels=True)
    ctx.profile(False)
    _, ga2 = mp.jacobian_adjoint(ctx, plan, B, ag, pg, rg, prec=prec)
    ctx.synchronize()
    assert kernels.get(name, (0, 0))[1] == 1
    assert kernels.get("k_uh_reduce", (0, 0))[1] == 1
    assert "k_uh_v" not in kernels and "k_reduce_partials" not in kernels
    # fixed split ranges and a fixed-order reduction: identical bits
    assert torch.equal(ga1, ga2)


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("bf16", 5e-3)])
def test_tucker_core_contraction_ragged(ctx, mp, prec, tol):
    # ranks (5, 6, 6): the core's contraction runs over R = 180 positions, 5.6
    # 32-position (FP32) stages and 2.8 64-position (BF16) stages; q = 160 takes
    # two M blocks
    dims, ranks, q, C = (16, 32, 48), (5, 6, 6), 160, 5
    core, fac = w.smooth_tucker_basis(dims, ranks, q, seed=31)
    core = core.astype(np.complex64).astype(np.complex128)
    fac = [f.astype(np.complex64).astype(np.complex128) for f in fac]
    tb = tucker.TuckerBasis(core, fac)
    mask = w.poisson_disc_mask_3d(*dims, R=3, calib=(6, 6), seed=32)
    idx = w.mask_to_indices(mask)
    Fs = fourier.CartesianSampling(dims, idx)
    N = int(np.prod(dims))
    a = w.random_coefficients(C, q, seed=33).astype(np.complex64).astype(np.complex128)
    p = w.random_image(N, seed=34).astype(np.complex64).astype(np.complex128)
    r = w.random_coefficients(C, idx.size, seed=35, decay=False).astype(np.complex64).astype(np.complex128)
    plan = mp.Plan(ctx, dims, sample_idx=idx)
    B = mp.TuckerBasis(ctx, core, fac)
    gp, ga = mp.jacobian_adjoint(ctx, plan, B, c64(a), c64(p), c64(r), prec=prec)
    rp, ra = op.jacobian_adjoint(Fs, tb, a, p, r)
    ctx.synchronize()
    assert rel(f64(gp), rp) < tol and rel(f64(ga), ra) < tol
