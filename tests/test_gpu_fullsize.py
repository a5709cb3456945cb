"""Element-wise GPU parity against the FP64 oracle at the full workload sizes.

* The 3D Tucker workload: 96 x 128 x 128 volume, 32 coils, ranks (32, 40, 40),
  q = 256, 3D Poisson-disc R = 8 with a 24 x 24 calibration box ("A Compression
  Scheme for Maxwell Basis", Eqs. 19-21; the operator of Eq. 5, its adjoint, the
  Jacobian of Eq. 7 and the Jacobian-adjoint display after it).  This is the only
  size that takes the 96-point pass along z, the coil-grouped x1 mode product
  and the coil-grouped core contraction.
* The batched exam's slice shapes: 192^2, 256^2 and 320^2 grids at 16 and 32
  coils with their q = 96 / 128 / 160 bases, through the recorded batch.

Tolerances: relative L2 <= 1e-5 (FP32 path), <= 5e-3 (BF16 path).
"""

import numpy as np
import pytest
import torch

import workloads as w
from oracle import fourier, operator as op, tucker

pytestmark = pytest.mark.gpu
TOL = {"fp32": 1e-5, "bf16": 5e-3}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def c64(x):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, dtype=np.complex64))).cuda()


def f64(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def q32(x):
    return np.asarray(x).astype(np.complex64).astype(np.complex128)


@pytest.fixture(scope="module")
def mp():
    import paper_2008_09042_gb300 as mp

    return mp


@pytest.fixture(scope="module")
def ctx(mp):
    return mp.Context(0)


@pytest.fixture(scope="module")
def c5():
    """Inputs of the 3D workload and the oracle's four operator outputs on them."""
    cfg = w.workload("cart3d_128x128x96_c32_tucker256")
    dims, C, q = cfg["dims"], cfg["C"], cfg["q"]
    core, fac = w.smooth_tucker_basis(dims, cfg["ranks"], q, seed=w.BASE_SEED)
    core, fac = q32(core), [q32(f) for f in fac]
    tb = tucker.TuckerBasis(core, fac)
    idx = w.mask_to_indices(w.poisson_disc_mask_3d(*dims, R=cfg["R"], calib=cfg["calib"], seed=w.BASE_SEED + 1))
    Fs = fourier.CartesianSampling(dims, idx)
    N = int(np.prod(dims))
    a = q32(w.random_coefficients(C, q, seed=31))
    da = q32(w.random_coefficients(C, q, seed=32))
    p = q32(w.random_ellipses(dims[1], dims[2], nz=dims[0], seed=33).ravel())
    dp = q32(w.random_image(N, seed=34))
    r = q32(w.random_coefficients(C, idx.size, seed=35, decay=False))
    ref = dict(y=op.forward(Fs, tb, a, p), x=op.adjoint(Fs, tb, a, r), dy=op.jacobian(Fs, tb, a, p, dp, da))
    ref["jp"], ref["ja"] = op.jacobian_adjoint(Fs, tb, a, p, r)
    return dict(dims=dims, C=C, q=q, core=core, fac=fac, idx=idx, a=a, da=da, p=p, dp=dp, r=r, ref=ref)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_tucker_operator_full_size(ctx, mp, c5, prec):
    tol = TOL[prec]
    plan = mp.Plan(ctx, c5["dims"], sample_idx=c5["idx"])
    B = mp.TuckerBasis(ctx, c5["core"], c5["fac"])
    ctx.reserve(plan, B, c5["C"])
    a, p, r = c64(c5["a"]), c64(c5["p"]), c64(c5["r"])
    ref = c5["ref"]
    assert rel(f64(mp.forward(ctx, plan, B, a, p, prec=prec)), ref["y"]) < tol
    assert rel(f64(mp.adjoint(ctx, plan, B, a, r, prec=prec)), ref["x"]) < tol
    assert rel(f64(mp.jacobian(ctx, plan, B, a, p, c64(c5["dp"]), c64(c5["da"]), prec=prec)), ref["dy"]) < tol
    gp, ga = mp.jacobian_adjoint(ctx, plan, B, a, p, r, prec=prec)
    assert rel(f64(gp), ref["jp"]) < tol
    assert rel(f64(ga), ref["ja"]) < tol
    ctx.synchronize()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_batched_exam_slice_shapes(ctx, mp, prec):
    cfg = w.workload("batched2d_64slices")
    shapes = [(192, 16), (256, 32), (320, 16), (320, 32)]
    slices, refs, bases = [], [], {}
    for i, (n, C) in enumerate(shapes):
        q = cfg["q_by_size"][n]
        U = q32(w.smooth_orthonormal_basis(n, n, q, seed=w.BASE_SEED + n))
        idx = w.mask_to_indices(w.poisson_disc_mask(n, n, 4 + i, calib=(24, 24), seed=w.BASE_SEED + 10 * n + i))
        plan = mp.Plan(ctx, (n, n), sample_idx=idx)
        if n not in bases:  # the two 320^2 slices share one basis: a grouped expansion
            bases[n] = mp.Basis(ctx, U.T)
        B = bases[n]
        a = q32(w.random_coefficients(C, q, seed=40 + i))
        p = q32(w.random_ellipses(n, n, seed=50 + i).ravel())
        slices.append(dict(plan=plan, basis=B, alpha=c64(a), p=c64(p),
                           y=torch.empty((C, idx.size), dtype=torch.complex64, device="cuda"),
                           x=torch.empty((n * n,), dtype=torch.complex64, device="cuda")))
        refs.append((fourier.CartesianSampling((n, n), idx), U, a, p))
    batch = mp.Batch(ctx, slices, kind="pair", prec=prec)
    assert batch.groups() == 1
    batch.run()
    ctx.synchronize()
    for s, (Fs, U, a, p) in zip(slices, refs):
        y_ref = op.forward(Fs, U, a, p)
        assert rel(f64(s["y"]), y_ref) < TOL[prec]
        # the batch's adjoint input is its own forward output
        assert rel(f64(s["x"]), op.adjoint(Fs, U, a, f64(s["y"]))) < TOL[prec]
    batch.close()
