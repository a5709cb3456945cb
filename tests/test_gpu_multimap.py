"""GPU parity of the forward model with several sets of maps (Discussion,
"Forward Model Extensions": y_k = F_s(sum_m U alpha_{m,k} (.) p_m)) and of its
MPI-BL solver, against the FP64 oracle.  FP32 operators: relative L2 <= 1e-5;
BF16: <= 5e-3; the solver: NRMSE <= 1e-3 on the per-coil signal sum_m s_{m,k} p_m
and on each set's images and coefficients."""

import numpy as np
import pytest
import torch

import workloads as w
from oracle import basis as obasis, fourier, operator as op, solvers

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


def _case(shape, C, q, M, seed):
    N = shape[0] * shape[1]
    U = w.smooth_orthonormal_basis(shape[0], shape[1], q, seed=seed).astype(np.complex64).astype(np.complex128)
    mask = w.poisson_disc_mask(shape[0], shape[1], 4, calib=(12, 12), seed=seed + 1)
    idx = w.mask_to_indices(mask)
    A = np.stack([w.random_coefficients(C, q, seed=seed + 2 + m) for m in range(M)]).astype(np.complex64)
    P = np.stack([w.random_image(N, seed=seed + 10 + m) for m in range(M)]).astype(np.complex64)
    dA = np.stack([w.random_coefficients(C, q, seed=seed + 20 + m) for m in range(M)]).astype(np.complex64)
    dP = np.stack([w.random_image(N, seed=seed + 30 + m) for m in range(M)]).astype(np.complex64)
    r = w.random_coefficients(C, idx.size, seed=seed + 40, decay=False).astype(np.complex64)
    f = lambda x: x.astype(np.complex128)  # noqa: E731
    return U, idx, f(A), f(P), f(dA), f(dP), f(r)


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("bf16", 5e-3)])
@pytest.mark.parametrize("shape,C,q,M", [((64, 64), 4, 32, 2), ((128, 96), 8, 48, 3), ((256, 256), 16, 128, 2)])
def test_operator_family_matches_oracle(ctx, mp, shape, C, q, M, prec, tol):
    U, idx, A, P, dA, dP, r = _case(shape, C, q, M, 50 + M)
    Fs = fourier.CartesianSampling(shape, idx)
    plan = mp.Plan(ctx, shape, sample_idx=idx)
    B = mp.Basis(ctx, U.T)
    Ag, Pg = c64(A), c64(P)
    assert rel(f64(mp.forward_maps(ctx, plan, B, Ag, Pg, prec=prec)), op.forward_multi(Fs, U, A, P)) < tol
    assert rel(f64(mp.adjoint_maps(ctx, plan, B, Ag, c64(r), prec=prec)), op.adjoint_multi(Fs, U, A, r)) < tol
    assert rel(f64(mp.jacobian_maps(ctx, plan, B, Ag, Pg, c64(dP), c64(dA), prec=prec)),
               op.jacobian_multi(Fs, U, A, P, dP, dA)) < tol
    gp, ga = mp.jacobian_adjoint_maps(ctx, plan, B, Ag, Pg, c64(r), prec=prec)
    rp, ra = op.jacobian_adjoint_multi(Fs, U, A, P, r)
    ctx.synchronize()
    assert rel(f64(gp), rp) < tol and rel(f64(ga), ra) < tol


def test_one_set_is_the_single_set_call(ctx, mp):
    shape, C, q = (64, 64), 4, 32
    U, idx, A, P, dA, dP, r = _case(shape, C, q, 1, 60)
    plan = mp.Plan(ctx, shape, sample_idx=idx)
    B = mp.Basis(ctx, U.T)
    y1 = mp.forward_maps(ctx, plan, B, c64(A), c64(P))
    y0 = mp.forward(ctx, plan, B, c64(A[0]), c64(P[0]))
    ctx.synchronize()
    assert torch.equal(y1, y0)


def test_sm_estimate_two_sets_matches_oracle(ctx, mp):
    # data from two sets of maps on different images, 30 dB noise
    ny = nx = 64
    C, q, M = 4, 32, 2
    b = obasis.build_maxwell_basis_2d(ny, nx, q, n_sites=32, n_exc=200, seed=0)
    U = b.U.astype(np.complex64).astype(np.complex128)
    a1 = solvers.project_onto_basis(U, obasis.coil_maps_2d(ny, nx, C))
    a2 = 0.3 * w.random_coefficients(C, q, seed=71)
    A_true = np.stack([a1, a2])
    P_true = np.stack([w.random_ellipses(ny, nx, seed=72).ravel(), w.random_ellipses(ny, nx, seed=73).ravel()])
    idx = w.mask_to_indices(w.vd_lines_mask(ny, nx, 2, 16, seed=74))
    Fs = fourier.CartesianSampling((ny, nx), idx)
    y0 = op.forward_multi(Fs, U, A_true, P_true)
    y = (y0 + w.complex_noise(y0.shape, w.noise_sigma_for_snr(y0, 30.0), seed=75)).astype(np.complex64)
    y = y.astype(np.complex128)
    plan = mp.Plan(ctx, (ny, nx), sample_idx=idx)
    B = mp.Basis(ctx, U.T)
    a, p, hist = mp.sm_estimate_maps(ctx, plan, B, c64(y), C, M, n_outer=12, n_cg=10)
    P_ref, A_ref, h_ref = solvers.irgn_multi(Fs, U, y, C, q, M, n_outer=12, n_cg=10)
    a, p = f64(a), f64(p)
    sig = sum(op.expand(U, a[m]) * p[m][None] for m in range(M))
    sig_ref = sum(op.expand(U, A_ref[m]) * P_ref[m][None] for m in range(M))
    assert rel(sig, sig_ref) < 1e-3
    for m in range(M):
        assert rel(a[m], A_ref[m]) < 1e-3
        assert rel(p[m], P_ref[m]) < 1e-3
    assert np.allclose(hist, h_ref, rtol=1e-3)
    # the single-set solve of the same data stops at a higher residual
    _, _, h1 = mp.sm_estimate_maps(ctx, plan, B, c64(y), C, 1, n_outer=12, n_cg=10)
    assert hist[-1] < h1[-1]
