"""GPU parity of dynamic MPI-L (frames with their own sampling, shared coil
maps, TV over the (t, y, x) grid) against the FP64 oracle: NRMSE <= 1e-3 on the
frames and the same rho decisions; T = 1 is the single-frame solve."""

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
def movie():
    # T frames of a 64 x 64 slice whose ellipses drift by a pixel per frame, each
    # frame sampled by its own variable-density line pattern (R = 4, 8 ACS lines)
    ny = nx = 64
    C, q, T = 4, 32, 4
    b = obasis.build_maxwell_basis_2d(ny, nx, q, n_sites=32, n_exc=200, seed=0)
    U = b.U.astype(np.complex64).astype(np.complex128)
    a = solvers.project_onto_basis(U, obasis.coil_maps_2d(ny, nx, C)).astype(np.complex64).astype(np.complex128)
    base = w.random_ellipses(ny, nx, seed=1)
    frames = np.stack([np.roll(base, t, axis=1).ravel() for t in range(T)]).astype(np.complex128)
    Fs_t, idx_t, ys = [], [], []
    for t in range(T):
        idx = w.mask_to_indices(w.vd_lines_mask(ny, nx, 4, 8, seed=10 + t))
        Fs = fourier.CartesianSampling((ny, nx), idx)
        y0 = op.forward(Fs, U, a, frames[t])
        sig = w.noise_sigma_for_snr(y0, 30.0)
        ys.append((y0 + w.complex_noise(y0.shape, sig, seed=20 + t)).astype(np.complex64).astype(np.complex128))
        Fs_t.append(Fs)
        idx_t.append(idx)
    y = np.stack(ys)
    sig = w.noise_sigma_for_snr(y, 30.0)
    eps = np.full((T, C), sig * np.sqrt(Fs_t[0].M))
    return dict(ny=ny, nx=nx, C=C, T=T, U=U, a=a, Fs_t=Fs_t, idx_t=idx_t, y=y, eps=eps)


def test_dynamic_image_solve_matches_oracle(ctx, mp, movie):
    m = movie
    plans = [mp.Plan(ctx, (m["ny"], m["nx"]), sample_idx=idx) for idx in m["idx_t"]]
    B = mp.Basis(ctx, m["U"].T)
    p, hist = mp.image_solve_dynamic(ctx, plans, B, c64(m["a"]), c64(m["y"]), m["eps"], n_outer=30, n_cg=5, n_tv=10)
    s = op.expand(m["U"], m["a"])
    p_ref, h_ref = solvers.admm_tv_dynamic(m["Fs_t"], s, m["y"], m["eps"], (m["ny"], m["nx"]),
                                           n_outer=30, n_cg=5, n_tv=10)
    assert nrmse(f64(p), p_ref) < 1e-3
    np.testing.assert_array_equal(hist[:, 2], h_ref[:, 2])  # same rho decisions


def test_one_frame_is_the_single_frame_solve(ctx, mp, movie):
    m = movie
    plan = mp.Plan(ctx, (m["ny"], m["nx"]), sample_idx=m["idx_t"][0])
    B = mp.Basis(ctx, m["U"].T)
    p1, h1 = mp.image_solve_dynamic(ctx, [plan], B, c64(m["a"]), c64(m["y"][:1]), m["eps"][:1], n_outer=10)
    p0, h0 = mp.image_solve(ctx, plan, B, c64(m["a"]), c64(m["y"][0]), m["eps"][0], n_outer=10)
    ctx.synchronize()
    assert torch.equal(p1[0], p0)
    np.testing.assert_array_equal(h1, h0)


def test_dynamic_rejects_mismatched_frames(ctx, mp, movie):
    m = movie
    B = mp.Basis(ctx, m["U"].T)
    plans = [mp.Plan(ctx, (m["ny"], m["nx"]), sample_idx=m["idx_t"][0]),
             mp.Plan(ctx, (m["ny"], m["nx"]), sample_idx=m["idx_t"][1][:-5])]  # fewer samples
    y = torch.zeros((2, m["C"], plans[0].M), dtype=torch.complex64, device="cuda")
    with pytest.raises(mp.MpiError, match="MPI_ERR_SHAPE"):
        mp.image_solve_dynamic(ctx, plans, B, c64(m["a"]), y, m["eps"][:2], n_outer=2)
