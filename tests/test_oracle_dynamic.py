"""Pins for the oracle's dynamic MPI-L (T frames with their own sampling, shared
coil maps, spatiotemporal TV; the constrained problem with a spatiotemporal
regulariser in "Regularized Density Reconstruction")."""

import numpy as np
from scipy.optimize import minimize

from oracle import fourier, solvers


def _frames(seed, T=2, ny=4, nx=4, n_samp=9, noise=0.05):
    rng = np.random.default_rng(seed)
    N = ny * nx
    yy, xx = np.mgrid[0:ny, 0:nx] / 4.0
    s = np.stack([np.exp(0.4j + 0.5 * xx) * (1 + 0.3 * yy), np.exp(-0.3j * yy) * (1.2 - 0.4 * xx)]).reshape(2, N)
    Fs_t, ys, ps = [], [], []
    for t in range(T):
        p = np.zeros((ny, nx))
        p[1:3, 1 + t % 2:3 + t % 2] = 1.0  # the object moves by a pixel from frame to frame
        p = p.ravel() + 0.05 * rng.normal(size=N)
        idx = np.sort(rng.choice(N, n_samp, replace=False))  # each frame its own pattern
        Fs = fourier.CartesianSampling((ny, nx), idx)
        Fs_t.append(Fs)
        ys.append(Fs.fwd(s * p[None]) + noise * (rng.normal(size=(2, n_samp)) + 1j * rng.normal(size=(2, n_samp))))
        ps.append(p)
    eps = np.full((T, 2), 0.25)
    return Fs_t, s, np.stack(ys), eps, (ny, nx)


def test_one_frame_is_admm_tv():
    Fs_t, s, y, eps, shape = _frames(1, T=1)
    p1, h1 = solvers.admm_tv_dynamic(Fs_t, s, y, eps, shape, n_outer=30, n_cg=8, n_tv=12)
    p0, h0 = solvers.admm_tv(Fs_t[0], s, y[0], eps[0], shape, n_outer=30, n_cg=8, n_tv=12)
    np.testing.assert_allclose(p1[0], p0, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(h1, h0, rtol=1e-12, atol=1e-12)


def test_rho_change_keeps_unscaled_dual():
    # residual balancing with scaled duals: every change of rho keeps rho * u
    events = []
    Fs_t, s, y, eps, shape = _frames(2, T=3)
    solvers.admm_tv_dynamic(Fs_t, s, y, eps, shape, n_outer=40, n_cg=6, n_tv=8, rho0=1e-3,
                            trace=lambda ev, rho, u0, uk: events.append((ev, rho, u0, uk)))
    changes = 0
    for (e1, r1, a1, b1), (e2, r2, a2, b2) in zip(events, events[1:]):
        if e2 == "rho":
            changes += 1
            np.testing.assert_allclose(r2 * a2, r1 * a1, rtol=1e-12, atol=1e-14)
            np.testing.assert_allclose(r2 * b2, r1 * b1, rtol=1e-12, atol=1e-14)
    assert changes > 0


def test_matches_generic_constrained_spatiotemporal_tv_minimiser():
    # min TV over (t, y, x) s.t. ||y_{k,t} - F_s^t S_k p_t|| <= eps_{k,t}, solved
    # independently by SLSQP on a smoothed TV (sqrt(|grad|^2 + delta)); the
    # oracle's ADMM must reach the same optimal value, feasibly.
    Fs_t, s, y, eps, shape = _frames(3, T=2)
    T, N = 2, Fs_t[0].N
    grid = (T,) + shape
    delta = 1e-12

    def unpack(z):
        return (z[:T * N] + 1j * z[T * N:]).reshape(T, N)

    def tv_smooth(z):
        g = solvers.grad_fd(unpack(z).reshape(grid))
        return float(np.sum(np.sqrt(np.sum(np.abs(g) ** 2, axis=0) + delta)))

    cons = [{"type": "ineq",
             "fun": lambda z, k=k, t=t: eps[t, k] ** 2 - np.sum(np.abs(y[t, k] - Fs_t[t].fwd(s[k] * unpack(z)[t])) ** 2)}
            for t in range(T) for k in range(2)]
    x0 = np.stack([np.sum(s.conj() * Fs_t[t].adj(y[t]), axis=0) / np.sum(np.abs(s) ** 2, axis=0) for t in range(T)])
    best = minimize(tv_smooth, np.concatenate([x0.real.ravel(), x0.imag.ravel()]), constraints=cons, method="SLSQP",
                    options=dict(maxiter=400, ftol=1e-14))
    p_ref = unpack(best.x)
    viol_ref = max(np.linalg.norm(y[t, k] - Fs_t[t].fwd(s[k] * p_ref[t])) / eps[t, k] for t in range(T) for k in range(2))
    assert viol_ref < 1 + 1e-6
    tv_ref = solvers.tv(p_ref.reshape(grid))
    p, _ = solvers.admm_tv_dynamic(Fs_t, s, y, eps, shape, n_outer=400, n_cg=2 * T * N, n_tv=100)
    viol = max(np.linalg.norm(y[t, k] - Fs_t[t].fwd(s[k] * p[t])) / eps[t, k] for t in range(T) for k in range(2))
    assert viol < 1 + 1e-4
    assert abs(solvers.tv(p.reshape(grid)) - tv_ref) < 1e-3 * tv_ref
