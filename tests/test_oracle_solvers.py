"""Pins for the oracle's solvers: CG, TV prox, ball projection, basis projection,
IRGN (MPI-BL, Eq. 6) and ADMM (MPI-L, Eqs. 8-11)."""

import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import basis, fourier, operator as op, solvers
import workloads as w


def _cn(rng, *shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def test_cg_solves_hpd_system():
    rng = np.random.default_rng(0)
    n = 12
    A = _cn(rng, n, n)
    A = A.conj().T @ A + n * np.eye(n)
    b = _cn(rng, n)
    (x,) = solvers.cg(lambda v: [A @ v[0]], (b,), (np.zeros(n),), n)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), atol=1e-9)


def test_grad_fd_adjoint_and_constant_kernel():
    rng = np.random.default_rng(1)
    x = _cn(rng, 5, 7)
    P = _cn(rng, 2, 5, 7)
    assert np.isclose(np.vdot(solvers.grad_fd(x), P), np.vdot(x, solvers.grad_fd_adj(P)))
    assert np.allclose(solvers.grad_fd(np.full((5, 7), 2.0 + 1j)), 0)


def test_tv_prox_matches_generic_minimiser():
    # brute force: minimise (1/2)||x - v||^2 + lam TV(x) over R^{2n} with BFGS
    rng = np.random.default_rng(2)
    shape = (3, 4)
    v = _cn(rng, *shape).ravel()
    lam = 0.3

    def obj(z):
        x = (z[:12] + 1j * z[12:]).reshape(shape)
        g = solvers.grad_fd(x)
        return 0.5 * np.sum(np.abs(x.ravel() - v) ** 2) + lam * np.sum(
            np.sqrt(np.sum(np.abs(g) ** 2, axis=0) + 1e-14))

    z0 = np.concatenate([v.real, v.imag])
    res = minimize(obj, z0, method="Powell", options=dict(xtol=1e-10, ftol=1e-14, maxiter=200000))
    x_ref = res.x[:12] + 1j * res.x[12:]
    x = solvers.tv_prox(v, lam, shape, 3000)
    f_ref = obj(np.concatenate([x_ref.real, x_ref.imag]))
    f_fgp = obj(np.concatenate([x.real, x.imag]))
    assert f_fgp <= f_ref + 1e-6
    assert np.linalg.norm(x - x_ref) < 1e-2 * np.linalg.norm(v)


def test_tv_prox_limits():
    rng = np.random.default_rng(3)
    v = _cn(rng, 6 * 6)
    np.testing.assert_allclose(solvers.tv_prox(v, 0.0, (6, 6), 10), v)
    c = np.full(36, 0.5 - 0.2j)
    np.testing.assert_allclose(solvers.tv_prox(c, 1.0, (6, 6), 10), c, atol=1e-14)
    # a huge weight flattens the image to its mean
    x = solvers.tv_prox(v, 1e4, (6, 6), 500)
    np.testing.assert_allclose(x, np.full(36, v.mean()), atol=1e-3)


def test_project_ball():
    rng = np.random.default_rng(4)
    y = _cn(rng, 3, 10)
    eps = np.array([0.5, 2.0, 100.0])
    z = y + _cn(rng, 3, 10)
    pz = solvers.project_ball(z, y, eps)
    d = np.linalg.norm(z - y, axis=1)
    for k in range(3):
        if d[k] <= eps[k]:
            np.testing.assert_allclose(pz[k], z[k])
        else:
            assert np.isclose(np.linalg.norm(pz[k] - y[k]), eps[k])
            # the projection lies on the segment from y to z
            t = (pz[k] - y[k]) / (z[k] - y[k])
            assert np.allclose(t, t[0]) and np.isclose(t[0].imag, 0)


def test_project_onto_basis():
    rng = np.random.default_rng(5)
    U = _cn(rng, 50, 6)  # not orthonormal: the Gram matrix matters
    a = _cn(rng, 3, 6)
    S = a @ U.T
    np.testing.assert_allclose(solvers.project_onto_basis(U, S), a, atol=1e-10)
    T = _cn(rng, 3, 50)
    a2 = solvers.project_onto_basis(U, T)
    ref = np.linalg.lstsq(U, T.T, rcond=None)[0].T
    np.testing.assert_allclose(a2, ref, atol=1e-10)
    np.testing.assert_allclose(solvers.project_onto_basis(U, a2 @ U.T), a2, atol=1e-10)


@pytest.fixture(scope="module")
def problem64():
    ny = nx = 32
    C, q = 4, 16
    b = basis.build_maxwell_basis_2d(ny, nx, q, n_sites=24, n_exc=160, seed=0)
    a_true = solvers.project_onto_basis(b.U, basis.coil_maps_2d(ny, nx, C))
    p_true = w.random_ellipses(ny, nx, seed=1).ravel()
    return ny, nx, C, q, b.U, a_true, p_true


def test_irgn_fully_sampled_fits_data(problem64):
    ny, nx, C, q, U, a_true, p_true = problem64
    Fs = fourier.CartesianSampling((ny, nx), np.arange(ny * nx))
    y = op.forward(Fs, U, a_true, p_true)
    p, a, hist = solvers.irgn(Fs, U, y, C, q, n_outer=12, n_cg=10)
    assert hist[-1] < 0.02 * hist[0]
    assert np.all(np.diff(hist[1:]) < 0)
    ci = op.expand(U, a) * p[None]
    ct = op.expand(U, a_true) * p_true[None]
    assert np.linalg.norm(ci - ct) / np.linalg.norm(ct) < 0.05


def test_admm_reduces_to_least_squares_when_constraints_are_tight(problem64):
    # Fully sampled, eps -> 0: the constraint set is the single point S p = F^H y,
    # so MPI-L returns the SENSE least-squares image, here the truth.
    ny, nx, C, q, U, a_true, p_true = problem64
    Fs = fourier.CartesianSampling((ny, nx), np.arange(ny * nx))
    s = op.expand(U, a_true)
    y = op.forward(Fs, U, a_true, p_true)
    errs = []
    for n_outer in (50, 150):
        p, hist = solvers.admm_tv(Fs, s, y, np.full(C, 1e-9), (ny, nx), n_outer=n_outer, n_cg=10)
        errs.append(np.linalg.norm(p - p_true) / np.linalg.norm(p_true))
    assert errs[1] < 5e-2 and errs[1] < 0.5 * errs[0]


def test_admm_meets_constraints_with_noise(problem64):
    ny, nx, C, q, U, a_true, p_true = problem64
    mask = w.vd_lines_mask(ny, nx, 2, 8, seed=2)
    Fs = fourier.CartesianSampling((ny, nx), w.mask_to_indices(mask))
    s = op.expand(U, a_true)
    y0 = op.forward(Fs, U, a_true, p_true)
    sig = w.noise_sigma_for_snr(y0, 30)
    y = y0 + w.complex_noise(y0.shape, sig, seed=3)
    eps = np.full(C, sig * np.sqrt(Fs.M))
    p, hist = solvers.admm_tv(Fs, s, y, eps, (ny, nx), n_outer=200, n_cg=5)
    viol = max(np.linalg.norm(y[k] - Fs.fwd(s[k] * p)) / eps[k] for k in range(C))
    # ADMM reaches the constraint set only in the limit; after 200 iterations
    # the data misfit is within 2x of the noise level (it starts near 6x after 50)
    assert viol < 2.0
    # the primal residual shrinks
    assert hist[-1, 0] < 0.1 * hist[0, 0]


def test_admm_rho_change_keeps_unscaled_dual(problem64):
    # Scaled ADMM carries u = lambda / rho.  Changing rho must leave the unscaled
    # dual lambda = rho u unchanged (residual balancing, He et al. 2000; Boyd et
    # al. 2011 Sec. 3.4.1): rho -> tau rho goes with u -> u / tau.  A rescaling
    # in the wrong direction changes rho u by tau^2 and fails here.
    ny, nx, C, q, U, a_true, p_true = problem64
    mask = w.vd_lines_mask(ny, nx, 2, 8, seed=2)
    Fs = fourier.CartesianSampling((ny, nx), w.mask_to_indices(mask))
    s = op.expand(U, a_true)
    y0 = op.forward(Fs, U, a_true, p_true)
    sig = w.noise_sigma_for_snr(y0, 30)
    y = y0 + w.complex_noise(y0.shape, sig, seed=3)
    eps = np.full(C, sig * np.sqrt(Fs.M))
    events = []
    solvers.admm_tv(Fs, s, y, eps, (ny, nx), n_outer=60, n_cg=5, rho0=1e-3,
                    trace=lambda ev, rho, u0, uk: events.append((ev, rho, u0, uk)))
    changes = 0
    for i, (ev, rho, u0, uk) in enumerate(events):
        if ev != "rho":
            continue
        pev, prho, pu0, puk = events[i - 1]
        assert pev == "dual" and rho != prho
        np.testing.assert_allclose(rho * u0, prho * pu0, rtol=1e-13, atol=0)
        np.testing.assert_allclose(rho * uk, prho * puk, rtol=1e-13, atol=0)
        changes += 1
    assert changes >= 2


def _tiny_tv_problem():
    # 4 x 4 image, 2 smooth coil maps, 10 of 16 k-space points, noise
    rng = np.random.default_rng(11)
    ny = nx = 4
    N = ny * nx
    yy, xx = np.mgrid[0:ny, 0:nx] / 4.0
    s = np.stack([np.exp(0.4j + 0.5 * xx) * (1 + 0.3 * yy), np.exp(-0.3j * yy) * (1.2 - 0.4 * xx)]).reshape(2, N)
    p_true = np.zeros((ny, nx))
    p_true[1:3, 1:4] = 1.0
    p_true = p_true.ravel() + 0.05 * rng.normal(size=N)
    idx = np.sort(rng.choice(N, 10, replace=False))
    Fs = fourier.CartesianSampling((ny, nx), idx)
    y = Fs.fwd(s * p_true[None]) + 0.05 * (rng.normal(size=(2, 10)) + 1j * rng.normal(size=(2, 10)))
    eps = np.array([0.25, 0.25])
    return Fs, s, y, eps, (ny, nx)


def test_admm_matches_generic_constrained_tv_minimiser():
    # Eq. 8 on a tiny problem: min TV(p) s.t. ||y_k - F_s S_k p|| <= eps_k,
    # solved independently by SLSQP on a smoothed TV (sqrt(|grad|^2 + delta),
    # delta = 1e-12, which moves the optimal value by at most N * 1e-6); the
    # oracle's ADMM must reach the same optimal value, feasibly.
    Fs, s, y, eps, shape = _tiny_tv_problem()
    N = Fs.N
    delta = 1e-12

    def unpack(z):
        return z[:N] + 1j * z[N:]

    def tv_smooth(z):
        g = solvers.grad_fd(unpack(z).reshape(shape))
        return float(np.sum(np.sqrt(np.sum(np.abs(g) ** 2, axis=0) + delta)))

    cons = [{"type": "ineq", "fun": lambda z, k=k: eps[k] ** 2 - np.sum(np.abs(y[k] - Fs.fwd(s[k] * unpack(z))) ** 2)}
            for k in range(2)]
    x0 = np.sum(s.conj() * Fs.adj(y), axis=0) / np.sum(np.abs(s) ** 2, axis=0)
    best = minimize(tv_smooth, np.concatenate([x0.real, x0.imag]), constraints=cons, method="SLSQP",
                    options=dict(maxiter=200, ftol=1e-14))
    p_ref = unpack(best.x)
    assert max(np.linalg.norm(y[k] - Fs.fwd(s[k] * p_ref)) / eps[k] for k in range(2)) < 1 + 1e-6
    tv_ref = solvers.tv(p_ref.reshape(shape))
    p, hist = solvers.admm_tv(Fs, s, y, eps, shape, n_outer=300, n_cg=2 * N, n_tv=100)
    viol = max(np.linalg.norm(y[k] - Fs.fwd(s[k] * p)) / eps[k] for k in range(2))
    assert viol < 1 + 1e-4
    assert abs(solvers.tv(p.reshape(shape)) - tv_ref) < 1e-4 * tv_ref
    assert np.linalg.norm(p - p_ref) < 5e-3 * np.linalg.norm(p_ref)


def test_irgn_step_is_regularised_least_squares():
    # One outer step of MPI-BL from a generic point, its CG run to convergence,
    # equals the dense minimiser of Eq. 6's objective
    #   (1/2)||r - J dx||^2 + a_0 ||p + dp||^2 + b_0 ||alpha + dalpha||^2,
    # solved here by stacking it as one least-squares problem over an explicit J
    # (built column by column from the Jacobian of Eq. 7).  A wrong factor in the
    # normal equations (J^H J + L instead of J^H J + 2 L) fails.
    rng = np.random.default_rng(12)
    ny = nx = 6
    N, C, q = ny * nx, 2, 3
    U = np.linalg.qr(_cn(rng, N, q))[0]
    idx = np.sort(rng.choice(N, 20, replace=False))
    Fs = fourier.CartesianSampling((ny, nx), idx)
    y = _cn(rng, C, idx.size)
    y *= 100.0 / np.linalg.norm(y)  # the oracle's data scale is then 1
    p0 = 1.0 + 0.3 * _cn(rng, N)
    a0 = 0.5 * _cn(rng, C, q)
    an, bn = 0.7, 0.4
    p1, a1, _ = solvers.irgn(Fs, U, y, C, q, n_outer=1, n_cg=3 * (N + C * q), a0=an, b0=bn,
                             p0=p0, alpha0=a0)
    # explicit J: columns are J applied to unit vectors of [dp; dalpha]
    n_unk = N + C * q
    J = np.empty((C * idx.size, n_unk), dtype=np.complex128)
    for j in range(n_unk):
        e = np.zeros(n_unk, dtype=np.complex128)
        e[j] = 1.0
        J[:, j] = op.jacobian(Fs, U, a0, p0, e[:N], e[N:].reshape(C, q)).ravel()
    r = (y - op.forward(Fs, U, a0, p0)).ravel()
    x0 = np.concatenate([p0, a0.ravel()])
    w_reg = np.concatenate([np.full(N, np.sqrt(2 * an)), np.full(C * q, np.sqrt(2 * bn))])
    A = np.vstack([J, np.diag(w_reg)])
    b = np.concatenate([r, -w_reg * x0])
    dx = np.linalg.lstsq(A, b, rcond=None)[0]
    np.testing.assert_allclose(np.concatenate([p1 - p0, (a1 - a0).ravel()]), dx, rtol=0, atol=1e-8 * np.abs(dx).max())
