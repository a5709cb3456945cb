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
