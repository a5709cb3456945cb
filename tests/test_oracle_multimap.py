"""Pins for the oracle's forward model with several sets of maps (Discussion,
"Forward Model Extensions": extra bilinear terms, y_k = F_s(sum_m U alpha_{m,k} p_m))
and its MPI-BL solver."""

import numpy as np

from oracle import fourier, operator as op, solvers


def _cn(rng, *shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def _case(seed, ny=6, nx=8, C=3, q=4, M=2, n_samp=30):
    rng = np.random.default_rng(seed)
    N = ny * nx
    U = np.linalg.qr(_cn(rng, N, q))[0]
    idx = np.sort(rng.choice(N, n_samp, replace=False))
    Fs = fourier.CartesianSampling((ny, nx), idx)
    A = _cn(rng, M, C, q)
    P = _cn(rng, M, N)
    return rng, Fs, U, A, P


def test_one_set_is_the_single_map_model():
    rng, Fs, U, A, P = _case(1, M=1)
    y = _cn(rng, 3, 30)
    dA, dP = _cn(rng, 1, 3, 4), _cn(rng, 1, 48)
    np.testing.assert_allclose(op.forward_multi(Fs, U, A, P), op.forward(Fs, U, A[0], P[0]), atol=1e-13)
    np.testing.assert_allclose(op.adjoint_multi(Fs, U, A, y)[0], op.adjoint(Fs, U, A[0], y), atol=1e-13)
    np.testing.assert_allclose(op.jacobian_multi(Fs, U, A, P, dP, dA),
                               op.jacobian(Fs, U, A[0], P[0], dP[0], dA[0]), atol=1e-13)
    gp, ga = op.jacobian_adjoint_multi(Fs, U, A, P, y)
    rp, ra = op.jacobian_adjoint(Fs, U, A[0], P[0], y)
    np.testing.assert_allclose(gp[0], rp, atol=1e-13)
    np.testing.assert_allclose(ga[0], ra, atol=1e-13)


def test_images_adjoint_dot_product():
    # <G(P), y> = sum_m <p_m, adjoint_multi(y)_m> for fixed maps (G is linear in P)
    rng, Fs, U, A, P = _case(2, M=3)
    y = _cn(rng, 3, 30)
    lhs = np.vdot(y, op.forward_multi(Fs, U, A, P))
    rhs = np.vdot(op.adjoint_multi(Fs, U, A, y), P)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_jacobian_is_the_exact_central_difference():
    # G is bilinear in (p_m, alpha_m) per term, so the central difference is exact
    rng, Fs, U, A, P = _case(3, M=2)
    dA, dP = _cn(rng, 2, 3, 4), _cn(rng, 2, 48)
    h = 0.37
    fd = (op.forward_multi(Fs, U, A + h * dA, P + h * dP) - op.forward_multi(Fs, U, A - h * dA, P - h * dP)) / (2 * h)
    np.testing.assert_allclose(op.jacobian_multi(Fs, U, A, P, dP, dA), fd, atol=1e-12 * np.abs(fd).max())


def test_jacobian_adjoint_dot_product():
    rng, Fs, U, A, P = _case(4, M=2)
    dA, dP = _cn(rng, 2, 3, 4), _cn(rng, 2, 48)
    r = _cn(rng, 3, 30)
    gp, ga = op.jacobian_adjoint_multi(Fs, U, A, P, r)
    lhs = np.vdot(r, op.jacobian_multi(Fs, U, A, P, dP, dA))
    rhs = np.vdot(gp, dP) + np.vdot(ga, dA)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_irgn_multi_with_one_set_is_irgn():
    rng, Fs, U, A, P = _case(5, M=1)
    y = _cn(rng, 3, 30)
    p1, a1, h1 = solvers.irgn(Fs, U, y, 3, 4, n_outer=4, n_cg=6)
    P2, A2, h2 = solvers.irgn_multi(Fs, U, y, 3, 4, 1, n_outer=4, n_cg=6)
    np.testing.assert_allclose(P2[0], p1, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(A2[0], a1, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(h2, h1, rtol=1e-12)


def test_irgn_multi_step_is_regularised_least_squares():
    # One outer step with two sets of maps from a generic point, its CG run to
    # convergence, equals the dense minimiser of
    #   (1/2)||r - J dx||^2 + a ||P + dP||^2 + b ||A + dA||^2
    # over an explicit J built column by column from jacobian_multi.  A wrong
    # factor, or a block of the right-hand side or of the penalty dropped, fails.
    rng = np.random.default_rng(12)
    ny = nx = 5
    N, C, q, M = ny * nx, 2, 3, 2
    U = np.linalg.qr(_cn(rng, N, q))[0]
    idx = np.sort(rng.choice(N, 18, replace=False))
    Fs = fourier.CartesianSampling((ny, nx), idx)
    y = _cn(rng, C, idx.size)
    y *= 100.0 / np.linalg.norm(y)  # the oracle's data scale is then 1
    P0 = 1.0 + 0.3 * _cn(rng, M, N)
    A0 = 0.5 * _cn(rng, M, C, q)
    an, bn = 0.7, 0.4
    n_unk = M * (N + C * q)
    P1, A1, _ = solvers.irgn_multi(Fs, U, y, C, q, M, n_outer=1, n_cg=3 * n_unk, a0=an, b0=bn, p0=P0, alpha0=A0)
    J = np.empty((C * idx.size, n_unk), dtype=np.complex128)
    for j in range(n_unk):
        e = np.zeros(n_unk, dtype=np.complex128)
        e[j] = 1.0
        J[:, j] = op.jacobian_multi(Fs, U, A0, P0, e[:M * N].reshape(M, N), e[M * N:].reshape(M, C, q)).ravel()
    r = (y - op.forward_multi(Fs, U, A0, P0)).ravel()
    x0 = np.concatenate([P0.ravel(), A0.ravel()])
    w_reg = np.concatenate([np.full(M * N, np.sqrt(2 * an)), np.full(M * C * q, np.sqrt(2 * bn))])
    dx = np.linalg.lstsq(np.vstack([J, np.diag(w_reg)]), np.concatenate([r, -w_reg * x0]), rcond=None)[0]
    got = np.concatenate([(P1 - P0).ravel(), (A1 - A0).ravel()])
    np.testing.assert_allclose(got, dx, rtol=0, atol=1e-8 * np.abs(dx).max())


def test_two_sets_fit_data_that_one_set_cannot():
    # data made with two sets of maps on different images: the two-set model
    # fits them far better than the single-set model (the point of the extension)
    rng = np.random.default_rng(7)
    ny = nx = 16
    N, C, q = ny * nx, 4, 6
    U = np.linalg.qr(_cn(rng, N, q))[0]
    Fs = fourier.CartesianSampling((ny, nx), np.arange(N))
    A_true = _cn(rng, 2, C, q)
    P_true = np.abs(_cn(rng, 2, N))
    y = op.forward_multi(Fs, U, A_true, P_true)
    _, _, h1 = solvers.irgn_multi(Fs, U, y, C, q, 1, n_outer=12, n_cg=20)
    _, _, h2 = solvers.irgn_multi(Fs, U, y, C, q, 2, n_outer=12, n_cg=20)
    assert h2[-1] < 0.5 * h1[-1]
