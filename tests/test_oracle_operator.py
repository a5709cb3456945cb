"""Pins for the oracle's bilinear operator, Jacobian and adjoints (Eqs. 3, 5, 7)."""

import numpy as np
import pytest

from oracle import fourier, operator as op, tucker
import workloads as w


def _setup(shape=(16, 16), C=3, q=6, seed=0, full=False):
    rng = np.random.default_rng(seed)
    N = int(np.prod(shape))
    U = np.linalg.qr(rng.normal(size=(N, q)) + 1j * rng.normal(size=(N, q)))[0]
    if full:
        idx = np.arange(N, dtype=np.int32)
    else:
        idx = w.mask_to_indices(w.poisson_disc_mask(shape[0], shape[1], 2.5, calib=(4, 4), seed=seed))
    Fs = fourier.CartesianSampling(shape, idx)
    a = rng.normal(size=(C, q)) + 1j * rng.normal(size=(C, q))
    p = rng.normal(size=N) + 1j * rng.normal(size=N)
    return rng, U, Fs, a, p


def _cn(rng, *shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def test_expand_brute_force():
    rng, U, Fs, a, p = _setup()
    s = op.expand(U, a)
    for k in range(a.shape[0]):
        ref = sum(U[:, j] * a[k, j] for j in range(U.shape[1]))
        np.testing.assert_allclose(s[k], ref, atol=1e-12)


def test_adjoint_dot_product():
    rng, U, Fs, a, p = _setup()
    y = _cn(rng, a.shape[0], Fs.M)
    lhs = np.vdot(op.forward(Fs, U, a, p), y)
    rhs = np.vdot(p, op.adjoint(Fs, U, a, y))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_jacobian_central_difference_is_exact():
    # G is bilinear, so (G(x + h d) - G(x - h d)) / 2h = J(x) d with no O(h^2) term.
    rng, U, Fs, a, p = _setup(seed=1)
    dp = _cn(rng, p.size)
    da = _cn(rng, *a.shape)
    h = 1e-3
    fd = (op.forward(Fs, U, a + h * da, p + h * dp) - op.forward(Fs, U, a - h * da, p - h * dp)) / (2 * h)
    J = op.jacobian(Fs, U, a, p, dp, da)
    assert np.linalg.norm(fd - J) <= 1e-10 * np.linalg.norm(J)
    # the second-order part is the product term: G(x+hd) - G(x) - h J d = h^2 G(dp, da)
    rem = op.forward(Fs, U, a + h * da, p + h * dp) - op.forward(Fs, U, a, p) - h * J
    np.testing.assert_allclose(rem, h * h * op.forward(Fs, U, da, dp), atol=1e-12)


def test_jacobian_adjoint_dot_product():
    rng, U, Fs, a, p = _setup(seed=2)
    dp = _cn(rng, p.size)
    da = _cn(rng, *a.shape)
    r = _cn(rng, a.shape[0], Fs.M)
    gp, ga = op.jacobian_adjoint(Fs, U, a, p, r)
    lhs = np.vdot(op.jacobian(Fs, U, a, p, dp, da), r)
    rhs = np.vdot(dp, gp) + np.vdot(da, ga)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_jacobian_adjoint_is_gradient_of_data_term():
    # f(x) = 1/2 ||G(x) - y||^2; its directional derivative along d equals
    # Re <J^H (G(x) - y), d>.
    rng, U, Fs, a, p = _setup(seed=3)
    y = _cn(rng, a.shape[0], Fs.M)
    dp = _cn(rng, p.size)
    da = _cn(rng, *a.shape)

    def f(pp, aa):
        return 0.5 * np.linalg.norm(op.forward(Fs, U, aa, pp) - y) ** 2

    h = 1e-6
    fd = (f(p + h * dp, a + h * da) - f(p - h * dp, a - h * da)) / (2 * h)
    gp, ga = op.jacobian_adjoint(Fs, U, a, p, op.forward(Fs, U, a, p) - y)
    an = (np.vdot(gp, dp) + np.vdot(ga, da)).real
    assert abs(fd - an) <= 1e-6 * abs(an)


def test_fully_sampled_closed_form():
    # With every sample taken F_s is unitary, so S^H F^H F S p = sum_k |s_k|^2 p.
    rng, U, Fs, a, p = _setup(full=True, seed=4)
    s = op.expand(U, a)
    got = op.adjoint(Fs, U, a, op.forward(Fs, U, a, p))
    np.testing.assert_allclose(got, np.sum(np.abs(s) ** 2, axis=0) * p, atol=1e-10)


def test_tucker_basis_operator_matches_dense():
    rng = np.random.default_rng(5)
    n = (4, 6, 8)
    r = (3, 4, 5)
    q = 7
    core = _cn(rng, *r, q)
    factors = [np.linalg.qr(_cn(rng, nk, rk))[0] for nk, rk in zip(n, r)]
    tb = tucker.TuckerBasis(core, factors)
    Ud = tb.dense()
    N = Ud.shape[0]
    a = _cn(rng, 2, q)
    np.testing.assert_allclose(op.expand(tb, a), op.expand(Ud, a), atol=1e-12)
    v = _cn(rng, 2, N)
    np.testing.assert_allclose(op.expand_adjoint(tb, v), op.expand_adjoint(Ud, v), atol=1e-12)
    idx = np.sort(rng.choice(N, size=N // 3, replace=False)).astype(np.int32)
    Fs = fourier.CartesianSampling(n, idx)
    p = _cn(rng, N)
    rr = _cn(rng, 2, Fs.M)
    g1 = op.jacobian_adjoint(Fs, tb, a, p, rr)
    g2 = op.jacobian_adjoint(Fs, Ud, a, p, rr)
    np.testing.assert_allclose(g1[0], g2[0], atol=1e-11)
    np.testing.assert_allclose(g1[1], g2[1], atol=1e-11)


@pytest.mark.parametrize("dims", [(8, 8), (4, 8, 8)])
def test_forward_direct_sum_tiny(dims):
    # y_k[m] = N^{-1/2} sum_n s_k[n] p[n] exp(-2 pi i sum_d (kk_d - n_d/2)(j_d - n_d/2)/n_d)
    rng = np.random.default_rng(6)
    N = int(np.prod(dims))
    q, C = 3, 2
    U = _cn(rng, N, q)
    a = _cn(rng, C, q)
    p = _cn(rng, N)
    idx = np.sort(rng.choice(N, size=N // 4, replace=False))
    Fs = fourier.CartesianSampling(dims, idx)
    y = op.forward(Fs, U, a, p)
    coords = np.array(np.unravel_index(np.arange(N), dims)).T - np.array(dims) // 2
    s = a @ U.T
    for m, flat in enumerate(idx[:10]):
        kk = np.array(np.unravel_index(flat, dims)) - np.array(dims) // 2
        ph = np.exp(-2j * np.pi * np.sum(coords * kk / np.array(dims), axis=1))
        for c in range(C):
            ref = np.sum(s[c] * p * ph) / np.sqrt(N)
            assert abs(y[c, m] - ref) < 1e-11
