"""Pins for the oracle's sampling operators (Eq. 1's F_s), independent of the oracle itself."""

import numpy as np
import pytest

from oracle import fourier, nufft
import workloads as w


def _np_centered(v, axes):
    # numpy's FFT with index shifts: an independent realisation of the centred
    # unitary DFT convention.
    out = np.fft.ifftshift(v, axes=axes)
    out = np.fft.fftn(out, axes=axes, norm="ortho")
    return np.fft.fftshift(out, axes=axes)


@pytest.mark.parametrize("shape", [(4, 8), (8, 8), (12, 16), (64, 64)])
def test_dft_matches_numpy_fft(shape):
    rng = np.random.default_rng(0)
    v = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    np.testing.assert_allclose(fourier.dft(v, 2), _np_centered(v, (0, 1)), atol=1e-12)


def test_dft_3d_matches_numpy_fft():
    rng = np.random.default_rng(1)
    v = rng.normal(size=(4, 8, 12)) + 1j * rng.normal(size=(4, 8, 12))
    np.testing.assert_allclose(fourier.dft(v, 3), _np_centered(v, (0, 1, 2)), atol=1e-12)


def test_dft_closed_forms():
    n = 16
    # a unit impulse at the centre (t = 0) has a flat spectrum n^{-1/2}
    d = np.zeros(n)
    d[n // 2] = 1.0
    np.testing.assert_allclose(fourier.dft(d[None], 1)[0], np.full(n, n ** -0.5), atol=1e-14)
    # a plane wave exp(+2 pi i k0 t / n) lands on bin k0 + n/2 with height sqrt(n)
    k0 = 3
    t = np.arange(n) - n // 2
    pw = np.exp(2j * np.pi * k0 * t / n)
    ref = np.zeros(n, complex)
    ref[k0 + n // 2] = np.sqrt(n)
    np.testing.assert_allclose(fourier.dft(pw[None], 1)[0], ref, atol=1e-12)


def test_parseval_and_inverse():
    rng = np.random.default_rng(2)
    v = rng.normal(size=(3, 8, 12)) + 1j * rng.normal(size=(3, 8, 12))
    k = fourier.dft(v, 2)
    assert np.isclose(np.linalg.norm(k), np.linalg.norm(v), rtol=1e-13)
    np.testing.assert_allclose(fourier.idft(k, 2), v, atol=1e-12)


def test_cartesian_sampling_adjoint_and_projection():
    rng = np.random.default_rng(3)
    mask = w.poisson_disc_mask(32, 32, 3, calib=(8, 8), seed=4)
    Fs = fourier.CartesianSampling((32, 32), w.mask_to_indices(mask))
    v = rng.normal(size=(2, 1024)) + 1j * rng.normal(size=(2, 1024))
    y = rng.normal(size=(2, Fs.M)) + 1j * rng.normal(size=(2, Fs.M))
    lhs = np.vdot(Fs.fwd(v), y)
    rhs = np.vdot(v, Fs.adj(y))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # F_s F_s^H = I on the samples (F unitary, rows selected)
    np.testing.assert_allclose(Fs.fwd(Fs.adj(y)), y, atol=1e-12)


def test_nudft_on_grid_equals_dft():
    n = 16
    kk = np.arange(n) - n // 2
    KY, KX = np.meshgrid(kk, kk, indexing="ij")
    k = np.stack([2 * np.pi * KX.ravel() / n, 2 * np.pi * KY.ravel() / n], axis=1)
    nu = fourier.DirectNUDFT((n, n), k)
    rng = np.random.default_rng(5)
    v = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    np.testing.assert_allclose(nu.fwd(v.ravel()), _np_centered(v, (0, 1)).ravel(), atol=1e-12)


def test_nudft_adjoint():
    n = 16
    k = w.golden_angle_radial(5, 32)
    nu = fourier.DirectNUDFT((n, n), k)
    rng = np.random.default_rng(6)
    v = rng.normal(size=n * n) + 1j * rng.normal(size=n * n)
    y = rng.normal(size=nu.M) + 1j * rng.normal(size=nu.M)
    lhs = np.vdot(nu.fwd(v), y)
    rhs = np.vdot(v, nu.adj(y))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_nudft_brute_force_tiny():
    n = 4
    k = np.array([[0.3, -1.1], [2.0, 0.5], [-3.1, 3.0]])
    rng = np.random.default_rng(7)
    v = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    ref = []
    for kx, ky in k:
        acc = 0j
        for yy in range(n):
            for xx in range(n):
                acc += v[yy, xx] * np.exp(-1j * (kx * (xx - n // 2) + ky * (yy - n // 2)))
        ref.append(acc / n)
    np.testing.assert_allclose(fourier.DirectNUDFT((n, n), k).fwd(v.ravel()), ref, atol=1e-12)


# --- Kaiser-Bessel gridding ---------------------------------------------------

def test_kb_deapod_is_fourier_transform_of_kernel():
    W, sigma, G = 6, 2.0, 64
    beta = nufft.kb_beta(W, sigma)
    u = np.linspace(-W / 2, W / 2, 200001)
    phi = nufft.kb_kernel(u, W, beta)
    for t in [0.0, 3.0, 10.0, 16.0]:
        integrand = phi * np.exp(-2j * np.pi * u * t / G)
        num = np.trapezoid(integrand, u).real
        assert np.isclose(nufft.kb_deapod(np.array([t]), W, beta, G)[0], num, rtol=1e-7)


def test_kb_beta_value():
    # beta = pi sqrt((W/sigma)^2 (sigma - 1/2)^2 - 0.8) at W = 6, sigma = 2
    assert np.isclose(nufft.kb_beta(6, 2.0), np.pi * np.sqrt(19.45))


def test_gridding_indices_brute_force():
    k = w.golden_angle_radial(7, 64).astype(np.float32)
    G, W = 128, 6
    idx = nufft.gridding_indices(k, G, W)
    for m in range(0, k.shape[0], 13):
        for ax in range(2):
            kap = float(np.float64(k[m, ax]) * (G / (2 * np.pi)))
            # taps are exactly the integers g with kap - W/2 < g <= kap + W/2
            gs = [g for g in range(-G, G) if kap - W / 2 < g <= kap + W / 2]
            assert len(gs) == W
            assert idx[m, ax] == (gs[0] + G // 2) % G


def test_kb_nufft_close_to_nudft():
    n = 32
    k = w.golden_angle_radial(16, 64).astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(8)
    v = rng.normal(size=(2, n * n)) + 1j * rng.normal(size=(2, n * n))
    kb = nufft.KBGriddingNUFFT((n, n), k, W=6, sigma=2.0)
    ex = fourier.DirectNUDFT((n, n), k)
    err = np.linalg.norm(kb.fwd(v) - ex.fwd(v)) / np.linalg.norm(ex.fwd(v))
    assert err < 1e-4
    y = rng.normal(size=(2, kb.M)) + 1j * rng.normal(size=(2, kb.M))
    erra = np.linalg.norm(kb.adj(y) - ex.adj(y)) / np.linalg.norm(ex.adj(y))
    assert erra < 1e-4


def test_kb_nufft_adjoint():
    n = 16
    k = w.golden_angle_radial(6, 32)
    kb = nufft.KBGriddingNUFFT((n, n), k)
    rng = np.random.default_rng(9)
    v = rng.normal(size=n * n) + 1j * rng.normal(size=n * n)
    y = rng.normal(size=kb.M) + 1j * rng.normal(size=kb.M)
    lhs = np.vdot(kb.fwd(v), y)
    rhs = np.vdot(v, kb.adj(y))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("shape", [(8, 12), (16, 32, 48), (6, 10, 4)])
def test_fast_mode_equals_explicit_matrices(shape):
    # the oracle's FFT fast mode (used only to time the CPU baseline) computes the
    # same F_s and F_s^H as the explicit separable DFT matrices
    rng = np.random.default_rng(7)
    N = int(np.prod(shape))
    idx = np.sort(rng.choice(N, N // 3, replace=False))
    slow = fourier.CartesianSampling(shape, idx)
    fast = fourier.CartesianSamplingFFT(shape, idx, workers=2)
    v = rng.normal(size=(3, N)) + 1j * rng.normal(size=(3, N))
    y = rng.normal(size=(3, idx.size)) + 1j * rng.normal(size=(3, idx.size))
    np.testing.assert_allclose(fast.fwd(v), slow.fwd(v), atol=1e-12)
    np.testing.assert_allclose(fast.adj(y), slow.adj(y), atol=1e-12)
