"""Pins for the oracle's Maxwell basis ("Maxwell Regularization") and Tucker compression."""

import os

import numpy as np
import pytest

from oracle import basis, tucker


def _num_grad(f, x, h=1e-6):
    g = []
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        g.append((f(x + e) - f(x - e)) / (2 * h))
    return np.array(g)


def test_dipole_fields_match_green_function_derivatives():
    # H_e = grad g x e and H_m = (grad grad g + k^2 g) m / (j k), checked against
    # finite differences of the scalar Green's function g = exp(-jkR)/(4 pi R).
    k = basis.wavenumber(128e6)
    src = np.array([[0.3, -0.1, 0.05]])
    pt = np.array([0.02, 0.04, -0.01])

    def g(r):
        R = np.linalg.norm(r - src[0])
        return np.exp(-1j * k * R) / (4 * np.pi * R)

    grad = _num_grad(g, pt, 1e-6)
    hess = np.array([_num_grad(lambda r, d=d: _num_grad(g, r, 1e-5)[d], pt, 1e-5) for d in range(3)])
    B = basis.dipole_b_fields(pt[None], src, k)[0]
    eye = np.eye(3)
    for i, e in enumerate(eye):
        H = np.cross(grad, e)
        assert np.isclose(B[i], (H[0] - 1j * H[1]) / np.sqrt(2), rtol=1e-6)
    for i, m in enumerate(eye):
        H = (hess @ m + k * k * g(pt) * m) / (1j * k)
        assert np.isclose(B[3 + i], (H[0] - 1j * H[1]) / np.sqrt(2), rtol=1e-4)


@pytest.fixture(scope="module")
def small_basis():
    return basis.build_maxwell_basis_2d(24, 24, 12, n_sites=16, n_exc=96, seed=3)


def test_basis_orthonormal_and_ordered(small_basis):
    U = small_basis.U
    np.testing.assert_allclose(U.conj().T @ U, np.eye(U.shape[1]), atol=1e-12)
    assert np.all(np.diff(small_basis.sv) <= 0)
    # the stored combination reproduces the basis from the dipole fields
    pts = basis.pixel_centroids(24, 24, small_basis.fov)
    np.testing.assert_allclose(small_basis.fields_at(pts), U, atol=1e-10)


def test_randomized_basis_captures_range_within_sigma_q_plus_1():
    # Eckart-Young (Eq. 16): the best rank-q approximation of K errs by sigma_{q+1};
    # the randomized basis must get within a small factor of it.
    ny = nx = 16
    q = 8
    b = basis.build_maxwell_basis_2d(ny, nx, q, n_sites=12, n_exc=72, seed=1)
    src = b.sources
    K = basis.dipole_b_fields(basis.pixel_centroids(ny, nx, b.fov), src, b.k)
    sK = np.linalg.svd(K, compute_uv=False)
    resid = K - b.U @ (b.U.conj().T @ K)
    err = np.linalg.norm(resid, 2)
    assert err >= sK[q] * (1 - 1e-9)
    assert err <= 3.0 * sK[q]


def _helmholtz_residual(fields_at, k, centre, h):
    offs = [np.array(v) * h for v in
            [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)]]
    pts = np.array([centre] + [centre + o for o in offs])
    u = fields_at(pts)
    lap = (np.sum(u[1:], axis=0) - 6 * u[0]) / h ** 2
    return np.abs(lap + k * k * u[0]), np.abs(lap)


def test_basis_vectors_solve_helmholtz(small_basis):
    k = small_basis.k
    centre = np.array([0.013, -0.021, 0.0])
    r1, lap1 = _helmholtz_residual(small_basis.fields_at, k, centre, 4e-3)
    r2, _ = _helmholtz_residual(small_basis.fields_at, k, centre, 2e-3)
    ratio = r1 / r2
    assert np.all((ratio > 3.5) & (ratio < 4.5)), ratio
    # a smooth non-solution of comparable size leaves an O(1) residual instead
    def bump(P):
        return np.exp(-np.sum(P ** 2, axis=1) / 0.05 ** 2)[:, None]

    rb, _ = _helmholtz_residual(bump, k, centre, 2e-3)
    rel_basis = r2 / np.abs(small_basis.fields_at(centre[None]))[0]
    rel_bump = rb[0] / np.abs(bump(centre[None]))[0, 0]
    assert rel_basis.max() < 1e-2 * rel_bump


def test_mode_product_brute_force():
    rng = np.random.default_rng(0)
    A = rng.normal(size=(3, 4, 5)) + 1j * rng.normal(size=(3, 4, 5))
    B = rng.normal(size=(6, 4)) + 1j * rng.normal(size=(6, 4))
    C = tucker.mode_product(A, B, 1)
    ref = np.zeros((3, 6, 5), complex)
    for i in range(3):
        for j in range(6):
            for kk in range(5):
                ref[i, j, kk] = sum(A[i, p, kk] * B[j, p] for p in range(4))
    np.testing.assert_allclose(C, ref, atol=1e-12)


def test_hosvd_full_rank_exact_and_truncation_bound():
    rng = np.random.default_rng(1)
    T = rng.normal(size=(6, 5, 4, 3)) + 1j * rng.normal(size=(6, 5, 4, 3))
    core, fac = tucker.hosvd(T)
    for f in fac:
        np.testing.assert_allclose(f.conj().T @ f, np.eye(f.shape[1]), atol=1e-12)
    np.testing.assert_allclose(tucker.tucker_full(core, fac), T, atol=1e-12)
    # smooth tensor: truncation at eps keeps the error below eps ||T|| (Eq. 21)
    b = basis.build_maxwell_basis_2d(16, 16, 6, n_sites=12, n_exc=60, seed=2)
    Ts = b.U.reshape(4, 4, 16, 6)
    for eps in [1e-2, 1e-4]:
        core, fac = tucker.hosvd(Ts, eps=eps)
        err = np.linalg.norm(tucker.tucker_full(core, fac) - Ts) / np.linalg.norm(Ts)
        assert err < eps


def test_table_s1_dense_ram_column():
    # Table S1 (supporting information): dense basis RAM for N = 6,266,880
    # voxels stored as complex128, in MiB.
    fix = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "table_s1_dense_ram.txt"),
                     comments="#")
    N = 6266880
    for q, mb in fix:
        assert round(N * q * 16 / 2 ** 20) == mb


def test_voxel_centroids_and_3d_builder_reduce_to_2d():
    # one slice of voxels is the 2D pixel grid, and the 3D builder with the 2D
    # sources and excitations gives the 2D basis (subspace) and singular values
    pts3 = basis.voxel_centroids(1, 6, 8, (0.01, 0.22, 0.22))
    np.testing.assert_allclose(pts3, basis.pixel_centroids(6, 8, (0.22, 0.22)), atol=0)
    src = basis.circle_sources(8, 1.5 * 0.5 * np.hypot(0.22, 0.22))
    om = (np.random.default_rng(4).normal(size=(48, 40)) + 1j * np.random.default_rng(5).normal(size=(48, 40)))
    b2 = basis.build_maxwell_basis_2d(12, 12, 6, n_sites=8, omega=om)
    U3, sv3, _ = basis.build_maxwell_basis_3d(1, 12, 12, 6, fov_m=(0.01, 0.22, 0.22), omega=om, sources=src)
    np.testing.assert_allclose(sv3, b2.sv, rtol=1e-12)
    assert np.linalg.norm(U3 - b2.U @ (b2.U.conj().T @ U3)) < 1e-10


def test_sphere_sources_on_the_sphere_and_spread():
    s = basis.sphere_sources(50, 0.3)
    np.testing.assert_allclose(np.linalg.norm(s, axis=1), 0.3, rtol=1e-12)
    assert abs(s.mean(axis=0)).max() < 0.02  # no hemisphere favoured
    d = np.linalg.norm(s[:, None] - s[None], axis=2) + np.eye(50)
    assert d.min() > 0.5 * 0.3 * np.sqrt(4 * np.pi / 50)  # no two sites much closer than the mean spacing
