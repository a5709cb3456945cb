"""Maxwell basis construction in FP64 ("Maxwell Regularization" section).

Test infrastructure (see the package header).

Steps, in the paper's order:

1. Sources outside the field of view: point electric and magnetic dipoles
   (three orientations each) at D sites on a circle of radius
   1.5 x the FOV half-diagonal in the slice plane.  (The paper discretises
   boundary currents with MARIE; point dipoles outside the FOV are the
   simplification taken here.)
2. Their magnetic field at the pixel centroids through the free-space dyadic
   Green's functions (Eqs. 17-18): H = grad g x j for an electric current
   element and H = (grad grad + k^2) g m / (j omega mu) for a magnetic one,
   g = exp(-j k R) / (4 pi R), k = omega sqrt(eps0 mu0).  Magnetic currents are
   weighted by the free-space impedance eta0 (m = eta0 m_hat), which makes the
   factor 1 / (j k); it only balances the two blocks of K = [K^hj K^hm] (Eq. 15).
3. Circular polarisation: the detected component b = (H_x - i H_y) / sqrt(2)
   (sign convention e^{+j omega t}, implied by the e^{-jkR} of g).
4. Randomized range finder: random complex amplitudes and phases on all the
   dipoles give L excitations Y = B Omega; the SVD of Y gives the basis as its
   q leading left singular vectors, ordered by singular value (Eq. 16:
   truncation error sigma_{q+1}).

Because every column of B is an exact source-free solution of the Helmholtz
equation inside the FOV, so is every basis vector; ``basis_fields_at`` lets the
tests evaluate a basis vector off the slice plane to check that.
"""

import numpy as np

C0 = 299792458.0
MU0 = 4e-7 * np.pi


def wavenumber(f_hz):
    """k = omega sqrt(eps0 mu0) = 2 pi f / c0."""
    return 2.0 * np.pi * f_hz / C0


def pixel_centroids(ny, nx, fov_m):
    """(N, 3) centroids of an ny x nx grid in the z = 0 plane, raster order."""
    dy = fov_m[0] / ny
    dx = fov_m[1] / nx
    y = (np.arange(ny) - ny / 2 + 0.5) * dy
    x = (np.arange(nx) - nx / 2 + 0.5) * dx
    Y, X = np.meshgrid(y, x, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), np.zeros(ny * nx)], axis=1)


def voxel_centroids(nz, ny, nx, fov_m):
    """(N, 3) centroids of an nz x ny x nx grid centred on the origin, raster
    order (x fastest, z slowest); fov_m = (fov_z, fov_y, fov_x)."""
    dz, dy, dx = fov_m[0] / nz, fov_m[1] / ny, fov_m[2] / nx
    z = (np.arange(nz) - nz / 2 + 0.5) * dz
    y = (np.arange(ny) - ny / 2 + 0.5) * dy
    x = (np.arange(nx) - nx / 2 + 0.5) * dx
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def sphere_sources(n_sites, radius):
    """n_sites points spread over a sphere (the Fibonacci lattice)."""
    i = np.arange(n_sites) + 0.5
    zc = 1.0 - 2.0 * i / n_sites
    rho = np.sqrt(1.0 - zc ** 2)
    th = np.pi * (3.0 - np.sqrt(5.0)) * i
    return radius * np.stack([rho * np.cos(th), rho * np.sin(th), zc], axis=1)


def circle_sources(n_sites, radius, z=0.0):
    th = 2.0 * np.pi * np.arange(n_sites) / n_sites
    return np.stack([radius * np.cos(th), radius * np.sin(th), np.full(n_sites, z)], axis=1)


def dipole_b_fields(points, sources, k):
    """Circularly polarised field of each source dipole at each point.

    Returns B of shape (P, S * 6): for every source site, columns are the
    electric dipoles along x, y, z then the magnetic dipoles along x, y, z.
    """
    points = np.asarray(points, dtype=np.float64)
    sources = np.asarray(sources, dtype=np.float64)
    Rv = points[:, None, :] - sources[None, :, :]  # (P, S, 3)
    R = np.linalg.norm(Rv, axis=2)
    Rh = Rv / R[:, :, None]
    g = np.exp(-1j * k * R) / (4.0 * np.pi * R)
    g1 = -(1j * k + 1.0 / R) * g  # dg/dR
    g2 = ((1j * k + 1.0 / R) ** 2 + 1.0 / R ** 2) * g  # d2g/dR2
    eye = np.eye(3)
    cols = []
    # Electric current element along e: H = grad g x e = g1 (Rh x e).
    for e in eye:
        H = g1[:, :, None] * np.cross(Rh, e[None, None, :])
        cols.append((H[..., 0] - 1j * H[..., 1]) / np.sqrt(2.0))
    # Magnetic current element eta0 m: H = (grad grad g + k^2 g) m / (j k),
    # grad grad g = (g2 - g1/R) Rh Rh^T + (g1/R) I.
    A = (g2 - g1 / R) / (1j * k)
    Bc = (g1 / R + k * k * g) / (1j * k)
    for m in eye:
        Rm = Rh @ m  # (P, S)
        H = A[:, :, None] * Rm[:, :, None] * Rh + Bc[:, :, None] * m[None, None, :]
        cols.append((H[..., 0] - 1j * H[..., 1]) / np.sqrt(2.0))
    B = np.stack(cols, axis=2)  # (P, S, 6)
    return B.reshape(points.shape[0], -1)


class MaxwellBasis2D:
    """Result of ``build_maxwell_basis_2d``.

    U      (N, q) orthonormal basis, raster order over (ny, nx)
    sv     singular values of the excitation matrix Y (all of them)
    comb   (6 D, q) coefficients such that U = B(pixels) @ comb
    """

    def __init__(self, U, sv, comb, sources, k, shape, fov):
        self.U, self.sv, self.comb = U, sv, comb
        self.sources, self.k, self.shape, self.fov = sources, k, shape, fov

    def fields_at(self, points):
        """Basis vectors evaluated at arbitrary points (P, 3) -> (P, q)."""
        return dipole_b_fields(points, self.sources, self.k) @ self.comb


def build_maxwell_basis_2d(ny, nx, q, fov_m=(0.22, 0.22), f_hz=128e6, n_sites=64,
                           n_exc=500, radius_factor=1.5, seed=0, omega=None):
    """Maxwell basis for a 2D slice (steps 1-4 of the module docstring).

    ``omega`` (6 D x L complex), when given, is the excitation matrix itself
    (rows in the column order of ``dipole_b_fields``); otherwise it is drawn
    from ``seed``."""
    k = wavenumber(f_hz)
    half_diag = 0.5 * np.hypot(fov_m[0], fov_m[1])
    src = circle_sources(n_sites, radius_factor * half_diag)
    pts = pixel_centroids(ny, nx, fov_m)
    B = dipole_b_fields(pts, src, k)  # (N, 6D)
    if omega is not None:
        Omega = np.asarray(omega, dtype=np.complex128)
        L = Omega.shape[1]
    else:
        rng = np.random.default_rng(seed)
        L = n_exc
        Omega = (rng.normal(size=(B.shape[1], L)) + 1j * rng.normal(size=(B.shape[1], L))) / np.sqrt(2.0)
    Y = B @ Omega
    Uy, sv, Vh = np.linalg.svd(Y, full_matrices=False)
    U = Uy[:, :q]
    comb = Omega @ (Vh[:q].conj().T / sv[:q][None, :])
    return MaxwellBasis2D(U, sv, comb, src, k, (ny, nx), fov_m)


def build_maxwell_basis_3d(nz, ny, nx, q, fov_m=(0.22, 0.22, 0.22), f_hz=128e6, n_sites=64, omega=None,
                           radius_factor=1.5, sources=None, seed=0, n_exc=500):
    """Maxwell basis of a 3D volume: the 2D steps with voxel centroids and, by
    default, dipole sites on a sphere of radius radius_factor x the FOV
    half-diagonal.  Returns (U (N, q), singular values, sources)."""
    k = wavenumber(f_hz)
    if sources is None:
        sources = sphere_sources(n_sites, radius_factor * 0.5 * np.sqrt(np.sum(np.square(fov_m))))
    pts = voxel_centroids(nz, ny, nx, fov_m)
    B = dipole_b_fields(pts, sources, k)
    if omega is None:
        rng = np.random.default_rng(seed)
        omega = (rng.normal(size=(B.shape[1], n_exc)) + 1j * rng.normal(size=(B.shape[1], n_exc))) / np.sqrt(2.0)
    Uy, sv, _ = np.linalg.svd(B @ np.asarray(omega, dtype=np.complex128), full_matrices=False)
    return Uy[:, :q], sv, np.asarray(sources)


def coil_maps_2d(ny, nx, C, fov_m=(0.22, 0.22), f_hz=128e6, radius_factor=1.2):
    """Ground-truth coil maps: C loop coils modelled as magnetic dipoles.

    Coil c sits at angle 2 pi c / C on a circle of radius radius_factor x the FOV
    half-diagonal with its moment pointing to the centre; its map is the
    circularly polarised field, normalised so that max over pixels of
    sqrt(sum_c |s_c|^2) is 1.  Returns (C, N).
    """
    k = wavenumber(f_hz)
    half_diag = 0.5 * np.hypot(fov_m[0], fov_m[1])
    src = circle_sources(C, radius_factor * half_diag)
    pts = pixel_centroids(ny, nx, fov_m)
    B = dipole_b_fields(pts, src, k).reshape(ny * nx, C, 6)
    th = 2.0 * np.pi * np.arange(C) / C
    mx, my = -np.cos(th), -np.sin(th)
    s = (B[:, :, 3] * mx[None, :] + B[:, :, 4] * my[None, :]).T
    s = s / np.sqrt(np.sum(np.abs(s) ** 2, axis=0)).max()
    return s
