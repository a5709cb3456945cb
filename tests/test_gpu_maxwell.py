"""GPU Maxwell basis construction against the FP64 oracle ("Maxwell
Regularization": Eqs. 15-18, Fig. 1's random boundary excitations).

Both sides take the same dipole sites and the same excitation matrix Omega
(seeded inputs).  Several bases are correct (each singular vector's phase is
free, and equal singular values would leave a rotation free), so the checks
are on what is unique: the singular values of B Omega (to 1e-10 of sigma_1,
the absolute accuracy of either FP64 computation) and the subspace of the q
leading vectors, ||U U^H - U_ref U_ref^H||_2 <= 1e-5, at truncations where
the spectrum has a gap.
"""

import numpy as np
import pytest
import torch

import workloads as w
from oracle import basis as ob

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mp():
    import paper_2008_09042_gb300 as mp

    return mp


@pytest.fixture(scope="module")
def ctx(mp):
    return mp.Context(0)


def _sources(n_sites, fov=(0.22, 0.22), radius_factor=1.5):
    return ob.circle_sources(n_sites, radius_factor * 0.5 * np.hypot(*fov))


def _sin_theta(U, Uref):
    """||U U^H - Uref Uref^H||_2 = ||(I - Uref Uref^H) U||_2 for orthonormal
    (N, q) bases, taken from the residual itself (U re-orthonormalised in
    FP64 first), not as sqrt(1 - cos^2), which would turn the complex64
    vectors' 1e-8 departures from unit length into 1e-4."""
    Uo = np.linalg.qr(U)[0]
    return float(np.linalg.norm(Uo - Uref @ (Uref.conj().T @ Uo), 2))


def _gpu_vs_oracle(ctx, mp, shape, n_sites, L, qs, seed):
    src = _sources(n_sites)
    om = w.random_excitations(6 * n_sites, L, seed=seed)
    qmax = max(qs)
    ref = ob.build_maxwell_basis_2d(shape[0], shape[1], qmax, n_sites=n_sites, omega=om)
    U, sv = mp.maxwell_basis_2d(ctx, shape, qmax, src, om)
    ctx.synchronize()
    U = U.cpu().numpy().astype(np.complex128).T  # (N, q)
    nsv = min(6 * n_sites, L)
    assert sv.shape == (nsv,)
    assert np.all(np.diff(sv) <= 0)
    assert np.max(np.abs(sv - ref.sv[:nsv])) <= 1e-10 * ref.sv[0]
    # complex64 vectors: orthonormal to single precision
    assert np.abs(U.conj().T @ U - np.eye(qmax)).max() < 1e-6
    for q in qs:
        assert ref.sv[q - 1] > 1.05 * ref.sv[q]  # a gap: the subspace is unique
        assert _sin_theta(U[:, :q], ref.U[:, :q]) < 1e-5, q
    return U, sv


def test_maxwell_basis_small(ctx, mp):
    # 24 x 24 pixels, 16 sites (96 dipoles), 96 excitations
    _gpu_vs_oracle(ctx, mp, (24, 24), 16, 96, [4, 8, 12], seed=3)


def test_maxwell_basis_64_fig1_excitations(ctx, mp):
    # 64 sites (384 dipoles) and Fig. 1's 500 excitations; q = 128 keeps
    # directions down to sigma ~ 3e-9 sigma_1
    _gpu_vs_oracle(ctx, mp, (64, 64), 64, 500, [32, 64, 128], seed=5)


def test_maxwell_basis_rectangular_fewer_excitations_than_dipoles(ctx, mp):
    # L = 120 < 6 D = 192: Y has at most L nonzero singular values
    _gpu_vs_oracle(ctx, mp, (48, 96), 32, 120, [16, 40], seed=7)


def test_maxwell_basis_full_size_256(ctx, mp):
    # the 256 x 256 workload's basis size: q = 128 from 500 excitations
    _gpu_vs_oracle(ctx, mp, (256, 256), 64, 500, [64, 128], seed=w.BASE_SEED)


def test_maxwell_basis_loads_and_is_reproducible(ctx, mp):
    src = _sources(16)
    om = w.random_excitations(96, 64, seed=11)
    U1, s1 = mp.maxwell_basis_2d(ctx, (32, 32), 16, src, om)
    U2, s2 = mp.maxwell_basis_2d(ctx, (32, 32), 16, src, om)
    ctx.synchronize()
    assert torch.equal(U1, U2) and np.array_equal(s1, s2)  # fixed-order FP64 reductions
    B = mp.Basis(ctx, U1)
    assert (B.N, B.q) == (1024, 16)


def test_maxwell_basis_rejects_bad_shapes(ctx, mp):
    src = _sources(16)
    om = w.random_excitations(96, 64, seed=1)
    with pytest.raises(mp.MpiError, match="MPI_ERR_SHAPE"):
        mp.maxwell_basis_2d(ctx, (8, 8), 4, src, om)  # N = 64 < 6 D = 96
    with pytest.raises(mp.MpiError, match="MPI_ERR_SHAPE"):
        mp.maxwell_basis_2d(ctx, (32, 32), 65, src, om)  # q > L
