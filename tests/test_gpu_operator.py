"""GPU parity of the encoding operator against the FP64 oracle.

Every case runs the CUDA path through the C ABI and compares element by
element with the oracle on the same seeded inputs.  Tolerance for the FP32 path:
relative L2 error <= 1e-5 on every output.
"""

import numpy as np
import pytest
import torch

import workloads as w
from oracle import basis as obasis, fourier, nufft, operator as op, solvers

pytestmark = pytest.mark.gpu
TOL = 1e-5


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def c64(x, dev="cuda"):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, dtype=np.complex64))).to(dev)


def f64(t):
    return t.detach().cpu().numpy().astype(np.complex128)


@pytest.fixture(scope="module")
def mp():
    import paper_2008_09042_gb300 as mp

    return mp


@pytest.fixture(scope="module")
def ctx(mp):
    return mp.Context(0)


def _case(ctx, mp, shape, C, q, mask, U=None, seed=0):
    rng = np.random.default_rng(seed)
    N = int(np.prod(shape))
    if U is None:
        U = w.smooth_orthonormal_basis(shape[-2], shape[-1], q, seed=seed) if len(shape) == 2 else \
            np.linalg.qr(rng.normal(size=(N, q)) + 1j * rng.normal(size=(N, q)))[0]
    # the problem is defined by the FP32 values the GPU receives
    U = U.astype(np.complex64).astype(np.complex128)
    idx = w.mask_to_indices(mask)
    Fs = fourier.CartesianSampling(shape, idx)
    a = w.random_coefficients(C, q, seed=seed + 1).astype(np.complex64).astype(np.complex128)
    p = w.random_image(N, seed=seed + 2).astype(np.complex64).astype(np.complex128)
    plan = mp.Plan(ctx, shape, sample_idx=idx)
    B = mp.Basis(ctx, U.T)
    return dict(U=U, Fs=Fs, a=a, p=p, plan=plan, B=B, C=C, q=q, N=N, M=idx.size, rng=rng)


def _check_all(ctx, mp, cs):
    U, Fs, a, p, plan, B = cs["U"], cs["Fs"], cs["a"], cs["p"], cs["plan"], cs["B"]
    rng = cs["rng"]
    C, q, N, M = cs["C"], cs["q"], cs["N"], cs["M"]
    ag, pg = c64(a), c64(p)
    # forward (Eq. 5)
    y = mp.forward(ctx, plan, B, ag, pg)
    assert rel(f64(y), op.forward(Fs, U, a, p)) < TOL
    # adjoint
    r = (rng.normal(size=(C, M)) + 1j * rng.normal(size=(C, M))).astype(np.complex64).astype(np.complex128)
    rg = c64(r)
    x = mp.adjoint(ctx, plan, B, ag, rg)
    assert rel(f64(x), op.adjoint(Fs, U, a, r)) < TOL
    # Jacobian (Eq. 7)
    dp = w.random_image(N, seed=7).astype(np.complex64).astype(np.complex128)
    da = w.random_coefficients(C, q, seed=8).astype(np.complex64).astype(np.complex128)
    dy = mp.jacobian(ctx, plan, B, ag, pg, c64(dp), c64(da))
    assert rel(f64(dy), op.jacobian(Fs, U, a, p, dp, da)) < TOL
    # Jacobian adjoint
    gp, ga = mp.jacobian_adjoint(ctx, plan, B, ag, pg, rg)
    rp, ra = op.jacobian_adjoint(Fs, U, a, p, r)
    assert rel(f64(gp), rp) < TOL
    assert rel(f64(ga), ra) < TOL
    # maps
    s = mp.basis_expand(ctx, B, ag)
    assert rel(f64(s), op.expand(U, a)) < TOL


def test_cartesian_64_vd_lines_maxwell_basis(ctx, mp):
    b = obasis.build_maxwell_basis_2d(64, 64, 32, n_sites=32, n_exc=200, seed=0)
    mask = w.vd_lines_mask(64, 64, 3, 16, seed=1)
    cs = _case(ctx, mp, (64, 64), 4, 32, mask, U=b.U)
    _check_all(ctx, mp, cs)


@pytest.mark.parametrize("shape,C,q", [((48, 96), 5, 20), ((32, 16), 17, 3), ((192, 64), 3, 40),
                                       ((128, 320), 2, 9)])
def test_cartesian_ragged_shapes(ctx, mp, shape, C, q):
    # coil counts that leave a partial coil block, non-square grids, radix-3/5 lengths
    mask = w.poisson_disc_mask(shape[0], shape[1], 3, calib=(8, 8), seed=3)
    cs = _case(ctx, mp, shape, C, q, mask, seed=4)
    _check_all(ctx, mp, cs)


def test_cartesian_full_size_256_c16_q128(ctx, mp):
    mask = w.poisson_disc_mask(256, 256, 6, calib=(24, 24), seed=5)
    cs = _case(ctx, mp, (256, 256), 16, 128, mask, seed=6)
    _check_all(ctx, mp, cs)


def test_cartesian_3d_volume_pipelined_line_passes(ctx, mp):
    # a 32 x 64 x 128 volume with 20 coils: thousands of 32-line tiles per pass,
    # which the library runs on persistent, software-pipelined CTAs
    shape, C, q = (32, 64, 128), 20, 4
    rng = np.random.default_rng(21)
    N = int(np.prod(shape))
    U = np.linalg.qr(rng.normal(size=(N, q)) + 1j * rng.normal(size=(N, q)))[0]
    mask = w.poisson_disc_mask_3d(*shape, R=4, calib=(8, 8), seed=22)
    cs = _case(ctx, mp, shape, C, q, mask, U=U, seed=23)
    U, Fs, a, p, plan, B = cs["U"], cs["Fs"], cs["a"], cs["p"], cs["plan"], cs["B"]
    ag, pg = c64(a), c64(p)
    assert rel(f64(mp.forward(ctx, plan, B, ag, pg)), op.forward(Fs, U, a, p)) < TOL
    r = w.random_coefficients(C, cs["M"], seed=24, decay=False).astype(np.complex64).astype(np.complex128)
    assert rel(f64(mp.adjoint(ctx, plan, B, ag, c64(r))), op.adjoint(Fs, U, a, r)) < TOL
    ctx.synchronize()


def test_fully_sampled_and_empty(ctx, mp):
    full = np.ones((32, 32), dtype=bool)
    cs = _case(ctx, mp, (32, 32), 3, 8, full, seed=9)
    _check_all(ctx, mp, cs)
    # fully sampled, unitary F: adjoint(forward(p)) = sum_k |s_k|^2 p
    ag, pg = c64(cs["a"]), c64(cs["p"])
    back = f64(mp.adjoint(ctx, cs["plan"], cs["B"], ag, mp.forward(ctx, cs["plan"], cs["B"], ag, pg)))
    s = op.expand(cs["U"], cs["a"])
    assert rel(back, np.sum(np.abs(s) ** 2, axis=0) * cs["p"]) < TOL
    # no samples at all: y is empty and the adjoint is exactly zero
    empty = np.zeros((32, 32), dtype=bool)
    ce = _case(ctx, mp, (32, 32), 2, 4, empty, seed=10)
    ag = c64(ce["a"])
    y = mp.forward(ctx, ce["plan"], ce["B"], ag, c64(ce["p"]))
    assert y.shape == (2, 0)
    x = mp.adjoint(ctx, ce["plan"], ce["B"], ag, torch.zeros((2, 0), dtype=torch.complex64, device="cuda"))
    assert torch.count_nonzero(x).item() == 0


def test_adjoint_dot_products_at_full_size(ctx, mp):
    # <G p, r> = <p, G^H r> and <J d, r> = <d, J^H r> hold at any size; checked
    # in FP64 from the FP32 outputs.
    mask = w.poisson_disc_mask(256, 256, 6, calib=(24, 24), seed=5)
    cs = _case(ctx, mp, (256, 256), 16, 128, mask, seed=11)
    ag, pg = c64(cs["a"]), c64(cs["p"])
    r = w.random_coefficients(16, cs["M"], seed=12, decay=False)
    rg = c64(r)
    r = r.astype(np.complex64).astype(np.complex128)
    lhs = np.vdot(f64(mp.forward(ctx, cs["plan"], cs["B"], ag, pg)), r)
    rhs = np.vdot(cs["p"], f64(mp.adjoint(ctx, cs["plan"], cs["B"], ag, rg)))
    assert abs(lhs - rhs) / abs(lhs) < 1e-5
    dp = c64(w.random_image(cs["N"], seed=13))
    da = c64(w.random_coefficients(16, 128, seed=14))
    gp, ga = mp.jacobian_adjoint(ctx, cs["plan"], cs["B"], ag, pg, rg)
    lhs = np.vdot(f64(mp.jacobian(ctx, cs["plan"], cs["B"], ag, pg, dp, da)), r)
    rhs = np.vdot(f64(dp), f64(gp)) + np.vdot(f64(da), f64(ga))
    assert abs(lhs - rhs) / abs(lhs) < 1e-5


def test_jacobian_central_difference_32_directions(ctx, mp):
    # G is bilinear: (G(x + h d) - G(x - h d)) / 2h = J d exactly; h = 1e-3,
    # 32 random directions, evaluated with the GPU forward.
    mask = w.poisson_disc_mask(64, 64, 4, calib=(12, 12), seed=15)
    cs = _case(ctx, mp, (64, 64), 4, 16, mask, seed=16)
    a, p = cs["a"], cs["p"]
    h = 1e-3
    for k in range(32):
        dp = w.random_image(cs["N"], seed=100 + k)
        da = w.random_coefficients(4, 16, seed=200 + k)
        yp = f64(mp.forward(ctx, cs["plan"], cs["B"], c64(a + h * da), c64(p + h * dp)))
        ym = f64(mp.forward(ctx, cs["plan"], cs["B"], c64(a - h * da), c64(p - h * dp)))
        J = f64(mp.jacobian(ctx, cs["plan"], cs["B"], c64(a), c64(p), c64(dp), c64(da)))
        # FP32 inputs perturbed by h: difference quotient error ~ eps32 |G| / h
        assert rel((yp - ym) / (2 * h), J) < 5e-3


def test_autograd_backward_is_jacobian_adjoint(ctx, mp):
    mask = w.poisson_disc_mask(64, 64, 3, calib=(12, 12), seed=17)
    cs = _case(ctx, mp, (64, 64), 3, 12, mask, seed=18)
    p = c64(cs["p"]).requires_grad_(True)
    a = c64(cs["a"]).requires_grad_(True)
    y = mp.mpi_operator(p, a, ctx, cs["plan"], cs["B"])
    target = c64(w.random_coefficients(3, cs["M"], seed=19, decay=False))
    loss = 0.5 * (y - target).abs().pow(2).sum()
    loss.backward()
    rp, ra = op.jacobian_adjoint(cs["Fs"], cs["U"], cs["a"], cs["p"],
                                 op.forward(cs["Fs"], cs["U"], cs["a"], cs["p"]) - f64(target))
    # torch's gradient of a real loss is the conjugate-Wirtinger one: J^H (G(x) - y)
    assert rel(f64(p.grad), rp) < 1e-4
    assert rel(f64(a.grad), ra) < 1e-4


def test_bad_arguments_rejected_before_launch(ctx, mp):
    idx = np.array([3, 2], dtype=np.int32)  # not increasing
    with pytest.raises(mp.MpiError):
        mp.Plan(ctx, (32, 32), sample_idx=idx)
    with pytest.raises(mp.MpiError):
        mp.Plan(ctx, (32, 32), sample_idx=np.array([0, 1024], dtype=np.int32))  # out of range
    with pytest.raises(mp.MpiError):
        mp.Plan(ctx, (30, 32), sample_idx=np.array([0], dtype=np.int32))  # unsupported length


@pytest.mark.parametrize("pinned", [False, True, "mixed"])
def test_host_buffer_calls_match_device_calls(ctx, mp, pinned):
    # mpi_forward_host / mpi_adjoint_host run the same kernels, on pinned host
    # buffers in place and on staged copies of pageable ones: results equal the
    # device-pointer calls bit for bit, and the oracle within the FP32
    # tolerance.  Pageable, pinned, and pinned alpha with pageable data.
    mask = w.poisson_disc_mask(64, 96, 4, calib=(12, 12), seed=60)
    cs = _case(ctx, mp, (64, 96), 5, 12, mask, seed=61)
    C, M = cs["C"], cs["M"]
    r = w.random_coefficients(C, M, seed=62, decay=False).astype(np.complex64)

    def host(x, pin):
        t = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64)))
        return t.pin_memory() if pin else t

    a_h = host(cs["a"], bool(pinned))
    p_h, r_h = host(cs["p"], pinned is True), host(r, pinned is True)
    y_h = mp.forward_host(ctx, cs["plan"], cs["B"], a_h, p_h)
    x_h = mp.adjoint_host(ctx, cs["plan"], cs["B"], a_h, r_h)
    assert not y_h.is_cuda and not x_h.is_cuda
    y_d = mp.forward(ctx, cs["plan"], cs["B"], a_h.cuda(), p_h.cuda())
    x_d = mp.adjoint(ctx, cs["plan"], cs["B"], a_h.cuda(), r_h.cuda())
    assert torch.equal(y_h, y_d.cpu()) and torch.equal(x_h, x_d.cpu())
    assert rel(y_h.numpy(), op.forward(cs["Fs"], cs["U"], cs["a"], cs["p"])) < TOL
    assert rel(x_h.numpy(), op.adjoint(cs["Fs"], cs["U"], cs["a"], r.astype(np.complex128))) < TOL
    with pytest.raises(TypeError):
        mp.forward_host(ctx, cs["plan"], cs["B"], a_h.cuda(), p_h)


def test_host_buffer_calls_without_samples(ctx, mp):
    # a plan with no samples: the forward's y and the adjoint's input are empty
    n, q, C = 32, 4, 3
    U = w.smooth_orthonormal_basis(n, n, q, seed=80)
    plan = mp.Plan(ctx, (n, n), sample_idx=np.zeros(0, dtype=np.int32))
    B = mp.Basis(ctx, U.T)
    a = torch.from_numpy(w.random_coefficients(C, q, seed=81).astype(np.complex64)).pin_memory()
    p = torch.from_numpy(w.random_image(n * n, seed=82).astype(np.complex64))
    y = mp.forward_host(ctx, plan, B, a, p)
    assert tuple(y.shape) == (C, 0)
    x = mp.adjoint_host(ctx, plan, B, a, y)
    assert torch.count_nonzero(x).item() == 0


def test_cartesian_rows_without_samples(ctx, mp):
    # Only every third k-space row is sampled: the adjoint's row pass skips the
    # empty rows and the pass along y reads them as zeros (the plan's row mask),
    # after a call that filled the workspace with non-zero values.
    shape = (96, 64)
    mask = np.zeros(shape, dtype=bool)
    mask[::3, :] = True
    mask[40:56, 24:40] = True  # calibration block: some rows sampled in part
    cs = _case(ctx, mp, shape, 4, 10, mask, seed=70)
    C, M = cs["C"], cs["M"]
    r = w.random_coefficients(C, M, seed=71, decay=False).astype(np.complex64).astype(np.complex128)
    ag, pg = c64(cs["a"]), c64(cs["p"])
    mp.forward(ctx, cs["plan"], cs["B"], ag, pg)  # leaves non-zero data in the workspace
    x = mp.adjoint(ctx, cs["plan"], cs["B"], ag, c64(r))
    assert rel(f64(x), op.adjoint(cs["Fs"], cs["U"], cs["a"], r)) < TOL
    y = mp.forward(ctx, cs["plan"], cs["B"], ag, pg)
    assert rel(f64(y), op.forward(cs["Fs"], cs["U"], cs["a"], cs["p"])) < TOL
    gp, ga = mp.jacobian_adjoint(ctx, cs["plan"], cs["B"], ag, pg, c64(r))
    rp, ra = op.jacobian_adjoint(cs["Fs"], cs["U"], cs["a"], cs["p"], r)
    assert rel(f64(gp), rp) < TOL and rel(f64(ga), ra) < TOL


def test_launch_count_grows(ctx, mp):
    before = ctx.launches()
    mask = w.poisson_disc_mask(32, 32, 3, calib=(8, 8), seed=20)
    cs = _case(ctx, mp, (32, 32), 2, 4, mask, seed=21)
    mp.forward(ctx, cs["plan"], cs["B"], c64(cs["a"]), c64(cs["p"]))
    torch.cuda.synchronize()
    assert ctx.launches() >= before + 3


# ----------------------------------------------------------------- radial

def _radial_case(ctx, mp, n, C, q, spokes, readout, seed=30):
    k = w.golden_angle_radial(spokes, readout).astype(np.float32)
    U = w.smooth_orthonormal_basis(n, n, q, seed=seed).astype(np.complex64).astype(np.complex128)
    a = w.random_coefficients(C, q, seed=seed + 1).astype(np.complex64).astype(np.complex128)
    p = w.random_image(n * n, seed=seed + 2).astype(np.complex64).astype(np.complex128)
    plan = mp.Plan(ctx, (n, n), traj=k, kb_width=6, oversamp=2.0)
    B = mp.Basis(ctx, U.T)
    kb = nufft.KBGriddingNUFFT((n, n), k.astype(np.float64), W=6, sigma=2.0)
    return dict(k=k, U=U, a=a, p=p, plan=plan, B=B, kb=kb, C=C, q=q, N=n * n, M=k.shape[0])


def test_radial_gridding_indices_bit_exact(ctx, mp):
    cs = _radial_case(ctx, mp, 64, 2, 8, 16, 128)
    got = cs["plan"].grid_index().cpu().numpy()
    ref = nufft.gridding_indices(cs["k"], 128, 6)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("n,C,q,spokes,readout", [(64, 3, 8, 16, 128), (256, 12, 96, 64, 512)])
def test_radial_operator_matches_fp64_gridding(ctx, mp, n, C, q, spokes, readout):
    cs = _radial_case(ctx, mp, n, C, q, spokes, readout)
    kb, U, a, p = cs["kb"], cs["U"], cs["a"], cs["p"]
    ag, pg = c64(a), c64(p)
    y = mp.forward(ctx, cs["plan"], cs["B"], ag, pg)
    assert rel(f64(y), op.forward(kb, U, a, p)) < TOL
    r = w.random_coefficients(C, cs["M"], seed=40, decay=False).astype(np.complex64).astype(np.complex128)
    x = mp.adjoint(ctx, cs["plan"], cs["B"], ag, c64(r))
    assert rel(f64(x), op.adjoint(kb, U, a, r)) < TOL
    gp, ga = mp.jacobian_adjoint(ctx, cs["plan"], cs["B"], ag, pg, c64(r))
    rp, ra = op.jacobian_adjoint(kb, U, a, p, r)
    assert rel(f64(gp), rp) < TOL and rel(f64(ga), ra) < TOL


@pytest.mark.parametrize("W,C,sigma", [(2, 5, 2.0), (3, 1, 2.0), (4, 4, 1.5), (7, 9, 2.0), (8, 2, 1.5), (6, 19, 2.0)])
def test_radial_kernel_widths_and_wrapped_windows(ctx, mp, W, C, sigma):
    # Every kernel width the plan accepts; coil counts that leave a ragged group
    # of four and one beyond sixteen (two coil chunks) in the spreading; a
    # 48-point grid (not a multiple of the 32-cell strips); and samples on the
    # k-space edge whose W x W footprints wrap around the grid's first row and
    # column.
    n, q = 32, 4
    rng = np.random.default_rng(50 + W)
    k = np.concatenate([
        w.golden_angle_radial(8, 64),
        rng.uniform(-np.pi, np.pi, size=(200, 2)),
        np.array([[-np.pi, -np.pi], [-np.pi, 0.0], [0.0, -np.pi], [np.pi * 0.999, -np.pi * 0.999]]),
    ]).astype(np.float32)
    U = w.smooth_orthonormal_basis(n, n, q, seed=W).astype(np.complex64).astype(np.complex128)
    a = w.random_coefficients(C, q, seed=W + 1).astype(np.complex64).astype(np.complex128)
    p = w.random_image(n * n, seed=W + 2).astype(np.complex64).astype(np.complex128)
    r = w.random_coefficients(C, k.shape[0], seed=W + 3, decay=False).astype(np.complex64).astype(np.complex128)
    plan = mp.Plan(ctx, (n, n), traj=k, kb_width=W, oversamp=sigma)
    B = mp.Basis(ctx, U.T)
    kb = nufft.KBGriddingNUFFT((n, n), k.astype(np.float64), W=W, sigma=sigma)
    assert rel(f64(mp.forward(ctx, plan, B, c64(a), c64(p))), op.forward(kb, U, a, p)) < TOL
    assert rel(f64(mp.adjoint(ctx, plan, B, c64(a), c64(r))), op.adjoint(kb, U, a, r)) < TOL


def test_radial_close_to_direct_nudft(ctx, mp):
    cs = _radial_case(ctx, mp, 64, 2, 8, 24, 128)
    ex = fourier.DirectNUDFT((64, 64), cs["k"].astype(np.float64))
    y = f64(mp.forward(ctx, cs["plan"], cs["B"], c64(cs["a"]), c64(cs["p"])))
    ref_exact = op.forward(ex, cs["U"], cs["a"], cs["p"])
    ref_kb = op.forward(cs["kb"], cs["U"], cs["a"], cs["p"])
    kb_err = rel(ref_kb, ref_exact)  # the gridding's own error, FP64
    assert rel(y, ref_exact) < kb_err + 1e-5


def test_destroy_context_before_children(mp):
    # a garbage collector may finalise a context before the plans, bases and
    # batches made on it; destroying them afterwards must only free their memory
    ctx2 = mp.Context(0)
    n, C, q = 32, 2, 4
    U = w.smooth_orthonormal_basis(n, n, q, seed=1)
    idx = w.mask_to_indices(w.poisson_disc_mask(n, n, 4, calib=(8, 8), seed=2))
    plan = mp.Plan(ctx2, (n, n), sample_idx=idx)
    B = mp.Basis(ctx2, U.T)
    a = c64(w.random_coefficients(C, q, seed=3))
    p = c64(w.random_image(n * n, seed=4))
    y = torch.empty((C, idx.size), dtype=torch.complex64, device="cuda")
    x = torch.empty((n * n,), dtype=torch.complex64, device="cuda")
    bt = mp.Batch(ctx2, [dict(plan=plan, basis=B, alpha=a, p=p, y=y, x=x)], kind="pair")
    bt.run()
    ctx2.close()
    bt.close()
    B.close()
    plan.close()


@pytest.mark.parametrize("choice", [8, 16, 32, -1])
@pytest.mark.parametrize("dims,C,q,R", [((256, 256), 6, 24, 6), ((128, 192), 5, 16, 4), ((96, 64), 4, 12, 3)])
def test_line_pass_kernels_match_oracle(mp, choice, dims, C, q, R):
    # every FFT line-pass kernel the autotuner chooses between, fixed in turn:
    # forward and adjoint against the oracle (row-masked passes along y included)
    ctx = mp.Context(0)
    ctx.set_line_kernel(choice)
    mask = w.poisson_disc_mask(dims[0], dims[1], R, calib=(8, 8), seed=17)
    cs = _case(ctx, mp, dims, C, q, mask, seed=18)
    ag, pg = c64(cs["a"]), c64(cs["p"])
    y = mp.forward(ctx, cs["plan"], cs["B"], ag, pg)
    assert rel(f64(y), op.forward(cs["Fs"], cs["U"], cs["a"], cs["p"])) < TOL
    r = w.random_coefficients(C, cs["M"], seed=19, decay=False).astype(np.complex64).astype(np.complex128)
    x = mp.adjoint(ctx, cs["plan"], cs["B"], ag, c64(r))
    assert rel(f64(x), op.adjoint(cs["Fs"], cs["U"], cs["a"], r)) < TOL
    ctx.synchronize()


def _volume_mask(dims, kind, seed):
    """3D sampling patterns for the plane passes: whole readouts on a
    Poisson-disc (kz, ky) set; the same with a random 60 % of the samples kept
    (rows partly sampled, some planes empty); or a dense centre (every row of
    the central planes sampled, more rows per plane than the pipelined kernel
    keeps in shared memory)."""
    nz, ny, nx = dims
    m = w.poisson_disc_mask_3d(nz, ny, nx, R=8, calib=(12, 12), seed=seed)
    if kind == "partial":
        rng = np.random.default_rng(seed + 1)
        m = m & (rng.random(m.shape) < 0.6)
        m[: nz // 4] = False  # a run of planes without samples
    elif kind == "dense":
        m[nz // 2 - 2: nz // 2 + 2] = True
    return m


@pytest.mark.parametrize("choice", [0, -2, -3])
@pytest.mark.parametrize("dims,kind", [
    ((64, 64, 128), "readouts"),
    ((64, 128, 128), "readouts"),
    ((96, 96, 96), "partial"),
    ((64, 128, 64), "partial"),
    ((64, 64, 96), "dense"),
    ((64, 128, 128), "dense"),
])
def test_line_pass_kernels_3d_volume(mp, choice, dims, kind):
    # the 3D path's passes along y and x: the pipelined plane kernel (0, where
    # each plane's rows with samples fit), one CTA per plane (-3, and 0 where
    # they do not) or the separate, tuned passes (-2)
    from oracle import tucker

    ctx = mp.Context(0)
    ctx.set_line_kernel(choice)
    ranks, q, C = (8, 12, 12), 16, 3
    core, fac = w.smooth_tucker_basis(dims, ranks, q, seed=27)
    core = core.astype(np.complex64).astype(np.complex128)
    fac = [f.astype(np.complex64).astype(np.complex128) for f in fac]
    tb = tucker.TuckerBasis(core, fac)
    idx = w.mask_to_indices(_volume_mask(dims, kind, seed=28))
    Fs = fourier.CartesianSampling(dims, idx)
    N = int(np.prod(dims))
    a = w.random_coefficients(C, q, seed=29).astype(np.complex64).astype(np.complex128)
    p = w.random_image(N, seed=30).astype(np.complex64).astype(np.complex128)
    r = w.random_coefficients(C, idx.size, seed=31, decay=False).astype(np.complex64).astype(np.complex128)
    plan = mp.Plan(ctx, dims, sample_idx=idx)
    B = mp.TuckerBasis(ctx, core, fac)
    ctx.profile(True)
    assert rel(f64(mp.forward(ctx, plan, B, c64(a), c64(p))), op.forward(Fs, tb, a, p)) < TOL
    assert rel(f64(mp.adjoint(ctx, plan, B, c64(a), c64(r))), op.adjoint(Fs, tb, a, r)) < TOL
    ctx.synchronize()
    _, kern = ctx.profile_read(kernels=True)
    ctx.profile(False)
    pipe = {k for k in kern if k.startswith("k_plane_pipe")}
    single = {k for k in kern if k.startswith("k_plane_yx")}
    if choice == -2:
        assert not pipe and not single
    elif choice == -3 or kind == "dense" and dims[1] == 128:
        assert single == {"k_plane_yx<fwd>", "k_plane_yx<inv>"} and not pipe
    else:
        assert pipe == {"k_plane_pipe<fwd>", "k_plane_pipe<inv>"} and not single
