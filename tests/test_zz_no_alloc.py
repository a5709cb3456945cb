"""The allocation-free forward entry point, through the C ABI.

mpi_forward_noalloc serves callers that cannot call cudaMalloc while running
(a fixed device-memory pool set up at start-up, or a real-time loop that must
not block in the allocator).  Its output must match mpi_forward's within the
operator tolerance on two calls in a row (the static scratch keeps the last
call's contents, which must not leak into the next result).  This file is
collected last on purpose.
"""

import ctypes

import numpy as np
import pytest
import torch

import workloads as w

pytestmark = pytest.mark.gpu
TOL = 1e-5


def _rel(a, b):
    a = a.cpu().numpy().astype(np.complex128)
    b = b.cpu().numpy().astype(np.complex128)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _slice(mp, ctx, n=256, q=64):
    plan = mp.Plan(ctx, (n, n), sample_idx=w.mask_to_indices(w.poisson_disc_mask(n, n, 6, calib=(24, 24), seed=1)))
    basis = mp.Basis(ctx, w.smooth_orthonormal_basis(n, n, q, seed=2).T)
    return plan, basis


def test_forward_noalloc_first_call_leaves_workspace_empty():
    # On a fresh context, before any other operator call: the allocation-free
    # forward must not grow the context's workspace, and its result must match
    # the allocating forward's (called afterwards).
    import paper_2008_09042_gb300 as mp
    from paper_2008_09042_gb300 import _lib

    lib = _lib.load()
    ctx = mp.Context(0)
    n, C, q = 256, 16, 64
    plan, basis = _slice(mp, ctx, n, q)
    assert ctx.workspace_bytes() == 0
    a = torch.from_numpy(w.random_coefficients(C, q, seed=30).astype(np.complex64)).cuda()
    p = torch.from_numpy(w.random_image(n * n, seed=31).astype(np.complex64)).cuda()
    y = torch.full((C, plan.M), float("nan"), dtype=torch.complex64, device="cuda")
    vp = ctypes.c_void_p
    st = lib.mpi_forward_noalloc(ctx.h, plan.h, basis.h, vp(a.data_ptr()), C, vp(p.data_ptr()), vp(y.data_ptr()))
    assert st == 0, lib.mpi_last_error(ctx.h)
    ctx.synchronize()
    assert ctx.workspace_bytes() == 0
    y_ref = mp.forward(ctx, plan, basis, a, p)
    torch.cuda.synchronize()
    assert _rel(y, y_ref) < TOL


def test_forward_noalloc_matches_forward_twice():
    import paper_2008_09042_gb300 as mp
    from paper_2008_09042_gb300 import _lib

    lib = _lib.load()
    ctx = mp.Context(0)
    n, C, q = 256, 16, 64
    plan, basis = _slice(mp, ctx, n, q)
    vp = ctypes.c_void_p
    for call in range(2):
        a = torch.from_numpy(w.random_coefficients(C, q, seed=10 + call).astype(np.complex64)).cuda()
        p = torch.from_numpy(w.random_image(n * n, seed=20 + call).astype(np.complex64)).cuda()
        y_ref = torch.empty((C, plan.M), dtype=torch.complex64, device="cuda")
        y = torch.full((C, plan.M), float("nan"), dtype=torch.complex64, device="cuda")
        st = lib.mpi_forward(ctx.h, plan.h, basis.h, vp(a.data_ptr()), C, vp(p.data_ptr()), vp(y_ref.data_ptr()), 0)
        assert st == 0
        st = lib.mpi_forward_noalloc(ctx.h, plan.h, basis.h, vp(a.data_ptr()), C, vp(p.data_ptr()),
                                     vp(y.data_ptr()))
        assert st == 0, lib.mpi_last_error(ctx.h)
        torch.cuda.synchronize()
        assert torch.isfinite(y.real).all() and torch.isfinite(y.imag).all()
        assert _rel(y, y_ref) < TOL


def test_forward_noalloc_rejects_oversize():
    import paper_2008_09042_gb300 as mp
    from paper_2008_09042_gb300 import _lib

    lib = _lib.load()
    ctx = mp.Context(0)
    n, C, q = 512, 9, 4  # C * N = 2,359,296 > 2,097,152
    plan = mp.Plan(ctx, (n, n), sample_idx=np.arange(0, n * n, 97, dtype=np.int32))
    basis = mp.Basis(ctx, np.eye(n * n, q, dtype=np.complex64).T)
    a = torch.zeros((C, q), dtype=torch.complex64, device="cuda")
    p = torch.zeros((n * n,), dtype=torch.complex64, device="cuda")
    y = torch.zeros((C, plan.M), dtype=torch.complex64, device="cuda")
    vp = ctypes.c_void_p
    st = lib.mpi_forward_noalloc(ctx.h, plan.h, basis.h, vp(a.data_ptr()), C, vp(p.data_ptr()), vp(y.data_ptr()))
    assert st == 2  # MPI_ERR_SHAPE
    assert b"static scratch" in lib.mpi_last_error(ctx.h)
