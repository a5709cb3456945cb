"""The bounded-wait failure path of the tensor-core kernels, made to run on a
GPU without faulting it.

With a short wait limit and the fault-injection hook that makes the FP32
expansion's copy producer issue no copy at all, the consumers' waits on the
stages never loaded run out: the kernel records MPI_ERR_TIMEOUT in the
context's device error word, drains the copies it issued, frees its tensor
memory and returns.  The host learns of it at mpi_ctx_synchronize, and the
next call on the same context must be correct.
"""

import numpy as np
import pytest
import torch

import workloads as w
from oracle import fourier, operator as op

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_wait_timeout_reported_and_context_recovers():
    import paper_2008_09042_gb300 as mp
    from paper_2008_09042_gb300._lib import MpiError

    ctx = mp.Context(0)
    n, C, q = 128, 8, 32
    U = w.smooth_orthonormal_basis(n, n, q, seed=41).astype(np.complex64)
    idx = w.mask_to_indices(w.poisson_disc_mask(n, n, 4, calib=(16, 16), seed=42))
    plan = mp.Plan(ctx, (n, n), sample_idx=idx)
    B = mp.Basis(ctx, U.T)
    assert mp.expand_path(ctx, B, C, "fp32") == "tf32x3"
    a = w.random_coefficients(C, q, seed=43).astype(np.complex64)
    p = w.random_image(n * n, seed=44).astype(np.complex64)
    ag, pg = torch.from_numpy(a).cuda(), torch.from_numpy(p).cuda()
    mp.forward(ctx, plan, B, ag, pg)  # everything loaded and tuned first
    ctx.synchronize()

    ctx.set_wait_limit(2_000_000)  # about 1 ms at 2 GHz
    ctx.inject_stall(0)  # no ring stage is loaded (at this size a CTA has one per tile)
    mp.forward(ctx, plan, B, ag, pg)
    with pytest.raises(MpiError) as e:
        ctx.synchronize()
    assert e.value.status == 6  # MPI_ERR_TIMEOUT
    ctx.synchronize()  # the error word was cleared

    ctx.inject_stall(-1)
    y = mp.forward(ctx, plan, B, ag, pg)
    ctx.synchronize()
    Fs = fourier.CartesianSampling((n, n), idx)
    ref = op.forward(Fs, U.astype(np.complex128), a.astype(np.complex128), p.astype(np.complex128))
    assert _rel(y.cpu().numpy().astype(np.complex128), ref) < 1e-5
    ctx.set_wait_limit(1 << 32)
