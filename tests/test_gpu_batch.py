"""Batched slices of uneven size and coil count replayed as one CUDA graph
(mpi_batch_*): every slice's result must equal the per-slice calls, and match
the FP64 oracle within the FP32 operator tolerance."""

import numpy as np
import pytest
import torch

import workloads as w
from oracle import fourier, operator as op

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_batch_pair_matches_single_calls(prec):
    import paper_2008_09042_gb300 as mp

    ctx = mp.Context(0)
    sizes = {64: 16, 96: 24, 128: 32}
    bases = {n: (w.smooth_orthonormal_basis(n, n, q, seed=n), None) for n, q in sizes.items()}
    bases = {n: (U, mp.Basis(ctx, U.T)) for n, (U, _) in bases.items()}
    rng = np.random.default_rng(0)
    slices, refs = [], []
    for i in range(7):
        n = [64, 96, 128][i % 3]
        C = [4, 8, 12][(i // 3) % 3]
        U, B = bases[n]
        q = sizes[n]
        idx = w.mask_to_indices(w.poisson_disc_mask(n, n, 4 + i % 3, calib=(8, 8), seed=i))
        plan = mp.Plan(ctx, (n, n), sample_idx=idx)
        a = torch.from_numpy(w.random_coefficients(C, q, seed=10 + i).astype(np.complex64)).cuda()
        p = torch.from_numpy(w.random_image(n * n, seed=20 + i).astype(np.complex64)).cuda()
        y = torch.empty((C, idx.size), dtype=torch.complex64, device="cuda")
        x = torch.empty((n * n,), dtype=torch.complex64, device="cuda")
        slices.append(dict(plan=plan, basis=B, alpha=a, p=p, y=y, x=x))
        refs.append((U, idx, n))
    batch = mp.Batch(ctx, slices, kind="pair", prec=prec)
    # the slices of each grid share a basis: one grouped expansion per grid and
    # direction, and every slice's four FFT / gather passes
    assert batch.groups() == 3
    assert batch.kernels() == 4 * len(slices) + 2 * 3
    for rep in range(2):
        for s in slices:
            s["y"].zero_()
            s["x"].zero_()
        batch.run()
        ctx.synchronize()
        for s, (U, idx, n) in zip(slices, refs):
            y1 = mp.forward(ctx, s["plan"], s["basis"], s["alpha"], s["p"], prec)
            x1 = mp.adjoint(ctx, s["plan"], s["basis"], s["alpha"], y1, prec)
            assert torch.equal(s["y"], y1) and torch.equal(s["x"], x1)
    # one slice against the oracle
    s, (U, idx, n) = slices[4], refs[4]
    Fs = fourier.CartesianSampling((n, n), idx)
    U64 = U.astype(np.complex64).astype(np.complex128)
    a64 = s["alpha"].cpu().numpy().astype(np.complex128)
    p64 = s["p"].cpu().numpy().astype(np.complex128)
    tol = 1e-5 if prec == "fp32" else 5e-3
    y_ref = op.forward(Fs, U64, a64, p64)
    assert rel(s["y"].cpu().numpy(), y_ref) < tol
    batch.close()
