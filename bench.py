"""Benchmark of the Maxwell Parallel Imaging encoding operator on GB300.

Metric: forward + adjoint operator pairs per second (one mpi_forward plus one
mpi_adjoint of the Maxwell-parameterised bilinear operator, Eq. 5, and its
adjoint).  The headline workload is the largest single-GPU configuration: the
3D Cartesian 96 x 128 x 128 volume with 32 coils, a Tucker-factored basis
(q = 256, ranks 32 / 40 / 40) and a 3D Poisson-disc mask (R = 8, 24 x 24
calibration), complex64 data.  The 2D Cartesian 256^2 / 16-coil slice, the
radial slice, the 64-slice batched exam and the reconstruction times are
secondary lines under "workloads".

One step = one forward + one adjoint with the inputs resident in HBM.  A
256 MiB buffer is written between timed steps (L2 flush; the 3D volume's
403 MB intermediates exceed L2 anyway).  Steps are timed with CUDA events on
the library's stream.  A second run of the same steps brackets every kernel
launch with the library's own events (on its stream) for the per-kernel times
and the roofline entry of the dominant kernel.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--workload NAME]

Multi-GPU: independent replicas (one volume per rank, no collective on the
data path); the value is the pairs of all ranks over the slowest rank's time.
"""

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as w  # noqa: E402

HEADLINE = "cart3d_128x128x96_c32_tucker256"
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0
# FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.07 GHz max SM clock
FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=HEADLINE, choices=[HEADLINE, "cart2d_256_c16_q128"])
    ap.add_argument("--prec", default="fp32", choices=["fp32", "bf16", "fp32_simt"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true", help="skip the 2D/radial/batched/recon lines")
    ap.add_argument("--profile-workload", default=None,
                    help="only run --steps forward+adjoint pairs of this workload, untimed, for an external profiler")
    ap.add_argument("--profile-op", default="pair", choices=["pair", "jacobian"],
                    help="with --profile-workload: forward+adjoint pairs, or Jacobian + Jacobian-adjoint pairs")
    ap.add_argument("--profile-coils", type=int, default=0,
                    help="with --profile-workload: run only the first N coils (a smaller case of the same "
                         "kernels for multi-pass profiler captures)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


# ----------------------------------------------------------------- workloads

def make_case(name, seed_offset=0):
    """Seeded host inputs of one workload (a dense 2D slice or the 3D Tucker volume)."""
    cfg = w.workload(name)
    base = w.BASE_SEED + seed_offset
    C, q = cfg["C"], cfg["q"]
    case = dict(name=name, cfg=cfg, C=C, q=q, dims=tuple(cfg["dims"]))
    if cfg["kind"] == "cartesian":
        ny, nx = cfg["dims"]
        case["U"] = w.smooth_orthonormal_basis(ny, nx, q, seed=base)
        if cfg["mask"] == "poisson":
            mask = w.poisson_disc_mask(ny, nx, cfg["R"], calib=cfg["calib"], seed=base + 1)
        else:
            mask = w.vd_lines_mask(ny, nx, cfg["R"], cfg["acs"], seed=base + 1)
        case["p"] = w.random_ellipses(ny, nx, seed=base + 3).ravel().astype(np.complex128)
        case["alpha"] = w.random_coefficients(C, q, seed=base + 2)
        case["tucker"] = False
        case["mask_desc"] = f"2D variable-density Poisson-disc R={cfg['R']} calib {cfg['calib']}"
    elif cfg["kind"] == "cartesian3d":
        dims = cfg["dims"]
        case["core"], case["fac"] = w.smooth_tucker_basis(dims, cfg["ranks"], q, seed=base)
        mask = w.poisson_disc_mask_3d(*dims, R=cfg["R"], calib=cfg["calib"], seed=base + 1)
        case["alpha"] = w.random_coefficients(C, q, seed=base + 2)
        case["p"] = w.random_ellipses(dims[1], dims[2], nz=dims[0], seed=base + 3).ravel().astype(np.complex128)
        case["tucker"] = True
        case["ranks"] = tuple(cfg["ranks"])
        case["mask_desc"] = (f"3D Poisson-disc over (ky, kz) R={cfg['R']} calib {cfg['calib']}, kx fully sampled")
    else:
        raise SystemExit(f"{name}: not a Cartesian workload")
    idx = w.mask_to_indices(mask)
    case["idx"] = idx
    case["N"] = int(np.prod(case["dims"]))
    case["M"] = int(idx.size)
    # fraction of k-space rows (x lines) holding samples
    nx = case["dims"][-1]
    rows = np.unique(idx // nx)
    case["row_frac"] = rows.size / (case["N"] // nx)
    return case


def gpu_objects(mp, ctx, dev, case):
    import torch

    plan = mp.Plan(ctx, case["dims"], sample_idx=case["idx"])
    basis = mp.TuckerBasis(ctx, case["core"], case["fac"]) if case["tucker"] else mp.Basis(ctx, case["U"].T)
    ctx.reserve(plan, basis, case["C"])
    a_d = torch.from_numpy(case["alpha"].astype(np.complex64)).to(dev)
    p_d = torch.from_numpy(case["p"].astype(np.complex64)).to(dev)
    return plan, basis, a_d, p_d


def basis_bytes(case, prec):
    """Bytes of the basis one expansion pass must read (dense U, or the Tucker core)."""
    ub = 4 if prec == "bf16" else 8
    if case["tucker"]:
        r1, r2, r3 = case["ranks"]
        return r1 * r2 * r3 * case["q"] * ub
    return case["N"] * case["q"] * ub


def pair_algorithmic_bytes(case, prec):
    """Algorithmic bytes of one forward + adjoint pair: per direction, the basis
    (or Tucker core) once, the per-coil image-side product once (C N complex64),
    the k-space samples (C M complex64), the image and the coefficients."""
    C, N, M, q = case["C"], case["N"], case["M"], case["q"]
    return 2 * (basis_bytes(case, prec) + 8 * C * N + 8 * C * M + 8 * N + 8 * C * q)


def kernel_bytes_per_pair(case, prec):
    """Algorithmic DRAM bytes per forward + adjoint pair of each kernel (by the
    name the library's per-kernel timing reports), for the roofline entry."""
    C, N, M, q = case["C"], case["N"], case["M"], case["q"]
    V = 8 * C * N          # one complex64 volume (or slice) per coil
    Y = 8 * C * M          # the k-space samples
    P = 8 * N              # the image
    f = case["row_frac"]   # k-space rows with samples
    out = {
        "k_fft_lines<z,fwd>": 2 * V, "k_fft_lines<z,inv>": 2 * V,
        "k_fft_lines<y,fwd>": V * (1 + f), "k_fft_lines<y,inv>": V * (1 + f),
        "k_rows_fwd_gather": f * V + Y, "k_rows_scatter_inv": Y + f * V,
        "k_pointwise<fwd>": 2 * V + P, "k_pointwise<adj>": 2 * V + P,
        # the per-plane kernel: passes along y and x with the gather (forward)
        # or the scatter (adjoint), one read and one write
        "k_plane_yx<fwd>": V + Y, "k_plane_yx<inv>": Y + V,
        # the same passes as the pipelined persistent kernel (TMA tiles)
        "k_plane_pipe<fwd>": V + Y, "k_plane_pipe<inv>": Y + V,
    }
    if case["tucker"]:
        n1, n2, n3 = case["dims"]
        r1, r2, r3 = case["ranks"]
        R = r1 * r2 * r3
        ob = 2 if prec == "bf16" else 4
        tc = "k_expand_tc" if prec == "bf16" else "k_expand_tf32x3"
        # per pair: the forward's and the adjoint's map chains
        out[f"{tc}<tucker core>"] = 2 * (basis_bytes(case, prec) + 8 * C * q + 8 * C * R)
        out["k_mode_last"] = 2 * (8 * C * R + 8 * C * r1 * r2 * n3)
        out["k_mode_b"] = 2 * (8 * C * r1 * r2 * n3 + 8 * C * r1 * n2 * n3)
        out["k_x1_operand"] = 2 * (8 * C * r1 * n2 * n3 + ob * C * n2 * n3 * 2 * r1)
        out[f"{tc}<tucker x1>"] = 2 * (ob * C * n2 * n3 * 2 * r1 + V)
        # the FP32 tensor-core chain (core -> x3 -> x2), each product written
        # in the next one's operand layout; twice per pair
        out["k_expand_tf32x3<tucker x3>"] = 2 * (8 * C * R + 8 * C * r1 * r2 * n3)
        # (BF16: the x2 product writes the x1 operand as BF16 rows)
        out["k_expand_tf32x3<tucker x2>"] = 2 * (8 * C * r1 * r2 * n3 + 2 * ob * C * r1 * n2 * n3)
        # the fused x1 kernels: operand in; forward: image in, DFT'd volume out;
        # adjoint: per-coil data in, image out
        pk = "bf16" if prec == "bf16" else "tf32x3"
        out[f"k_tucker_x1<{pk},fwd+dft_z>"] = ob * C * n2 * n3 * 2 * r1 + P + V
        out[f"k_tucker_x1<{pk},idft_z+adj>"] = ob * C * n2 * n3 * 2 * r1 + V + P
    else:
        per = basis_bytes(case, prec) + 8 * C * q + V + P
        for k in ("k_expand_tf32x3", "k_expand_tc", "k_expand"):
            out[k] = 2 * per
    return out


# ------------------------------------------------------------- measurement

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            d = json.load(open(path))
            return float(d.get("hbm_gbs")), float(d.get("bf16_tflops")), "measured"
        except Exception:
            pass
    return FALLBACK_HBM_GBS, FALLBACK_BF16_TFLOPS, "fallback"


def ncu_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summary, if it was taken on the kernel's current source; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path)).get(f"{workload}/{kernel}")
    if not d:
        return None
    src = os.path.join(ROOT, "paper_2008_09042_gb300", "csrc", d["source"])
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    return d["bytes_per_launch"] if sha == d.get("source_sha") else None


def reduce_max(value, device=None):
    """Max of a scalar over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, units_per_rank, slowest_ms):
    """Whole-job throughput of independent replicas: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / (slowest_ms / 1000.0)


def run_pair(mp, ctx, plan, basis, a_d, p_d, prec, y, x):
    mp.forward(ctx, plan, basis, a_d, p_d, prec, out=y)
    mp.adjoint(ctx, plan, basis, a_d, y, prec, out=x)


def time_pairs(mp, ctx, plan, basis, a_d, p_d, prec, steps, warmup, flush, stream):
    """Mean ms of one forward + adjoint pair (CUDA events, L2 flushed between pairs)."""
    import torch

    C = a_d.shape[0]
    y = torch.empty((C, plan.M), dtype=torch.complex64, device=a_d.device)
    x = torch.empty((plan.N,), dtype=torch.complex64, device=a_d.device)
    for _ in range(warmup):
        run_pair(mp, ctx, plan, basis, a_d, p_d, prec, y, x)
    torch.cuda.synchronize()
    total = 0.0
    for _ in range(steps):
        flush.zero_()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        run_pair(mp, ctx, plan, basis, a_d, p_d, prec, y, x)
        e.record(stream)
        e.synchronize()
        total += s.elapsed_time(e)
    ctx.synchronize()
    return total / steps


def kernel_profile(mp, ctx, plan, basis, a_d, p_d, prec, steps, flush):
    """Per-kernel device time over `steps` pairs, each launch bracketed by the
    library's events on its stream: {name: {ms_per_pair, launches_per_pair,
    us_per_launch}} and the family sums."""
    import torch

    C = a_d.shape[0]
    y = torch.empty((C, plan.M), dtype=torch.complex64, device=a_d.device)
    x = torch.empty((plan.N,), dtype=torch.complex64, device=a_d.device)
    ctx.profile(True)
    ctx.profile_read(reset=True)
    for _ in range(steps):
        flush.zero_()
        run_pair(mp, ctx, plan, basis, a_d, p_d, prec, y, x)
    fam, kern = ctx.profile_read(reset=True, kernels=True)
    ctx.profile(False)
    per = {k: {"ms_per_pair": v[0] / steps, "launches_per_pair": v[1] / steps, "us_per_launch": 1e3 * v[0] / v[1]}
           for k, v in kern.items() if v[1]}
    return per, {k: v[0] / steps for k, v in fam.items() if v[1]}


def roofline_entry(case, prec, per_kernel, hbm_gbs, peak_src, workload):
    """Roofline of the dominant kernel (largest share of the pair's kernel time)
    whose algorithmic bytes are tabulated; every kernel is HBM-bound here."""
    table = kernel_bytes_per_pair(case, prec)
    total = sum(v["ms_per_pair"] for v in per_kernel.values())
    ranked = sorted(per_kernel.items(), key=lambda kv: -kv[1]["ms_per_pair"])
    for name, v in ranked:
        if name not in table:
            continue
        b_launch = table[name] / v["launches_per_pair"]
        t_launch = v["us_per_launch"] * 1e-6
        achieved = b_launch / t_launch / 1e9
        return {"bound": "hbm", "achieved": achieved, "peak": hbm_gbs, "unit": "GB/s", "frac": achieved / hbm_gbs,
                "traffic": ncu_traffic(name, workload), "kernel": name,
                "peak_source": f"{peak_src} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                "algorithmic_bytes_per_launch": b_launch, "avg_launch_us": v["us_per_launch"],
                "launches_per_pair": v["launches_per_pair"],
                "share_of_kernel_time": v["ms_per_pair"] / total if total else None,
                "dominant_overall": ranked[0][0]}
    return None


# ---------------------------------------------------------------- CPU oracle

def cpu_oracle_pairs(case, budget_s=15.0, sample_coils=None, max_pairs=50):
    """Forward+adjoint pairs/s of the FP64 oracle in its fast mode (scipy.fft
    with every host core, threaded BLAS) on this host, over a bounded sample:
    whole pairs restricted to `sample_coils` coils (the per-coil work dominates;
    the value is scaled to whole pairs by sample_coils / C)."""
    from oracle import fourier, operator as op, tucker

    C = case["C"]
    cs = min(sample_coils or C, C)
    Fs = fourier.CartesianSamplingFFT(case["dims"], case["idx"])
    U = tucker.TuckerBasis(case["core"], case["fac"]) if case["tucker"] else case["U"]
    a = case["alpha"][:cs]
    p = case["p"]
    n = 0
    t0 = time.perf_counter()
    while n < max_pairs:
        y = op.forward(Fs, U, a, p)
        op.adjoint(Fs, U, a, y)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    value = n * (cs / C) / dt
    desc = (f"{n} forward+adjoint pairs of the {case['name']} workload restricted to {cs} of its {C} coils "
            f"({dt:.1f} s; value scaled by {cs}/{C}); complex128 numpy oracle, fast mode: scipy.fft with "
            f"{os.cpu_count()} workers, threaded BLAS")
    return value, desc


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def host_threads():
    try:
        from threadpoolctl import threadpool_info

        info = threadpool_info()
        return max([i.get("num_threads", 1) for i in info] + [os.cpu_count() or 1])
    except Exception:
        return os.cpu_count()


# --------------------------------------------------------- secondary lines

def slice_line(mp, ctx, dev, flush, stream, name, prec_list=("fp32", "bf16"), steps=10, warmup=3):
    """A 2D Cartesian workload: pairs/s per precision, with the roofline of its
    dominant kernel."""
    case = make_case(name)
    plan, basis, a_d, p_d = gpu_objects(mp, ctx, dev, case)
    hbm, _, src = load_peaks()
    out = {}
    for prec in prec_list:
        ms = time_pairs(mp, ctx, plan, basis, a_d, p_d, prec, steps, warmup, flush, stream)
        per, _ = kernel_profile(mp, ctx, plan, basis, a_d, p_d, prec, steps, flush)
        out[prec] = {"value": 1000.0 / ms, "unit": "pairs/s", "ms_per_pair": ms,
                     "roofline": roofline_entry(case, prec, per, hbm, src, name),
                     "kernels": {k: round(v["ms_per_pair"] * 1e3, 2) for k, v in per.items()},
                     "pair_hbm_frac": pair_algorithmic_bytes(case, prec) / (ms * 1e-3) / 1e9 / hbm}
    return out


def jacobian_line(mp, ctx, dev, flush, stream, name="cart2d_256_c16_q128", steps=10, warmup=3,
                  precs=("fp32", "bf16", "fp32_simt")):
    """Jacobian + Jacobian-adjoint pairs (the operator of every IRGN CG
    iteration) per precision, with the roofline of the adjoint's coefficient
    block dalpha = U^H v (k_uh_tc on the tensor cores; k_uh_v, the CUDA-core
    form, under fp32_simt)."""
    import torch

    case = make_case(name)
    plan, basis, a_d, p_d = gpu_objects(mp, ctx, dev, case)
    C, N, q = case["C"], case["N"], case["q"]
    hbm, _, src = load_peaks()
    g = torch.Generator().manual_seed(w.BASE_SEED + 77)
    dp = torch.randn(N, dtype=torch.complex64, generator=g).to(dev)
    da = torch.randn((C, q), dtype=torch.complex64, generator=g).to(dev)
    r = torch.empty((C, plan.M), dtype=torch.complex64, device=dev)
    gp = torch.empty((N,), dtype=torch.complex64, device=dev)
    ga = torch.empty((C, q), dtype=torch.complex64, device=dev)

    def run(prec):
        mp.jacobian(ctx, plan, basis, a_d, p_d, dp, da, prec, out=r)
        mp.jacobian_adjoint(ctx, plan, basis, a_d, p_d, r, prec, out_p=gp, out_alpha=ga)

    out = {}
    for prec in precs:
        for _ in range(warmup):
            run(prec)
        torch.cuda.synchronize()
        total = 0.0
        for _ in range(steps):
            flush.zero_()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            run(prec)
            e.record(stream)
            e.synchronize()
            total += s.elapsed_time(e)
        ms = total / steps
        ctx.profile(True)
        ctx.profile_read(reset=True)
        for _ in range(steps):
            flush.zero_()
            run(prec)
        _, kern = ctx.profile_read(reset=True, kernels=True)
        ctx.profile(False)
        per = {k: (v[0] / steps, v[1] / steps) for k, v in kern.items() if v[1]}
        uh = {"fp32": "k_uh_tc<tf32x3>", "bf16": "k_uh_tc<bf16>", "fp32_simt": "k_uh_v"}[prec]
        entry = {"value": 1000.0 / ms, "unit": "Jacobian + adjoint pairs/s", "ms_per_pair": ms,
                 "kernels": {k: round(v[0] * 1e3, 2) for k, v in per.items()}}
        if uh in per and not case["tucker"]:
            # algorithmic bytes: the basis (FP32 view 8 N q, BF16 view 4 N q) and v (8 C N) once
            ub = (4 if prec == "bf16" else 8) * N * q
            b = ub + 8 * C * N
            t = per[uh][0] * 1e-3 / per[uh][1]
            entry["uh_roofline"] = {"bound": "hbm", "kernel": uh, "achieved": b / t / 1e9, "peak": hbm,
                                    "unit": "GB/s", "frac": b / t / 1e9 / hbm, "algorithmic_bytes_per_launch": b,
                                    "avg_launch_us": t * 1e6, "launches_per_pair": per[uh][1],
                                    "peak_source": f"{src} HBM copy bandwidth"}
        out[prec] = entry
    return out


def multimap_line(mp, ctx, dev, flush, stream, name="cart2d_256_c16_q128", M=2, steps=10, warmup=3):
    """The forward model with M sets of maps (extra bilinear terms) on a 2D
    workload: forward + adjoint (in the M images) pairs per second."""
    import torch

    case = make_case(name)
    plan, basis, a_d, p_d = gpu_objects(mp, ctx, dev, case)
    C, N, q = case["C"], case["N"], case["q"]
    g = torch.Generator().manual_seed(w.BASE_SEED + 91)
    A = torch.stack([a_d] + [0.3 * torch.randn((C, q), dtype=torch.complex64, generator=g).to(dev)
                             for _ in range(M - 1)]).contiguous()
    P = torch.stack([p_d] + [torch.randn(N, dtype=torch.complex64, generator=g).to(dev) for _ in range(M - 1)])
    P = P.contiguous()
    y = torch.empty((C, plan.M), dtype=torch.complex64, device=dev)
    x = torch.empty((M, N), dtype=torch.complex64, device=dev)
    out = {"sets": M}
    for prec in ("fp32", "bf16"):
        def run():
            mp.forward_maps(ctx, plan, basis, A, P, prec, out=y)
            mp.adjoint_maps(ctx, plan, basis, A, y, prec, out=x)
        for _ in range(warmup):
            run()
        torch.cuda.synchronize()
        total = 0.0
        for _ in range(steps):
            flush.zero_()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            run()
            e.record(stream)
            e.synchronize()
            total += s.elapsed_time(e)
        ms = total / steps
        out[prec] = {"value": 1000.0 / ms, "unit": "pairs/s", "ms_per_pair": ms}
    return out


def maxwell_basis_line(mp, ctx, n=256, q=128, n_sites=64, L=500, reps=3):
    """The Maxwell basis of an n x n slice built on the GPU (64 dipole sites x 6
    dipoles, Fig. 1's 500 excitations): wall time per build (it synchronises),
    its agreement with the FP64 oracle (singular values; subspace of the q
    leading vectors), and the oracle's own time on this host."""
    import torch

    src = w.circle_sites(n_sites, 1.5 * 0.5 * np.hypot(0.22, 0.22))
    om = w.random_excitations(6 * n_sites, L, seed=w.BASE_SEED)
    mp.maxwell_basis_2d(ctx, (n, n), q, src, om)  # warm-up (module load, first allocations)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        U, sv = mp.maxwell_basis_2d(ctx, (n, n), q, src, om)
        times.append(time.perf_counter() - t0)
    from oracle import basis as ob  # the CPU baseline of this line

    t0 = time.perf_counter()
    ref = ob.build_maxwell_basis_2d(n, n, q, n_sites=n_sites, omega=om)
    t_cpu = time.perf_counter() - t0
    Uo = np.linalg.qr(U.cpu().numpy().astype(np.complex128).T)[0]
    sin_theta = float(np.linalg.norm(Uo - ref.U @ (ref.U.conj().T @ Uo), 2))
    nsv = sv.size
    return {"shape": [n, n], "q": q, "dipoles": 6 * n_sites, "excitations": L,
            "value": float(np.median(times)), "unit": "s per basis build (GPU, FP64)",
            "cpu_baseline": {"kind": "oracle", "value": t_cpu, "unit": "s per basis build", "cores": host_threads(),
                             "sample": "one whole build: complex128 numpy, LAPACK SVD of B Omega"},
            "vs_oracle": {"sv_max_abs_err_over_sigma1": float(np.max(np.abs(sv - ref.sv[:nsv])) / ref.sv[0]),
                          "subspace_sin_theta": sin_theta, "sigma_q_over_sigma1": float(ref.sv[q - 1] / ref.sv[0])}}


def dynamic_line(mp, ctx, dev, n=256, C=16, q=128, T=8, R=4, n_outer=50, n_cg=5, n_tv=10, reps=3):
    """Dynamic MPI-L on a movie of T frames of an n x n slice (each frame its own
    variable-density line pattern, shared maps, TV over (t, y, x)): time per
    movie through mpi_image_solve_dynamic (solver graph replayed)."""
    import torch

    base = w.BASE_SEED + 300
    B = mp.Basis(ctx, w.smooth_orthonormal_basis(n, n, q, seed=base).T)
    a = torch.from_numpy(w.random_coefficients(C, q, seed=base + 1).astype(np.complex64)).to(dev)
    plans = [mp.Plan(ctx, (n, n), sample_idx=w.mask_to_indices(w.vd_lines_mask(n, n, R, 16, seed=base + 10 + t)))
             for t in range(T)]
    M = plans[0].M
    g = torch.Generator().manual_seed(base + 2)
    y = (torch.randn((T, C, M), dtype=torch.complex64, generator=g) * 0.01).to(dev)
    eps = np.full((T, C), 0.01 * np.sqrt(M))
    out = {"frames": T, "shape": [n, n], "C": C, "q": q, "iterations": f"{n_outer} ADMM x {n_cg} CG x {n_tv} TV"}
    for prec in ("fp32", "bf16"):
        mp.image_solve_dynamic(ctx, plans, B, a, y, eps, n_outer=n_outer, n_cg=n_cg, n_tv=n_tv, prec=prec)  # records
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            mp.image_solve_dynamic(ctx, plans, B, a, y, eps, n_outer=n_outer, n_cg=n_cg, n_tv=n_tv, prec=prec)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) / reps * 1e3
        out[prec] = {"ms_per_movie": ms, "ms_per_frame": ms / T}
    return out


def table_s1_line(mp, ctx, shape=(192, 192, 170), cases=((75, 16, 96), (200, 40, 256)), eps=1e-4, reps=10):
    """Supporting Table S1's setting: a 192 x 192 x 170 volume, a Maxwell basis of q
    columns built on the GPU (dipole sites on a sphere; 6 D dipoles, L
    excitations), compressed on the GPU to eps = 1e-4; its ranks, memory, the
    error of the compressed basis, and the matrix-vector product U alpha (one
    coil) with the Tucker and the dense basis.  The paper's numbers (V100,
    MARIE basis) are context: the source model differs."""
    import torch

    out = {"shape": list(shape), "eps": eps}
    fov = (0.22, 0.22, 0.22 * shape[2] / shape[0])
    for q, D, L in cases:
        src = w.sphere_sites(D, 1.5 * 0.5 * np.sqrt(np.sum(np.square(fov))))
        om = w.random_excitations(6 * D, L, seed=w.BASE_SEED + q)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        U, sv = mp.maxwell_basis_3d(ctx, shape, q, src, om, fov=fov)
        torch.cuda.synchronize()
        t_basis = time.perf_counter() - t0
        t0 = time.perf_counter()
        B = mp.tucker_compress(ctx, U, shape, eps)
        torch.cuda.synchronize()
        t_comp = time.perf_counter() - t0
        r = B.ranks
        ram = (q * r[0] * r[1] * r[2] + sum(n * rk for n, rk in zip(shape, r))) * 8 / 1e6
        err2 = tot2 = 0.0
        for c0 in range(0, q, 25):
            c1 = min(q, c0 + 25)
            eye = torch.zeros((c1 - c0, q), dtype=torch.complex64, device=U.device)
            eye[torch.arange(c1 - c0), torch.arange(c0, c1)] = 1
            S = mp.basis_expand(ctx, B, eye)
            err2 += float(torch.sum(torch.abs(S - U[c0:c1]) ** 2))
            tot2 += float(torch.sum(torch.abs(U[c0:c1]) ** 2))
        Bd = mp.Basis(ctx, U)
        a = torch.randn((1, q), dtype=torch.complex64, device=U.device)
        mvp = {}
        for name, basis in (("tucker", B), ("dense", Bd)):
            for prec in ("fp32", "bf16"):
                for _ in range(3):
                    mp.basis_expand(ctx, basis, a, prec=prec)
                torch.cuda.synchronize()
                s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s_.record()
                for _ in range(reps):
                    mp.basis_expand(ctx, basis, a, prec=prec)
                e_.record()
                e_.synchronize()
                mvp[f"{name}_{prec}_ms"] = s_.elapsed_time(e_) / reps
        out[f"q{q}"] = {"dipoles": 6 * D, "excitations": L, "basis_build_s": t_basis, "compress_s": t_comp,
                        "ranks": list(r), "tucker_MB": ram, "dense_MB": 8 * q * int(np.prod(shape)) / 1e6,
                        "bound": B.bound, "error": float(np.sqrt(err2 / tot2)), "mvp": mvp}
        del Bd, B, U
        torch.cuda.empty_cache()
    return out


def radial_line(mp, ctx, dev, flush, stream, steps=10, warmup=3):
    """radial 256^2, 12 coils, q = 96, 64 golden-angle spokes x 512 samples, KB W = 6, sigma = 2."""
    import torch

    base = w.BASE_SEED
    cfg = w.workload("radial2d_256_c12_q96")
    n = cfg["dims"][0]
    k = w.golden_angle_radial(cfg["spokes"], cfg["readout"]).astype(np.float32)
    plan = mp.Plan(ctx, (n, n), traj=k, kb_width=cfg["W"], oversamp=cfg["sigma"])
    B = mp.Basis(ctx, w.smooth_orthonormal_basis(n, n, cfg["q"], seed=base).T)
    a = torch.from_numpy(w.random_coefficients(cfg["C"], cfg["q"], seed=base + 1).astype(np.complex64)).to(dev)
    p = torch.from_numpy(w.random_ellipses(n, n, seed=base + 2).ravel().astype(np.complex64)).to(dev)
    out = {}
    for prec in ("fp32", "bf16"):
        ms = time_pairs(mp, ctx, plan, B, a, p, prec, steps, warmup, flush, stream)
        per, _ = kernel_profile(mp, ctx, plan, B, a, p, prec, steps, flush)
        out[prec] = {"value": 1000.0 / ms, "unit": "pairs/s", "ms_per_pair": ms,
                     "kernels": {k: round(v["ms_per_pair"] * 1e3, 2) for k, v in per.items()}}
    return out


def batched_slices(mp, ctx, dev, flush, stream, steps=5, warmup=2):
    """The 64-slice mixed exam: grids from {128, 192, 256, 320}^2, coils from
    {8, 16, 32}, q by grid size, Poisson-disc R in 4..8; all slices' forward +
    adjoint replayed as one CUDA graph.  Slice pairs/s per precision, and the
    exam's algorithmic bytes over its time against HBM peak."""
    import torch

    cfg = w.workload("batched2d_64slices")
    rng = np.random.default_rng(w.BASE_SEED)
    sizes = rng.choice(cfg["sizes"], size=cfg["slices"])
    coils = rng.choice(cfg["coils"], size=cfg["slices"])
    Rs = rng.integers(cfg["R_range"][0], cfg["R_range"][1] + 1, size=cfg["slices"])
    bases, masks = {}, {}
    slices = []
    exam_bytes = {"fp32": 0, "bf16": 0}
    for i in range(cfg["slices"]):
        n, C, R = int(sizes[i]), int(coils[i]), int(Rs[i])
        q = cfg["q_by_size"][n]
        if n not in bases:
            bases[n] = mp.Basis(ctx, w.smooth_orthonormal_basis(n, n, q, seed=w.BASE_SEED + n).T)
        if (n, R) not in masks:  # one mask per (grid, R), shared by the slices that draw it
            masks[(n, R)] = mp.Plan(ctx, (n, n), sample_idx=w.mask_to_indices(
                w.poisson_disc_mask(n, n, R, calib=(24, 24), seed=w.BASE_SEED + 10 * n + R)))
        plan = masks[(n, R)]
        a = torch.from_numpy(w.random_coefficients(C, q, seed=w.BASE_SEED + 100 + i).astype(np.complex64)).to(dev)
        p = torch.from_numpy(w.random_ellipses(n, n, seed=w.BASE_SEED + 200 + i).ravel().astype(np.complex64)).to(dev)
        slices.append(dict(plan=plan, basis=bases[n], alpha=a, p=p,
                           y=torch.empty((C, plan.M), dtype=torch.complex64, device=dev),
                           x=torch.empty((n * n,), dtype=torch.complex64, device=dev)))
        for prec in exam_bytes:
            ub = 4 if prec == "bf16" else 8
            exam_bytes[prec] += 2 * (n * n * q * ub + 8 * C * n * n + 8 * C * plan.M + 8 * n * n + 8 * C * q)
    hbm, _, src = load_peaks()
    out = {"slices": cfg["slices"], "coils_total": int(coils.sum()),
           "grid_counts": {int(k): int((sizes == k).sum()) for k in cfg["sizes"]}}
    _, bf16_peak, _ = load_peaks()
    for prec in ("fp32", "bf16"):
        n_rec = len(ctx.tuning_records())
        batch = mp.Batch(ctx, slices, kind="pair", prec=prec)
        # the grouped expansions' timings from the batch's tuning records
        grouped = []
        for rec in ctx.tuning_records()[n_rec:]:
            m = re.match(r"grouped expansion \((\d+) slices, N=(\d+), q=(\d+), sumC=(\d+), (\w+)\):.* chose (\d+) "
                         r"\(([\d.]+) us\)", rec)
            if not m:
                continue
            ns, N, q, sumC, pr, ctas, us = m.groups()
            N, q, sumC, us = int(N), int(q), int(sumC), float(us)
            flops = 2.0 * N * (2 * q) * (2 * sumC)  # the real-ified GEMM, counted once
            ub = (2 if prec == "bf16" else 4) * N * 2 * q
            byts = ub + 8 * sumC * N + 8 * sumC * q + 8 * int(ns) * N  # basis, per-coil images out, alpha, images in
            grouped.append({"slices": int(ns), "N": N, "q": q, "coils": sumC, "ctas_per_row": int(ctas),
                            "us_per_launch": us, "tflops": flops / (us * 1e-6) / 1e12,
                            "frac_of_bf16_tensor_peak": flops / (us * 1e-6) / 1e12 / bf16_peak,
                            "hbm_gbs": byts / (us * 1e-6) / 1e9, "frac_of_hbm_peak": byts / (us * 1e-6) / 1e9 / hbm})
        for _ in range(warmup):
            batch.run()
        torch.cuda.synchronize()
        total = 0.0
        for _ in range(steps):
            flush.zero_()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            batch.run()
            e.record(stream)
            e.synchronize()
            total += s.elapsed_time(e)
        ctx.synchronize()
        ms = total / steps
        achieved = exam_bytes[prec] / (ms * 1e-3) / 1e9
        out[prec] = {"value": cfg["slices"] * 1000.0 / ms, "unit": "slice pairs/s", "ms_per_exam": ms,
                     "graph_kernels": batch.kernels(), "grouped_launches_per_direction": batch.groups(),
                     "grouped_expansion": grouped,
                     "roofline": {"bound": "hbm", "kernel": "whole exam (every kernel of the replayed graph)",
                                  "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                                  "algorithmic_bytes_per_exam": exam_bytes[prec], "traffic": None,
                                  "peak_source": f"{src} HBM copy bandwidth"}}
        batch.close()
    return out


def recon_per_slice(mp, ctx, dev, names=("cart2d_64_c4_q32", "cart2d_256_c16_q128", "cart2d_320_c16_q100",
                                         "radial2d_256_c12_q96"),
                    precs=("fp32", "bf16", "mixed"), reps=2):
    """MPI-BL (20 IRGN x 10 CG) + MPI-L (50 ADMM x 5 CG x 10 TV) wall time per
    slice for each precision, on data and against reconstructions the FP64
    oracle made (tests/golden/recon_<workload>.npz, written by
    tests/golden/make_recon_golden.py): NRMSE of the coil images s_k (.) p
    (MPI-BL) and of the image (MPI-L) against the oracle's."""
    import torch

    out = {"iterations": "20 IRGN x 10 CG + 50 ADMM x 5 CG x 10 TV",
           "reference": "FP64 oracle reconstruction of the same data (stored fixture)"}
    for name in names:
        path = os.path.join(ROOT, "tests", "golden", f"recon_{name}.npz")
        if not os.path.exists(path):
            out[name] = {"unavailable": f"{os.path.relpath(path, ROOT)} missing"}
            continue
        g = np.load(path)
        cfg, U, samp, _, _ = w.recon_case(name)
        ny, nx = cfg["dims"]
        C = cfg["C"]
        if cfg["kind"] == "radial":
            plan = mp.Plan(ctx, (ny, nx), traj=samp, kb_width=cfg["W"], oversamp=cfg["sigma"])
        else:
            plan = mp.Plan(ctx, (ny, nx), sample_idx=samp)
        B = mp.Basis(ctx, U.T)
        y = torch.from_numpy(np.ascontiguousarray(g["y"])).to(dev)
        eps = g["eps"]
        ref_ci = (g["alpha_bl"].astype(np.complex128) @ U.T) * g["p_bl"].astype(np.complex128)[None]
        ref_p = g["p_l"].astype(np.complex128)
        res = {}
        for prec in precs:
            times = []
            for _ in range(reps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                a, p, _ = mp.sm_estimate(ctx, plan, B, y, C, n_outer=cfg["n_irgn"], n_cg=10, prec=prec)
                img, _ = mp.image_solve(ctx, plan, B, a, y, eps, n_outer=cfg["n_admm"], n_cg=5, n_tv=10, prec=prec)
                torch.cuda.synchronize()
                times.append(time.perf_counter() - t0)
            ci = (a.cpu().numpy().astype(np.complex128) @ U.T) * p.cpu().numpy().astype(np.complex128)[None]
            x = img.cpu().numpy().astype(np.complex128)
            res[prec] = {"ms_per_slice": 1000.0 * min(times),
                         "nrmse_coil_images_vs_oracle": float(np.linalg.norm(ci - ref_ci) / np.linalg.norm(ref_ci)),
                         "nrmse_image_vs_oracle": float(np.linalg.norm(x - ref_p) / np.linalg.norm(ref_p))}
        out[name] = {"dims": list(cfg["dims"]), "C": C, "q": cfg["q"], "M": int(plan.M), **res}
        del plan, B
    return out


# --------------------------------------------------------------------- arms

def run_reference(args):
    """The oracle (this build's reference arm: the paper ships no code) timed on
    the host cores in its fast mode; each step one forward+adjoint pair of the
    workload restricted to a few coils, the value scaled to whole pairs."""
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    case = make_case(args.workload)
    from oracle import fourier, operator as op, tucker

    C = case["C"]
    cs = min(4, C)
    Fs = fourier.CartesianSamplingFFT(case["dims"], case["idx"])
    U = tucker.TuckerBasis(case["core"], case["fac"]) if case["tucker"] else case["U"]
    a, p = case["alpha"][:cs], case["p"]
    for _ in range(args.warmup):
        op.adjoint(Fs, U, a, op.forward(Fs, U, a, p))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        op.adjoint(Fs, U, a, op.forward(Fs, U, a, p))
    dt = time.perf_counter() - t0
    value = args.steps * (cs / C) / dt
    sample = (f"each step one forward+adjoint pair of the {case['name']} workload restricted to {cs} of its {C} "
              f"coils (value scaled by {cs}/{C}); complex128 numpy oracle, fast mode: scipy.fft with "
              f"{os.cpu_count()} workers, threaded BLAS")
    line = {
        "impl": "reference", "metric": "MPI forward+adjoint operator pairs per second",
        "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": case["name"], "N": case["N"], "C": C, "q": case["q"], "M": case["M"]},
        "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": host_threads(), "kind": "oracle",
                         "cpu": cpu_model(), "sample": sample},
        "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    import paper_2008_09042_gb300 as mp

    case = make_case(args.workload, seed_offset=rank)
    C, q, N, M = case["C"], case["q"], case["N"], case["M"]
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    ctx = mp.Context(local_rank, stream=stream)
    plan, basis, a_d, p_d = gpu_objects(mp, ctx, dev, case)
    y_d = torch.empty((C, M), dtype=torch.complex64, device=dev)
    x_d = torch.empty((N,), dtype=torch.complex64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step():
        run_pair(mp, ctx, plan, basis, a_d, p_d, args.prec, y_d, x_d)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(local_rank)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = ctx.launches()
    for k in range(args.steps):
        flush.zero_()
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = ctx.launches() - launches0
    total_ms = reduce_max(sum(s.elapsed_time(e) for s, e in evs), dev)
    value = replica_throughput(world, args.steps, total_ms)
    # Per-launch kernel durations: the same K steps again, each launch bracketed by
    # the library's own events on its stream.  A separate region, because the
    # extra event records between launches slow the step they sit in.
    per_kernel, families = kernel_profile(mp, ctx, plan, basis, a_d, p_d, args.prec, args.steps, flush)
    clk = clocks.stop()

    # ---- end to end through the C ABI's host-buffer calls (mpi_forward_host,
    # mpi_adjoint_host): pinned host inputs in, host outputs back, each call
    # returning once its result is in host memory.  Host wall clock per step.
    a_h = torch.from_numpy(case["alpha"].astype(np.complex64)).pin_memory()
    p_h = torch.from_numpy(case["p"].astype(np.complex64)).pin_memory()
    y_h = torch.empty((C, M), dtype=torch.complex64).pin_memory()
    x_h = torch.empty((N,), dtype=torch.complex64).pin_memory()

    def e2e_step():
        mp.forward_host(ctx, plan, basis, a_h, p_h, args.prec, out=y_h)
        mp.adjoint_host(ctx, plan, basis, a_h, y_h, args.prec, out=x_h)

    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    e2e_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        e2e_ms += (time.perf_counter() - t0) * 1e3
    e2e_ms = reduce_max(e2e_ms, dev)
    e2e_value = replica_throughput(world, args.steps, e2e_ms)
    h2d = (2 * C * q + N + C * M) * 8  # alpha for each call, p, y
    d2h = (C * M + N) * 8

    hbm_gbs, bf16_tflops, peak_src = load_peaks()
    roof = roofline_entry(case, args.prec, per_kernel, hbm_gbs, peak_src, case["name"])
    pair_bytes = pair_algorithmic_bytes(case, args.prec)
    ms_pair = total_ms / args.steps
    if case["tucker"]:
        basis_desc = (f"smooth orthonormal stand-in of the Maxwell basis shape, Tucker-factored: core "
                      f"{case['ranks']} x q={q}, factors {case['dims'][0]}x{case['ranks'][0]}, "
                      f"{case['dims'][1]}x{case['ranks'][1]}, {case['dims'][2]}x{case['ranks'][2]} (complex64)")
    else:
        basis_desc = "smooth orthonormal stand-in of the Maxwell basis shape (complex64 [q][N])"
    line = {
        "metric": "MPI forward+adjoint operator pairs per second",
        "value": value, "unit": "pairs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_pair, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16+f32" if args.prec == "bf16" else "f32",
        "data": "synthetic",
        "config": {"workload": case["name"], "dims": list(case["dims"]), "N": N, "C": C, "q": q, "M": M,
                   "mask": case["mask_desc"], "basis": basis_desc, "expansion_precision": args.prec,
                   "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"replicas x{world}"},
        "e2e": {"value": e2e_value, "unit": "pairs/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": roof,
        "pair_roofline": {"bound": "hbm", "algorithmic_bytes_per_pair": pair_bytes,
                          "achieved": pair_bytes / (ms_pair * 1e-3) / 1e9, "peak": hbm_gbs, "unit": "GB/s",
                          "frac": pair_bytes / (ms_pair * 1e-3) / 1e9 / hbm_gbs},
        "kernel_us_per_pair": {k: round(v["ms_per_pair"] * 1e3, 1) for k, v in
                               sorted(per_kernel.items(), key=lambda kv: -kv[1]["ms_per_pair"])},
        "clocks": clk,
        "autotune": ctx.tuning_records(),
    }
    if not args.no_secondary:
        wl = {}
        others = {HEADLINE, "cart2d_256_c16_q128"} - {case["name"]}
        for other in sorted(others):
            wl[other] = slice_line(mp, ctx, dev, flush, stream, other) if other != HEADLINE else None
        if case["name"] == HEADLINE:
            for prec in ("bf16",):
                ms = time_pairs(mp, ctx, plan, basis, a_d, p_d, prec, max(3, args.steps // 2), 2, flush, stream)
                wl[f"{case['name']}/{prec}"] = {"value": 1000.0 / ms, "unit": "pairs/s", "ms_per_pair": ms}
        wl = {k: v for k, v in wl.items() if v is not None}
        wl["radial2d_256_c12_q96"] = radial_line(mp, ctx, dev, flush, stream)
        wl["cart2d_256_c16_q128/jacobian"] = jacobian_line(mp, ctx, dev, flush, stream)
        wl[f"{HEADLINE}/jacobian"] = jacobian_line(mp, ctx, dev, flush, stream, name=HEADLINE,
                                                   precs=("fp32", "bf16"), steps=5)
        wl["maxwell_basis_2d_256_q128"] = maxwell_basis_line(mp, ctx)
        wl["cart2d_256_c16_q128/two_sets_of_maps"] = multimap_line(mp, ctx, dev, flush, stream)
        wl["dynamic_mpi_l_256_c16_q128_t8"] = dynamic_line(mp, ctx, dev)
        try:
            wl["table_s1_192x192x170"] = table_s1_line(mp, ctx)
        except Exception as exc:  # reported, not fatal to the headline
            wl["table_s1_192x192x170"] = {"error": str(exc)}
        wl["batched2d_64slices"] = batched_slices(mp, ctx, dev, flush, stream)
        line["workloads"] = wl
        line["recon"] = recon_per_slice(mp, ctx, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, desc = cpu_oracle_pairs(case, sample_coils=4 if case["tucker"] else None)
        line["cpu_baseline"] = {"value": v, "unit": "pairs/s", "cores": host_threads(), "kind": "oracle",
                                "cpu": cpu_model(), "sample": desc}
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def profile_workload(args):
    """Forward+adjoint pairs of one workload, nothing timed: the command an
    external profiler (ncu) wraps to capture that workload's kernels."""
    import torch
    import paper_2008_09042_gb300 as mp

    dev = torch.device("cuda", 0)
    ctx = mp.Context(0)
    base = w.BASE_SEED
    name = args.profile_workload
    if name.startswith("radial2d"):
        cfg = w.workload(name)
        n = cfg["dims"][0]
        k = w.golden_angle_radial(cfg["spokes"], cfg["readout"]).astype(np.float32)
        plan = mp.Plan(ctx, (n, n), traj=k, kb_width=cfg["W"], oversamp=cfg["sigma"])
        B = mp.Basis(ctx, w.smooth_orthonormal_basis(n, n, cfg["q"], seed=base).T)
        a = torch.from_numpy(w.random_coefficients(cfg["C"], cfg["q"], seed=base + 2).astype(np.complex64)).to(dev)
        pd = torch.from_numpy(w.random_ellipses(n, n, seed=base + 2).ravel().astype(np.complex64)).to(dev)
        ctx.reserve(plan, B, cfg["C"])
    else:
        case = make_case(name)
        plan, B, a, pd = gpu_objects(mp, ctx, dev, case)
    if args.profile_coils > 0:
        a = a[: args.profile_coils].contiguous()
    if args.profile_op == "jacobian":
        da = (0.5 * a).contiguous()
        dp = (0.25 * pd).contiguous()
        for _ in range(args.steps):
            dy = mp.jacobian(ctx, plan, B, a, pd, dp, da, args.prec)
            mp.jacobian_adjoint(ctx, plan, B, a, pd, dy, args.prec)
    else:
        for _ in range(args.steps):
            y = mp.forward(ctx, plan, B, a, pd, args.prec)
            mp.adjoint(ctx, plan, B, a, y, args.prec)
    ctx.synchronize()
    what = "Jacobian + Jacobian-adjoint" if args.profile_op == "jacobian" else "forward+adjoint"
    print(f"{name}: {args.steps} {what} pairs ({args.prec})", flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_workload:
        return profile_workload(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
