// C ABI entry points: argument checks, workspace, and the order of kernel
// passes for each operator (Theory section, Eqs. 1, 5, 7 and the
// Jacobian-adjoint display after Eq. 7).
#include <math.h>
#include <string.h>

#include <cuda.h>

#include <algorithm>
#include <string>
#include <vector>

#include "mpi_internal.h"

// ------------------------------------------------------------------ helpers

mpi_status set_err(mpi_ctx* ctx, mpi_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}

mpi_status cuda_check(mpi_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return MPI_OK;
  return set_err(ctx, MPI_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool fft_length_supported(int n) {
  for (int i = 0; i < kNumFftLengths; ++i)
    if (kFftLengths[i] == n) return true;
  return false;
}

void ctx_adopt(mpi_ctx* ctx, mpi_ctx** slot) { ctx->children.push_back(slot); }

void ctx_release(mpi_ctx** slot) {
  mpi_ctx* ctx = *slot;
  if (!ctx) return;
  auto& v = ctx->children;
  v.erase(std::remove(v.begin(), v.end(), slot), v.end());
  *slot = nullptr;
}

const float2* twiddle_table(const mpi_ctx* ctx, int n) {
  for (int i = 0; i < kNumFftLengths; ++i)
    if (kFftLengths[i] == n) return ctx->twiddles + ctx->tw_offset[i];
  return nullptr;
}

mpi_status ensure_work(mpi_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->work_bytes) return MPI_OK;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_check(ctx, e, "workspace sync");
  if (ctx->work) cudaFree(ctx->work);
  ctx->work = nullptr;
  ctx->work_bytes = 0;
  ctx->tune_scratch = nullptr;
  ctx->tune_scratch_bytes = 0;
  const size_t want = std::max(bytes, (size_t)1 << 20);
  e = cudaMalloc(&ctx->work, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, MPI_ERR_OOM, "workspace allocation failed");
  }
  ctx->work_bytes = want;
  return MPI_OK;
}

void prof_begin(mpi_ctx* ctx, int family) {
  if (!ctx->profiling || ctx->ev_used >= (int)ctx->ev_begin.size()) return;
  cudaEventRecord(ctx->ev_begin[ctx->ev_used], ctx->stream);
  ctx->pending_family = family;
}

void prof_end(mpi_ctx* ctx, const char* name) {
  if (!ctx->profiling || ctx->pending_family < 0 || ctx->ev_used >= (int)ctx->ev_begin.size()) return;
  cudaEventRecord(ctx->ev_end[ctx->ev_used], ctx->stream);
  ctx->ev_family[ctx->ev_used] = ctx->pending_family;
  ctx->ev_name[ctx->ev_used] = name;
  ctx->ev_used++;
  ctx->pending_family = -1;
}

namespace {

constexpr int kProfileSlots = 16384;

struct DeviceGuard {
  explicit DeviceGuard(int dev) { cudaSetDevice(dev); }
};

bool bad_ptr(const void* p) { return p == nullptr; }

size_t partial_elems(const mpi_ctx* ctx, const mpi_basis* basis, int C) {
  if (!basis) return 0;
  const mpi_basis* b = basis->tucker ? basis->core : basis;
  return std::max(uh_v_partial_elems(ctx, b->N, b->q, C), uh_tc_partial_elems(ctx, b->N, b->q, C));
}

size_t op_work_bytes(const mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis, int C) {
  const size_t cn = (size_t)C * plan->N;
  size_t grid = 0;
  if (plan->kind == MPI_TRAJ_RADIAL) grid = nufft_grid_elems(plan, C);
  size_t partial = partial_elems(ctx, basis, C);
  size_t tucker = (basis && basis->tucker) ? 2 * cn + tucker_work_elems(basis, C) : 0;
  return (2 * cn + grid + partial + tucker) * sizeof(float2) + 4096;
}

mpi_status check_op(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis, int C,
                    mpi_precision prec) {
  if (!ctx) return MPI_ERR_ARG;
  if (!plan || !basis) return set_err(ctx, MPI_ERR_ARG, "null plan or basis");
  if (plan->ctx != ctx || basis->ctx != ctx) return set_err(ctx, MPI_ERR_ARG, "plan/basis from another context");
  if (C < 1) return set_err(ctx, MPI_ERR_ARG, "C must be >= 1");
  if (basis->N != plan->N) return set_err(ctx, MPI_ERR_SHAPE, "basis N differs from plan N");
  if (prec != MPI_PREC_FP32 && prec != MPI_PREC_BF16 && prec != MPI_PREC_FP32_SIMT)
    return set_err(ctx, MPI_ERR_ARG, "bad precision");
  const mpi_basis* eb = basis->tucker ? basis->core : basis;
  if (prec == MPI_PREC_BF16 && !eb->Ubf)
    return set_err(ctx, MPI_ERR_UNSUPPORTED, "BF16 expansion unavailable: " + eb->bf16_err);
  return MPI_OK;
}

}  // namespace

extern "C" int mpi_expand_path(const mpi_basis* basis, int C, int jacobian, mpi_precision prec) {
  if (!basis || C < 1) return -1;
  const mpi_basis* eb = basis->tucker ? basis->core : basis;
  const int mode = jacobian ? EX_JFWD : EX_FWD;
  switch (prec) {
    case MPI_PREC_BF16:
      return MPI_EXPAND_BF16;
    case MPI_PREC_FP32:
      return tf32_group(eb, mode, C) > 0 ? MPI_EXPAND_TF32X3 : MPI_EXPAND_FFMA;
    case MPI_PREC_FP32_SIMT:
      return MPI_EXPAND_FFMA;
    default:
      return -1;
  }
}

// FP32: the 3xTF32 tensor-core kernel where the shape fits its shared-memory
// budget, else the CUDA-core FFMA kernel.  BF16: the BF16 tensor-core kernel.
// FP32_SIMT: the FFMA kernel.
mpi_status expand(mpi_ctx* ctx, const mpi_basis* basis, int mode, const ExpandArgs& a, mpi_precision prec) {
  if (prec == MPI_PREC_BF16) return launch_expand_tc(ctx, basis, mode, a);
  if (prec == MPI_PREC_FP32) {
    const int g = tf32_group(basis, mode, a.C);
    if (g == a.C) return launch_expand_tf32(ctx, basis, mode, a);
    // coil groups in one launch: each grid row takes its slice of alpha (dalpha)
    // and of the per-coil output
    if (g > 0) return launch_expand_tf32(ctx, basis, mode, a, g);
  }
  if (a.kname && strncmp(a.kname, "k_expand_t", 10) == 0) {  // a tensor-core label: profile under the FFMA name
    ExpandArgs f = a;
    f.kname = "k_expand";
    return launch_expand(ctx, mode, f);
  }
  return launch_expand(ctx, mode, a);
}

mpi_status uh_v(mpi_ctx* ctx, const mpi_basis* b, const float2* V, int C, float2* dalpha, float2* partials,
                size_t partial_cap, mpi_precision prec) {
  if (prec != MPI_PREC_FP32_SIMT && uh_tc_supported(b, prec))
    return launch_uh_tc(ctx, b, V, C, dalpha, partials, partial_cap, prec);
  return launch_uh_v(ctx, b->U, b->N, b->q, V, C, dalpha, partials, partial_cap);
}

namespace {

ExpandArgs base_args(const mpi_plan* plan, const mpi_basis* basis, int C) {
  ExpandArgs a;
  a.U = basis->U;
  a.N = basis->N;
  a.q = basis->q;
  a.nx = plan->nx;
  a.ny = plan->ny;
  a.C = C;
  if (plan->kind == MPI_TRAJ_CARTESIAN) {
    a.centre = 1;
    a.scale = 1.0f / sqrtf((float)plan->N);
  } else {
    a.centre = 0;  // the NUFFT passes handle centring and scale themselves
    a.scale = 1.0f;
  }
  return a;
}

// k-space -> image-side grid (inverse FFT passes) into `w` [C][N].
mpi_status kspace_to_image(mpi_ctx* ctx, const mpi_plan* plan, const float2* y, int C, float2* w,
                           float2* grid) {
  if (plan->kind == MPI_TRAJ_RADIAL) return nufft_adjoint(ctx, plan, y, C, w, grid);
  if (ctx->plane_pass && plane_pass_supported(plan)) {  // 3D: the passes along x and y per plane, then z
    mpi_status st = launch_plane_yx(ctx, plan, w, C, (float2*)y, true);
    return st ? st : launch_fft_z(ctx, w, C, plan->nz, plan->ny, plan->nx, true);
  }
  mpi_status st = launch_rows_scatter_inv(ctx, plan, y, C, w);
  if (st) return st;
  st = launch_fft_cols(ctx, w, C, plan->nz, plan->ny, plan->nx, true, plan->row_has);
  if (st) return st;
  if (plan->ndim == 3) st = launch_fft_z(ctx, w, C, plan->nz, plan->ny, plan->nx, true);
  return st;
}

// image-side grid `v` [C][N] (already multiplied by sign and scale) -> k-space y.
mpi_status image_to_kspace(mpi_ctx* ctx, const mpi_plan* plan, float2* v, int C, float2* y,
                           float2* grid) {
  if (plan->kind == MPI_TRAJ_RADIAL) return nufft_forward(ctx, plan, v, C, y, grid);
  mpi_status st = MPI_OK;
  if (plan->ndim == 3) st = launch_fft_z(ctx, v, C, plan->nz, plan->ny, plan->nx, false);
  if (st) return st;
  if (ctx->plane_pass && plane_pass_supported(plan)) return launch_plane_yx(ctx, plan, v, C, y, false);
  st = launch_fft_cols(ctx, v, C, plan->nz, plan->ny, plan->nx, false, plan->row_has);
  if (st) return st;
  return launch_rows_fwd_gather(ctx, plan, v, C, y);
}

struct Work {
  float2* A;
  float2* B;
  float2* grid;
  float2* partials;
  size_t partial_cap;
  float2* S;   // Tucker: per-coil maps [C][N]
  float2* dS;  // Tucker: per-coil Jacobian maps [C][N]
  float2* T;   // Tucker: core / mode-product intermediates
};

mpi_status carve_work(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis, int C, Work* w) {
  mpi_status st = ensure_work(ctx, op_work_bytes(ctx, plan, basis, C));
  if (st) return st;
  const size_t cn = (size_t)C * plan->N;
  float2* base = (float2*)ctx->work;
  w->A = base;
  w->B = base + cn;
  // the line passes run on A; B is free while they run (the autotuner's scratch)
  ctx->tune_scratch = w->B;
  ctx->tune_scratch_bytes = cn * sizeof(float2);
  size_t grid = plan->kind == MPI_TRAJ_RADIAL ? nufft_grid_elems(plan, C) : 0;
  w->grid = base + 2 * cn;
  w->partials = base + 2 * cn + grid;
  w->partial_cap = partial_elems(ctx, basis, C);
  w->S = w->partials + w->partial_cap;
  w->dS = w->S + cn;
  w->T = w->dS + cn;
  return MPI_OK;
}

// Expansion fused with the point-wise products for dense bases; for Tucker
// bases the maps are materialised first and combined point-wise.
mpi_status run_expand(mpi_ctx* ctx, const mpi_basis* basis, int mode, const ExpandArgs& a, mpi_precision prec,
                      const Work& w) {
  if (!basis->tucker) return expand(ctx, basis, mode, a, prec);
  // With the x1 product on the CUDA cores, the forward fuses it with its
  // point-wise step; on the tensor cores the maps are written and combined below.
  if (tucker_fusable(mode) && !tucker_x1_on_tensor_cores(basis, a.C, prec))
    return tucker_fused(ctx, basis, mode, a, w.T, prec);
  mpi_status st = tucker_maps(ctx, basis, a.alpha, a.C, w.S, w.T, prec);
  if (st) return st;
  if (mode == EX_JFWD && (st = tucker_maps(ctx, basis, a.dalpha, a.C, w.dS, w.T, prec))) return st;
  return launch_pointwise(ctx, mode, a, w.S, w.dS);
}

}  // namespace

// ---------------------------------------------------------------- context

extern "C" mpi_status mpi_ctx_create(mpi_ctx** out, int device, void* cuda_stream) {
  if (!out) return MPI_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return MPI_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return MPI_ERR_CUDA;
  mpi_ctx* ctx = new mpi_ctx();
  ctx->device = device;
  ctx->stream = (cudaStream_t)cuda_stream;
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  // twiddle tables exp(-2 pi i m / n) for every supported length, from FP64
  std::vector<float2> host;
  for (int i = 0; i < kNumFftLengths; ++i) {
    const int n = kFftLengths[i];
    ctx->tw_offset[i] = (int)host.size();
    for (int m = 0; m < n; ++m) {
      const double ang = -2.0 * M_PI * (double)m / (double)n;
      host.push_back(make_float2((float)cos(ang), (float)sin(ang)));
    }
  }
  cudaError_t e = cudaMalloc(&ctx->twiddles, host.size() * sizeof(float2) + 256);
  if (e == cudaSuccess)
    e = cudaMemcpy(ctx->twiddles, host.data(), host.size() * sizeof(float2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    ctx->dev_err = (int*)((char*)ctx->twiddles + ((host.size() * sizeof(float2) + 127) & ~(size_t)127));
    e = cudaMemset(ctx->dev_err, 0, sizeof(int));
  }
  // The allocation-free forward's static scratch lives in a module of its own,
  // which the driver would otherwise load (and reserve 16 MiB for) at that
  // call's first use; load it now, while allocating is allowed.
  if (e == cudaSuccess) e = noalloc_preload();
  if (e == cudaSuccess) {
    ctx->tf32_read = tf32_reading_probe(ctx);
    ctx->tf32x3 = ctx->tf32_read == MPI_TF32_READ_TRUNCATE;
    if (ctx->tf32_read == MPI_TF32_READ_FAILED) e = cudaErrorLaunchFailure;  // no kernel of this library runs
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (ctx->twiddles) cudaFree(ctx->twiddles);
    delete ctx;
    return MPI_ERR_CUDA;
  }
  *out = ctx;
  return MPI_OK;
}

extern "C" mpi_status mpi_ctx_destroy(mpi_ctx* ctx) {
  if (!ctx) return MPI_ERR_ARG;
  DeviceGuard g(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (size_t i = 0; i < ctx->ev_begin.size(); ++i) {
    cudaEventDestroy(ctx->ev_begin[i]);
    cudaEventDestroy(ctx->ev_end[i]);
  }
  solver_cache_clear(ctx);
  for (mpi_ctx** slot : ctx->children) *slot = nullptr;  // orphan the children still alive
  if (ctx->work) cudaFree(ctx->work);
  if (ctx->stage) cudaFree(ctx->stage);
  if (ctx->twiddles) cudaFree(ctx->twiddles);
  delete ctx;
  return MPI_OK;
}

extern "C" mpi_status mpi_ctx_set_stream(mpi_ctx* ctx, void* stream) {
  if (!ctx) return MPI_ERR_ARG;
  ctx->stream = (cudaStream_t)stream;
  return MPI_OK;
}

extern "C" mpi_status mpi_ctx_synchronize(mpi_ctx* ctx) {
  if (!ctx) return MPI_ERR_ARG;
  DeviceGuard g(ctx->device);
  mpi_status st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "stream synchronize");
  if (st) return st;
  int err = 0;
  st = cuda_check(ctx, cudaMemcpy(&err, ctx->dev_err, sizeof(int), cudaMemcpyDeviceToHost), "error word");
  if (st) return st;
  if (err) {
    cudaMemset(ctx->dev_err, 0, sizeof(int));
    return set_err(ctx, MPI_ERR_TIMEOUT, "a kernel gave up on a bounded barrier wait (device error word set)");
  }
  return MPI_OK;
}

extern "C" mpi_status mpi_ctx_reserve(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis, int C) {
  if (!ctx) return MPI_ERR_ARG;
  if (!plan || !basis || C < 1) return set_err(ctx, MPI_ERR_ARG, "reserve: bad arguments");
  DeviceGuard g(ctx->device);
  // operators plus the solver state (IRGN/ADMM vectors)
  size_t extra = ((size_t)12 * plan->N + (size_t)8 * C * std::max(plan->M, 1) +
                  (size_t)8 * C * basis->q + 1024) * sizeof(float2);
  return ensure_work(ctx, op_work_bytes(ctx, plan, basis, C) + extra);
}

extern "C" mpi_status mpi_ctx_profile(mpi_ctx* ctx, int enable) {
  if (!ctx) return MPI_ERR_ARG;
  DeviceGuard g(ctx->device);
  if (enable && ctx->ev_begin.empty()) {
    ctx->ev_begin.resize(kProfileSlots);
    ctx->ev_end.resize(kProfileSlots);
    ctx->ev_family.assign(kProfileSlots, 0);
    ctx->ev_name.assign(kProfileSlots, nullptr);
    for (int i = 0; i < kProfileSlots; ++i) {
      if (cudaEventCreate(&ctx->ev_begin[i]) != cudaSuccess || cudaEventCreate(&ctx->ev_end[i]) != cudaSuccess) {
        cudaGetLastError();
        ctx->ev_begin.resize(i);
        ctx->ev_end.resize(i);
        return set_err(ctx, MPI_ERR_CUDA, "event creation failed");
      }
    }
  }
  ctx->profiling = enable != 0;
  ctx->pending_family = -1;
  return MPI_OK;
}

namespace {

// Folds the timed launches recorded since the last fold into the per-family
// and per-kernel sums (the caller has synchronised the stream).
void prof_fold(mpi_ctx* ctx) {
  for (int i = 0; i < ctx->ev_used; ++i) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, ctx->ev_begin[i], ctx->ev_end[i]) == cudaSuccess) {
      ctx->prof_ms[ctx->ev_family[i]] += t;
      ctx->prof_launches[ctx->ev_family[i]] += 1;
      const std::string nm = ctx->ev_name[i] ? ctx->ev_name[i] : "?";
      auto it = std::find_if(ctx->prof_kernels.begin(), ctx->prof_kernels.end(),
                             [&](const std::pair<std::string, std::pair<double, int64_t>>& k) { return k.first == nm; });
      if (it == ctx->prof_kernels.end()) {
        ctx->prof_kernels.push_back({nm, {0.0, 0}});
        it = ctx->prof_kernels.end() - 1;
      }
      it->second.first += t;
      it->second.second += 1;
    } else {
      cudaGetLastError();
    }
  }
  ctx->ev_used = 0;
}

}  // namespace

extern "C" mpi_status mpi_ctx_profile_read(mpi_ctx* ctx, int family, double* ms, int64_t* launches, int reset) {
  if (!ctx) return MPI_ERR_ARG;
  if (family < 0 || family >= KF_COUNT || !ms || !launches) return set_err(ctx, MPI_ERR_ARG, "bad profile query");
  DeviceGuard g(ctx->device);
  mpi_status st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "profile sync");
  if (st) return st;
  prof_fold(ctx);
  *ms = ctx->prof_ms[family];
  *launches = ctx->prof_launches[family];
  if (reset) {
    for (int k = 0; k < KF_COUNT; ++k) {
      ctx->prof_ms[k] = 0;
      ctx->prof_launches[k] = 0;
    }
    ctx->prof_kernels.clear();
  }
  return MPI_OK;
}

extern "C" mpi_status mpi_ctx_profile_kernel(mpi_ctx* ctx, int index, const char** name, double* ms,
                                             int64_t* launches) {
  if (!ctx) return MPI_ERR_ARG;
  if (!name || !ms || !launches) return set_err(ctx, MPI_ERR_ARG, "bad profile query");
  DeviceGuard g(ctx->device);
  mpi_status st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "profile sync");
  if (st) return st;
  prof_fold(ctx);
  if (index < 0 || index >= (int)ctx->prof_kernels.size()) return MPI_ERR_ARG;
  const auto& k = ctx->prof_kernels[index];
  *name = k.first.c_str();
  *ms = k.second.first;
  *launches = k.second.second;
  return MPI_OK;
}

extern "C" const char* mpi_last_error(const mpi_ctx* ctx) {
  if (!ctx) return "null context";
  return ctx->err.c_str();
}

extern "C" int64_t mpi_ctx_launch_count(const mpi_ctx* ctx) { return ctx ? ctx->launches : -1; }

extern "C" mpi_status mpi_ctx_set_autotune(mpi_ctx* ctx, int enable) {
  if (!ctx) return MPI_ERR_ARG;
  ctx->autotune = enable != 0;
  return MPI_OK;
}

extern "C" mpi_status mpi_ctx_set_wait_limit(mpi_ctx* ctx, int64_t cycles) {
  if (!ctx) return MPI_ERR_ARG;
  if (cycles < 1000) return set_err(ctx, MPI_ERR_ARG, "wait limit below 1000 cycles");
  ctx->wait_cycles = cycles;
  return MPI_OK;
}

extern "C" int mpi_ctx_tf32_reading(const mpi_ctx* ctx) { return ctx ? ctx->tf32_read : -1; }

extern "C" mpi_status mpi_ctx_set_tf32x3(mpi_ctx* ctx, int enable) {
  if (!ctx) return MPI_ERR_ARG;
  if (enable && ctx->tf32_read != MPI_TF32_READ_TRUNCATE)
    return set_err(ctx, MPI_ERR_UNSUPPORTED, "3xTF32 needs the truncating reading of FP32 kind::tf32 operands");
  ctx->tf32x3 = enable != 0;
  return MPI_OK;
}

extern "C" mpi_status mpi_ctx_inject_stall(mpi_ctx* ctx, int stages) {
  if (!ctx) return MPI_ERR_ARG;
  ctx->stall_after = stages < 0 ? -1 : stages;
  return MPI_OK;
}

extern "C" mpi_status mpi_ctx_set_line_kernel(mpi_ctx* ctx, int choice) {
  if (!ctx) return MPI_ERR_ARG;
  if (choice != 0 && choice != 8 && choice != 16 && choice != 32 && choice != -1 && choice != -2 && choice != -3)
    return set_err(ctx, MPI_ERR_ARG, "line kernel choice must be 0, 8, 16, 32, -1, -2 or -3");
  // -2: separate passes along y and x in 3D (no plane kernel), tuned line passes;
  // -3: the plane kernel with one CTA per plane instead of the pipelined one
  ctx->plane_pass = choice != -2;
  ctx->plane_pipe = choice != -3;
  ctx->line_kernel = choice == -2 ? 0 : choice;
  return MPI_OK;
}

extern "C" mpi_status mpi_ctx_tuning_record(const mpi_ctx* ctx, int index, const char** text_out) {
  if (!ctx || !text_out) return MPI_ERR_ARG;
  if (index < 0 || index >= (int)ctx->tuned.size()) return MPI_ERR_ARG;
  *text_out = ctx->tuned[index].what.c_str();
  return MPI_OK;
}

extern "C" int64_t mpi_ctx_workspace_bytes(const mpi_ctx* ctx) {
  return ctx ? (int64_t)(ctx->work_bytes + ctx->stage_bytes) : -1;
}

// ------------------------------------------------------------------- plan

extern "C" mpi_status mpi_plan_create(mpi_ctx* ctx, const mpi_plan_desc* d, mpi_plan** out) {
  if (!ctx) return MPI_ERR_ARG;
  if (!d || !out) return set_err(ctx, MPI_ERR_ARG, "null plan descriptor or output");
  *out = nullptr;
  DeviceGuard g(ctx->device);
  if (d->ndim != 2 && d->ndim != 3) return set_err(ctx, MPI_ERR_SHAPE, "ndim must be 2 or 3");
  const int nz = d->ndim == 3 ? d->dims[0] : 1, ny = d->dims[1], nx = d->dims[2];
  if (nz < 1 || ny < 1 || nx < 1) return set_err(ctx, MPI_ERR_SHAPE, "non-positive dimension");
  const long long Nll = (long long)nz * ny * nx;
  if (Nll > (1LL << 31) - 1) return set_err(ctx, MPI_ERR_SHAPE, "grid too large");
  if (d->M < 0) return set_err(ctx, MPI_ERR_ARG, "M < 0");
  mpi_plan* plan = new mpi_plan();
  plan->ctx = ctx;
  plan->device = ctx->device;
  plan->ndim = d->ndim;
  plan->nz = nz;
  plan->ny = ny;
  plan->nx = nx;
  plan->N = (int)Nll;
  plan->kind = d->kind;
  plan->M = d->M;
  mpi_status st = MPI_OK;
  if (d->kind == MPI_TRAJ_CARTESIAN) {
    if (!fft_length_supported(nx) || !fft_length_supported(ny) || (d->ndim == 3 && !fft_length_supported(nz))) {
      delete plan;
      return set_err(ctx, MPI_ERR_SHAPE, "unsupported Cartesian FFT length");
    }
    if (d->M > 0 && !d->sample_idx) {
      delete plan;
      return set_err(ctx, MPI_ERR_ARG, "null sample_idx");
    }
    for (int m = 0; m < d->M; ++m) {
      const int32_t v = d->sample_idx[m];
      if (v < 0 || v >= plan->N || (m > 0 && v <= d->sample_idx[m - 1])) {
        delete plan;
        return set_err(ctx, MPI_ERR_ARG, "sample_idx must be strictly increasing and in [0, N)");
      }
    }
    plan->n_rows = nz * ny;
    std::vector<int32_t> row_ptr(plan->n_rows + 1, 0);
    int m = 0;
    for (int r = 0; r < plan->n_rows; ++r) {
      row_ptr[r] = m;
      const long long end = (long long)(r + 1) * nx;
      while (m < d->M && d->sample_idx[m] < end) ++m;
    }
    row_ptr[plan->n_rows] = m;
    // row mask only where some k-space row has no samples (3D masks sample
    // whole readouts at a fraction of the (kz, ky) rows)
    std::vector<uint8_t> row_has(plan->n_rows);
    bool any_empty = false;
    for (int r = 0; r < plan->n_rows; ++r) {
      row_has[r] = row_ptr[r + 1] > row_ptr[r] ? 1 : 0;
      any_empty |= !row_has[r];
    }
    cudaError_t e = cudaMalloc(&plan->row_ptr, row_ptr.size() * sizeof(int32_t));
    if (e == cudaSuccess)
      e = cudaMemcpy(plan->row_ptr, row_ptr.data(), row_ptr.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && any_empty) e = cudaMalloc(&plan->row_has, row_has.size());
    if (e == cudaSuccess && any_empty)
      e = cudaMemcpy(plan->row_has, row_has.data(), row_has.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && d->ndim == 3) {
      // per kz plane, the rows with samples (the pipelined plane passes keep
      // only those rows of a plane in shared memory)
      std::vector<int32_t> cnt(nz, 0);
      std::vector<int16_t> slot((size_t)nz * ny, (int16_t)-1);
      for (int kz = 0; kz < nz; ++kz)
        for (int ky = 0; ky < ny; ++ky)
          if (row_has[(size_t)kz * ny + ky]) slot[(size_t)kz * ny + ky] = (int16_t)cnt[kz]++;
      plan->plane_kmax = nz > 0 ? *std::max_element(cnt.begin(), cnt.end()) : 0;
      const int kcap = std::max(plan->plane_kmax, 1);
      std::vector<int4> rows((size_t)nz * kcap, make_int4(-1, 0, 0, 0));
      for (int kz = 0; kz < nz; ++kz)
        for (int ky = 0; ky < ny; ++ky) {
          const int s = slot[(size_t)kz * ny + ky];
          const int r = kz * ny + ky;
          if (s >= 0) rows[(size_t)kz * kcap + s] = make_int4(ky, row_ptr[r], row_ptr[r + 1], 0);
        }
      e = cudaMalloc(&plan->plane_rows, rows.size() * sizeof(int4));
      if (e == cudaSuccess) e = cudaMalloc(&plan->plane_nrows, cnt.size() * sizeof(int32_t));
      if (e == cudaSuccess) e = cudaMalloc(&plan->plane_slot, slot.size() * sizeof(int16_t));
      if (e == cudaSuccess)
        e = cudaMemcpy(plan->plane_rows, rows.data(), rows.size() * sizeof(int4), cudaMemcpyHostToDevice);
      if (e == cudaSuccess)
        e = cudaMemcpy(plan->plane_nrows, cnt.data(), cnt.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
      if (e == cudaSuccess)
        e = cudaMemcpy(plan->plane_slot, slot.data(), slot.size() * sizeof(int16_t), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && d->M > 0) {
      e = cudaMalloc(&plan->idx, (size_t)d->M * sizeof(int32_t));
      if (e == cudaSuccess)
        e = cudaMemcpy(plan->idx, d->sample_idx, (size_t)d->M * sizeof(int32_t), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) st = cuda_check(ctx, e, "plan upload");
  } else if (d->kind == MPI_TRAJ_RADIAL) {
    if (d->ndim != 2 || nx != ny) {
      delete plan;
      return set_err(ctx, MPI_ERR_SHAPE, "radial plans are 2D square");
    }
    if (d->M > 0 && !d->traj) {
      delete plan;
      return set_err(ctx, MPI_ERR_ARG, "null trajectory");
    }
    if (d->kb_width < 2 || d->kb_width > 8) {
      delete plan;
      return set_err(ctx, MPI_ERR_ARG, "kb_width must be in [2, 8]");
    }
    plan->W = d->kb_width;
    plan->G = (int)lround((double)d->oversamp * nx);
    if (!fft_length_supported(plan->G) || plan->G < nx || (plan->G - nx) % 2) {
      delete plan;
      return set_err(ctx, MPI_ERR_SHAPE, "unsupported oversampled grid size");
    }
    for (int m = 0; m < 2 * d->M; ++m) {
      const float v = d->traj[m];
      if (!(v >= -3.14159274f && v <= 3.14159274f)) {
        delete plan;
        return set_err(ctx, MPI_ERR_ARG, "trajectory outside [-pi, pi]");
      }
    }
    st = nufft_plan_init(ctx, plan, d->traj);
  } else {
    delete plan;
    return set_err(ctx, MPI_ERR_ARG, "unknown trajectory kind");
  }
  if (st != MPI_OK) {
    mpi_plan_destroy(plan);
    return st;
  }
  ctx_adopt(ctx, &plan->ctx);  // only a fully made plan is tracked
  *out = plan;
  return MPI_OK;
}

extern "C" mpi_status mpi_plan_destroy(mpi_plan* plan) {
  if (!plan) return MPI_ERR_ARG;
  DeviceGuard g(plan->device);
  if (plan->ctx) {  // else the context is gone, and it drained its stream when it went
    cudaStreamSynchronize(plan->ctx->stream);
    solver_cache_forget(plan->ctx, plan);
    ctx_release(&plan->ctx);
  }
  void* ptrs[] = {plan->idx,        plan->row_ptr,     plan->row_has,    plan->plane_rows, plan->plane_nrows,
                  plan->plane_slot, plan->traj,        plan->gstart,     plan->gw,         plan->deap,
                  plan->cell_ptr,   plan->cell_rank,   plan->cell_sx,    plan->cell_w,     plan->cell_dense,
                  plan->tile_items, plan->tile_samples};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete plan;
  return MPI_OK;
}

extern "C" mpi_status mpi_plan_grid_index(mpi_ctx* ctx, const mpi_plan* plan, int32_t* out_dev) {
  if (!ctx) return MPI_ERR_ARG;
  if (!plan || bad_ptr(out_dev)) return set_err(ctx, MPI_ERR_ARG, "null argument");
  if (plan->kind != MPI_TRAJ_RADIAL) return set_err(ctx, MPI_ERR_ARG, "not a radial plan");
  DeviceGuard g(ctx->device);
  if (plan->M == 0) return MPI_OK;
  return cuda_check(ctx,
                    cudaMemcpyAsync(out_dev, plan->gstart, (size_t)plan->M * 2 * sizeof(int32_t),
                                    cudaMemcpyDeviceToDevice, ctx->stream),
                    "grid index copy");
}

// ------------------------------------------------------------------ basis

extern "C" mpi_status mpi_basis_load_dense(mpi_ctx* ctx, const mpi_c32* U, int N, int q, int on_device,
                                           mpi_basis** out) {
  if (!ctx) return MPI_ERR_ARG;
  if (!U || !out) return set_err(ctx, MPI_ERR_ARG, "null basis pointer");
  if (N < 4 || (N % 4) || q < 1 || q > 256) return set_err(ctx, MPI_ERR_SHAPE, "need N >= 4 divisible by 4 and 1 <= q <= 256");
  *out = nullptr;
  DeviceGuard g(ctx->device);
  mpi_basis* b = new mpi_basis();
  b->ctx = ctx;
  b->device = ctx->device;
  b->N = N;
  b->q = q;
  const size_t bytes = (size_t)N * q * sizeof(float2);
  cudaError_t e = cudaMalloc(&b->U, bytes);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->U, U, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    mpi_status st = cuda_check(ctx, e, "basis upload");
    if (b->U) cudaFree(b->U);
    delete b;
    return st == MPI_OK ? MPI_ERR_CUDA : st;
  }
  // BF16 operand copy for the tensor-core path; without it only FP32 is served
  if (tc_basis_prepare(ctx, b) != MPI_OK) {
    b->bf16_err = ctx->err;
    if (b->Ubf) cudaFree(b->Ubf);
    b->Ubf = nullptr;
    tc_basis_release(b);
  }
  // FP32 operand copy for the 3xTF32 tensor-core path; without it FP32 runs on CUDA cores
  if (tf32_basis_prepare(ctx, b) != MPI_OK) {
    if (b->Uf32) cudaFree(b->Uf32);
    b->Uf32 = nullptr;
    tf32_basis_release(b);
  }
  // views of U for the tensor-core U^H V; without them it runs on the CUDA cores
  if (uh_tc_prepare(ctx, b) != MPI_OK) uh_tc_release(b);
  e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    mpi_status st = cuda_check(ctx, e, "basis conversion");
    mpi_basis_destroy(b);
    return st;
  }
  ctx_adopt(ctx, &b->ctx);  // only a fully made basis is tracked
  *out = b;
  return MPI_OK;
}

extern "C" mpi_status mpi_basis_load_tucker(mpi_ctx* ctx, const mpi_c32* core, const mpi_c32* U1, const mpi_c32* U2,
                                            const mpi_c32* U3, const int n[3], const int r[3], int q, int on_device,
                                            mpi_basis** out) {
  if (!ctx) return MPI_ERR_ARG;
  if (!core || !U1 || !U2 || !U3 || !n || !r || !out) return set_err(ctx, MPI_ERR_ARG, "null Tucker argument");
  *out = nullptr;
  for (int k = 0; k < 3; ++k)
    if (n[k] < 1 || r[k] < 1 || r[k] > n[k] || r[k] > 128)
      return set_err(ctx, MPI_ERR_SHAPE, "Tucker ranks must satisfy 1 <= r_k <= min(n_k, 128)");
  if (n[1] > 256 || n[2] > 256 || n[0] > 256)
    return set_err(ctx, MPI_ERR_SHAPE, "Tucker factor lengths above 256 are not supported");
  const long long R = (long long)r[0] * r[1] * r[2];
  const long long N = (long long)n[0] * n[1] * n[2];
  if (R % 4 || N % 4 || N > (1LL << 31) - 1) return set_err(ctx, MPI_ERR_SHAPE, "Tucker sizes (R, N must be multiples of 4)");
  DeviceGuard g(ctx->device);
  mpi_basis* cb = nullptr;
  mpi_status st = mpi_basis_load_dense(ctx, core, (int)R, q, on_device, &cb);
  if (st) return st;
  mpi_basis* b = new mpi_basis();
  b->ctx = ctx;
  b->device = ctx->device;
  b->N = (int)N;
  b->q = q;
  b->tucker = true;
  b->core = cb;
  const mpi_c32* src[3] = {U1, U2, U3};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
    b->n[k] = n[k];
    b->r[k] = r[k];
    const size_t bytes = (size_t)n[k] * r[k] * sizeof(float2);
    e = cudaMalloc(&b->F[k], bytes);
    if (e == cudaSuccess)
      e = cudaMemcpy(b->F[k], src[k], bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    st = cuda_check(ctx, e, "Tucker factor upload");
    mpi_basis_destroy(b);
    return st;
  }
  if ((st = tucker_conj_factors(ctx, b))) {
    mpi_basis_destroy(b);
    return st;
  }
  ctx_adopt(ctx, &b->ctx);  // only a fully made basis is tracked
  *out = b;
  return MPI_OK;
}

extern "C" mpi_status mpi_basis_destroy(mpi_basis* b) {
  if (!b) return MPI_ERR_ARG;
  DeviceGuard g(b->device);
  if (b->ctx) {  // else the context is gone, and it drained its stream when it went
    cudaStreamSynchronize(b->ctx->stream);
    solver_cache_forget(b->ctx, b);
    ctx_release(&b->ctx);
  }
  if (b->U) cudaFree(b->U);
  if (b->Ubf) cudaFree(b->Ubf);
  tc_basis_release(b);
  if (b->Uf32) cudaFree(b->Uf32);
  tf32_basis_release(b);
  uh_tc_release(b);
  for (int k = 0; k < 3; ++k) {
    if (b->F[k]) cudaFree(b->F[k]);
    if (b->Fh[k]) cudaFree(b->Fh[k]);
  }
  if (b->core) mpi_basis_destroy(b->core);
  delete (CUtensorMap*)b->op_map;
  tucker_chain_release(b);
  delete b;
  return MPI_OK;
}

// --------------------------------------------------------------- operators

extern "C" mpi_status mpi_basis_expand(mpi_ctx* ctx, const mpi_basis* basis, const mpi_c32* alpha, int C,
                                       mpi_c32* maps, mpi_precision prec) {
  if (!ctx) return MPI_ERR_ARG;
  if (!basis || bad_ptr(alpha) || bad_ptr(maps) || C < 1) return set_err(ctx, MPI_ERR_ARG, "bad argument");
  if (prec != MPI_PREC_FP32 && prec != MPI_PREC_BF16 && prec != MPI_PREC_FP32_SIMT)
    return set_err(ctx, MPI_ERR_ARG, "bad precision");
  const mpi_basis* eb = basis->tucker ? basis->core : basis;
  if (prec == MPI_PREC_BF16 && !eb->Ubf)
    return set_err(ctx, MPI_ERR_UNSUPPORTED, "BF16 expansion unavailable: " + eb->bf16_err);
  DeviceGuard g(ctx->device);
  if (basis->tucker) {
    mpi_status st = ensure_work(ctx, tucker_work_elems(basis, C) * sizeof(float2) + 4096);
    if (st) return st;
    return tucker_maps(ctx, basis, (const float2*)alpha, C, (float2*)maps, (float2*)ctx->work, prec);
  }
  ExpandArgs a;
  a.U = basis->U;
  a.N = basis->N;
  a.q = basis->q;
  a.C = C;
  a.alpha = (const float2*)alpha;
  a.out = (float2*)maps;
  return expand(ctx, basis, EX_MAPS, a, prec);
}

extern "C" mpi_status mpi_forward(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis,
                                  const mpi_c32* alpha, int C, const mpi_c32* p, mpi_c32* y,
                                  mpi_precision prec) {
  mpi_status st = check_op(ctx, plan, basis, C, prec);
  if (st) return st;
  if (bad_ptr(alpha) || bad_ptr(p) || (plan->M > 0 && bad_ptr(y))) return set_err(ctx, MPI_ERR_ARG, "null pointer");
  DeviceGuard g(ctx->device);
  Work w;
  if ((st = carve_work(ctx, plan, basis, C, &w))) return st;
  ExpandArgs a = base_args(plan, basis, C);
  a.alpha = (const float2*)alpha;
  a.p = (const float2*)p;
  a.out = w.A;
  if (tucker_x1_fused_supported(basis, plan, C, prec)) {
    // x1 product, point-wise step and the DFT along z in one tensor-core pass,
    // then the passes along y and x
    void* op = nullptr;
    void* map = nullptr;
    if ((st = tucker_x1_operand(ctx, basis, a.alpha, C, w.T, prec, &op, &map))) return st;
    if ((st = tucker_x1_fused_launch(ctx, basis, plan, false, C, map, a.p, nullptr, w.A, a.scale, prec))) return st;
    if (ctx->plane_pass && plane_pass_supported(plan)) return launch_plane_yx(ctx, plan, w.A, C, (float2*)y, false);
    if ((st = launch_fft_cols(ctx, w.A, C, plan->nz, plan->ny, plan->nx, false, plan->row_has))) return st;
    return launch_rows_fwd_gather(ctx, plan, w.A, C, (float2*)y);
  }
  if ((st = run_expand(ctx, basis, EX_FWD, a, prec, w))) return st;
  return image_to_kspace(ctx, plan, w.A, C, (float2*)y, w.grid);
}

extern "C" mpi_status mpi_adjoint(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis,
                                  const mpi_c32* alpha, int C, const mpi_c32* y, mpi_c32* p_out,
                                  mpi_precision prec) {
  mpi_status st = check_op(ctx, plan, basis, C, prec);
  if (st) return st;
  if (bad_ptr(alpha) || bad_ptr(p_out) || (plan->M > 0 && bad_ptr(y))) return set_err(ctx, MPI_ERR_ARG, "null pointer");
  DeviceGuard g(ctx->device);
  Work w;
  if ((st = carve_work(ctx, plan, basis, C, &w))) return st;
  ExpandArgs a = base_args(plan, basis, C);
  a.alpha = (const float2*)alpha;
  a.w = w.A;
  a.out = (float2*)p_out;
  if (tucker_x1_fused_supported(basis, plan, C, prec)) {
    // inverse passes along x and y, then one tensor-core pass: the inverse DFT
    // along z, the maps' x1 product and the sum over coils of conj(s_c) w_c
    if (ctx->plane_pass && plane_pass_supported(plan)) {
      if ((st = launch_plane_yx(ctx, plan, w.A, C, (float2*)y, true))) return st;
    } else {
      if ((st = launch_rows_scatter_inv(ctx, plan, (const float2*)y, C, w.A))) return st;
      if ((st = launch_fft_cols(ctx, w.A, C, plan->nz, plan->ny, plan->nx, true, plan->row_has))) return st;
    }
    void* op = nullptr;
    void* map = nullptr;
    if ((st = tucker_x1_operand(ctx, basis, a.alpha, C, w.T, prec, &op, &map))) return st;
    return tucker_x1_fused_launch(ctx, basis, plan, true, C, map, nullptr, w.A, a.out, a.scale, prec);
  }
  if ((st = kspace_to_image(ctx, plan, (const float2*)y, C, w.A, w.grid))) return st;
  return run_expand(ctx, basis, EX_ADJ, a, prec, w);
}

namespace {

// Device staging for the host-buffer calls: grown like the workspace, with a
// stream sync before the old buffer is freed.
mpi_status ensure_stage(mpi_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->stage_bytes) return MPI_OK;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_check(ctx, e, "staging sync");
  if (ctx->stage) cudaFree(ctx->stage);
  ctx->stage = nullptr;
  ctx->stage_bytes = 0;
  e = cudaMalloc(&ctx->stage, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, MPI_ERR_OOM, "staging allocation failed");
  }
  ctx->stage_bytes = bytes;
  return MPI_OK;
}

// Device address of a host buffer the GPU can access in place (pinned and
// mapped, e.g. from cudaHostAlloc), or null for pageable memory.  On GB300 the
// kernels then read and write it directly over the coherent CPU-GPU link.
const void* mapped_host(const void* h) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, h) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// One host-buffer operator call.  Pinned buffers are used in place; pageable
// ones go through the staging buffer: alpha [C][q] and the input (n_in
// elements) copied in, the output (n_out elements) copied back.  `op` runs on
// the device addresses; the call waits for the stream before returning.
// `reread_in`: the kernels read the input more than once (the 3D forward reads
// the image once per coil), so it is copied to the device even when pinned.
template <class Op>
mpi_status host_call(mpi_ctx* ctx, const mpi_basis* basis, int C, const mpi_c32* alpha, const mpi_c32* in,
                     size_t n_in, mpi_c32* out, size_t n_out, Op op, bool reread_in = false) {
  const size_t n_alpha = (size_t)C * basis->q;
  // an empty input or output (no samples) is passed through as given
  const mpi_c32* da = (const mpi_c32*)mapped_host(alpha);
  const mpi_c32* di = n_in ? (reread_in ? nullptr : (const mpi_c32*)mapped_host(in)) : in;
  mpi_c32* dout = n_out ? (mpi_c32*)mapped_host(out) : out;
  const bool stage_a = !da, stage_i = n_in && !di, copy_out = n_out && !dout;
  const size_t a_off = 0, i_off = (n_alpha + 1) & ~(size_t)1, o_off = i_off + ((n_in + 1) & ~(size_t)1);
  if (stage_a || stage_i || copy_out) {
    mpi_status st = ensure_stage(ctx, (o_off + n_out) * sizeof(mpi_c32));
    if (st) return st;
  }
  mpi_c32* d = (mpi_c32*)ctx->stage;
  cudaError_t e = cudaSuccess;
  if (stage_a) {
    e = cudaMemcpyAsync(d + a_off, alpha, n_alpha * sizeof(mpi_c32), cudaMemcpyHostToDevice, ctx->stream);
    da = d + a_off;
  }
  if (e == cudaSuccess && stage_i) {
    e = cudaMemcpyAsync(d + i_off, in, n_in * sizeof(mpi_c32), cudaMemcpyHostToDevice, ctx->stream);
    di = d + i_off;
  }
  if (e != cudaSuccess) return cuda_check(ctx, e, "host input copy");
  if (copy_out) dout = d + o_off;
  mpi_status st = op(da, di, dout);
  if (st) return st;
  if (copy_out) e = cudaMemcpyAsync(out, dout, n_out * sizeof(mpi_c32), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  return e == cudaSuccess ? MPI_OK : cuda_check(ctx, e, "host output copy");
}

}  // namespace

extern "C" mpi_status mpi_forward_host(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis,
                                       const mpi_c32* alpha, int C, const mpi_c32* p, mpi_c32* y,
                                       mpi_precision prec) {
  mpi_status st = check_op(ctx, plan, basis, C, prec);
  if (st) return st;
  if (bad_ptr(alpha) || bad_ptr(p) || (plan->M > 0 && bad_ptr(y))) return set_err(ctx, MPI_ERR_ARG, "null pointer");
  DeviceGuard g(ctx->device);
  return host_call(ctx, basis, C, alpha, p, (size_t)plan->N, y, (size_t)C * plan->M,
                   [&](const mpi_c32* da, const mpi_c32* dp, mpi_c32* dy) {
                     return mpi_forward(ctx, plan, basis, da, C, dp, dy, prec);
                   },
                   tucker_x1_fused_supported(basis, plan, C, prec));
}

extern "C" mpi_status mpi_adjoint_host(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis,
                                       const mpi_c32* alpha, int C, const mpi_c32* y, mpi_c32* p_out,
                                       mpi_precision prec) {
  mpi_status st = check_op(ctx, plan, basis, C, prec);
  if (st) return st;
  if (bad_ptr(alpha) || bad_ptr(p_out) || (plan->M > 0 && bad_ptr(y))) return set_err(ctx, MPI_ERR_ARG, "null pointer");
  DeviceGuard g(ctx->device);
  return host_call(ctx, basis, C, alpha, y, (size_t)C * plan->M, p_out, (size_t)plan->N,
                   [&](const mpi_c32* da, const mpi_c32* dy, mpi_c32* dp) {
                     return mpi_adjoint(ctx, plan, basis, da, C, dy, dp, prec);
                   });
}

extern "C" mpi_status mpi_jacobian(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis,
                                   const mpi_c32* alpha, int C, const mpi_c32* p, const mpi_c32* dp,
                                   const mpi_c32* dalpha, mpi_c32* dy, mpi_precision prec) {
  mpi_status st = check_op(ctx, plan, basis, C, prec);
  if (st) return st;
  if (bad_ptr(alpha) || bad_ptr(p) || bad_ptr(dp) || bad_ptr(dalpha) || (plan->M > 0 && bad_ptr(dy)))
    return set_err(ctx, MPI_ERR_ARG, "null pointer");
  DeviceGuard g(ctx->device);
  Work w;
  if ((st = carve_work(ctx, plan, basis, C, &w))) return st;
  ExpandArgs a = base_args(plan, basis, C);
  a.alpha = (const float2*)alpha;
  a.dalpha = (const float2*)dalpha;
  a.p = (const float2*)p;
  a.dp = (const float2*)dp;
  a.out = w.A;
  if (tucker_x1_fused_supported(basis, plan, C, prec)) {
    // J = F_s(S(dalpha) p + S(alpha) dp): the forward's fused x1 pass (maps,
    // point-wise step, DFT along z) once per term, the second adding into the
    // first, then the passes along y and x
    void* op = nullptr;
    void* map = nullptr;
    if ((st = tucker_x1_operand(ctx, basis, a.dalpha, C, w.T, prec, &op, &map))) return st;
    if ((st = tucker_x1_fused_launch(ctx, basis, plan, false, C, map, a.p, nullptr, w.A, a.scale, prec))) return st;
    if ((st = tucker_x1_operand(ctx, basis, a.alpha, C, w.T, prec, &op, &map))) return st;
    if ((st = tucker_x1_fused_launch(ctx, basis, plan, false, C, map, a.dp, nullptr, w.A, a.scale, prec, true)))
      return st;
    if (ctx->plane_pass && plane_pass_supported(plan)) return launch_plane_yx(ctx, plan, w.A, C, (float2*)dy, false);
    if ((st = launch_fft_cols(ctx, w.A, C, plan->nz, plan->ny, plan->nx, false, plan->row_has))) return st;
    return launch_rows_fwd_gather(ctx, plan, w.A, C, (float2*)dy);
  }
  if ((st = run_expand(ctx, basis, EX_JFWD, a, prec, w))) return st;
  return image_to_kspace(ctx, plan, w.A, C, (float2*)dy, w.grid);
}

extern "C" mpi_status mpi_jacobian_adjoint(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis,
                                           const mpi_c32* alpha, int C, const mpi_c32* p, const mpi_c32* r,
                                           mpi_c32* dp, mpi_c32* dalpha, mpi_precision prec) {
  mpi_status st = check_op(ctx, plan, basis, C, prec);
  if (st) return st;
  if (bad_ptr(alpha) || bad_ptr(p) || bad_ptr(dp) || bad_ptr(dalpha) || (plan->M > 0 && bad_ptr(r)))
    return set_err(ctx, MPI_ERR_ARG, "null pointer");
  DeviceGuard g(ctx->device);
  Work w;
  if ((st = carve_work(ctx, plan, basis, C, &w))) return st;
  if (tucker_jadj_tc_supported(basis, plan, C, prec)) {
    // the inverse passes along x and y; dp = the adjoint's fused x1 pass (inverse
    // DFT along z, maps, sum over coils); dalpha = the conjugate chain on the
    // tensor cores from the same per-coil data
    if (ctx->plane_pass && plane_pass_supported(plan)) {
      if ((st = launch_plane_yx(ctx, plan, w.A, C, (float2*)r, true))) return st;
    } else {
      if ((st = launch_rows_scatter_inv(ctx, plan, (const float2*)r, C, w.A))) return st;
      if ((st = launch_fft_cols(ctx, w.A, C, plan->nz, plan->ny, plan->nx, true, plan->row_has))) return st;
    }
    const float scale = base_args(plan, basis, C).scale;
    void* op = nullptr;
    void* map = nullptr;
    if ((st = tucker_x1_operand(ctx, basis, (const float2*)alpha, C, w.T, prec, &op, &map))) return st;
    if ((st = tucker_x1_fused_launch(ctx, basis, plan, true, C, map, nullptr, w.A, (float2*)dp, scale, prec)))
      return st;
    return tucker_jadj_alpha(ctx, basis, plan, w.A, (const float2*)p, scale, C, w.B, (float2*)dalpha, w.T,
                             w.partials, w.partial_cap);
  }
  if ((st = kspace_to_image(ctx, plan, (const float2*)r, C, w.A, w.grid))) return st;
  ExpandArgs a = base_args(plan, basis, C);
  a.alpha = (const float2*)alpha;
  a.p = (const float2*)p;
  a.w = w.A;
  a.out = (float2*)dp;
  a.vout = w.B;
  if ((st = run_expand(ctx, basis, EX_JADJ, a, prec, w))) return st;
  if (basis->tucker)
    return tucker_adjoint(ctx, basis, w.B, C, (float2*)dalpha, w.T, w.partials, w.partial_cap, prec);
  return uh_v(ctx, basis, w.B, C, (float2*)dalpha, w.partials, w.partial_cap, prec);
}

// ----------------------------------------------------- several sets of maps
//
// y_k = F_s(sum_m (U alpha_{m,k}) (.) p_m) (the forward model with extra
// bilinear terms, Discussion: "Forward Model Extensions").  Dense bases.  The
// image-side sum is formed by the expansion epilogues: two sets per launch
// through the Jacobian's two-product epilogue (s (.) dp + ds (.) p with
// (alpha, dp, dalpha, p) = (alpha_m, p_m, alpha_{m+1}, p_{m+1})), further
// launches adding into the same buffer.

namespace {

mpi_status check_maps(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis, int M, int C, mpi_precision prec) {
  mpi_status st = check_op(ctx, plan, basis, C, prec);
  if (st) return st;
  if (M < 1) return set_err(ctx, MPI_ERR_ARG, "M must be >= 1");
  if (basis->tucker && M > 1) return set_err(ctx, MPI_ERR_UNSUPPORTED, "several sets of maps: dense bases only");
  return MPI_OK;
}

}  // namespace

extern "C" mpi_status mpi_forward_maps(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis, int M,
                                       const mpi_c32* alpha, int C, const mpi_c32* p, mpi_c32* y,
                                       mpi_precision prec) {
  mpi_status st = check_maps(ctx, plan, basis, M, C, prec);
  if (st) return st;
  if (bad_ptr(alpha) || bad_ptr(p) || (plan->M > 0 && bad_ptr(y))) return set_err(ctx, MPI_ERR_ARG, "null pointer");
  if (M == 1) return mpi_forward(ctx, plan, basis, alpha, C, p, y, prec);
  DeviceGuard g(ctx->device);
  Work w;
  if ((st = carve_work(ctx, plan, basis, C, &w))) return st;
  const size_t Cq = (size_t)C * basis->q, N = (size_t)plan->N;
  for (int m = 0; m < M; m += 2) {
    ExpandArgs a = base_args(plan, basis, C);
    a.out = w.A;
    a.accumulate = m > 0;
    a.alpha = (const float2*)alpha + m * Cq;
    if (m + 1 < M) {
      a.dp = (const float2*)p + m * N;
      a.dalpha = (const float2*)alpha + (m + 1) * Cq;
      a.p = (const float2*)p + (m + 1) * N;
      if ((st = expand(ctx, basis, EX_JFWD, a, prec))) return st;
    } else {
      a.p = (const float2*)p + m * N;
      if ((st = expand(ctx, basis, EX_FWD, a, prec))) return st;
    }
  }
  return image_to_kspace(ctx, plan, w.A, C, (float2*)y, w.grid);
}

extern "C" mpi_status mpi_adjoint_maps(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis, int M,
                                       const mpi_c32* alpha, int C, const mpi_c32* y, mpi_c32* p_out,
                                       mpi_precision prec) {
  mpi_status st = check_maps(ctx, plan, basis, M, C, prec);
  if (st) return st;
  if (bad_ptr(alpha) || bad_ptr(p_out) || (plan->M > 0 && bad_ptr(y)))
    return set_err(ctx, MPI_ERR_ARG, "null pointer");
  if (M == 1) return mpi_adjoint(ctx, plan, basis, alpha, C, y, p_out, prec);
  DeviceGuard g(ctx->device);
  Work w;
  if ((st = carve_work(ctx, plan, basis, C, &w))) return st;
  if ((st = kspace_to_image(ctx, plan, (const float2*)y, C, w.A, w.grid))) return st;
  const size_t Cq = (size_t)C * basis->q, N = (size_t)plan->N;
  for (int m = 0; m < M; ++m) {
    ExpandArgs a = base_args(plan, basis, C);
    a.alpha = (const float2*)alpha + m * Cq;
    a.w = w.A;
    a.out = (float2*)p_out + m * N;
    if ((st = expand(ctx, basis, EX_ADJ, a, prec))) return st;
  }
  return MPI_OK;
}

extern "C" mpi_status mpi_jacobian_maps(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis, int M,
                                        const mpi_c32* alpha, int C, const mpi_c32* p, const mpi_c32* dp,
                                        const mpi_c32* dalpha, mpi_c32* dy, mpi_precision prec) {
  mpi_status st = check_maps(ctx, plan, basis, M, C, prec);
  if (st) return st;
  if (bad_ptr(alpha) || bad_ptr(p) || bad_ptr(dp) || bad_ptr(dalpha) || (plan->M > 0 && bad_ptr(dy)))
    return set_err(ctx, MPI_ERR_ARG, "null pointer");
  if (M == 1) return mpi_jacobian(ctx, plan, basis, alpha, C, p, dp, dalpha, dy, prec);
  DeviceGuard g(ctx->device);
  Work w;
  if ((st = carve_work(ctx, plan, basis, C, &w))) return st;
  const size_t Cq = (size_t)C * basis->q, N = (size_t)plan->N;
  for (int m = 0; m < M; ++m) {
    ExpandArgs a = base_args(plan, basis, C);
    a.out = w.A;
    a.accumulate = m > 0;
    a.alpha = (const float2*)alpha + m * Cq;
    a.dalpha = (const float2*)dalpha + m * Cq;
    a.p = (const float2*)p + m * N;
    a.dp = (const float2*)dp + m * N;
    if ((st = expand(ctx, basis, EX_JFWD, a, prec))) return st;
  }
  return image_to_kspace(ctx, plan, w.A, C, (float2*)dy, w.grid);
}

extern "C" mpi_status mpi_jacobian_adjoint_maps(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis, int M,
                                                const mpi_c32* alpha, int C, const mpi_c32* p, const mpi_c32* r,
                                                mpi_c32* dp, mpi_c32* dalpha, mpi_precision prec) {
  mpi_status st = check_maps(ctx, plan, basis, M, C, prec);
  if (st) return st;
  if (bad_ptr(alpha) || bad_ptr(p) || bad_ptr(dp) || bad_ptr(dalpha) || (plan->M > 0 && bad_ptr(r)))
    return set_err(ctx, MPI_ERR_ARG, "null pointer");
  if (M == 1) return mpi_jacobian_adjoint(ctx, plan, basis, alpha, C, p, r, dp, dalpha, prec);
  DeviceGuard g(ctx->device);
  Work w;
  if ((st = carve_work(ctx, plan, basis, C, &w))) return st;
  if ((st = kspace_to_image(ctx, plan, (const float2*)r, C, w.A, w.grid))) return st;
  const size_t Cq = (size_t)C * basis->q, N = (size_t)plan->N;
  for (int m = 0; m < M; ++m) {
    ExpandArgs a = base_args(plan, basis, C);
    a.alpha = (const float2*)alpha + m * Cq;
    a.p = (const float2*)p + m * N;
    a.w = w.A;
    a.out = (float2*)dp + m * N;
    a.vout = w.B;
    if ((st = expand(ctx, basis, EX_JADJ, a, prec))) return st;
    if ((st = uh_v(ctx, basis, w.B, C, (float2*)dalpha + m * Cq, w.partials, w.partial_cap, prec))) return st;
  }
  return MPI_OK;
}

// ----------------------------------------------------------- grouped batches

bool rows_supported(const mpi_basis* basis, int Cmax, mpi_precision prec) {
  if (basis->tucker || Cmax < 1) return false;
  if (prec == MPI_PREC_BF16) return basis->Ubf && 2 * ((2 * Cmax + 15) / 16 * 8) <= 256;
  if (prec == MPI_PREC_FP32) return tf32_supported(basis, EX_FWD, Cmax) && tf32_supported(basis, EX_ADJ, Cmax);
  return false;
}

mpi_status expand_rows(mpi_ctx* ctx, const mpi_plan* plan0, const mpi_basis* basis, int mode, const ExpandRow* rows,
                       int nrows, int Cmax, mpi_precision prec, int row_ctas) {
  if (!rows_supported(basis, Cmax, prec)) return set_err(ctx, MPI_ERR_UNSUPPORTED, "grouped expansion: shape");
  if (nrows < 1 || nrows > 65535) return set_err(ctx, MPI_ERR_SHAPE, "grouped expansion: row count");
  ExpandArgs a = base_args(plan0, basis, Cmax);
  a.rows = rows;
  a.nrows = nrows;
  a.row_ctas = row_ctas;
  a.kname = mode == EX_FWD ? "k_expand<grouped fwd>" : "k_expand<grouped adj>";
  if (prec == MPI_PREC_BF16) return launch_expand_tc(ctx, basis, mode, a);
  return launch_expand_tf32(ctx, basis, mode, a);
}

mpi_status plan_image_to_kspace(mpi_ctx* ctx, const mpi_plan* plan, float2* v, int C, float2* y) {
  if (plan->kind != MPI_TRAJ_CARTESIAN) return set_err(ctx, MPI_ERR_UNSUPPORTED, "grouped batch: Cartesian plans");
  return image_to_kspace(ctx, plan, v, C, y, nullptr);
}

mpi_status plan_kspace_to_image(mpi_ctx* ctx, const mpi_plan* plan, const float2* y, int C, float2* w) {
  if (plan->kind != MPI_TRAJ_CARTESIAN) return set_err(ctx, MPI_ERR_UNSUPPORTED, "grouped batch: Cartesian plans");
  return kspace_to_image(ctx, plan, y, C, w, nullptr);
}
