// Batched operator application over many slices of uneven grid size and coil
// count, replayed as one CUDA graph.
//
// mpi_batch_create orders the slices by basis (slices of the same grid share
// one Maxwell basis), sizes the context workspace for the largest slice, and
// records every kernel of every slice's operator calls into one graph by stream
// capture on a private stream.  mpi_batch_run launches that graph on the
// context's stream.  The captured pointers are the caller's buffers, which must
// stay valid for the life of the batch.
//
// Grouped expansion: consecutive slices on Cartesian plans that share a dense
// basis (FP32 or BF16, every slice's coils within one tensor-core pass) form a
// group.  The group's basis expansion is one launch whose grid rows are its
// slices (a device table gives each row its coefficients, image, per-coil data
// and output); the rows stream the same basis tiles in step, so the basis is
// read from DRAM about once per group instead of once per slice.  Each slice's
// per-coil images live in a batch-owned buffer between the expansion and the
// slice's FFT passes.  How many CTAs each row gets is chosen at creation by
// timing the candidates (an autotuner decision the context records).
#include <algorithm>
#include <cstdio>
#include <numeric>
#include <string>
#include <vector>

#include "mpi_internal.h"

struct mpi_batch {
  mpi_ctx* ctx = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int n = 0;
  int64_t kernels = 0;  // kernels per replay
  void* buf = nullptr;   // per-coil images of one group [sum C][N]
  void* rows = nullptr;  // row tables of every group (device)
  int groups = 0;        // grouped launches per direction
};

namespace {

mpi_status record_slice(mpi_ctx* ctx, const mpi_batch_slice& s, int kind, mpi_precision prec) {
  mpi_status st = MPI_OK;
  if (kind & MPI_BATCH_FORWARD)
    st = mpi_forward(ctx, s.plan, s.basis, s.alpha, s.C, s.p, s.y, prec);
  if (st == MPI_OK && (kind & MPI_BATCH_ADJOINT))
    st = mpi_adjoint(ctx, s.plan, s.basis, s.alpha, s.C, s.y, s.x, prec);
  return st;
}

struct Group {
  std::vector<int> idx;  // slices, in recording order
  int Cmax = 0;
  long sumC = 0;
  size_t fwd_rows = 0, adj_rows = 0;  // offsets (rows) into the device row table
  int row_ctas = 0;
};

bool groupable(const mpi_batch_slice& s, mpi_precision prec) {
  return s.plan->kind == MPI_TRAJ_CARTESIAN && !s.basis->tucker && rows_supported(s.basis, s.C, prec);
}

// The group's forward and adjoint expansions, and its slices' FFT passes.
mpi_status record_group(mpi_ctx* ctx, const mpi_batch_slice* sl, const Group& g, int kind, mpi_precision prec,
                        const ExpandRow* rows, float2* buf) {
  const mpi_batch_slice& s0 = sl[g.idx[0]];
  const long N = s0.plan->N;
  const int nr = (int)g.idx.size();
  mpi_status st = MPI_OK;
  if (kind & MPI_BATCH_FORWARD) {
    st = expand_rows(ctx, s0.plan, s0.basis, EX_FWD, rows + g.fwd_rows, nr, g.Cmax, prec, g.row_ctas);
    long off = 0;
    for (int i = 0; i < nr && st == MPI_OK; ++i) {
      const mpi_batch_slice& s = sl[g.idx[i]];
      st = plan_image_to_kspace(ctx, s.plan, buf + off * N, s.C, (float2*)s.y);
      off += s.C;
    }
  }
  if (st == MPI_OK && (kind & MPI_BATCH_ADJOINT)) {
    long off = 0;
    for (int i = 0; i < nr && st == MPI_OK; ++i) {
      const mpi_batch_slice& s = sl[g.idx[i]];
      st = plan_kspace_to_image(ctx, s.plan, (const float2*)s.y, s.C, buf + off * N);
      off += s.C;
    }
    if (st == MPI_OK) st = expand_rows(ctx, s0.plan, s0.basis, EX_ADJ, rows + g.adj_rows, nr, g.Cmax, prec, g.row_ctas);
  }
  return st;
}

// CTAs per row for a group's expansion: every candidate timed over three
// launches of the group's forward expansion (between events on the context's
// stream, after one warm-up launch), the fastest kept.
mpi_status tune_group(mpi_ctx* ctx, const mpi_batch_slice* sl, Group& g, mpi_precision prec,
                      const ExpandRow* rows) {
  const mpi_batch_slice& s0 = sl[g.idx[0]];
  const int nr = (int)g.idx.size();
  const int sms = std::max(ctx->num_sms, 1);
  std::vector<int> cands;
  for (int c : {std::max(1, sms / nr), std::max(1, 2 * sms / nr), std::max(1, sms / (2 * nr))})
    if (std::find(cands.begin(), cands.end(), c) == cands.end()) cands.push_back(c);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, MPI_ERR_CUDA, "grouped batch: tuning events");
  }
  std::string rec = std::string("grouped expansion (") + std::to_string(nr) + " slices, N=" +
                    std::to_string(s0.plan->N) + ", q=" + std::to_string(s0.basis->q) + ", sumC=" +
                    std::to_string(g.sumC) + ", " + (prec == MPI_PREC_BF16 ? "bf16" : "fp32") + "):";
  float best = 1e30f;
  int pick = cands[0];
  mpi_status st = MPI_OK;
  for (int c : cands) {
    st = expand_rows(ctx, s0.plan, s0.basis, EX_FWD, rows + g.fwd_rows, nr, g.Cmax, prec, c);
    if (st) break;
    cudaEventRecord(e0, ctx->stream);
    for (int r = 0; r < 3 && st == MPI_OK; ++r)
      st = expand_rows(ctx, s0.plan, s0.basis, EX_FWD, rows + g.fwd_rows, nr, g.Cmax, prec, c);
    cudaEventRecord(e1, ctx->stream);
    if (st) break;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      st = cuda_check(ctx, cudaGetLastError(), "grouped batch tuning");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    char buf[64];
    snprintf(buf, sizeof(buf), " %d CTAs/row %.2f us;", c, ms / 3 * 1e3);
    rec += buf;
    if (ms < best) {
      best = ms;
      pick = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st) return st;
  g.row_ctas = pick;
  mpi_ctx::TuneRecord tr{};
  tr.key[0] = -1;  // not a line-pass record
  tr.choice = pick;
  char buf[64];
  snprintf(buf, sizeof(buf), " chose %d (%.2f us)", pick, best / 3 * 1e3);
  tr.what = rec + buf;
  ctx->tuned.push_back(tr);
  return MPI_OK;
}

}  // namespace

extern "C" mpi_status mpi_batch_create(mpi_ctx* ctx, const mpi_batch_slice* slices, int n, int kind,
                                       mpi_precision prec, mpi_batch** out) {
  if (!ctx) return MPI_ERR_ARG;
  if (!slices || n < 1 || !out || kind < 1 || kind > 3) return set_err(ctx, MPI_ERR_ARG, "batch: bad argument");
  *out = nullptr;
  cudaSetDevice(ctx->device);
  for (int i = 0; i < n; ++i) {
    const mpi_batch_slice& s = slices[i];
    if (!s.plan || !s.basis || !s.alpha || s.C < 1 || !s.p || !s.x || (s.plan->M > 0 && !s.y))
      return set_err(ctx, MPI_ERR_ARG, "batch: incomplete slice " + std::to_string(i));
    // reserve the workspace outside the capture (no allocation may happen inside it)
    mpi_status st = mpi_ctx_reserve(ctx, s.plan, s.basis, s.C);
    if (st) return st;
  }
  // tune the slices' FFT line passes now: no tuning happens inside the capture
  for (int i = 0; i < n; ++i) {
    mpi_status st = mpi_ctx_reserve(ctx, slices[i].plan, slices[i].basis, slices[i].C);
    if (st == MPI_OK) st = tune_line_passes(ctx, slices[i].plan, slices[i].C);
    if (st) return st;
  }
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return slices[a].basis < slices[b].basis; });

  // groups: runs of groupable slices on one basis (and one grid); the rest alone
  std::vector<Group> groups;
  std::vector<int> solo;
  std::vector<std::pair<int, int>> seq;  // recording order: (0, group) or (1, slice)
  for (int i = 0; i < n;) {
    int j = i;
    const mpi_batch_slice& a = slices[order[i]];
    while (j < n && slices[order[j]].basis == a.basis && groupable(slices[order[j]], prec) && groupable(a, prec) &&
           slices[order[j]].plan->N == a.plan->N && slices[order[j]].plan->nx == a.plan->nx)
      ++j;
    if (j - i >= 2) {
      Group g;
      for (int k = i; k < j; ++k) {
        g.idx.push_back(order[k]);
        g.Cmax = std::max(g.Cmax, slices[order[k]].C);
        g.sumC += slices[order[k]].C;
      }
      if (rows_supported(a.basis, g.Cmax, prec)) {
        seq.push_back({0, (int)groups.size()});
        groups.push_back(g);
        i = j;
        continue;
      }
    }
    seq.push_back({1, order[i]});
    ++i;
  }

  mpi_batch* bt = new mpi_batch();
  bt->ctx = ctx;
  bt->n = n;
  bt->groups = (int)groups.size();
  // the group buffer and the row tables
  size_t buf_elems = 0, nrows = 0;
  for (Group& g : groups) {
    buf_elems = std::max(buf_elems, (size_t)g.sumC * slices[g.idx[0]].plan->N);
    g.fwd_rows = nrows;
    g.adj_rows = nrows + g.idx.size();
    nrows += 2 * g.idx.size();
  }
  cudaError_t e = cudaSuccess;
  if (!groups.empty()) {
    e = cudaMalloc(&bt->buf, buf_elems * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&bt->rows, nrows * sizeof(ExpandRow));
    if (e != cudaSuccess) {
      cudaGetLastError();
      mpi_batch_destroy(bt);
      return set_err(ctx, MPI_ERR_OOM, "batch: group buffers");
    }
    std::vector<ExpandRow> host(nrows);
    float2* buf = (float2*)bt->buf;
    for (const Group& g : groups) {
      long off = 0;
      const long N = slices[g.idx[0]].plan->N;
      for (size_t r = 0; r < g.idx.size(); ++r) {
        const mpi_batch_slice& s = slices[g.idx[r]];
        host[g.fwd_rows + r] = ExpandRow{(const float2*)s.alpha, (const float2*)s.p, nullptr, buf + off * N, s.C, 0};
        host[g.adj_rows + r] = ExpandRow{(const float2*)s.alpha, nullptr, buf + off * N, (float2*)s.x, s.C, 0};
        off += s.C;
      }
    }
    e = cudaMemcpy(bt->rows, host.data(), nrows * sizeof(ExpandRow), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      mpi_status st = cuda_check(ctx, e, "batch: row tables");
      mpi_batch_destroy(bt);
      return st;
    }
    for (Group& g : groups) {
      mpi_status st = tune_group(ctx, slices, g, prec, (const ExpandRow*)bt->rows);
      if (st) {
        mpi_batch_destroy(bt);
        return st;
      }
    }
  }

  cudaStream_t cap = nullptr, user = ctx->stream;
  e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    mpi_batch_destroy(bt);
    return cuda_check(ctx, e, "batch stream");
  }
  // the capture must not wait on work still queued on the user's stream
  e = cudaStreamSynchronize(user);
  const bool prof = ctx->profiling;
  ctx->profiling = false;
  ctx->stream = cap;
  const int64_t l0 = ctx->launches;
  mpi_status st = MPI_OK;
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    for (size_t i = 0; i < seq.size() && st == MPI_OK; ++i) {
      if (seq[i].first == 0)
        st = record_group(ctx, slices, groups[seq[i].second], kind, prec, (const ExpandRow*)bt->rows,
                          (float2*)bt->buf);
      else
        st = record_slice(ctx, slices[seq[i].second], kind, prec);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cap, &g);
    if (st == MPI_OK && e2 == cudaSuccess) {
      bt->graph = g;
      e2 = cudaGraphInstantiate(&bt->exec, g, 0);
    } else if (g) {
      cudaGraphDestroy(g);
    }
    if (st == MPI_OK && e2 != cudaSuccess) st = cuda_check(ctx, e2, "batch graph capture");
  } else {
    st = cuda_check(ctx, e, "batch capture begin");
  }
  bt->kernels = ctx->launches - l0;
  ctx->launches = l0;
  ctx->stream = user;
  ctx->profiling = prof;
  cudaStreamDestroy(cap);
  if (st != MPI_OK) {
    mpi_batch_destroy(bt);
    return st;
  }
  ctx_adopt(ctx, &bt->ctx);
  *out = bt;
  return MPI_OK;
}

extern "C" mpi_status mpi_batch_run(mpi_ctx* ctx, mpi_batch* bt) {
  if (!ctx) return MPI_ERR_ARG;
  if (!bt || bt->ctx != ctx || !bt->exec) return set_err(ctx, MPI_ERR_ARG, "batch: bad handle");
  cudaSetDevice(ctx->device);
  cudaError_t e = cudaGraphLaunch(bt->exec, ctx->stream);
  if (e != cudaSuccess) return cuda_check(ctx, e, "batch graph launch");
  ctx->launches += bt->kernels;
  return MPI_OK;
}

extern "C" int64_t mpi_batch_kernel_count(const mpi_batch* bt) { return bt ? bt->kernels : -1; }

extern "C" int mpi_batch_group_count(const mpi_batch* bt) { return bt ? bt->groups : -1; }

extern "C" mpi_status mpi_batch_destroy(mpi_batch* bt) {
  if (!bt) return MPI_ERR_ARG;
  if (bt->ctx && (bt->buf || bt->rows)) cudaStreamSynchronize(bt->ctx->stream);  // a replay may still run
  ctx_release(&bt->ctx);
  if (bt->exec) cudaGraphExecDestroy(bt->exec);
  if (bt->graph) cudaGraphDestroy(bt->graph);
  if (bt->buf) cudaFree(bt->buf);
  if (bt->rows) cudaFree(bt->rows);
  delete bt;
  return MPI_OK;
}
