// Internal declarations shared by the CUDA translation units of libmpi_gb300.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "mpi_gb300.h"

// Supported FFT lengths (per axis) and the offset of each one's twiddle table
// exp(-2 pi i m / n), m < n, inside the context's table buffer.
static const int kFftLengths[] = {16, 32, 48, 64, 96, 128, 192, 256, 320, 512};
static const int kNumFftLengths = sizeof(kFftLengths) / sizeof(int);
// Bytes reserved per context for the tensor-core coefficient operand image.

// Kernel families for the optional per-launch event timing.
enum KernelFamily { KF_EXPAND = 0, KF_UHV = 1, KF_FFT_ROWS = 2, KF_FFT_LINES = 3, KF_NUFFT = 4,
                    KF_SOLVER = 5, KF_OTHER = 6, KF_COUNT = 7 };

struct mpi_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  void* work = nullptr;  // scratch between kernel passes
  size_t work_bytes = 0;
  void* stage = nullptr;  // device copies of host-buffer calls' inputs and outputs
  size_t stage_bytes = 0;
  float2* twiddles = nullptr;  // all tables back to back
  int tw_offset[kNumFftLengths] = {0};
  int num_sms = 0;
  int* dev_err = nullptr;  // device error word written by kernels whose waits time out
  void* solver_cache = nullptr;  // recorded solver graphs (solvers.cu)
  int64_t launches = 0;
  bool pdl = true;  // launch operator kernels with programmatic stream serialization
  // The `ctx` fields of the plans, bases and batches made on this context; the
  // context clears them when it is destroyed, so that destroying a child after
  // its context (in any order a caller's garbage collector picks) only frees
  // the child's own memory.
  std::vector<mpi_ctx**> children;
  std::string err;
  // profiling: event pairs around launches while enabled
  bool profiling = false;
  std::vector<cudaEvent_t> ev_begin, ev_end;
  std::vector<int> ev_family;
  std::vector<const char*> ev_name;  // kernel name of each timed launch (string literals)
  std::vector<std::pair<std::string, std::pair<double, int64_t>>> prof_kernels;  // per-name sums
  int ev_used = 0;
  int pending_family = -1;
  double prof_ms[KF_COUNT] = {0};
  int64_t prof_launches[KF_COUNT] = {0};
  // Autotuned launch shapes (fft.cu): one record per pass shape, with the
  // candidates' measured times.  Tuning runs on `tune_scratch` (a workspace
  // buffer the operator calls are not using at that point), never while the
  // stream is being captured, and only while `autotune` is set.
  bool autotune = true;
  int line_kernel = 0;  // fixed line-pass choice (8, 16, 32 lines, -1 register two-step), 0 = tuned
  bool plane_pass = true;  // 3D: the passes along y and x in one kernel per plane where it applies
  bool plane_pipe = true;  // ... as the pipelined persistent kernel (TMA tiles) where it applies
  long long wait_cycles = 4LL << 30;  // bounded-wait limit of the tensor-core kernels (SM clock cycles)
  int stall_after = -1;               // fault injection in the 3xTF32 expansion's producer (-1: off)
  int tf32_read = MPI_TF32_READ_FAILED;  // the tensor core's reading of FP32 kind::tf32 operands (probed)
  bool tf32x3 = false;                   // 3xTF32 kernels on (only with the truncating reading)
  void* tune_scratch = nullptr;
  size_t tune_scratch_bytes = 0;
  struct TuneRecord {
    long key[10];
    int choice;
    int n;
    int cand[4];
    float us[4];
    std::string what;
  };
  std::vector<TuneRecord> tuned;
};

struct mpi_plan {
  mpi_ctx* ctx = nullptr;
  int device = 0;
  int ndim = 2;
  int nz = 1, ny = 0, nx = 0;
  int N = 0;
  int kind = MPI_TRAJ_CARTESIAN;
  int M = 0;
  // Cartesian: sorted sample list and, per k-space row (nz * ny rows of nx), the
  // first sample of that row (rows + 1 entries).
  int32_t* idx = nullptr;
  int32_t* row_ptr = nullptr;
  uint8_t* row_has = nullptr;  // [n_rows]: 1 where the k-space row has samples; null when every row has some
  int n_rows = 0;
  // 3D: per kz plane, its k-space rows with samples in order of ky:
  // plane_rows [nz][max(plane_kmax, 1)] = {ky, first sample, end of samples, 0}
  // (unused entries ky = -1), plane_nrows [nz] their number, plane_slot
  // [nz][ny] each row's position in its plane's list (-1: no samples).
  int4* plane_rows = nullptr;
  int32_t* plane_nrows = nullptr;
  int16_t* plane_slot = nullptr;
  int plane_kmax = 0;
  // Radial (Kaiser-Bessel gridding)
  int W = 0, G = 0;
  float* traj = nullptr;      // [M][2]
  int32_t* gstart = nullptr;  // [M][2] first tap, array index in [0, G)
  float* gw = nullptr;        // [M][2][W] separable kernel weights
  float* deap = nullptr;      // [n] 1 / Phi(t), t = j - n/2
  // Spreading index: the samples in order of their first-tap cell sy * G + sx
  // (stable in m; cell_rank [M] gives each sample's position), CSR offsets per
  // cell (cell_ptr [G * G + 1]), each sorted sample's sx (cell_sx [M]) and
  // weights (cell_w [M][2][W]), and the cells whose W x W window holds many
  // samples (cell_dense [n_dense], spread one warp per cell).
  int32_t* cell_ptr = nullptr;
  int32_t* cell_rank = nullptr;
  int32_t* cell_sx = nullptr;
  float* cell_w = nullptr;
  int32_t* cell_dense = nullptr;
  int n_dense = 0;
  // Interpolation work list: the samples sorted by the 32 x 32 tile of their
  // first tap (tile_samples [M]); items [n_tile_items][3] = (tile, first
  // sorted sample, count), dense tiles split into chunks.
  int32_t* tile_items = nullptr;
  int32_t* tile_samples = nullptr;
  int n_tile_items = 0;
};

struct mpi_basis {
  mpi_ctx* ctx = nullptr;
  int device = 0;
  int N = 0, q = 0;
  float2* U = nullptr;  // [q][N] FP32 complex
  __nv_bfloat16* Ubf = nullptr;  // BF16 operand copy [N][Kp] (tensor-core path)
  size_t Ubf_bytes = 0;
  int Kp = 0;                    // padded K = round_up(2 q, 64)
  void* tmap = nullptr;          // CUtensorMap of Ubf (owned)
  float* Uf32 = nullptr;         // FP32 operand copy [N][Kp32] (3xTF32 tensor-core path)
  int Kp32 = 0;                  // padded K: round_up(2 q, 64) for a basis, round_up(2 q, 32) for a chain operand view
  void* tmap32 = nullptr;        // CUtensorMap of Uf32 (owned)
  // U^H V on the tensor cores (tc_uh.cu): tensor maps of the interleaved view
  // [q][2N] of U (FP32, in place) and of its BF16 copy Uview_bf
  void* umap32 = nullptr;
  void* umap_bf = nullptr;
  void* Uview_bf = nullptr;
  std::string bf16_err;          // why the BF16 copy is missing, if it is
  // Tucker-factored basis (3D): N = n1 n2 n3; the core (r1 r2 r3 x q) is held
  // as an internal dense basis `core`; factors F[k] = U_k [n_k][r_k].
  bool tucker = false;
  int n[3] = {0, 0, 0}, r[3] = {0, 0, 0};
  float2* F[3] = {nullptr, nullptr, nullptr};
  float2* Fh[3] = {nullptr, nullptr, nullptr};  // U_k^H [r_k][n_k] (the conjugate products' coefficient rows)
  mpi_basis* core = nullptr;
  // Tensor map of the flattened x1 operand in the workspace (tucker.cu), kept
  // while the workspace address, coil count and precision stay the same.
  void* op_map = nullptr;
  const void* op_map_ptr = nullptr;
  int op_map_C = -1, op_map_prec = -1;
  void* chain_maps = nullptr;  // tensor maps of the FP32 tensor-core mode-product chain (tucker.cu)
};

// ------------------------------------------------------------------ helpers

mpi_status set_err(mpi_ctx* ctx, mpi_status st, const std::string& msg);
mpi_status cuda_check(mpi_ctx* ctx, cudaError_t e, const char* what);
// Make sure ctx->work holds at least `bytes`; grows (after a stream sync) if needed.
mpi_status ensure_work(mpi_ctx* ctx, size_t bytes);
const float2* twiddle_table(const mpi_ctx* ctx, int n);
bool fft_length_supported(int n);

// Record the start event of the next launch (when profiling is on).
void prof_begin(mpi_ctx* ctx, int family);
// Record the end event of the launch just issued (`name`: the kernel's name,
// a string literal, for the per-kernel sums).
void prof_end(mpi_ctx* ctx, const char* name = nullptr);

#define MPI_PROF(ctx, fam) prof_begin((ctx), (fam))

// Launches `kern` on the context's stream with programmatic stream
// serialization, so that its launch and its prologue overlap the tail of the
// previous kernel.  Every kernel launched this way calls mpi_ptx::pdl_wait()
// before touching global data that earlier stream work reads or writes.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(mpi_ctx* ctx, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              Args&&... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = ctx->stream;
  cfg.attrs = attr;
  cfg.numAttrs = ctx->pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

#define MPI_LAUNCH_CHECK(ctx, what)                                   \
  do {                                                                \
    (ctx)->launches++;                                                \
    prof_end((ctx), (what));                                          \
    cudaError_t e__ = cudaGetLastError();                             \
    if (e__ != cudaSuccess) return cuda_check((ctx), e__, (what));    \
  } while (0)

// ------------------------------------------------------- expansion kernels

enum ExpandMode { EX_MAPS = 0, EX_FWD = 1, EX_JFWD = 2, EX_ADJ = 3, EX_JADJ = 4, EX_SCATTER = 5, EX_SCATTER_ADD = 6 };

// EX_SCATTER (3xTF32 kernel): the real and imaginary parts of output (row n,
// column pair j) go to the FP32 array `out` at
//   (n / (L0 L1)) s_hi + ((n / L0) % L1) s_mid + n % L0 + j s_col   and  + im,
// which writes a product straight into the real-ified K-major operand layout
// the next contraction streams (the Tucker mode-product chain).
struct ScatterMap {
  int L0 = 1, L1 = 1;
  long s_hi = 0, s_mid = 0, s_col = 0;
  int im = 0;
  bool bf16 = false;  // write BF16 values (the same element offsets) instead of FP32
};

// One row of a grouped expansion launch (grid row blockIdx.y): a slice that
// shares the basis, with its own coefficients, image, per-coil data and output.
struct ExpandRow {
  const float2* alpha;
  const float2* p;
  const float2* w;
  float2* out;
  int C;
  int pad;
};

struct ExpandArgs {
  const float2* U = nullptr;  // [q][N]
  int N = 0, q = 0;
  int nx = 1, ny = 1;          // grid, for the (-1)^(x+y+z) centring sign
  int centre = 0;              // apply the centring sign
  float scale = 1.f;           // N^{-1/2} (and the n/2-odd sign) for F_s
  const float2* alpha = nullptr;   // [C][q]
  const float2* dalpha = nullptr;  // [C][q] (Jacobian)
  int C = 0;
  const float2* p = nullptr;   // [N]
  const float2* dp = nullptr;  // [N]
  const float2* w = nullptr;   // [C][N] adjoint input (after inverse FFT passes)
  float2* out = nullptr;       // maps / v [C][N], or image [N]
  float2* vout = nullptr;      // Jacobian adjoint: conj(p) w [C][N]
  int* err = nullptr;          // device error word (bounded-wait timeouts)
  // Maps-mode output remap for a flattened Tucker operand (tensor-core kernels
  // only): pixel n = c B + b of coil row i goes to out[c tuck_stride + i B + b].
  int tuck_B = 0;
  long tuck_stride = 0;
  const char* kname = nullptr;  // name of the launch in the per-kernel timing (default: the kernel's)
  ScatterMap sc;                // EX_SCATTER output map
  int accumulate = 0;           // EX_FWD / EX_JFWD: add into out instead of storing (several sets of maps)
  // Grouped launch (tensor-core kernels): device table of nrows rows, C = the
  // largest row's coil count; row_ctas CTAs per row (0: the SMs shared out).
  const ExpandRow* rows = nullptr;
  int nrows = 0;
  int row_ctas = 0;
  // 3xTF32 EX_SCATTER_ADD: split K into this many parts (grid rows, >= 2), each
  // adding its partial products into `out` (scattered as EX_SCATTER), which the
  // caller has zeroed
  int ksplit = 0;
};

mpi_status launch_expand(mpi_ctx* ctx, int mode, const ExpandArgs& a);
// Precision dispatch over the FFMA, 3xTF32 and BF16 expansion kernels.
mpi_status expand(mpi_ctx* ctx, const mpi_basis* basis, int mode, const ExpandArgs& a, mpi_precision prec);
// Child bookkeeping (see mpi_ctx::children).
void ctx_adopt(mpi_ctx* ctx, mpi_ctx** slot);
void ctx_release(mpi_ctx** slot);
// BF16 tensor-core expansion (tcgen05); same modes and arguments.
mpi_status launch_expand_tc(mpi_ctx* ctx, const mpi_basis* b, int mode, const ExpandArgs& a);
mpi_status tc_basis_prepare(mpi_ctx* ctx, mpi_basis* b);
void tc_basis_release(mpi_basis* b);
// FP32-accurate tensor-core expansion (3xTF32); same modes and arguments.
// With group_coils > 0 (< C), one launch runs the coils in groups of that size
// (grid rows), each row streaming the same basis tiles in step.
mpi_status launch_expand_tf32(mpi_ctx* ctx, const mpi_basis* b, int mode, const ExpandArgs& a, int group_coils = 0);
bool tf32_supported(const mpi_basis* b, int mode, int C);
// Whether the 3xTF32 scatter expansion of all C coils fits one launch with K split in `ksplit` parts.
bool tf32_ksplit_supported(const mpi_basis* b, int mode, int C, int ksplit);
// Measures how the tensor core reads an FP32 operand of kind::tf32 (one MMA on
// the context's stream, synchronised); returns an MPI_TF32_READ_* value.
int tf32_reading_probe(mpi_ctx* ctx);
// Coils per launch of the 3xTF32 kernel: C when the whole call fits, else the
// largest group that fits (forward-type modes only), or 0.
int tf32_group(const mpi_basis* b, int mode, int C);
mpi_status tf32_basis_prepare(mpi_ctx* ctx, mpi_basis* b);
void tf32_basis_release(mpi_basis* b);
// Tensor maps of a K-major operand [rows][Kp] (BF16 or FP32) laid out as the
// tensor-core kernels read their basis copies; `map` is a CUtensorMap.
bool tc_encode_operand_map(void* map, void* ptr, long rows, int Kp);
// BF16 operand rows of K values (K a multiple of 8) read as 64-element boxes;
// columns past K read as zeros.
bool tc_encode_operand_map_k(void* map, void* ptr, long rows, int K);
bool tf32_encode_operand_map(void* map, void* ptr, long rows, int Kp);
// FP32 operand of `rows` rows of K (a multiple of 4) values, read by the 3xTF32
// kernel as Kp = round_up(K, 64) columns (the rest zero-filled by the copy engine).
bool tf32_encode_operand_map_k(void* map, void* ptr, long rows, int K);
// dalpha[c][j] = sum_n conj(U[j][n]) V[c][n]; partials in `work_partials`.
mpi_status launch_uh_v(mpi_ctx* ctx, const float2* U, int N, int q, const float2* V, int C,
                       float2* dalpha, float2* work_partials, size_t partial_cap_elems);
size_t uh_v_partial_elems(const mpi_ctx* ctx, int N, int q, int C);
// dalpha_c = U^H V_c on the tensor cores (3xTF32 for FP32, BF16 for BF16);
// V is [C][N] complex.  Prepared at basis load (tensor maps, the BF16 view).
mpi_status uh_tc_prepare(mpi_ctx* ctx, mpi_basis* b);
void uh_tc_release(mpi_basis* b);
bool uh_tc_supported(const mpi_basis* b, mpi_precision prec);
size_t uh_tc_partial_elems(const mpi_ctx* ctx, int N, int q, int C);
mpi_status launch_uh_tc(mpi_ctx* ctx, const mpi_basis* b, const float2* V, int C, float2* dalpha,
                        float2* partials, size_t partial_cap, mpi_precision prec);
// One-sided Jacobi SVD of the nj (even) columns of an FP64 L x nj column-major
// matrix M (maxwell.cu): rotations accumulated into V (nj x nj), final column
// norms (the singular values, column order) into sig_host.
mpi_status jacobi_columns(mpi_ctx* ctx, double2* M, int L, int nj, double2* V, double* sig_dev, int* flag,
                          std::vector<double>& sig_host, const char* what);
// core [q][r1][r2][r3] = T x1 U1^H x2 U2^H x3 U3^H for a dense tensor T
// [q][n1][n2][n3] and factors F_k [n_k][r_k] (tucker.cu, FP32 mode products);
// tmp holds q r1 (n2 n3 + r2 n3) complex values.
mpi_status tucker_project(mpi_ctx* ctx, const float2* T, int q, const int n[3], const int r[3], const float2* F0,
                          const float2* F1, const float2* F2, float2* core, float2* tmp);
// Grouped batch pieces (api.cu): one expansion launch over the rows of slices
// that share `basis` (grid geometry from plan0), and a Cartesian plan's
// image -> k-space / k-space -> image passes on a caller buffer.
mpi_status expand_rows(mpi_ctx* ctx, const mpi_plan* plan0, const mpi_basis* basis, int mode, const ExpandRow* rows,
                       int nrows, int Cmax, mpi_precision prec, int row_ctas);
bool rows_supported(const mpi_basis* basis, int Cmax, mpi_precision prec);
mpi_status plan_image_to_kspace(mpi_ctx* ctx, const mpi_plan* plan, float2* v, int C, float2* y);
mpi_status plan_kspace_to_image(mpi_ctx* ctx, const mpi_plan* plan, const float2* y, int C, float2* w);
// U^H V on the tensor cores where the basis and precision allow, else on the CUDA cores.
mpi_status uh_v(mpi_ctx* ctx, const mpi_basis* b, const float2* V, int C, float2* dalpha, float2* partials,
                size_t partial_cap, mpi_precision prec);

// Tucker basis: per-coil maps, the adjoint contraction, point-wise epilogues.
size_t tucker_work_elems(const mpi_basis* b, int C);
mpi_status tucker_maps(mpi_ctx* ctx, const mpi_basis* b, const float2* alpha, int C, float2* maps, float2* tmp,
                       mpi_precision prec);
// The forward pass of a Tucker basis with the last mode product fused with the
// point-wise step (no per-coil maps stored); tucker_fusable says which modes.
bool tucker_fusable(int mode);
// Whether the x1 mode product of this basis runs on the tensor-core kernels.
bool tucker_x1_on_tensor_cores(const mpi_basis* b, int C, mpi_precision prec);
mpi_status tucker_fused(mpi_ctx* ctx, const mpi_basis* b, int mode, const ExpandArgs& a, float2* tmp,
                        mpi_precision prec);
mpi_status tucker_adjoint(mpi_ctx* ctx, const mpi_basis* b, const float2* V, int C, float2* dalpha, float2* tmp,
                          float2* partials, size_t partial_cap, mpi_precision prec);
mpi_status launch_pointwise(mpi_ctx* ctx, int mode, const ExpandArgs& a, const float2* S, const float2* dS);
void tucker_chain_release(mpi_basis* b);
bool tucker_chain_on_tensor_cores(const mpi_basis* b, int C);
// The flattened x1 operand of alpha's maps and its tensor map (see tucker.cu).
mpi_status tucker_x1_operand(mpi_ctx* ctx, const mpi_basis* b, const float2* alpha, int C, float2* tmp,
                             mpi_precision prec, void** op_out, void** map_out);
// The x1 product on the tensor cores fused with the forward's point-wise step
// and DFT along z (out = vhat [C][n1][n2 n3]), or with the inverse DFT along z
// of `wk` [C][n1][n2 n3] and the adjoint's sum over coils of conj(s_c) w_c
// (out = image [N]) (tc_tucker.cu).
bool tucker_x1_fused_supported(const mpi_basis* b, const mpi_plan* plan, int C, mpi_precision prec);
// Tucker: Fh[k] = U_k^H, made at basis load.
mpi_status tucker_conj_factors(mpi_ctx* ctx, mpi_basis* b);
// The Jacobian-adjoint's coefficient block on the tensor cores (FP32): from the
// per-coil data after the inverse passes along x and y.
bool tucker_jadj_tc_supported(const mpi_basis* b, const mpi_plan* plan, int C, mpi_precision prec);
mpi_status tucker_jadj_alpha(mpi_ctx* ctx, const mpi_basis* b, const mpi_plan* plan, const float2* wk,
                             const float2* p, float scale, int C, float2* opbuf, float2* dalpha, float2* tmp,
                             float2* partials, size_t partial_cap);
mpi_status tucker_x1_fused_launch(mpi_ctx* ctx, const mpi_basis* b, const mpi_plan* plan, bool adjoint, int C,
                                  const void* map, const float2* p, const float2* wk, float2* out, float scale,
                                  mpi_precision prec, bool accumulate = false);

// Loads the module holding the allocation-free forward's static scratch on the
// current device (noalloc.cu); called once per context at creation.
cudaError_t noalloc_preload();

// Drop recorded solver graphs that reference `object` (a plan or basis), or all of them.
void solver_cache_forget(mpi_ctx* ctx, const void* object);
void solver_cache_clear(mpi_ctx* ctx);

// ------------------------------------------------------------ FFT passes

// In-place FFT along the y axis of `data` [C][nz][ny][nx] (unnormalised).
// With row_has ([nz][ny], 1 where the k-space row has samples): inverse, rows
// without samples are read as zeros (the adjoint's row pass does not write
// them); forward, only rows with samples are stored (the row pass reads no
// other row).
mpi_status launch_fft_cols(mpi_ctx* ctx, float2* data, int C, int nz, int ny, int nx, bool inverse,
                           const uint8_t* row_has = nullptr);
// FFT along y over the oversampled radial grid [C][G][G] with the centred
// n x n window folded in: forward reads the image src [C][n][n] (padding,
// deapodisation and sign on the fly); inverse writes only the window into dst.
mpi_status launch_fft_cols_window(mpi_ctx* ctx, float2* grid, int C, int G, const float2* src, float2* dst,
                                  const float* deap, int n, bool inverse);
// Tunes the line passes the operators run on this plan with C coils (in the
// workspace, which must already hold them) so that a stream capture that
// follows records the tuned kernels.
mpi_status tune_line_passes(mpi_ctx* ctx, const mpi_plan* plan, int C);
// The passes along y and x of every (coil, kz) plane of a 3D volume in one
// kernel (plane in shared memory): forward, data [C][nz][ny][nx] (already
// transformed along z) -> samples y; inverse, samples -> data (to be
// transformed along z).  Planes of 64 / 96 / 128 squared.
bool plane_pass_supported(const mpi_plan* plan);
// The passes along y and x of the (coil, kz) planes: the pipelined kernel where
// ctx->plane_pipe is set and it applies, else one CTA per plane.
mpi_status launch_plane_yx(mpi_ctx* ctx, const mpi_plan* plan, float2* data, int C, float2* y, bool inverse);
// In-place FFT along z of [C][nz][ny][nx].
mpi_status launch_fft_z(mpi_ctx* ctx, float2* data, int C, int nz, int ny, int nx, bool inverse);
// Forward: FFT along x of every row, centring sign on k, gather of the sampled points.
mpi_status launch_rows_fwd_gather(mpi_ctx* ctx, const mpi_plan* plan, const float2* data, int C,
                                  float2* y);
// Adjoint: zero-fill every row from the samples, centring sign, inverse FFT along x.
mpi_status launch_rows_scatter_inv(mpi_ctx* ctx, const mpi_plan* plan, const float2* y, int C,
                                   float2* data);

// ------------------------------------------------------------- NUFFT (radial)

mpi_status nufft_plan_init(mpi_ctx* ctx, mpi_plan* plan, const float* traj_host);
// Radial workspace: the C oversampled grids, then the coil-grouped sorted copy
// of the k-space samples that spreading reads.
size_t nufft_grid_elems(const mpi_plan* plan, int C);
mpi_status nufft_forward(mpi_ctx* ctx, const mpi_plan* plan, const float2* img_deap_src, int C,
                         float2* y, float2* grid);
mpi_status nufft_adjoint(mpi_ctx* ctx, const mpi_plan* plan, const float2* y, int C,
                         float2* img_out, float2* grid);
