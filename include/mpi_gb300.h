/*
 * mpi_gb300.h -- C ABI of the GB300 (sm_103a) Maxwell Parallel Imaging encoding operator.
 *
 * Operator (Theory, "Regularized Nonlinear Inversion", Eq. 5):
 *   G(p, alpha_1..alpha_C) = [ F_s( (U alpha_k) (.) p ) ]_{k=1..C}
 * with p in C^N the image, U in C^{N x q} the Maxwell basis, alpha_k in C^q the
 * coefficients of coil k, (.) the element-wise product and F_s in C^{M x N} the
 * undersampled Fourier operator of one coil (Eq. 1: F = I_C (x) F_s).
 *
 * Conventions shared by every call
 *   - complex numbers are interleaved float pairs (mpi_c32, 8 bytes);
 *   - arrays are C order: p [N] raster (x fastest, then y, then z), alpha [C][q],
 *     maps [C][N], k-space data y [C][M];
 *   - F_s is the centred unitary DFT (forward sign e^{-i}, index origin at n/2 on
 *     every axis, scale N^{-1/2}) followed by selection of the sampled points;
 *     for radial sampling it is the Kaiser-Bessel gridding NUFFT of the same
 *     non-uniform DFT;
 *   - pointers named in "device" are caller-owned device memory; the library never
 *     frees them, never keeps them after the call returns, overwrites outputs
 *     (never accumulates) and enqueues all work on the context's stream without
 *     synchronising (results are ready when that stream is);
 *   - every call checks its arguments before launching anything and returns
 *     MPI_ERR_ARG / MPI_ERR_SHAPE without side effects on a bad argument;
 *     CUDA failures return MPI_ERR_CUDA; mpi_last_error() gives the text;
 *   - a context is not thread-safe; distinct contexts are independent.
 */
#ifndef MPI_GB300_H
#define MPI_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { float x, y; } mpi_c32;
typedef struct { double x, y; } mpi_c64;

typedef enum {
  MPI_OK = 0,
  MPI_ERR_ARG = 1,
  MPI_ERR_SHAPE = 2,
  MPI_ERR_CUDA = 3,
  MPI_ERR_OOM = 4,
  MPI_ERR_NOT_CONVERGED = 5,
  MPI_ERR_TIMEOUT = 6,
  MPI_ERR_UNSUPPORTED = 7
} mpi_status;

typedef enum { MPI_TRAJ_CARTESIAN = 0, MPI_TRAJ_RADIAL = 1 } mpi_traj_kind;

/* Arithmetic of the basis expansion U alpha (the only dense contraction).
 * FP32: FP32 in and out at FP32 accuracy; on the tensor cores as three TF32
 * products per term (hi*hi + hi*lo + lo*hi of the split operands, FP32
 * accumulation) where the coefficient operand fits the kernel's shared-memory
 * budget (2 C <= 256, or 4 C <= 256 for the Jacobian, and 2 q <= 256 or so),
 * else on the CUDA cores.  BF16: tensor cores, BF16 basis and coefficients,
 * FP32 accumulation.  FP32_SIMT: always the CUDA-core FFMA kernel.  FFT,
 * gridding and reductions are FP32 in all three.
 * MIXED (the solvers only): BF16 operators inside the CG iterations, FP32 for
 * the outer residuals and the right-hand sides (IRGN: r = y - G(x) and
 * J^H r - 2 L x of every Gauss-Newton step; ADMM: A p, the right-hand side and
 * each p-update's starting residual), so the outer iterations refine the
 * solution against FP32 residuals; operator calls reject it. */
typedef enum { MPI_PREC_FP32 = 0, MPI_PREC_BF16 = 1, MPI_PREC_FP32_SIMT = 2, MPI_PREC_MIXED = 3 } mpi_precision;

typedef struct mpi_ctx mpi_ctx;
typedef struct mpi_plan mpi_plan;
typedef struct mpi_basis mpi_basis;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`, enqueueing on `cuda_stream`
 * (a cudaStream_t; NULL = legacy default stream).  The context owns a growable
 * device workspace (scratch between kernel passes); it grows on a call that
 * needs more, which synchronises the stream once -- call mpi_ctx_reserve first
 * to size it up front. */
mpi_status mpi_ctx_create(mpi_ctx** out, int device, void* cuda_stream);
mpi_status mpi_ctx_destroy(mpi_ctx* ctx);
mpi_status mpi_ctx_set_stream(mpi_ctx* ctx, void* cuda_stream);
/* Wait for the context's stream, then read the context's device error word:
 * a kernel whose bounded barrier wait ran out sets it (and exits early), in
 * which case this returns MPI_ERR_TIMEOUT and clears the word. */
mpi_status mpi_ctx_synchronize(mpi_ctx* ctx);
/* Size the workspace for operator calls with `C` coils on this plan and basis. */
mpi_status mpi_ctx_reserve(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis, int C);
/* Text of the last error on this context (static storage inside ctx; never NULL). */
const char* mpi_last_error(const mpi_ctx* ctx);
/* Number of kernels this context has launched since creation (for accounting). */
int64_t mpi_ctx_launch_count(const mpi_ctx* ctx);
/* Bytes of device memory the context currently holds for its growable workspace
 * and host-call staging buffer (0 until an operator call or mpi_ctx_reserve
 * grows them); -1 for a null context.  Library bookkeeping, no paper passage. */
int64_t mpi_ctx_workspace_bytes(const mpi_ctx* ctx);
/* Bounded waits.  Every mbarrier wait of the tensor-core kernels gives up after
 * `cycles` SM clock cycles (default 2^32, about 2 s at 2 GHz; at least 1000):
 * the kernel then records MPI_ERR_TIMEOUT in the context's device error word,
 * waits (bounded) for the copies it issued, frees its tensor memory and
 * returns; mpi_ctx_synchronize reports the timeout and clears the word, and the
 * context stays usable.  mpi_ctx_inject_stall(ctx, k) is a fault-injection
 * hook for testing that path: with k >= 0 the FP32 tensor-core expansion's
 * copy producer stops after k ring stages, so the waits on the stages it never
 * loads run out (the failure is made by withholding work; nothing faults);
 * k < 0 switches it off.  Library machinery, no paper passage. */
mpi_status mpi_ctx_set_wait_limit(mpi_ctx* ctx, int64_t cycles);
mpi_status mpi_ctx_inject_stall(mpi_ctx* ctx, int stages);
/* How the tensor core reads an FP32 shared-memory operand of a kind::tf32 MMA.
 * The FP32 tensor-core kernels (the 3xTF32 split x = hi(x) + lo(x) behind the
 * FP32 basis expansion of Eq. 5, its Jacobian forms of Eq. 7 and the
 * Jacobian-adjoint display after it, the Tucker mode products of Eq. 19 and
 * the coefficient block U^H v) feed each raw FP32 tile as hi(x) and add lo(x)
 * separately, which is exact only if the tensor core reads the FP32 value as
 * its upper 19 bits (truncation).  mpi_ctx_create measures the reading with
 * one MMA on 128 test values (ties, values just above and below a TF32 step,
 * both signs) and returns it here: MPI_TF32_READ_TRUNCATE (measured on GB300),
 * _NEAREST_EVEN, _NEAREST_AWAY, _FULL (all 23 bits), _OTHER, or _FAILED (the
 * probe did not run).  Only MPI_TF32_READ_TRUNCATE enables the 3xTF32 kernels;
 * any other reading sends every FP32 call to the CUDA-core FP32 kernels (the
 * paths MPI_PREC_FP32_SIMT takes, and for Tucker bases the CUDA-core mode
 * products), so FP32 results keep their accuracy on any device.  -1 for a
 * null context.  mpi_ctx_set_tf32x3(ctx, 0) switches the 3xTF32 kernels off
 * for later calls (graphs already recorded by solvers or batches keep the
 * kernels they were recorded with); (ctx, 1) switches them back on and is
 * MPI_ERR_UNSUPPORTED unless the probe found truncation.  Library machinery,
 * no paper passage. */
enum { MPI_TF32_READ_FAILED = -2, MPI_TF32_READ_TRUNCATE = 0, MPI_TF32_READ_NEAREST_EVEN = 1,
       MPI_TF32_READ_NEAREST_AWAY = 2, MPI_TF32_READ_FULL = 3, MPI_TF32_READ_OTHER = 4 };
int mpi_ctx_tf32_reading(const mpi_ctx* ctx);
mpi_status mpi_ctx_set_tf32x3(mpi_ctx* ctx, int enable);
/* Launch-shape autotuning (on by default).  The first operator call that runs an
 * FFT line pass of a new shape (length, stride, line count, row mask) times each
 * candidate tile width of that pass with CUDA events on a free workspace buffer
 * (never while the stream is being captured, never in mpi_forward_noalloc) and
 * keeps the fastest for the context's later calls.  enable = 0 switches tuning
 * off (untuned shapes take a fixed default).  mpi_ctx_tuning_record returns the
 * text of the `index`-th decision (shape, candidates and their times; valid for
 * the context's lifetime), MPI_ERR_ARG past the last.  Library machinery, no
 * paper passage. */
mpi_status mpi_ctx_set_autotune(mpi_ctx* ctx, int enable);
/* Fixes the FFT line passes' kernel instead of tuning it: 8, 16 or 32 lines per
 * CTA (shared-memory Stockham passes), -1 the register two-step pass along y
 * (lengths 64, 96, 128, 192, 256), 0 back to tuning.  A pass the choice does
 * not cover keeps its tuned or default kernel.  3D Tucker volumes with planes
 * of 64, 96 or 128 squared run the passes along y and x as one kernel over
 * the (coil, kz) planes unless the choice is -2 (separate, tuned passes): a
 * persistent kernel that streams the planes through shared memory in TMA
 * tiles where each plane's rows with samples fit beside the tiles, else, and
 * always with the choice -3, one CTA per plane.  MPI_ERR_ARG for other
 * values. */
mpi_status mpi_ctx_set_line_kernel(mpi_ctx* ctx, int choice);
mpi_status mpi_ctx_tuning_record(const mpi_ctx* ctx, int index, const char** text_out);
/* Per-launch device timing: while enabled, every kernel the context launches is
 * bracketed by two CUDA events on the context's stream (16384 launches at most
 * between reads; later ones are not timed).  mpi_ctx_profile_read synchronises
 * the stream and returns, for one kernel family, the summed device time (ms) and
 * the number of timed launches since the last reset; reset != 0 clears the sums.
 * Families: 0 basis expansion, 1 U^H V contraction, 2 row FFT passes, 3 strided
 * FFT passes, 4 NUFFT gridding, 5 solver vector kernels, 6 other. */
mpi_status mpi_ctx_profile(mpi_ctx* ctx, int enable);
mpi_status mpi_ctx_profile_read(mpi_ctx* ctx, int family, double* ms_out, int64_t* launches_out,
                                int reset);
/* Per-kernel sums of the same timing: entry `index` (0, 1, ... in order of first
 * launch) gives the kernel's name (valid until the next reset), its summed device
 * time (ms) and its timed launches since the last reset.  Synchronises the
 * stream.  MPI_ERR_ARG once `index` is past the last kernel.  Library
 * bookkeeping, no paper passage. */
mpi_status mpi_ctx_profile_kernel(mpi_ctx* ctx, int index, const char** name_out, double* ms_out,
                                  int64_t* launches_out);

/* ------------------------------------------------------------------- plan */

/* Geometry and sampling of F_s (Eq. 1).  Host pointers; the plan copies them.
 *   ndim        2 or 3
 *   dims        (nz, ny, nx); nz = 1 when ndim = 2.  Cartesian FFT axes must have
 *               lengths in {16, 32, 48, 64, 96, 128, 192, 256, 320, 512}
 *   kind        MPI_TRAJ_CARTESIAN or MPI_TRAJ_RADIAL (2D square only)
 *   M           samples per coil (M >= 0; M = 0 gives empty k-space)
 *   sample_idx  Cartesian: M strictly increasing flat indices into the centred
 *               k-space grid (raster order, same layout as the image);
 *               checked: sorted, unique, in [0, N) -- else MPI_ERR_ARG
 *   traj        radial: M x 2 floats (kx, ky) in radians per pixel, [-pi, pi)
 *   kb_width    radial: Kaiser-Bessel width W (2..8)
 *   oversamp    radial: grid oversampling sigma (grid = sigma * n, must be a
 *               supported FFT length) */
typedef struct {
  int ndim;
  int dims[3];
  int kind;
  int M;
  const int32_t* sample_idx;
  const float* traj;
  int kb_width;
  float oversamp;
} mpi_plan_desc;

mpi_status mpi_plan_create(mpi_ctx* ctx, const mpi_plan_desc* desc, mpi_plan** out);
mpi_status mpi_plan_destroy(mpi_plan* plan);
/* Radial plans: the first grid tap of every sample and axis, int32 [M][2]
 * (x, y), array index in [0, G): floor(k G / 2 pi) - W/2 + 1 + G/2 taken in FP64,
 * wrapped mod G (device pointer out). */
mpi_status mpi_plan_grid_index(mpi_ctx* ctx, const mpi_plan* plan, int32_t* out_dev);

/* ------------------------------------------------------------------ basis */

/* Dense basis U in C^{N x q} (Maxwell Regularization section: s_k ~ U alpha_k),
 * given column-major as [q][N] (basis vector j contiguous).  `U` is a host
 * pointer when on_device = 0, else a device pointer.  The basis keeps its own
 * copies (FP32, and a BF16 copy for MPI_PREC_BF16). */
mpi_status mpi_basis_load_dense(mpi_ctx* ctx, const mpi_c32* U, int N, int q, int on_device,
                                mpi_basis** out);
/* Tucker-factored basis for a 3D grid (n1, n2, n3) = (nz, ny, nx) ("A Compression
 * Scheme for Maxwell Basis", Eqs. 19-20): basis column j reshaped onto the grid
 * is G_j x1 U1 x2 U2 x3 U3, with the core G given as [q][r1][r2][r3] (the core
 * slice of column j contiguous) and factors U_k as [n_k][r_k] (row-major), all
 * complex64; host pointers when on_device = 0, else device pointers.  Limits:
 * 1 <= r_k <= min(n_k, 128), n_k <= 256, r1 r2 r3 and n1 n2 n3 multiples of 4,
 * q <= 256.  The
 * operators expand maps as (G x4 alpha_c^T) x1 U1 x2 U2 x3 U3 (the core
 * contraction in FP32 or on BF16 tensor cores, the mode products in FP32). */
mpi_status mpi_basis_load_tucker(mpi_ctx* ctx, const mpi_c32* core, const mpi_c32* U1, const mpi_c32* U2,
                                 const mpi_c32* U3, const int n[3], const int r[3], int q, int on_device,
                                 mpi_basis** out);
mpi_status mpi_basis_destroy(mpi_basis* basis);

/* Maxwell basis of a 2D slice built on the GPU (Maxwell Regularization
 * section: the dyadic Green's functions of Eqs. 17-18, the field operator of
 * Eq. 15 sampled by random boundary excitations as in Fig. 1, truncation by
 * singular value as in Eq. 16).
 *   Pixels: ny x nx centroids of a field of view fov_y x fov_x metres centred
 *   on the origin in the z = 0 plane, raster order (x fastest).
 *   Sources: n_sites points (host, double [n_sites][3], metres), each with three
 *   electric and three magnetic point dipoles (x, y, z); column 6 s + t of the
 *   field matrix B (N x 6 n_sites) is the circularly polarised field
 *   (H_x - i H_y) / sqrt(2) of dipole t of site s, with k = 2 pi f_hz / c0 and
 *   the magnetic dipoles scaled by the free-space impedance.
 *   omega: host, complex128 [6 n_sites][L] row-major, the random excitation
 *   amplitudes (row order = the column order of B).
 * Result: the q leading left singular vectors of Y = B omega, ordered by
 * singular value, as a device array U_out [q][N] complex64 (the layout
 * mpi_basis_load_dense takes; each vector's phase is arbitrary), and all
 * min(6 n_sites, L) singular values of Y in descending order into sv_out
 * (host, double).  Computed in FP64 (Householder QR of B, X = R omega, one-sided
 * Jacobi SVD of X, Q applied to the leading vectors), so subspaces with singular
 * values down to about 1e-15 sigma_1 are resolved where the gaps allow.
 * Allocates its FP64 workspace (about 16 N (6 n_sites + q) bytes) and
 * synchronises the context's stream; do not call it during stream capture.
 * Fields that are identically zero (three of the six per site when the sites
 * lie in the slice plane) are dropped with their rows of omega; they add only
 * zero singular values.
 * Errors: MPI_ERR_SHAPE unless 6 n_sites <= N and q <= min(number of nonzero
 * fields, L); MPI_ERR_OOM; MPI_ERR_CUDA if the Jacobi sweeps do not converge
 * (60 sweeps). */
mpi_status mpi_maxwell_basis_2d(mpi_ctx* ctx, int ny, int nx, double fov_y, double fov_x, double f_hz,
                                const double* sources, int n_sites, const mpi_c64* omega, int L, int q,
                                mpi_c32* U_out, double* sv_out);
/* The same for a 3D volume of nz x ny x nx voxels (fov_z x fov_y x fov_x metres,
 * centred on the origin, raster order x fastest, z slowest): U_out [q][N] with
 * N = nz ny nx is the dense basis tensor [q][nz][ny][nx] that
 * mpi_tucker_compress takes. */
mpi_status mpi_maxwell_basis_3d(mpi_ctx* ctx, int nz, int ny, int nx, double fov_z, double fov_y, double fov_x,
                                double f_hz, const double* sources, int n_sites, const mpi_c64* omega, int L, int q,
                                mpi_c32* U_out, double* sv_out);

/* Tucker compression of a dense basis on the GPU ("A Compression Scheme for
 * Maxwell Basis", Eqs. 19-21): T (device, complex64 [q][n1][n2][n3], i.e. a
 * dense basis [q][N] on an n1 x n2 x n3 grid, n1 slowest) -> a Tucker basis
 * (*out, owned by the caller, as from mpi_basis_load_tucker).  HOSVD: U_k = the
 * leading eigenvectors of the mode-k Gram matrix T_(k) T_(k)^H (formed in FP64
 * with a fixed summation order), r_k = the fewest with discarded eigenvalues
 * summing to at most eps^2 ||T||^2 / 3, core = T x1 U1^H x2 U2^H x3 U3^H (FP32).
 * Then ||T - T~|| <= bound ||T|| with bound = sqrt(sum_k tail_k) / ||T|| <= eps
 * (Eq. 21).  r3 is raised where needed to make r1 r2 r3 a multiple of 4 (the
 * Tucker basis layout); ranks_out receives the ranks used, bound_out the bound
 * for them.  Limits: n_k <= 256, q <= 256, n1 n2 n3 a multiple of 4; a rank above
 * 128 is MPI_ERR_UNSUPPORTED.  Allocates its workspace (about 16 q r1 n2 n3
 * bytes for the mode products) and synchronises the context's stream. */
mpi_status mpi_tucker_compress(mpi_ctx* ctx, const mpi_c32* T, const int n[3], int q, double eps,
                               mpi_basis** out, int ranks_out[3], double* bound_out);

/* Which kernel carries the dense contraction U alpha (for a Tucker basis, the
 * core contraction) for C coils at precision `prec`; `jacobian` != 0 asks
 * about the Jacobian's forward pass, which expands alpha and dalpha together.
 * The forward-type passes run in coil groups when all C coils do not fit one
 * tensor-core launch; the adjoint passes run on the CUDA cores in that case.
 * Returns MPI_EXPAND_FFMA (CUDA-core FP32), MPI_EXPAND_TF32X3 (tensor cores,
 * FP32-accurate split) or MPI_EXPAND_BF16 (tensor cores, BF16 operands), or -1
 * for a null basis, C < 1 or an unknown precision.  Host-side query: no device
 * work. */
enum { MPI_EXPAND_FFMA = 0, MPI_EXPAND_TF32X3 = 1, MPI_EXPAND_BF16 = 2 };
int mpi_expand_path(const mpi_basis* basis, int C, int jacobian, mpi_precision prec);

/* ------------------------------------------------------- operator (device) */

/* maps[k] = U alpha_k for k < C (Eq. 5 inside F_s(.)).  alpha [C][q], maps [C][N]. */
mpi_status mpi_basis_expand(mpi_ctx* ctx, const mpi_basis* basis, const mpi_c32* alpha, int C,
                            mpi_c32* maps, mpi_precision prec);

/* y = G(p, alpha) (Eq. 5).  alpha [C][q], p [N], y [C][M]. */
mpi_status mpi_forward(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis,
                       const mpi_c32* alpha, int C, const mpi_c32* p, mpi_c32* y,
                       mpi_precision prec);

/* p_out = S^H F^H y = sum_k conj(U alpha_k) (.) F_s^H y_k (adjoint of Eq. 1 in p).
 * y [C][M], p_out [N]. */
mpi_status mpi_adjoint(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis,
                       const mpi_c32* alpha, int C, const mpi_c32* y, mpi_c32* p_out,
                       mpi_precision prec);

/* mpi_forward and mpi_adjoint on HOST buffers (the same operators, Eq. 5 and the
 * adjoint of Eq. 1 in p, and the same layouts:
 * alpha [C][q]; forward p [N] -> y [C][M]; adjoint y [C][M] -> p_out [N]).  The
 * kernels read and write pinned (page-locked, mapped) host buffers in place,
 * over the coherent CPU-GPU link; pageable buffers are copied through a device
 * staging buffer that the context owns (grown on demand, freed with the
 * context).  The call runs the operator on the context's stream and
 * synchronises the stream before it returns, so the output is ready in host
 * memory.  Errors: as mpi_forward / mpi_adjoint;
 * MPI_ERR_OOM if the staging buffer cannot be allocated; MPI_ERR_CUDA if a copy
 * fails.  Not for use inside stream capture (it synchronises). */
mpi_status mpi_forward_host(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis,
                            const mpi_c32* alpha, int C, const mpi_c32* p, mpi_c32* y,
                            mpi_precision prec);
mpi_status mpi_adjoint_host(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis,
                            const mpi_c32* alpha, int C, const mpi_c32* y, mpi_c32* p_out,
                            mpi_precision prec);

/* dy = J(p, alpha)[dp; dalpha] = [F_s(U alpha_k (.) dp + p (.) U dalpha_k)]_k (Eq. 7). */
mpi_status mpi_jacobian(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis,
                        const mpi_c32* alpha, int C, const mpi_c32* p, const mpi_c32* dp,
                        const mpi_c32* dalpha, mpi_c32* dy, mpi_precision prec);

/* Allocation-free variant of mpi_forward (Cartesian plans, FP32 expansion).
 * The paper has no counterpart: this exists for callers that cannot call
 * cudaMalloc once running -- a service whose device memory is carved up at
 * start-up by its own pool allocator, or a real-time loop that must not block in
 * the driver's allocator (cudaMalloc may synchronise the device and can fail at
 * an unpredictable point).  mpi_forward may grow the context workspace; this
 * call never allocates: its [C][N] intermediate lives in a 16 MiB static device
 * array inside the library.  mpi_ctx_create loads the module holding that array
 * on its device (the driver loads modules lazily, and the first use would
 * otherwise reserve the 16 MiB inside this call); from then on every GPU with a
 * context holds the array until the process exits.  Each call asks for the
 * array's device address (cudaGetSymbolAddress, no allocation once the module
 * is resident) with the context's device current; after a device reset the
 * first call loads the module again.  Make the first call before any stream
 * capture.  Limit: C * N <= 2,097,152, else MPI_ERR_SHAPE (nothing is
 * launched).  Radial plans and Tucker bases return MPI_ERR_UNSUPPORTED.  The
 * expansion is mpi_forward's FP32 one (3xTF32 tensor cores where the shape
 * fits).  Every call,
 * from any context, shares the one array: calls whose work overlaps on the GPU
 * (different streams, or concurrent host threads) race and corrupt each other's
 * results; serialise them.  The caller still passes every input and output
 * (device pointers), as for mpi_forward. */
mpi_status mpi_forward_noalloc(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis,
                               const mpi_c32* alpha, int C, const mpi_c32* p, mpi_c32* y);

/* [dp; dalpha] = J^H(p, alpha) r (the display after Eq. 7; ^H on a vector inside
 * (.) is the element-wise conjugate):
 *   dp        = sum_k conj(U alpha_k) (.) F_s^H r_k            [N]
 *   dalpha_k  = U^H (conj(p) (.) F_s^H r_k)                     [C][q]
 * Coil maps are recomputed from alpha, never stored. */
mpi_status mpi_jacobian_adjoint(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis,
                                const mpi_c32* alpha, int C, const mpi_c32* p, const mpi_c32* r,
                                mpi_c32* dp, mpi_c32* dalpha, mpi_precision prec);

/* Several sets of maps (Discussion, "Forward Model Extensions": extra bilinear
 * terms in the signal equation), M >= 1 sets on a dense basis:
 *   y_k = F_s( sum_m (U alpha_{m,k}) (.) p_m )
 * alpha [M][C][q] (set m's coefficients contiguous), p [M][N], all device
 * pointers; M = 1 is the single-set call.  The products are summed image-side
 * in the expansion epilogues, so F_s runs once per coil whatever M.
 * MPI_ERR_UNSUPPORTED for Tucker bases with M > 1. */
mpi_status mpi_forward_maps(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis, int M,
                            const mpi_c32* alpha, int C, const mpi_c32* p, mpi_c32* y, mpi_precision prec);
/* The adjoint in the images: p_out[m] = sum_k conj(U alpha_{m,k}) (.) F_s^H y_k, [M][N]. */
mpi_status mpi_adjoint_maps(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis, int M,
                            const mpi_c32* alpha, int C, const mpi_c32* y, mpi_c32* p_out, mpi_precision prec);
/* J[dp; dalpha] = [F_s(sum_m U alpha_{m,k} (.) dp_m + p_m (.) U dalpha_{m,k})]_k
 * (Eq. 7 summed over the sets); dp [M][N], dalpha [M][C][q], dy [C][M_samples]. */
mpi_status mpi_jacobian_maps(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis, int M,
                             const mpi_c32* alpha, int C, const mpi_c32* p, const mpi_c32* dp,
                             const mpi_c32* dalpha, mpi_c32* dy, mpi_precision prec);
/* J^H r per set: dp[m] = sum_k conj(U alpha_{m,k}) (.) F_s^H r_k,
 * dalpha[m][k] = U^H (conj(p_m) (.) F_s^H r_k); F_s^H runs once. */
mpi_status mpi_jacobian_adjoint_maps(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis, int M,
                                     const mpi_c32* alpha, int C, const mpi_c32* p, const mpi_c32* r,
                                     mpi_c32* dp, mpi_c32* dalpha, mpi_precision prec);

/* alpha_k = (U^H U)^{-1} U^H maps_k: projection of given maps onto the basis
 * (Fig. 2 caption).  Gram matrix, Cholesky factor and triangular solves in FP64.
 * maps [C][N] -> alpha [C][q]. */
mpi_status mpi_basis_project(mpi_ctx* ctx, const mpi_basis* basis, const mpi_c32* maps, int C,
                             mpi_c32* alpha);

/* ------------------------------------------------------------------ batches */

/* Many slices of uneven grid size and coil count (e.g. a multi-slice exam),
 * each a set of caller-owned device buffers: y = G_s(p) and/or x = G_s^H(y). */
typedef struct {
  const mpi_plan* plan;
  const mpi_basis* basis;  /* slices of one grid size may share one basis */
  int C;
  const mpi_c32* alpha;    /* [C][q] */
  const mpi_c32* p;        /* [N] forward input */
  mpi_c32* y;              /* [C][M] forward output and adjoint input */
  mpi_c32* x;              /* [N] adjoint output */
} mpi_batch_slice;

typedef enum { MPI_BATCH_FORWARD = 1, MPI_BATCH_ADJOINT = 2, MPI_BATCH_PAIR = 3 } mpi_batch_kind;
typedef struct mpi_batch mpi_batch;

/* Record every kernel of the n slices' operator calls (forward, adjoint, or the
 * forward followed by the adjoint of its output) into one CUDA graph.  Slices
 * are ordered by basis so that a shared basis stays L2-resident; the context
 * workspace is sized first, so replays allocate nothing.  The slice descriptors
 * are copied; their buffers must stay valid while the batch exists.  Waits for
 * the context's stream once. */
mpi_status mpi_batch_create(mpi_ctx* ctx, const mpi_batch_slice* slices, int n, int kind,
                            mpi_precision prec, mpi_batch** out);
/* Launch the recorded graph once on the context's stream (asynchronous). */
mpi_status mpi_batch_run(mpi_ctx* ctx, mpi_batch* batch);
/* Kernels one replay launches (-1 for a NULL batch). */
int64_t mpi_batch_kernel_count(const mpi_batch* batch);
/* Grouped expansion launches per direction in the batch (slices on Cartesian
 * plans sharing a dense basis, FP32 or BF16, are expanded by one launch per
 * group whose grid rows are the slices), or -1 for a null handle. */
int mpi_batch_group_count(const mpi_batch* batch);
mpi_status mpi_batch_destroy(mpi_batch* batch);

/* ----------------------------------------------------------------- solvers */

/* MPI-BL: IRGN for (p, alpha) (Eq. 6) with CG on the normal equations
 *   (J^H J + 2 diag(a_n I, b_n I)) dx = J^H r - 2 diag(a_n I, b_n I) x,
 * r = y_s - G(x), y_s = y * (scale_target / ||y||), a_n = max(a0 d^n, floor),
 * b_n = max(b0 d^n, floor), x <- x + gamma dx, start p = 1, alpha = 0.
 * Outputs: alpha_out [C][q]; p_out [N] divided by the data scale;
 * resid_out (host, may be NULL) [n_outer + 1] residual norms in scaled units. */
typedef struct {
  int n_outer, n_cg;
  double a0, b0, decay, floor_, gamma, scale_target;
} mpi_irgn_params;

mpi_status mpi_sm_estimate(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis,
                           const mpi_c32* y, int C, const mpi_irgn_params* prm,
                           mpi_c32* alpha_out, mpi_c32* p_out, double* resid_out,
                           mpi_precision prec);
/* MPI-BL with M sets of maps (the model of mpi_forward_maps): the same IRGN with
 * the unknowns x = [p_1 .. p_M ; alpha_1 .. alpha_M], Eq. 6's penalties on every
 * image (alpha_n) and every coefficient set (beta_n).  Start: p_m = 1, alpha_1 = 0
 * and, for m >= 2, the first basis coefficient of every coil 0.1 (sets that start
 * proportional to the first stay proportional).  Outputs alpha_out [M][C][q],
 * p_out [M][N] (device); resid_out as mpi_sm_estimate.  M = 1 is mpi_sm_estimate. */
mpi_status mpi_sm_estimate_maps(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis, int M,
                                const mpi_c32* y, int C, const mpi_irgn_params* prm, mpi_c32* alpha_out,
                                mpi_c32* p_out, double* resid_out, mpi_precision prec);

/* MPI-L: constrained TV reconstruction (Eq. 8) by scaled ADMM (Eq. 11):
 *   z0 = prox_{TV/rho}(p + u0)        (n_tv FGP iterations from zero)
 *   zk = Pi_{C(y_k, eps_k)}(F_s S_k p + u_k)
 *   p  = (I + sum S_k^H F_s^H F_s S_k)^{-1}(z0 - u0 + sum S_k^H F_s^H (zk - u_k))
 *        (n_cg CG iterations from the previous p)
 *   u  = u + A p - z ; residual-balancing rho (mu, tau).
 * Start p = z = u = 0.  eps: host [C] (FP64).  hist_out (host, may be NULL)
 * [n_outer][3] (primal, dual, rho). */
typedef struct {
  int n_outer, n_cg, n_tv;
  double rho0, mu, tau;
} mpi_admm_params;

mpi_status mpi_image_solve(mpi_ctx* ctx, const mpi_plan* plan, const mpi_basis* basis,
                           const mpi_c32* alpha, int C, const mpi_c32* y, const double* eps,
                           const mpi_admm_params* prm, mpi_c32* p_out, double* hist_out,
                           mpi_precision prec);
/* Dynamic MPI-L (the constrained problem with a spatiotemporal regulariser
 * that closes the "Regularized Density Reconstruction" section): T frames p_t
 * of one 2D grid share the coil maps (alpha), frame t is sampled by plans[t]
 * (equal sample counts M), and
 *   min R(p)  s.t.  ||y_{k,t} - F_s^t S_k p_t|| <= eps_{k,t}  for all k, t,
 * with R the isotropic TV over the (t, y, x) grid of the frames (the frame
 * axis weighted like the spatial ones).  The steps of mpi_image_solve with
 * the data blocks of all frames.  y: device [T][C][M]; eps: host [T][C];
 * p_out: device [T][N]; hist_out as mpi_image_solve.  T = 1 is mpi_image_solve.
 * MPI_ERR_SHAPE unless every plan is 2D with the first plan's grid and M. */
mpi_status mpi_image_solve_dynamic(mpi_ctx* ctx, const mpi_plan* const* plans, int T, const mpi_basis* basis,
                                   const mpi_c32* alpha, int C, const mpi_c32* y, const double* eps,
                                   const mpi_admm_params* prm, mpi_c32* p_out, double* hist_out,
                                   mpi_precision prec);

/* TV prox alone: x = argmin (1/2)||x - v||^2 + lam TV(x) by n_iter FGP
 * iterations (the z0 update of Eq. 11).  v, x device [N] on the plan's grid. */
mpi_status mpi_tv_prox(mpi_ctx* ctx, const mpi_plan* plan, const mpi_c32* v, double lam,
                       int n_iter, mpi_c32* x);

#ifdef __cplusplus
}
#endif

#endif /* MPI_GB300_H */
