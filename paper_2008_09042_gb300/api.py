"""Python face of the C ABI: contexts, plans, bases and the operator calls.

Tensors are torch complex64 CUDA tensors (contiguous); the calls pass their
device pointers and the current torch stream to the library, which does all
the work in its own kernels.
"""

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import PREC, check, load


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else ctypes.c_void_p(0)


def _need(t, shape, name):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.dtype != torch.complex64 or not t.is_cuda or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous complex64 CUDA tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t


class Context:
    """A library context bound to a CUDA device and stream."""

    def __init__(self, device=0, stream=None):
        self.lib = load()
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = ctypes.c_void_p()
        st = self.lib.mpi_ctx_create(ctypes.byref(h), device, ctypes.c_void_p(stream.cuda_stream))
        check(None, st)
        self.h = h

    def set_stream(self, stream):
        self.stream = stream
        check(self.h, self.lib.mpi_ctx_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream)))

    def synchronize(self):
        check(self.h, self.lib.mpi_ctx_synchronize(self.h))

    def launches(self):
        return int(self.lib.mpi_ctx_launch_count(self.h))

    def set_autotune(self, enable=True):
        check(self.h, self.lib.mpi_ctx_set_autotune(self.h, 1 if enable else 0))

    def set_wait_limit(self, cycles):
        """Bounded-wait limit of the tensor-core kernels, in SM clock cycles."""
        check(self.h, self.lib.mpi_ctx_set_wait_limit(self.h, int(cycles)))

    def inject_stall(self, stages=-1):
        """Fault injection for tests of the timeout path: the FP32 tensor-core
        expansion's copy producer stops after `stages` ring stages (-1: off)."""
        check(self.h, self.lib.mpi_ctx_inject_stall(self.h, int(stages)))

    TF32_READINGS = {-2: "failed", 0: "truncate", 1: "nearest_even", 2: "nearest_away", 3: "full", 4: "other"}

    def tf32_reading(self):
        """How the tensor core reads FP32 operands of kind::tf32, as measured when
        the context was made ("truncate" enables the 3xTF32 kernels)."""
        return self.TF32_READINGS.get(int(self.lib.mpi_ctx_tf32_reading(self.h)), "other")

    def set_tf32x3(self, enable=True):
        """Switch the 3xTF32 tensor-core kernels off (FP32 then runs on the CUDA
        cores) or back on (only where the probe found the truncating reading)."""
        check(self.h, self.lib.mpi_ctx_set_tf32x3(self.h, 1 if enable else 0))

    def set_line_kernel(self, choice=0):
        """Fix the FFT line passes' kernel: 8, 16, 32 (lines per CTA), -1 (register
        two-step pass along y) or 0 (tuned)."""
        check(self.h, self.lib.mpi_ctx_set_line_kernel(self.h, int(choice)))

    def tuning_records(self):
        """Text of every launch-shape decision the autotuner made on this context."""
        out = []
        while True:
            t = ctypes.c_char_p()
            if self.lib.mpi_ctx_tuning_record(self.h, len(out), ctypes.byref(t)):
                return out
            out.append(t.value.decode())

    def workspace_bytes(self):
        """Device bytes held by the context's growable workspace and staging buffer."""
        return int(self.lib.mpi_ctx_workspace_bytes(self.h))

    FAMILIES = {"expand": 0, "uh_v": 1, "fft_rows": 2, "fft_lines": 3, "nufft": 4, "solver": 5, "other": 6}

    def profile(self, enable=True):
        check(self.h, self.lib.mpi_ctx_profile(self.h, 1 if enable else 0))

    def profile_read(self, reset=False, kernels=False):
        """{family: (ms, launches)} summed since the last reset; with ``kernels``
        also {kernel name: (ms, launches)}, returned as a second value."""
        out = {}
        for name, fam in self.FAMILIES.items():
            ms = ctypes.c_double()
            n = ctypes.c_int64()
            check(self.h, self.lib.mpi_ctx_profile_read(self.h, fam, ctypes.byref(ms), ctypes.byref(n), 0))
            out[name] = (ms.value, n.value)
        per_kernel = {}
        if kernels:
            i = 0
            while True:
                nm = ctypes.c_char_p()
                ms = ctypes.c_double()
                n = ctypes.c_int64()
                if self.lib.mpi_ctx_profile_kernel(self.h, i, ctypes.byref(nm), ctypes.byref(ms), ctypes.byref(n)):
                    break
                per_kernel[nm.value.decode()] = (ms.value, n.value)
                i += 1
        if reset:
            ms = ctypes.c_double()
            n = ctypes.c_int64()
            check(self.h, self.lib.mpi_ctx_profile_read(self.h, 0, ctypes.byref(ms), ctypes.byref(n), 1))
        return (out, per_kernel) if kernels else out

    def reserve(self, plan, basis, C):
        check(self.h, self.lib.mpi_ctx_reserve(self.h, plan.h, basis.h, C))

    def close(self):
        if getattr(self, "h", None):
            self.lib.mpi_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """Geometry and sampling of F_s."""

    def __init__(self, ctx, dims, sample_idx=None, traj=None, kb_width=6, oversamp=2.0):
        self.ctx = ctx
        dims = tuple(int(d) for d in dims)
        if len(dims) == 2:
            self.ndim, full = 2, (1,) + dims
        elif len(dims) == 3:
            self.ndim, full = 3, dims
        else:
            raise ValueError("dims must have 2 or 3 entries")
        self.dims = dims
        self.N = int(np.prod(dims))
        d = _lib.PlanDesc()
        d.ndim = self.ndim
        d.dims[0], d.dims[1], d.dims[2] = full
        keep = []
        if traj is None:
            idx = np.ascontiguousarray(np.asarray(sample_idx, dtype=np.int32))
            keep.append(idx)
            d.kind = _lib.TRAJ_CARTESIAN
            d.M = int(idx.size)
            d.sample_idx = idx.ctypes.data if idx.size else None
            self.kind = "cartesian"
        else:
            k = np.ascontiguousarray(np.asarray(traj, dtype=np.float32).reshape(-1, 2))
            keep.append(k)
            d.kind = _lib.TRAJ_RADIAL
            d.M = int(k.shape[0])
            d.traj = k.ctypes.data if k.size else None
            d.kb_width = int(kb_width)
            d.oversamp = float(oversamp)
            self.kind = "radial"
        self.M = int(d.M)
        h = ctypes.c_void_p()
        check(ctx.h, ctx.lib.mpi_plan_create(ctx.h, ctypes.byref(d), ctypes.byref(h)))
        self.h = h

    def grid_index(self):
        out = torch.empty((self.M, 2), dtype=torch.int32, device=f"cuda:{self.ctx.device}")
        check(self.ctx.h, self.ctx.lib.mpi_plan_grid_index(self.ctx.h, self.h, _ptr(out)))
        return out

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.mpi_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Basis:
    """Dense basis U (N x q) held by the library as [q][N] complex64."""

    def __init__(self, ctx, U_qN):
        self.ctx = ctx
        if isinstance(U_qN, torch.Tensor):
            t = U_qN.to(device=f"cuda:{ctx.device}", dtype=torch.complex64).contiguous()
        else:
            t = torch.from_numpy(np.ascontiguousarray(np.asarray(U_qN, dtype=np.complex64))).to(
                f"cuda:{ctx.device}")
        q, N = t.shape
        self.q, self.N = int(q), int(N)
        h = ctypes.c_void_p()
        check(ctx.h, ctx.lib.mpi_basis_load_dense(ctx.h, _ptr(t), self.N, self.q, 1, ctypes.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.mpi_basis_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class TuckerBasis(Basis):
    """Tucker-factored basis: core (r1, r2, r3, q) and factors U_k (n_k, r_k).

    The library takes the core as [q][r1][r2][r3]; this constructor transposes.
    """

    def __init__(self, ctx, core, factors):
        self.ctx = ctx
        core = np.asarray(core)
        r = core.shape[:3]
        self.q = int(core.shape[3])
        n = tuple(int(f.shape[0]) for f in factors)
        self.N = int(np.prod(n))
        core_q = np.ascontiguousarray(np.moveaxis(core, 3, 0).astype(np.complex64))
        fac = [np.ascontiguousarray(np.asarray(f, dtype=np.complex64)) for f in factors]
        keep = [core_q] + fac
        n_arr = (ctypes.c_int * 3)(*n)
        r_arr = (ctypes.c_int * 3)(*[int(x) for x in r])
        h = ctypes.c_void_p()
        check(ctx.h, ctx.lib.mpi_basis_load_tucker(ctx.h, core_q.ctypes.data, fac[0].ctypes.data, fac[1].ctypes.data,
                                                   fac[2].ctypes.data, n_arr, r_arr, self.q, 0, ctypes.byref(h)))
        del keep
        self.h = h


def basis_expand(ctx, basis, alpha, prec="fp32", out=None):
    C = alpha.shape[0]
    _need(alpha, (C, basis.q), "alpha")
    out = out if out is not None else torch.empty((C, basis.N), dtype=torch.complex64, device=alpha.device)
    check(ctx.h, ctx.lib.mpi_basis_expand(ctx.h, basis.h, _ptr(alpha), C, _ptr(out), PREC[prec]))
    return out


def forward(ctx, plan, basis, alpha, p, prec="fp32", out=None):
    C = alpha.shape[0]
    _need(alpha, (C, basis.q), "alpha")
    _need(p, (plan.N,), "p")
    out = out if out is not None else torch.empty((C, plan.M), dtype=torch.complex64, device=p.device)
    check(ctx.h, ctx.lib.mpi_forward(ctx.h, plan.h, basis.h, _ptr(alpha), C, _ptr(p), _ptr(out), PREC[prec]))
    return out


def adjoint(ctx, plan, basis, alpha, y, prec="fp32", out=None):
    C = alpha.shape[0]
    _need(alpha, (C, basis.q), "alpha")
    _need(y, (C, plan.M), "y")
    out = out if out is not None else torch.empty((plan.N,), dtype=torch.complex64, device=y.device)
    check(ctx.h, ctx.lib.mpi_adjoint(ctx.h, plan.h, basis.h, _ptr(alpha), C, _ptr(y), _ptr(out), PREC[prec]))
    return out


def _need_host(t, shape, name):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.dtype != torch.complex64 or t.is_cuda or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous complex64 CPU tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t


def forward_host(ctx, plan, basis, alpha, p, prec="fp32", out=None):
    """forward() on host tensors: the library copies the inputs in and y out
    (mpi_forward_host); returns when y is ready in host memory."""
    C = alpha.shape[0]
    _need_host(alpha, (C, basis.q), "alpha")
    _need_host(p, (plan.N,), "p")
    out = out if out is not None else torch.empty((C, plan.M), dtype=torch.complex64)
    _need_host(out, (C, plan.M), "out")
    check(ctx.h, ctx.lib.mpi_forward_host(ctx.h, plan.h, basis.h, _ptr(alpha), C, _ptr(p), _ptr(out),
                                          PREC[prec]))
    return out


def adjoint_host(ctx, plan, basis, alpha, y, prec="fp32", out=None):
    """adjoint() on host tensors (mpi_adjoint_host); returns when the image is
    ready in host memory."""
    C = alpha.shape[0]
    _need_host(alpha, (C, basis.q), "alpha")
    _need_host(y, (C, plan.M), "y")
    out = out if out is not None else torch.empty((plan.N,), dtype=torch.complex64)
    _need_host(out, (plan.N,), "out")
    check(ctx.h, ctx.lib.mpi_adjoint_host(ctx.h, plan.h, basis.h, _ptr(alpha), C, _ptr(y), _ptr(out),
                                          PREC[prec]))
    return out


def jacobian(ctx, plan, basis, alpha, p, dp, dalpha, prec="fp32", out=None):
    C = alpha.shape[0]
    for t, s, n in ((alpha, (C, basis.q), "alpha"), (dalpha, (C, basis.q), "dalpha"),
                    (p, (plan.N,), "p"), (dp, (plan.N,), "dp")):
        _need(t, s, n)
    out = out if out is not None else torch.empty((C, plan.M), dtype=torch.complex64, device=p.device)
    check(ctx.h, ctx.lib.mpi_jacobian(ctx.h, plan.h, basis.h, _ptr(alpha), C, _ptr(p), _ptr(dp), _ptr(dalpha),
                                      _ptr(out), PREC[prec]))
    return out


def jacobian_adjoint(ctx, plan, basis, alpha, p, r, prec="fp32", out_p=None, out_alpha=None):
    C = alpha.shape[0]
    _need(alpha, (C, basis.q), "alpha")
    _need(p, (plan.N,), "p")
    _need(r, (C, plan.M), "r")
    out_p = out_p if out_p is not None else torch.empty((plan.N,), dtype=torch.complex64, device=p.device)
    out_alpha = out_alpha if out_alpha is not None else torch.empty((C, basis.q), dtype=torch.complex64,
                                                                    device=p.device)
    check(ctx.h, ctx.lib.mpi_jacobian_adjoint(ctx.h, plan.h, basis.h, _ptr(alpha), C, _ptr(p), _ptr(r),
                                              _ptr(out_p), _ptr(out_alpha), PREC[prec]))
    return out_p, out_alpha


EXPAND_PATHS = {0: "ffma", 1: "tf32x3", 2: "bf16"}


def expand_path(ctx, basis, C, prec="fp32", jacobian=False):
    """Which kernel carries the contraction U alpha for C coils: "ffma", "tf32x3" or "bf16"."""
    r = ctx.lib.mpi_expand_path(basis.h, int(C), int(bool(jacobian)), PREC[prec])
    if r < 0:
        raise ValueError("mpi_expand_path: bad arguments")
    return EXPAND_PATHS[r]


def maxwell_basis_2d(ctx, shape, q, sources, omega, fov=(0.22, 0.22), f_hz=128e6):
    """Maxwell basis of an ny x nx slice built on the GPU (mpi_maxwell_basis_2d).

    sources: (D, 3) dipole sites in metres; omega: (6 D, L) complex excitation
    amplitudes.  Returns (U, sv): U the (q, N) complex64 device tensor of the q
    leading left singular vectors of B omega (load it with Basis(ctx, U)), sv
    the min(6 D, L) singular values (numpy, descending)."""
    ny, nx = shape
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.float64))
    om = np.ascontiguousarray(np.asarray(omega, dtype=np.complex128))
    D = src.shape[0]
    if src.shape != (D, 3) or om.ndim != 2 or om.shape[0] != 6 * D:
        raise ValueError("sources must be (D, 3) and omega (6 D, L)")
    L = om.shape[1]
    U = torch.empty((q, ny * nx), dtype=torch.complex64, device=f"cuda:{ctx.device}")
    sv = np.zeros(min(6 * D, L), dtype=np.float64)
    check(ctx.h, ctx.lib.mpi_maxwell_basis_2d(ctx.h, ny, nx, float(fov[0]), float(fov[1]), float(f_hz),
                                             src.ctypes.data, D, om.ctypes.data, L, q, _ptr(U),
                                             sv.ctypes.data))
    return U, sv


def maxwell_basis_3d(ctx, shape, q, sources, omega, fov=(0.22, 0.22, 0.22), f_hz=128e6):
    """Maxwell basis of an nz x ny x nx volume built on the GPU (mpi_maxwell_basis_3d).
    Returns (U (q, N) complex64 device tensor, singular values)."""
    nz, ny, nx = shape
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.float64))
    om = np.ascontiguousarray(np.asarray(omega, dtype=np.complex128))
    D = src.shape[0]
    if src.shape != (D, 3) or om.ndim != 2 or om.shape[0] != 6 * D:
        raise ValueError("sources must be (D, 3) and omega (6 D, L)")
    L = om.shape[1]
    U = torch.empty((q, nz * ny * nx), dtype=torch.complex64, device=f"cuda:{ctx.device}")
    sv = np.zeros(min(6 * D, L), dtype=np.float64)
    check(ctx.h, ctx.lib.mpi_maxwell_basis_3d(ctx.h, nz, ny, nx, float(fov[0]), float(fov[1]), float(fov[2]),
                                             float(f_hz), src.ctypes.data, D, om.ctypes.data, L, q, _ptr(U),
                                             sv.ctypes.data))
    return U, sv


class CompressedBasis(Basis):
    """A Tucker basis made by mpi_tucker_compress (held by the library)."""

    def __init__(self, ctx, handle, shape, q, ranks, bound):
        self.ctx, self.h = ctx, handle
        self.n, self.q, self.N = tuple(shape), int(q), int(np.prod(shape))
        self.ranks, self.bound = tuple(ranks), float(bound)


def tucker_compress(ctx, T, shape, eps=1e-4):
    """HOSVD compression of a dense basis T (q, n1 n2 n3) on the GPU to accuracy
    eps (Eq. 21).  Returns a CompressedBasis with .ranks and .bound."""
    q = int(T.shape[0])
    t = T.to(device=f"cuda:{ctx.device}", dtype=torch.complex64).contiguous()
    if t.shape[1] != int(np.prod(shape)):
        raise ValueError("T must be (q, n1 n2 n3)")
    n_arr = (ctypes.c_int * 3)(*[int(x) for x in shape])
    r_arr = (ctypes.c_int * 3)()
    bound = ctypes.c_double()
    h = ctypes.c_void_p()
    check(ctx.h, ctx.lib.mpi_tucker_compress(ctx.h, _ptr(t), n_arr, q, float(eps), ctypes.byref(h), r_arr,
                                             ctypes.byref(bound)))
    return CompressedBasis(ctx, h, shape, q, tuple(r_arr), bound.value)


def basis_project(ctx, basis, maps):
    C = maps.shape[0]
    _need(maps, (C, basis.N), "maps")
    out = torch.empty((C, basis.q), dtype=torch.complex64, device=maps.device)
    check(ctx.h, ctx.lib.mpi_basis_project(ctx.h, basis.h, _ptr(maps), C, _ptr(out)))
    return out


class MPIOperator(torch.autograd.Function):
    """y = G(p, alpha) with a backward that calls the library's J^H kernel.

    G is complex-bilinear (no conjugates), so the vector-Jacobian product torch
    asks for is J^H applied to the incoming gradient.
    """

    @staticmethod
    def forward(fctx, p, alpha, ctx, plan, basis, prec):
        fctx.save_for_backward(p, alpha)
        fctx.lib_ctx, fctx.plan, fctx.basis, fctx.prec = ctx, plan, basis, prec
        return forward(ctx, plan, basis, alpha.contiguous(), p.contiguous(), prec)

    @staticmethod
    def backward(fctx, gy):
        p, alpha = fctx.saved_tensors
        gp, ga = jacobian_adjoint(fctx.lib_ctx, fctx.plan, fctx.basis, alpha.contiguous(), p.contiguous(),
                                  gy.contiguous(), fctx.prec)
        return gp, ga, None, None, None, None


def mpi_operator(p, alpha, ctx, plan, basis, prec="fp32"):
    return MPIOperator.apply(p, alpha, ctx, plan, basis, prec)


def sm_estimate(ctx, plan, basis, y, C, n_outer=20, n_cg=10, a0=1.0, b0=1.0, decay=0.5, floor=1e-6, gamma=1.0,
                scale_target=100.0, prec="fp32"):
    """MPI-BL (IRGN, Eq. 6).  Returns (alpha [C][q], p [N], residual history (n_outer + 1,))."""
    _need(y, (C, plan.M), "y")
    prm = _lib.IrgnParams(n_outer, n_cg, a0, b0, decay, floor, gamma, scale_target)
    alpha = torch.empty((C, basis.q), dtype=torch.complex64, device=y.device)
    p = torch.empty((plan.N,), dtype=torch.complex64, device=y.device)
    hist = np.zeros(n_outer + 1, dtype=np.float64)
    check(ctx.h, ctx.lib.mpi_sm_estimate(ctx.h, plan.h, basis.h, _ptr(y), C, ctypes.byref(prm), _ptr(alpha), _ptr(p),
                                         hist.ctypes.data_as(ctypes.c_void_p), PREC[prec]))
    return alpha, p, hist


def forward_maps(ctx, plan, basis, alpha, p, prec="fp32", out=None):
    """y_k = F_s(sum_m U alpha[m, k] (.) p[m]) for M sets of maps: alpha (M, C, q), p (M, N)."""
    M, C = alpha.shape[0], alpha.shape[1]
    _need(alpha, (M, C, basis.q), "alpha")
    _need(p, (M, plan.N), "p")
    out = out if out is not None else torch.empty((C, plan.M), dtype=torch.complex64, device=p.device)
    check(ctx.h, ctx.lib.mpi_forward_maps(ctx.h, plan.h, basis.h, M, _ptr(alpha), C, _ptr(p), _ptr(out), PREC[prec]))
    return out


def adjoint_maps(ctx, plan, basis, alpha, y, prec="fp32", out=None):
    """The adjoint in the M images: (M, N)."""
    M, C = alpha.shape[0], alpha.shape[1]
    _need(alpha, (M, C, basis.q), "alpha")
    _need(y, (C, plan.M), "y")
    out = out if out is not None else torch.empty((M, plan.N), dtype=torch.complex64, device=y.device)
    check(ctx.h, ctx.lib.mpi_adjoint_maps(ctx.h, plan.h, basis.h, M, _ptr(alpha), C, _ptr(y), _ptr(out), PREC[prec]))
    return out


def jacobian_maps(ctx, plan, basis, alpha, p, dp, dalpha, prec="fp32", out=None):
    M, C = alpha.shape[0], alpha.shape[1]
    for t, sh, n in ((alpha, (M, C, basis.q), "alpha"), (dalpha, (M, C, basis.q), "dalpha"),
                     (p, (M, plan.N), "p"), (dp, (M, plan.N), "dp")):
        _need(t, sh, n)
    out = out if out is not None else torch.empty((C, plan.M), dtype=torch.complex64, device=p.device)
    check(ctx.h, ctx.lib.mpi_jacobian_maps(ctx.h, plan.h, basis.h, M, _ptr(alpha), C, _ptr(p), _ptr(dp),
                                           _ptr(dalpha), _ptr(out), PREC[prec]))
    return out


def jacobian_adjoint_maps(ctx, plan, basis, alpha, p, r, prec="fp32"):
    """J^H r per set of maps: ((M, N), (M, C, q))."""
    M, C = alpha.shape[0], alpha.shape[1]
    _need(alpha, (M, C, basis.q), "alpha")
    _need(p, (M, plan.N), "p")
    _need(r, (C, plan.M), "r")
    gp = torch.empty((M, plan.N), dtype=torch.complex64, device=p.device)
    ga = torch.empty((M, C, basis.q), dtype=torch.complex64, device=p.device)
    check(ctx.h, ctx.lib.mpi_jacobian_adjoint_maps(ctx.h, plan.h, basis.h, M, _ptr(alpha), C, _ptr(p), _ptr(r),
                                                   _ptr(gp), _ptr(ga), PREC[prec]))
    return gp, ga


def sm_estimate_maps(ctx, plan, basis, y, C, M, n_outer=20, n_cg=10, a0=1.0, b0=1.0, decay=0.5, floor=1e-6,
                     gamma=1.0, scale_target=100.0, prec="fp32"):
    """MPI-BL with M sets of maps.  Returns (alpha (M, C, q), p (M, N), residual history)."""
    _need(y, (C, plan.M), "y")
    prm = _lib.IrgnParams(n_outer, n_cg, a0, b0, decay, floor, gamma, scale_target)
    alpha = torch.empty((M, C, basis.q), dtype=torch.complex64, device=y.device)
    p = torch.empty((M, plan.N), dtype=torch.complex64, device=y.device)
    hist = np.zeros(n_outer + 1, dtype=np.float64)
    check(ctx.h, ctx.lib.mpi_sm_estimate_maps(ctx.h, plan.h, basis.h, M, _ptr(y), C, ctypes.byref(prm), _ptr(alpha),
                                              _ptr(p), hist.ctypes.data_as(ctypes.c_void_p), PREC[prec]))
    return alpha, p, hist


def image_solve(ctx, plan, basis, alpha, y, eps, n_outer=50, n_cg=5, n_tv=10, rho0=1.0, mu=10.0, tau=2.0,
                prec="fp32"):
    """MPI-L (ADMM-TV, Eqs. 8-11).  Returns (p [N], history (n_outer, 3) of primal, dual, rho)."""
    C = alpha.shape[0]
    _need(alpha, (C, basis.q), "alpha")
    _need(y, (C, plan.M), "y")
    eps = np.ascontiguousarray(np.asarray(eps, dtype=np.float64).reshape(C))
    prm = _lib.AdmmParams(n_outer, n_cg, n_tv, rho0, mu, tau)
    p = torch.empty((plan.N,), dtype=torch.complex64, device=y.device)
    hist = np.zeros((max(n_outer, 1), 3), dtype=np.float64)
    check(ctx.h, ctx.lib.mpi_image_solve(ctx.h, plan.h, basis.h, _ptr(alpha), C, _ptr(y),
                                         eps.ctypes.data_as(ctypes.c_void_p), ctypes.byref(prm), _ptr(p),
                                         hist.ctypes.data_as(ctypes.c_void_p), PREC[prec]))
    return p, hist[:n_outer]


def image_solve_dynamic(ctx, plans, basis, alpha, y, eps, n_outer=50, n_cg=5, n_tv=10, rho0=1.0, mu=10.0, tau=2.0,
                        prec="fp32"):
    """Dynamic MPI-L: frames sampled by plans[t], shared maps, spatiotemporal TV.
    y (T, C, M), eps (T, C).  Returns (p (T, N), history (n_outer, 3))."""
    T = len(plans)
    C = alpha.shape[0]
    _need(alpha, (C, basis.q), "alpha")
    _need(y, (T, C, plans[0].M), "y")
    eps = np.ascontiguousarray(np.asarray(eps, dtype=np.float64).reshape(T, C))
    prm = _lib.AdmmParams(n_outer, n_cg, n_tv, rho0, mu, tau)
    hs = (ctypes.c_void_p * T)(*[pl.h.value if isinstance(pl.h, ctypes.c_void_p) else pl.h for pl in plans])
    p = torch.empty((T, plans[0].N), dtype=torch.complex64, device=y.device)
    hist = np.zeros((max(n_outer, 1), 3), dtype=np.float64)
    check(ctx.h, ctx.lib.mpi_image_solve_dynamic(ctx.h, hs, T, basis.h, _ptr(alpha), C, _ptr(y),
                                                 eps.ctypes.data_as(ctypes.c_void_p), ctypes.byref(prm), _ptr(p),
                                                 hist.ctypes.data_as(ctypes.c_void_p), PREC[prec]))
    return p, hist[:n_outer]


def tv_prox(ctx, plan, v, lam, n_iter):
    """argmin (1/2)||x - v||^2 + lam TV(x) by n_iter FGP iterations."""
    _need(v, (plan.N,), "v")
    x = torch.empty_like(v)
    check(ctx.h, ctx.lib.mpi_tv_prox(ctx.h, plan.h, _ptr(v), float(lam), int(n_iter), _ptr(x)))
    return x


class Batch:
    """Many slices' operator calls recorded into one CUDA graph (mpi_batch_*).

    ``slices`` is a list of dicts with keys plan, basis, alpha, p, y, x (device
    tensors that must outlive the batch); kind is "forward", "adjoint" or "pair".
    """

    KINDS = {"forward": 1, "adjoint": 2, "pair": 3}

    def __init__(self, ctx, slices, kind="pair", prec="fp32"):
        self.ctx = ctx
        self.slices = slices  # keep the tensors alive
        arr = (_lib.BatchSlice * len(slices))()
        for i, s in enumerate(slices):
            arr[i].plan = s["plan"].h.value
            arr[i].basis = s["basis"].h.value
            arr[i].C = int(s["alpha"].shape[0])
            arr[i].alpha = s["alpha"].data_ptr()
            arr[i].p = s["p"].data_ptr()
            arr[i].y = s["y"].data_ptr() if s["y"].numel() else None
            arr[i].x = s["x"].data_ptr()
        h = ctypes.c_void_p()
        check(ctx.h, ctx.lib.mpi_batch_create(ctx.h, arr, len(slices), self.KINDS[kind], PREC[prec],
                                              ctypes.byref(h)))
        self.h = h

    def run(self):
        check(self.ctx.h, self.ctx.lib.mpi_batch_run(self.ctx.h, self.h))

    def kernels(self):
        return int(self.ctx.lib.mpi_batch_kernel_count(self.h))

    def groups(self):
        """Grouped expansion launches per direction (slices sharing a basis)."""
        return int(self.ctx.lib.mpi_batch_group_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.mpi_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
