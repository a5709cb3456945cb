"""The two solvers that drive the encoding operator, in FP64.

Test infrastructure (see the package header).

MPI-BL (sensitivity estimation): IRGN on the Maxwell-parameterised model.  At
each outer step the penalised Gauss-Newton sub-problem of Eq. 6 is solved by CG
on its normal equations (Theory, "Regularized Nonlinear Inversion").

MPI-L (density reconstruction): the constrained problem of Eq. 8 solved by
scaled ADMM with the splitting A = [I; F_s S_1; ...; F_s S_C], B = -I
(Eqs. 9-11): TV prox for z_0, l2-ball projections for z_k, a CG solve for p,
the dual update, and a residual-balancing rho (He et al. 2000; Boyd et al. 2011).

Readings of what the paper leaves open (all fixed numbers are choices, not
the paper's):
* Eq. 6's objective is (1/2)||r - J dx||^2 + a_n||p + dp||^2 + b_n sum||alpha_k + dalpha_k||^2;
  setting its gradient to zero gives (J^H J + 2 L_n) dx = J^H r - 2 L_n x,
  L_n = diag(a_n I_N, b_n I_{Cq}).
* Start p = 1, alpha = 0 (the convention of the NLINV method the section
  builds on); a_n = a_0 d^n, b_n = b_0 d^n with a floor; step gamma = 1 (no
  line search); the data are scaled to ||y|| = 100 and the scale is put back
  on p at the end.
* CG: fixed iteration count from zero; a zero curvature or residual makes the
  step 0 instead of dividing by zero.
* The z_0 update of Eq. 11 is printed as prox(z_0^n - (p^n + u_0^n)); with
  A p + B z = 0 and B = -I the scaled-form update is prox(p^n + u_0^n), which is
  what is computed.
* R = isotropic TV with forward differences and a zero difference at the last
  sample (Neumann), on complex images: TV(x) = sum sqrt(sum_d |D_d x|^2).  Its prox
  is computed by n_tv iterations of FGP (Beck and Teboulle 2009) from P = 0.
* rho: primal residual ||A p - z||; the z-block is updated first and p second,
  so the dual residual is rho ||A (p - p_prev)|| (Boyd et al. 2011, Sec. 3.3,
  with the roles of the two blocks exchanged);
  if primal > mu dual then rho *= tau, u /= tau; if dual > mu primal then
  rho /= tau, u *= tau (mu = 10, tau = 2).  ADMM starts from p = z = u = 0.
"""

import numpy as np

from . import operator as op


def _dot(a, b):
    return np.vdot(np.ravel(a), np.ravel(b))


def cg(apply_A, b, x0, n_iter):
    """Plain CG for a Hermitian positive definite operator (Shewchuk 1994).

    ``b`` and ``x0`` are tuples of arrays (the blocks of one vector).
    """
    x = [np.array(v, dtype=np.complex128, copy=True) for v in x0]
    Ax = apply_A(x)
    r = [bi - ai for bi, ai in zip(b, Ax)]
    d = [ri.copy() for ri in r]
    rr = sum(_dot(ri, ri).real for ri in r)
    for _ in range(n_iter):
        Ad = apply_A(d)
        dAd = sum(_dot(di, adi).real for di, adi in zip(d, Ad))
        a = rr / dAd if dAd > 0 else 0.0
        x = [xi + a * di for xi, di in zip(x, d)]
        r = [ri - a * adi for ri, adi in zip(r, Ad)]
        rr_new = sum(_dot(ri, ri).real for ri in r)
        beta = rr_new / rr if rr > 0 else 0.0
        d = [ri + beta * di for ri, di in zip(r, d)]
        rr = rr_new
    return x


def irgn(Fs, U, y, C, q, n_outer=20, n_cg=10, a0=1.0, b0=1.0, decay=0.5,
         floor=1e-6, gamma=1.0, scale_target=100.0, p0=None, alpha0=None):
    """MPI-BL: returns (p, alpha, history of ||y - G(x^n)|| in the scaled units).

    ``p0`` / ``alpha0`` replace the default start (p = 1, alpha = 0); ``p0`` is
    given in the units of the scaled data."""
    y = np.asarray(y, dtype=np.complex128)
    N = Fs.N
    ny = np.linalg.norm(y)
    scale = scale_target / ny if ny > 0 else 1.0
    ys = y * scale
    p = np.ones(N, dtype=np.complex128) if p0 is None else np.array(p0, dtype=np.complex128)
    alpha = np.zeros((C, q), dtype=np.complex128) if alpha0 is None else np.array(alpha0, dtype=np.complex128)
    hist = []
    for n in range(n_outer):
        an = max(a0 * decay ** n, floor)
        bn = max(b0 * decay ** n, floor)
        r = ys - op.forward(Fs, U, alpha, p)
        hist.append(np.linalg.norm(r))
        gp, ga = op.jacobian_adjoint(Fs, U, alpha, p, r)
        rhs = (gp - 2.0 * an * p, ga - 2.0 * bn * alpha)

        def normal(d, p=p, alpha=alpha, an=an, bn=bn):
            jd = op.jacobian(Fs, U, alpha, p, d[0], d[1])
            hp, ha = op.jacobian_adjoint(Fs, U, alpha, p, jd)
            return [hp + 2.0 * an * d[0], ha + 2.0 * bn * d[1]]

        dp, da = cg(normal, rhs, (np.zeros(N), np.zeros((C, q))), n_cg)
        p = p + gamma * dp
        alpha = alpha + gamma * da
    hist.append(np.linalg.norm(ys - op.forward(Fs, U, alpha, p)))
    return p / scale, alpha, np.array(hist)


def irgn_multi(Fs, U, y, C, q, M, n_outer=20, n_cg=10, a0=1.0, b0=1.0, decay=0.5,
               floor=1e-6, gamma=1.0, scale_target=100.0, p0=None, alpha0=None):
    """MPI-BL with M sets of maps (the forward model with extra bilinear terms,
    "Forward Model Extensions"): the unknowns are x = (p_1..p_M, alpha_1..alpha_M),
    Eq. 6's penalties apply alpha_n to every image and beta_n to every set of
    coefficients, and each step solves the same regularised normal equations.

    Start (the paper is silent): p_m = 1 for every set, alpha_1 = 0, and for
    m >= 2 the first basis coefficient of every coil 0.1.  Sets that start
    proportional, (p_m, alpha_m) = c (p_1, alpha_1), stay proportional (their
    Jacobian columns are parallel), so the extra sets must start off that line;
    p_m = 0 with alpha_m = 0 is a stationary point of the block.  M = 1 is
    ``irgn``.  Returns ((M, N) images, (M, C, q) coefficients, residual
    history), images in the units of y."""
    y = np.asarray(y, dtype=np.complex128)
    N = Fs.N
    ny = np.linalg.norm(y)
    scale = scale_target / ny if ny > 0 else 1.0
    ys = y * scale
    P = np.ones((M, N), dtype=np.complex128) if p0 is None else np.array(p0, dtype=np.complex128)
    if alpha0 is None:
        A = np.zeros((M, C, q), dtype=np.complex128)
        A[1:, :, 0] = 0.1
    else:
        A = np.array(alpha0, dtype=np.complex128)
    hist = []
    for n in range(n_outer):
        an = max(a0 * decay ** n, floor)
        bn = max(b0 * decay ** n, floor)
        r = ys - op.forward_multi(Fs, U, A, P)
        hist.append(np.linalg.norm(r))
        gp, ga = op.jacobian_adjoint_multi(Fs, U, A, P, r)
        rhs = (gp - 2.0 * an * P, ga - 2.0 * bn * A)

        def normal(d, P=P, A=A, an=an, bn=bn):
            jd = op.jacobian_multi(Fs, U, A, P, d[0], d[1])
            hp, ha = op.jacobian_adjoint_multi(Fs, U, A, P, jd)
            return [hp + 2.0 * an * d[0], ha + 2.0 * bn * d[1]]

        dP, dA = cg(normal, rhs, (np.zeros((M, N)), np.zeros((M, C, q))), n_cg)
        P = P + gamma * dP
        A = A + gamma * dA
    hist.append(np.linalg.norm(ys - op.forward_multi(Fs, U, A, P)))
    return P / scale, A, np.array(hist)


# --- TV prox (FGP) -----------------------------------------------------------

def grad_fd(x):
    """Forward differences along every axis, zero at the last sample."""
    out = np.zeros((x.ndim,) + x.shape, dtype=np.complex128)
    for ax in range(x.ndim):
        sl_hi = [slice(None)] * x.ndim
        sl_lo = [slice(None)] * x.ndim
        sl_hi[ax] = slice(1, None)
        sl_lo[ax] = slice(0, -1)
        out[(ax,) + tuple(sl_lo)] = x[tuple(sl_hi)] - x[tuple(sl_lo)]
    return out


def grad_fd_adj(P):
    """Adjoint of ``grad_fd`` (minus the discrete divergence)."""
    nd = P.shape[0]
    x = np.zeros(P.shape[1:], dtype=np.complex128)
    for ax in range(nd):
        sl_hi = [slice(None)] * nd
        sl_lo = [slice(None)] * nd
        sl_hi[ax] = slice(1, None)
        sl_lo[ax] = slice(0, -1)
        d = P[ax][tuple(sl_lo)]
        x[tuple(sl_hi)] += d
        x[tuple(sl_lo)] -= d
    return x


def tv(x):
    g = grad_fd(x)
    return float(np.sum(np.sqrt(np.sum(np.abs(g) ** 2, axis=0))))


def tv_prox(v, lam, shape, n_iter):
    """argmin_x (1/2)||x - v||^2 + lam TV(x) by n_iter FGP iterations."""
    b = np.asarray(v, dtype=np.complex128).reshape(shape)
    if lam <= 0:
        return b.ravel().copy()
    nd = len(shape)
    L = 4.0 * nd  # ||grad_fd||^2 <= 4 * ndim
    P = np.zeros((nd,) + tuple(shape), dtype=np.complex128)
    R = P.copy()
    t = 1.0
    for _ in range(n_iter):
        x = b - lam * grad_fd_adj(R)
        Pn = R + grad_fd(x) / (L * lam)
        mag = np.sqrt(np.sum(np.abs(Pn) ** 2, axis=0))
        Pn = Pn / np.maximum(1.0, mag)[None]
        tn = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        R = Pn + ((t - 1.0) / tn) * (Pn - P)
        P, t = Pn, tn
    return (b - lam * grad_fd_adj(P)).ravel()


def project_ball(z, y, eps):
    """Pi_{C(y, eps)}(z) = y + eps (z - y) / max(||z - y||, eps), per coil row."""
    d = z - y
    nrm = np.linalg.norm(d, axis=-1)
    return y + (eps / np.maximum(nrm, eps))[:, None] * d


def admm_tv(Fs, s, y, eps, shape, n_outer=50, n_cg=5, n_tv=10, rho0=1.0, mu=10.0, tau=2.0, trace=None):
    """MPI-L: returns (p, history of (primal, dual, rho)).

    ``trace``, if given, is called as trace(event, rho, u0, uk) after each dual
    update (event "dual") and after each change of rho (event "rho"), with
    copies of the scaled dual variables."""
    s = np.asarray(s, dtype=np.complex128)
    y = np.asarray(y, dtype=np.complex128)
    eps = np.asarray(eps, dtype=np.float64)
    N = Fs.N
    C = s.shape[0]
    M = y.shape[1]
    p = np.zeros(N, dtype=np.complex128)
    u0 = np.zeros(N, dtype=np.complex128)
    uk = np.zeros((C, M), dtype=np.complex128)
    rho = rho0

    def AH(w0, wk):
        return w0 + np.sum(s.conj() * Fs.adj(wk), axis=0)

    def normal(v):
        return [v[0] + np.sum(s.conj() * Fs.adj(Fs.fwd(s * v[0][None, :])), axis=0)]

    hist = []
    Apk = np.zeros((C, M), dtype=np.complex128)
    for _ in range(n_outer):
        z0n = tv_prox(p + u0, 1.0 / rho, shape, n_tv)
        zkn = project_ball(Apk + uk, y, eps)
        rhs = AH(z0n - u0, zkn - uk)
        p_prev, Apk_prev = p, Apk
        (p,) = cg(normal, (rhs,), (p,), n_cg)
        Apk = Fs.fwd(s * p[None, :])
        u0 = u0 + p - z0n
        uk = uk + Apk - zkn
        if trace is not None:
            trace("dual", rho, u0.copy(), uk.copy())
        r_norm = np.sqrt(np.linalg.norm(p - z0n) ** 2 + np.linalg.norm(Apk - zkn) ** 2)
        s_norm = rho * np.sqrt(np.linalg.norm(p - p_prev) ** 2 + np.linalg.norm(Apk - Apk_prev) ** 2)
        hist.append((r_norm, s_norm, rho))
        if r_norm > mu * s_norm:
            rho *= tau
            u0 = u0 / tau
            uk = uk / tau
            if trace is not None:
                trace("rho", rho, u0.copy(), uk.copy())
        elif s_norm > mu * r_norm:
            rho /= tau
            u0 = u0 * tau
            uk = uk * tau
            if trace is not None:
                trace("rho", rho, u0.copy(), uk.copy())
    return p, np.array(hist)


def admm_tv_dynamic(Fs_t, s, y, eps, shape, n_outer=50, n_cg=5, n_tv=10, rho0=1.0, mu=10.0, tau=2.0,
                    trace=None):
    """Dynamic MPI-L (the constrained problem with a spatiotemporal regulariser
    that closes the "Regularized Density Reconstruction" section): T frames
    p_t share the coil maps s, frame t is sampled by its own Fs_t[t], and
        min_p R(p)  s.t.  ||y_{k,t} - F_s^t S_k p_t|| <= eps_{k,t}  for all k, t,
    with R the isotropic TV over the (t, y, x) grid of the T frames (the
    frame axis weighted like the spatial ones; (y, x) alone when T = 1).  The
    ADMM steps of Eq. 11 with A = [I; (F_s^t S_k)_{k,t}], residual-balancing
    rho as in ``admm_tv``.  y (T, C, M), eps (T, C); returns ((T, N) frames,
    history of (primal, dual, rho)).  T = 1 is ``admm_tv``."""
    s = np.asarray(s, dtype=np.complex128)
    y = np.asarray(y, dtype=np.complex128)
    eps = np.asarray(eps, dtype=np.float64)
    T, C, M = y.shape
    N = Fs_t[0].N
    grid = tuple(shape) if T == 1 else (T,) + tuple(shape)
    p = np.zeros((T, N), dtype=np.complex128)
    u0 = np.zeros((T, N), dtype=np.complex128)
    uk = np.zeros((T, C, M), dtype=np.complex128)
    rho = rho0

    def fwd(v):
        return np.stack([Fs_t[t].fwd(s * v[t][None, :]) for t in range(T)])

    def adj(w):
        return np.stack([np.sum(s.conj() * Fs_t[t].adj(w[t]), axis=0) for t in range(T)])

    def normal(v):
        return [v[0] + adj(fwd(v[0]))]

    hist = []
    Apk = np.zeros((T, C, M), dtype=np.complex128)
    for _ in range(n_outer):
        z0n = tv_prox(p + u0, 1.0 / rho, grid, n_tv).reshape(T, N)
        zkn = project_ball((Apk + uk).reshape(T * C, M), y.reshape(T * C, M), eps.reshape(T * C)).reshape(T, C, M)
        rhs = (z0n - u0) + adj(zkn - uk)
        p_prev, Apk_prev = p, Apk
        (p,) = cg(normal, (rhs,), (p,), n_cg)
        Apk = fwd(p)
        u0 = u0 + p - z0n
        uk = uk + Apk - zkn
        if trace is not None:
            trace("dual", rho, u0.copy(), uk.copy())
        r_norm = np.sqrt(np.linalg.norm(p - z0n) ** 2 + np.linalg.norm(Apk - zkn) ** 2)
        s_norm = rho * np.sqrt(np.linalg.norm(p - p_prev) ** 2 + np.linalg.norm(Apk - Apk_prev) ** 2)
        hist.append((r_norm, s_norm, rho))
        if r_norm > mu * s_norm:
            rho *= tau
            u0 = u0 / tau
            uk = uk / tau
            if trace is not None:
                trace("rho", rho, u0.copy(), uk.copy())
        elif s_norm > mu * r_norm:
            rho /= tau
            u0 = u0 * tau
            uk = uk * tau
            if trace is not None:
                trace("rho", rho, u0.copy(), uk.copy())
    return p, np.array(hist)


def project_onto_basis(U, S):
    """alpha_k = (U^H U)^{-1} U^H s_k via a Cholesky factor of the Gram matrix
    (the projection in the Fig. 2 caption).  S is (C, N); returns (C, q)."""
    U = np.asarray(U, dtype=np.complex128)
    G = U.conj().T @ U
    L = np.linalg.cholesky(G)
    rhs = U.conj().T @ np.asarray(S, dtype=np.complex128).T  # (q, C)
    w = np.linalg.solve(L, rhs)
    return np.linalg.solve(L.conj().T, w).T
