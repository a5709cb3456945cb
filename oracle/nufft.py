"""Kaiser-Bessel gridding NUFFT for 2D radial sampling, in FP64.

Test infrastructure (see the package header).

The paper only assumes that a non-Cartesian F is available (Results, "2D
synthetic radial sequences"); it does not fix an implementation.  This module
is the gridding approximation of the direct NUDFT of ``fourier.DirectNUDFT``,
written step by step:

1. divide the image by the kernel's continuous Fourier transform Phi(t)
   (deapodisation), t = j - n/2;
2. zero-pad it, centred, into a G x G grid, G = sigma * n;
3. take the unnormalised centred DFT of the grid (explicit matrices);
4. interpolate at kappa = k G / (2 pi) with the separable kernel
   phi(u) = I0(beta sqrt(1 - (2u/W)^2)) / I0(beta), |u| <= W/2, over the W grid
   points floor(kappa) - W/2 + 1 ... floor(kappa) + W/2 (periodic wrap);
5. scale by N^{-1/2}.

beta = pi sqrt((W/sigma)^2 (sigma - 1/2)^2 - 0.8) (Beatty, Nishimura and Pauly,
IEEE TMI 2005).  Phi(t) = W sinh(z) / (z I0(beta)), z = sqrt(beta^2 - (pi W t/G)^2),
the Fourier transform of phi at frequency t/G cycles per grid unit.

The grid positions kappa and the start indices floor(kappa) are taken in FP64
from the float32 trajectory, so the integer decisions are bit-identical to any
implementation that does the same FP64 multiply.
"""

import numpy as np
from scipy.special import i0

from .fourier import dft, idft


def kb_beta(W, sigma):
    return np.pi * np.sqrt((W / sigma) ** 2 * (sigma - 0.5) ** 2 - 0.8)


def kb_kernel(u, W, beta):
    u = np.asarray(u, dtype=np.float64)
    a = 1.0 - (2.0 * u / W) ** 2
    out = np.zeros_like(u)
    ok = a >= 0.0
    out[ok] = i0(beta * np.sqrt(a[ok])) / i0(beta)
    return out


def kb_deapod(t, W, beta, G):
    """Phi(t): continuous Fourier transform of ``kb_kernel`` at t / G cycles."""
    x = (np.pi * W * np.asarray(t, dtype=np.float64) / G) ** 2
    z2 = beta ** 2 - x
    out = np.empty_like(x)
    pos = z2 > 0
    z = np.sqrt(np.abs(z2))
    out[pos] = np.sinh(z[pos]) / z[pos]
    neg = ~pos
    out[neg] = np.where(z[neg] > 0, np.sin(z[neg]) / np.where(z[neg] > 0, z[neg], 1.0), 1.0)
    return W * out / i0(beta)


def grid_positions(k, G):
    """kappa = k * (G / (2 pi)) in FP64 and the first of the W grid indices.

    Returns (kappa, start) where start = floor(kappa) - W/2 + 1 is a centred
    grid index (add G/2 and wrap to get the array index).  ``k`` is the float32
    trajectory (rad/pixel).
    """
    k64 = np.asarray(k, dtype=np.float32).astype(np.float64)
    kappa = k64 * (float(G) / (2.0 * np.pi))
    return kappa, np.floor(kappa).astype(np.int64)


def gridding_indices(k, G, W):
    """Array index (0..G-1) of the first kernel tap per sample and axis (int32).

    Shape (M, 2), columns (x, y).  Tap a covers (start + a) mod G.
    """
    _, fl = grid_positions(k, G)
    return np.mod(fl - W // 2 + 1 + G // 2, G).astype(np.int32)


class KBGriddingNUFFT:
    def __init__(self, shape, k, W=6, sigma=2.0):
        self.shape = tuple(shape)
        ny, nx = self.shape
        if ny != nx:
            raise ValueError("square grids only")
        self.n = nx
        self.N = ny * nx
        self.W = int(W)
        self.G = int(round(sigma * nx))
        self.beta = kb_beta(W, sigma)
        kappa, fl = grid_positions(k, self.G)
        self.M = kappa.shape[0]
        taps = np.arange(self.W) - self.W // 2 + 1  # centred offsets from floor
        gc = fl[:, :, None] + taps[None, None, :]  # (M, 2, W) centred index
        self.gidx = np.mod(gc + self.G // 2, self.G)  # array index
        self.wts = kb_kernel(kappa[:, :, None] - gc, self.W, self.beta)  # (M, 2, W)
        t = np.arange(nx) - nx // 2
        self.deap = kb_deapod(t, self.W, self.beta, self.G)

    def _grid_fwd(self, img):
        n, G = self.n, self.G
        w = img / (self.deap[:, None] * self.deap[None, :])
        grid = np.zeros((G, G), dtype=np.complex128)
        o = G // 2 - n // 2
        grid[o:o + n, o:o + n] = w
        return dft(grid, 2) * G  # unnormalised centred DFT

    def fwd(self, v):
        v = np.asarray(v, dtype=np.complex128)
        lead = v.shape[:-1]
        vv = v.reshape((-1,) + self.shape)
        gx, gy = self.gidx[:, 0, :], self.gidx[:, 1, :]
        wx, wy = self.wts[:, 0, :], self.wts[:, 1, :]
        out = np.empty((vv.shape[0], self.M), dtype=np.complex128)
        for c in range(vv.shape[0]):
            Wg = self._grid_fwd(vv[c])
            vals = Wg[gy[:, :, None], gx[:, None, :]]  # (M, W, W)
            out[c] = np.einsum("ma,mb,mab->m", wy, wx, vals)
        return out.reshape(lead + (self.M,)) / np.sqrt(self.N)

    def adj(self, y):
        y = np.asarray(y, dtype=np.complex128)
        lead = y.shape[:-1]
        yy = y.reshape((-1, self.M))
        n, G = self.n, self.G
        gx, gy = self.gidx[:, 0, :], self.gidx[:, 1, :]
        wx, wy = self.wts[:, 0, :], self.wts[:, 1, :]
        out = np.empty((yy.shape[0], n, n), dtype=np.complex128)
        o = G // 2 - n // 2
        for c in range(yy.shape[0]):
            grid = np.zeros((G, G), dtype=np.complex128)
            contrib = wy[:, :, None] * wx[:, None, :] * yy[c][:, None, None]
            np.add.at(grid, (np.broadcast_to(gy[:, :, None], contrib.shape),
                             np.broadcast_to(gx[:, None, :], contrib.shape)), contrib)
            img = idft(grid, 2) * G
            out[c] = img[o:o + n, o:o + n] / (self.deap[:, None] * self.deap[None, :])
        return out.reshape(lead + (self.N,)) / np.sqrt(self.N)
