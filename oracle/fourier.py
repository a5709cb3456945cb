"""Sampling operators F_s in FP64 (Eq. 1: F = I_C (x) F_s, F_s in C^{K x N}).

Test infrastructure (see the package header).

The paper leaves the DFT convention open.  Reading taken here: forward sign
e^{-i}, centred indices (j - n/2) on both the image and the k-space axis, and a
unitary scale n^{-1/2} per axis, so that the fully sampled F is unitary
(Parseval holds).  Each axis transform is an explicit n x n matrix product; no
FFT is used.
"""

import numpy as np


def centered_dft_matrix(n):
    """F[k, j] = n^{-1/2} exp(-2 pi i (k - n/2)(j - n/2) / n)."""
    t = np.arange(n) - n // 2
    return np.exp(-2j * np.pi * np.outer(t, t) / n) / np.sqrt(n)


def dft(v, ndim):
    """Centred unitary DFT over the last ``ndim`` axes of v (separable matrices)."""
    out = np.asarray(v, dtype=np.complex128)
    for ax in range(out.ndim - ndim, out.ndim):
        F = centered_dft_matrix(out.shape[ax])
        out = np.moveaxis(np.tensordot(out, F, axes=([ax], [1])), -1, ax)
    return out


def idft(v, ndim):
    """Adjoint (= inverse) of ``dft``."""
    out = np.asarray(v, dtype=np.complex128)
    for ax in range(out.ndim - ndim, out.ndim):
        F = centered_dft_matrix(out.shape[ax]).conj()
        out = np.moveaxis(np.tensordot(out, F, axes=([ax], [0])), -1, ax)
    return out


class CartesianSampling:
    """F_s = (row selection by the sorted raster index list) o (centred DFT).

    ``shape`` is the image grid ((ny, nx) or (nz, ny, nx)); ``idx`` the sorted
    flat indices of the sampled k-space points (centred order).
    """

    def __init__(self, shape, idx):
        self.shape = tuple(shape)
        self.idx = np.asarray(idx, dtype=np.int64)
        self.N = int(np.prod(self.shape))
        self.M = int(self.idx.size)

    def fwd(self, v):
        """v: (..., N) -> (..., M)."""
        v = np.asarray(v, dtype=np.complex128)
        lead = v.shape[:-1]
        k = dft(v.reshape(lead + self.shape), len(self.shape)).reshape(lead + (self.N,))
        return k[..., self.idx]

    def adj(self, y):
        """y: (..., M) -> (..., N): zero-fill then inverse centred DFT."""
        y = np.asarray(y, dtype=np.complex128)
        lead = y.shape[:-1]
        k = np.zeros(lead + (self.N,), dtype=np.complex128)
        k[..., self.idx] = y
        return idft(k.reshape(lead + self.shape), len(self.shape)).reshape(lead + (self.N,))


class CartesianSamplingFFT(CartesianSampling):
    """The same F_s as ``CartesianSampling`` with the centred DFT taken by FFTs
    (``scipy.fft``, ``workers`` threads): the oracle's fast mode, used only to
    time a CPU baseline.  The centred transform is the plain DFT of the
    index-shifted array, shifted back: F_c v = fftshift(fft(ifftshift(v))) with
    the unitary scale; pinned against the explicit matrices by the tests."""

    def __init__(self, shape, idx, workers=None):
        super().__init__(shape, idx)
        import os

        self.workers = workers or os.cpu_count()

    def _fft(self, v, inverse):
        import scipy.fft as sfft

        axes = tuple(range(v.ndim - len(self.shape), v.ndim))
        v = sfft.ifftshift(v, axes=axes)
        v = (sfft.ifftn if inverse else sfft.fftn)(v, axes=axes, norm="ortho", workers=self.workers)
        return sfft.fftshift(v, axes=axes)

    def fwd(self, v):
        v = np.asarray(v, dtype=np.complex128)
        lead = v.shape[:-1]
        k = self._fft(v.reshape(lead + self.shape), False).reshape(lead + (self.N,))
        return k[..., self.idx]

    def adj(self, y):
        y = np.asarray(y, dtype=np.complex128)
        lead = y.shape[:-1]
        k = np.zeros(lead + (self.N,), dtype=np.complex128)
        k[..., self.idx] = y
        return self._fft(k.reshape(lead + self.shape), True).reshape(lead + (self.N,))


class DirectNUDFT:
    """Direct non-uniform DFT for 2D radial sampling.

    y_m = N^{-1/2} sum_j v_j exp(-i (kx_m tx_j + ky_m ty_j)), t = index - n/2,
    k in radians per pixel.  On Cartesian grid points k = 2 pi (kk - n/2)/n this
    equals the centred DFT above.  The exponential separates over x and y, so
    the sum is done as one matrix product per axis (exact, no approximation).
    """

    def __init__(self, shape, k):
        self.shape = tuple(shape)
        ny, nx = self.shape
        self.N = ny * nx
        k = np.asarray(k, dtype=np.float64)
        self.M = k.shape[0]
        tx = np.arange(nx) - nx // 2
        ty = np.arange(ny) - ny // 2
        self.Ex = np.exp(-1j * np.outer(k[:, 0], tx))  # (M, nx)
        self.Ey = np.exp(-1j * np.outer(k[:, 1], ty))  # (M, ny)

    def fwd(self, v):
        v = np.asarray(v, dtype=np.complex128)
        lead = v.shape[:-1]
        ny, nx = self.shape
        vv = v.reshape((-1, ny, nx))
        out = np.empty((vv.shape[0], self.M), dtype=np.complex128)
        for c in range(vv.shape[0]):
            A = vv[c] @ self.Ex.T  # (ny, M): sum over x
            out[c] = np.einsum("my,ym->m", self.Ey, A)
        return out.reshape(lead + (self.M,)) / np.sqrt(self.N)

    def adj(self, y):
        y = np.asarray(y, dtype=np.complex128)
        lead = y.shape[:-1]
        ny, nx = self.shape
        yy = y.reshape((-1, self.M))
        out = np.empty((yy.shape[0], ny, nx), dtype=np.complex128)
        for c in range(yy.shape[0]):
            out[c] = (self.Ey.conj() * yy[c][:, None]).T @ self.Ex.conj()
        return out.reshape(lead + (self.N,)) / np.sqrt(self.N)
