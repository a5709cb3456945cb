"""Writes the reconstruction fixtures `recon_<workload>.npz` with the FP64 oracle.

For each 2D workload (Cartesian, or radial with the oracle's FP64 Kaiser-Bessel
gridding NUFFT): seeded truth (the smooth orthonormal stand-in
basis, decaying random coefficients, a random-ellipse phantom), data
y = F_s(U alpha_k (.) p) + complex Gaussian noise at the workload's SNR (the
forward model of Eq. 5), rounded to complex64 as the GPU receives it, and the
oracle's reconstruction of it: MPI-BL (IRGN, Eq. 6; 20 outer x 10 CG
iterations) and then MPI-L (ADMM-TV, Eqs. 8-11; 50 outer x 5 CG x 10 TV
iterations) with the MPI-BL maps and eps_k = sigma sqrt(M).  The oracle runs
in its FFT fast mode (equal to the explicit DFT matrices, see
test_fast_mode_equals_explicit_matrices).  Only oracle/ and workloads/ are
used.  `bench.py` reads these files to time the GPU solvers on the same data
and report their distance from the oracle's reconstructions.

    python tests/golden/make_recon_golden.py [workload ...]
"""

import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as w  # noqa: E402
from oracle import fourier, nufft, operator as op, solvers  # noqa: E402

DEFAULT = ["cart2d_64_c4_q32", "cart2d_256_c16_q128", "cart2d_320_c16_q100", "radial2d_256_c12_q96"]


def main(names):
    for name in names:
        t0 = time.time()
        cfg, U, samp, a_true, p_true = w.recon_case(name)
        ny, nx = cfg["dims"]
        if cfg["kind"] == "radial":
            Fs = nufft.KBGriddingNUFFT((ny, nx), samp.astype(np.float64), W=cfg["W"], sigma=cfg["sigma"])
            n_samp = samp.shape[0]
        else:
            Fs = fourier.CartesianSamplingFFT((ny, nx), samp)
            n_samp = samp.size
        y0 = op.forward(Fs, U, a_true, p_true)
        sig = w.noise_sigma_for_snr(y0, cfg["snr_db"])
        y = (y0 + w.complex_noise(y0.shape, sig, seed=w.RECON_SEED + 4)).astype(np.complex64)
        y64 = y.astype(np.complex128)
        eps = np.full(cfg["C"], sig * np.sqrt(n_samp))
        p_bl, a_bl, hist = solvers.irgn(Fs, U, y64, cfg["C"], cfg["q"], n_outer=cfg["n_irgn"], n_cg=10)
        s_bl = op.expand(U, a_bl).astype(np.complex64).astype(np.complex128)
        p_l, _ = solvers.admm_tv(Fs, s_bl, y64, eps, (ny, nx), n_outer=cfg["n_admm"], n_cg=5, n_tv=10)
        out = os.path.join(HERE, f"recon_{name}.npz")
        np.savez_compressed(out, y=y, eps=eps, alpha_bl=a_bl.astype(np.complex64), p_bl=p_bl.astype(np.complex64),
                            p_l=p_l.astype(np.complex64), hist_bl=hist)
        print(f"{name}: {out} ({os.path.getsize(out) / 1e6:.1f} MB, {time.time() - t0:.0f} s)", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:] or DEFAULT)
