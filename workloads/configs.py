"""The five synthetic workloads the encoding operator is built and measured on.

Shapes follow the paper's experiments (2D Cartesian brain slices, golden-angle
radial, Table S1's 3D volume) scaled to the sizes listed here; every input is
seeded and synthetic.
"""

WORKLOADS = {
    "cart2d_64_c4_q32": dict(
        kind="cartesian", dims=(64, 64), C=4, q=32, mask="vd_lines", R=3, acs=16,
        snr_db=30.0, n_irgn=20, n_admm=50,
    ),
    "cart2d_256_c16_q128": dict(
        kind="cartesian", dims=(256, 256), C=16, q=128, mask="poisson", R=6, calib=(24, 24),
        snr_db=30.0, n_irgn=20, n_admm=50,
    ),
    # the paper's 2D Cartesian timing shape (320 x 320, 16 coils, R = 2 with 16
    # ACS lines, q = 100), used for reconstruction times
    "cart2d_320_c16_q100": dict(
        kind="cartesian", dims=(320, 320), C=16, q=100, mask="vd_lines", R=2, acs=16,
        snr_db=30.0, n_irgn=20, n_admm=50,
    ),
    "radial2d_256_c12_q96": dict(
        kind="radial", dims=(256, 256), C=12, q=96, spokes=64, readout=512, W=6, sigma=2.0,
        snr_db=30.0, n_irgn=20, n_admm=50,
    ),
    "batched2d_64slices": dict(
        kind="batched", slices=64, sizes=(128, 192, 256, 320), coils=(8, 16, 32),
        q_by_size={128: 64, 192: 96, 256: 128, 320: 160}, R_range=(4, 8),
    ),
    "cart3d_128x128x96_c32_tucker256": dict(
        kind="cartesian3d", dims=(96, 128, 128), C=32, q=256, ranks=(32, 40, 40),
        mask="poisson3d", R=8, calib=(24, 24),
    ),
}


def workload(name):
    return dict(WORKLOADS[name], name=name)
