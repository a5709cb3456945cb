"""FP64 CPU oracle for the Maxwell Parallel Imaging encoding operator.

TEST INFRASTRUCTURE.  This package is a plain, slow, obviously correct
complex128 restatement of what the paper computes.  Only the test suite,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` leg
of ``bench.py`` may import it.  The CUDA library shares no code with it: no
kernels, headers, tables or pre/post-processing.  The only shared module is
``workloads`` (seeded inputs, none of the method's arithmetic).

Modules
-------
fourier   centred unitary DFT by explicit separable DFT matrices, Cartesian
          sampling (Eq. 1 and the definition of F_s), direct non-uniform DFT.
nufft     Kaiser-Bessel gridding NUFFT in FP64 (the radial F_s realised the way
          the GPU realises it, used for the tight parity bound).
operator  basis expansion, G, its adjoint, the Jacobian and its adjoint
          (Eqs. 1, 3, 5, 7 and the Jacobian-adjoint display after Eq. 7).
basis     Maxwell basis from dipole sources through the free-space Green's
          function, circular polarisation and a randomized SVD
          ("Maxwell Regularization" section).
tucker    HOSVD of the basis tensor and Tucker-factored expansion
          ("A Compression Scheme for Maxwell Basis" section).
solvers   IRGN with CG on the normal equations (MPI-BL, Eq. 6), scaled ADMM
          with TV prox and l2-ball projection (MPI-L, Eqs. 8-11), Gram /
          Cholesky basis projection (Fig. 2 caption).

Equation numbers count the numbered displays of the paper in order (Eq. 1 the
forward model y = F S p + n, ..., Eq. 11 the ADMM updates, Eqs. 17-18 the
free-space dyadic Green's functions, Eq. 21 the Tucker error bound).

Parity status: every function is pinned by a ``-m "not gpu"`` test against a
closed form, an invariant or brute force, except the reconstruction quality
against ground truth, which the paper reports only as figures ("parity
unpinned" for that comparison only).
"""
