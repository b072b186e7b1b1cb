"""Oracle: a plain, slow, FP64 CPU restatement of the paper's method.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import, call, link or run anything in this package.  The product path (the CUDA
library and its binding) never uses it, and it shares no code with that path: the two meet only
through the seeded inputs of the ``workloads`` module.

Modules
  layers      discretisation of the empty grating, the 7x7-block matrix A (Sec. 3, Eq. matA),
              its SVD pseudo-inverse (Sec. 5, Eq. applypA), Bragg amplitudes and flux (Sec. 6)
  inclusions  disk scattering coefficients (Sec. 4.1), the translation operator T (Sec. 4.2,
              Eq. trans), the coupling matrices B and C (Sec. 5, Eqs. matB, matC)
  solver      the preconditioned Schur system (Sec. 5) solved densely by LU or matrix-free by GMRES
  m2l         a small C/OpenMP direct-sum translation used by the matrix-free solver at large M

Every function cites the passage it follows.  Bessel and Hankel functions come from
scipy.special (a library primitive).  Readings of passages that are ambiguous are listed in the
docstrings where they are used.
"""
