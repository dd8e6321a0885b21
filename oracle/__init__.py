"""FP64 CPU oracle for the matrix-free Q_k Laplacian (test infrastructure only).

This package is the independent checker of the GPU library.  It is plain,
slow and written to be read against the method's definition:

* the bilinear form a(u, v) = (a(x) grad u, grad v) of Eq. (1) (Sec. 2.4),
  extended with the variable coefficient a(x) of the workloads;
* the cell loop of the step-4 listing (Sec. 2.4): element matrix and
  right-hand side by full, non-factorised quadrature;
* the matrix-free statement of Sec. 3.6: the operator action equals the
  action of the assembled matrix, so the oracle assembles the global sparse
  matrix, condenses the constraints and multiplies;
* the single-precision solver wrapped in a double-precision correction of
  Sec. 6.1, and the Chebyshev smoother named in Sec. 3.5 / Sec. 6.1.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import, call, link or execute anything in this package.
It shares no code with the CUDA library and never imports it.

Modules: ``rules`` (1D quadrature and Lagrange bases), ``mesh``
(structured and octree meshes, DoF numbering, constraints), ``fem``
(assembly, condensation, SpMV, PCG, Chebyshev, defect correction, L2
error), ``_native`` (ctypes binding of ``oracle.c``).
"""
