"""Oracle: a plain, slow, CPU FP64 restatement of the method of arXiv 2102.03515.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  It shares
no code with the CUDA library ``paper_2102_03515_gb300`` and never imports it.

* :mod:`oracle.core`  -- C core (Kuhn mesh, P1 assembly, Jacobi-PCG, dense
  Cholesky, error norms), loaded through ctypes.
* :mod:`oracle.amg`   -- numpy/scipy smoothed-aggregation hierarchy, V-cycle and
  (flexible) PCG.
* :mod:`oracle.refine` -- longest-edge bisection with conforming closure (the local
  refinement of the adaptive runs, Sec. 4.2-4.3).
"""
