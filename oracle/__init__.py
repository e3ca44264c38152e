"""FP64 oracle for the singly periodic Spectral Ewald (SE1P) method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package.
The product path (the CUDA library and its Python binding) never imports it
and shares no code, header, table or constant generator with it.

  direct.py / ewald1p_direct.c  plain direct Ewald1P sums (Section 2.1, App. A)
  se1p_algorithm.py             numpy restatement of Algorithms 1-3 (Section 3)
"""
