"""FP64 CPU oracle for the domain-wall solver.

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow reference every
result of the CUDA library is checked against.  Only the test-suite, the smoke
check (``__graft_entry__.smoke``) and the benchmark's CPU-baseline and
reference legs import, call, link or run anything in this directory; the
library's product path never does.  The oracle shares no code with the CUDA
implementation (no kernels, headers, helpers, tables or constants); the only
common dependency is the seeded input generator
``paper_2602_14454_gb300.inputs``, which contains no solver arithmetic.

Modules
  _clib   builds and loads ``wilson.c`` (the 4D Wilson operator in plain C)
  dwf     domain-wall and Neff operators written block by block from the
          printed matrices, even-odd Schur route, source/projection maps,
          CGNR, dense helpers
  net     the gauge-covariant stencil network (forward, loss, backward) in FP64

Every function says which passage of the paper it follows.  Functions with
no independent check say "parity unpinned" in their docstring.
"""
