"""Plain FP64 CPU oracle for the treecode boundary-element Poisson-Boltzmann solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call, link
or run anything in this package: only the tests, the smoke check and the
benchmark's CPU-baseline leg use it.  It shares no code with the CUDA library
(no kernels, headers, helpers, tables or constant generators); the two read
the same synthetic inputs from ``synth`` and nothing else.

Every function cites the part of Cooper, Bardhan & Barba (arXiv:1309.4018,
"A biomolecular electrostatics solver using Python, GPUs and boundary elements
that can handle solvent-filled cavities and Stern layers") it follows.

Parity status: every function is pinned by a test against something other
than itself (closed forms, quadrature exactness, brute-force integration,
invariants); see tests/test_oracle_*.py.
"""
