"""FP64 CPU oracle for the rid-preconditioned Davidson solve of the TDDFT response problem.

TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
Python binding) imports, links or runs anything in this package; only the test
suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg of
``bench.py`` use it.  It shares no code with the CUDA path: its only common
dependency is the seeded input generator in ``synth/``.

Contents
  operators  the response Hessians of Eq. hessian (f^xc = 0) built densely from
             the four-index definition (Eq. pqrs), and the same operators as
             matrix-free products over the density-fitted factors; the ris
             operator of Eq. TDDFT-ris_approx with the exchange energy window
             of Sec. 3.1
  dense      plain-definition results on small inputs: TDA eigenpairs (Eq. TDA),
             Casida eigenpairs (Eq. Casida), dynamic polarizability
             (Eq. TDDFT_polar)
  davidson   the preconditioned Davidson algorithm of Sec. 2.1 (Eqs. 1-4,
             Eq. residual, Eq. precondition) for TDA, Casida and the
             polarizability linear systems, with the diagonal and the rid
             preconditioners

Every function cites the passage it follows.  Parity status of each function
is listed in the module docstrings; functions without an external pin say
"parity unpinned".
"""
