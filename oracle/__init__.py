"""CPU oracle for the random-circuit state-vector method (arXiv:1804.04797).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code,
constants or tables with the CUDA library; the two meet only on the seeded
inputs from ``paper_1804_04797_gb300.inputs`` (lattice shapes, seeds, bitstrings).

Modules
  circuit  -- independent re-implementation of the lattice circuit rules (§2, gate set
              and fixed CZ positions per layer) used to check the library's generator.
  statevec -- complex128 numpy state vector: the pair update of §2, CZ, the
              brute-force Kronecker-product unitary, branch (cut) amplitudes by the
              CZ = P0 (x) I + P1 (x) Z decomposition (§2, Fig. 2), reductions.
  csim     -- ctypes loader of ``sv_oracle.c`` (the same complex128 algorithm in C
              with OpenMP, for 24-30 qubit cases and the CPU baseline timing).
"""
