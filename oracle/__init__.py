"""FP64 reference oracle — TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously correct CPU restatement of what the circuit engine
computes (arXiv 2205.10091, "TensorCircuit"), in complex128/float64 numpy.
Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA engine; the only
common module is the seeded input generator
``paper_2205_10091_b300.workloads``, which describes work and holds none of
the method's arithmetic.

Modules:
  statevector  gate definitions, gate application, Pauli-sum expectation
  gradients    parameter-shift and central finite-difference gradients
  noise        Philox4x32-10, Pauli-channel trajectory selection, density matrix
  tensornet    light cone, naive pairwise contraction, windowed state vector

Parity status per function is stated in each module header.
"""
