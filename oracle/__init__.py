"""Plain, slow, FP64 CPU oracle for the sliced bucket-elimination QAOA simulator.

TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's CPU
baseline leg import this package; the CUDA library and its Python binding never
do, and nothing here imports them. The two sides share only the seeded input
generators (paper_2012_02430_gb300.inputs), which hold none of the method's
arithmetic.

Modules (each cites the passage of the paper it follows):
  network      Sec. IV.A-B: gates as tensors, the line graph with diagonal gates
  ordering     Sec. IV.B, Sec. V.A.1: greedy min-fill / min-degree, width
  slicing      Sec. VI.C-D, Alg. 1: step-dependent slicing search
  contract     Alg. 1, Eq. 2: bucket elimination with explicit slicing
  ledger       Alg. 1: per-step FLOP/byte accounting of the sliced schedule
  statevector  Sec. III.A: brute-force 2^N statevector
  energy       Sec. III.A-B: lightcone energy and the closed-form p=1 energy
"""
