"""Plain FP64 CPU oracle for the CV-ADAPT-VQE hot path (arXiv 2606.05297).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
the cpu_baseline / reference legs of bench.py, never by the product package.
It shares no code with paper_2606_05297_gb300 (the CUDA path); the only module
both sides read is paper_2606_05297_gb300.workloads, which generates seeded
synthetic inputs and holds none of the method's arithmetic.

Modules:
  core       ctypes binding of cvq_oracle.c (sector, ladder strings, expm,
             energy, Eq. (grad) screen, adjoint ansatz gradient)
  operators  Hamiltonian and pool generators as ladder strings (Sec. II.B, III)
  dense      dense full-Fock-space Kronecker reference and exact diagonalisation
  bfgs       BFGS with strong-Wolfe line search (Sec. IV.A optimiser)
  adapt      CV-ADAPT-VQE loop (Sec. IV.B) on top of core
"""
