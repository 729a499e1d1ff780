"""CPU oracle of the close-coupling Hamiltonian build and its eigenpairs.

ORACLE / TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and
the `cpu_baseline` / reference leg of `bench.py` may import anything here.  The
product path (the CUDA library and its Python binding) never imports it and
shares no code with it.

Modules:
  fock     second-quantised Hamiltonian applied by definition (tiny systems)
  brute    uncontracted determinant build + explicit T^T H T (Eq. 3-5)
  coracle  ctypes front end of hb_oracle.c: bitstring Slater-Condon rules
           (Section 2.1) and the structured prototype / contract / expand build
           (Eq. 6-8, classes 1-8)
  eig      dense eigen reference and a plain Davidson iteration
  mlp      FP64 reference of the preconditioner-correction network
"""
