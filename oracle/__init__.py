"""FP64 CPU oracle for the closed-shell Kohn-Sham SCF of arXiv 2311.01135.

TEST INFRASTRUCTURE ONLY.  The tests, `__graft_entry__.smoke()` and the
benchmark's `cpu_baseline` / `--impl reference` legs are the only code that may
import, call, link or execute anything under this directory.  The product
(the CUDA library and its Python binding) shares no code with it.

Modules:
  basis  - STO-3G and 6-31G tables and shell model (packing order)
  ints   - FP64 McMurchie-Davidson integrals (ints.c), Schwarz screening, the
           canonical packed two-electron store
  grid   - Treutler-Ahlrichs M4 radial x Gauss-Legendre/uniform angular
           atom-centred grids with Becke partitioning
  xc     - B3LYP(VWN5) energy density; potentials by complex-step
           differentiation of the energy density
  scf    - AO evaluation, J/K, V_xc and the SCF driver (SAD or core guess, DIIS)

Parity status per function is listed in the module headers; every function
here has at least one pin in tests/test_oracle_*.py except the whole-method
absolute B3LYP energy, whose parity is unpinned beyond the invariants (the
paper prints no energies), and the single outer exponents of the 6-31G heavy
atoms (parity unpinned).
"""
