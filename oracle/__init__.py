"""FP64 CPU oracle for the ppRPA hot path.

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
timed CPU-baseline leg of the benchmark may import this package; the product
path (the CUDA library and its Python binding) never does, and this package
imports nothing from the product.

Every function cites the passage of the LibppRPA paper (arXiv 2512.12515) it
follows.  Matrix elements are built element by element from their
definitions and diagonalised densely, so a reader can check each step
against the equations by eye.

Parity status per function (what pins it; see tests/test_oracle_pins.py):

* ao_to_mo, eri_phys, build_matrix, solve_full, solve_full_shifted,
  correlation_energy: pinned by the spin-orbital brute force, the
  two-electron determinant CI, the B = 0 limit, root counting, the
  correlation-energy identity, the uniform-shift identity and the
  second-order (MP2-type) limit.
* grad_omega: pinned by central finite differences and by the trace rule of
  the two-electron density matrix.
* grad_omega_ab (alpha-beta subspace): pinned by central finite differences of its
  roots (addition and removal) and by the uniform-shift rule (each spin's energy
  gradient sums to 1).
* grad_ao: pinned by central finite differences of a root through the whole
  chain (AO integrals or MO coefficients -> L -> M -> omega).
* ri_sigma / davidson: pinned by the explicit matrix (sigma) and by full
  diagonalisation (Davidson roots).
* fractional_slots, fractional_integrals: pinned by the spin-orbital brute force
  written element by element from the fractional matrix elements (its spectrum is the
  union of the folded singlet roots and three copies of the triplet roots), and by
  integer occupations reducing to the ordinary path.
* build_matrix_ab (spin-unrestricted alpha-beta subspace): pinned by the
  restricted limit (alpha = beta: singlet roots plus one copy of the triplet
  roots) and by the spin-orbital brute force of a spin-unrestricted reference
  (its spectrum is the union of the three subspaces).
* two_e_density, nto: pinned by the trace rule, by the epsilon gradient (the
  diagonal), by reconstructing X and Y from their NTOs and by the identity
  X X^T + X^T X = C^p1 L C^p1^T + C^p2 L C^p2^T between the two definitions.
* two_e_density_ab, nto_ab (alpha-beta subspace): pinned by each spin's trace rule,
  by the alpha and beta energy gradients of grad_omega_ab (the diagonals), by
  reconstructing X and Y from their NTOs and by the weight sum rule.
* matrix_rows / explicit_matrix_ri, shifted_lambda_min, roots_near (stability at
  workload sizes): pinned by build_matrix (rows), dense symmetric eigenvalues of
  M - mu W, and the dense spectrum of solve_full (roots and their norm signs).
* eigenvector phase: fixed by convention (largest-magnitude component
  positive); parity unpinned beyond that convention.
"""
from .pprpa_ref import (  # noqa: F401
    active_orbitals,
    fractional_slots,
    fractional_integrals,
    ao_to_mo,
    ao_to_mo_rows,
    grad_ao,
    pair_list,
    eri_phys,
    build_matrix,
    build_matrix_ab,
    matrix_blocks,
    solve_full,
    solve_full_shifted,
    correlation_energy,
    grad_omega,
    grad_omega_ab,
    two_e_density_diag,
    two_e_density,
    two_e_density_ab,
    nto,
    nto_ab,
    nto_weights,
    diag_of_matrix,
)
from .brute import (  # noqa: F401
    spinorb_matrix,
    spinorb_matrix_fractional,
    spinorb_matrix_unrestricted,
    two_electron_ci,
    mp2_pair_energy,
)
from .davidson_ref import ri_sigma, ri_sigma_rows, davidson  # noqa: F401
from .stability import (  # noqa: F401
    matrix_rows, explicit_matrix_ri, shifted_lambda_min, roots_near, block_shift_window,
    classified_spectrum)
