"""CPU FP64 oracle for the NAO band step -- TEST INFRASTRUCTURE ONLY.

This package is the slow, plain reference that the CUDA path is checked against.  Only the
test-suite, the smoke check and the CPU-baseline leg of the benchmark may import it; the
product path (the C-ABI library and its Python binding) never does, and shares no code,
table or helper with it.

Every function follows the paper's Band_DFT_Col (Sec. 3, Parts 1-6) and its Eigen_HH
steps (Householder tridiagonalization, Procedures 1-6; an implicit-QL tridiagonal eigensolver;
rearrangement of eigenvectors; normalization), written out in numpy, float64/complex128.

Pins (tests/test_oracle_pins.py) tie it to things other than itself: closed-form chain
bands, exact characteristic-polynomial roots for n <= 6, hand-computed Bloch sums,
closed-form Fermi levels and plane-wave density matrices, and invariants.
"""
from .band import (  # noqa: F401
    bloch_sum,
    householder_tridiagonalize,
    tridiagonal_eigensolve,
    rearrange_eigenvectors,
    eigen_hh,
    generalized_eigensolve,
    fermi_occupations,
    density_matrix,
    band_step,
)
