"""Site-by-site product of fields of 3x3 complex matrices, z(s) = x(s) y(s).

This is the first kernel of the paper's performance section (Sec. 5): a
product of two LatticeColourMatrix fields, benchmarked against memory
footprint. The definition is the ordinary matrix product at every site,
z_ik = sum_j x_ij y_jk, with no coupling between sites; 198 real flops per
site (9 entries, each 3 complex products and 2 complex additions).

Fields are arrays ``[..., 3, 3]`` of complex128 (any leading site shape).
Pins (tests/test_oracle_su3.py): an explicit triple loop on a small field, the
identity, SU(3) closure (unitary with unit determinant), the determinant and
trace-cyclicity identities and the non-commutativity that a transposed
operand would break.
"""
from __future__ import annotations

import numpy as np

FLOP_PER_SITE = 198


def su3_mul(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """z = x y at every site (matrix product over the last two axes)."""
    return np.matmul(x, y)
