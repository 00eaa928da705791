"""Shamir domain-wall (five-dimensional chiral) Dirac operator.

The paper benchmarks the domain-wall operator as the "L_s replicated Wilson
dslash" (Sec. 3, Table 4) and notes that the gauge field is reused L_s times
(Sec. 3, Fig. xc30 caption); it does not write the operator down. Textbook
Shamir form, with the reading chosen here (5D field psi[s, ...], s = 0..L_s-1):

  D_DW psi(s) = D_W(-M5) psi(s) + psi(s) - P_- psi(s+1) - P_+ psi(s-1)
              = M5op psi(s) - H psi(s) / 2,

  M5op = (5 - M5) - P_- S_up - P_+ S_down      (site-local in 4D)
  (S_up psi)(s)   = psi(s+1),  (S_up psi)(L_s-1) = -mf psi(0)
  (S_down psi)(s) = psi(s-1),  (S_down psi)(0)   = -mf psi(L_s-1)

The hop H acts on each s-slice with the same links. P_+- = (1 +- gamma_5)/2.
Adjoint: S_up^dag = S_down, so M5op^dag = (5 - M5) - P_- S_down - P_+ S_up and
D_DW^dag = M5op^dag - H^dag / 2.

Even-odd on the 4D parity, with M5op the (site-diagonal) even-even and
odd-odd block:

  M_hat = M5op - H_eo M5op^-1 H_oe / 4,
  b_hat_e = b_e + H_eo M5op^-1 b_o / 2,   x_o = M5op^-1 (b_o + H_oe x_e / 2).

M5op^-1 is applied by a dense LU solve of the L_s x L_s matrix of each
chirality. Pins: Gamma_5 R hermiticity, the L_s = 1 reduction to Wilson with
mass 1 - M5 + mf, the closed-form free-field determinant on a periodic 2^4
lattice, an explicit-loop dense matrix on a small 5D lattice, and the
full-system residual of the even-odd solve (tests/test_oracle_dwf.py).
"""
from __future__ import annotations

import numpy as np

from . import wilson
from .gamma import GAMMA5, P_MINUS, P_PLUS, spin_apply


def s_up(psi: np.ndarray, mf: float) -> np.ndarray:
    out = np.roll(psi, -1, axis=0)
    out[-1] *= -mf
    return out


def s_down(psi: np.ndarray, mf: float) -> np.ndarray:
    out = np.roll(psi, 1, axis=0)
    out[0] *= -mf
    return out


def m5op(psi: np.ndarray, M5: float, mf: float, dagger: bool = False) -> np.ndarray:
    """Site-local fifth-dimension part of D_DW (diagonal 5 - M5)."""
    up, down = s_up(psi, mf), s_down(psi, mf)
    if dagger:
        up, down = down, up
    return (5.0 - M5) * psi - spin_apply(P_MINUS, up) - spin_apply(P_PLUS, down)


def m5op_matrix(Ls: int, M5: float, mf: float, chirality: int, dagger: bool = False):
    """L_s x L_s matrix of M5op on one chirality (+1: spins 0,1; -1: spins 2,3)."""
    d = 5.0 - M5
    up = np.zeros((Ls, Ls))
    for s in range(Ls):
        if s + 1 < Ls:
            up[s, s + 1] = 1.0
        else:
            up[s, 0] = -mf
    down = up.T.copy()
    shift_op = down if chirality > 0 else up
    if dagger:
        shift_op = shift_op.T
    return d * np.eye(Ls) - shift_op


def m5op_inv(psi: np.ndarray, M5: float, mf: float, dagger: bool = False) -> np.ndarray:
    """M5op^-1 psi by a dense LU solve per chirality along the s axis."""
    Ls = psi.shape[0]
    out = np.empty_like(psi)
    for chir, spins in ((+1, slice(0, 2)), (-1, slice(2, 4))):
        mat = m5op_matrix(Ls, M5, mf, chir, dagger)
        part = psi[..., spins, :]
        rhs = part.reshape(Ls, -1)
        out[..., spins, :] = np.linalg.solve(mat, rhs).reshape(part.shape)
    return out


def dirac(U, psi, M5, mf, bc, dagger: bool = False):
    """D_DW psi for a 5D field psi[s, t, z, y, x, spin, colour]."""
    return m5op(psi, M5, mf, dagger) - 0.5 * wilson.hop(U, psi, bc, dagger)


def dirac_dag_dirac(U, psi, M5, mf, bc):
    return dirac(U, dirac(U, psi, M5, mf, bc), M5, mf, bc, dagger=True)


def gamma5_reflect(psi: np.ndarray) -> np.ndarray:
    """(R gamma_5 psi)(s) = gamma_5 psi(L_s - 1 - s)."""
    return spin_apply(GAMMA5, psi[::-1])


# --------------------------------------------------------------- even / odd

def schur(U, psi_e, M5, mf, bc, dagger: bool = False):
    """M_hat psi_e = M5op psi_e - H_eo M5op^-1 H_oe psi_e / 4 (or its adjoint)."""
    tmp = wilson.hop_eo(U, psi_e, bc, 1, dagger)
    tmp = m5op_inv(tmp, M5, mf, dagger)
    return (m5op(wilson.restrict(psi_e, 0), M5, mf, dagger)
            - 0.25 * wilson.hop_eo(U, tmp, bc, 0, dagger))


def schur_dag_schur(U, psi_e, M5, mf, bc):
    return schur(U, schur(U, psi_e, M5, mf, bc), M5, mf, bc, dagger=True)


def prepare_source(U, b, M5, mf, bc):
    tmp = m5op_inv(wilson.restrict(b, 1), M5, mf)
    return wilson.restrict(b, 0) + 0.5 * wilson.hop_eo(U, tmp, bc, 0)


def reconstruct(U, x_e, b, M5, mf, bc):
    rhs = wilson.restrict(b, 1) + 0.5 * wilson.hop_eo(U, x_e, bc, 1)
    return wilson.restrict(x_e, 0) + m5op_inv(rhs, M5, mf)
