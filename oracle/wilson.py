"""Wilson-Dirac operator, its hopping term and the even-odd Schur complement.

Definitions (textbook; the paper only names the "Wilson Fermion Action" and
benchmarks "Wilson and Domain Wall fermion operators", Sec. 3 and Sec. 4):

  hopping term   (H psi)(x) = sum_mu [ (1 - gamma_mu) U_mu(x) psi(x + mu)
                                     + (1 + gamma_mu) U_mu(x - mu)^dag psi(x - mu) ]
  dagger         (H^dag psi)(x): the same with (1 - gamma) and (1 + gamma) swapped,
                 which equals gamma_5 H gamma_5
  Wilson         D_W = (4 + m) - H / 2           (lattice spacing 1, r = 1)
  kappa form     M_kappa = 1 - kappa H = 2 kappa D_W,   kappa = 1 / (2m + 8)

Readings where the paper is silent: the forward hop carries (1 - gamma_mu);
boundary phases bc[mu] = +-1 multiply every hop that wraps around direction
mu, in both directions (antiperiodic time is bc = (1, 1, 1, -1)).

Even-odd: parity(x) = (x + y + z + t) mod 2. With c = 4 + m,

  D_W = [[c, -H_eo/2], [-H_oe/2, c]]
  M_hat = c - H_eo H_oe / (4c)                   (Schur complement on even sites)
  b_hat_e = b_e + H_eo b_o / (2c),   x_o = (b_o + H_oe x_e / 2) / c

Fields here are full-lattice arrays; an even-parity field is a full-lattice
array that is zero on odd sites. Pins: plane-wave closed form at unit links,
free spectrum, gamma_5-hermiticity, gauge covariance and an explicit-loop
dense matrix (tests/test_oracle_wilson.py); full-system residual of the
even-odd solve (tests/test_oracle_eo.py).
"""
from __future__ import annotations

import numpy as np

from .gamma import GAMMA5, one_minus_gamma, one_plus_gamma, spin_apply


def site_axis(mu: int) -> int:
    """Array axis of coordinate ``mu`` in ``[..., t, z, y, x, a, b]`` arrays."""
    return -3 - mu


def _edge(f: np.ndarray, mu: int, index: int) -> tuple:
    sl = [slice(None)] * f.ndim
    sl[f.ndim + site_axis(mu)] = index
    return tuple(sl)


def shift(f: np.ndarray, mu: int, sign: int, bc) -> np.ndarray:
    """g(x) = bc-phase * f(x + sign * mu_hat): the field seen one hop away."""
    ax = site_axis(mu)
    g = np.roll(f, -sign, axis=ax)
    if bc[mu] != 1.0:
        length = f.shape[ax]
        wrapped = length - 1 if sign > 0 else 0
        g[_edge(g, mu, wrapped)] *= bc[mu]
    return g


def colour_apply(u: np.ndarray, f: np.ndarray) -> np.ndarray:
    """(U f)(x) for link matrices ``u[..., a, b]`` and field ``f[..., spin, b]``."""
    return np.einsum("...ab,...sb->...sa", u, f)


def colour_apply_dag(u: np.ndarray, f: np.ndarray) -> np.ndarray:
    """(U^dag f)(x)."""
    return np.einsum("...ba,...sb->...sa", u.conj(), f)


def hop(U: np.ndarray, psi: np.ndarray, bc, dagger: bool = False) -> np.ndarray:
    """Hopping term H psi (or H^dag psi). ``psi`` may carry leading axes (s, rhs);
    the links are shared across them."""
    out = np.zeros(psi.shape, dtype=np.complex128)
    for mu in range(4):
        fwd_spin = one_plus_gamma(mu) if dagger else one_minus_gamma(mu)
        bwd_spin = one_minus_gamma(mu) if dagger else one_plus_gamma(mu)
        u_mu = U[..., mu, :, :]
        out += spin_apply(fwd_spin, colour_apply(u_mu, shift(psi, mu, +1, bc)))
        u_back = np.roll(u_mu, 1, axis=site_axis(mu))  # U_mu(x - mu)
        out += spin_apply(bwd_spin, colour_apply_dag(u_back, shift(psi, mu, -1, bc)))
    return out


def dirac(U: np.ndarray, psi: np.ndarray, mass: float, bc, dagger: bool = False) -> np.ndarray:
    """D_W psi = (4 + m) psi - H psi / 2 (or its adjoint)."""
    return (4.0 + mass) * psi - 0.5 * hop(U, psi, bc, dagger)


def dirac_dag_dirac(U, psi, mass, bc):
    return dirac(U, dirac(U, psi, mass, bc), mass, bc, dagger=True)


def gamma5(psi: np.ndarray) -> np.ndarray:
    return spin_apply(GAMMA5, psi)


# --------------------------------------------------------------- even / odd

def parity_field(dims) -> np.ndarray:
    """parity(x) = (x + y + z + t) mod 2 on the (T, Z, Y, X) grid."""
    x, y, z, t = dims
    tt, zz, yy, xx = np.meshgrid(np.arange(t), np.arange(z), np.arange(y), np.arange(x),
                                 indexing="ij")
    return (xx + yy + zz + tt) % 2


def restrict(psi: np.ndarray, parity: int) -> np.ndarray:
    """Zero every site whose parity differs from ``parity``."""
    t, z, y, x = psi.shape[-6:-2]
    mask = parity_field((x, y, z, t)) == parity
    return psi * mask[..., None, None]


def hop_eo(U, psi, bc, out_parity: int, dagger: bool = False):
    """H_{out,in} psi: hop from sites of parity 1-out_parity to sites of out_parity."""
    return restrict(hop(U, restrict(psi, 1 - out_parity), bc, dagger), out_parity)


def schur(U, psi_e, mass, bc, dagger: bool = False):
    """M_hat psi_e = c psi_e - H_eo H_oe psi_e / (4c) on even sites (or its adjoint,
    c - H^dag_eo H^dag_oe / (4c))."""
    c = 4.0 + mass
    tmp = hop_eo(U, psi_e, bc, 1, dagger)
    return c * restrict(psi_e, 0) - hop_eo(U, tmp, bc, 0, dagger) / (4.0 * c)


def schur_dag_schur(U, psi_e, mass, bc):
    return schur(U, schur(U, psi_e, mass, bc), mass, bc, dagger=True)


def prepare_source(U, b, mass, bc):
    """b_hat_e = b_e + H_eo b_o / (2c)."""
    c = 4.0 + mass
    return restrict(b, 0) + hop_eo(U, restrict(b, 1), bc, 0) / (2.0 * c)


def reconstruct(U, x_e, b, mass, bc):
    """Full solution from the even half: x_o = (b_o + H_oe x_e / 2) / c."""
    c = 4.0 + mass
    x_o = (restrict(b, 1) + 0.5 * hop_eo(U, x_e, bc, 1)) / c
    return restrict(x_e, 0) + x_o
