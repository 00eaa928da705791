"""Pins for the oracle's Shamir domain-wall operator (CPU only)."""
import numpy as np
import pytest

from oracle import dwf, wilson
from synthetic import gauge_field, gaussian_spinor
from tests.brute import dwf_dense

BC_AP = (1.0, 1.0, 1.0, -1.0)


def test_ls1_reduces_to_wilson():
    """L_s = 1: D_DW = D_W with mass 1 - M5 + mf."""
    dims = (4, 4, 2, 4)
    U = gauge_field(dims, "haar", 61)
    psi = gaussian_spinor(dims, 62, lead=(1,))
    M5, mf = 1.8, 0.02
    out = dwf.dirac(U, psi, M5, mf, BC_AP)
    np.testing.assert_allclose(out[0], wilson.dirac(U, psi[0], 1 - M5 + mf, BC_AP), atol=1e-13)


def test_gamma5_reflection_hermiticity():
    """D_DW^dag = (R gamma_5) D_DW (R gamma_5)."""
    dims = (4, 2, 2, 4)
    U = gauge_field(dims, "haar", 63)
    psi = gaussian_spinor(dims, 64, lead=(6,))
    M5, mf = 1.8, 0.02
    lhs = dwf.dirac(U, psi, M5, mf, BC_AP, dagger=True)
    rhs = dwf.gamma5_reflect(dwf.dirac(U, dwf.gamma5_reflect(psi), M5, mf, BC_AP))
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)


@pytest.mark.parametrize("dagger", [False, True])
def test_dense_brute_force(dagger):
    dims, Ls = (2, 2, 2, 4), 4
    M5, mf = 1.8, 0.02
    U = gauge_field(dims, "haar", 65)
    D = dwf_dense(U, dims, Ls, M5, mf, BC_AP)
    if dagger:
        D = D.conj().T
    psi = gaussian_spinor(dims, 66, lead=(Ls,))
    out = dwf.dirac(U, psi, M5, mf, BC_AP, dagger=dagger)
    np.testing.assert_allclose(out.reshape(-1), D @ psi.reshape(-1), atol=1e-12)


@pytest.mark.parametrize("dagger", [False, True])
def test_m5_inverse(dagger):
    dims, Ls = (2, 2, 2, 2), 8
    psi = gaussian_spinor(dims, 67, lead=(Ls,))
    out = dwf.m5op(dwf.m5op_inv(psi, 1.8, 0.02, dagger), 1.8, 0.02, dagger)
    np.testing.assert_allclose(out, psi, atol=1e-12)


def test_eo_solve_gives_full_solution():
    dims, Ls = (2, 2, 2, 4), 4
    M5, mf = 1.8, 0.1
    U = gauge_field(dims, "haar", 68)
    b = gaussian_spinor(dims, 69, lead=(Ls,))
    par = wilson.parity_field(dims).reshape(-1)
    even = np.nonzero(par == 0)[0]
    V = par.size
    idx = ((np.arange(Ls)[:, None, None] * V + even[None, :, None]) * 12
           + np.arange(12)[None, None, :]).reshape(-1)
    n = idx.size
    basis = np.zeros((n,) + b.shape, dtype=np.complex128)
    basis.reshape(n, -1)[np.arange(n), idx] = 1.0
    Mhat = np.array([dwf.schur(U, basis[k], M5, mf, BC_AP).reshape(-1)[idx] for k in range(n)]).T
    bhat = dwf.prepare_source(U, b, M5, mf, BC_AP).reshape(-1)[idx]
    xe = np.zeros(b.size, dtype=np.complex128)
    xe[idx] = np.linalg.solve(Mhat, bhat)
    x = dwf.reconstruct(U, xe.reshape(b.shape), b, M5, mf, BC_AP)
    res = b - dwf.dirac(U, x, M5, mf, BC_AP)
    assert np.linalg.norm(res) < 1e-11 * np.linalg.norm(b)
    # Schur adjoint is the true adjoint
    a = wilson.restrict(gaussian_spinor(dims, 70, lead=(Ls,)), 0)
    c = wilson.restrict(gaussian_spinor(dims, 71, lead=(Ls,)), 0)
    lhs = np.vdot(a.ravel(), dwf.schur(U, c, M5, mf, BC_AP).ravel())
    rhs = np.vdot(dwf.schur(U, a, M5, mf, BC_AP, dagger=True).ravel(), c.ravel())
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)


@pytest.mark.parametrize("Ls,M5,mf", [(5, 1.8, 0.02), (4, 1.3, 0.1), (3, 0.5, -0.3)])
def test_free_field_determinant_closed_form(Ls, M5, mf):
    """Free field on a periodic 2^4 lattice: every momentum p has components in {0, pi},
    so sin p = 0 and the hop is diagonal, H = 2 sum_mu cos p_mu = 2 (4 - 2k) with k the
    number of pi components. The operator is then block-diagonal in chirality with
    blocks d_k - T, d_k = 1 - M5 + 2k, T a cyclic shift in s whose weights multiply to
    -mf, and det(d - T) = d^Ls + mf (characteristic polynomial of a weighted cycle).
    Each chirality carries 2 spins x 3 colours, and C(4, k) momenta have k pi components:
    det D_DW = prod_k ((1 - M5 + 2k)^Ls + mf)^(12 C(4, k))."""
    from math import comb

    from synthetic import unit_gauge
    dims = (2, 2, 2, 2)
    U = unit_gauge(dims)
    shape = (Ls, 2, 2, 2, 2, 4, 3)
    n = int(np.prod(shape))
    D = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[j] = 1.0
        D[:, j] = dwf.dirac(U, e.reshape(shape), M5, mf, (1.0, 1.0, 1.0, 1.0)).reshape(-1)
        e[j] = 0.0
    sign, logabs = np.linalg.slogdet(D)
    factors = [(1 - M5 + 2 * k) ** Ls + mf for k in range(5)]
    mult = [12 * comb(4, k) for k in range(5)]
    want_log = sum(m * np.log(abs(f)) for f, m in zip(factors, mult))
    want_sign = np.prod([np.sign(f) ** m for f, m in zip(factors, mult)])
    assert logabs == pytest.approx(want_log, rel=1e-12, abs=1e-9)
    assert abs(sign - want_sign) < 1e-9
