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
