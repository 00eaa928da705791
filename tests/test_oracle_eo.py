"""Pins for the oracle's even-odd Schur complement (CPU only)."""
import numpy as np

from oracle import wilson
from synthetic import gauge_field, gaussian_spinor
from tests.brute import wilson_dense

BC_AP = (1.0, 1.0, 1.0, -1.0)


def _even_indices(dims):
    par = wilson.parity_field(dims).reshape(-1)
    even_sites = np.nonzero(par == 0)[0]
    return (even_sites[:, None] * 12 + np.arange(12)[None, :]).reshape(-1)


def test_schur_solve_gives_full_solution():
    """Solving M_hat x_e = b_hat_e densely, then reconstructing x_o, solves D_W x = b."""
    dims = (4, 2, 2, 4)
    m = 0.2
    U = gauge_field(dims, "haar", 51)
    b = gaussian_spinor(dims, 52)
    idx = _even_indices(dims)
    n = idx.size
    basis = np.zeros((n,) + b.shape, dtype=np.complex128)
    flat = basis.reshape(n, -1)
    flat[np.arange(n), idx] = 1.0
    Mhat = np.array([wilson.schur(U, basis[k], m, BC_AP).reshape(-1)[idx] for k in range(n)]).T
    bhat = wilson.prepare_source(U, b, m, BC_AP).reshape(-1)[idx]
    xe_vec = np.linalg.solve(Mhat, bhat)
    xe = np.zeros(b.size, dtype=np.complex128)
    xe[idx] = xe_vec
    x = wilson.reconstruct(U, xe.reshape(b.shape), b, m, BC_AP)
    res = b - wilson.dirac(U, x, m, BC_AP)
    assert np.linalg.norm(res) < 1e-12 * np.linalg.norm(b)
    # the reconstructed solution equals the dense full-lattice solve
    D = wilson_dense(U, dims, m, BC_AP)
    np.testing.assert_allclose(x.reshape(-1), np.linalg.solve(D, b.reshape(-1)), atol=1e-11)


def test_schur_determinant_identity():
    """det D_W = c^(12 Vh) det M_hat on a 2^4 lattice (block LU of D_W)."""
    dims = (2, 2, 2, 2)
    m = 0.4
    c = 4 + m
    U = gauge_field(dims, "haar", 53)
    D = wilson_dense(U, dims, m, BC_AP)
    idx = _even_indices(dims)
    n = idx.size
    shape = (2, 2, 2, 2, 4, 3)
    basis = np.zeros((n,) + shape, dtype=np.complex128)
    basis.reshape(n, -1)[np.arange(n), idx] = 1.0
    Mhat = np.array([wilson.schur(U, basis[k], m, BC_AP).reshape(-1)[idx] for k in range(n)]).T
    s1, l1 = np.linalg.slogdet(D)
    s2, l2 = np.linalg.slogdet(Mhat)
    assert abs((l1 - (l2 + n * np.log(c)))) < 1e-10
    assert abs(s1 - s2) < 1e-10


def test_schur_adjoint():
    dims = (4, 4, 2, 4)
    U = gauge_field(dims, "haar", 54)
    a = wilson.restrict(gaussian_spinor(dims, 55), 0)
    b = wilson.restrict(gaussian_spinor(dims, 56), 0)
    lhs = np.vdot(a.ravel(), wilson.schur(U, b, 0.1, BC_AP).ravel())
    rhs = np.vdot(wilson.schur(U, a, 0.1, BC_AP, dagger=True).ravel(), b.ravel())
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)
