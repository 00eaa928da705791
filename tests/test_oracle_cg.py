"""Pins for the oracle's conjugate gradient (CPU only)."""
import numpy as np

from oracle import cg, wilson
from synthetic import gauge_field, gaussian_spinor
from tests.brute import wilson_dense

BC_AP = (1.0, 1.0, 1.0, -1.0)


def test_cg_matches_dense_solve():
    dims = (4, 2, 2, 4)
    m = 0.1
    U = gauge_field(dims, "haar", 81)
    b = gaussian_spinor(dims, 82)
    x, info = cg.cg(lambda v: wilson.dirac_dag_dirac(U, v, m, BC_AP), b, 1e-12, 5000)
    D = wilson_dense(U, dims, m, BC_AP)
    xd = np.linalg.solve(D.conj().T @ D, b.reshape(-1))
    assert info.converged and info.true_rel_residual <= 1e-12
    assert np.linalg.norm(x.reshape(-1) - xd) <= 1e-9 * np.linalg.norm(xd)
    assert 0 < info.iterations < b.size


def test_cg_on_hermitian_matrix_exact_termination():
    """On a well-separated n x n HPD matrix CG terminates in at most ~n steps."""
    rng = np.random.default_rng(83)
    n = 12
    q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    a = q @ np.diag(np.linspace(1, 4, n)) @ q.conj().T
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x, info = cg.cg(lambda v: a @ v, b, 1e-13, 100)
    np.testing.assert_allclose(x, np.linalg.solve(a, b), atol=1e-11)
    assert info.iterations <= n + 2


def test_cg_zero_source():
    b = np.zeros((2, 2, 2, 2, 4, 3), dtype=np.complex128)
    x, info = cg.cg(lambda v: v, b, 1e-10, 10)
    assert info.iterations == 0 and np.all(x == 0)
