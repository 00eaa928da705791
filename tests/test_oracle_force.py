"""Pins for the oracle's pseudofermion force (CPU only)."""
import numpy as np
import pytest

from oracle import force, wilson
from synthetic import gauge_field, gaussian_spinor, make_rng, random_gauge_transform, random_su3_algebra
from tests.brute import wilson_dense

BC_AP = (1.0, 1.0, 1.0, -1.0)


def _exact_action(U, phi, m, dims):
    D = wilson_dense(U, dims, m, BC_AP)
    x = np.linalg.solve(D.conj().T @ D, phi.reshape(-1))
    return float(np.vdot(phi.reshape(-1), x).real)


def _expm_i_hermitian(h, eps):
    w, v = np.linalg.eigh(h)
    return np.einsum("...ij,...j,...kj->...ik", v, np.exp(1j * eps * w), v.conj())


@pytest.mark.parametrize("dims", [(2, 2, 2, 4), (4, 2, 2, 2)])
def test_force_matches_central_finite_difference(dims):
    """dS/deps of S(exp(i eps T) U) at eps = 0 equals sum_links tr(T F)."""
    m = 0.05
    U = gauge_field(dims, "haar", 91)
    phi = gaussian_spinor(dims, 92)
    S, grad, F, X, Y = force.force(U, phi, m, BC_AP, tol=1e-14)
    assert abs(S - _exact_action(U, phi, m, dims)) < 1e-10 * abs(S)
    rng = make_rng(93)
    for _ in range(2):
        T = random_su3_algebra(rng, U.size // 9).reshape(U.shape)
        analytic = np.einsum("...ab,...ba->...", T, F).sum().real
        eps = 1e-5
        sp = _exact_action(_expm_i_hermitian(T, eps) @ U, phi, m, dims)
        sm = _exact_action(_expm_i_hermitian(T, -eps) @ U, phi, m, dims)
        fd = (sp - sm) / (2 * eps)
        assert abs(fd - analytic) < 1e-6 * max(1.0, abs(analytic)), (fd, analytic)


def test_wirtinger_gradient_matches_finite_difference():
    """dS = Re sum conj(dU) G for an arbitrary complex link perturbation dU."""
    dims = (2, 2, 2, 4)
    m = 0.1
    U = gauge_field(dims, "haar", 94)
    phi = gaussian_spinor(dims, 95)
    _, grad, _, _, _ = force.force(U, phi, m, BC_AP, tol=1e-14)
    rng = make_rng(96)
    dU = rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape)
    eps = 1e-6
    fd = (_exact_action(U + eps * dU, phi, m, dims) - _exact_action(U - eps * dU, phi, m, dims)) / (2 * eps)
    analytic = np.vdot(dU.ravel(), grad.ravel()).real
    assert abs(fd - analytic) < 1e-6 * abs(analytic)


def test_force_is_traceless_hermitian_and_gauge_covariant():
    dims = (4, 2, 2, 4)
    m = 0.05
    U = gauge_field(dims, "haar", 97)
    phi = gaussian_spinor(dims, 98)
    _, _, F, _, _ = force.force(U, phi, m, BC_AP, tol=1e-13)
    np.testing.assert_allclose(F, np.conj(np.swapaxes(F, -1, -2)), atol=1e-12)
    np.testing.assert_allclose(np.trace(F, axis1=-2, axis2=-1), 0, atol=1e-12)
    g = random_gauge_transform(dims, 99)
    Ug = np.empty_like(U)
    for mu in range(4):
        g_fwd = np.roll(g, -1, axis=wilson.site_axis(mu))
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ np.conj(np.swapaxes(g_fwd, -1, -2))
    phig = np.einsum("...ab,...sb->...sa", g, phi)
    _, _, Fg, _, _ = force.force(Ug, phig, m, BC_AP, tol=1e-13)
    gd = np.conj(np.swapaxes(g, -1, -2))
    expect = g[..., None, :, :] @ F @ gd[..., None, :, :]
    np.testing.assert_allclose(Fg, expect, atol=1e-9)
