"""Checks on the seeded input generators (CPU only)."""
import numpy as np

from synthetic import exp_i_hermitian_su3, gauge_field, gaussian_spinor, haar_su3, make_rng


def test_haar_su3_is_special_unitary():
    u = haar_su3(make_rng(1), 2000)
    eye = np.broadcast_to(np.eye(3), u.shape)
    np.testing.assert_allclose(u @ np.conj(np.swapaxes(u, 1, 2)), eye, atol=1e-13)
    np.testing.assert_allclose(np.linalg.det(u), 1.0, atol=1e-13)


def test_haar_moments():
    """Haar SU(3): E[U_ij] = 0 and E[|U_ij|^2] = 1/3."""
    u = haar_su3(make_rng(2), 200000)
    assert np.abs(u.mean(axis=0)).max() < 0.01
    np.testing.assert_allclose((np.abs(u) ** 2).mean(axis=0), 1.0 / 3.0, atol=0.01)


def test_exp_field_is_special_unitary_and_near_one():
    u = exp_i_hermitian_su3(make_rng(3), 2000, 0.3)
    eye = np.broadcast_to(np.eye(3), u.shape)
    np.testing.assert_allclose(u @ np.conj(np.swapaxes(u, 1, 2)), eye, atol=1e-13)
    np.testing.assert_allclose(np.linalg.det(u), 1.0, atol=1e-13)
    assert np.abs(np.trace(u, axis1=1, axis2=2).real.mean() / 3.0 - 1) < 0.3


def test_seeded_determinism_and_shapes():
    a = gauge_field((4, 2, 2, 6), "haar", 5)
    b = gauge_field((4, 2, 2, 6), "haar", 5)
    assert a.shape == (6, 2, 2, 4, 4, 3, 3)
    np.testing.assert_array_equal(a, b)
    s = gaussian_spinor((4, 2, 2, 6), 6, lead=(3,))
    assert s.shape == (3, 6, 2, 2, 4, 4, 3)
    assert abs(s.real.std() - 1) < 0.05 and abs(s.imag.std() - 1) < 0.05
