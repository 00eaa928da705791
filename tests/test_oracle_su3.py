"""Pins for the oracle's SU(3) x SU(3) field product (CPU only)."""
import numpy as np

from oracle import su3
from synthetic import gauge_field, make_rng


def _fields(n, seed):
    U = gauge_field((2, 2, 2, 4), "haar", seed)  # [t, z, y, x, mu, 3, 3]
    return U.reshape(-1, 3, 3)[:n]


def test_explicit_loop():
    rng = make_rng(1301)
    x = rng.standard_normal((5, 3, 3)) + 1j * rng.standard_normal((5, 3, 3))
    y = rng.standard_normal((5, 3, 3)) + 1j * rng.standard_normal((5, 3, 3))
    z = su3.su3_mul(x, y)
    for s in range(5):
        for i in range(3):
            for k in range(3):
                want = sum(x[s, i, j] * y[s, j, k] for j in range(3))
                assert abs(z[s, i, k] - want) < 1e-14


def test_identity_and_order():
    x = _fields(16, 1302)
    y = _fields(16, 1303)
    eye = np.broadcast_to(np.eye(3), x.shape)
    np.testing.assert_allclose(su3.su3_mul(x, eye), x, atol=1e-15)
    np.testing.assert_allclose(su3.su3_mul(eye, x), x, atol=1e-15)
    # SU(3) does not commute: a transposed or swapped operand is caught here
    assert np.abs(su3.su3_mul(x, y) - su3.su3_mul(y, x)).max() > 1e-2
    assert np.abs(su3.su3_mul(x, y) - np.swapaxes(su3.su3_mul(np.swapaxes(x, -1, -2), y), -1, -2)).max() > 1e-2


def test_group_closure_and_invariants():
    x = _fields(128, 1304)
    y = _fields(128, 1305)
    z = su3.su3_mul(x, y)
    eye = np.eye(3)
    np.testing.assert_allclose(z @ np.conj(np.swapaxes(z, -1, -2)), np.broadcast_to(eye, z.shape), atol=1e-13)
    np.testing.assert_allclose(np.linalg.det(z), 1.0, atol=1e-13)
    # tr(xy) = tr(yx) and det(xy) = det(x) det(y) for general complex matrices
    rng = make_rng(1306)
    a = rng.standard_normal((8, 3, 3)) + 1j * rng.standard_normal((8, 3, 3))
    b = rng.standard_normal((8, 3, 3)) + 1j * rng.standard_normal((8, 3, 3))
    np.testing.assert_allclose(np.trace(su3.su3_mul(a, b), axis1=-2, axis2=-1),
                               np.trace(su3.su3_mul(b, a), axis1=-2, axis2=-1), rtol=1e-13)
    np.testing.assert_allclose(np.linalg.det(su3.su3_mul(a, b)), np.linalg.det(a) * np.linalg.det(b), rtol=1e-12)
