"""Pins for the oracle's Wilson gauge action, gauge force and link update (CPU only)."""
import numpy as np
import pytest

from oracle import gauge, wilson
from synthetic import gauge_field, make_rng, random_gauge_transform, random_su3_algebra, unit_gauge

BETA = 5.6


def _transform(U, g):
    Ug = np.empty_like(U)
    for mu in range(4):
        g_fwd = np.roll(g, -1, axis=wilson.site_axis(mu))
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ np.conj(np.swapaxes(g_fwd, -1, -2))
    return Ug


def test_unit_links():
    U = unit_gauge((4, 2, 2, 4))
    assert gauge.mean_plaquette(U) == pytest.approx(1.0, abs=1e-15)
    assert gauge.action(U, BETA) == pytest.approx(0.0, abs=1e-12)
    assert np.abs(gauge.force(U, BETA)).max() < 1e-15


@pytest.mark.parametrize("mu", [0, 3])
@pytest.mark.parametrize("theta", [0.3, 1.7])
def test_single_twisted_link_closed_form(mu, theta):
    """One link diag(e^{i th}, e^{-i th}, 1) on unit links: six plaquettes have
    Re tr = 1 + 2 cos th, so S_g = 6 beta (1 - (1 + 2 cos th) / 3) = 4 beta (1 - cos th)."""
    U = unit_gauge((4, 4, 2, 4))
    U[1, 0, 1, 2, mu] = np.diag([np.exp(1j * theta), np.exp(-1j * theta), 1.0])
    assert gauge.action(U, BETA) == pytest.approx(4 * BETA * (1 - np.cos(theta)), rel=1e-13)


def test_staple_counts_every_plaquette_four_times():
    U = gauge_field((2, 4, 2, 4), "haar", 1501)
    lhs = sum(np.trace(U[..., mu, :, :] @ gauge.staple(U, mu), axis1=-2, axis2=-1).real.sum() for mu in range(4))
    rhs = 4 * sum(np.trace(gauge.plaquette_field(U, mu, nu), axis1=-2, axis2=-1).real.sum()
                  for mu in range(4) for nu in range(mu + 1, 4))
    assert lhs == pytest.approx(rhs, rel=1e-13)


def test_gauge_invariance():
    dims = (4, 2, 4, 2)
    U = gauge_field(dims, "haar", 1502)
    g = random_gauge_transform(dims, 1503)
    assert gauge.action(_transform(U, g), BETA) == pytest.approx(gauge.action(U, BETA), rel=1e-12)


def test_force_matches_central_finite_difference():
    dims = (2, 4, 2, 4)
    U = gauge_field(dims, "exp", 1504, eps=0.5)
    T = random_su3_algebra(make_rng(1505), U.size // 9).reshape(U.shape)
    F = gauge.force(U, BETA)
    analytic = np.einsum("...ij,...ji->...", T, F).real.sum()
    h = 1e-5
    sp = gauge.action(gauge.update_links(U, T, h), BETA)
    sm = gauge.action(gauge.update_links(U, T, -h), BETA)
    assert (sp - sm) / (2 * h) == pytest.approx(analytic, rel=1e-7)


def test_force_is_traceless_hermitian_and_covariant():
    dims = (2, 2, 4, 4)
    U = gauge_field(dims, "haar", 1506)
    F = gauge.force(U, BETA)
    np.testing.assert_allclose(F, gauge.dag(F), atol=1e-13)
    np.testing.assert_allclose(np.trace(F, axis1=-2, axis2=-1), 0, atol=1e-13)
    g = random_gauge_transform(dims, 1507)
    Fg = gauge.force(_transform(U, g), BETA)
    expect = g[..., None, :, :] @ F @ gauge.dag(g)[..., None, :, :]
    np.testing.assert_allclose(Fg, expect, atol=1e-12)


def test_exponential_against_series():
    P = random_su3_algebra(make_rng(1508), 64)
    for eps in (0.05, 0.4):
        series = np.zeros_like(P)
        term = np.broadcast_to(np.eye(3, dtype=complex), P.shape).copy()
        for k in range(40):
            series += term
            term = term @ (1j * eps * P) / (k + 1)
        E = gauge.expm_i(P, eps)
        np.testing.assert_allclose(E, series, atol=1e-14)
        np.testing.assert_allclose(E @ gauge.dag(E), np.broadcast_to(np.eye(3), E.shape), atol=1e-14)
        np.testing.assert_allclose(np.linalg.det(E), 1.0, atol=1e-14)


def test_kinetic_energy():
    P = random_su3_algebra(make_rng(1509), 10)
    assert gauge.kinetic(P) == pytest.approx(0.5 * sum(np.sum(np.abs(p) ** 2) for p in P), rel=1e-13)
