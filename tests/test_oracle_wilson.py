"""Pins for the oracle's gamma matrices and Wilson operator (CPU only)."""
import itertools

import numpy as np
import pytest

from oracle import gamma, wilson
from synthetic import gauge_field, gaussian_spinor, random_gauge_transform, unit_gauge
from tests.brute import wilson_dense

BC_AP = (1.0, 1.0, 1.0, -1.0)


def _vec(f):
    return f.reshape(-1)


def test_gamma_algebra():
    g = gamma.GAMMA
    for a, b in itertools.product(range(4), range(4)):
        anti = g[a] @ g[b] + g[b] @ g[a]
        np.testing.assert_allclose(anti, 2.0 * np.eye(4) * (a == b), atol=1e-15)
    for a in range(4):
        np.testing.assert_allclose(g[a], g[a].conj().T, atol=0)
    np.testing.assert_allclose(gamma.GAMMA5, np.diag([1, 1, -1, -1]), atol=1e-15)
    for a in range(4):
        np.testing.assert_allclose(gamma.GAMMA5 @ g[a] + g[a] @ gamma.GAMMA5, 0, atol=1e-15)


@pytest.mark.parametrize("p", [(0, 0, 0, 0), (1, 0, 0, 0), (0, 2, 1, 0), (1, 1, 1, 2), (3, 2, 1, 5)])
def test_plane_wave_closed_form(p):
    """At unit links D_W e^{ipx} u = e^{ipx} [m + sum(1 - cos p) + i sum gamma sin p] u,
    p_mu = 2 pi n / L in space and (2n + 1) pi / L in the antiperiodic time direction."""
    dims = (4, 4, 4, 6)
    m = 0.1
    U = unit_gauge(dims)
    mom = [2 * np.pi * p[k] / dims[k] for k in range(3)] + [(2 * p[3] + 1) * np.pi / dims[3]]
    X, Y, Z, T = dims
    tt, zz, yy, xx = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    phase = np.exp(1j * (mom[0] * xx + mom[1] * yy + mom[2] * zz + mom[3] * tt))
    rng = np.random.default_rng(7)
    u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    psi = phase[..., None, None] * u
    out = wilson.dirac(U, psi, m, BC_AP)
    k = (m + sum(1 - np.cos(q) for q in mom)) * np.eye(4) + 1j * sum(
        np.sin(mom[mu]) * gamma.GAMMA[mu] for mu in range(4))
    expect = phase[..., None, None] * (k @ u)
    np.testing.assert_allclose(out, expect, atol=1e-13)


def test_free_spectrum():
    """Spectrum at unit links: m + sum(1 - cos p) +- i sqrt(sum sin^2 p), each value 6-fold."""
    dims = (2, 2, 2, 4)
    m = 0.2
    U = unit_gauge(dims)
    V = 32
    basis = np.eye(12 * V).reshape(12 * V, 4, 2, 2, 2, 4, 3)  # (n, T, Z, Y, X, s, c)
    cols = [_vec(wilson.dirac(U, basis[n], m, BC_AP)) for n in range(12 * V)]
    D = np.array(cols).T
    ev = np.linalg.eigvals(D)
    expect = []
    for n in itertools.product(range(2), range(2), range(2), range(4)):
        mom = [2 * np.pi * n[k] / 2 for k in range(3)] + [(2 * n[3] + 1) * np.pi / 4]
        re = m + sum(1 - np.cos(q) for q in mom)
        im = np.sqrt(sum(np.sin(q) ** 2 for q in mom))
        expect += [re + 1j * im] * 6 + [re - 1j * im] * 6
    key = lambda z: (round(z.real, 8), round(z.imag, 8))  # noqa: E731
    np.testing.assert_allclose(sorted(ev, key=key), sorted(expect, key=key), atol=1e-10)


def test_gamma5_hermiticity():
    dims = (4, 4, 4, 4)
    U = gauge_field(dims, "haar", 11)
    psi = gaussian_spinor(dims, 12)
    chi = gaussian_spinor(dims, 13)
    np.testing.assert_allclose(wilson.hop(U, psi, BC_AP, dagger=True),
                               wilson.gamma5(wilson.hop(U, wilson.gamma5(psi), BC_AP)), atol=1e-12)
    lhs = np.vdot(_vec(chi), _vec(wilson.dirac(U, psi, 0.1, BC_AP)))
    rhs = np.vdot(_vec(wilson.dirac(U, chi, 0.1, BC_AP, dagger=True)), _vec(psi))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


def test_gauge_covariance():
    """D[U^g](g psi) = g D[U] psi with U^g_mu(x) = g(x) U_mu(x) g(x + mu)^dag."""
    dims = (4, 4, 4, 6)
    U = gauge_field(dims, "haar", 21)
    g = random_gauge_transform(dims, 22)
    psi = gaussian_spinor(dims, 23)
    Ug = np.empty_like(U)
    for mu in range(4):
        g_fwd = np.roll(g, -1, axis=wilson.site_axis(mu))
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ np.conj(np.swapaxes(g_fwd, -1, -2))
    gpsi = np.einsum("...ab,...sb->...sa", g, psi)
    lhs = wilson.dirac(Ug, gpsi, 0.05, BC_AP)
    rhs = np.einsum("...ab,...sb->...sa", g, wilson.dirac(U, psi, 0.05, BC_AP))
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 4), (2, 4, 4, 2)])
@pytest.mark.parametrize("dagger", [False, True])
def test_dense_brute_force(dims, dagger):
    U = gauge_field(dims, "haar", 31)
    m = 0.3
    D = wilson_dense(U, dims, m, BC_AP)
    if dagger:
        D = D.conj().T
    for seed in (32, 33):
        psi = gaussian_spinor(dims, seed)
        out = wilson.dirac(U, psi, m, BC_AP, dagger=dagger)
        np.testing.assert_allclose(_vec(out), D @ _vec(psi), atol=1e-12)


def test_kappa_normalisation():
    """M_kappa = 1 - kappa H equals 2 kappa D_W, kappa = 1/(2m + 8)."""
    dims = (4, 4, 2, 4)
    U = gauge_field(dims, "haar", 41)
    psi = gaussian_spinor(dims, 42)
    m = 0.1
    kappa = 1.0 / (2 * m + 8)
    lhs = psi - kappa * wilson.hop(U, psi, BC_AP)
    np.testing.assert_allclose(lhs, 2 * kappa * wilson.dirac(U, psi, m, BC_AP), atol=1e-13)
