"""Pins for the oracle's G-parity Wilson operator (CPU only)."""
import itertools

import numpy as np
import pytest

from oracle import gparity, wilson
from oracle.gamma import GAMMA, GAMMA5
from synthetic import gauge_field, gaussian_spinor, random_gauge_transform, unit_gauge

MASS = 0.1


def _axis(mu):
    return 3 - mu  # axis of coordinate mu in [t, z, y, x, ...]


@pytest.mark.parametrize("mu_g", [0, 1, 2, 3])
@pytest.mark.parametrize("dagger", [False, True])
def test_single_direction_equals_doubled_lattice(mu_g, dagger):
    """G-parity in one direction = Wilson on the lattice doubled there, links U then U*,
    antiperiodic wrap of the doubled extent."""
    dims = (2, 4, 2, 4)
    bc = (1.0, -1.0, 1.0, -1.0)
    U = gauge_field(dims, "haar", 1801)
    psi2 = gaussian_spinor(dims, 1802, lead=(2,))
    out = gparity.dirac(U, psi2, MASS, bc, (mu_g,), dagger)
    ax = _axis(mu_g)
    U2 = np.concatenate([U, np.conj(U)], axis=ax)
    psi_d = np.concatenate([psi2[0], psi2[1]], axis=ax)
    bc2 = list(bc)
    bc2[mu_g] = -1.0
    ref = wilson.dirac(U2, psi_d, MASS, tuple(bc2), dagger)
    np.testing.assert_allclose(np.concatenate([out[0], out[1]], axis=ax), ref, atol=1e-12)


def _plane_wave(dims, p, u):
    X, Y, Z, T = dims
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    ph = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))
    return ph[..., None, None] * u


@pytest.mark.parametrize("gdirs", [(0, 1), (0, 1, 2)])
@pytest.mark.parametrize("which", [+1, -1])
def test_free_field_twisted_plane_waves(gdirs, which):
    """At unit links Phi_pm = Psi_0 +- i Psi_1 decouple and pick up -+i at each G-parity
    boundary, so e^{ipx} u with p_mu = (2 pi n -+ pi/2) / L_mu there is an eigenmode with
    D(p) = 4 + m - sum_mu (cos p_mu - i gamma_mu sin p_mu)."""
    dims = (4, 4, 4, 4)
    bc = (1.0, 1.0, 1.0, -1.0)
    rng = np.random.default_rng(1803)
    u = rng.standard_normal((4, 3)) + 1j * rng.standard_normal((4, 3))
    p = []
    for mu in range(4):
        L = dims[mu]
        n = 1 if mu % 2 else 0
        if mu in gdirs:
            p.append((2 * np.pi * n - which * np.pi / 2) / L)
        else:
            p.append((2 * np.pi * n + (np.pi if bc[mu] < 0 else 0.0)) / L)
    phi = _plane_wave(dims, p, u)
    psi2 = np.stack([phi / 2, phi / (2j) * which])  # Psi_0 = Phi / 2, Psi_1 = which * Phi / (2i)
    Dp = (4 + MASS) * np.eye(4, dtype=complex)
    for mu in range(4):
        Dp -= np.cos(p[mu]) * np.eye(4) - 1j * np.sin(p[mu]) * GAMMA[mu]
    expect = np.stack([_plane_wave(dims, p, Dp @ u) / 2, _plane_wave(dims, p, Dp @ u) / (2j) * which])
    out = gparity.dirac(unit_gauge(dims), psi2, MASS, bc, gdirs)
    np.testing.assert_allclose(out, expect, atol=1e-12)


@pytest.mark.parametrize("gdirs", [(1,), (0, 2), (0, 1, 2)])
def test_gamma5_hermiticity(gdirs):
    dims = (4, 2, 4, 2)
    bc = (1.0, 1.0, 1.0, -1.0)
    U = gauge_field(dims, "haar", 1804)
    a = gaussian_spinor(dims, 1805, lead=(2,))
    b = gaussian_spinor(dims, 1806, lead=(2,))
    g5 = lambda f: np.einsum("st,...tc->...sc", GAMMA5, f)  # noqa: E731
    np.testing.assert_allclose(gparity.dirac(U, a, MASS, bc, gdirs, dagger=True),
                               g5(gparity.dirac(U, g5(a), MASS, bc, gdirs)), atol=1e-12)
    lhs = np.vdot(b, gparity.dirac(U, a, MASS, bc, gdirs))
    rhs = np.vdot(gparity.dirac(U, b, MASS, bc, gdirs, dagger=True), a)
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)


@pytest.mark.parametrize("gdirs", [(2,), (0, 3), (0, 1, 2)])
def test_gauge_covariance(gdirs):
    """Psi_0 -> g Psi_0, Psi_1 -> g* Psi_1, and a link U_mu(x) -> g(x) U g(x+mu)^dag, with
    g(x+mu) replaced by g*(x+mu) when the link crosses a G-parity boundary (flavour 1 sees
    the conjugate transformation)."""
    dims = (4, 4, 2, 4)
    bc = (1.0, 1.0, 1.0, -1.0)
    U = gauge_field(dims, "haar", 1807)
    g = random_gauge_transform(dims, 1808)
    psi2 = gaussian_spinor(dims, 1809, lead=(2,))
    Ug = np.empty_like(U)
    for mu in range(4):
        g_fwd = np.roll(g, -1, axis=wilson.site_axis(mu))
        if mu in gdirs:
            edge = [slice(None)] * g_fwd.ndim
            edge[_axis(mu)] = dims[mu] - 1
            g_fwd[tuple(edge)] = np.conj(g_fwd[tuple(edge)])
        Ug[..., mu, :, :] = g @ U[..., mu, :, :] @ np.conj(np.swapaxes(g_fwd, -1, -2))
    gs = np.stack([g, np.conj(g)])
    apply = lambda f: np.einsum("f...ab,f...sb->f...sa", gs, f)  # noqa: E731
    lhs = gparity.dirac(Ug, apply(psi2), MASS, bc, gdirs)
    rhs = apply(gparity.dirac(U, psi2, MASS, bc, gdirs))
    np.testing.assert_allclose(lhs, rhs, atol=1e-12)


def test_no_twist_is_two_independent_flavours_with_conjugate_links():
    dims = (2, 2, 4, 4)
    bc = (1.0, 1.0, 1.0, -1.0)
    U = gauge_field(dims, "haar", 1810)
    psi2 = gaussian_spinor(dims, 1811, lead=(2,))
    out = gparity.dirac(U, psi2, MASS, bc, ())
    np.testing.assert_allclose(out[0], wilson.dirac(U, psi2[0], MASS, bc), atol=1e-12)
    np.testing.assert_allclose(out[1], wilson.dirac(np.conj(U), psi2[1], MASS, bc), atol=1e-12)
