"""Pins for the oracle's HMC trajectory (CPU only): reversibility and the
O(eps^2) energy violation of both integrators, with and without the Wilson
pseudofermion. A force inconsistent with the action (wrong sign or factor)
leaves an O(1) energy violation and fails the scaling test."""
import numpy as np
import pytest

from oracle import hmc, wilson
from synthetic import gauge_field, gaussian_spinor, make_rng, random_su3_algebra

BC = (1.0, 1.0, 1.0, -1.0)
BETA, MASS = 5.6, 0.2


def _setup(dims, seed, fermion):
    U = gauge_field(dims, "exp", seed, eps=0.3)
    P = random_su3_algebra(make_rng(seed + 1), U.size // 9).reshape(U.shape)
    phi = None
    if fermion:
        eta = gaussian_spinor(dims, seed + 2) / np.sqrt(2.0)
        phi = wilson.dirac(U, eta, MASS, BC, dagger=True)
    return U, P, phi


@pytest.mark.parametrize("integrator", [hmc.LEAPFROG, hmc.MINNORM2])
@pytest.mark.parametrize("fermion", [False, True])
def test_reversibility(integrator, fermion):
    dims = (2, 2, 2, 4)
    U, P, phi = _setup(dims, 1601, fermion)
    U1, P1, H0, H1, _ = hmc.trajectory(U, P, phi, MASS, BC, BETA, 0.5, 4, integrator, fermion)
    U2, P2, H2, H3, _ = hmc.trajectory(U1, -P1, phi, MASS, BC, BETA, 0.5, 4, integrator, fermion)
    np.testing.assert_allclose(U2, U, atol=1e-11)
    np.testing.assert_allclose(P2, -P, atol=1e-10)
    assert H3 == pytest.approx(H0, rel=1e-11)


@pytest.mark.parametrize("integrator", [hmc.LEAPFROG, hmc.MINNORM2])
@pytest.mark.parametrize("fermion", [False, True])
def test_energy_violation_is_second_order(integrator, fermion):
    """|dH| falls by 4 per halving of eps (tau = 0.5, 8 -> 16 -> 32 steps); the
    minimum-norm integrator's violation is several times smaller."""
    dims = (2, 2, 2, 4)
    U, P, phi = _setup(dims, 1611, fermion)
    dh = []
    for n in (8, 16, 32):
        _, _, H0, H1, nforce = hmc.trajectory(U, P, phi, MASS, BC, BETA, 0.5, n, integrator, fermion)
        dh.append(abs(H1 - H0))
        assert nforce == (n + 1 if integrator == hmc.LEAPFROG else 2 * n + 1)
    r1, r2 = dh[0] / dh[1], dh[1] / dh[2]
    assert 2.8 < r1 < 5.0 and 3.5 < r2 < 4.5, dh
    assert dh[2] < (0.03 if integrator == hmc.LEAPFROG else 0.005)
