"""Wilson gauge action, gauge force, link update and HMC trajectories on the
GPU against the oracle (oracle/gauge.py, oracle/hmc.py) on the same seeded
inputs: gauge field, momenta and pseudofermion are drawn on the host and fed
to both sides."""
import numpy as np
import pytest

from oracle import gauge as og
from oracle import hmc as oh
from oracle import wilson
from synthetic import gauge_field, gaussian_spinor, make_rng, random_su3_algebra

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
BC = (1.0, 1.0, 1.0, -1.0)
BETA, MASS = 5.6, 0.2


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1512_03487_gb300 as L
    from paper_1512_03487_gb300 import fields
    L.fields = fields
    return L


def _momenta(U, seed):
    return random_su3_algebra(make_rng(seed), U.size // 9).reshape(U.shape)


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (4, 2, 6, 4), (8, 4, 4, 6)])
def test_plaquette_force_update_kinetic(L, dims):
    F = L.fields
    lat = L.lattice(dims, bc=BC)
    U = gauge_field(dims, "haar", 1701)
    P = _momenta(U, 1702)
    Ud = F.gauge_to_device(U, lat, 0, 18)
    Pd = F.gauge_to_device(P, lat, 0, 18)
    ws = F.empty(L.lqcd_reduce_workspace_bytes(lat))
    assert L.lqcd_plaquette(Ud, lat, ws) == pytest.approx(og.mean_plaquette(U), abs=1e-14)
    assert L.lqcd_momentum_kinetic(Pd, lat, ws) == pytest.approx(og.kinetic(P), rel=1e-13)
    Fd = F.empty(L.lqcd_gauge_bytes(lat, 0, 18))
    L.lqcd_gauge_force(Fd, Ud, lat, BETA)
    assert _rel(F.gauge_to_host(Fd, lat, 0, 18), og.force(U, BETA)) <= 1e-13
    for eps in (0.07, 1.3):  # 1.3 exercises the scaling-and-squaring branch
        Ue = F.gauge_to_device(U, lat, 0, 18)
        L.lqcd_gauge_exp_update(Ue, Pd, eps, lat)
        assert _rel(F.gauge_to_host(Ue, lat, 0, 18), og.update_links(U, P, eps)) <= 1e-13


def _trajectory(L, U, P, phi, dims, integrator, nsteps, tau, fermion, sloppy=0, tol=1e-14):
    F = L.fields
    lat = L.lattice(dims, bc=BC)
    op = L.operator(mass=MASS)
    prm = L.solver_params(tol=tol, maxiter=20000, sloppy_prec=sloppy, sloppy_recon=12 if sloppy else 18,
                          delta=1e-5 if sloppy else 0.1)
    hp = L.hmc_params(BETA, tau, nsteps, integrator, int(fermion))
    Ud = F.gauge_to_device(U, lat, 0, 18)
    Pd = F.gauge_to_device(P, lat, 0, 18)
    phid = F.spinor_to_device(phi, lat, 0, 2) if fermion else None
    ws = F.empty(L.lqcd_hmc_workspace_bytes(lat, op, prm))
    info = L.lqcd_hmc_trajectory(Ud, Pd, phid, lat, op, hp, prm, ws)
    return F.gauge_to_host(Ud, lat, 0, 18), F.gauge_to_host(Pd, lat, 0, 18), info


def _inputs(dims, seed, fermion):
    U = gauge_field(dims, "exp", seed, eps=0.3)
    P = _momenta(U, seed + 1)
    phi = None
    if fermion:
        eta = gaussian_spinor(dims, seed + 2) / np.sqrt(2.0)
        phi = wilson.dirac(U, eta, MASS, BC, dagger=True)
    return U, P, phi


@pytest.mark.parametrize("integrator", [0, 1])
@pytest.mark.parametrize("fermion", [False, True])
def test_trajectory_matches_oracle(L, integrator, fermion):
    dims, nsteps, tau = (4, 4, 2, 4), 3, 0.3
    U, P, phi = _inputs(dims, 1711, fermion)
    U1, P1, info = _trajectory(L, U, P, phi, dims, integrator, nsteps, tau, fermion)
    Uo, Po, H0, H1, nforce = oh.trajectory(U, P, phi, MASS, BC, BETA, tau, nsteps, integrator, fermion)
    assert info.status == 0 and info.force_evaluations == nforce
    assert _rel(U1, Uo) <= 1e-11
    assert _rel(P1, Po) <= 1e-10
    assert info.H0 == pytest.approx(H0, rel=1e-12)
    assert abs((info.H1 - info.H0) - (H1 - H0)) <= 1e-9 * abs(H0)
    if fermion:
        assert info.cg_iterations > 0 and info.fermion0 > 0


def test_reversibility_and_mixed_precision_solves(L):
    """Forward, momentum flip, forward again returns to the start; FP32-inner
    solves (to the same FP64 tolerance) change dH only at the solver's
    tolerance."""
    dims = (4, 4, 4, 4)
    U, P, phi = _inputs(dims, 1721, True)
    U1, P1, i1 = _trajectory(L, U, P, phi, dims, 1, 4, 0.4, True, sloppy=1, tol=1e-12)
    U2, P2, i2 = _trajectory(L, U1, -P1, phi, dims, 1, 4, 0.4, True, sloppy=1, tol=1e-12)
    assert _rel(U2, U) <= 1e-9 and _rel(P2, -P) <= 1e-8
    assert abs(i2.H1 - i1.H0) <= 1e-8 * abs(i1.H0)
    _, _, i64 = _trajectory(L, U, P, phi, dims, 1, 4, 0.4, True, sloppy=0, tol=1e-12)
    assert abs((i1.H1 - i1.H0) - (i64.H1 - i64.H0)) <= 1e-7 * abs(i64.H0)


@pytest.mark.parametrize("integrator", [0, 1])
def test_energy_violation_scales_as_eps_squared(L, integrator):
    dims = (8, 8, 8, 8)
    U, P, phi = _inputs(dims, 1731, True)
    dh = []
    for n in (16, 32):  # eps = 1/32, 1/64: the asymptotic regime for this start far from equilibrium
        _, _, info = _trajectory(L, U, P, phi, dims, integrator, n, 0.5, True, sloppy=1, tol=1e-12)
        dh.append(abs(info.H1 - info.H0))
    assert 3.3 < dh[0] / dh[1] < 4.7, dh
