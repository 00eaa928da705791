"""G-parity Wilson operator on the GPU against the oracle (oracle/gparity.py):
the hop on each checkerboard and on the full lattice, the even-odd Schur
operator, and even-odd CG solves that must reach the FP64 true residual of the
full G-parity system. Two flavours are the n5 = 2 inner index."""
import numpy as np
import pytest

from oracle import gparity, wilson
from synthetic import gauge_field, gaussian_spinor
from tests.layout import rel_l2, to_cb

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL = {0: 1e-12, 1: 1e-5}
BC = (1.0, 1.0, 1.0, -1.0)
MASKS = {1: (0,), 6: (1, 2), 7: (0, 1, 2), 15: (0, 1, 2, 3)}


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1512_03487_gb300 as L
    from paper_1512_03487_gb300 import fields
    L.fields = fields
    return L


def _restrict(psi2, parity):
    return np.stack([wilson.restrict(psi2[f], parity) for f in range(2)])


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("recon", [18, 12])
@pytest.mark.parametrize("dagger", [0, 1])
@pytest.mark.parametrize("subset", [0, 1, 2])
@pytest.mark.parametrize("mask", [1, 6, 15])
def test_hop_matches_oracle(L, prec, recon, dagger, subset, mask):
    dims = (6, 4, 4, 6)
    gd = MASKS[mask]
    U = gauge_field(dims, "haar", 1901)
    psi2 = gaussian_spinor(dims, 1902, lead=(2,))
    F = L.fields
    lat = L.lattice(dims, n5=2, bc=BC)
    op = L.operator(prec=prec, recon=recon, gparity=mask)
    g = F.gauge_to_device(U, lat, prec, recon)
    if subset == 2:
        fin = F.spinor_to_device(psi2, lat, prec, 2)
        expect = gparity.hop(U, psi2, BC, gd, bool(dagger))
    else:
        src = 1 - subset
        fin = F.spinor_to_device(to_cb(psi2, src), lat, prec, src)
        expect = to_cb(gparity.hop(U, _restrict(psi2, src), BC, gd, bool(dagger)), subset)
    out = F.empty(L.lqcd_spinor_bytes(lat, prec, subset))
    L.lqcd_dslash(out, fin, g, lat, op, subset, dagger)
    assert rel_l2(F.spinor_to_host(out, lat, prec, subset), expect) <= TOL[prec]


def _schur(U, psi_e, m, gd, dagger=False):
    """M_hat psi_e = c psi_e - H_eo H_oe psi_e / (4c) for a two-flavour even field (full-lattice arrays)."""
    c = 4.0 + m
    t = _restrict(gparity.hop(U, psi_e, BC, gd, dagger), 1)
    return c * psi_e - _restrict(gparity.hop(U, t, BC, gd, dagger), 0) / (4 * c)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dagger", [0, 1])
def test_schur_operator(L, prec, dagger):
    dims, m, mask = (4, 4, 6, 4), 0.1, 7
    U = gauge_field(dims, "haar", 1911)
    psi_e = _restrict(gaussian_spinor(dims, 1912, lead=(2,)), 0)
    F = L.fields
    lat = L.lattice(dims, n5=2, bc=BC)
    op = L.operator(mass=m, prec=prec, recon=12, gparity=mask)
    g = F.gauge_to_device(U, lat, prec, 12)
    out = F.empty(L.lqcd_spinor_bytes(lat, prec, 0))
    tmp = F.empty(L.lqcd_operator_workspace_bytes(lat, op, 0))
    L.lqcd_M(out, F.spinor_to_device(to_cb(psi_e, 0), lat, prec, 0), g, lat, op, 0, dagger, tmp)
    expect = to_cb(_schur(U, psi_e, m, MASKS[mask], bool(dagger)), 0)
    assert rel_l2(F.spinor_to_host(out, lat, prec, 0), expect) <= TOL[prec]


@pytest.mark.parametrize("sloppy", [0, 1])
@pytest.mark.parametrize("mask", [1, 7])
@pytest.mark.parametrize("solver", ["cg", "cgnr"])
def test_even_odd_solve_full_residual(L, sloppy, mask, solver):
    """b_hat = prepare(b); CG on M_hat^dag M_hat with source M_hat^dag b_hat (or CGNR on
    b_hat, whose start applies M_hat^dag with FP32 arithmetic on the FP64 links); reconstruct
    x_o; the oracle's G-parity operator must give |b - D x| / |b| <= 1e-9 on the full lattice."""
    dims, m = (4, 4, 4, 8), 0.05
    gd = MASKS[mask]
    U = gauge_field(dims, "haar", 1921)
    b = gaussian_spinor(dims, 1922, lead=(2,))
    F = L.fields
    lat = L.lattice(dims, n5=2, bc=BC)
    op = L.operator(mass=m, gparity=mask)
    prm = L.solver_params(tol=1e-11, maxiter=5000, sloppy_prec=sloppy, sloppy_recon=12 if sloppy else 18,
                          delta=1e-5 if sloppy else 0.1)
    g64 = F.gauge_to_device(U, lat, 0, 18)
    gs = F.gauge_to_device(U, lat, 1, 12) if sloppy else g64
    bd = F.spinor_to_device(b, lat, 0, 2)
    tmp = F.empty(L.lqcd_operator_workspace_bytes(lat, op, 0))
    bhat = F.empty(L.lqcd_spinor_bytes(lat, 0, 0))
    src = F.empty(L.lqcd_spinor_bytes(lat, 0, 0))
    L.lqcd_eo_prepare(bhat, bd, g64, lat, op, tmp)
    L.lqcd_M(src, bhat, g64, lat, op, 0, 1, tmp)
    x = F.empty(L.lqcd_spinor_bytes(lat, 0, 2))
    ws = F.empty(L.lqcd_cg_workspace_bytes(lat, op, prm, 0))
    if solver == "cg":
        info = L.lqcd_cg_solve(x, src, g64, gs, lat, op, prm, 0, ws)
    else:
        info = L.lqcd_cgnr_solve(x, bhat, g64, gs, lat, op, prm, 0, ws)
    L.lqcd_eo_reconstruct(x, bd, g64, lat, op, tmp)
    xh = F.spinor_to_host(x, lat, 0, 2)
    res = np.linalg.norm(b - gparity.dirac(U, xh, m, BC, gd)) / np.linalg.norm(b)
    assert info.status == 0 and res <= 1e-9, (info.iterations, res)


@pytest.mark.parametrize("sloppy", [0, 1])
def test_eo_solve_gparity(L, sloppy):
    """lqcd_eo_solve with G-parity: the odd half comes from the last update's
    G-parity hop H_oe x_e; the oracle's two-flavour operator gives the full
    system's residual <= 1e-10."""
    dims, m, mask = (4, 4, 4, 8), 0.05, 6
    gd = MASKS[mask]
    U = gauge_field(dims, "haar", 1931)
    b = gaussian_spinor(dims, 1932, lead=(2,))
    F = L.fields
    lat = L.lattice(dims, n5=2, bc=BC)
    op = L.operator(mass=m, gparity=mask)
    prm = L.solver_params(tol=1e-10, maxiter=5000, sloppy_prec=sloppy, sloppy_recon=12 if sloppy else 18,
                          delta=3e-6 if sloppy else 0.1)
    g64 = F.gauge_to_device(U, lat, 0, 18)
    gs = F.gauge_to_device(U, lat, 1, 12) if sloppy else g64
    x = F.empty(L.lqcd_spinor_bytes(lat, 0, 2))
    ws = F.empty(L.lqcd_eo_solve_workspace_bytes(lat, op, prm))
    info = L.lqcd_eo_solve(x, F.spinor_to_device(b, lat, 0, 2), g64, gs, lat, op, prm, ws)
    xh = F.spinor_to_host(x, lat, 0, 2)
    res = np.linalg.norm(b - gparity.dirac(U, xh, m, BC, gd)) / np.linalg.norm(b)
    assert info.status == 0 and res <= 1e-10, (info.iterations, res)
