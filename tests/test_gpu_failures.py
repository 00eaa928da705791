"""Failure detection of the solvers, made on the host side: a NaN in the
source, a wall-clock limit, an iteration cap. Each must come back as its
status code with the GPU context still usable (a following solve converges).
Nothing here faults, traps or hangs a GPU: the NaN only travels through the
reductions, whose finaliser closes the iteration gate, and the time limit is
checked by the host between graph launches."""
import numpy as np
import pytest

from oracle import cg as ocg
from oracle import wilson
from synthetic import gauge_field, gaussian_spinor
from tests.layout import from_cb, to_cb

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
BC = (1.0, 1.0, 1.0, -1.0)
ERR_NOT_CONVERGED, ERR_NAN, ERR_TIMEOUT = -3, -4, -5


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1512_03487_gb300 as L
    from paper_1512_03487_gb300 import fields
    L.fields = fields
    return L


def _solve(L, U, b, dims, m, cgnr=False, **kw):
    F = L.fields
    lat = L.lattice(dims, bc=BC)
    op = L.operator(mass=m)
    prm = L.solver_params(**kw)
    g64 = F.gauge_to_device(U, lat, 0, 18)
    gs = F.gauge_to_device(U, lat, prm.sloppy_prec, prm.sloppy_recon) if prm.sloppy_prec else g64
    bd = F.spinor_to_device(b, lat, 0, 0)
    x = F.empty(L.lqcd_spinor_bytes(lat, 0, 0))
    ws = F.empty(L.lqcd_cg_workspace_bytes(lat, op, prm, 0))
    solve = L.lqcd_cgnr_solve if cgnr else L.lqcd_cg_solve
    info = solve(x, bd, g64, gs, lat, op, prm, 0, ws, raise_on_error=False)
    torch.cuda.synchronize()
    return F.spinor_to_host(x, lat, 0, 0), info


def _healthy(L, U, b, dims, m):
    x, info = _solve(L, U, b, dims, m, tol=1e-10, maxiter=2000)
    assert info.status == 0, L.lqcd_last_error()
    res = ocg.true_residual(lambda v: wilson.schur_dag_schur(U, v, m, BC), from_cb(x, 0), from_cb(b, 0))
    assert res <= 1e-10


@pytest.mark.parametrize("sloppy,use_graph", [(0, 1), (1, 1), (2, 1), (1, 0)])
def test_nan_in_source_is_reported(L, sloppy, use_graph):
    dims, m = (4, 4, 4, 8), 0.1
    U = gauge_field(dims, "haar", 801)
    b = to_cb(gaussian_spinor(dims, 802, lead=(1,)), 0)
    bad = b.copy()
    bad.reshape(-1)[17] = np.nan
    _, info = _solve(L, U, bad, dims, m, tol=1e-10, maxiter=500, sloppy_prec=sloppy,
                     sloppy_recon=12 if sloppy else 18, use_graph=use_graph)
    assert info.status == ERR_NAN, (info.status, L.lqcd_last_error())
    assert "NaN" in L.lqcd_last_error()
    _healthy(L, U, b, dims, m)


def test_wall_clock_limit(L):
    """A limit far below one chunk's duration stops the solve at the first host
    check (before or after the first graph launch) with LQCD_ERR_TIMEOUT."""
    dims, m = (8, 8, 8, 8), 0.01
    U = gauge_field(dims, "haar", 811)
    b = to_cb(gaussian_spinor(dims, 812, lead=(1,)), 0)
    _, info = _solve(L, U, b, dims, m, tol=1e-12, maxiter=20000, check_interval=4, timeout_ms=1e-3)
    assert info.status == ERR_TIMEOUT, (info.status, L.lqcd_last_error())
    assert info.iterations <= 8
    _healthy(L, U, b, (8, 8, 8, 8), m)


def test_iteration_cap_reports_true_residual(L):
    dims, m = (4, 4, 4, 8), 0.05
    U = gauge_field(dims, "haar", 821)
    b = to_cb(gaussian_spinor(dims, 822, lead=(1,)), 0)
    x, info = _solve(L, U, b, dims, m, tol=1e-12, maxiter=10, sloppy_prec=1, sloppy_recon=12, check_interval=3)
    assert info.status == ERR_NOT_CONVERGED
    res = ocg.true_residual(lambda v: wilson.schur_dag_schur(U, v, m, BC), from_cb(x, 0), from_cb(b, 0))
    # the reported residual is the FP64 true residual of the returned x
    assert abs(res - info.true_rel_residual) <= 1e-6 * res
    _healthy(L, U, b, dims, m)


@pytest.mark.parametrize("sloppy,delta_mid,use_graph", [(0, 0.0, 1), (1, 0.0, 1), (2, 0.003, 1), (2, 0.003, 0)])
def test_cgnr_nan_zero_and_cap(L, sloppy, delta_mid, use_graph):
    """CGNR and the three-level scheme on the failure paths: a NaN in b is
    reported (it reaches |b|^2 and the start M^dag b), a zero b returns x = 0 at
    once, and the iteration cap ends with the FP64 system residual
    ||b - M x|| / ||b|| of the returned x; the context stays usable."""
    dims, m = (4, 4, 4, 8), 0.05
    U = gauge_field(dims, "haar", 831)
    b = to_cb(gaussian_spinor(dims, 832, lead=(1,)), 0)
    kw = dict(tol=1e-12, sloppy_prec=sloppy, sloppy_recon=12 if sloppy else 18, delta=1e-5 if sloppy else 0.1,
              delta_mid=delta_mid, use_graph=use_graph, cgnr=True)
    bad = b.copy()
    bad.reshape(-1)[5] = np.nan
    _, info = _solve(L, U, bad, dims, m, maxiter=500, **kw)
    assert info.status == ERR_NAN, (info.status, L.lqcd_last_error())
    x, info = _solve(L, U, np.zeros_like(b), dims, m, maxiter=500, **kw)
    assert info.status == 0 and info.iterations == 0 and not np.any(x)
    x, info = _solve(L, U, b, dims, m, maxiter=12, check_interval=5, **kw)
    assert info.status == ERR_NOT_CONVERGED
    xe, be = from_cb(x, 0), from_cb(b, 0)
    res = np.linalg.norm(be - wilson.schur(U, xe, m, BC)) / np.linalg.norm(be)
    assert abs(res - info.true_rel_residual) <= 1e-9 * res
    _healthy(L, U, b, dims, m)


def test_eo_solve_iteration_cap_returns_full_solution(L):
    """lqcd_eo_solve stopped by the iteration cap still returns the full
    solution of its last FP64 update: the odd half is what lqcd_eo_reconstruct
    gives for the returned even half, and the reported residual is the full
    system's, ||b_hat - M_hat x_e|| / ||b|| for the returned x_e."""
    from tests.layout import rel_l2
    dims, m = (4, 4, 4, 8), 0.05
    U = gauge_field(dims, "haar", 841)
    b = gaussian_spinor(dims, 842, lead=(1,))
    F = L.fields
    lat = L.lattice(dims, bc=BC)
    op = L.operator(mass=m)
    prm = L.solver_params(tol=1e-12, maxiter=10, sloppy_prec=1, sloppy_recon=12, delta=3e-6, check_interval=4)
    g64 = F.gauge_to_device(U, lat, 0, 18)
    gs = F.gauge_to_device(U, lat, 1, 12)
    bd = F.spinor_to_device(b, lat, 0, 2)
    x = F.empty(L.lqcd_spinor_bytes(lat, 0, 2))
    ws = F.empty(L.lqcd_eo_solve_workspace_bytes(lat, op, prm))
    info = L.lqcd_eo_solve(x, bd, g64, gs, lat, op, prm, ws, raise_on_error=False)
    assert info.status == ERR_NOT_CONVERGED
    xh = F.spinor_to_host(x, lat, 0, 2)
    tmp = F.empty(L.lqcd_operator_workspace_bytes(lat, op, 0))
    x2 = x.clone()
    L.lqcd_eo_reconstruct(x2, bd, g64, lat, op, tmp)
    assert rel_l2(F.spinor_to_host(x2, lat, 0, 2), xh) <= 1e-13
    xe = wilson.restrict(xh, 0)
    bh = wilson.prepare_source(U, b, m, BC)
    res = np.linalg.norm(bh - wilson.schur(U, xe, m, BC)) / np.linalg.norm(b)
    assert abs(res - info.true_rel_residual) <= 1e-9 * res
    res_full = np.linalg.norm(b - wilson.dirac(U, xh, m, BC)) / np.linalg.norm(b)
    assert abs(res_full - info.true_rel_residual) <= 1e-9 * res
    _healthy(L, U, to_cb(b, 0), dims, m)
