"""GPU conjugate-gradient solves against the FP64 oracle.

Every solve must reach an FP64 true residual <= tol, recomputed here by the
oracle from the returned x (not trusted from the solver), and x must match the
oracle's own CG solution to the accuracy the tolerance implies.
"""
import numpy as np
import pytest

from oracle import cg as ocg
from oracle import dwf, wilson
from synthetic import gauge_field, gaussian_spinor
from tests.layout import from_cb, rel_l2, to_cb

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
BC = (1.0, 1.0, 1.0, -1.0)


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1512_03487_gb300 as L
    from paper_1512_03487_gb300 import fields
    L.fields = fields
    return L


def _solve(L, U, b, lat, op, prm, subset, sloppy_recon=18):
    F = L.fields
    g64 = F.gauge_to_device(U, lat, 0, op.recon)
    gs = F.gauge_to_device(U, lat, prm.sloppy_prec, sloppy_recon) if prm.sloppy_prec != 0 else g64
    bd = F.spinor_to_device(b, lat, 0, subset)
    x = F.empty(L.lqcd_spinor_bytes(lat, 0, subset))
    ws = F.empty(L.lqcd_cg_workspace_bytes(lat, op, prm, subset))
    info = L.lqcd_cg_solve(x, bd, g64, gs, lat, op, prm, subset, ws, raise_on_error=False)
    return F.spinor_to_host(x, lat, 0, subset), info


@pytest.mark.parametrize("use_graph", [1, 0])
def test_fp64_unpreconditioned_cg_8x4(L, use_graph):
    """Plain Wilson CG on M^dag M, 8^4, Haar links, m = 0.1, FP64, tol 1e-10."""
    dims, m = (8, 8, 8, 8), 0.1
    U = gauge_field(dims, "haar", 101)
    b = gaussian_spinor(dims, 102, lead=(1,))
    lat = L.lattice(dims, bc=BC)
    op = L.operator(mass=m)
    prm = L.solver_params(tol=1e-10, maxiter=2000, use_graph=use_graph)
    x, info = _solve(L, U, b, lat, op, prm, L.LQCD_FULL)
    assert info.status == 0
    A = lambda v: wilson.dirac_dag_dirac(U, v, m, BC)  # noqa: E731
    assert ocg.true_residual(A, x, b) <= 1e-10
    assert abs(info.true_rel_residual - ocg.true_residual(A, x, b)) < 1e-11
    xo, oinfo = ocg.cg(A, b, 1e-12, 5000)
    assert rel_l2(x, xo) < 1e-8
    assert abs(info.iterations - oinfo.iterations) <= 0.1 * oinfo.iterations + 20


@pytest.mark.parametrize("sloppy,recon", [(0, 18), (1, 18), (1, 12), (2, 18), (2, 12)])
def test_eo_cg_mixed_precision(L, sloppy, recon):
    """Even-odd Wilson CG, exp(0.3 i H) links, m = 0.01: FP64 and mixed FP32 /
    FP16 inner solves all reach an FP64 true residual <= 1e-10."""
    dims, m = (8, 4, 4, 8), 0.01
    U = gauge_field(dims, "exp", 111, eps=0.3)
    b = gaussian_spinor(dims, 112, lead=(1,))
    be = to_cb(b, 0)
    lat = L.lattice(dims, bc=BC)
    op = L.operator(mass=m)
    prm = L.solver_params(tol=1e-10, maxiter=5000, sloppy_prec=sloppy, sloppy_recon=recon, delta=0.1)
    x, info = _solve(L, U, be, lat, op, prm, L.LQCD_EVEN, sloppy_recon=recon)
    assert info.status == 0, L.lqcd_last_error()
    A = lambda v: wilson.schur_dag_schur(U, v, m, BC)  # noqa: E731
    res = ocg.true_residual(A, from_cb(x, 0), from_cb(be, 0))
    assert res <= 1e-10
    if sloppy != 0:
        assert info.reliable_updates >= 2


def test_multi_rhs_cg(L):
    """n5 = 3 independent right-hand sides sharing one gauge field, FP16 inner."""
    dims, m, n = (4, 4, 4, 8), 0.05, 3
    U = gauge_field(dims, "haar", 121)
    b = gaussian_spinor(dims, 122, lead=(n,))
    b[1] *= 1e-3  # very different scales per RHS
    lat = L.lattice(dims, n5=n, bc=BC)
    op = L.operator(mass=m)
    prm = L.solver_params(tol=1e-10, maxiter=2000, sloppy_prec=2, sloppy_recon=12)
    be = to_cb(b, 0)
    x, info = _solve(L, U, be, lat, op, prm, L.LQCD_EVEN, sloppy_recon=12)
    assert info.status == 0, L.lqcd_last_error()
    for k in range(n):
        A = lambda v: wilson.schur_dag_schur(U, v, m, BC)  # noqa: E731
        assert ocg.true_residual(A, from_cb(x[k:k + 1], 0), from_cb(be[k:k + 1], 0)) <= 1e-10


@pytest.mark.parametrize("sloppy", [0, 1])
def test_dwf_cg(L, sloppy):
    dims, Ls, M5, mf = (4, 4, 4, 4), 8, 1.8, 0.02
    U = gauge_field(dims, "haar", 131)
    b = gaussian_spinor(dims, 132, lead=(Ls,))
    lat = L.lattice(dims, n5=Ls, bc=BC)
    op = L.operator(kind=L.LQCD_DWF, M5=M5, mf=mf)
    prm = L.solver_params(tol=1e-10, maxiter=5000, sloppy_prec=sloppy, sloppy_recon=18)
    be = to_cb(b, 0)
    x, info = _solve(L, U, be, lat, op, prm, L.LQCD_EVEN)
    assert info.status == 0, L.lqcd_last_error()
    A = lambda v: dwf.schur_dag_schur(U, v, M5, mf, BC)  # noqa: E731
    assert ocg.true_residual(A, from_cb(x, 0), from_cb(be, 0)) <= 1e-10


def test_full_system_solve_via_schur(L):
    """Solve D_W x = b: b_hat = prepare(b), CG on M_hat^dag M_hat with source
    M_hat^dag b_hat, reconstruct x_o; the oracle checks ||b - D_W x|| / ||b||."""
    dims, m = (6, 4, 4, 6), 0.05
    U = gauge_field(dims, "haar", 141)
    b = gaussian_spinor(dims, 142, lead=(1,))
    lat = L.lattice(dims, bc=BC)
    op = L.operator(mass=m)
    F = L.fields
    g = F.gauge_to_device(U, lat, 0, 18)
    bd = F.spinor_to_device(b, lat, 0, 2)
    tmp = F.empty(L.lqcd_operator_workspace_bytes(lat, op, 0))
    bhat = F.empty(L.lqcd_spinor_bytes(lat, 0, 0))
    L.lqcd_eo_prepare(bhat, bd, g, lat, op, tmp)
    src = F.empty(L.lqcd_spinor_bytes(lat, 0, 0))
    L.lqcd_M(src, bhat, g, lat, op, 0, 1, tmp)
    prm = L.solver_params(tol=1e-12, maxiter=3000, sloppy_prec=1)
    x = F.empty(L.lqcd_spinor_bytes(lat, 0, 2))
    ws = F.empty(L.lqcd_cg_workspace_bytes(lat, op, prm, 0))
    gs = F.gauge_to_device(U, lat, 1, 18)
    info = L.lqcd_cg_solve(x, src, g, gs, lat, op, prm, 0, ws)
    assert info.status == 0
    L.lqcd_eo_reconstruct(x, bd, g, lat, op, tmp)
    xh = F.spinor_to_host(x, lat, 0, 2)
    res = b - wilson.dirac(U, xh, m, BC)
    assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(b)


def test_zero_source_and_not_converged(L):
    dims = (4, 4, 4, 4)
    U = gauge_field(dims, "haar", 151)
    lat = L.lattice(dims, bc=BC)
    op = L.operator(mass=0.1)
    prm = L.solver_params(tol=1e-10, maxiter=100)
    zero = np.zeros((1, 4, 4, 4, 2, 4, 3), dtype=np.complex128)
    x, info = _solve(L, U, zero, lat, op, prm, 0)
    assert info.status == 0 and info.iterations == 0 and not np.any(x)
    b = to_cb(gaussian_spinor(dims, 152, lead=(1,)), 0)
    prm = L.solver_params(tol=1e-14, maxiter=3, check_interval=2)
    x, info = _solve(L, U, b, lat, op, prm, 0)
    assert info.status == -3  # LQCD_ERR_NOT_CONVERGED
    assert 3 <= info.iterations <= 4
    assert 0 < info.true_rel_residual < 1
