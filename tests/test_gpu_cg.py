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


@pytest.mark.parametrize("recon64,use_graph,subset", [(18, 1, "even"), (12, 1, "even"), (18, 0, "even"),
                                                     (18, 1, "full")])
def test_three_level_fp16(L, recon64, use_graph, subset):
    """FP16 inner iteration with intermediate FP32-arithmetic residual
    replacements (delta_mid) and FP64 reliable updates only every five decades
    (delta 1e-5): the FP64 true residual still reaches 1e-10, the replacements
    run, and the FP64 updates stay as few as the FP32 inner solve needs. A wrong
    replacement operator (it runs only inside the solve) would leave the
    iterated residual inconsistent with x_s and cost FP64 updates and
    iterations, which the bounds below catch."""
    dims, m = (8, 4, 4, 8), 0.01
    U = gauge_field(dims, "exp", 111, eps=0.3)
    b = gaussian_spinor(dims, 112, lead=(1,))
    lat = L.lattice(dims, bc=BC)
    op = L.operator(mass=m, recon=recon64)
    if subset == "even":
        src, sub = to_cb(b, 0), L.LQCD_EVEN
        A = lambda v: wilson.schur_dag_schur(U, v, m, BC)  # noqa: E731
        check = lambda x: ocg.true_residual(A, from_cb(x, 0), from_cb(src, 0))  # noqa: E731
    else:
        src, sub = b, L.LQCD_FULL
        A = lambda v: wilson.dirac_dag_dirac(U, v, m, BC)  # noqa: E731
        check = lambda x: ocg.true_residual(A, x, src)  # noqa: E731
    prm = L.solver_params(tol=1e-10, maxiter=5000, sloppy_prec=2, sloppy_recon=12, delta=1e-5,
                          delta_mid=0.003, use_graph=use_graph)
    x, info = _solve(L, U, src, lat, op, prm, sub, sloppy_recon=12)
    assert info.status == 0, L.lqcd_last_error()
    res = check(x)
    assert res <= 1e-10
    assert abs(info.true_rel_residual - res) < 1e-11
    assert info.residual_replacements >= 1
    assert info.reliable_updates <= 3
    p64 = L.solver_params(tol=1e-10, maxiter=5000)
    _, i64 = _solve(L, U, src, lat, op, p64, sub)
    assert info.iterations <= 1.25 * i64.iterations + 10, (info.iterations, i64.iterations)
    # without the middle level, FP16 needs an FP64 update every two to three decades
    plain = L.solver_params(tol=1e-10, maxiter=5000, sloppy_prec=2, sloppy_recon=12, delta=0.003,
                            use_graph=use_graph)
    _, ip = _solve(L, U, src, lat, op, plain, sub, sloppy_recon=12)
    assert ip.status == 0 and ip.residual_replacements == 0
    assert info.reliable_updates < ip.reliable_updates


def test_three_level_multi_rhs(L):
    """The replacement level with n5 = 3 independent systems of very different
    scales (each keeps its own replacement maximum)."""
    dims, m, n = (4, 4, 4, 8), 0.05, 3
    U = gauge_field(dims, "haar", 121)
    b = gaussian_spinor(dims, 122, lead=(n,))
    b[1] *= 1e-3
    lat = L.lattice(dims, n5=n, bc=BC)
    op = L.operator(mass=m)
    prm = L.solver_params(tol=1e-10, maxiter=2000, sloppy_prec=2, sloppy_recon=12, delta=1e-5, delta_mid=0.003)
    be = to_cb(b, 0)
    x, info = _solve(L, U, be, lat, op, prm, L.LQCD_EVEN, sloppy_recon=12)
    assert info.status == 0, L.lqcd_last_error()
    assert info.residual_replacements >= 1
    for k in range(n):
        A = lambda v: wilson.schur_dag_schur(U, v, m, BC)  # noqa: E731
        assert ocg.true_residual(A, from_cb(x[k:k + 1], 0), from_cb(be[k:k + 1], 0)) <= 1e-10


def test_three_level_dwf(L):
    """Domain wall, FP16 inner with replacements (M5 epilogue on FP64 links)."""
    dims, Ls, M5, mf = (4, 4, 4, 4), 8, 1.8, 0.02
    U = gauge_field(dims, "haar", 131)
    b = gaussian_spinor(dims, 132, lead=(Ls,))
    lat = L.lattice(dims, n5=Ls, bc=BC)
    op = L.operator(kind=L.LQCD_DWF, M5=M5, mf=mf)
    prm = L.solver_params(tol=1e-10, maxiter=5000, sloppy_prec=2, sloppy_recon=12, delta=1e-5, delta_mid=0.003)
    be = to_cb(b, 0)
    x, info = _solve(L, U, be, lat, op, prm, L.LQCD_EVEN, sloppy_recon=12)
    assert info.status == 0, L.lqcd_last_error()
    assert info.residual_replacements >= 1
    A = lambda v: dwf.schur_dag_schur(U, v, M5, mf, BC)  # noqa: E731
    assert ocg.true_residual(A, from_cb(x, 0), from_cb(be, 0)) <= 1e-10


def _solve_nr(L, U, b, lat, op, prm, subset, sloppy_recon=12):
    F = L.fields
    g64 = F.gauge_to_device(U, lat, 0, op.recon)
    gs = F.gauge_to_device(U, lat, prm.sloppy_prec, sloppy_recon) if prm.sloppy_prec != 0 else g64
    bd = F.spinor_to_device(b, lat, 0, subset)
    x = F.empty(L.lqcd_spinor_bytes(lat, 0, subset))
    ws = F.empty(L.lqcd_cg_workspace_bytes(lat, op, prm, subset))
    info = L.lqcd_cgnr_solve(x, bd, g64, gs, lat, op, prm, subset, ws, raise_on_error=False)
    return F.spinor_to_host(x, lat, 0, subset), info


def _system_residual(apply_m, x, b):
    """||b - M x|| / ||b|| in FP64 (the oracle's own operator): CGNR's exit test."""
    return float(np.linalg.norm((b - apply_m(x)).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("case", ["fp64", "fp32", "fp16_three_level", "full_fp32", "nograph_fp16", "dwf_fp32",
                                  "mrhs_fp16_three_level"])
def test_cgnr(L, case):
    """CGNR for M_hat x = b_hat (or M x = b): the reliable updates recompute
    b - M x and its norm in FP64, which decide the exit; M^dag b and
    M^dag (b - M x) only seed the recurrence, in the inner arithmetic. The
    solve meets the system residual ||b - M x|| / ||b|| that the oracle
    computes from x, reports it, and x is the oracle's solution."""
    dims, m = (8, 4, 4, 8), 0.01
    sloppy, dmid, delta, subset, n5 = 1, 0.0, 1e-5, L.LQCD_EVEN, 1
    if case == "fp64":
        sloppy, delta = 0, 0.1
    elif case in ("fp16_three_level", "nograph_fp16", "mrhs_fp16_three_level"):
        sloppy, dmid = 2, 0.003
    elif case == "full_fp32":
        subset = L.LQCD_FULL
    if case == "mrhs_fp16_three_level":
        dims, n5 = (4, 4, 4, 8), 3
    U = gauge_field(dims, "exp", 141, eps=0.3)
    if case == "dwf_fp32":
        dims, n5, M5, mf = (4, 4, 4, 4), 8, 1.8, 0.02
        U = gauge_field(dims, "haar", 142)
        op = L.operator(kind=L.LQCD_DWF, M5=M5, mf=mf)
        Mx = lambda v: dwf.schur(U, v, M5, mf, BC)  # noqa: E731
        Md = lambda v: dwf.schur(U, v, M5, mf, BC, dagger=True)  # noqa: E731
    else:
        op = L.operator(mass=m)
        if subset == L.LQCD_EVEN:
            Mx = lambda v: wilson.schur(U, v, m, BC)  # noqa: E731
            Md = lambda v: wilson.schur(U, v, m, BC, dagger=True)  # noqa: E731
        else:
            Mx = lambda v: wilson.dirac(U, v, m, BC)  # noqa: E731
            Md = lambda v: wilson.dirac(U, v, m, BC, dagger=True)  # noqa: E731
    b = gaussian_spinor(dims, 143, lead=(n5,))
    if n5 == 3:
        b[1] *= 1e-3
    lat = L.lattice(dims, n5=n5, bc=BC)
    prm = L.solver_params(tol=1e-10, maxiter=5000, sloppy_prec=sloppy, sloppy_recon=12, delta=delta,
                          delta_mid=dmid, use_graph=0 if case == "nograph_fp16" else 1)
    src = to_cb(b, 0) if subset == L.LQCD_EVEN else b
    x, info = _solve_nr(L, U, src, lat, op, prm, subset)
    assert info.status == 0, L.lqcd_last_error()
    if dmid:
        assert info.residual_replacements >= 1
    full = (lambda v: from_cb(v, 0)) if subset == L.LQCD_EVEN else (lambda v: v)  # noqa: E731
    if case == "dwf_fp32":
        res = _system_residual(Mx, full(x), full(src))
        assert res <= 1e-10
        assert abs(res - info.true_rel_residual) < 1e-12
        return
    worst = 0.0
    for k in range(n5):
        res = _system_residual(Mx, full(x[k:k + 1]), full(src[k:k + 1]))
        assert res <= 1e-10, (k, res)
        worst = max(worst, res)
        xo, _ = ocg.cg(lambda v: Md(Mx(v)), Md(full(src[k:k + 1])), 1e-13, 5000)
        assert rel_l2(full(x[k:k + 1]), xo) < 1e-6
    assert abs(worst - info.true_rel_residual) < 1e-12


@pytest.mark.parametrize("case", ["fp64", "fp32", "fp16_three_level", "nograph_fp16", "mrhs_fp32", "dwf_fp32",
                                  "dwf6_fp16_three_level", "zero"])
def test_eo_solve_full_system(L, case):
    """lqcd_eo_solve: prepare, CGNR, odd half (for Wilson from the last reliable
    update's H_oe x_e, with no hop of its own). The oracle's full operator gives
    ||b - D x|| / ||b|| <= 1e-10 on the whole lattice, and the odd half equals
    what lqcd_eo_reconstruct computes from the returned even half."""
    dims, m, n5 = (8, 4, 4, 8), 0.01, 1
    sloppy, dmid, delta, kind = 1, 0.0, 1e-5, 0
    if case == "fp64":
        sloppy, delta = 0, 0.1
    elif case in ("fp16_three_level", "nograph_fp16"):
        sloppy, dmid = 2, 0.003
    elif case == "mrhs_fp32":
        dims, n5 = (4, 4, 4, 8), 3
    U = gauge_field(dims, "exp", 151, eps=0.3)
    if case.startswith("dwf"):
        # L_s = 8 runs M5op^-1 in the hop's epilogue, L_s = 6 the closed-form kernel
        dims, n5, kind = (4, 4, 4, 4), (6 if case.startswith("dwf6") else 8), 1
        U = gauge_field(dims, "haar", 152)
        if case == "dwf6_fp16_three_level":
            sloppy, dmid = 2, 0.003
    F = L.fields
    lat = L.lattice(dims, n5=n5, bc=BC)
    op = L.operator(kind=kind, mass=m, M5=1.8, mf=0.02)
    b = gaussian_spinor(dims, 153, lead=(n5,))
    if case == "zero":
        b = np.zeros_like(b)
    prm = L.solver_params(tol=1e-10, maxiter=5000, sloppy_prec=sloppy, sloppy_recon=12, delta=delta,
                          delta_mid=dmid, use_graph=0 if case == "nograph_fp16" else 1)
    g64 = F.gauge_to_device(U, lat, 0, 18)
    gs = F.gauge_to_device(U, lat, sloppy, 12) if sloppy else g64
    bd = F.spinor_to_device(b, lat, 0, 2)
    x = F.empty(L.lqcd_spinor_bytes(lat, 0, 2))
    ws = F.empty(L.lqcd_eo_solve_workspace_bytes(lat, op, prm))
    info = L.lqcd_eo_solve(x, bd, g64, gs, lat, op, prm, ws, raise_on_error=False)
    assert info.status == 0, L.lqcd_last_error()
    xh = F.spinor_to_host(x, lat, 0, 2)
    if case == "zero":
        assert not np.any(xh)
        return
    D = (lambda v: dwf.dirac(U, v, 1.8, 0.02, BC)) if kind else (lambda v: wilson.dirac(U, v, m, BC))  # noqa: E731
    for k in range(n5 if kind == 0 else 1):
        sl = slice(k, k + 1) if kind == 0 else slice(None)
        res = np.linalg.norm(b[sl] - D(xh[sl])) / np.linalg.norm(b[sl])
        assert res <= 1e-10, (k, res)
    # the odd half against lqcd_eo_reconstruct applied to the returned even half
    tmp = F.empty(L.lqcd_operator_workspace_bytes(lat, op, 0))
    x2 = x.clone()
    L.lqcd_eo_reconstruct(x2, bd, g64, lat, op, tmp)
    assert rel_l2(F.spinor_to_host(x2, lat, 0, 2), xh) <= 1e-13


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
