"""Parity at the benchmark sizes, in the launch configuration bench.py times.

24^3 x 48 (the bench workload): every output of the FP16 and FP32 12-real hop
against the oracle, and the bench's solve (CGNR, FP16 three levels) and the
two-level CG: normal-equation and full-system FP64 residuals from the oracle.
16^4 x L_s = 16 (domain wall) and 32^4 x 12 RHS: the L_s-replicated /
multi-RHS hop on sampled slices. The force kernel at 16^4 and 24^3 x 32 on the
same X, Y as the oracle.
"""
import numpy as np
import pytest

from oracle import force as oforce
from oracle import wilson
from synthetic import config_seed, gauge_field, gaussian_spinor
from tests.layout import rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
BC = (1.0, 1.0, 1.0, -1.0)
DIMS = (24, 24, 24, 48)


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1512_03487_gb300 as L
    from paper_1512_03487_gb300 import fields
    L.fields = fields
    return L


@pytest.fixture(scope="module")
def bench_fields():
    U = gauge_field(DIMS, "exp", config_seed(1, 0), eps=0.3)
    b = gaussian_spinor(DIMS, config_seed(1, 1), lead=(1,))
    return U, b


def _cb_flat(full, parity, dims):
    """Sites of one parity of [..., T, Z, Y, X, 4, 3] in lexicographic order."""
    X, Y, Z, T = dims
    par = wilson.parity_field(dims).reshape(-1)
    idx = np.nonzero(par == parity)[0]
    return full.reshape(full.shape[:-6] + (X * Y * Z * T, 4, 3))[..., idx, :, :]


@pytest.mark.parametrize("prec,tol", [(2, 3e-3), (1, 1e-5)])
def test_bench_size_hop_all_outputs(L, bench_fields, prec, tol):
    U, b = bench_fields
    F = L.fields
    lat = L.lattice(DIMS, bc=BC)
    op = L.operator(prec=prec, recon=12)
    g = F.gauge_to_device(U, lat, prec, 12)
    src = _cb_flat(b, 1, DIMS).reshape(F.host_spinor_shape(lat, 1))
    fin = F.spinor_to_device(src, lat, prec, 1)
    out = F.empty(L.lqcd_spinor_bytes(lat, prec, 0))
    L.lqcd_dslash(out, fin, g, lat, op, 0, 0)
    got = F.spinor_to_host(out, lat, prec, 0)
    expect = _cb_flat(wilson.hop_eo(U, b, BC, 0), 0, DIMS)
    assert rel_l2(got, expect) <= tol


@pytest.mark.parametrize("solver", ["cgnr_three_level", "cg_fp16"])
def test_bench_size_mixed_solve_residual(L, bench_fields, solver):
    """The bench step -- lqcd_eo_solve: CGNR on b_hat with FP16 / 12-real inner
    iteration, FP32 replacements (delta_mid 0.003) and FP64 reliable updates
    (delta 3e-6), check interval 64, odd half from the last update's hop -- and
    the two-level CG on M_hat^dag b_hat: the residuals the oracle recomputes
    from x (even-odd system and full system for the former, normal equations
    for the latter) meet the tolerance."""
    U, b = bench_fields
    F = L.fields
    m = 0.01
    lat = L.lattice(DIMS, bc=BC)
    op = L.operator(mass=m)
    g64 = F.gauge_to_device(U, lat, 0, 18)
    g16 = F.gauge_to_device(U, lat, 2, 12)
    bd = F.spinor_to_device(b, lat, 0, 2)
    tmp = F.empty(L.lqcd_operator_workspace_bytes(lat, op, 0))
    bhat = F.empty(L.lqcd_spinor_bytes(lat, 0, 0))
    L.lqcd_eo_prepare(bhat, bd, g64, lat, op, tmp)
    x = F.empty(L.lqcd_spinor_bytes(lat, 0, 2))
    if solver == "cgnr_three_level":
        # the bench's call: lqcd_eo_solve (prepare, CGNR, odd half from the last update's hop)
        prm = L.solver_params(tol=1e-10, maxiter=20000, sloppy_prec=2, sloppy_recon=12, delta=3e-6,
                              delta_mid=0.003, check_interval=64, update_prec=L.LQCD_F64_DF)
        ws = F.empty(L.lqcd_eo_solve_workspace_bytes(lat, op, prm))
        info = L.lqcd_eo_solve(x, bd, g64, g16, lat, op, prm, ws)
        assert info.residual_replacements >= 1 and info.reliable_updates == 2
    else:
        src = F.empty(L.lqcd_spinor_bytes(lat, 0, 0))
        L.lqcd_M(src, bhat, g64, lat, op, 0, 1, tmp)
        prm = L.solver_params(tol=1e-10, maxiter=20000, sloppy_prec=2, sloppy_recon=12, check_interval=32)
        ws = F.empty(L.lqcd_cg_workspace_bytes(lat, op, prm, 0))
        info = L.lqcd_cg_solve(x, src, g64, g16, lat, op, prm, 0, ws)
    assert info.status == 0 and info.true_rel_residual <= 1e-10
    if solver != "cgnr_three_level":
        L.lqcd_eo_reconstruct(x, bd, g64, lat, op, tmp)
    xh = F.spinor_to_host(x, lat, 0, 2)
    xe = wilson.restrict(xh, 0)
    bh = wilson.prepare_source(U, b, m, BC)
    s = bh - wilson.schur(U, xe, m, BC)
    res = b - wilson.dirac(U, xh, m, BC)
    if solver == "cgnr_three_level":
        # the exit test is ||b_hat - M_hat x_e|| <= tol ||b||: with the odd half reconstructed the
        # full system's residual is the same vector, and true_rel_residual reports ||b - D x|| / ||b||
        assert np.linalg.norm(s) <= 1e-10 * np.linalg.norm(b)
        assert abs(np.linalg.norm(s) / np.linalg.norm(b) - info.true_rel_residual) <= 1e-12
        assert abs(np.linalg.norm(res) / np.linalg.norm(b) - info.true_rel_residual) <= 1e-12
        assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(b)
    else:
        # normal-equation residual of the even half, from the oracle's own operators
        r = wilson.schur(U, s, m, BC, dagger=True)
        s0 = wilson.schur(U, bh, m, BC, dagger=True)
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(s0)
        # ||b - D x|| <= ||M_hat^-dag|| tol ||...||: the normal-equation tolerance 1e-10 bounds it loosely
        assert np.linalg.norm(res) <= 1e-8 * np.linalg.norm(b)


def test_dwf_size_hop_sampled_slices(L):
    dims, Ls = (16, 16, 16, 16), 16
    U = gauge_field(dims, "haar", config_seed(2, 0))
    psi = gaussian_spinor(dims, config_seed(2, 1), lead=(Ls,))
    F = L.fields
    lat = L.lattice(dims, n5=Ls, bc=BC)
    op = L.operator(kind=L.LQCD_DWF, M5=1.8, mf=0.02, prec=1, recon=12)
    g = F.gauge_to_device(U, lat, 1, 12)
    fin = F.spinor_to_device(_cb_flat(psi, 1, dims).reshape(F.host_spinor_shape(lat, 1)), lat, 1, 1)
    out = F.empty(L.lqcd_spinor_bytes(lat, 1, 0))
    L.lqcd_dslash(out, fin, g, lat, op, 0, 0)
    got = F.spinor_to_host(out, lat, 1, 0)
    for s in (0, 7, 15):
        expect = _cb_flat(wilson.hop_eo(U, psi[s], BC, 0), 0, dims)
        assert rel_l2(got[s].reshape(expect.shape), expect) <= 1e-5


def test_multi_rhs_size_hop_sampled_rhs(L):
    dims, n = (32, 32, 32, 32), 12
    U = gauge_field(dims, "haar", config_seed(3, 0))
    F = L.fields
    lat = L.lattice(dims, n5=n, bc=BC)
    op = L.operator(prec=2, recon=12)
    g = F.gauge_to_device(U, lat, 2, 12)
    rhs = gaussian_spinor(dims, config_seed(3, 1), lead=(n,))
    fin = F.spinor_to_device(_cb_flat(rhs, 1, dims).reshape(F.host_spinor_shape(lat, 1)), lat, 2, 1)
    del rhs
    out = F.empty(L.lqcd_spinor_bytes(lat, 2, 0))
    L.lqcd_dslash(out, fin, g, lat, op, 0, 0)
    got = F.spinor_to_host(out, lat, 2, 0)
    rhs = gaussian_spinor(dims, config_seed(3, 1), lead=(n,))
    for k in (0, 11):
        expect = _cb_flat(wilson.hop_eo(U, rhs[k], BC, 0), 0, dims)
        assert rel_l2(got[k].reshape(expect.shape), expect) <= 3e-3


@pytest.mark.parametrize("dims", [(16, 16, 16, 16), (24, 24, 24, 32)])
def test_force_kernel_bench_sizes(L, dims):
    """The force kernel on the two force workloads' sizes, on the same X, Y as the oracle."""
    U = gauge_field(dims, "haar", config_seed(4, 0))
    X = gaussian_spinor(dims, config_seed(4, 1))
    Y = gaussian_spinor(dims, config_seed(4, 2))
    F = L.fields
    lat = L.lattice(dims, bc=BC)
    op = L.operator(mass=0.05)
    g = F.gauge_to_device(U, lat, 0, 18)
    out = F.empty(L.lqcd_gauge_bytes(lat, 0, 18))
    L.lqcd_force(out, g, F.spinor_to_device(X[None], lat, 0, 2), F.spinor_to_device(Y[None], lat, 0, 2), lat, op,
                 L.LQCD_FORCE_TA)
    got = F.gauge_to_host(out, lat, 0, 18)
    _, F_o = oforce.force_terms(U, X, Y, BC)
    assert rel_l2(got, F_o) <= 1e-12


def test_dwf_size_solve_full_system_residual(L):
    """The bench's domain-wall solve at full size: 16^4 x L_s = 16, M5 = 1.8,
    mf = 0.02, Haar links, lqcd_eo_solve with FP32 / 12-real inner storage and
    FP64 reliable updates (delta 3e-6, check interval 64). The oracle recomputes
    ||b - D_DW x|| / ||b|| from the returned x on the whole 5D lattice."""
    from oracle import dwf
    dims, Ls, M5, mf = (16, 16, 16, 16), 16, 1.8, 0.02
    U = gauge_field(dims, "haar", config_seed(2, 0))
    b = gaussian_spinor(dims, config_seed(2, 1), lead=(Ls,))
    F = L.fields
    lat = L.lattice(dims, n5=Ls, bc=BC)
    op = L.operator(kind=L.LQCD_DWF, M5=M5, mf=mf)
    g64 = F.gauge_to_device(U, lat, 0, 18)
    g32 = F.gauge_to_device(U, lat, 1, 12)
    bd = F.spinor_to_device(b, lat, 0, 2)
    prm = L.solver_params(tol=1e-10, maxiter=20000, sloppy_prec=1, sloppy_recon=12, delta=3e-6, check_interval=64)
    ws = F.empty(L.lqcd_eo_solve_workspace_bytes(lat, op, prm))
    x = F.empty(L.lqcd_spinor_bytes(lat, 0, 2))
    info = L.lqcd_eo_solve(x, bd, g64, g32, lat, op, prm, ws)
    assert info.status == 0 and info.true_rel_residual <= 1e-10
    del ws, g32
    xh = F.spinor_to_host(x, lat, 0, 2)
    res = np.linalg.norm(b - dwf.dirac(U, xh, M5, mf, BC)) / np.linalg.norm(b)
    assert res <= 1e-10, res


def test_multi_rhs_size_solves_sampled_columns(L):
    """The bench's 12-right-hand-side workload at full size (32^4, Haar links,
    m = 0.01): the full systems D x_k = b_k by lqcd_eo_solve (FP16 storage,
    FP32 replacements, double-float reliable updates) and the batched CG on
    M_hat^dag M_hat x_k = b_k,e by lqcd_cg_solve (FP16 storage, three levels).
    The oracle recomputes ||b_k - D x_k|| / ||b_k|| for columns 0 and 11 and
    the normal-equation residual for column 5 (each column is an independent
    system, so any column checks the batched solve)."""
    dims, n, m = (32, 32, 32, 32), 12, 0.01
    U = gauge_field(dims, "haar", config_seed(3, 0))
    F = L.fields
    lat = L.lattice(dims, n5=n, bc=BC)
    op = L.operator(mass=m)
    g64 = F.gauge_to_device(U, lat, 0, 18)
    g16 = F.gauge_to_device(U, lat, 2, 12)
    rhs = gaussian_spinor(dims, config_seed(3, 1), lead=(n,))
    bd = F.spinor_to_device(rhs, lat, 0, 2)
    be = F.spinor_to_device(_cb_flat(rhs, 0, dims).reshape(F.host_spinor_shape(lat, 0)), lat, 0, 0)
    pe = L.solver_params(tol=1e-10, maxiter=20000, sloppy_prec=2, sloppy_recon=12, delta=3e-6, delta_mid=0.003,
                         check_interval=64, update_prec=L.LQCD_F64_DF)
    ws = F.empty(L.lqcd_eo_solve_workspace_bytes(lat, op, pe))
    x = F.empty(L.lqcd_spinor_bytes(lat, 0, 2))
    info = L.lqcd_eo_solve(x, bd, g64, g16, lat, op, pe, ws)
    assert info.status == 0 and info.true_rel_residual <= 1e-10
    del ws
    xh = F.spinor_to_host(x, lat, 0, 2)
    del x
    for k in (0, 11):
        res = np.linalg.norm(rhs[k] - wilson.dirac(U, xh[k], m, BC)) / np.linalg.norm(rhs[k])
        assert res <= 1e-10, (k, res)
    del xh
    pc = L.solver_params(tol=1e-10, maxiter=20000, sloppy_prec=2, sloppy_recon=12, delta=1e-5, delta_mid=0.003,
                         check_interval=64, update_prec=L.LQCD_F64_DF)
    ws = F.empty(L.lqcd_cg_workspace_bytes(lat, op, pc, 0))
    xe = F.empty(L.lqcd_spinor_bytes(lat, 0, 0))
    info = L.lqcd_cg_solve(xe, be, g64, g16, lat, op, pc, 0, ws)
    assert info.status == 0 and info.true_rel_residual <= 1e-10
    del ws
    xeh = F.spinor_to_host(xe, lat, 0, 0)
    k = 5
    par = wilson.parity_field(dims).reshape(-1) == 0
    full_x = np.zeros(rhs.shape[1:], dtype=np.complex128)
    full_x.reshape(-1, 4, 3)[par] = xeh[k].reshape(-1, 4, 3)
    b_e = wilson.restrict(rhs[k], 0)
    r = b_e - wilson.schur_dag_schur(U, full_x, m, BC)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b_e)
