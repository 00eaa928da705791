"""Block CG over the right-hand sides of a multi-RHS field: every column must
reach its own FP64 true residual, recomputed by the oracle from the returned
solution, including degenerate blocks (a zero column, two equal columns)."""
import numpy as np
import pytest

from oracle import cg as ocg
from oracle import wilson
from synthetic import gauge_field, gaussian_spinor
from tests.layout import from_cb, to_cb

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


def _block_solve(L, U, b, dims, m, sloppy, recon=12, tol=1e-10, maxiter=3000, update_prec=0):
    F = L.fields
    n = b.shape[0]
    lat = L.lattice(dims, n5=n, bc=BC)
    op = L.operator(mass=m)
    prm = L.solver_params(tol=tol, maxiter=maxiter, sloppy_prec=sloppy, sloppy_recon=recon, delta=0.01,
                          check_interval=16, update_prec=update_prec)
    g64 = F.gauge_to_device(U, lat, 0, 18)
    gs = F.gauge_to_device(U, lat, sloppy, recon) if sloppy else g64
    bd = F.spinor_to_device(b, lat, 0, 0)
    x = F.empty(L.lqcd_spinor_bytes(lat, 0, 0))
    ws = F.empty(L.lqcd_block_cg_workspace_bytes(lat, op, prm))
    info = L.lqcd_block_cg_solve(x, bd, g64, gs, lat, op, prm, ws, raise_on_error=False)
    return F.spinor_to_host(x, lat, 0, 0), info


def _check_columns(U, x, b, m, tol=1e-10):
    for k in range(b.shape[0]):
        if not np.any(b[k]):
            assert not np.any(x[k])
            continue
        res = ocg.true_residual(lambda v: wilson.schur_dag_schur(U, v, m, BC), from_cb(x[k:k + 1], 0),
                                from_cb(b[k:k + 1], 0))
        assert res <= tol, (k, res)


@pytest.mark.parametrize("sloppy,update_prec", [(0, 0), (1, 0), (2, 0), (1, 3), (2, 3)])
def test_block_cg_reaches_tolerance(L, sloppy, update_prec):
    """FP64, FP32 and FP16 inner operators; reliable updates on the FP64 pipe or
    in double-float arithmetic (update_prec 3)."""
    dims, m, n = (4, 4, 4, 8), 0.05, 6
    U = gauge_field(dims, "haar", 701)
    b = to_cb(gaussian_spinor(dims, 702, lead=(n,)), 0)
    x, info = _block_solve(L, U, b, dims, m, sloppy, update_prec=update_prec)
    assert info.status == 0, L.lqcd_last_error()
    _check_columns(U, x, b, m)
    assert info.true_rel_residual <= 1e-10


@pytest.mark.parametrize("n", [1, 3, 5, 9, 13, 16])
@pytest.mark.parametrize("sloppy", [0, 1])
def test_block_cg_every_gram_tile(L, n, sloppy):
    """Block sizes that take each register tile of the Gram kernel (1 x 1 for
    N <= 4 up to 4 x 4 for N <= 16, with ragged last tiles), on a lattice whose
    40 4D sites per checkerboard leave a partial last pass of staged sites."""
    dims, m = (2, 2, 2, 10), 0.1
    U = gauge_field(dims, "haar", 731 + n)
    b = to_cb(gaussian_spinor(dims, 732 + n, lead=(n,)), 0)
    x, info = _block_solve(L, U, b, dims, m, sloppy, update_prec=3 if sloppy else 0)
    assert info.status == 0, L.lqcd_last_error()
    _check_columns(U, x, b, m)


def test_block_cg_needs_no_more_iterations_than_independent_cg(L):
    dims, m, n = (4, 4, 4, 8), 0.02, 8
    U = gauge_field(dims, "exp", 711, eps=0.3)
    b = to_cb(gaussian_spinor(dims, 712, lead=(n,)), 0)
    xb, ib = _block_solve(L, U, b, dims, m, 0)
    F = L.fields
    lat = L.lattice(dims, n5=n, bc=BC)
    op = L.operator(mass=m)
    prm = L.solver_params(tol=1e-10, maxiter=3000)
    g = F.gauge_to_device(U, lat, 0, 18)
    x = F.empty(L.lqcd_spinor_bytes(lat, 0, 0))
    ws = F.empty(L.lqcd_cg_workspace_bytes(lat, op, prm, 0))
    ii = L.lqcd_cg_solve(x, F.spinor_to_device(b, lat, 0, 0), g, g, lat, op, prm, 0, ws)
    assert ib.status == 0 and ii.status == 0
    assert ib.iterations <= ii.iterations
    _check_columns(U, xb, b, m)


def test_block_cg_degenerate_columns(L):
    """A zero column and two identical columns make the block Gram matrices
    singular; the solve must still converge column by column."""
    dims, m, n = (4, 4, 2, 4), 0.1, 4
    U = gauge_field(dims, "haar", 721)
    b = to_cb(gaussian_spinor(dims, 722, lead=(n,)), 0)
    b[1] = 0.0
    b[3] = b[2]
    x, info = _block_solve(L, U, b, dims, m, 1)
    assert info.status == 0, L.lqcd_last_error()
    _check_columns(U, x, b, m)
    np.testing.assert_allclose(x[3], x[2], rtol=0, atol=1e-9 * np.abs(x[2]).max())
