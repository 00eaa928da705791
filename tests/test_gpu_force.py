"""GPU fermion force against the FP64 oracle."""
import numpy as np
import pytest

from oracle import force as oforce
from oracle import wilson
from synthetic import gauge_field, gaussian_spinor
from tests.layout import rel_l2

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


@pytest.mark.parametrize("dims,recon", [((4, 4, 4, 4), 18), ((6, 4, 2, 6), 12)])
def test_force_kernel_matches_oracle(L, dims, recon):
    """Same X, Y on both sides: the kernel alone against the oracle formula."""
    U = gauge_field(dims, "haar", 201)
    X = gaussian_spinor(dims, 202)
    Y = gaussian_spinor(dims, 203)
    lat = L.lattice(dims, bc=BC)
    op = L.operator(mass=0.05, recon=recon)
    F = L.fields
    g = F.gauge_to_device(U, lat, 0, recon)
    Xd = F.spinor_to_device(X[None], lat, 0, 2)
    Yd = F.spinor_to_device(Y[None], lat, 0, 2)
    grad_o, F_o = oforce.force_terms(U, X, Y, BC)
    for kind, ref in ((L.LQCD_FORCE_TA, F_o), (L.LQCD_FORCE_GRAD, grad_o)):
        out = F.empty(L.lqcd_gauge_bytes(lat, 0, 18))
        L.lqcd_force(out, g, Xd, Yd, lat, op, kind)
        got = F.gauge_to_host(out, lat, 0, 18)
        assert rel_l2(got, ref) <= 1e-12


def test_force_end_to_end(L):
    """X from the GPU CG (FP64, tol 1e-12), Y = M X, force; compared with the
    oracle's own solve and force."""
    dims, m = (4, 4, 4, 6), 0.05
    U = gauge_field(dims, "haar", 211)
    phi = gaussian_spinor(dims, 212)
    lat = L.lattice(dims, bc=BC)
    op = L.operator(mass=m)
    F = L.fields
    g = F.gauge_to_device(U, lat, 0, 18)
    phid = F.spinor_to_device(phi[None], lat, 0, 2)
    prm = L.solver_params(tol=1e-12, maxiter=5000)
    X = F.empty(L.lqcd_spinor_bytes(lat, 0, 2))
    ws = F.empty(L.lqcd_cg_workspace_bytes(lat, op, prm, 2))
    L.lqcd_cg_solve(X, phid, g, g, lat, op, prm, 2, ws)
    Y = F.empty(L.lqcd_spinor_bytes(lat, 0, 2))
    L.lqcd_M(Y, X, g, lat, op, 2, 0, None)
    out = F.empty(L.lqcd_gauge_bytes(lat, 0, 18))
    L.lqcd_force(out, g, X, Y, lat, op, L.LQCD_FORCE_TA)
    got = F.gauge_to_host(out, lat, 0, 18)
    S, grad_o, F_o, X_o, Y_o = oforce.force(U, phi, m, BC, tol=1e-13)
    assert rel_l2(F.spinor_to_host(X, lat, 0, 2)[0], X_o) < 1e-9
    assert rel_l2(got, F_o) < 1e-9
    np.testing.assert_allclose(np.trace(got, axis1=-2, axis2=-1), 0, atol=1e-12)
    assert wilson is not None
