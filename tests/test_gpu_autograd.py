"""The force behind torch.autograd: gradient against the oracle and against
finite differences of the GPU action itself."""
import numpy as np
import pytest

from oracle import force as oforce
from synthetic import gauge_field, gaussian_spinor, make_rng
from tests.layout import rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
BC = (1.0, 1.0, 1.0, -1.0)


@pytest.fixture(scope="module")
def AG():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_03487_gb300 import autograd
    return autograd


def _inputs(dims, seed):
    U = gauge_field(dims, "haar", seed)
    phi = gaussian_spinor(dims, seed + 1)
    return U, phi


@pytest.mark.parametrize("checkpoint", [False, True])
def test_autograd_gradient_matches_oracle(AG, checkpoint):
    dims, m = (4, 4, 4, 4), 0.05
    U, phi = _inputs(dims, 301)
    Ut = torch.tensor(U, device="cuda", requires_grad=True)
    pt = torch.tensor(phi, device="cuda")
    S = AG.fermion_action(Ut, pt, m, BC, tol=1e-13, checkpoint=checkpoint)
    S.backward()
    S_o, grad_o, F_o, _, _ = oforce.force(U, phi, m, BC, tol=1e-13)
    assert abs(S.item() - S_o) <= 1e-10 * abs(S_o)
    assert rel_l2(Ut.grad.cpu().numpy(), grad_o) <= 1e-9


def test_autograd_gradient_matches_gpu_finite_difference(AG):
    dims, m = (4, 4, 2, 4), 0.1
    U, phi = _inputs(dims, 311)
    Ut = torch.tensor(U, device="cuda", requires_grad=True)
    pt = torch.tensor(phi, device="cuda")
    S = AG.fermion_action(Ut, pt, m, BC, tol=1e-14)
    S.backward()
    rng = make_rng(312)
    dU = torch.tensor(rng.standard_normal(U.shape) + 1j * rng.standard_normal(U.shape), device="cuda")
    eps = 1e-5
    with torch.no_grad():
        sp = AG.fermion_action(Ut + eps * dU, pt, m, BC, tol=1e-14).item()
        sm = AG.fermion_action(Ut - eps * dU, pt, m, BC, tol=1e-14).item()
    fd = (sp - sm) / (2 * eps)
    analytic = torch.sum((dU.conj() * Ut.grad).real).item()
    assert abs(fd - analytic) <= 1e-5 * abs(analytic)


def test_traceless_hermitian_force(AG):
    dims, m = (4, 4, 4, 6), 0.05
    U, phi = _inputs(dims, 321)
    S, F = AG.force_traceless_hermitian(torch.tensor(U, device="cuda"), torch.tensor(phi, device="cuda"), m, BC,
                                        tol=1e-13)
    S_o, _, F_o, _, _ = oforce.force(U, phi, m, BC, tol=1e-13)
    assert rel_l2(F.cpu().numpy(), F_o) <= 1e-9
    assert abs(S.item() - S_o) <= 1e-10 * abs(S_o)
    Fh = F.cpu().numpy()
    np.testing.assert_allclose(Fh, np.conj(np.swapaxes(Fh, -1, -2)), atol=1e-12)


def test_spinor_dot_re_matches_numpy():
    """lqcd_spinor_dot_re (the action's S = Re <phi, X>) against numpy's
    Re sum conj(a) b on a ragged lattice; the reduction is deterministic, so two
    calls agree bit for bit."""
    import numpy as np

    import paper_1512_03487_gb300 as L
    from paper_1512_03487_gb300 import fields as F
    from synthetic import gaussian_spinor
    dims = (6, 4, 2, 10)
    lat = L.lattice(dims)
    a = gaussian_spinor(dims, 71, lead=(1,))
    b = gaussian_spinor(dims, 72, lead=(1,))
    ad = F.spinor_to_device(a, lat, 0, L.LQCD_FULL)
    bd = F.spinor_to_device(b, lat, 0, L.LQCD_FULL)
    ws = F.empty(L.lqcd_reduce_workspace_bytes(lat))
    got = L.lqcd_spinor_dot_re(ad, bd, lat, ws)
    expect = float(np.real(np.vdot(a, b)))
    assert abs(got - expect) <= 1e-12 * np.sqrt(np.vdot(a, a).real * np.vdot(b, b).real)
    assert L.lqcd_spinor_dot_re(ad, bd, lat, ws) == got
