"""GPU parity of the hop, the Dirac operators and the even-odd helpers against
the FP64 oracle, through the C ABI.

Tolerances (relative L2 against the FP64 oracle on the same inputs):
  FP64  1e-12  (rounding-order differences only)
  FP32  1e-5   (FP32 storage and arithmetic, unit roundoff 6e-8)
  FP16  3e-3   (FP16 storage: unit roundoff 2^-11 = 4.9e-4 of the site norm for
               spinors, of 1 for links; the output error is a few times that)
"""
import numpy as np
import pytest

from oracle import dwf, wilson
from synthetic import gauge_field, gaussian_spinor
from tests.layout import from_cb, rel_l2, to_cb

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {0: 1e-12, 1: 1e-5, 2: 3e-3}
BC = (1.0, 1.0, 1.0, -1.0)


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1512_03487_gb300 as L
    from paper_1512_03487_gb300 import fields
    L.fields = fields
    return L


def _hop_case(L, dims, n5, prec, recon, dagger, subset, seed=1):
    U = gauge_field(dims, "haar", seed)
    psi = gaussian_spinor(dims, seed + 1, lead=(n5,))
    lat = L.lattice(dims, n5=n5, bc=BC)
    op = L.operator(prec=prec, recon=recon)
    F = L.fields
    g = F.gauge_to_device(U, lat, prec, recon)
    if subset == L.LQCD_FULL:
        fin = F.spinor_to_device(psi, lat, prec, L.LQCD_FULL)
        expect = wilson.hop(U, psi, BC, dagger)
    else:
        src_par = 1 - subset
        fin = F.spinor_to_device(to_cb(psi, src_par), lat, prec, src_par)
        expect = to_cb(wilson.hop(U, wilson.restrict(psi, src_par), BC, dagger), subset)
    out = F.empty(L.lqcd_spinor_bytes(lat, prec, subset))
    L.lqcd_dslash(out, fin, g, lat, op, subset, dagger)
    got = F.spinor_to_host(out, lat, prec, subset)
    return got, expect


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("recon", [18, 12])
@pytest.mark.parametrize("dagger", [0, 1])
@pytest.mark.parametrize("subset", [0, 1, 2])
def test_hop_matches_oracle(L, prec, recon, dagger, subset):
    got, expect = _hop_case(L, (6, 4, 4, 6), 1, prec, recon, dagger, subset)
    assert rel_l2(got, expect) <= TOL[prec]


@pytest.mark.parametrize("dims", [(4, 2, 6, 2), (2, 2, 2, 2), (8, 6, 2, 4)])
@pytest.mark.parametrize("n5", [1, 3])
def test_hop_degenerate_shapes(L, dims, n5):
    """Extent-2 directions (forward and backward neighbour are the same site),
    a single partial block, and an inner dimension n5 > 1 (L_s-replicated /
    multi-RHS hop)."""
    for subset in (0, 1, 2):
        got, expect = _hop_case(L, dims, n5, 0, 18, 0, subset, seed=7)
        assert rel_l2(got, expect) <= TOL[0]
        got, expect = _hop_case(L, dims, n5, 1, 12, 1, subset, seed=9)
        assert rel_l2(got, expect) <= TOL[1]


def test_pack_roundtrip(L):
    dims = (6, 4, 4, 6)
    lat = L.lattice(dims, n5=2)
    F = L.fields
    psi = gaussian_spinor(dims, 5, lead=(2,))
    for prec in (0, 1, 2):
        back = F.spinor_to_host(F.spinor_to_device(psi, lat, prec, 2), lat, prec, 2)
        assert rel_l2(back, psi) <= {0: 0, 1: 1e-7, 2: 1e-3}[prec]
        cb = to_cb(psi, 1)
        back = F.spinor_to_host(F.spinor_to_device(cb, lat, prec, 1), lat, prec, 1)
        assert rel_l2(back, cb) <= {0: 0, 1: 1e-7, 2: 1e-3}[prec]
    U = gauge_field(dims, "haar", 6)
    for prec in (0, 1, 2):
        for recon in (18, 12):
            back = F.gauge_to_host(F.gauge_to_device(U, lat, prec, recon), lat, prec, recon)
            tol = {0: 1e-14, 1: 2e-7, 2: 2e-3}[prec]
            assert np.abs(back - U).max() <= tol * (4 if recon == 12 else 1)
    # the package's checkerboard helper agrees with the test's own
    np.testing.assert_array_equal(F.checkerboard(psi, 1), to_cb(psi, 1))


def _field(L, arr, lat, prec, subset):
    return L.fields.spinor_to_device(arr, lat, prec, subset)


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("dagger", [0, 1])
def test_wilson_operators(L, prec, dagger):
    dims, m = (6, 4, 4, 6), 0.1
    U = gauge_field(dims, "haar", 11)
    psi = gaussian_spinor(dims, 12, lead=(1,))
    lat = L.lattice(dims, bc=BC)
    op = L.operator(mass=m, prec=prec, recon=18)
    F = L.fields
    g = F.gauge_to_device(U, lat, prec, 18)
    # full operator
    out = F.empty(L.lqcd_spinor_bytes(lat, prec, 2))
    L.lqcd_M(out, _field(L, psi, lat, prec, 2), g, lat, op, 2, dagger, None)
    expect = wilson.dirac(U, psi, m, BC, dagger=bool(dagger))
    assert rel_l2(F.spinor_to_host(out, lat, prec, 2), expect) <= TOL[prec]
    # Schur complement on even sites
    pe = to_cb(psi, 0)
    tmp = F.empty(L.lqcd_operator_workspace_bytes(lat, op, 0))
    out = F.empty(L.lqcd_spinor_bytes(lat, prec, 0))
    L.lqcd_M(out, _field(L, pe, lat, prec, 0), g, lat, op, 0, dagger, tmp)
    expect = to_cb(wilson.schur(U, from_cb(pe, 0), m, BC, dagger=bool(dagger)), 0)
    assert rel_l2(F.spinor_to_host(out, lat, prec, 0), expect) <= TOL[prec]


@pytest.mark.parametrize("subset", [0, 2])
def test_wilson_mdagm(L, subset):
    dims, m = (4, 4, 4, 6), 0.05
    U = gauge_field(dims, "haar", 13)
    psi = gaussian_spinor(dims, 14, lead=(1,))
    lat = L.lattice(dims, bc=BC)
    op = L.operator(mass=m)
    F = L.fields
    g = F.gauge_to_device(U, lat, 0, 18)
    arr = psi if subset == 2 else to_cb(psi, 0)
    out = F.empty(L.lqcd_spinor_bytes(lat, 0, subset))
    tmp = F.empty(L.lqcd_operator_workspace_bytes(lat, op, subset))
    L.lqcd_MdagM(out, _field(L, arr, lat, 0, subset), g, lat, op, subset, tmp)
    if subset == 2:
        expect = wilson.dirac_dag_dirac(U, psi, m, BC)
    else:
        expect = to_cb(wilson.schur_dag_schur(U, from_cb(arr, 0), m, BC), 0)
    assert rel_l2(F.spinor_to_host(out, lat, 0, subset), expect) <= TOL[0]


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("dagger", [0, 1])
@pytest.mark.parametrize("Ls", [6, 2, 8, 16, 32])
def test_dwf_operators(L, prec, dagger, Ls):
    """Full and Schur domain-wall operators; L_s = 6 takes the closed-form M5op^-1
    kernel, the powers of two up to 32 the warp-shuffle scan."""
    dims, M5, mf = (4, 4, 2, 6), 1.8, 0.02
    U = gauge_field(dims, "haar", 21)
    psi = gaussian_spinor(dims, 22, lead=(Ls,))
    lat = L.lattice(dims, n5=Ls, bc=BC)
    op = L.operator(kind=L.LQCD_DWF, M5=M5, mf=mf, prec=prec, recon=12)
    F = L.fields
    g = F.gauge_to_device(U, lat, prec, 12)
    out = F.empty(L.lqcd_spinor_bytes(lat, prec, 2))
    L.lqcd_M(out, _field(L, psi, lat, prec, 2), g, lat, op, 2, dagger, None)
    expect = dwf.dirac(U, psi, M5, mf, BC, dagger=bool(dagger))
    assert rel_l2(F.spinor_to_host(out, lat, prec, 2), expect) <= TOL[prec]
    pe = to_cb(psi, 0)
    tmp = F.empty(L.lqcd_operator_workspace_bytes(lat, op, 0))
    out = F.empty(L.lqcd_spinor_bytes(lat, prec, 0))
    L.lqcd_M(out, _field(L, pe, lat, prec, 0), g, lat, op, 0, dagger, tmp)
    expect = to_cb(dwf.schur(U, from_cb(pe, 0), M5, mf, BC, dagger=bool(dagger)), 0)
    assert rel_l2(F.spinor_to_host(out, lat, prec, 0), expect) <= TOL[prec]


@pytest.mark.parametrize("kind", [0, 1])
def test_eo_prepare_and_reconstruct(L, kind):
    dims = (4, 4, 2, 6)
    n5 = 1 if kind == 0 else 4
    U = gauge_field(dims, "haar", 31)
    b = gaussian_spinor(dims, 32, lead=(n5,))
    x = gaussian_spinor(dims, 33, lead=(n5,))
    lat = L.lattice(dims, n5=n5, bc=BC)
    op = L.operator(kind=kind, mass=0.1, M5=1.8, mf=0.05)
    F = L.fields
    g = F.gauge_to_device(U, lat, 0, 18)
    bd = _field(L, b, lat, 0, 2)
    tmp = F.empty(L.lqcd_operator_workspace_bytes(lat, op, 0))
    bhat = F.empty(L.lqcd_spinor_bytes(lat, 0, 0))
    L.lqcd_eo_prepare(bhat, bd, g, lat, op, tmp)
    if kind == 0:
        expect = wilson.prepare_source(U, b, 0.1, BC)
    else:
        expect = dwf.prepare_source(U, b, 1.8, 0.05, BC)
    assert rel_l2(F.spinor_to_host(bhat, lat, 0, 0), to_cb(expect, 0)) <= TOL[0]
    xd = _field(L, x, lat, 0, 2)  # only the even half is read
    L.lqcd_eo_reconstruct(xd, bd, g, lat, op, tmp)
    if kind == 0:
        expect = wilson.reconstruct(U, wilson.restrict(x, 0), b, 0.1, BC)
    else:
        expect = dwf.reconstruct(U, wilson.restrict(x, 0), b, 1.8, 0.05, BC)
    assert rel_l2(F.spinor_to_host(xd, lat, 0, 2), expect) <= TOL[0]
