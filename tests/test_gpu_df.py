"""GPU parity of the double-float (LQCD_F64_DF) Wilson operator: FP64 fields,
arithmetic in pairs of FP32 numbers (about 48 significant bits).

Bars: against the FP64 oracle, relative L2 <= 1e-12 (the FP64 bar, which
only rounding order may use); against the library's own FP64 hop on the same
inputs, <= 1e-13, a few times the 2^-46 per-operation bound of the
double-float addition summed over a hop's 8 directions. A mixed-precision solve
whose reliable updates run in double-float arithmetic must still reach the
oracle-recomputed FP64 true residual: its exit test is on b - A x computed
within a few 1e-15 |b| of the FP64 value.
"""
import numpy as np
import pytest

from oracle import dwf, wilson
from synthetic import gauge_field, gaussian_spinor
from tests.layout import rel_l2, to_cb

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

BC = (1.0, 1.0, 1.0, -1.0)
DF = 3


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1512_03487_gb300 as L
    from paper_1512_03487_gb300 import fields
    L.fields = fields
    assert L.LQCD_F64_DF == DF
    return L


@pytest.mark.parametrize("recon", [18, 12])
@pytest.mark.parametrize("dagger", [0, 1])
@pytest.mark.parametrize("subset", [0, 1, 2])
@pytest.mark.parametrize("field", ["haar", "exp"])
def test_df_hop_matches_oracle_and_fp64(L, recon, dagger, subset, field):
    dims = (6, 4, 2, 10)  # Vh = 240: one full and one partial block
    U = gauge_field(dims, field, 3, eps=0.3)
    psi = gaussian_spinor(dims, 4, lead=(1,)) * 1e3  # magnitudes away from 1
    lat = L.lattice(dims, bc=BC)
    F = L.fields
    g = F.gauge_to_device(U, lat, 0, recon)
    if subset == L.LQCD_FULL:
        fin = F.spinor_to_device(psi, lat, 0, L.LQCD_FULL)
        expect = wilson.hop(U, psi, BC, dagger)
    else:
        fin = F.spinor_to_device(to_cb(psi, 1 - subset), lat, 0, 1 - subset)
        expect = to_cb(wilson.hop(U, wilson.restrict(psi, 1 - subset), BC, dagger), subset)
    got = {}
    for prec in (0, DF):
        out = F.empty(L.lqcd_spinor_bytes(lat, 0, subset))
        L.lqcd_dslash(out, fin, g, lat, L.operator(prec=prec, recon=recon), subset, dagger)
        got[prec] = F.spinor_to_host(out, lat, 0, subset)
    assert rel_l2(got[DF], expect) <= 1e-12
    assert rel_l2(got[DF], got[0]) <= 1e-13
    assert rel_l2(got[DF], got[0]) > 0.0 or np.array_equal(got[DF], got[0])


@pytest.mark.parametrize("subset", [0, 2])
@pytest.mark.parametrize("dagger", [0, 1])
def test_df_operator_matches_oracle(L, subset, dagger):
    """lqcd_M: the full operator (xpay over both checkerboards) and the Schur
    complement (plain hop, then the xpay hop) in double-float arithmetic."""
    dims, m = (4, 4, 6, 8), 0.05
    U = gauge_field(dims, "haar", 11)
    psi = gaussian_spinor(dims, 12, lead=(1,))
    lat = L.lattice(dims, bc=BC)
    op = L.operator(mass=m, prec=DF, recon=18)
    F = L.fields
    g = F.gauge_to_device(U, lat, 0, 18)
    if subset == L.LQCD_FULL:
        fin = F.spinor_to_device(psi, lat, 0, L.LQCD_FULL)
        expect = wilson.dirac(U, psi, m, BC, dagger)
        tmp = None
    else:
        fin = F.spinor_to_device(to_cb(psi, 0), lat, 0, L.LQCD_EVEN)
        expect = to_cb(wilson.schur(U, wilson.restrict(psi, 0), m, BC, dagger), 0)
        tmp = F.empty(L.lqcd_operator_workspace_bytes(lat, op, L.LQCD_EVEN))
    out = F.empty(L.lqcd_spinor_bytes(lat, 0, subset))
    L.lqcd_M(out, fin, g, lat, op, subset, dagger, tmp)
    assert rel_l2(F.spinor_to_host(out, lat, 0, subset), expect) <= 1e-12


def test_df_split_edge_values(L):
    """Zeros, signs, values spanning 1e-30 .. 1e30 and exact powers of two go
    through the split and the recombination: a hop on a field with a single
    nonzero site (component value v + i v / 7) and unit links agrees with the
    FP64 hop and the oracle to 2e-14 |v| (the split keeps 48 of the 53 bits)."""
    dims = (4, 2, 2, 4)
    lat = L.lattice(dims, bc=(1.0, 1.0, 1.0, 1.0))
    F = L.fields
    U = gauge_field(dims, "unit", 0)
    g = F.gauge_to_device(U, lat, 0, 18)
    for v in (0.0, 1.0, -2.0 ** -20, 3.0e-30, -7.5e29, 1.0 / 3.0, np.pi * 1e5):
        psi = np.zeros((1, dims[3], dims[2], dims[1], dims[0], 4, 3), dtype=np.complex128)
        psi[0, 1, 0, 1, 2, 0, 1] = v + 1j * v / 7.0  # site (x, y, z, t) = (2, 1, 0, 1), spin 0, colour 1
        fin = F.spinor_to_device(psi, lat, 0, L.LQCD_FULL)
        res = {}
        for prec in (0, DF):
            out = F.empty(L.lqcd_spinor_bytes(lat, 0, L.LQCD_FULL))
            L.lqcd_dslash(out, fin, g, lat, L.operator(prec=prec, recon=18), L.LQCD_FULL, 0)
            res[prec] = F.spinor_to_host(out, lat, 0, L.LQCD_FULL)
        scale = max(abs(v), 1e-300)
        assert np.max(np.abs(res[DF] - res[0])) <= 2e-14 * scale
        expect = wilson.hop(U, psi, (1.0, 1.0, 1.0, 1.0))
        assert np.max(np.abs(res[DF] - expect)) <= 2e-14 * scale


@pytest.mark.parametrize("sloppy", [1, 2])
def test_df_reliable_updates_solve(L, sloppy):
    """lqcd_eo_solve with FP32 / FP16 inner storage and double-float reliable
    updates and source preparation: the oracle's FP64 full-system residual of x
    is below the tolerance, with no more than one extra reliable update over the
    FP64-update solve."""
    dims, m = (6, 4, 4, 10), 0.05
    U = gauge_field(dims, "exp", 21, eps=0.3)
    b = gaussian_spinor(dims, 22, lead=(1,))
    lat = L.lattice(dims, bc=BC)
    op = L.operator(mass=m)
    F = L.fields
    g64 = F.gauge_to_device(U, lat, 0, 18)
    gs = F.gauge_to_device(U, lat, sloppy, 12)
    bd = F.spinor_to_device(b, lat, 0, L.LQCD_FULL)
    infos = {}
    for up in (0, DF):
        prm = L.solver_params(tol=1e-10, maxiter=3000, sloppy_prec=sloppy, sloppy_recon=12, delta=1e-3,
                              delta_mid=0.01 if sloppy == 2 else 0.0, update_prec=up)
        ws = F.empty(L.lqcd_eo_solve_workspace_bytes(lat, op, prm))
        x = F.empty(L.lqcd_spinor_bytes(lat, 0, L.LQCD_FULL))
        info = L.lqcd_eo_solve(x, bd, g64, gs, lat, op, prm, ws)
        xh = F.spinor_to_host(x, lat, 0, L.LQCD_FULL)
        res = np.linalg.norm(b - wilson.dirac(U, xh, m, BC)) / np.linalg.norm(b)
        assert res <= 1e-10, (up, res)
        infos[up] = info
    assert abs(infos[DF].reliable_updates - infos[0].reliable_updates) <= 1


@pytest.mark.parametrize("Ls", [4, 8])
@pytest.mark.parametrize("subset", [0, 2])
@pytest.mark.parametrize("dagger", [0, 1])
def test_df_domain_wall_operator_matches_oracle(L, Ls, subset, dagger):
    """Domain wall in double-float arithmetic (18-real links, L_s dividing 32):
    the full operator (M5op epilogue) and the Schur complement (M5op^-1 fused
    into the first hop by the warp-shuffle scan on double-float pairs, then the
    M5op hop), against the oracle's dense-LU M5op^-1 and the FP64 operator."""
    dims, M5, mf = (4, 2, 6, 8), 1.8, 0.02
    U = gauge_field(dims, "haar", 41)
    psi = gaussian_spinor(dims, 42, lead=(Ls,))
    lat = L.lattice(dims, n5=Ls, bc=BC)
    F = L.fields
    g = F.gauge_to_device(U, lat, 0, 18)
    if subset == L.LQCD_FULL:
        fin = F.spinor_to_device(psi, lat, 0, L.LQCD_FULL)
        expect = dwf.dirac(U, psi, M5, mf, BC, dagger)
    else:
        fin = F.spinor_to_device(to_cb(psi, 0), lat, 0, L.LQCD_EVEN)
        expect = to_cb(dwf.schur(U, wilson.restrict(psi, 0), M5, mf, BC, dagger), 0)
    got = {}
    for prec in (0, DF):
        op = L.operator(kind=L.LQCD_DWF, M5=M5, mf=mf, prec=prec, recon=18)
        tmp = None if subset == L.LQCD_FULL else F.empty(L.lqcd_operator_workspace_bytes(lat, op, L.LQCD_EVEN))
        out = F.empty(L.lqcd_spinor_bytes(lat, 0, subset))
        L.lqcd_M(out, fin, g, lat, op, subset, dagger, tmp)
        got[prec] = F.spinor_to_host(out, lat, 0, subset)
    assert rel_l2(got[DF], expect) <= 1e-12
    assert rel_l2(got[DF], got[0]) <= 1e-13


def test_df_domain_wall_rejections(L):
    """Double-float domain wall needs 18-real links and L_s dividing 32 (the
    fused M5op^-1): other forms are rejected on the host, before any launch."""
    dims = (4, 2, 2, 4)
    F = L.fields
    for Ls, recon in ((6, 18), (4, 12)):
        lat = L.lattice(dims, n5=Ls, bc=BC)
        op = L.operator(kind=L.LQCD_DWF, M5=1.8, mf=0.02, prec=DF, recon=recon)
        g = F.empty(L.lqcd_gauge_bytes(lat, 0, recon))
        fin = F.empty(L.lqcd_spinor_bytes(lat, 0, L.LQCD_FULL))
        out = F.empty(L.lqcd_spinor_bytes(lat, 0, L.LQCD_FULL))
        with pytest.raises(L.LqcdError):
            L.lqcd_M(out, fin, g, lat, op, L.LQCD_FULL, 0, None)


@pytest.mark.parametrize("Ls", [4, 6])
def test_df_domain_wall_solve(L, Ls):
    """lqcd_eo_solve on a domain-wall system with FP32 inner storage and
    update_prec = LQCD_F64_DF: double-float reliable updates where L_s divides 32
    (4), FP64 ones otherwise (6); the oracle's full-system residual of x meets
    the tolerance either way."""
    dims, M5, mf = (4, 4, 2, 8), 1.8, 0.05
    U = gauge_field(dims, "haar", 51)
    b = gaussian_spinor(dims, 52, lead=(Ls,))
    lat = L.lattice(dims, n5=Ls, bc=BC)
    op = L.operator(kind=L.LQCD_DWF, M5=M5, mf=mf)
    F = L.fields
    g64 = F.gauge_to_device(U, lat, 0, 18)
    g32 = F.gauge_to_device(U, lat, 1, 12)
    bd = F.spinor_to_device(b, lat, 0, L.LQCD_FULL)
    prm = L.solver_params(tol=1e-10, maxiter=5000, sloppy_prec=1, sloppy_recon=12, delta=1e-3, update_prec=DF)
    ws = F.empty(L.lqcd_eo_solve_workspace_bytes(lat, op, prm))
    x = F.empty(L.lqcd_spinor_bytes(lat, 0, L.LQCD_FULL))
    info = L.lqcd_eo_solve(x, bd, g64, g32, lat, op, prm, ws)
    xh = F.spinor_to_host(x, lat, 0, L.LQCD_FULL)
    res = np.linalg.norm(b - dwf.dirac(U, xh, M5, mf, BC)) / np.linalg.norm(b)
    assert res <= 1e-10, res
    assert info.true_rel_residual <= 1e-10
