"""GPU tests of the launch-shape autotuner of the FP32 / FP16 hop.

Every shape computes the hop's arithmetic in the same order (one site per
thread with 128 or 256 threads per block and register caps, one site per
thread with the links of each 4D site staged in shared memory, one site per
thread with its two spin components paired in packed FP32x2 instructions, or
two sites per thread in packed FP32x2 instructions), so a table that forces a shape must change
nothing in a hop's result: hops agree exactly across shapes and with the FP64
oracle within the storage precision's tolerance. Only the grouping of the
block partial sums of the solver's reductions depends on the block size (an
FP64 rounding difference), so a whole mixed-precision solve takes the same
iterations up to one and reaches an oracle-recomputed FP64 residual below its
tolerance with every shape.
"""
import itertools

import numpy as np
import pytest

from oracle import cg as ocg
from oracle import dwf, wilson
from synthetic import gauge_field, gaussian_spinor
from tests.layout import rel_l2, to_cb

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {1: 1e-5, 2: 3e-3}
BC = (1.0, 1.0, 1.0, -1.0)
NSHAPES = 9


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1512_03487_gb300 as L
    from paper_1512_03487_gb300 import fields
    L.fields = fields
    yield L
    L.lqcd_tune_clear()


def _keys(dims, n5):
    X, Y, Z, T = dims
    for prec, recon, dag, epi, red, full in itertools.product((1, 2), (12, 18), (0, 1), range(4), range(3), (0, 1)):
        yield (f"hop prec={prec} recon={recon} dagger={dag} epi={epi} red={red} full={full} "
               f"lat={X}x{Y}x{Z}x{T} n5={n5}")


def _force(L, tmp_path, dims, n5, shape):
    """Load a table that sets every hop key of this lattice to one shape."""
    path = tmp_path / f"force_{shape}.txt"
    path.write_text("".join(f"{shape}\t{k}\n" for k in _keys(dims, n5)))
    L.lqcd_tune_load(str(path))


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("recon", [12, 18])
@pytest.mark.parametrize("n5", [1, 4, 12])
def test_every_shape_gives_identical_hops(L, tmp_path, prec, recon, n5):
    """Ragged lattice (Vh = 90 per 4D checkerboard: several blocks and a partial
    one for every shape), both daggers, single checkerboard and full field; with
    n5 = 4 and 12 the link-staging shape shares each 4D site's links across its
    n5 threads, 4D sites straddling block boundaries for n5 = 12."""
    dims = (6, 2, 6, 10)
    U = gauge_field(dims, "haar", 21)
    psi = gaussian_spinor(dims, 22, lead=(n5,))
    lat = L.lattice(dims, n5=n5, bc=BC)
    op = L.operator(prec=prec, recon=recon)
    F = L.fields
    g = F.gauge_to_device(U, lat, prec, recon)
    fin_full = F.spinor_to_device(psi, lat, prec, L.LQCD_FULL)
    fin_odd = F.spinor_to_device(to_cb(psi, 1), lat, prec, L.LQCD_ODD)
    results = {}
    for shape in range(NSHAPES):
        _force(L, tmp_path, dims, n5, shape)
        for dag in (0, 1):
            out_full = F.empty(L.lqcd_spinor_bytes(lat, prec, L.LQCD_FULL))
            L.lqcd_dslash(out_full, fin_full, g, lat, op, L.LQCD_FULL, dag)
            out_even = F.empty(L.lqcd_spinor_bytes(lat, prec, L.LQCD_EVEN))
            L.lqcd_dslash(out_even, fin_odd, g, lat, op, L.LQCD_EVEN, dag)
            results[shape, dag] = (F.spinor_to_host(out_full, lat, prec, L.LQCD_FULL),
                                   F.spinor_to_host(out_even, lat, prec, L.LQCD_EVEN))
        key = (f"hop prec={prec} recon={recon} dagger=1 epi=0 red=0 full=1 "
               f"lat={dims[0]}x{dims[1]}x{dims[2]}x{dims[3]} n5={n5}")
        assert L.lqcd_tune_get(key) == shape  # a loaded entry is never re-timed
    for dag in (0, 1):
        expect_full = wilson.hop(U, psi, BC, dag)
        expect_even = to_cb(wilson.hop(U, wilson.restrict(psi, 1), BC, dag), 0)
        for shape in range(NSHAPES):
            got_full, got_even = results[shape, dag]
            assert rel_l2(got_full, expect_full) <= TOL[prec]
            assert rel_l2(got_even, expect_even) <= TOL[prec]
            np.testing.assert_array_equal(got_full, results[0, dag][0])
            np.testing.assert_array_equal(got_even, results[0, dag][1])


@pytest.mark.parametrize("prec", [1, 2])
def test_every_shape_domain_wall_operators(L, tmp_path, prec):
    """The M5op and fused M5op^-1 epilogues (L_s = 4 lanes of a 4D site in the
    scan, for both sites of a thread) under every shape, against the oracle's
    dense-LU M5op^-1."""
    dims, Ls, M5, mf = (4, 2, 6, 10), 4, 1.8, 0.02
    U = gauge_field(dims, "haar", 31)
    psi = gaussian_spinor(dims, 32, lead=(Ls,))
    lat = L.lattice(dims, n5=Ls, bc=BC)
    op = L.operator(kind=L.LQCD_DWF, M5=M5, mf=mf, prec=prec, recon=12)
    F = L.fields
    g = F.gauge_to_device(U, lat, prec, 12)
    fin = F.spinor_to_device(to_cb(psi, 0), lat, prec, L.LQCD_EVEN)
    tmp = F.empty(L.lqcd_operator_workspace_bytes(lat, op, L.LQCD_EVEN))
    first = {}
    for shape in range(NSHAPES):
        _force(L, tmp_path, dims, Ls, shape)
        for dag in (0, 1):
            out = F.empty(L.lqcd_spinor_bytes(lat, prec, L.LQCD_EVEN))
            L.lqcd_M(out, fin, g, lat, op, L.LQCD_EVEN, dag, tmp)
            got = F.spinor_to_host(out, lat, prec, L.LQCD_EVEN)
            expect = to_cb(dwf.schur(U, wilson.restrict(psi, 0), M5, mf, BC, dag), 0)
            assert rel_l2(got, expect) <= TOL[prec]
            if shape == 0:
                first[dag] = got
            np.testing.assert_array_equal(got, first[dag])


def test_every_shape_same_solve(L, tmp_path):
    """Mixed-precision even-odd CGNR (FP16 storage, FP32 replacements, FP64
    updates) with every in-iteration hop (plain, norm-reducing, fused update)
    forced to each shape: the same iteration counts (up to one, from the block
    partials' grouping), and the oracle's FP64 full-system residual of every
    returned x is below the tolerance."""
    dims, m = (6, 4, 4, 10), 0.05
    U = gauge_field(dims, "haar", 41)
    b = gaussian_spinor(dims, 42, lead=(1,))
    lat = L.lattice(dims, bc=BC)
    op = L.operator(mass=m)
    F = L.fields
    g64 = F.gauge_to_device(U, lat, 0, 18)
    g16 = F.gauge_to_device(U, lat, 2, 12)
    bd = F.spinor_to_device(b, lat, 0, L.LQCD_FULL)
    prm = L.solver_params(tol=1e-10, maxiter=2000, sloppy_prec=2, sloppy_recon=12, delta=1e-4, delta_mid=0.01)
    ws = F.empty(L.lqcd_eo_solve_workspace_bytes(lat, op, prm))
    iters = []
    for shape in range(NSHAPES):
        _force(L, tmp_path, dims, 1, shape)
        L.lqcd_release_caches()  # graphs captured under another shape
        x = F.empty(L.lqcd_spinor_bytes(lat, 0, L.LQCD_FULL))
        info = L.lqcd_eo_solve(x, bd, g64, g16, lat, op, prm, ws)
        xh = F.spinor_to_host(x, lat, 0, L.LQCD_FULL)
        res = np.linalg.norm(b - wilson.dirac(U, xh, m, BC)) / np.linalg.norm(b)
        assert res <= 1e-10, (shape, res)
        iters.append(info.iterations)
    assert max(iters) - min(iters) <= 1, iters


def test_solver_tuning_pass_records_its_hops(L):
    """With an empty table, the first mixed solve times its in-iteration hops
    (the norm-reducing M_hat hop and the fused-update M_hat^dag hop) in its
    tuning pass, and the captured iterations then use the recorded shapes."""
    L.lqcd_tune_clear()
    dims, m = (4, 4, 6, 8), 0.1
    U = gauge_field(dims, "haar", 51)
    b = gaussian_spinor(dims, 52, lead=(1,))
    lat = L.lattice(dims, bc=BC)
    op = L.operator(mass=m)
    F = L.fields
    g64 = F.gauge_to_device(U, lat, 0, 18)
    g32 = F.gauge_to_device(U, lat, 1, 12)
    be = F.spinor_to_device(to_cb(b, 0), lat, 0, L.LQCD_EVEN)
    prm = L.solver_params(tol=1e-10, maxiter=2000, sloppy_prec=1, sloppy_recon=12, delta=1e-3)
    ws = F.empty(L.lqcd_cg_workspace_bytes(lat, op, prm, L.LQCD_EVEN))
    x = F.empty(L.lqcd_spinor_bytes(lat, 0, L.LQCD_EVEN))
    L.lqcd_release_caches()
    L.lqcd_cg_solve(x, be, g64, g32, lat, op, prm, L.LQCD_EVEN, ws)
    lat_s = "x".join(str(d) for d in dims)
    for dag, epi, red in ((0, 0, 0), (0, 1, 1), (1, 0, 0), (1, 1, 2)):
        v = L.lqcd_tune_get(f"hop prec=1 recon=12 dagger={dag} epi={epi} red={red} full=0 lat={lat_s} n5=1")
        assert 0 <= v < NSHAPES, (dag, epi, red, v)
    xh = F.spinor_to_host(x, lat, 0, L.LQCD_EVEN)
    full_x = np.zeros_like(b)
    full_b = np.zeros_like(b)
    par = wilson.parity_field(dims).reshape(-1) == 0
    full_x.reshape(1, -1, 4, 3)[:, par] = xh.reshape(1, -1, 4, 3)
    full_b.reshape(1, -1, 4, 3)[:, par] = to_cb(b, 0).reshape(1, -1, 4, 3)
    res = ocg.true_residual(lambda v: wilson.schur_dag_schur(U, v, m, BC), full_x, full_b)
    assert res <= 1e-10


def test_tuning_disabled_keeps_the_table(L):
    L.lqcd_tune_clear()
    L.lqcd_tune_set_enabled(False)
    try:
        dims = (4, 4, 4, 4)
        lat = L.lattice(dims, bc=BC)
        op = L.operator(prec=1, recon=12)
        F = L.fields
        g = F.gauge_to_device(gauge_field(dims, "haar", 61), lat, 1, 12)
        fin = F.spinor_to_device(to_cb(gaussian_spinor(dims, 62, lead=(1,)), 1), lat, 1, L.LQCD_ODD)
        out = F.empty(L.lqcd_spinor_bytes(lat, 1, L.LQCD_EVEN))
        L.lqcd_dslash(out, fin, g, lat, op, L.LQCD_EVEN, 0)
        torch.cuda.synchronize()
        assert L.lqcd_tune_entries() == 0
    finally:
        L.lqcd_tune_set_enabled(True)
