"""Multigrid pieces on the GPU against the oracle (oracle/mg.py) on the same
seeded inputs -- block orthonormalisation, restriction, prolongation, the
Galerkin coarse operator and its stencil -- and multigrid-preconditioned GCR
solves that must reach the FP64 true residual of the full Wilson system."""
import numpy as np
import pytest

from oracle import mg, wilson
from synthetic import gauge_field, gaussian_spinor, make_rng

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
BC = (1.0, 1.0, 1.0, -1.0)
TOL = {0: 1e-12, 1: 2e-6}


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1512_03487_gb300 as L
    from paper_1512_03487_gb300 import fields
    L.fields = fields
    return L


def _vecs_to_device(L, V, lat, prec):
    return torch.cat([L.fields.spinor_to_device(v, lat, prec, 2) for v in V])


def _vecs_to_host(L, buf, nv, lat, prec):
    fb = L.lqcd_spinor_bytes(lat, prec, 2)
    return np.stack([L.fields.spinor_to_host(buf[k * fb:(k + 1) * fb], lat, prec, 2)[0] for k in range(nv)])


def _rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


CASES = [((4, 4, 4, 8), 2, 3), ((8, 4, 4, 4), 4, 2), ((8, 8, 8, 8), 4, 4)]


@pytest.mark.parametrize("dims,b,nv", CASES)
def test_block_orthonormalize(L, dims, b, nv):
    lat = L.lattice(dims, bc=BC)
    V = gaussian_spinor(dims, 2101, lead=(nv,))
    buf = _vecs_to_device(L, V, lat, 0)
    L.lqcd_mg_block_orthonormalize(buf, nv, b, lat)
    assert _rel(_vecs_to_host(L, buf, nv, lat, 0), mg.orthonormalize(V, b)) <= 1e-12


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dims,b,nv", CASES)
def test_restrict_prolong(L, prec, dims, b, nv):
    lat = L.lattice(dims, bc=BC)
    P = mg.orthonormalize(gaussian_spinor(dims, 2111, lead=(nv,)), b)
    psi = gaussian_spinor(dims, 2112)
    Pd = _vecs_to_device(L, P, lat, prec)
    if prec == 1:  # the oracle works on the FP32-rounded inputs
        P = P.astype(np.complex64).astype(np.complex128)
        psi = psi.astype(np.complex64).astype(np.complex128)
    ctype = torch.complex128 if prec == 0 else torch.complex64
    cd = mg.coarse_dims(dims, b)
    c = torch.empty(int(np.prod(cd)) * 2 * nv, dtype=ctype, device="cuda")
    L.lqcd_mg_restrict(c, L.fields.spinor_to_device(psi, lat, prec, 2), Pd, nv, b, prec, lat)
    assert _rel(c.cpu().numpy().reshape(-1), mg.restrict(P, psi, b).reshape(-1)) <= TOL[prec]
    ch = make_rng(2113).standard_normal((int(np.prod(cd)) * 2 * nv, 2)) @ np.array([1.0, 1j])
    f = L.fields.empty(L.lqcd_spinor_bytes(lat, prec, 2))
    L.lqcd_mg_prolong(f, torch.from_numpy(ch.astype(np.complex128 if prec == 0 else np.complex64)).cuda(), Pd, nv, b,
                      prec, lat)
    expect = mg.prolong(P, ch.reshape(tuple(reversed(cd)) + (2 * nv,)), b)
    assert _rel(L.fields.spinor_to_host(f, lat, prec, 2)[0], expect) <= TOL[prec]


@pytest.mark.parametrize("dims,b,nv", CASES)
def test_coarse_build_and_apply(L, dims, b, nv):
    m = 0.07
    lat = L.lattice(dims, bc=BC)
    U = gauge_field(dims, "haar", 2121)
    P = mg.orthonormalize(gaussian_spinor(dims, 2122, lead=(nv,)), b)
    Yo = mg.coarse_operator(U, m, BC, P, b)
    g64 = L.fields.gauge_to_device(U, lat, 0, 18)
    Y = torch.empty(L.lqcd_mg_coarse_op_bytes(lat, nv, b, 0) // 16, dtype=torch.complex128, device="cuda")
    L.lqcd_mg_coarse_build(Y, g64, _vecs_to_device(L, P, lat, 0), nv, b, lat, L.operator(mass=m))
    assert _rel(Y.cpu().numpy(), Yo.reshape(-1)) <= 1e-12
    cd = mg.coarse_dims(dims, b)
    c = make_rng(2123).standard_normal((int(np.prod(cd)) * 2 * nv, 2)) @ np.array([1.0, 1j])
    cs = c.reshape(tuple(reversed(cd)) + (2 * nv,))
    for prec, ctype, ntype in ((0, torch.complex128, np.complex128), (1, torch.complex64, np.complex64)):
        Yd = torch.from_numpy(Yo.reshape(-1).astype(ntype)).cuda()
        cin = torch.from_numpy(c.astype(ntype)).cuda()
        out = torch.empty_like(cin)
        for dagger in (0, 1):
            L.lqcd_mg_coarse_apply(out, cin, Yd, nv, b, prec, dagger, lat)
            Yr = Yo.astype(ntype).astype(np.complex128)
            cr = cs.astype(ntype).astype(np.complex128)
            assert _rel(out.cpu().numpy(), mg.coarse_apply(Yr, cr, bool(dagger)).reshape(-1)) <= TOL[prec] * 5


@pytest.mark.parametrize("kind,m,b,nv", [("exp", 0.01, 4, 8), ("haar", 0.1, 2, 6)])
def test_mg_solve_reaches_tolerance(L, kind, m, b, nv):
    dims = (8, 8, 8, 16)
    lat = L.lattice(dims, bc=BC)
    U = gauge_field(dims, kind, 2131, eps=0.3)
    src = gaussian_spinor(dims, 2132)
    F = L.fields
    op = L.operator(mass=m)
    mgp = L.mg_params(block=b, nvec=nv, setup_iters=30, post_smooth=4, coarse_iters=30, restart=12)
    g64 = F.gauge_to_device(U, lat, 0, 18)
    g32 = F.gauge_to_device(U, lat, 1, 12)
    rnd = _vecs_to_device(L, gaussian_spinor(dims, 2133, lead=(nv,)), lat, 0)
    ws = F.empty(L.lqcd_mg_workspace_bytes(lat, op, mgp))
    L.lqcd_mg_setup(g64, g32, rnd, lat, op, mgp, ws)
    x = F.empty(L.lqcd_spinor_bytes(lat, 0, 2))
    info = L.lqcd_mg_solve(x, F.spinor_to_device(src, lat, 0, 2), g64, g32, lat, op, mgp,
                           L.solver_params(tol=1e-10, maxiter=300), ws)
    xh = F.spinor_to_host(x, lat, 0, 2)[0]
    res = np.linalg.norm(src - wilson.dirac(U, xh, m, BC)) / np.linalg.norm(src)
    assert info.status == 0 and res <= 1e-10, (info.iterations, res)
    assert info.iterations < 120
