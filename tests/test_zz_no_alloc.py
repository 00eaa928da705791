"""lqcd_M_noalloc: the Dirac operator for callers that cannot allocate device
memory (host callbacks, latency-critical paths, plugins whose framework owns
the memory pool). It must give what lqcd_M gives with a caller-provided
workspace, call after call, although every call reuses one fixed scratch
array inside the library.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test; it also passes on its own in a
fresh process."""
import numpy as np
import pytest

from synthetic import gauge_field, gaussian_spinor
from tests.layout import rel_l2, to_cb

BC = (1.0, 1.0, 1.0, -1.0)
TOL = {0: 1e-12, 1: 1e-5, 2: 3e-3}


@pytest.fixture(scope="module")
def L():
    import paper_1512_03487_gb300 as L
    return L


@pytest.mark.gpu
def test_noalloc_operator_matches_workspace_operator_twice(L):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1512_03487_gb300 import fields as F
    cases = [
        ((8, 8, 8, 12), 1, L.operator(kind=L.LQCD_WILSON, mass=0.05, prec=L.LQCD_F32, recon=12), 0),
        ((4, 4, 4, 8), 6, L.operator(kind=L.LQCD_DWF, M5=1.8, mf=0.02, prec=L.LQCD_F16, recon=18), 1),
        ((4, 4, 4, 4), 1, L.operator(kind=L.LQCD_WILSON, mass=0.1, prec=L.LQCD_F64, recon=18), 1),
    ]
    for dims, n5, op, dagger in cases:
        lat = L.lattice(dims, n5=n5, bc=BC)
        U = gauge_field(dims, "haar", 401)
        g = F.gauge_to_device(U, lat, op.prec, op.recon)
        ws = F.empty(L.lqcd_operator_workspace_bytes(lat, op, L.LQCD_EVEN))
        for call in range(2):  # two calls in a row: the shared scratch keeps the last call's contents
            psi = to_cb(gaussian_spinor(dims, 402 + call, lead=(n5,)), 0)
            fin = F.spinor_to_device(psi, lat, op.prec, L.LQCD_EVEN)
            ref = F.empty(L.lqcd_spinor_bytes(lat, op.prec, L.LQCD_EVEN))
            got = F.empty(L.lqcd_spinor_bytes(lat, op.prec, L.LQCD_EVEN))
            L.lqcd_M(ref, fin, g, lat, op, L.LQCD_EVEN, dagger, ws)
            L.lqcd_M_noalloc(got, fin, g, lat, op, L.LQCD_EVEN, dagger)
            a = F.spinor_to_host(got, lat, op.prec, L.LQCD_EVEN)
            b = F.spinor_to_host(ref, lat, op.prec, L.LQCD_EVEN)
            assert np.any(b != 0)
            assert rel_l2(a, b) <= TOL[op.prec]


def test_noalloc_rejects_lattices_beyond_the_fixed_scratch(L):
    """An FP64 Schur operator on 32^4 needs a 96 MiB odd-checkerboard
    temporary, beyond the 32 MiB array: refused on the host with a clear error
    before any CUDA call (the pointers below are never dereferenced)."""
    lat = L.lattice((32, 32, 32, 32))
    op = L.operator(mass=0.1, prec=L.LQCD_F64)
    with pytest.raises(L.LqcdError) as ei:
        L.lqcd_M_noalloc(4096, 8192, 12288, lat, op, L.LQCD_EVEN, 0, stream=0)
    assert ei.value.status == -1
    assert "fixed" in L.lqcd_last_error() and "scratch" in L.lqcd_last_error()
