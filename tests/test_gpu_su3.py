"""SU(3) x SU(3) field product on the GPU against the oracle: FP64 and FP32,
general complex and SU(3) fields, ragged site counts, n5 > 1, aliasing, and a
sampled check at a size far beyond L2."""
import numpy as np
import pytest

from oracle import su3
from synthetic import gauge_field, make_rng

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL = {0: 1e-14, 1: 2e-6}


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1512_03487_gb300 as L
    from paper_1512_03487_gb300 import fields
    L.fields = fields
    return L


def _random(shape, seed, kind):
    if kind == "su3":
        n = int(np.prod(shape))
        dims = (2, 2, 2, 2 * ((n + 63) // 64))
        U = gauge_field(dims, "haar", seed).reshape(-1, 3, 3)[:n]
        return U.reshape(shape + (3, 3))
    rng = make_rng(seed)
    return rng.standard_normal(shape + (3, 3)) + 1j * rng.standard_normal(shape + (3, 3))


def _max_rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dims,n5", [((4, 4, 4, 4), 1), ((2, 2, 2, 6), 3), ((6, 2, 4, 2), 1), ((8, 8, 8, 16), 2)])
@pytest.mark.parametrize("kind", ["gauss", "su3"])
def test_su3_mul_matches_oracle(L, prec, dims, n5, kind):
    F = L.fields
    lat = L.lattice(dims, n5=n5)
    shape = F.host_colour_matrix_shape(lat)[:-2]
    x = _random(shape, 1401, kind)
    y = _random(shape, 1402, kind)
    xd = F.colour_matrix_to_device(x, lat, prec)
    yd = F.colour_matrix_to_device(y, lat, prec)
    zd = F.empty(L.lqcd_colour_matrix_bytes(lat, prec))
    L.lqcd_su3_mul(zd, xd, yd, lat, prec)
    z = F.colour_matrix_to_host(zd, lat, prec)
    if prec == 1:  # compare with the product of the FP32-rounded inputs
        x = x.astype(np.complex64).astype(np.complex128)
        y = y.astype(np.complex64).astype(np.complex128)
    assert _max_rel(z, su3.su3_mul(x, y)) <= TOL[prec]


@pytest.mark.parametrize("prec", [0, 1])
def test_su3_mul_in_place(L, prec):
    F = L.fields
    lat = L.lattice((4, 4, 2, 6), n5=1)
    shape = F.host_colour_matrix_shape(lat)[:-2]
    x = _random(shape, 1411, "gauss")
    y = _random(shape, 1412, "gauss")
    xd = F.colour_matrix_to_device(x, lat, prec)
    yd = F.colour_matrix_to_device(y, lat, prec)
    L.lqcd_su3_mul(xd, xd, yd, lat, prec)  # x <- x y
    L.lqcd_su3_mul(yd, xd, yd, lat, prec)  # y <- (x y) y
    if prec == 1:
        x = x.astype(np.complex64).astype(np.complex128)
        y = y.astype(np.complex64).astype(np.complex128)
    xy = su3.su3_mul(x, y)
    assert _max_rel(F.colour_matrix_to_host(xd, lat, prec), xy) <= TOL[prec]
    assert _max_rel(F.colour_matrix_to_host(yd, lat, prec), su3.su3_mul(xy, y)) <= 3 * TOL[prec]


def test_su3_mul_fullsize_sampled(L):
    """40^4 FP32 (2.56 M sites, 184 MB per field, beyond L2): 4096 sampled sites against the oracle."""
    F = L.fields
    dims = (40, 40, 40, 40)
    lat = L.lattice(dims)
    n = int(np.prod(dims))
    rng = make_rng(1421)
    x = rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))
    y = rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))
    xd = F.colour_matrix_to_device(x, lat, 1)
    yd = F.colour_matrix_to_device(y, lat, 1)
    zd = F.empty(L.lqcd_colour_matrix_bytes(lat, 1))
    L.lqcd_su3_mul(zd, xd, yd, lat, 1)
    z = F.colour_matrix_to_host(zd, lat, 1).reshape(n, 3, 3)
    idx = rng.choice(n, 4096, replace=False)
    xs = x[idx].astype(np.complex64).astype(np.complex128)
    ys = y[idx].astype(np.complex64).astype(np.complex128)
    assert _max_rel(z[idx], su3.su3_mul(xs, ys)) <= TOL[1]
    del xd, yd, zd
    torch.cuda.empty_cache()
