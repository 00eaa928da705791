"""Pins for the oracle's multigrid pieces (CPU only): aggregation identities and
the Galerkin coarse operator against the dense product P^dag D P."""
import numpy as np
import pytest

from oracle import mg
from synthetic import gauge_field, gaussian_spinor, make_rng
from tests.brute import wilson_dense

BC = (1.0, 1.0, 1.0, -1.0)


def _coarse_random(cdims, nc, seed):
    rng = make_rng(seed)
    shape = tuple(reversed(cdims)) + (nc,)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("dims,b,nv", [((4, 4, 4, 4), 2, 3), ((4, 2, 2, 4), 2, 2), ((8, 4, 4, 4), 4, 4)])
def test_restriction_and_prolongation(dims, b, nv):
    V = gaussian_spinor(dims, 2001, lead=(nv,))
    P = mg.orthonormalize(V, b)
    cd = mg.coarse_dims(dims, b)
    c = _coarse_random(cd, 2 * nv, 2002)
    np.testing.assert_allclose(mg.restrict(P, mg.prolong(P, c, b), b), c, atol=1e-12)   # R P = 1
    for k in range(nv):  # the near-null vectors lie in the range of P: P R v = v
        np.testing.assert_allclose(mg.prolong(P, mg.restrict(P, V[k], b), b), V[k], atol=1e-12)
    # Gram-Schmidt order: P_0 on each aggregate and chirality is V_0 normalised there
    B0 = mg._blocked(V[0:1], b)[0]
    P0 = mg._blocked(P[0:1], b)[0]
    for spins in mg.CHIRAL_SPINS:
        sp = list(spins)
        nrm = np.sqrt(np.sum(np.abs(B0[..., sp, :]) ** 2, axis=(-6, -5, -4, -3, -2, -1)))
        np.testing.assert_allclose(P0[..., sp, :], B0[..., sp, :] / nrm[..., None, None, None, None, None, None],
                                   atol=1e-12)


def _dense_prolongator(P, dims, b):
    cd = mg.coarse_dims(dims, b)
    nc = 2 * P.shape[0]
    ncoarse = int(np.prod(cd)) * nc
    cols = []
    for j in range(ncoarse):
        e = np.zeros(ncoarse, dtype=complex)
        e[j] = 1.0
        cols.append(mg.prolong(P, e.reshape(tuple(reversed(cd)) + (nc,)), b).reshape(-1))
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("dims,b,nv", [((4, 2, 2, 4), 2, 2), ((4, 4, 2, 2), 2, 1), ((4, 4, 4, 4), 4, 2)])
def test_coarse_operator_is_galerkin_product(dims, b, nv):
    """The 9-point stencil of Y equals P^dag D P built from the dense Wilson matrix,
    including coarse extents 1 and 2 where the stencil wraps onto itself."""
    m = 0.1
    U = gauge_field(dims, "haar", 2011)
    P = mg.orthonormalize(gaussian_spinor(dims, 2012, lead=(nv,)), b)
    Y = mg.coarse_operator(U, m, BC, P, b)
    Pm = _dense_prolongator(P, dims, b)
    Dc = Pm.conj().T @ wilson_dense(U, dims, m, BC) @ Pm
    cd = mg.coarse_dims(dims, b)
    c = _coarse_random(cd, 2 * nv, 2013)
    np.testing.assert_allclose(mg.coarse_apply(Y, c).reshape(-1), Dc @ c.reshape(-1), atol=1e-11)
    np.testing.assert_allclose(mg.coarse_apply(Y, c, dagger=True).reshape(-1), Dc.conj().T @ c.reshape(-1),
                               atol=1e-11)


def test_coarse_gamma5_hermiticity():
    """Chirality-preserving aggregation keeps gamma_5-hermiticity: with s = diag(1 (+), -1 (-))
    on the coarse components, D_c^dag = s D_c s."""
    dims, b, nv, m = (4, 4, 4, 4), 2, 2, 0.05
    U = gauge_field(dims, "exp", 2021, eps=0.4)
    P = mg.orthonormalize(gaussian_spinor(dims, 2022, lead=(nv,)), b)
    Y = mg.coarse_operator(U, m, BC, P, b)
    s = np.concatenate([np.ones(nv), -np.ones(nv)])
    c = _coarse_random(mg.coarse_dims(dims, b), 2 * nv, 2023)
    np.testing.assert_allclose(mg.coarse_apply(Y, c, dagger=True), s * mg.coarse_apply(Y, s * c), atol=1e-12)
