"""Seeded generators for the synthetic lattices the method is exercised on.

Host layouts (complex128, C order) shared by every consumer:

* gauge field  ``U[t, z, y, x, mu, row, col]``, ``mu`` = 0..3 for x, y, z, t;
* spinor field ``psi[..., t, z, y, x, spin, colour]`` with optional leading
  axes ``[rhs, s]`` for multi-right-hand-side and five-dimensional fields.

Random numbers come from numpy's PCG64 generator. The stream order is the C
order of the array being filled, real part before imaginary part, so a given
seed always produces the same field. Nothing here knows about Dirac operators.
"""
from __future__ import annotations

import concurrent.futures as cf
import os

import numpy as np

#: Base seed; the workload with index ``k`` uses ``BASE_SEED + k``.
BASE_SEED = 1512034870


def config_seed(index: int, stream: int = 0) -> int:
    """Seed for workload ``index`` and sub-stream ``stream`` (links, source, ...)."""
    return BASE_SEED + index + 1000 * stream


def make_rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def lattice_volume(dims) -> int:
    x, y, z, t = dims
    return x * y * z * t


def _complex_gaussian(rng: np.random.Generator, shape) -> np.ndarray:
    """Complex Gaussian with unit-variance real and imaginary parts."""
    re_im = rng.standard_normal(tuple(shape) + (2,))
    return re_im[..., 0] + 1j * re_im[..., 1]


def _chunked(fn, *arrays, chunk: int = 65536):
    """Apply ``fn`` to matching row-chunks of ``arrays`` on a thread pool and
    concatenate. numpy's batched linear algebra releases the GIL, so chunks run
    in parallel; the result is identical to ``fn(*arrays)``."""
    n = arrays[0].shape[0]
    if n <= chunk:
        return fn(*arrays)
    starts = range(0, n, chunk)
    workers = max(1, min(len(starts), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:
        parts = list(ex.map(lambda s0: fn(*(a[s0:s0 + chunk] for a in arrays)), starts))
    return np.concatenate(parts, axis=0)


def _su3_from_gaussian(z: np.ndarray) -> np.ndarray:
    q = np.empty_like(z)
    for j in range(3):
        v = z[:, :, j].copy()
        for k in range(j):
            proj = np.einsum("ni,ni->n", q[:, :, k].conj(), v)
            v -= proj[:, None] * q[:, :, k]
        v /= np.linalg.norm(v, axis=1)[:, None]
        q[:, :, j] = v
    det = np.linalg.det(q)
    q /= np.power(det, 1.0 / 3.0)[:, None, None]
    return q


def haar_su3(rng: np.random.Generator, n: int) -> np.ndarray:
    """``n`` Haar-distributed SU(3) matrices, shape (n, 3, 3).

    A complex Gaussian 3x3 matrix is orthonormalised column by column
    (Gram-Schmidt, i.e. the Q of a QR decomposition whose R has a positive
    real diagonal), which is Haar on U(3); dividing by the principal cube root
    of the determinant maps it to SU(3) and keeps left invariance, hence the
    Haar measure on SU(3).
    """
    z = _complex_gaussian(rng, (n, 3, 3))
    return _chunked(_su3_from_gaussian, z)


def _hermitian_from_gaussian(a: np.ndarray) -> np.ndarray:
    h = 0.5 * (a + np.conj(np.swapaxes(a, 1, 2)))
    tr = np.trace(h, axis1=1, axis2=2).real / 3.0
    h -= tr[:, None, None] * np.eye(3)[None]
    return h


def random_su3_algebra(rng: np.random.Generator, n: int) -> np.ndarray:
    """``n`` random traceless Hermitian 3x3 matrices H = (A + A^dag)/2 - tr/3."""
    return _hermitian_from_gaussian(_complex_gaussian(rng, (n, 3, 3)))


def exp_i_hermitian_su3(rng: np.random.Generator, n: int, eps: float) -> np.ndarray:
    """``n`` matrices exp(i * eps * H), H from :func:`random_su3_algebra`.

    The exponential is taken exactly through the Hermitian eigendecomposition
    H = V diag(w) V^dag, so the result is unitary with det = exp(i eps tr H) = 1
    up to rounding.
    """
    h = random_su3_algebra(rng, n)

    def expo(hc):
        w, v = np.linalg.eigh(hc)
        return np.einsum("nij,nj,nkj->nik", v, np.exp(1j * eps * w), v.conj())

    return _chunked(expo, h)


def gauge_field(dims, kind: str, seed: int, eps: float = 0.3) -> np.ndarray:
    """Gauge field of shape (T, Z, Y, X, 4, 3, 3).

    ``kind`` is ``"haar"`` (independent Haar SU(3) links), ``"exp"``
    (exp(i eps H) links, a smooth field near unit links) or ``"unit"``.
    """
    x, y, z, t = dims
    n = x * y * z * t * 4
    if kind == "unit":
        return unit_gauge(dims)
    rng = make_rng(seed)
    if kind == "haar":
        links = haar_su3(rng, n)
    elif kind == "exp":
        links = exp_i_hermitian_su3(rng, n, eps)
    else:
        raise ValueError(f"unknown gauge kind {kind!r}")
    return links.reshape(t, z, y, x, 4, 3, 3)


def unit_gauge(dims) -> np.ndarray:
    x, y, z, t = dims
    u = np.zeros((t, z, y, x, 4, 3, 3), dtype=np.complex128)
    u[..., :, :] = np.eye(3)
    return u


def gaussian_spinor(dims, seed: int, lead=()) -> np.ndarray:
    """Gaussian spinor field of shape ``lead + (T, Z, Y, X, 4, 3)``."""
    x, y, z, t = dims
    rng = make_rng(seed)
    return _complex_gaussian(rng, tuple(lead) + (t, z, y, x, 4, 3))


def random_gauge_transform(dims, seed: int) -> np.ndarray:
    """Haar SU(3) matrix per site, shape (T, Z, Y, X, 3, 3)."""
    x, y, z, t = dims
    rng = make_rng(seed)
    return haar_su3(rng, x * y * z * t).reshape(t, z, y, x, 3, 3)
