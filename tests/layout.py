"""Test-side conversions between full-lattice arrays and one-parity arrays.

Written independently of the library's own helper: a site of parity p is
listed at position lex // 2 of its parity's array, lex = x + X (y + Y (z + Z t)).
"""
import itertools

import numpy as np


def to_cb(full: np.ndarray, parity: int) -> np.ndarray:
    T, Z, Y, X = full.shape[-6:-2]
    lead = full.shape[:-6]
    out = np.zeros(lead + (T, Z, Y, X // 2, 4, 3), dtype=np.complex128)
    for t, z, y, x in itertools.product(range(T), range(Z), range(Y), range(X)):
        if (x + y + z + t) % 2 == parity:
            out[..., t, z, y, x // 2, :, :] = full[..., t, z, y, x, :, :]
    return out


def from_cb(cb: np.ndarray, parity: int) -> np.ndarray:
    T, Z, Y, Xh = cb.shape[-6:-2]
    lead = cb.shape[:-6]
    out = np.zeros(lead + (T, Z, Y, 2 * Xh, 4, 3), dtype=np.complex128)
    for t, z, y, x in itertools.product(range(T), range(Z), range(Y), range(2 * Xh)):
        if (x + y + z + t) % 2 == parity:
            out[..., t, z, y, x, :, :] = cb[..., t, z, y, x // 2, :, :]
    return out


def rel_l2(a, b) -> float:
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))
