"""Euclidean Dirac matrices in a chiral (DeGrand-Rossi type) basis.

The paper uses spin-projected Wilson kernels (Sec. 2.6, the Compressor that
spin-projects communicated fields) but never fixes a basis. Reading taken here:

    gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]   (k = 1, 2, 3 -> x, y, z)
    gamma_4 = [[0, 1], [1, 0]]                    (t)
    gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1, 1, -1, -1)

so the chiral projectors P_+ = (1 + gamma_5)/2 and P_- = (1 - gamma_5)/2 keep
spin components (0, 1) and (2, 3). Pinned by tests: Hermiticity,
{gamma_mu, gamma_nu} = 2 delta_mu_nu, and gamma_5 equal to the product.
"""
import numpy as np

_S1 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_S2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_S3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)


def _block(a, b, c, d):
    return np.block([[a, b], [c, d]])


#: GAMMA[mu] for mu = 0..3 (x, y, z, t).
GAMMA = np.array(
    [_block(_Z2, -1j * s, 1j * s, _Z2) for s in (_S1, _S2, _S3)]
    + [_block(_Z2, _I2, _I2, _Z2)]
)
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
ID4 = np.eye(4, dtype=np.complex128)
P_PLUS = 0.5 * (ID4 + GAMMA5)
P_MINUS = 0.5 * (ID4 - GAMMA5)


def one_minus_gamma(mu: int) -> np.ndarray:
    return ID4 - GAMMA[mu]


def one_plus_gamma(mu: int) -> np.ndarray:
    return ID4 + GAMMA[mu]


def spin_apply(m: np.ndarray, f: np.ndarray) -> np.ndarray:
    """Apply a 4x4 spin matrix to a field ``f[..., spin, colour]``."""
    return np.einsum("st,...tc->...sc", m, f)
