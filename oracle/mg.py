"""Two-level adaptive multigrid pieces for the Wilson operator: aggregation,
block orthonormalisation of near-null vectors, restriction / prolongation and
the Galerkin coarse-grid operator with its 9-point stencil (the paper shows a
coarse-grid operator of an adaptive multigrid inverter as its stencil example,
Sec. 2, and lists multigrid-preconditioned CG / GCR, Sec. 4; the definitions
are the standard aggregation-based ones).

Aggregates: blocks of b^4 fine sites (b divides every extent), each split by
chirality (spins 0, 1 = chirality +, spins 2, 3 = chirality - in the chiral
basis, gamma_5 = diag(1, 1, -1, -1)). Given Nv fine vectors v_k, the
prolongator P has, per aggregate and chirality, the Nv columns obtained by
orthonormalising v_k restricted there (Gram-Schmidt order: QR with a positive
real diagonal of R), so a coarse site carries Nc = 2 Nv components, ordered
(chirality, k) with chirality + first.

  restriction   c(X)[(s, k)] = sum_{x in X, spin in s} P_k(x)^dag psi(x)
  prolongation  psi(x) = sum_k P_k(x)|_{s(x)} c(X(x))[(s, k)]
  coarse op     D_c = P^dag D P: a 9-point stencil on the coarse lattice,
                (D_c c)(X) = sum_{d in {0, +-mu}} Y_d(X) c(X + d), with
                Y_{+mu}(X) = -1/2 sum_{x in X, x + mu not in X} P(x)^dag (1 - gamma_mu) U_mu(x) P(x + mu)
                Y_{-mu}(X) = -1/2 sum_{x in X, x - mu not in X} P(x)^dag (1 + gamma_mu) U_mu(x - mu)^dag P(x - mu)
                Y_0(X)     = (4 + m) 1 - 1/2 sum of the same terms for hops inside X,
                boundary phases included in the hops that wrap.

Layouts: fine vectors V[Nv, t, z, y, x, spin, colour]; coarse fields
c[T, Z, Y, X, Nc]; Y[9, T, Z, Y, X, Nc, Nc] with d = 0 the self term and
d = 1 + 2 mu (+mu), 2 + 2 mu (-mu).

Pins (tests/test_oracle_mg.py): P^dag P = 1 within every aggregate, R P = 1,
the stencil against the dense product P^dag D P on small lattices (built from
the explicit-loop dense Wilson matrix), and the coarse operator's
gamma_5-hermiticity analogue.
"""
from __future__ import annotations

import numpy as np

from . import wilson
from .gamma import one_minus_gamma, one_plus_gamma, spin_apply

CHIRAL_SPINS = ((0, 1), (2, 3))


def coarse_dims(dims, b):
    for L in dims:
        if L % b:
            raise ValueError("block size must divide every extent")
    return tuple(L // b for L in dims)


def _blocked(f: np.ndarray, b: int) -> np.ndarray:
    """[..., T, Z, Y, X, s, c] -> [..., T/b, Z/b, Y/b, X/b, b, b, b, b, s, c]."""
    lead = f.shape[:-6]
    T, Z, Y, X = f.shape[-6:-2]
    g = f.reshape(lead + (T // b, b, Z // b, b, Y // b, b, X // b, b) + f.shape[-2:])
    n = len(lead)
    order = list(range(n)) + [n + 0, n + 2, n + 4, n + 6, n + 1, n + 3, n + 5, n + 7, n + 8, n + 9]
    return g.transpose(order)


def _unblocked(g: np.ndarray, b: int) -> np.ndarray:
    lead = g.shape[:-10]
    n = len(lead)
    order = list(range(n)) + [n + 0, n + 4, n + 1, n + 5, n + 2, n + 6, n + 3, n + 7, n + 8, n + 9]
    h = g.transpose(order)
    Tc, Zc, Yc, Xc = g.shape[n:n + 4]
    return h.reshape(lead + (Tc * b, Zc * b, Yc * b, Xc * b) + g.shape[-2:])


def orthonormalize(V: np.ndarray, b: int) -> np.ndarray:
    """P from Nv vectors V[Nv, t, z, y, x, 4, 3]: per aggregate and chirality the
    columns of Q in V_block = Q R (QR with a positive real diagonal of R)."""
    Nv = V.shape[0]
    G = _blocked(V, b)  # [Nv, Tc, Zc, Yc, Xc, b, b, b, b, 4, 3]
    out = np.zeros_like(G)
    for s, spins in enumerate(CHIRAL_SPINS):
        sub = G[..., list(spins), :]  # [Nv, Tc..Xc, b^4, 2, 3]
        A = np.moveaxis(sub.reshape(Nv, *sub.shape[1:5], -1), 0, -1)  # [Tc..Xc, n, Nv]
        Q, R = np.linalg.qr(A)
        d = np.diagonal(R, axis1=-2, axis2=-1)
        Q = Q * (d / np.abs(d))[..., None, :]  # Q R = (Q L)(L^-1 R), L = d/|d|: diag(L^-1 R) = |d| > 0
        Qv = np.moveaxis(Q, -1, 0).reshape(sub.shape)
        out[..., list(spins), :] = Qv
    return _unblocked(out, b)


def restrict(P: np.ndarray, psi: np.ndarray, b: int) -> np.ndarray:
    """Coarse field [Tc, Zc, Yc, Xc, 2 Nv] of a fine field psi[t, z, y, x, 4, 3]."""
    Nv = P.shape[0]
    Gp = _blocked(P, b)
    Gs = _blocked(psi, b)
    out = []
    for spins in CHIRAL_SPINS:
        sp = list(spins)
        out.append(np.einsum("k...abcdsx,...abcdsx->...k", np.conj(Gp[..., sp, :]), Gs[..., sp, :]))
    return np.concatenate(out, axis=-1)


def prolong(P: np.ndarray, c: np.ndarray, b: int) -> np.ndarray:
    """Fine field psi[t, z, y, x, 4, 3] from a coarse field c[Tc, Zc, Yc, Xc, 2 Nv]."""
    Nv = P.shape[0]
    Gp = _blocked(P, b)
    out = np.zeros(Gp.shape[1:], dtype=complex)
    for s, spins in enumerate(CHIRAL_SPINS):
        sp = list(spins)
        out[..., sp, :] = np.einsum("k...abcdsx,...k->...abcdsx", Gp[..., sp, :], c[..., s * Nv:(s + 1) * Nv])
    return _unblocked(out, b)


def _project_blocks(P: np.ndarray, w: np.ndarray, mask: np.ndarray, b: int) -> np.ndarray:
    """sum over fine sites of each aggregate with mask: P^dag w, for w[Nc', t, z, y, x, 4, 3]
    (a fine field per coarse basis vector): returns [Tc, Zc, Yc, Xc, Nc, Nc']."""
    Nv = P.shape[0]
    Gp = _blocked(P * mask[None, ..., None, None], b)
    Gw = _blocked(w, b)
    rows = []
    for spins in CHIRAL_SPINS:
        sp = list(spins)
        rows.append(np.einsum("k...abcdsx,j...abcdsx->...kj", np.conj(Gp[..., sp, :]), Gw[..., sp, :]))
    return np.concatenate(rows, axis=-2)


def _basis_fields(P: np.ndarray) -> np.ndarray:
    """The Nc fine fields P e_(s, k): P_k restricted to chirality s, [Nc, t, z, y, x, 4, 3]."""
    out = []
    for spins in CHIRAL_SPINS:
        for k in range(P.shape[0]):
            f = np.zeros_like(P[k])
            f[..., list(spins), :] = P[k][..., list(spins), :]
            out.append(f)
    return np.stack(out)


def coarse_operator(U: np.ndarray, mass: float, bc, P: np.ndarray, b: int) -> np.ndarray:
    """Y[9, Tc, Zc, Yc, Xc, Nc, Nc] of D_c = P^dag D_W P (see the module docstring)."""
    dims = (U.shape[3], U.shape[2], U.shape[1], U.shape[0])
    cdims = coarse_dims(dims, b)
    Nc = 2 * P.shape[0]
    B = _basis_fields(P)  # [Nc, t, z, y, x, 4, 3]
    Y = np.zeros((9,) + tuple(reversed(cdims)) + (Nc, Nc), dtype=complex)
    ones = np.ones(U.shape[:4])
    Y[0] = _project_blocks(P, (4.0 + mass) * B, ones, b)
    for mu in range(4):
        ax = wilson.site_axis(mu)
        coord = np.indices(U.shape[:4])[3 - mu]  # fine coordinate along mu, shaped [t, z, y, x]
        fwd_out = (coord % b) == b - 1           # x + mu lies in the next aggregate
        bwd_out = (coord % b) == 0               # x - mu lies in the previous aggregate
        u = U[..., mu, :, :]
        # forward hop term (1 - gamma_mu) U_mu(x) B(x + mu), boundary phase included
        Bf = wilson.shift(B, mu, +1, bc)
        hf = -0.5 * spin_apply(one_minus_gamma(mu), np.einsum("...ab,n...sb->n...sa", u, Bf))
        # backward hop term (1 + gamma_mu) U_mu(x - mu)^dag B(x - mu)
        ub = np.roll(u, 1, axis=ax)  # U_mu(x - mu); link arrays [t, z, y, x, 3, 3] share the site axes
        Bb = wilson.shift(B, mu, -1, bc)
        hb = -0.5 * spin_apply(one_plus_gamma(mu), np.einsum("...ba,n...sb->n...sa", np.conj(ub), Bb))
        Y[1 + 2 * mu] += _project_blocks(P, hf, fwd_out.astype(float), b)
        Y[0] += _project_blocks(P, hf, (~fwd_out).astype(float), b)
        Y[2 + 2 * mu] += _project_blocks(P, hb, bwd_out.astype(float), b)
        Y[0] += _project_blocks(P, hb, (~bwd_out).astype(float), b)
    return Y


def coarse_apply(Y: np.ndarray, c: np.ndarray, dagger: bool = False) -> np.ndarray:
    """(D_c c)(X) = sum_d Y_d(X) c(X + d); with dagger the adjoint stencil
    (D_c^dag c)(X) = sum_d Y_{-d}(X + d)^dag c(X + d)."""
    out = np.einsum("...ij,...j->...i", Y[0] if not dagger else np.conj(np.swapaxes(Y[0], -1, -2)), c)
    for mu in range(4):
        ax = -2 - mu  # coarse arrays are [Tc, Zc, Yc, Xc, Nc]
        cp = np.roll(c, -1, axis=ax)  # c(X + mu)
        cm = np.roll(c, 1, axis=ax)   # c(X - mu)
        if not dagger:
            out += np.einsum("...ij,...j->...i", Y[1 + 2 * mu], cp)
            out += np.einsum("...ij,...j->...i", Y[2 + 2 * mu], cm)
        else:
            # the coupling X <- X + mu of D_c^dag is Y_{-mu}(X + mu)^dag
            ym = np.roll(Y[2 + 2 * mu], -1, axis=ax - 1)
            yp = np.roll(Y[1 + 2 * mu], 1, axis=ax - 1)
            out += np.einsum("...ji,...j->...i", np.conj(ym), cp)
            out += np.einsum("...ji,...j->...i", np.conj(yp), cm)
    return out
