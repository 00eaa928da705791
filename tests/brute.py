"""Explicit-loop dense matrices of the Wilson and domain-wall operators.

Independent of the oracle's array code: every matrix element is placed by
integer coordinate arithmetic and np.kron of a 4x4 spin block with a 3x3
colour block, so a mistake in the oracle's shifts, spin matrices or link
indexing shows up as a mismatch. Only usable on tiny lattices.
"""
import itertools

import numpy as np

from oracle.gamma import GAMMA, P_MINUS, P_PLUS

ID4 = np.eye(4)


def lex(coord, dims):
    x, y, z, t = coord
    X, Y, Z, T = dims
    return x + X * (y + Y * (z + Z * t))


def sites(dims):
    X, Y, Z, T = dims
    for t, z, y, x in itertools.product(range(T), range(Z), range(Y), range(X)):
        yield (x, y, z, t)


def wilson_dense(U, dims, mass, bc):
    """D_W as a (12V x 12V) matrix, dof index = lex*12 + spin*3 + colour."""
    V = int(np.prod(dims))
    D = np.zeros((12 * V, 12 * V), dtype=np.complex128)
    for coord in sites(dims):
        i = lex(coord, dims)
        D[12 * i:12 * i + 12, 12 * i:12 * i + 12] += (4.0 + mass) * np.eye(12)
        x, y, z, t = coord
        for mu in range(4):
            L = dims[mu]
            fwd = list(coord)
            fwd[mu] = (coord[mu] + 1) % L
            ph_f = bc[mu] if coord[mu] == L - 1 else 1.0
            bwd = list(coord)
            bwd[mu] = (coord[mu] - 1) % L
            ph_b = bc[mu] if coord[mu] == 0 else 1.0
            j = lex(fwd, dims)
            k = lex(bwd, dims)
            u_here = U[t, z, y, x, mu]
            bx, by, bz, bt = bwd
            u_back = U[bt, bz, by, bx, mu]
            D[12 * i:12 * i + 12, 12 * j:12 * j + 12] += -0.5 * ph_f * np.kron(ID4 - GAMMA[mu], u_here)
            D[12 * i:12 * i + 12, 12 * k:12 * k + 12] += -0.5 * ph_b * np.kron(ID4 + GAMMA[mu], u_back.conj().T)
    return D


def dwf_dense(U, dims, Ls, M5, mf, bc):
    """Shamir D_DW as a (12 V Ls)^2 matrix, dof index = (s*V + lex)*12 + spin*3 + colour."""
    V = int(np.prod(dims))
    n4 = 12 * V
    W = wilson_dense(U, dims, -M5, bc)
    D = np.zeros((n4 * Ls, n4 * Ls), dtype=np.complex128)
    pm = np.kron(np.eye(V), np.kron(P_MINUS, np.eye(3)))
    pp = np.kron(np.eye(V), np.kron(P_PLUS, np.eye(3)))
    for s in range(Ls):
        blk = slice(s * n4, (s + 1) * n4)
        D[blk, blk] += W + np.eye(n4)
        up = s + 1
        if up < Ls:
            D[blk, up * n4:(up + 1) * n4] += -pm
        else:
            D[blk, 0:n4] += mf * pm
        dn = s - 1
        if dn >= 0:
            D[blk, dn * n4:(dn + 1) * n4] += -pp
        else:
            D[blk, (Ls - 1) * n4:Ls * n4] += mf * pp
    return D
