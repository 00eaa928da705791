"""Pseudofermion action S = phi^dag (M^dag M)^-1 phi behind torch.autograd.

``FermionAction.apply(U, phi, mass, bc)`` returns the real scalar S for a
Wilson operator M = D_W; its backward gives the gauge-link gradient in the
convention torch uses for complex leaves (dS = Re sum conj(dU) U.grad) from the
library's force kernel. The solve X = (M^dag M)^-1 phi is an FP64 CG on the
GPU; backward needs X and Y = M X, which are either kept from the forward
pass or, with ``checkpoint=True``, recomputed by a second solve so that no
solution vector is held between forward and backward. For this scalar the
adjoint solve (M^dag M)^-1 (dS/dX) reuses X itself, because M^dag M is
Hermitian and dS/dX is phi.

All tensors are complex128 CUDA tensors in the host layouts of include/lqcd.h:
U[t, z, y, x, mu, row, col], phi[t, z, y, x, spin, colour].
"""
from __future__ import annotations

import torch

from . import api
from . import fields as F


def _lattice(U, bc):
    T, Z, Y, X = U.shape[:4]
    return api.lattice((X, Y, Z, T), n5=1, bc=bc)


def _solve(U_dev, phi_dev, lat, op, tol, maxiter):
    prm = api.solver_params(tol=tol, maxiter=maxiter, sloppy_prec=api.LQCD_F64, use_graph=1)
    X = F.empty(api.lqcd_spinor_bytes(lat, api.LQCD_F64, api.LQCD_FULL))
    ws = F.empty(api.lqcd_cg_workspace_bytes(lat, op, prm, api.LQCD_FULL))
    info = api.lqcd_cg_solve(X, phi_dev, U_dev, U_dev, lat, op, prm, api.LQCD_FULL, ws)
    Y = F.empty(api.lqcd_spinor_bytes(lat, api.LQCD_F64, api.LQCD_FULL))
    api.lqcd_M(Y, X, U_dev, lat, op, api.LQCD_FULL, 0, None)
    return X, Y, info


def _pack(U, phi, lat):
    U_dev = F.empty(api.lqcd_gauge_bytes(lat, api.LQCD_F64, 18))
    api.lqcd_gauge_pack(U_dev, api.LQCD_F64, 18, torch.view_as_real(U.detach().contiguous()), lat)
    phi_dev = F.empty(api.lqcd_spinor_bytes(lat, api.LQCD_F64, api.LQCD_FULL))
    api.lqcd_spinor_pack(phi_dev, api.LQCD_F64, api.LQCD_FULL, torch.view_as_real(phi.detach().contiguous()), lat)
    return U_dev, phi_dev


def _action(X, phi_dev, lat):
    """S = Re <phi, X>, reduced in FP64 by the library (lqcd_spinor_dot_re)."""
    ws = F.empty(api.lqcd_reduce_workspace_bytes(lat))
    S = api.lqcd_spinor_dot_re(phi_dev, X, lat, ws)
    return torch.tensor(S, dtype=torch.float64, device=X.device)


class FermionAction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, phi, mass: float, bc=(1.0, 1.0, 1.0, -1.0), tol: float = 1e-12,
                maxiter: int = 20000, checkpoint: bool = False):
        if not (U.is_cuda and phi.is_cuda and U.dtype == torch.complex128 and phi.dtype == torch.complex128):
            raise TypeError("FermionAction expects complex128 CUDA tensors")
        lat = _lattice(U, bc)
        op = api.operator(kind=api.LQCD_WILSON, mass=mass, prec=api.LQCD_F64, recon=18)
        U_dev, phi_dev = _pack(U, phi, lat)
        X, Y, info = _solve(U_dev, phi_dev, lat, op, tol, maxiter)
        S = _action(X, phi_dev, lat)
        ctx.lat, ctx.op, ctx.tol, ctx.maxiter, ctx.checkpoint = lat, op, tol, maxiter, checkpoint
        ctx.solve_info = (info.iterations, info.true_rel_residual)
        if checkpoint:
            ctx.save_for_backward(U, phi)
            ctx.XY = None
        else:
            ctx.save_for_backward(U, phi)
            ctx.XY = (U_dev, X, Y)
        return S

    @staticmethod
    def backward(ctx, grad_out):
        U, phi = ctx.saved_tensors
        lat, op = ctx.lat, ctx.op
        if ctx.XY is None:
            U_dev, phi_dev = _pack(U, phi, lat)
            X, Y, _ = _solve(U_dev, phi_dev, lat, op, ctx.tol, ctx.maxiter)
        else:
            U_dev, X, Y = ctx.XY
            ctx.XY = None
        out = F.empty(api.lqcd_gauge_bytes(lat, api.LQCD_F64, 18))
        api.lqcd_force(out, U_dev, X, Y, lat, op, api.LQCD_FORCE_GRAD)
        g = torch.empty(U.numel() * 2, dtype=torch.float64, device=U.device)
        api.lqcd_gauge_unpack(g, out, api.LQCD_F64, 18, lat)
        grad_U = torch.view_as_complex(g.view(*U.shape, 2)) * grad_out
        return grad_U, None, None, None, None, None, None


def fermion_action(U, phi, mass, bc=(1.0, 1.0, 1.0, -1.0), tol=1e-12, maxiter=20000, checkpoint=False):
    return FermionAction.apply(U, phi, mass, tuple(bc), tol, maxiter, checkpoint)


def force_traceless_hermitian(U, phi, mass, bc=(1.0, 1.0, 1.0, -1.0), tol=1e-12, maxiter=20000):
    """(S, F) with F[t, z, y, x, mu] the traceless Hermitian force, dS = eps tr(T F)
    under U -> exp(i eps T) U (the HMC force)."""
    lat = _lattice(U, bc)
    op = api.operator(kind=api.LQCD_WILSON, mass=mass, prec=api.LQCD_F64, recon=18)
    U_dev, phi_dev = _pack(U, phi, lat)
    X, Y, _ = _solve(U_dev, phi_dev, lat, op, tol, maxiter)
    out = F.empty(api.lqcd_gauge_bytes(lat, api.LQCD_F64, 18))
    api.lqcd_force(out, U_dev, X, Y, lat, op, api.LQCD_FORCE_TA)
    g = torch.empty(U.numel() * 2, dtype=torch.float64, device=U.device)
    api.lqcd_gauge_unpack(g, out, api.LQCD_F64, 18, lat)
    return _action(X, phi_dev, lat), torch.view_as_complex(g.view(*U.shape, 2))
