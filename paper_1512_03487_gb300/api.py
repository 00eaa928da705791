"""Thin Python binding of the C ABI in ``include/lqcd.h``.

Every ``lqcd_*`` function here has the name and argument order of the C entry
point; it only marshals arguments (torch tensors -> device pointers, the
current torch stream -> cudaStream_t) and turns a non-zero status into
:class:`LqcdError`. All computation happens in the CUDA library. PyTorch is
used for device memory and streams only.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np

from . import _lib
from ._lib import (  # noqa: F401  (re-exported constants and structs)
    LQCD_DWF, LQCD_EVEN, LQCD_F16, LQCD_F32, LQCD_F64, LQCD_F64_DF, LQCD_FORCE_GRAD, LQCD_FORCE_TA, LQCD_FULL,
    LQCD_LEAPFROG, LQCD_MINNORM2, LQCD_ODD, LQCD_WILSON, lqcd_hmc_info, lqcd_hmc_params, lqcd_lattice,
    lqcd_mg_params, lqcd_operator, lqcd_solve_info, lqcd_solver_params,
)

lib = _lib.load()


class LqcdError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"lqcd status {status}: {message}")
        self.status = status


def _check(status: int) -> None:
    if status != 0:
        raise LqcdError(status, lib.lqcd_last_error().decode())


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()  # torch tensor


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream or None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


# ------------------------------------------------------------------ structs

def lattice(dims: Sequence[int], n5: int = 1, bc: Sequence[float] = (1.0, 1.0, 1.0, -1.0)) -> lqcd_lattice:
    lat = lqcd_lattice()
    for k in range(4):
        lat.dims[k] = int(dims[k])
        lat.bc[k] = float(bc[k])
    lat.n5 = int(n5)
    return lat


def operator(kind: int = LQCD_WILSON, mass: float = 0.0, M5: float = 1.8, mf: float = 0.02,
             prec: int = LQCD_F64, recon: int = 18, gparity: int = 0) -> lqcd_operator:
    return lqcd_operator(kind=kind, mass=mass, M5=M5, mf=mf, prec=prec, recon=recon, gparity=gparity)


def solver_params(tol: float = 1e-10, maxiter: int = 10000, sloppy_prec: int = LQCD_F64,
                  sloppy_recon: int = 18, delta: float = 0.1, check_interval: int = 16,
                  use_graph: int = 1, timeout_ms: float = 0.0, delta_mid: float = 0.0,
                  update_prec: int = LQCD_F64) -> lqcd_solver_params:
    return lqcd_solver_params(tol=tol, maxiter=maxiter, sloppy_prec=sloppy_prec, sloppy_recon=sloppy_recon,
                              delta=delta, check_interval=check_interval, use_graph=use_graph,
                              timeout_ms=timeout_ms, delta_mid=delta_mid, update_prec=update_prec)


# ------------------------------------------------------------------ library

def lqcd_version() -> str:
    return lib.lqcd_version().decode()


def lqcd_last_error() -> str:
    return lib.lqcd_last_error().decode()


def lqcd_launch_count() -> int:
    return int(lib.lqcd_launch_count())


def lqcd_release_caches() -> None:
    lib.lqcd_release_caches()


def lqcd_spinor_bytes(lat, prec, subset) -> int:
    return int(lib.lqcd_spinor_bytes(C.byref(lat), prec, subset))


def lqcd_gauge_bytes(lat, prec, recon) -> int:
    return int(lib.lqcd_gauge_bytes(C.byref(lat), prec, recon))


def lqcd_operator_workspace_bytes(lat, op, subset) -> int:
    return int(lib.lqcd_operator_workspace_bytes(C.byref(lat), C.byref(op), subset))


def lqcd_cg_workspace_bytes(lat, op, params, subset) -> int:
    return int(lib.lqcd_cg_workspace_bytes(C.byref(lat), C.byref(op), C.byref(params), subset))


# ------------------------------------------------------------------ layout

def lqcd_spinor_pack(dst, prec, subset, src, lat, stream=None):
    _check(lib.lqcd_spinor_pack(_ptr(dst), prec, subset, _ptr(src), C.byref(lat), _stream(stream)))


def lqcd_spinor_unpack(dst, src, prec, subset, lat, stream=None):
    _check(lib.lqcd_spinor_unpack(_ptr(dst), _ptr(src), prec, subset, C.byref(lat), _stream(stream)))


def lqcd_gauge_pack(dst, prec, recon, src, lat, stream=None):
    _check(lib.lqcd_gauge_pack(_ptr(dst), prec, recon, _ptr(src), C.byref(lat), _stream(stream)))


def lqcd_gauge_unpack(dst, src, prec, recon, lat, stream=None):
    _check(lib.lqcd_gauge_unpack(_ptr(dst), _ptr(src), prec, recon, C.byref(lat), _stream(stream)))


def lqcd_spinor_upload(dst, prec, subset, src_host, staging, lat, stream=None):
    _check(lib.lqcd_spinor_upload(_ptr(dst), prec, subset, _ptr(src_host), _ptr(staging), C.byref(lat),
                                  _stream(stream)))


def lqcd_spinor_download(dst_host, src, prec, subset, staging, lat, stream=None):
    _check(lib.lqcd_spinor_download(_ptr(dst_host), _ptr(src), prec, subset, _ptr(staging), C.byref(lat),
                                    _stream(stream)))


def lqcd_gauge_upload(dst, prec, recon, src_host, staging, lat, stream=None):
    _check(lib.lqcd_gauge_upload(_ptr(dst), prec, recon, _ptr(src_host), _ptr(staging), C.byref(lat),
                                 _stream(stream)))


# ------------------------------------------------------------------ operators

def lqcd_dslash(out, inp, gauge, lat, op, out_subset, dagger, stream=None):
    _check(lib.lqcd_dslash(_ptr(out), _ptr(inp), _ptr(gauge), C.byref(lat), C.byref(op), out_subset,
                           int(dagger), _stream(stream)))


def lqcd_M(out, inp, gauge, lat, op, subset, dagger, tmp, stream=None):
    _check(lib.lqcd_M(_ptr(out), _ptr(inp), _ptr(gauge), C.byref(lat), C.byref(op), subset, int(dagger),
                      _ptr(tmp), _stream(stream)))


def lqcd_M_noalloc(out, inp, gauge, lat, op, subset, dagger, stream=None):
    """lqcd_M without a workspace argument, for callers that cannot allocate
    device memory; the temporaries live in a fixed array inside the library."""
    _check(lib.lqcd_M_noalloc(_ptr(out), _ptr(inp), _ptr(gauge), C.byref(lat), C.byref(op), subset,
                              int(dagger), _stream(stream)))


def lqcd_MdagM(out, inp, gauge, lat, op, subset, tmp, stream=None):
    _check(lib.lqcd_MdagM(_ptr(out), _ptr(inp), _ptr(gauge), C.byref(lat), C.byref(op), subset, _ptr(tmp),
                          _stream(stream)))


def lqcd_eo_prepare(bhat, b_full, gauge, lat, op, tmp, stream=None):
    _check(lib.lqcd_eo_prepare(_ptr(bhat), _ptr(b_full), _ptr(gauge), C.byref(lat), C.byref(op), _ptr(tmp),
                               _stream(stream)))


def lqcd_eo_reconstruct(x_full, b_full, gauge, lat, op, tmp, stream=None):
    _check(lib.lqcd_eo_reconstruct(_ptr(x_full), _ptr(b_full), _ptr(gauge), C.byref(lat), C.byref(op),
                                   _ptr(tmp), _stream(stream)))


def lqcd_cg_solve(x, b, gauge, gauge_sloppy, lat, op, params, subset, workspace, stream=None,
                  raise_on_error=True) -> lqcd_solve_info:
    info = lqcd_solve_info()
    nbytes = workspace.numel() * workspace.element_size()
    st = lib.lqcd_cg_solve(_ptr(x), _ptr(b), _ptr(gauge), _ptr(gauge_sloppy), C.byref(lat), C.byref(op),
                           C.byref(params), subset, C.byref(info), _ptr(workspace), nbytes, _stream(stream))
    if raise_on_error:
        _check(st)
    return info


def lqcd_cgnr_solve(x, b, gauge, gauge_sloppy, lat, op, params, subset, workspace, stream=None,
                    raise_on_error=True) -> lqcd_solve_info:
    info = lqcd_solve_info()
    nbytes = workspace.numel() * workspace.element_size()
    st = lib.lqcd_cgnr_solve(_ptr(x), _ptr(b), _ptr(gauge), _ptr(gauge_sloppy), C.byref(lat), C.byref(op),
                             C.byref(params), subset, C.byref(info), _ptr(workspace), nbytes, _stream(stream))
    if raise_on_error:
        _check(st)
    return info


def lqcd_eo_solve_workspace_bytes(lat, op, params) -> int:
    return int(lib.lqcd_eo_solve_workspace_bytes(C.byref(lat), C.byref(op), C.byref(params)))


def lqcd_eo_solve(x, b, gauge, gauge_sloppy, lat, op, params, workspace, stream=None,
                  raise_on_error=True) -> lqcd_solve_info:
    info = lqcd_solve_info()
    nbytes = workspace.numel() * workspace.element_size()
    st = lib.lqcd_eo_solve(_ptr(x), _ptr(b), _ptr(gauge), _ptr(gauge_sloppy), C.byref(lat), C.byref(op),
                           C.byref(params), C.byref(info), _ptr(workspace), nbytes, _stream(stream))
    if raise_on_error:
        _check(st)
    return info


def lqcd_block_cg_workspace_bytes(lat, op, params) -> int:
    return int(lib.lqcd_block_cg_workspace_bytes(C.byref(lat), C.byref(op), C.byref(params)))


def lqcd_block_cg_solve(x, b, gauge, gauge_sloppy, lat, op, params, workspace, stream=None,
                        raise_on_error=True) -> lqcd_solve_info:
    info = lqcd_solve_info()
    nbytes = workspace.numel() * workspace.element_size()
    st = lib.lqcd_block_cg_solve(_ptr(x), _ptr(b), _ptr(gauge), _ptr(gauge_sloppy), C.byref(lat), C.byref(op),
                                 C.byref(params), C.byref(info), _ptr(workspace), nbytes, _stream(stream))
    if raise_on_error:
        _check(st)
    return info


def batch_items(entries):
    """Array of lqcd_batch_item from dicts with keys lat, mass, gauge,
    gauge_sloppy (may be None), x, b (tensors or device pointers)."""
    arr = (_lib.lqcd_batch_item * len(entries))()
    for i, e in enumerate(entries):
        arr[i].lat = e["lat"]
        arr[i].mass = float(e["mass"])
        arr[i].gauge = _ptr(e["gauge"])
        arr[i].gauge_sloppy = _ptr(e.get("gauge_sloppy"))
        arr[i].x = _ptr(e["x"])
        arr[i].b = _ptr(e["b"])
    return arr


def lqcd_batch_cg_workspace_bytes(n, items, recon, params) -> int:
    return int(lib.lqcd_batch_cg_workspace_bytes(n, C.cast(items, C.c_void_p), recon, C.byref(params)))


def lqcd_batch_cg_solve(n, items, recon, params, workspace, stream=None, raise_on_error=True):
    infos = (lqcd_solve_info * n)()
    nbytes = workspace.numel() * workspace.element_size()
    st = lib.lqcd_batch_cg_solve(n, C.cast(items, C.c_void_p), recon, C.byref(params), C.cast(infos, C.c_void_p),
                                 _ptr(workspace), nbytes, _stream(stream))
    if raise_on_error:
        _check(st)
    return list(infos)


def lqcd_tune_save(path: str) -> None:
    _check(lib.lqcd_tune_save(path.encode()))


def lqcd_tune_load(path: str) -> None:
    _check(lib.lqcd_tune_load(path.encode()))


def lqcd_tune_entries() -> int:
    return int(lib.lqcd_tune_entries())


def lqcd_tune_get(key: str) -> int:
    return int(lib.lqcd_tune_get(key.encode()))


def lqcd_tune_clear() -> None:
    lib.lqcd_tune_clear()


def lqcd_tune_set_enabled(on: bool) -> None:
    lib.lqcd_tune_set_enabled(1 if on else 0)


def lqcd_colour_matrix_bytes(lat, prec) -> int:
    return int(lib.lqcd_colour_matrix_bytes(C.byref(lat), prec))


def lqcd_colour_matrix_pack(dst, prec, src, lat, stream=None):
    _check(lib.lqcd_colour_matrix_pack(_ptr(dst), prec, _ptr(src), C.byref(lat), _stream(stream)))


def lqcd_colour_matrix_unpack(dst, src, prec, lat, stream=None):
    _check(lib.lqcd_colour_matrix_unpack(_ptr(dst), _ptr(src), prec, C.byref(lat), _stream(stream)))


def lqcd_su3_mul(z, x, y, lat, prec, stream=None):
    _check(lib.lqcd_su3_mul(_ptr(z), _ptr(x), _ptr(y), C.byref(lat), prec, _stream(stream)))


def hmc_params(beta: float, tau: float, nsteps: int, integrator: int = LQCD_MINNORM2,
               fermion: int = 1) -> lqcd_hmc_params:
    return lqcd_hmc_params(beta=beta, tau=tau, nsteps=nsteps, integrator=integrator, fermion=fermion)


def lqcd_reduce_workspace_bytes(lat) -> int:
    return int(lib.lqcd_reduce_workspace_bytes(C.byref(lat)))


def lqcd_plaquette(gauge, lat, workspace, stream=None) -> float:
    out = C.c_double()
    nbytes = workspace.numel() * workspace.element_size()
    _check(lib.lqcd_plaquette(C.byref(out), _ptr(gauge), C.byref(lat), _ptr(workspace), nbytes, _stream(stream)))
    return out.value


def lqcd_spinor_dot_re(a, b, lat, workspace, stream=None) -> float:
    out = C.c_double()
    nbytes = workspace.numel() * workspace.element_size()
    _check(lib.lqcd_spinor_dot_re(C.byref(out), _ptr(a), _ptr(b), C.byref(lat), _ptr(workspace), nbytes,
                                  _stream(stream)))
    return out.value


def lqcd_momentum_kinetic(mom, lat, workspace, stream=None) -> float:
    out = C.c_double()
    nbytes = workspace.numel() * workspace.element_size()
    _check(lib.lqcd_momentum_kinetic(C.byref(out), _ptr(mom), C.byref(lat), _ptr(workspace), nbytes,
                                     _stream(stream)))
    return out.value


def lqcd_gauge_force(out, gauge, lat, beta, stream=None):
    _check(lib.lqcd_gauge_force(_ptr(out), _ptr(gauge), C.byref(lat), float(beta), _stream(stream)))


def lqcd_gauge_exp_update(gauge, mom, eps, lat, stream=None):
    _check(lib.lqcd_gauge_exp_update(_ptr(gauge), _ptr(mom), float(eps), C.byref(lat), _stream(stream)))


def lqcd_hmc_workspace_bytes(lat, op, params) -> int:
    return int(lib.lqcd_hmc_workspace_bytes(C.byref(lat), C.byref(op), C.byref(params)))


def lqcd_hmc_trajectory(gauge, mom, phi, lat, op, hmc, params, workspace, stream=None,
                        raise_on_error=True) -> lqcd_hmc_info:
    info = lqcd_hmc_info()
    nbytes = workspace.numel() * workspace.element_size()
    st = lib.lqcd_hmc_trajectory(_ptr(gauge), _ptr(mom), _ptr(phi), C.byref(lat), C.byref(op), C.byref(hmc),
                                 C.byref(params), C.byref(info), _ptr(workspace), nbytes, _stream(stream))
    if raise_on_error:
        _check(st)
    return info


def mg_params(block: int = 4, nvec: int = 12, setup_iters: int = 40, pre_smooth: int = 0, post_smooth: int = 4,
              coarse_iters: int = 30, restart: int = 16) -> lqcd_mg_params:
    return lqcd_mg_params(block=block, nvec=nvec, setup_iters=setup_iters, pre_smooth=pre_smooth,
                          post_smooth=post_smooth, coarse_iters=coarse_iters, restart=restart)


def lqcd_mg_coarse_bytes(lat, nvec, block, prec) -> int:
    return int(lib.lqcd_mg_coarse_bytes(C.byref(lat), nvec, block, prec))


def lqcd_mg_coarse_op_bytes(lat, nvec, block, prec) -> int:
    return int(lib.lqcd_mg_coarse_op_bytes(C.byref(lat), nvec, block, prec))


def lqcd_mg_block_orthonormalize(vecs, nvec, block, lat, stream=None):
    _check(lib.lqcd_mg_block_orthonormalize(_ptr(vecs), nvec, block, C.byref(lat), _stream(stream)))


def lqcd_mg_restrict(coarse, fine, vecs, nvec, block, prec, lat, stream=None):
    _check(lib.lqcd_mg_restrict(_ptr(coarse), _ptr(fine), _ptr(vecs), nvec, block, prec, C.byref(lat),
                                _stream(stream)))


def lqcd_mg_prolong(fine, coarse, vecs, nvec, block, prec, lat, stream=None):
    _check(lib.lqcd_mg_prolong(_ptr(fine), _ptr(coarse), _ptr(vecs), nvec, block, prec, C.byref(lat),
                               _stream(stream)))


def lqcd_mg_coarse_build(Y, gauge, vecs, nvec, block, lat, op, stream=None):
    _check(lib.lqcd_mg_coarse_build(_ptr(Y), _ptr(gauge), _ptr(vecs), nvec, block, C.byref(lat), C.byref(op),
                                    _stream(stream)))


def lqcd_mg_coarse_apply(out, inp, Y, nvec, block, prec, dagger, lat, stream=None):
    _check(lib.lqcd_mg_coarse_apply(_ptr(out), _ptr(inp), _ptr(Y), nvec, block, prec, int(dagger), C.byref(lat),
                                    _stream(stream)))


def lqcd_mg_workspace_bytes(lat, op, mg) -> int:
    return int(lib.lqcd_mg_workspace_bytes(C.byref(lat), C.byref(op), C.byref(mg)))


def lqcd_mg_setup(gauge64, gauge32, random_vectors, lat, op, mg, workspace, stream=None):
    nbytes = workspace.numel() * workspace.element_size()
    _check(lib.lqcd_mg_setup(_ptr(gauge64), _ptr(gauge32), _ptr(random_vectors), C.byref(lat), C.byref(op),
                             C.byref(mg), _ptr(workspace), nbytes, _stream(stream)))


def lqcd_mg_solve(x, b, gauge64, gauge32, lat, op, mg, params, workspace, stream=None,
                  raise_on_error=True) -> lqcd_solve_info:
    info = lqcd_solve_info()
    nbytes = workspace.numel() * workspace.element_size()
    st = lib.lqcd_mg_solve(_ptr(x), _ptr(b), _ptr(gauge64), _ptr(gauge32), C.byref(lat), C.byref(op), C.byref(mg),
                           C.byref(params), C.byref(info), _ptr(workspace), nbytes, _stream(stream))
    if raise_on_error:
        _check(st)
    return info


def lqcd_force(out, gauge, X, Y, lat, op, kind, stream=None):
    _check(lib.lqcd_force(_ptr(out), _ptr(gauge), _ptr(X), _ptr(Y), C.byref(lat), C.byref(op), kind,
                          _stream(stream)))
