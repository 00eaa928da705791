"""Device field allocation and host <-> device transfer helpers.

Device memory comes from PyTorch's caching allocator (a uint8 tensor per
field); the layout conversion itself is done by the library's pack / unpack
kernels. Host arrays are complex128 numpy arrays in the layouts documented in
``include/lqcd.h``.
"""
from __future__ import annotations

import numpy as np
import torch

from . import api


def empty(nbytes: int, device="cuda") -> torch.Tensor:
    """Uninitialised device buffer (torch allocations are 512-byte aligned)."""
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def host_spinor_shape(lat, subset: int):
    X, Y, Z, T = (lat.dims[k] for k in range(4))
    if subset == api.LQCD_FULL:
        return (lat.n5, T, Z, Y, X, 4, 3)
    return (lat.n5, T, Z, Y, X // 2, 4, 3)


def host_gauge_shape(lat):
    X, Y, Z, T = (lat.dims[k] for k in range(4))
    return (T, Z, Y, X, 4, 3, 3)


def _as_device_f64(a) -> torch.Tensor:
    if isinstance(a, torch.Tensor):
        t = a if a.dtype == torch.complex128 else a.to(torch.complex128)
        return torch.view_as_real(t.contiguous().cuda()).reshape(-1)
    arr = np.ascontiguousarray(a, dtype=np.complex128)
    return torch.from_numpy(arr.view(np.float64).reshape(-1)).cuda()


def spinor_to_device(psi, lat, prec: int, subset: int, stream=None) -> torch.Tensor:
    shape = host_spinor_shape(lat, subset)
    if tuple(np.shape(psi)) != shape:
        psi = np.reshape(psi, shape)
    staging = _as_device_f64(psi)
    dst = empty(api.lqcd_spinor_bytes(lat, prec, subset))
    api.lqcd_spinor_pack(dst, prec, subset, staging, lat, stream)
    return dst


def spinor_to_host(field: torch.Tensor, lat, prec: int, subset: int, stream=None) -> np.ndarray:
    shape = host_spinor_shape(lat, subset)
    n = int(np.prod(shape))
    staging = torch.empty(2 * n, dtype=torch.float64, device="cuda")
    api.lqcd_spinor_unpack(staging, field, prec, subset, lat, stream)
    return staging.cpu().numpy().view(np.complex128).reshape(shape)


def gauge_to_device(U, lat, prec: int, recon: int, stream=None) -> torch.Tensor:
    staging = _as_device_f64(U)
    dst = empty(api.lqcd_gauge_bytes(lat, prec, recon))
    api.lqcd_gauge_pack(dst, prec, recon, staging, lat, stream)
    return dst


def gauge_to_host(field: torch.Tensor, lat, prec: int, recon: int, stream=None) -> np.ndarray:
    shape = host_gauge_shape(lat)
    n = int(np.prod(shape))
    staging = torch.empty(2 * n, dtype=torch.float64, device="cuda")
    api.lqcd_gauge_unpack(staging, field, prec, recon, lat, stream)
    return staging.cpu().numpy().view(np.complex128).reshape(shape)


def host_colour_matrix_shape(lat):
    X, Y, Z, T = (int(lat.dims[k]) for k in range(4))
    return (int(lat.n5), T, Z, Y, X, 3, 3)


def colour_matrix_to_device(M, lat, prec: int, stream=None) -> torch.Tensor:
    staging = _as_device_f64(M)
    dst = empty(api.lqcd_colour_matrix_bytes(lat, prec))
    api.lqcd_colour_matrix_pack(dst, prec, staging, lat, stream)
    return dst


def colour_matrix_to_host(field: torch.Tensor, lat, prec: int, stream=None) -> np.ndarray:
    shape = host_colour_matrix_shape(lat)
    staging = torch.empty(2 * int(np.prod(shape)), dtype=torch.float64, device="cuda")
    api.lqcd_colour_matrix_unpack(staging, field, prec, lat, stream)
    return staging.cpu().numpy().view(np.complex128).reshape(shape)


def checkerboard(full: np.ndarray, parity: int) -> np.ndarray:
    """Sites of one parity of a full-lattice array ``[..., T, Z, Y, X, 4, 3]``
    in lexicographic order, shaped ``[..., T, Z, Y, X/2, 4, 3]``."""
    T, Z, Y, X = full.shape[-6:-2]
    t, z, y, x = np.meshgrid(np.arange(T), np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    idx = np.nonzero(((x + y + z + t) % 2).reshape(-1) == parity)[0]
    flat = full.reshape(full.shape[:-6] + (T * Z * Y * X, 4, 3))
    return flat[..., idx, :, :].reshape(full.shape[:-6] + (T, Z, Y, X // 2, 4, 3))
