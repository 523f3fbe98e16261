"""Direct summation u_i = sum_{j != i} G(x_i, x_j) q_j (Section 1, Eq. (1)).

Oracle (test infrastructure only). Two independent implementations:

* ``direct_sum_numpy`` — dense numpy blocks from ``kernels.kernel_matrix``.
* ``direct_sum``       — the plain C/OpenMP loop in ``direct.c``.

Both return u at the requested targets (all points when ``targets`` is None)
with the same (m x nrhs, Fortran-order) layout as q.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import kernels
from .build import LIB_PATH, build

_KIND_CODE = {"laplace2d": 0, "laplace3d": 1, "helmholtz3d": 2, "helmholtz2d": 3}
_lib = None


def _load():
    global _lib
    if _lib is None:
        path = LIB_PATH if os.path.exists(LIB_PATH) else build()
        lib = ctypes.CDLL(path)
        lib.oracle_direct_sum.restype = None
        lib.oracle_direct_sum.argtypes = [
            ctypes.c_int, ctypes.c_double, ctypes.c_int,
            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int,
            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def _as_2d(q: np.ndarray) -> np.ndarray:
    return q[:, None] if q.ndim == 1 else q


def direct_sum_numpy(kind: str, x: np.ndarray, q: np.ndarray, targets=None,
                     kappa: float = 0.0, block: int = 2048) -> np.ndarray:
    """u = A q with A_ij = G(x_i, x_j), zero diagonal, numpy blocks."""
    x = np.asarray(x, dtype=np.float64)
    q2 = _as_2d(np.asarray(q))
    tidx = np.arange(x.shape[0]) if targets is None else np.asarray(targets)
    dtype = np.complex128 if (kernels.is_complex(kind) or np.iscomplexobj(q2)) else np.float64
    u = np.zeros((tidx.shape[0], q2.shape[1]), dtype=dtype)
    for t0 in range(0, tidx.shape[0], block):
        xt = x[tidx[t0:t0 + block]]
        for s0 in range(0, x.shape[0], block):
            g = kernels.kernel_matrix(kind, xt, x[s0:s0 + block], kappa)
            u[t0:t0 + block] += g @ q2[s0:s0 + block]
    return np.asfortranarray(u if q.ndim == 2 else u[:, 0])


def direct_sum(kind: str, x: np.ndarray, q: np.ndarray, targets=None,
               kappa: float = 0.0) -> np.ndarray:
    """u = A q evaluated by the C/OpenMP loop (FP64 / complex128)."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    n, dim = x.shape
    squeeze = q.ndim == 1
    q2 = _as_2d(np.asarray(q))
    nrhs = q2.shape[1]
    cplx = kernels.is_complex(kind)
    if cplx:
        qf = np.asfortranarray(q2.astype(np.complex128))
    else:
        if np.iscomplexobj(q2):
            raise ValueError("complex charges need a complex kernel")
        qf = np.asfortranarray(q2.astype(np.float64))
    xt = x if targets is None else np.ascontiguousarray(x[np.asarray(targets)])
    m = xt.shape[0]
    u = np.zeros((m, nrhs), dtype=qf.dtype, order="F")
    lib.oracle_direct_sum(_KIND_CODE[kind], float(kappa), dim,
                          x.ctypes.data, n, qf.ctypes.data, nrhs,
                          xt.ctypes.data, m, u.ctypes.data)
    return u[:, 0] if squeeze else u
