"""Python binding of the C-ABI: argument marshalling only.

``SkelFMM`` owns one plan handle (tree + interpolative decompositions on the
host, operators uploaded to the GPU once). ``apply`` / ``apply_transpose``
take torch tensors (CUDA or CPU; CPU tensors go through the C-ABI's host
staging) or numpy arrays and call ``skel_apply`` / ``skel_apply_transpose``;
every step of the apply runs in the library's CUDA kernels. ``SkelApply`` is a
``torch.autograd.Function`` whose backward is the transpose apply.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import SkelKernel, SkelOptions, SkelPlanDims, SkelStats, SkelTimings, SkelTuning, check

PHASES = ("permute_in", "upward", "translations", "reduce", "downward", "permute_out")

_DTYPES = {("fp64", False): torch.float64, ("fp64", True): torch.complex128,
           ("fp32", False): torch.float32, ("fp32", True): torch.complex64,
           ("fp32_tc", False): torch.float32, ("fp32_tc", True): torch.complex64}


def _options(proxy_p, nrhs_max, host_only, num_threads, device_build=False, store_tiles=False, store_stages=0,
             updown_tc=False):
    return SkelOptions(int(proxy_p), int(nrhs_max), int(bool(host_only)), int(num_threads), int(bool(device_build)),
                       int(store_tiles), int(store_stages), int(bool(updown_tc)))


class SkelFMM:
    """One skeletonized-FMM plan (Algorithm 1 done, ready for Algorithm 2).

    ``device_build=True`` runs Algorithm 1 (proxy matrices, pivoted QR, T) on
    the current CUDA device instead of the host cores. ``store_tiles`` keeps
    the tensor-core translations' kernel values on the device so that FP32_TC
    applies read them instead of evaluating the kernel: 1 (or True) every
    tile's values (same result bit for bit), 2 the symmetric store (each
    block two tiles share held once; same result up to FP32 rounding).
    ``store_stages`` (4, 5 or 8, 0 = 4): the per-tile store kernel's form
    (skel_options.store_stages; same result; the autotuner may change it).
    ``updown_tc``: FP32_TC applies also run the upward / downward skeleton
    GEMMs on the tensor cores (less accurate than the CUDA-core default on
    these cancelling sums; see skel_options.updown_tc).
    """

    def __init__(self, points, kernel: str = "laplace3d", tol: float = 1e-6, leaf_size: int = 128,
                 kappa: float = 0.0, proxy_p: int = 0, nrhs_max: int = 32, host_only: bool = False,
                 num_threads: int = 0, device_build: bool = False, store_tiles: bool = False, store_stages: int = 0,
                 updown_tc: bool = False, _handle=None):
        self._lib = _lib.load()
        self.kernel = kernel
        self.kappa = float(kappa)
        self.is_complex = kernel in ("helmholtz3d", "helmholtz2d")
        self.nrhs_max = int(nrhs_max)
        if _handle is not None:
            self._h = _handle
        else:
            pts = np.ascontiguousarray(points, dtype=np.float64)
            n, dim = pts.shape
            h = ctypes.c_void_p()
            opts = _options(proxy_p, nrhs_max, host_only, num_threads, device_build, store_tiles, store_stages,
                            updown_tc)
            check(self._lib.skel_build(pts.ctypes.data, n, dim, SkelKernel(_lib.KERNELS[kernel], self.kappa),
                                       float(tol), int(leaf_size), ctypes.byref(opts), ctypes.byref(h)))
            self._h = h
        self.n = self.info()["n_points"]

    # ---- construction from an external plan --------------------------------------
    @classmethod
    def from_plan(cls, points, kernel: str, plan: dict, kappa: float = 0.0, nrhs_max: int = 32,
                  host_only: bool = False, store_tiles: bool = False, store_stages: int = 0,
                  updown_tc: bool = False):
        """Handle from a plan in the skel.h exchange format (dict of arrays)."""
        lib = _lib.load()
        pts = np.ascontiguousarray(points, dtype=np.float64)
        n, dim = pts.shape
        arr = {
            "level": np.ascontiguousarray(plan["level"], dtype=np.int32),
            "coord": np.ascontiguousarray(plan["coord"], dtype=np.int32),
            "parent": np.ascontiguousarray(plan["parent"], dtype=np.int64),
            "is_leaf": np.ascontiguousarray(plan["is_leaf"], dtype=np.int8),
            "idx_ptr": np.ascontiguousarray(plan["idx_ptr"], dtype=np.int64),
            "idx": np.ascontiguousarray(plan["idx"], dtype=np.int64),
            "piv": np.ascontiguousarray(plan["piv"], dtype=np.int64),
            "k": np.ascontiguousarray(plan["k"], dtype=np.int32),
            "T_ptr": np.ascontiguousarray(plan["T_ptr"], dtype=np.int64),
        }
        T = np.asarray(plan["T"])
        T = np.ascontiguousarray(T.view(np.float64) if np.iscomplexobj(T) else T, dtype=np.float64)
        center = np.ascontiguousarray(plan["center"], dtype=np.float64)
        nb = arr["level"].shape[0]
        h = ctypes.c_void_p()
        opts = _options(0, nrhs_max, host_only, 0, False, store_tiles, store_stages, updown_tc)
        check(lib.skel_plan_import(pts.ctypes.data, n, dim, SkelKernel(_lib.KERNELS[kernel], float(kappa)),
                                   center.ctypes.data, float(plan["side"]), nb,
                                   *[arr[k].ctypes.data for k in ("level", "coord", "parent", "is_leaf",
                                                                  "idx_ptr", "idx", "piv", "k", "T_ptr")],
                                   T.ctypes.data, ctypes.byref(opts), ctypes.byref(h)))
        return cls(None, kernel, kappa=kappa, nrhs_max=nrhs_max, _handle=h)

    # ---- queries --------------------------------------------------------------------------
    def info(self) -> dict:
        s = SkelStats()
        check(self._lib.skel_info(self._h, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in SkelStats._fields_}

    def export_plan(self) -> dict:
        d = SkelPlanDims()
        check(self._lib.skel_plan_get_dims(self._h, ctypes.byref(d)))
        nb, ni, nt, dim = d.n_boxes, d.n_index, d.n_T, d.dim
        out = {
            "level": np.zeros(nb, np.int32), "coord": np.zeros(nb * dim, np.int32),
            "parent": np.zeros(nb, np.int64), "is_leaf": np.zeros(nb, np.int8),
            "idx_ptr": np.zeros(nb + 1, np.int64), "idx": np.zeros(ni, np.int64),
            "piv": np.zeros(ni, np.int64), "k": np.zeros(nb, np.int32),
            "T_ptr": np.zeros(nb + 1, np.int64), "T": np.zeros(nt * (2 if d.is_complex else 1), np.float64),
        }
        check(self._lib.skel_plan_export(self._h, *[out[k].ctypes.data for k in (
            "level", "coord", "parent", "is_leaf", "idx_ptr", "idx", "piv", "k", "T_ptr", "T")]))
        if d.is_complex:
            out["T"] = out["T"].view(np.complex128)
        out["coord"] = out["coord"].reshape(nb, dim)
        out["center"] = np.array(d.center[:dim])
        out["side"] = d.side
        return out

    def neighbors(self, which: int):
        nb = self.info()["n_boxes"]
        ptr = np.zeros(nb + 1, np.int64)
        check(self._lib.skel_neighbors_export(self._h, which, ptr.ctypes.data, None))
        lst = np.zeros(int(ptr[-1]), np.int64)
        check(self._lib.skel_neighbors_export(self._h, which, ptr.ctypes.data, lst.ctypes.data))
        return ptr, lst

    def set_profiling(self, max_applies: int) -> None:
        """Record phase events for the next `max_applies` applies (0 = off)."""
        check(self._lib.skel_set_profiling(self._h, int(max_applies)))

    def last_timings(self) -> dict:
        """Phase durations (ms, summed over the captured applies), launches, applies;
        ``main_near`` / ``main_launches``: the main translation kernel inside ``translations``."""
        t = SkelTimings()
        check(self._lib.skel_last_timings(self._h, ctypes.byref(t)))
        out = {p: t.ms[i] for i, p in enumerate(PHASES)}
        out["launches"] = t.launches
        out["n_applies"] = t.n_applies
        out["main_near"] = t.ms_main
        out["main_launches"] = t.main_launches
        return out

    def device_status(self) -> None:
        """Raise SkelError(SKEL_ERR_TIMEOUT) if a bounded device wait gave up."""
        check(self._lib.skel_device_status(self._h))

    def autotune(self, nrhs: int | None = None, allow_store: bool = True, stream=None) -> dict:
        """Measure and keep the fastest kernel variants for FP32 applies of nrhs
        right-hand sides (skel_autotune): per-level up/down variants and, for
        the tensor-core path, stored or on-the-fly kernel tiles."""
        if stream is None and torch.cuda.is_available():
            stream = torch.cuda.current_stream().cuda_stream
        t = SkelTuning()
        check(self._lib.skel_autotune(self._h, int(nrhs or self.nrhs_max), int(bool(allow_store)),
                                      ctypes.c_void_p(stream or 0), ctypes.byref(t)))
        return {f: getattr(t, f) for f, _ in SkelTuning._fields_}

    def apply_into(self, q_cm, u_cm, nrhs: int, precision: str = "fp32_tc", transpose: bool = False,
                   stream=None) -> None:
        """Apply on preallocated column-major buffers (raw data pointers, no copies).

        q_cm, u_cm: tensors whose memory is the n x nrhs column-major layout of
        skel.h (for example the .t() of a contiguous (nrhs, n) tensor).
        """
        if stream is None and q_cm.is_cuda:
            stream = torch.cuda.current_stream(q_cm.device).cuda_stream
        fn = self._lib.skel_apply_transpose if transpose else self._lib.skel_apply
        check(fn(self._h, ctypes.c_void_p(q_cm.data_ptr()), ctypes.c_void_p(u_cm.data_ptr()), int(nrhs),
                 _lib.PRECISIONS[precision], ctypes.c_void_p(stream or 0)))

    # ---- apply ------------------------------------------------------------------------------
    def _call(self, fn, q, precision: str, stream):
        dtype = _DTYPES[(precision, self.is_complex)]
        is_np = isinstance(q, np.ndarray)
        qt = torch.from_numpy(np.asarray(q)) if is_np else q
        if qt.shape[0] != self.n or qt.dim() not in (1, 2):
            raise ValueError(f"q must have shape ({self.n},) or ({self.n}, nrhs)")
        squeeze = qt.dim() == 1
        q2 = qt.reshape(self.n, 1) if squeeze else qt
        nrhs = q2.shape[1]
        # column-major n x nrhs: each right-hand side contiguous
        qc = q2.to(dtype).t().contiguous()
        uc = torch.empty_like(qc)
        if stream is None and qc.is_cuda:
            stream = torch.cuda.current_stream(qc.device).cuda_stream
        check(fn(self._h, ctypes.c_void_p(qc.data_ptr()), ctypes.c_void_p(uc.data_ptr()), nrhs,
                 _lib.PRECISIONS[precision], ctypes.c_void_p(stream or 0)))
        u = uc.t()
        u = u.reshape(self.n) if squeeze else u
        return u.numpy() if is_np else u

    def apply(self, q, precision: str = "fp64", stream=None):
        """u = A~ q (Algorithm 2)."""
        return self._call(self._lib.skel_apply, q, precision, stream)

    def apply_transpose(self, ubar, precision: str = "fp64", stream=None):
        """A~^T ubar (plain transpose, no conjugation)."""
        return self._call(self._lib.skel_apply_transpose, ubar, precision, stream)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.skel_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SkelApply(torch.autograd.Function):
    """u = A~ q with backward q_grad = A~^H u_grad = conj(A~^T conj(u_grad))."""

    @staticmethod
    def forward(ctx, q, fmm: SkelFMM, precision: str = "fp64"):
        ctx.fmm = fmm
        ctx.precision = precision
        return fmm.apply(q, precision)

    @staticmethod
    def backward(ctx, g):
        fmm = ctx.fmm
        if fmm.is_complex:
            gq = torch.conj(fmm.apply_transpose(torch.conj(g).resolve_conj(), ctx.precision))
            return gq.resolve_conj(), None, None
        return fmm.apply_transpose(g, ctx.precision), None, None


class SkelBatch:
    """Many independent point sets: one plan each, applied together.

    ``apply_into`` queues every set's apply (or transpose apply) on one stream
    through ``skel_apply_batch``, without host synchronisation, so that a
    whole batch and its adjoint can be captured into one CUDA graph
    (``capture``).
    """

    def __init__(self, point_sets, kernel: str = "laplace2d", tol: float = 1e-7, leaf_size: int = 64,
                 kappa: float = 0.0, nrhs_max: int = 4, num_threads: int = 0, device_build: bool = False,
                 host_only: bool = False):
        self._lib = _lib.load()
        # every set's plan in one skel_build_batch call (the host phases of
        # the sets run in parallel)
        pts = [np.ascontiguousarray(p, dtype=np.float64) for p in point_sets]
        if not pts:
            raise ValueError("no point sets")
        dim = pts[0].shape[1]
        if any(p.ndim != 2 or p.shape[1] != dim for p in pts):
            raise ValueError("every set must be an (n_i, dim) array of one dim")
        ns = len(pts)
        pp = (ctypes.c_void_p * ns)(*[p.ctypes.data for p in pts])
        nn = (ctypes.c_int64 * ns)(*[p.shape[0] for p in pts])
        out = (ctypes.c_void_p * ns)()
        opts = _options(0, nrhs_max, host_only, num_threads, device_build)
        check(self._lib.skel_build_batch(ns, pp, nn, dim, SkelKernel(_lib.KERNELS[kernel], float(kappa)), float(tol),
                                         int(leaf_size), ctypes.byref(opts), out))
        self.plans = [SkelFMM(None, kernel, tol, leaf_size, kappa=kappa, nrhs_max=nrhs_max,
                              _handle=ctypes.c_void_p(out[i])) for i in range(ns)]
        self.sizes = [f.n for f in self.plans]
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        self.kernel, self.kappa, self.nrhs_max = kernel, float(kappa), int(nrhs_max)
        self._hs = (ctypes.c_void_p * len(self.plans))(*[f._h.value for f in self.plans])

    def merged(self, nrhs_max: int | None = None, store_tiles: bool = False, host_only: bool = False) -> SkelFMM:
        """One plan over every set (skel_merge): each phase of the apply is a
        single launch over all sets. Its q and u are N x nrhs column-major with
        the sets' points one after the other (set i: rows offsets[i] ..
        offsets[i+1]); each set's values equal its own apply bit for bit."""
        nm = int(nrhs_max or self.nrhs_max)
        h = ctypes.c_void_p()
        opts = _options(0, nm, host_only, 0, False, store_tiles)
        check(self._lib.skel_merge(self._hs, len(self.plans), ctypes.byref(opts), ctypes.byref(h)))
        return SkelFMM(None, self.kernel, kappa=self.kappa, nrhs_max=nm, _handle=h)

    def apply_into(self, qs, us, nrhs: int, precision: str = "fp32_tc", transpose: bool = False, stream=None):
        """qs[i], us[i]: device tensors holding set i's n_i x nrhs column-major buffers."""
        if len(qs) != len(self.plans) or len(us) != len(self.plans):
            raise ValueError("one q and one u per set")
        if stream is None:
            stream = torch.cuda.current_stream(qs[0].device).cuda_stream if qs else 0
        qp = (ctypes.c_void_p * len(qs))(*[t.data_ptr() for t in qs])
        up = (ctypes.c_void_p * len(us))(*[t.data_ptr() for t in us])
        check(self._lib.skel_apply_batch(self._hs, len(self.plans), qp, up, int(nrhs), _lib.PRECISIONS[precision],
                                         int(bool(transpose)), ctypes.c_void_p(stream)))

    def capture(self, qs, us, nrhs: int, precision: str = "fp32_tc", adjoint_qs=None, adjoint_us=None):
        """A CUDA graph of the batched apply (and, if given, the batched
        transpose apply on adjoint_qs -> adjoint_us). Replay with .replay()."""
        self.apply_into(qs, us, nrhs, precision)              # warm-up outside the capture
        if adjoint_qs is not None:
            self.apply_into(adjoint_qs, adjoint_us, nrhs, precision, transpose=True)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                self.apply_into(qs, us, nrhs, precision)
                if adjoint_qs is not None:
                    self.apply_into(adjoint_qs, adjoint_us, nrhs, precision, transpose=True)
        return g

    def close(self):
        for f in self.plans:
            f.close()


def skel_apply(q, fmm: SkelFMM, precision: str = "fp64"):
    """Differentiable apply (backward = transpose apply)."""
    return SkelApply.apply(q, fmm, precision)
