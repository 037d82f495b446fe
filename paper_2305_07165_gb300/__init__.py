"""GB300 machine fast Gauss transform: thin Python binding of libfgt.so.

The transform (paper Section 4.2, Algorithm 4; periodic variant Section 5)
runs entirely in the library's CUDA kernels; this module only marshals
arguments through the C ABI declared in ``include/fgt.h``.  PyTorch supplies
device memory and streams.  There is no CPU fallback: every call that needs
the GPU raises if the library or the device is missing.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

__all__ = ["Plan", "PointPlan", "FGTError", "Tuning", "lib", "build_gaussian_tree", "BC_FREE", "BC_PERIODIC", "PREC_FP64", "PREC_SPLIT", "PREC_FP64_TC", "MODE_FUSED",
           "MODE_HIERARCHICAL", "gauss_legendre", "params", "nf_for_range", "legendre_gauss_integrals",
           "spherical_bessel", "legendre_fourier_integrals", "analyze", "HostPlan", "Batch"]

BC_FREE, BC_PERIODIC = 0, 1
PREC_FP64, PREC_SPLIT, PREC_FP64_TC = 0, 1, 2
MODE_FUSED, MODE_HIERARCHICAL = 0, 1
_STATUS = {0: "FGT_OK", 1: "FGT_ERR_ARG", 2: "FGT_ERR_TREE", 3: "FGT_ERR_OOM", 4: "FGT_ERR_CUDA",
           5: "FGT_ERR_TIMEOUT", 6: "FGT_ERR_STATE"}


class FGTError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Tree(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("k", ctypes.c_int32), ("n_leaves", ctypes.c_int64),
                ("leaf_level", ctypes.c_void_p), ("leaf_coord", ctypes.c_void_p)]


class PlanInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("d", "k", "bc", "cutoff_level", "fourier", "max_level", "n_f",
                                              "n_p", "modes_1d", "modes_half")] + \
               [(n, ctypes.c_double) for n in ("delta", "tol", "eps_pw", "D0", "R", "h")] + \
               [(n, ctypes.c_int64) for n in ("n_leaves", "n_boxes", "n_pw_leaves", "n_anchor_boxes",
                                              "n_form_blocks", "n_direct_pairs", "n_gather_pairs", "form_flops",
                                              "eval_flops", "gather_flops", "direct_flops", "device_bytes")] + \
               [("prec", ctypes.c_int32), ("mode", ctypes.c_int32), ("launches", ctypes.c_int32)] + \
               [("n_merge_items", ctypes.c_int64), ("n_push_items", ctypes.c_int64),
                ("n_tc_eval_blocks", ctypes.c_int64), ("n_tc_form_blocks", ctypes.c_int64),
                ("n_sliced_jobs", ctypes.c_int64)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class PointInfo(ctypes.Structure):
    """fgt_point_info."""
    _fields_ = [(n, ctypes.c_int32) for n in ("cutoff_level", "proxy_order", "modes_1d")] + \
               [(n, ctypes.c_int64) for n in ("n_boxes", "n_dense_boxes", "n_incoming_boxes", "n_direct_pairs")] + \
               [("cutoff_length", ctypes.c_double), ("prec", ctypes.c_int32)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class Tuning(ctypes.Structure):
    """Launch-shape knobs of a plan (fgt_tuning)."""
    _fields_ = [(n, ctypes.c_int32) for n in ("form_group", "eval_rows16", "eval_rows_large", "near_phase")] + \
               [("ms", ctypes.c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_lib = None
_lock = threading.Lock()


def lib():
    """Load (building first if the sources are newer) the in-tree libfgt.so, or its bounds-checked
    build libfgt_checked.so when the environment has FGT_LIB=checked."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            if os.environ.get("FGT_LIB") == "checked":
                path = _build.CHECKED_LIB
            L = ctypes.CDLL(path)
            vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
            L.fgt_plan_create_ex.argtypes = [i32, dbl, dbl, dbl, i32, i32, i32, ctypes.POINTER(_Tree), vp]
            L.fgt_plan_create_host.argtypes = [i32, dbl, dbl, dbl, i32, i32, i32, ctypes.POINTER(_Tree), vp]
            L.fgt_plan_host_array.argtypes = [vp, ctypes.c_char_p, vp, vp]
            L.fgt_plan_analyze.argtypes = [i32, dbl, dbl, dbl, i32, i32, i32, ctypes.POINTER(_Tree),
                                           ctypes.POINTER(PlanInfo)]
            L.fgt_plan_get_info.argtypes = [vp, ctypes.POINTER(PlanInfo)]
            L.fgt_plan_set_precision.argtypes = [vp, i32]
            L.fgt_plan_set_mode.argtypes = [vp, i32]
            L.fgt_plan_device_bytes.argtypes = [vp]
            L.fgt_plan_device_bytes.restype = ctypes.c_size_t
            L.fgt_execute.argtypes = [vp, vp, vp]
            L.fgt_execute_async.argtypes = [vp, vp, vp, vp]
            L.fgt_execute_host.argtypes = [vp, vp, vp, vp]
            L.fgt_execute_host_async.argtypes = [vp, vp, vp, vp]
            L.fgt_host_sync.argtypes = [vp]
            L.fgt_execute_noalloc.argtypes = [vp, vp, vp, vp]
            L.fgt_execute_noalloc.restype = ctypes.c_int
            L.fgt_batch_create.argtypes = [vp, i32, vp]
            L.fgt_batch_create_mode.argtypes = [vp, i32, i32, vp]
            L.fgt_batch_status.argtypes = [vp, vp]
            L.fgt_batch_get_info.argtypes = [vp, vp, vp, vp]
            L.fgt_selftest_batch_timeout.argtypes = [vp]
            for name in ("fgt_batch_create_mode", "fgt_batch_status", "fgt_batch_get_info",
                         "fgt_selftest_batch_timeout"):
                getattr(L, name).restype = ctypes.c_int
            L.fgt_batch_execute.argtypes = [vp, vp, vp, vp]
            L.fgt_batch_destroy.argtypes = [vp]
            L.fgt_batch_destroy.restype = None
            L.fgt_execute_batch.argtypes = [vp, vp, vp, i32, vp]
            for name in ("fgt_batch_create", "fgt_batch_execute", "fgt_execute_batch"):
                getattr(L, name).restype = ctypes.c_int
            L.fgt_plan_set_profiling.argtypes = [vp, i32]
            L.fgt_plan_read_profile.argtypes = [vp, vp, vp]
            L.fgt_plan_autotune.argtypes = [vp, vp, vp, vp, i32, ctypes.POINTER(Tuning)]
            L.fgt_plan_set_output_tree.argtypes = [vp, ctypes.POINTER(_Tree)]
            L.fgt_leaf_errors.argtypes = [i32, i32, i64, vp, vp, vp, vp]
            L.fgt_build_gaussian_tree.argtypes = [i32, i32, i32, vp, vp, vp, i32, dbl, i32, i32, vp,
                                                  ctypes.POINTER(vp)]
            L.fgt_built_tree_get.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                             ctypes.POINTER(vp)]
            L.fgt_built_tree_copy_sigma.argtypes = [vp, vp, vp]
            L.fgt_point_plan_create.argtypes = [i32, dbl, dbl, i64, vp, i64, vp, i32, i32, ctypes.POINTER(vp)]
            L.fgt_point_execute.argtypes = [vp, vp, vp, vp]
            L.fgt_point_plan_get_info.argtypes = [vp, ctypes.POINTER(PointInfo)]
            L.fgt_point_destroy.argtypes = [vp]
            L.fgt_point_destroy.restype = None
            L.fgt_built_tree_destroy.argtypes = [vp]
            L.fgt_built_tree_destroy.restype = None
            L.fgt_merge_children.argtypes = [i32, i32, i64, vp, vp, vp, vp]
            L.fgt_plan_get_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
            L.fgt_plan_set_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
            L.fgt_destroy.argtypes = [vp]
            L.fgt_destroy.restype = None
            L.fgt_last_error.restype = ctypes.c_char_p
            L.fgt_device_status.argtypes = [vp]
            L.fgt_check_status.argtypes = [vp, vp, vp]
            L.fgt_selftest_tc_timeout.argtypes = []
            L.fgt_gauss_legendre.argtypes = [i32, vp, vp]
            L.fgt_params.argtypes = [dbl, dbl, i32, vp, vp, vp, vp, vp, vp]
            L.fgt_nf_for_range.argtypes = [dbl, dbl]
            L.fgt_nf_for_range.restype = ctypes.c_int32
            L.fgt_legendre_gauss_integrals.argtypes = [dbl, dbl, i32, vp]
            L.fgt_spherical_bessel.argtypes = [dbl, i32, vp]
            L.fgt_legendre_fourier_integrals.argtypes = [dbl, i32, vp, vp]
            for name in ("fgt_plan_create_ex", "fgt_plan_create_host", "fgt_plan_host_array", "fgt_plan_analyze", "fgt_plan_get_info", "fgt_plan_set_precision",
                         "fgt_plan_set_mode", "fgt_execute", "fgt_execute_async", "fgt_execute_host", "fgt_execute_host_async", "fgt_host_sync",
                         "fgt_gauss_legendre", "fgt_params", "fgt_legendre_gauss_integrals",
                         "fgt_spherical_bessel", "fgt_legendre_fourier_integrals", "fgt_plan_set_profiling",
                         "fgt_plan_read_profile", "fgt_plan_autotune", "fgt_plan_get_tuning",
                         "fgt_plan_set_tuning", "fgt_plan_set_output_tree", "fgt_leaf_errors",
                         "fgt_merge_children", "fgt_build_gaussian_tree", "fgt_built_tree_get",
                         "fgt_built_tree_copy_sigma", "fgt_point_plan_create", "fgt_point_execute",
                         "fgt_point_plan_get_info"):
                getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


def _check(status):
    if status != 0:
        raise FGTError(status, lib().fgt_last_error().decode(errors="replace"))


def check_status() -> dict:
    """fgt_check_status: in the bounds-checked build, the first failing access's source line and the
    failure count since the last call (cleared); {"checked": 0, ...} in the normal build."""
    site, count, checked = ctypes.c_uint(0), ctypes.c_uint(0), ctypes.c_int(0)
    _check(lib().fgt_check_status(ctypes.byref(site), ctypes.byref(count), ctypes.byref(checked)))
    return {"checked": checked.value, "site": site.value, "count": count.value}


def device_status() -> int:
    """fgt_device_status: 1 if a wait of a tensor-core kernel ran out since the last call, else 0
    (and clears it)."""
    v = ctypes.c_int(0)
    _check(lib().fgt_device_status(ctypes.byref(v)))
    return v.value


def selftest_batch_timeout() -> int:
    """Runs the persistent batch kernel on one item whose dependency nothing satisfies (a wait of
    about a millisecond); returns the status it reports (FGT_ERR_TIMEOUT)."""
    v = ctypes.c_int()
    _check(lib().fgt_selftest_batch_timeout(ctypes.byref(v)))
    return v.value


def selftest_tc_timeout() -> None:
    """fgt_selftest_tc_timeout: a bounded wait that runs out on purpose and sets the status word."""
    _check(lib().fgt_selftest_tc_timeout())


def _tree_struct(d, k, level, coord):
    lev = np.ascontiguousarray(level, dtype=np.int32)
    crd = np.ascontiguousarray(coord, dtype=np.int32).reshape(-1)
    if crd.size != lev.size * d:
        raise ValueError("coord must have n_leaves * d entries")
    t = _Tree(d, k, lev.size, lev.ctypes.data, crd.ctypes.data)
    return t, (lev, crd)


def analyze(d, k, delta, tol, level, coord, bc=BC_FREE, prec=PREC_FP64, mode=MODE_FUSED, eps_pw=0.0) -> dict:
    """Host-only planning (no GPU): validates the tree and returns the plan info."""
    t, keep = _tree_struct(d, k, level, coord)
    info = PlanInfo()
    _check(lib().fgt_plan_analyze(d, delta, tol, eps_pw, bc, prec, mode, ctypes.byref(t), ctypes.byref(info)))
    return info.as_dict()


class HostPlan:
    """A plan built without a GPU: lists and tables kept in host memory for inspection."""

    def __init__(self, d, k, delta, tol, level, coord, bc=BC_FREE, prec=PREC_FP64, mode=MODE_FUSED, eps_pw=0.0):
        self.d, self.k = d, k
        t, keep = _tree_struct(d, k, level, coord)
        self._h = ctypes.c_void_p()
        _check(lib().fgt_plan_create_host(d, delta, tol, eps_pw, bc, prec, mode, ctypes.byref(t),
                                          ctypes.byref(self._h)))

    def info(self) -> dict:
        info = PlanInfo()
        _check(lib().fgt_plan_get_info(self._h, ctypes.byref(info)))
        return info.as_dict()

    def array(self, name, dtype):
        p, n = ctypes.c_void_p(), ctypes.c_size_t()
        _check(lib().fgt_plan_host_array(self._h, name.encode(), ctypes.byref(p), ctypes.byref(n)))
        if n.value == 0:
            return np.zeros(0, dtype=dtype)
        buf = (ctypes.c_char * n.value).from_address(p.value)
        return np.frombuffer(bytes(buf), dtype=dtype).copy()

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().fgt_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """A box-FGT plan on the current CUDA device.

    level: int32 [n_leaves]; coord: int32 [n_leaves, d]; k: nodes per dimension.
    ``plan(sigma)`` takes a CUDA float64 tensor [n_leaves, k**d] and returns u.
    """

    def __init__(self, d, k, delta, tol, level, coord, bc=BC_FREE, prec=PREC_FP64, mode=MODE_FUSED, eps_pw=0.0):
        import torch
        if not torch.cuda.is_available():
            raise FGTError(4, "no CUDA device: the box FGT runs only on the GPU")
        torch.cuda.current_device()  # make sure the primary context exists before the library uses it
        self.d, self.k, self.delta, self.tol, self.bc = d, k, delta, tol, bc
        t, keep = _tree_struct(d, k, level, coord)
        self.n_leaves = int(keep[0].size)
        self._src_level, self._src_coord = keep[0], keep[1]
        self._h = ctypes.c_void_p()
        _check(lib().fgt_plan_create_ex(d, delta, tol, eps_pw, bc, prec, mode, ctypes.byref(t),
                                        ctypes.byref(self._h)))

    @property
    def n_points(self):
        return self.n_leaves * self.k ** self.d

    def info(self) -> dict:
        info = PlanInfo()
        _check(lib().fgt_plan_get_info(self._h, ctypes.byref(info)))
        return info.as_dict()

    def set_precision(self, prec):
        _check(lib().fgt_plan_set_precision(self._h, prec))

    def set_mode(self, mode):
        _check(lib().fgt_plan_set_mode(self._h, mode))

    PHASES = ("form", "merge", "gather", "push", "evaluate", "near")

    def set_profiling(self, on=True):
        _check(lib().fgt_plan_set_profiling(self._h, int(bool(on))))

    def read_profile(self):
        """(summed ms per phase, number of executions) since profiling was switched on / last read."""
        ms = np.zeros(6)
        n = ctypes.c_int()
        _check(lib().fgt_plan_read_profile(self._h, ms.ctypes.data, ctypes.byref(n)))
        return dict(zip(self.PHASES, ms.tolist())), n.value

    def device_bytes(self) -> int:
        return int(lib().fgt_plan_device_bytes(self._h))

    def _check_tensor(self, x, name):
        import torch
        if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != torch.float64 or not x.is_contiguous():
            raise TypeError(f"{name} must be a contiguous CUDA float64 tensor")
        n = self.n_out_points if name == "out" else self.n_points
        if x.numel() != n:
            raise ValueError(f"{name} must hold {n} values ({'output' if name == 'out' else 'source'} leaves x k**d)")

    # ---- output tree (Algorithms 5 and 6): u at the nodes of a tree refining the source tree
    n_out_leaves = None

    @property
    def n_out_points(self):
        return (self.n_out_leaves if self.n_out_leaves is not None else self.n_leaves) * self.k ** self.d

    def set_output_tree(self, level=None, coord=None):
        """Evaluate u at the leaves of an output tree: non-overlapping boxes, each inside (or equal
        to) one source leaf, not necessarily covering them (fgt_plan_set_output_tree).  None
        restores the source tree.  execute() then returns u as [n_out_leaves, k**d]."""
        if level is None:
            _check(lib().fgt_plan_set_output_tree(self._h, None))
            self.n_out_leaves = None
            return
        t, keep = _tree_struct(self.d, self.k, level, coord)
        _check(lib().fgt_plan_set_output_tree(self._h, ctypes.byref(t)))
        self.n_out_leaves = int(keep[0].size)

    def execute(self, sigma, out=None, stream=None):
        """Enqueue u = transform(sigma) on `stream` (default: torch's current stream)."""
        import torch
        self._check_tensor(sigma, "sigma")
        if out is None:
            out = torch.empty((self.n_out_points // self.k ** self.d, self.k ** self.d), dtype=sigma.dtype,
                              device=sigma.device)
        self._check_tensor(out, "out")
        s = stream if stream is not None else torch.cuda.current_stream(sigma.device)
        _check(lib().fgt_execute_async(self._h, sigma.data_ptr(), out.data_ptr(), ctypes.c_void_p(s.cuda_stream)))
        return out

    __call__ = execute

    def autotune(self, sigma, out=None, reps=3, stream=None) -> dict:
        """Time the plan's launch-shape knobs on this input (fgt_plan_autotune) and keep the
        fastest; returns the chosen knobs and the step time measured with them."""
        import torch
        self._check_tensor(sigma, "sigma")
        if out is None:
            out = torch.empty_like(sigma)
        self._check_tensor(out, "out")
        s = stream if stream is not None else torch.cuda.current_stream(sigma.device)
        t = Tuning()
        _check(lib().fgt_plan_autotune(self._h, ctypes.c_void_p(sigma.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(s.cuda_stream), int(reps), ctypes.byref(t)))
        return t.as_dict()

    def tuning(self) -> dict:
        t = Tuning()
        _check(lib().fgt_plan_get_tuning(self._h, ctypes.byref(t)))
        return t.as_dict()

    def set_tuning(self, **knobs):
        t = Tuning()
        _check(lib().fgt_plan_get_tuning(self._h, ctypes.byref(t)))
        for k, v in knobs.items():
            setattr(t, k, v)
        _check(lib().fgt_plan_set_tuning(self._h, ctypes.byref(t)))

    def execute_noalloc(self, sigma, out, stream=None):
        """Same transform through fgt_execute_noalloc: the expansions live in the library's fixed
        64 MiB device array, nothing is allocated.  Calls that overlap on the GPU race."""
        import torch
        self._check_tensor(sigma, "sigma")
        self._check_tensor(out, "out")
        s = stream if stream is not None else torch.cuda.current_stream(sigma.device)
        _check(lib().fgt_execute_noalloc(self._h, sigma.data_ptr(), out.data_ptr(), ctypes.c_void_p(s.cuda_stream)))
        return out

    def execute_host(self, sigma, out, stream=None):
        """End to end through the C ABI: host (ideally pinned) float64 arrays in and out."""
        import torch
        for x, n in ((sigma, "sigma"), (out, "out")):
            if isinstance(x, torch.Tensor):
                want = self.n_out_points if n == "out" else self.n_points
                if x.is_cuda or x.dtype != torch.float64 or not x.is_contiguous() or x.numel() != want:
                    raise TypeError(f"{n} must be a contiguous host float64 tensor of {want} values")
            else:
                raise TypeError(f"{n} must be a host torch tensor")
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(lib().fgt_execute_host(self._h, sigma.data_ptr(), out.data_ptr(), ctypes.c_void_p(s.cuda_stream)))
        return out

    def execute_host_async(self, sigma, out, stream=None):
        """Pipelined host-buffer transform (fgt_execute_host_async): returns at once; sigma and out
        stay untouched until host_sync().  Successive calls overlap copies with transforms."""
        import torch
        for x, n in ((sigma, "sigma"), (out, "out")):
            want = self.n_out_points if n == "out" else self.n_points
            if (not isinstance(x, torch.Tensor) or x.is_cuda or x.dtype != torch.float64 or not x.is_contiguous()
                    or x.numel() != want):
                raise TypeError(f"{n} must be a contiguous host float64 tensor of {want} values")
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(lib().fgt_execute_host_async(self._h, sigma.data_ptr(), out.data_ptr(), ctypes.c_void_p(s.cuda_stream)))
        return out

    def host_sync(self):
        """fgt_host_sync: wait until every pipelined host call on this plan has written its output."""
        _check(lib().fgt_host_sync(self._h))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().fgt_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


BATCH_GRAPH, BATCH_PERSISTENT = 0, 1
ERR_TIMEOUT = 5


class Batch:
    """Independent transforms in one launch.

    mode BATCH_GRAPH: one CUDA graph, each transform a parallel branch (captured on the first call,
    recaptured only when a tensor pointer changes).  mode BATCH_PERSISTENT: one persistent kernel
    over a device work queue of every transform's (phase, block) items, with per-transform phase
    counters and bounded waits (``status()`` reports a wait that ran out).  ``batch(sigmas, outs)``
    enqueues all transforms on the current stream.
    """

    def __init__(self, plans, mode=BATCH_GRAPH):
        self.plans = list(plans)
        self.mode = mode
        arr = (ctypes.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        self._h = ctypes.c_void_p()
        _check(lib().fgt_batch_create_mode(arr, len(self.plans), int(mode), ctypes.byref(self._h)))

    def status(self) -> int:
        """0, or FGT_ERR_TIMEOUT when a dependency wait of the persistent kernel ran out since the
        last call (read and cleared; synchronous)."""
        v = ctypes.c_int()
        _check(lib().fgt_batch_status(self._h, ctypes.byref(v)))
        return v.value

    def info(self) -> dict:
        m, n, g = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int()
        _check(lib().fgt_batch_get_info(self._h, ctypes.byref(m), ctypes.byref(n), ctypes.byref(g)))
        return {"mode": m.value, "items": n.value, "grid": g.value}

    def execute(self, sigmas, outs, stream=None):
        import torch
        if len(sigmas) != len(self.plans) or len(outs) != len(self.plans):
            raise ValueError("one sigma and one output per plan")
        for p, s, o in zip(self.plans, sigmas, outs):
            p._check_tensor(s, "sigma")
            p._check_tensor(o, "out")
        n = len(self.plans)
        sp = (ctypes.c_void_p * n)(*[s.data_ptr() for s in sigmas])
        up = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
        st = stream if stream is not None else torch.cuda.current_stream()
        _check(lib().fgt_batch_execute(self._h, sp, up, ctypes.c_void_p(st.cuda_stream)))
        return outs

    __call__ = execute

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().fgt_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- host-side table helpers (no GPU)

def gauss_legendre(k):
    x, w = np.zeros(k), np.zeros(k)
    _check(lib().fgt_gauss_legendre(k, x.ctypes.data, w.ctypes.data))
    return x, w


def params(delta, eps, bc=BC_FREE):
    lc, nf, npp = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    D0, R, h = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().fgt_params(delta, eps, bc, ctypes.byref(lc), ctypes.byref(D0), ctypes.byref(R), ctypes.byref(h),
                            ctypes.byref(nf), ctypes.byref(npp)))
    return dict(cutoff_level=lc.value, D0=D0.value, R=R.value, h=h.value, n_f=nf.value, n_p=npp.value)


def nf_for_range(eps, R):
    return int(lib().fgt_nf_for_range(eps, R))


def legendre_gauss_integrals(lam, t, nmax):
    out = np.zeros(nmax + 1)
    _check(lib().fgt_legendre_gauss_integrals(lam, t, nmax, out.ctypes.data))
    return out


def spherical_bessel(x, nmax):
    out = np.zeros(nmax + 1)
    _check(lib().fgt_spherical_bessel(x, nmax, out.ctypes.data))
    return out


def legendre_fourier_integrals(t, nmax):
    re, im = np.zeros(nmax + 1), np.zeros(nmax + 1)
    _check(lib().fgt_legendre_fourier_integrals(t, nmax, re.ctypes.data, im.ctypes.data))
    return re + 1j * im


def build_gaussian_tree(d, k, centers, alphas, amps=None, periodic=False, eps=1e-10, min_level=0, max_level=12,
                        stream=None):
    """Algorithm 3 on the GPU (fgt_build_gaussian_tree) for sigma = sum_i a_i exp(-|x - c_i|^2 / alpha_i):
    returns (level int32 [n], coord int32 [n, d], sigma CUDA float64 [n, k**d]) of the 2:1-balanced
    tree whose leaves resolve sigma to eps ||sigma||_2 by the error monitor of eq. (funerr)."""
    import torch
    c = np.ascontiguousarray(centers, dtype=np.float64).reshape(-1, d)
    a = np.ascontiguousarray(alphas, dtype=np.float64).reshape(-1)
    w = None if amps is None else np.ascontiguousarray(amps, dtype=np.float64).reshape(-1)
    if len(a) != len(c) or (w is not None and len(w) != len(c)):
        raise ValueError("one alpha (and amplitude) per centre")
    torch.cuda.current_device()
    st = stream if stream is not None else torch.cuda.current_stream()
    h = ctypes.c_void_p()
    _check(lib().fgt_build_gaussian_tree(d, k, len(a), c.ctypes.data, a.ctypes.data,
                                         None if w is None else w.ctypes.data, int(bool(periodic)), float(eps),
                                         int(min_level), int(max_level), ctypes.c_void_p(st.cuda_stream),
                                         ctypes.byref(h)))
    try:
        n = ctypes.c_int64()
        pl, pc, ps = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _check(lib().fgt_built_tree_get(h, ctypes.byref(n), ctypes.byref(pl), ctypes.byref(pc), ctypes.byref(ps)))
        nl = n.value
        level = np.ctypeslib.as_array((ctypes.c_int32 * nl).from_address(pl.value)).copy() if nl else np.zeros(0, np.int32)
        coord = (np.ctypeslib.as_array((ctypes.c_int32 * (nl * d)).from_address(pc.value)).copy().reshape(nl, d)
                 if nl else np.zeros((0, d), np.int32))
        sigma = torch.empty((nl, k ** d), dtype=torch.float64, device="cuda")
        _check(lib().fgt_built_tree_copy_sigma(h, ctypes.c_void_p(sigma.data_ptr()), ctypes.c_void_p(st.cuda_stream)))
        st.synchronize()
    finally:
        lib().fgt_built_tree_destroy(h)
    return level, coord, sigma


class PointPlan:
    """The discrete Gauss transform u_i = sum_j exp(-|x_i - y_j|^2/delta) q_j in free space
    (fgt_point_plan_create / fgt_point_execute): sources and targets fixed at creation (host
    arrays [n, d]), weights and results as CUDA float64 tensors in the callers' point orders.
    prec: PREC_FP64, or PREC_SPLIT (tol >= 1e-7) for FP32 Lagrange weights, anterpolation,
    interpolation and expansions around FP64 proxy values, direct pairs and results."""

    def __init__(self, d, delta, tol, src, tgt, n_s=64, prec=PREC_FP64):
        import torch
        if not torch.cuda.is_available():
            raise FGTError(4, "no CUDA device: the point FGT runs only on the GPU")
        torch.cuda.current_device()
        y = np.ascontiguousarray(src, dtype=np.float64).reshape(-1, d)
        x = np.ascontiguousarray(tgt, dtype=np.float64).reshape(-1, d)
        self.d, self.n_src, self.n_tgt = d, len(y), len(x)
        self._h = ctypes.c_void_p()
        _check(lib().fgt_point_plan_create(d, float(delta), float(tol), len(y), y.ctypes.data, len(x), x.ctypes.data,
                                           int(n_s), int(prec), ctypes.byref(self._h)))

    def info(self) -> dict:
        i = PointInfo()
        _check(lib().fgt_point_plan_get_info(self._h, ctypes.byref(i)))
        return i.as_dict()

    def execute(self, q, out=None, stream=None):
        import torch
        if not (isinstance(q, torch.Tensor) and q.is_cuda and q.dtype == torch.float64 and q.is_contiguous()
                and q.numel() == self.n_src):
            raise TypeError(f"q must be a contiguous CUDA float64 tensor of {self.n_src} values")
        if out is None:
            out = torch.empty(self.n_tgt, dtype=torch.float64, device=q.device)
        if not (out.is_cuda and out.dtype == torch.float64 and out.is_contiguous() and out.numel() == self.n_tgt):
            raise TypeError(f"out must be a contiguous CUDA float64 tensor of {self.n_tgt} values")
        s = stream if stream is not None else torch.cuda.current_stream(q.device)
        _check(lib().fgt_point_execute(self._h, ctypes.c_void_p(q.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(s.cuda_stream)))
        return out

    __call__ = execute

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().fgt_point_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
