"""Python binding of the GB300 Cartesian FMM C ABI (include/fmm_gb300.h).

Argument marshalling only: every step of the method runs in the CUDA
library ``libfmm_gb300.so``; PyTorch provides device memory and streams.
The names mirror the C entry points (fmm_create_tree -> create_tree, ...).
There is no CPU fallback: if the library is missing, loading fails loudly.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfmm_gb300.so")

FMM_OK, FMM_EINVAL, FMM_ENOMEM, FMM_EORDER, FMM_ECUDA, FMM_ETIMEOUT, FMM_EBUDGET, FMM_ESTATE = (
    0, -1, -2, -3, -4, -5, -6, -7)
PRECISIONS = {"fp64": 0, "fp32": 1, "3xtf32": 2}
PHASES = ["keys", "sort", "cells", "lists", "dtables", "upward", "fold", "m2l", "l2l", "l2p", "p2p"]
ARRAYS = {"keys": (0, torch.int64, 1), "perm": (1, torch.int32, 1), "level": (2, torch.int32, 1),
          "coord": (3, torch.int32, 3), "range": (4, torch.int32, 2), "parent": (5, torch.int32, 1),
          "child": (6, torch.int32, 2), "centre": (7, torch.float64, 3),
          "half": (8, torch.float64, 1), "m2l": (9, torch.int32, 2), "p2p": (10, torch.int32, 2),
          "multipole": (11, torch.float64, 0), "local": (12, torch.float64, 0),
          "system": (13, torch.int32, 1)}


class FMMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (status %d)" % (msg, status))
        self.status = status


class TreeInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("ncells", C.c_int64), ("nleaves", C.c_int64),
                ("nlevels", C.c_int32), ("source_order", C.c_int32), ("n_m2l", C.c_int64),
                ("n_p2p", C.c_int64), ("n_p2p_interactions", C.c_int64),
                ("n_doffsets", C.c_int64), ("theta", C.c_double), ("lo", C.c_double * 3),
                ("side", C.c_double), ("device_bytes", C.c_int64), ("nsystems", C.c_int64),
                ("tc_tiles", C.c_int64), ("tc_rows", C.c_int64), ("tc_chunks", C.c_int64),
                ("bh_m2p", C.c_int64), ("bh_p2p", C.c_int64), ("source_order_hi", C.c_int64)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["lo"] = list(self.lo)
        return d


class Tuning(C.Structure):
    _fields_ = [("p2p_variant", C.c_int), ("m2l_tensor", C.c_int), ("tc_chunk_rows", C.c_int),
                ("candidates", C.c_int), ("ms_per_evaluate", C.c_float), ("m2l_harmonic", C.c_int),
                ("p2p_targets", C.c_int), ("m2l_tiled", C.c_int)]


_lib = None
_lock = threading.Lock()


def lib():
    """Load libfmm_gb300.so (built by ``__graft_entry__.build()``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError("libfmm_gb300.so is not built (%s); run __graft_entry__.build()"
                                  % LIB_PATH)
            L = C.CDLL(LIB_PATH)
            vp, i64, dbl, i32 = C.c_void_p, C.c_int64, C.c_double, C.c_int
            L.fmm_create_tree.argtypes = [C.POINTER(vp), i32, vp, i32, i32, C.c_size_t]
            L.fmm_set_sources.argtypes = [vp, vp, vp, i64, i32]
            L.fmm_evaluate.argtypes = [vp, i32, dbl, i32, i32, vp, vp]
            L.fmm_destroy.argtypes = [vp]
            L.fmm_status_string.argtypes = [i32]
            L.fmm_status_string.restype = C.c_char_p
            L.fmm_last_error.argtypes = [vp]
            L.fmm_last_error.restype = C.c_char_p
            L.fmm_get_info.argtypes = [vp, C.POINTER(TreeInfo)]
            L.fmm_copy_array.argtypes = [vp, i32, vp, C.c_size_t, C.POINTER(C.c_size_t)]
            L.fmm_set_profiling.argtypes = [vp, i32]
            L.fmm_get_phase_times.argtypes = [vp, C.POINTER(C.c_float)]
            L.fmm_launch_count.argtypes = [vp]
            L.fmm_launch_count.restype = i64
            L.fmm_direct_sum.argtypes = [vp, vp, vp, i64, i32, vp, i64, vp, vp]
            L.fmm_morton_order.argtypes = [vp, vp, i64, vp, vp]
            for f in ("fmm_create_tree", "fmm_set_sources", "fmm_evaluate", "fmm_destroy",
                      "fmm_get_info", "fmm_copy_array", "fmm_set_profiling", "fmm_get_phase_times",
                      "fmm_direct_sum", "fmm_morton_order"):
                getattr(L, f).restype = i32
            _lib = L
    return _lib


def _check(status, handle=None, what=""):
    if status != FMM_OK:
        msg = lib().fmm_last_error(handle).decode() if handle is not None else ""
        base = lib().fmm_status_string(status).decode()
        raise FMMError(status, "%s: %s%s" % (what, base, (" -- " + msg) if msg else ""))


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _dev_f64(x, name, shape1=None):
    if not (isinstance(x, torch.Tensor) and x.is_cuda and x.dtype == torch.float64):
        raise TypeError("%s must be a CUDA float64 tensor" % name)
    if not x.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if shape1 is not None and (x.dim() != 2 or x.shape[1] != shape1):
        raise ValueError("%s must have shape (n, %d)" % (name, shape1))
    return x


def source_terms(s: int, s_hi: int = None) -> int:
    """Moments per particle of the orders s..s_hi (s_hi = s: one order)."""
    hi = s if s_hi is None else s_hi
    return sum((k + 1) * (k + 2) // 2 for k in range(s, hi + 1))


class FMMTree:
    """One system: fmm_create_tree / fmm_set_sources / fmm_evaluate."""

    def __init__(self, device=0, stream=None, max_leaf=64, precision="fp64", mem_budget_bytes=0):
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        self.stream = stream
        self.precision = precision
        h = C.c_void_p()
        st = lib().fmm_create_tree(C.byref(h), self.device.index or 0, _stream_ptr(stream),
                                   int(max_leaf), PRECISIONS[precision], int(mem_budget_bytes))
        if st != FMM_OK:
            raise FMMError(st, "create_tree: %s -- %s" % (lib().fmm_status_string(st).decode(),
                                                          lib().fmm_last_error(None).decode()))
        self._h = h
        self.n = 0
        self.s = None
        self._keep = None

    def set_sources(self, positions, moments, source_order: int):
        _dev_f64(positions, "positions", 3)
        if moments is not None:
            _dev_f64(moments, "moments", source_terms(source_order))
        n = positions.shape[0]
        st = lib().fmm_set_sources(self._h, _ptr(positions), _ptr(moments), n, int(source_order))
        _check(st, self._h, "set_sources")
        self.n, self.s, self.s_hi = n, source_order, source_order

    def set_sources_mixed(self, positions, moments, s_lo: int, s_hi: int):
        """Every particle carries the moments of the orders s_lo..s_hi (graded order)."""
        _dev_f64(positions, "positions", 3)
        _dev_f64(moments, "moments", source_terms(s_lo, s_hi))
        n = positions.shape[0]
        fn = lib().fmm_set_sources_mixed
        fn.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_int]
        fn.restype = C.c_int
        _check(fn(self._h, _ptr(positions), _ptr(moments), n, int(s_lo), int(s_hi)), self._h,
               "set_sources_mixed")
        self.n, self.s, self.s_hi = n, s_lo, s_hi

    def set_sources_batch(self, positions, moments, offsets, source_order: int):
        """A forest of independent systems; ``offsets`` is a host int sequence of count+1."""
        _dev_f64(positions, "positions", 3)
        _dev_f64(moments, "moments", source_terms(source_order))
        off = (C.c_int64 * len(offsets))(*[int(x) for x in offsets])
        fn = lib().fmm_set_sources_batch
        fn.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int64), C.c_int, C.c_int]
        fn.restype = C.c_int
        st = fn(self._h, _ptr(positions), _ptr(moments), off, len(offsets) - 1, int(source_order))
        _check(st, self._h, "set_sources_batch")
        self.n, self.s, self.s_hi = int(offsets[-1]), source_order, source_order

    def evaluate(self, p: int, theta: float, want_potential=True, want_field=True,
                 potential=None, field=None):
        """Returns (potential or None, field or None) as CUDA float64 tensors."""
        if want_potential and potential is None:
            potential = torch.empty(self.n, dtype=torch.float64, device=self.device)
        if want_field and field is None:
            field = torch.empty((self.n, 3), dtype=torch.float64, device=self.device)
        st = lib().fmm_evaluate(self._h, int(p), float(theta), int(bool(want_potential)),
                                int(bool(want_field)), _ptr(potential if want_potential else None),
                                _ptr(field if want_field else None))
        _check(st, self._h, "evaluate")
        return (potential if want_potential else None), (field if want_field else None)

    def evaluate_bh(self, p: int, theta: float, want_potential=True, want_field=True,
                    potential=None, field=None):
        """Multipolar Barnes-Hut of order p (FP64); returns like evaluate()."""
        if want_potential and potential is None:
            potential = torch.empty(self.n, dtype=torch.float64, device=self.device)
        if want_field and field is None:
            field = torch.empty((self.n, 3), dtype=torch.float64, device=self.device)
        fn = lib().fmm_evaluate_bh
        fn.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_int, C.c_void_p, C.c_void_p]
        fn.restype = C.c_int
        st = fn(self._h, int(p), float(theta), int(bool(want_potential)), int(bool(want_field)),
                _ptr(potential if want_potential else None), _ptr(field if want_field else None))
        _check(st, self._h, "evaluate_bh")
        return (potential if want_potential else None), (field if want_field else None)

    def update_moments(self, moments):
        """Replace the moments of the current tree (caller's order); keeps tree, lists, caches."""
        _dev_f64(moments, "moments", source_terms(self.s, getattr(self, "s_hi", self.s)))
        if moments.shape[0] != self.n:
            raise ValueError("moments must have %d rows" % self.n)
        fn = lib().fmm_update_moments
        fn.argtypes = [C.c_void_p, C.c_void_p]
        fn.restype = C.c_int
        _check(fn(self._h, _ptr(moments)), self._h, "update_moments")

    def evaluate_graph(self, p: int, theta: float, want_potential=True, want_field=True,
                       potential=None, field=None):
        """fmm_evaluate replayed as one CUDA graph launch while (p, theta, flags, outputs)
        stay the same.  Output tensors are allocated once per parameter set and reused."""
        key = (int(p), float(theta), bool(want_potential), bool(want_field))
        cache = getattr(self, "_graph_out", None)
        if potential is None and field is None and cache and cache[0] == key:
            potential, field = cache[1], cache[2]
        if want_potential and potential is None:
            potential = torch.empty(self.n, dtype=torch.float64, device=self.device)
        if want_field and field is None:
            field = torch.empty((self.n, 3), dtype=torch.float64, device=self.device)
        self._graph_out = (key, potential, field)
        fn = lib().fmm_evaluate_graph
        fn.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_int, C.c_void_p, C.c_void_p]
        fn.restype = C.c_int
        st = fn(self._h, int(p), float(theta), int(bool(want_potential)), int(bool(want_field)),
                _ptr(potential if want_potential else None), _ptr(field if want_field else None))
        _check(st, self._h, "evaluate_graph")
        return (potential if want_potential else None), (field if want_field else None)

    def autotune(self, p: int, theta: float, want_potential=True, want_field=True, reps=3):
        """Time the handle's kernel variants on its own workload; keep the fastest."""
        pot = torch.empty(self.n, dtype=torch.float64, device=self.device) if want_potential else None
        fld = torch.empty((self.n, 3), dtype=torch.float64, device=self.device) if want_field else None
        out = Tuning()
        fn = lib().fmm_autotune
        fn.argtypes = [C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                       C.c_int, C.POINTER(Tuning)]
        fn.restype = C.c_int
        st = fn(self._h, int(p), float(theta), int(bool(want_potential)), int(bool(want_field)),
                _ptr(pot), _ptr(fld), int(reps), C.byref(out))
        _check(st, self._h, "autotune")
        return {k: getattr(out, k) for k, _ in out._fields_}

    def set_tuning(self, p2p_variant: int = -1, m2l_tensor: int = -1, tc_chunk_rows: int = -1,
                   m2l_harmonic: int = -1, p2p_targets: int = -1, m2l_tiled: int = -1):
        """Applies a tuning without timing (-1 keeps the current setting)."""
        tu = Tuning()
        tu.p2p_variant, tu.m2l_tensor, tu.tc_chunk_rows = int(p2p_variant), int(m2l_tensor), int(tc_chunk_rows)
        tu.m2l_harmonic = int(m2l_harmonic)
        tu.p2p_targets = int(p2p_targets)
        tu.m2l_tiled = int(m2l_tiled)
        fn = lib().fmm_set_tuning
        fn.argtypes = [C.c_void_p, C.POINTER(Tuning)]
        fn.restype = C.c_int
        _check(fn(self._h, C.byref(tu)), self._h, "set_tuning")

    def info(self) -> dict:
        inf = TreeInfo()
        _check(lib().fmm_get_info(self._h, C.byref(inf)), self._h, "get_info")
        return inf.as_dict()

    def copy_array(self, name: str, width: int = None) -> torch.Tensor:
        """Host copy of an internal array (keys, perm, cells, lists, M, L)."""
        ident, dtype, cols = ARRAYS[name]
        if name in ("multipole", "local") and self.precision != "fp64":
            dtype = torch.float32          # scaled FP32 expansions
        need = C.c_size_t()
        inf = self.info()
        rows = {"keys": inf["n"], "perm": inf["n"], "m2l": inf["n_m2l"], "p2p": inf["n_p2p"]}.get(
            name, inf["ncells"])
        elem = torch.empty((), dtype=dtype).element_size()
        if cols == 0:
            cols = width if width else 1
        out = torch.empty((rows, cols) if cols > 1 else (rows,), dtype=dtype)
        st = lib().fmm_copy_array(self._h, ident, C.c_void_p(out.data_ptr()),
                                  out.numel() * elem, C.byref(need))
        _check(st, self._h, "copy_array(%s)" % name)
        return out

    def set_profiling(self, enable=True):
        _check(lib().fmm_set_profiling(self._h, int(bool(enable))), self._h, "set_profiling")

    def phase_times(self) -> dict:
        buf = (C.c_float * len(PHASES))()
        _check(lib().fmm_get_phase_times(self._h, buf), self._h, "get_phase_times")
        return {k: float(v) for k, v in zip(PHASES, buf)}

    def launch_count(self) -> int:
        return int(lib().fmm_launch_count(self._h))

    def destroy(self):
        h, self._h = getattr(self, "_h", None), None
        if h:
            lib().fmm_destroy(h)

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def create_tree(device=0, stream=None, max_leaf=64, precision="fp64", mem_budget_bytes=0):
    return FMMTree(device, stream, max_leaf, precision, mem_budget_bytes)


def direct_sum(positions, moments, source_order, targets=None, want_potential=True,
               want_field=True, stream=None, source_order_hi=None):
    """FP64 O(N^2) sum on the GPU at ``targets`` (int32 CUDA tensor or None); sources of
    the orders source_order..source_order_hi per particle when the latter is given."""
    _dev_f64(positions, "positions", 3)
    _dev_f64(moments, "moments", source_terms(source_order, source_order_hi))
    n = positions.shape[0]
    if targets is not None:
        if not (targets.is_cuda and targets.dtype == torch.int32):
            raise TypeError("targets must be a CUDA int32 tensor")
        nt = targets.shape[0]
    else:
        nt = n
    phi = torch.empty(nt, dtype=torch.float64, device=positions.device) if want_potential else None
    E = torch.empty((nt, 3), dtype=torch.float64, device=positions.device) if want_field else None
    if source_order_hi is None:
        st = lib().fmm_direct_sum(_stream_ptr(stream), _ptr(positions), _ptr(moments), n,
                                  int(source_order), _ptr(targets), nt, _ptr(phi), _ptr(E))
    else:
        fn = lib().fmm_direct_sum_mixed
        fn.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_int, C.c_void_p,
                       C.c_int64, C.c_void_p, C.c_void_p]
        fn.restype = C.c_int
        st = fn(_stream_ptr(stream), _ptr(positions), _ptr(moments), n, int(source_order),
                int(source_order_hi), _ptr(targets), nt, _ptr(phi), _ptr(E))
    _check(st, None, "direct_sum")
    return phi, E


def check_rsqrt(x, stream=None):
    """(library 1/sqrt(x), CUDA rsqrt(x)) for a CUDA float64 tensor x > 0."""
    fn = lib().fmm_check_rsqrt
    fn.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
    fn.restype = C.c_int
    own, ref = torch.empty_like(x), torch.empty_like(x)
    _check(fn(_stream_ptr(stream), _ptr(x), x.numel(), _ptr(own), _ptr(ref)), None, "check_rsqrt")
    return own, ref


def check_umma(A, B, kbn, a_tmem=False, passes=3):
    """Tensor-core self-check: D [128 x N] from CUDA float32 A [128 x 8 len(kbn)]
    and B [N x 8 len(kbn)]; K-block kb contributes to columns n < kbn[kb]."""
    fn = lib().fmm_check_umma
    fn.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int,
                   C.c_int]
    fn.restype = C.c_int
    for name, t in (("A", A), ("B", B)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32
                and t.is_contiguous() and t.dim() == 2):
            raise TypeError("%s must be a contiguous 2-D CUDA float32 tensor" % name)
    N = B.shape[0]
    kb = (C.c_int * len(kbn))(*[int(v) for v in kbn])
    D = torch.empty((128, N), dtype=torch.float32, device=A.device)
    _check(fn(_ptr(A), _ptr(B), _ptr(D), len(kbn), N, C.cast(kb, C.c_void_p), int(bool(a_tmem)),
              int(passes)), None, "check_umma")
    return D


def morton_order(positions, stream=None):
    """(keys uint64-as-int64 [n], perm int32 [n]) as CUDA tensors."""
    _dev_f64(positions, "positions", 3)
    n = positions.shape[0]
    keys = torch.empty(n, dtype=torch.int64, device=positions.device)
    perm = torch.empty(n, dtype=torch.int32, device=positions.device)
    st = lib().fmm_morton_order(_stream_ptr(stream), _ptr(positions), n, _ptr(keys), _ptr(perm))
    _check(st, None, "morton_order")
    return keys, perm


NOALLOC_MAX_POINTS = 1 << 20


def noalloc_entry():
    """The C entry point fmm_morton_order_noalloc with its argument types."""
    f = lib().fmm_morton_order_noalloc
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    return f


def morton_order_noalloc(positions, keys_out, perm_out, stream=None):
    """Morton order into caller-provided outputs with no device allocation
    (the library's fixed scratch array; see fmm_morton_order_noalloc)."""
    _dev_f64(positions, "positions", 3)
    n = positions.shape[0]
    st = noalloc_entry()(_stream_ptr(stream), _ptr(positions), n, _ptr(keys_out), _ptr(perm_out))
    _check(st, None, "morton_order_noalloc")
    return keys_out, perm_out


# ------------------------------------------------------------------ serving
class Request(C.Structure):
    _fields_ = [("positions", C.c_void_p), ("moments", C.c_void_p), ("n", C.c_int64),
                ("source_order", C.c_int), ("p", C.c_int), ("theta", C.c_double),
                ("max_leaf", C.c_int), ("want_potential", C.c_int), ("want_field", C.c_int),
                ("potential", C.c_void_p), ("field", C.c_void_p)]


class RequestResult(C.Structure):
    _fields_ = [("ticket", C.c_int64), ("status", C.c_int), ("slot", C.c_int),
                ("submit_s", C.c_double), ("start_s", C.c_double), ("end_s", C.c_double),
                ("device_bytes", C.c_int64), ("message", C.c_char * 128)]


class ServerStats(C.Structure):
    _fields_ = [("completed", C.c_int64), ("failed", C.c_int64), ("queued", C.c_int64),
                ("running", C.c_int64), ("device_bytes", C.c_int64),
                ("peak_device_bytes", C.c_int64), ("particles_done", C.c_int64),
                ("busy_span_s", C.c_double)]


def _server_fns():
    L = lib()
    vp = C.c_void_p
    L.fmm_server_create.argtypes = [C.POINTER(vp), C.c_int, C.c_int, C.c_int, C.c_size_t]
    L.fmm_server_submit.argtypes = [vp, C.POINTER(Request), C.POINTER(C.c_int64)]
    L.fmm_server_poll.argtypes = [vp, C.c_int64, C.POINTER(C.c_int)]
    L.fmm_server_wait.argtypes = [vp, C.c_int64, C.POINTER(RequestResult)]
    L.fmm_server_get_stats.argtypes = [vp, C.POINTER(ServerStats)]
    L.fmm_server_destroy.argtypes = [vp]
    for f in ("fmm_server_create", "fmm_server_submit", "fmm_server_poll", "fmm_server_wait",
              "fmm_server_get_stats", "fmm_server_destroy"):
        getattr(L, f).restype = C.c_int
    return L


class Server:
    """fmm_server_*: continuous batching of evaluation requests on one GPU.

    ``submit`` takes numpy arrays (kept alive here until ``wait``) and returns a
    ticket; ``wait`` returns (phi, E, result-dict)."""

    def __init__(self, device=0, slots=4, precision="fp64", mem_budget_bytes=0):
        import numpy as np  # noqa: F401
        L = _server_fns()
        h = C.c_void_p()
        st = L.fmm_server_create(C.byref(h), int(device), int(slots), PRECISIONS[precision],
                                 int(mem_budget_bytes))
        if st != FMM_OK:
            raise FMMError(st, "server_create: %s" % L.fmm_status_string(st).decode())
        self._h, self._L = h, L
        self._live = {}

    def submit(self, positions, moments, source_order, p, theta=0.5, max_leaf=64,
               want_potential=True, want_field=True):
        import numpy as np
        pos = np.ascontiguousarray(positions, dtype=np.float64)
        mom = np.ascontiguousarray(moments, dtype=np.float64)
        n = pos.shape[0]
        phi = np.empty(n) if want_potential else None
        E = np.empty((n, 3)) if want_field else None
        r = Request(pos.ctypes.data if n else None, mom.ctypes.data if n else None, n,
                    int(source_order), int(p), float(theta), int(max_leaf),
                    int(bool(want_potential)), int(bool(want_field)),
                    phi.ctypes.data if (phi is not None and n) else None,
                    E.ctypes.data if (E is not None and n) else None)
        t = C.c_int64()
        st = self._L.fmm_server_submit(self._h, C.byref(r), C.byref(t))
        if st != FMM_OK:
            raise FMMError(st, "server_submit: %s" % self._L.fmm_status_string(st).decode())
        self._live[t.value] = (pos, mom, phi, E)
        return t.value

    def done(self, ticket) -> bool:
        d = C.c_int()
        _check(self._L.fmm_server_poll(self._h, int(ticket), C.byref(d)), None, "server_poll")
        return bool(d.value)

    def wait(self, ticket):
        res = RequestResult()
        st = self._L.fmm_server_wait(self._h, int(ticket), C.byref(res))
        pos, mom, phi, E = self._live.pop(ticket)
        info = {"status": res.status, "slot": res.slot, "submit_s": res.submit_s,
                "start_s": res.start_s, "end_s": res.end_s, "device_bytes": res.device_bytes,
                "message": res.message.decode(errors="replace")}
        if st != FMM_OK:
            raise FMMError(st, "request %d: %s" % (ticket, info["message"]))
        return phi, E, info

    def stats(self) -> dict:
        s = ServerStats()
        _check(self._L.fmm_server_get_stats(self._h, C.byref(s)), None, "server_stats")
        return {k: getattr(s, k) for k, _ in s._fields_}

    def close(self):
        h, self._h = getattr(self, "_h", None), None
        if h:
            self._L.fmm_server_destroy(h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
