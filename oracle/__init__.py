"""CPU FP64 oracle for the Cartesian-Taylor FMM (Pepper & Fangohr, fmmgen).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The library path
never calls it, and it shares no code with the CUDA path.

This module is argument marshalling around ``fmm_oracle.c`` (plain C, FP64,
OpenMP over independent outputs) plus numpy views of its results.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fmm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE: no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            L.orc_ntot.argtypes = [C.c_int]
            L.orc_ntot.restype = C.c_int
            L.orc_index.argtypes = [C.c_int, C.c_int, C.c_int]
            L.orc_index.restype = C.c_int
            L.orc_multi_index.argtypes = [C.c_int] + [C.POINTER(C.c_int)] * 3
            L.orc_derivatives.argtypes = [C.c_double] * 3 + [C.c_int, _f64p]
            L.orc_n_multipole.argtypes = [C.c_int, C.c_int]
            L.orc_n_multipole.restype = C.c_int
            L.orc_n_local.argtypes = [C.c_int]
            L.orc_n_local.restype = C.c_int
            L.orc_p2m.argtypes = [C.c_int, C.c_int, _f64p, C.c_int64, _f64p, _f64p, _f64p]
            L.orc_m2m.argtypes = [C.c_int, C.c_int, _f64p, _f64p, _f64p, _f64p]
            L.orc_m2l.argtypes = [C.c_int, C.c_int, _f64p, _f64p, _f64p, _f64p]
            L.orc_l2l.argtypes = [C.c_int, _f64p, _f64p, _f64p, _f64p]
            L.orc_l2p.argtypes = [C.c_int, _f64p, _f64p, _f64p, _f64p, _f64p]
            L.orc_p2p_pair.argtypes = [C.c_int, _f64p, _f64p, _f64p, _f64p, _f64p]
            L.orc_direct.argtypes = [C.c_int, C.c_int64, _f64p, _f64p, C.c_int64, C.c_void_p,
                                     _f64p, _f64p]
            L.orc_tree_build.argtypes = [C.c_int64, _f64p, C.c_int]
            L.orc_tree_build.restype = C.c_void_p
            L.orc_tree_lists.argtypes = [C.c_void_p, C.c_double]
            L.orc_tree_free.argtypes = [C.c_void_p]
            L.orc_tree_sizes.argtypes = [C.c_void_p, _i64p]
            L.orc_tree_box.argtypes = [C.c_void_p, _f64p]
            L.orc_tree_particles.argtypes = [C.c_void_p, _u64p, _i64p]
            L.orc_tree_cells.argtypes = [C.c_void_p, _i32p, _i64p, _i64p, _i64p, _i64p, _i64p,
                                         _i32p, _f64p, _f64p]
            L.orc_tree_get_lists.argtypes = [C.c_void_p, _i64p, _i64p]
            L.orc_fmm.argtypes = [C.c_void_p, _f64p, C.c_int, C.c_int, _f64p, C.c_int64,
                                  C.c_void_p, _f64p, _f64p]
            L.orc_fmm.restype = C.c_int
            L.orc_m2p.argtypes = [C.c_int, C.c_int, _f64p, _f64p, _f64p, _f64p, _f64p]
            L.orc_p2m_orders.argtypes = [C.c_int, C.c_int, C.c_int, _f64p, C.c_int64, _f64p, _f64p,
                                         _f64p]
            L.orc_p2p_pair_orders.argtypes = [C.c_int, C.c_int, _f64p, _f64p, _f64p, _f64p, _f64p]
            L.orc_direct_orders.argtypes = [C.c_int, C.c_int, C.c_int64, _f64p, _f64p, C.c_int64,
                                            C.c_void_p, _f64p, _f64p]
            L.orc_fmm_orders.argtypes = [C.c_void_p, _f64p, C.c_int, C.c_int, C.c_int, _f64p,
                                         C.c_int64, C.c_void_p, _f64p, _f64p]
            L.orc_fmm_orders.restype = C.c_int
            L.orc_bh_orders.argtypes = [C.c_void_p, _f64p, C.c_int, C.c_int, C.c_int, _f64p,
                                        C.c_double, C.c_int64, C.c_void_p, _f64p, _f64p]
            L.orc_bh_orders.restype = C.c_int
            L.orc_bh.argtypes = [C.c_void_p, _f64p, C.c_int, C.c_int, _f64p, C.c_double,
                                 C.c_int64, C.c_void_p, _f64p, _f64p]
            L.orc_bh.restype = C.c_int
            L.orc_num_threads.restype = C.c_int
            _lib = L
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ------------------------------------------------------------ index helpers
def ntot(p: int) -> int:
    return lib().orc_ntot(p)


def index(nx: int, ny: int, nz: int) -> int:
    return lib().orc_index(nx, ny, nz)


def multi_index(idx: int):
    a, b, c = C.c_int(), C.c_int(), C.c_int()
    lib().orc_multi_index(idx, C.byref(a), C.byref(b), C.byref(c))
    return a.value, b.value, c.value


def n_multipole(s: int, p: int) -> int:
    return lib().orc_n_multipole(s, p)


def n_local(p: int) -> int:
    return lib().orc_n_local(p)


def num_threads() -> int:
    return lib().orc_num_threads()


# ---------------------------------------------------------------- operators
def derivatives(R, order: int) -> np.ndarray:
    D = np.zeros(ntot(order))
    lib().orc_derivatives(float(R[0]), float(R[1]), float(R[2]), order, D)
    return D


def n_source(s, s_hi=None) -> int:
    """Moments per particle of the source orders s..s_hi (all shells, graded order)."""
    return ntot(s if s_hi is None else s_hi) - ntot(s - 1)


def p2m(s, p, centre, pos, S, s_hi=None):
    pos, S = _f64(pos).reshape(-1, 3), _f64(S)
    M = np.zeros(n_multipole(s, p))
    lib().orc_p2m_orders(s, s if s_hi is None else s_hi, p, _f64(centre), len(pos), pos.ravel(),
                         S.ravel(), M)
    return M


def m2m(s, p, zc, zp, Mc, Mp=None):
    Mp = np.zeros(n_multipole(s, p)) if Mp is None else _f64(Mp).copy()
    lib().orc_m2m(s, p, _f64(zc), _f64(zp), _f64(Mc), Mp)
    return Mp


def m2l(s, p, zt, zs, Ms, Lt=None):
    Lt = np.zeros(n_local(p)) if Lt is None else _f64(Lt).copy()
    lib().orc_m2l(s, p, _f64(zt), _f64(zs), _f64(Ms), Lt)
    return Lt


def l2l(p, zp, zc, Lp, Lc=None):
    Lc = np.zeros(n_local(p)) if Lc is None else _f64(Lc).copy()
    lib().orc_l2l(p, _f64(zp), _f64(zc), _f64(Lp), Lc)
    return Lc


def l2p(p, z, L, x):
    phi, g = np.zeros(1), np.zeros(3)
    lib().orc_l2p(p, _f64(z), _f64(L), _f64(x), phi, g)
    return phi[0], g


def m2p(s, p, z, M, x):
    """Multipole of order p (s <= |m| <= p) at centre z evaluated at x: (phi, grad phi)."""
    f, g = np.zeros(1), np.zeros(3)
    lib().orc_m2p(s, p, _f64(z), _f64(M), _f64(x), f, g)
    return float(f[0]), g


def p2p_pair(s, xt, xs, S, s_hi=None):
    phi, g = np.zeros(1), np.zeros(3)
    lib().orc_p2p_pair_orders(s, s if s_hi is None else s_hi, _f64(xt), _f64(xs), _f64(S), phi, g)
    return phi[0], g


def direct(pos, S, s, targets=None, s_hi=None):
    """Compensated O(N^2) sum; returns (phi[nt], E[nt,3]) at ``targets``.  Sources
    of the orders s..s_hi (s_hi = s: a single order)."""
    pos, S = _f64(pos).reshape(-1, 3), _f64(S)
    n = len(pos)
    if targets is None:
        nt, tp = n, None
    else:
        targets = np.ascontiguousarray(targets, dtype=np.int64)
        nt, tp = len(targets), targets.ctypes.data
    phi, E = np.zeros(nt), np.zeros((nt, 3))
    if nt:
        lib().orc_direct_orders(s, s if s_hi is None else s_hi, n, pos.ravel(), S.ravel(), nt, tp,
                                phi, E.reshape(-1))
    return phi, E


# --------------------------------------------------------------------- tree
class Tree:
    """Octree + dual-tree interaction lists built by the oracle."""

    def __init__(self, pos, ncrit: int):
        self.pos = _f64(pos).reshape(-1, 3)
        self.ncrit = ncrit
        self._h = lib().orc_tree_build(len(self.pos), self.pos.ravel(), ncrit)
        sz = np.zeros(5, dtype=np.int64)
        lib().orc_tree_sizes(self._h, sz)
        self.n, self.ncells, self.nlevels = int(sz[0]), int(sz[1]), int(sz[2])
        box = np.zeros(4)
        lib().orc_tree_box(self._h, box)
        self.lo, self.side = box[:3].copy(), float(box[3])
        self.keys = np.zeros(self.n, dtype=np.uint64)
        self.perm = np.zeros(self.n, dtype=np.int64)
        if self.n:
            lib().orc_tree_particles(self._h, self.keys, self.perm)
        nc = self.ncells
        self.level = np.zeros(nc, dtype=np.int32)
        self.ci = np.zeros((nc, 3), dtype=np.int64)
        self.begin = np.zeros(nc, dtype=np.int64)
        self.end = np.zeros(nc, dtype=np.int64)
        self.parent = np.zeros(nc, dtype=np.int64)
        self.child_first = np.zeros(nc, dtype=np.int64)
        self.nchild = np.zeros(nc, dtype=np.int32)
        self.centre = np.zeros((nc, 3))
        self.halfw = np.zeros(nc)
        if nc:
            lib().orc_tree_cells(self._h, self.level, self.ci.reshape(-1), self.begin, self.end,
                                 self.parent, self.child_first, self.nchild,
                                 self.centre.reshape(-1), self.halfw)
        self.theta = None
        self.m2l = np.zeros((0, 2), dtype=np.int64)
        self.p2p = np.zeros((0, 2), dtype=np.int64)

    def lists(self, theta: float):
        lib().orc_tree_lists(self._h, float(theta))
        sz = np.zeros(5, dtype=np.int64)
        lib().orc_tree_sizes(self._h, sz)
        self.m2l = np.zeros((int(sz[3]), 2), dtype=np.int64)
        self.p2p = np.zeros((int(sz[4]), 2), dtype=np.int64)
        lib().orc_tree_get_lists(self._h, self.m2l.reshape(-1), self.p2p.reshape(-1))
        self.theta = theta
        return self.m2l, self.p2p

    def fmm(self, S, s: int, p: int, targets=None, s_hi=None):
        """FP64 FMM on this tree; (phi, E) at ``targets`` (original indices).  Sources of
        the orders s..s_hi (the expansion's lowest order is s)."""
        if self.theta is None:
            raise RuntimeError("call lists(theta) first")
        S = _f64(S)
        if targets is None:
            nt, tp = self.n, None
        else:
            targets = np.ascontiguousarray(targets, dtype=np.int64)
            nt, tp = len(targets), targets.ctypes.data
        phi, E = np.zeros(nt), np.zeros((nt, 3))
        rc = lib().orc_fmm_orders(self._h, self.pos.ravel(), s, s if s_hi is None else s_hi, p,
                                  S.ravel(), nt, tp, phi, E.reshape(-1))
        if rc != 0:
            raise ValueError("oracle FMM rejected s=%d p=%d" % (s, p))
        return phi, E

    def bh(self, S, s: int, p: int, theta: float, targets=None, s_hi=None):
        """FP64 multipolar Barnes-Hut on this tree (order p, opening angle theta):
        (phi, E) at ``targets`` (original indices)."""
        S = _f64(S)
        if targets is None:
            nt, tp = self.n, None
        else:
            targets = np.ascontiguousarray(targets, dtype=np.int64)
            nt, tp = len(targets), targets.ctypes.data
        phi, E = np.zeros(nt), np.zeros((nt, 3))
        rc = lib().orc_bh_orders(self._h, self.pos.ravel(), s, s if s_hi is None else s_hi, p,
                                 S.ravel(), float(theta), nt, tp, phi, E.reshape(-1))
        if rc != 0:
            raise ValueError("oracle BH rejected s=%d p=%d theta=%g" % (s, p, theta))
        return phi, E

    def __del__(self):
        h, self._h = getattr(self, "_h", None), None
        if h and _lib is not None:
            _lib.orc_tree_free(h)


def bh(pos, S, s, p, theta, ncrit, targets=None, s_hi=None):
    return Tree(pos, ncrit).bh(S, s, p, theta, targets, s_hi)


def fmm(pos, S, s, p, theta, ncrit, targets=None, s_hi=None):
    """Convenience: build the oracle tree and lists, then evaluate."""
    t = Tree(pos, ncrit)
    t.lists(theta)
    return t.fmm(S, s, p, targets, s_hi)
