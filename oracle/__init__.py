"""Python access to the plain-C FP64 oracle (``hg_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by ``__graft_entry__.smoke``
and by the CPU-baseline leg of ``bench.py``.  The product library never
imports or calls anything here.

The shared object is compiled on first use (or by ``build()``) with
``gcc -O2 -ffp-contract=off`` so that every multiply and add is rounded on its
own, as the arithmetic contract in ``hg_oracle.c`` requires.
"""
from __future__ import annotations

import concurrent.futures as _cf
import ctypes as C
import dataclasses
import math
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libhg_oracle.so")
_lock = threading.Lock()
_lib = None

RAY_STEPLIMIT = 1
RAY_LOST = 2
RAY_BADINPUT = 4
RAY_OVERFLOW = 8


def build(force: bool = False) -> str:
    """Compile the oracle library (plain C, FP64, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class _Model(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_table", C.c_int32), ("p", C.c_double * 8),
                ("table", C.POINTER(C.c_double)), ("m_tot", C.c_double),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3)]


class _Params(C.Structure):
    _fields_ = [("kind", C.c_int32), ("use_delta", C.c_int32), ("use_tau", C.c_int32), ("use_q", C.c_int32),
                ("delta_max", C.c_double), ("tau_max", C.c_double), ("q_max", C.c_double),
                ("kappa", C.c_double), ("max_level", C.c_int32), ("n_ran", C.c_int32),
                ("seed", C.c_uint64), ("max_nodes", C.c_int64), ("split_axis", C.c_int32),
                ("split_plane", C.c_int32)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)
_I32 = C.POINTER(C.c_int32)


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        sig = {
            "or_rho_true_batch": (None, [C.POINTER(_Model), C.c_int64, _D, _D]),
            "or_build": (C.c_int, [C.POINTER(_Model), C.POINTER(_Params), C.POINTER(_P)]),
            "or_tree_wrap": (C.c_int, [C.c_int32, C.c_int64, _D, _D, _I32, _I32, C.c_int64, _D, C.POINTER(_P)]),
            "or_tree_free": (None, [_P]),
            "or_tree_n_nodes": (C.c_int64, [_P]),
            "or_tree_n_leaves": (C.c_int64, [_P]),
            "or_tree_export": (None, [_P, _I32, _I64, _I32, _I32, _D, _D, _D, _D, _D, _D, _D, _I64]),
            "or_node_stats": (None, [C.POINTER(_Model), C.POINTER(_Params), _I32, _I64, _D]),
            "or_locate_batch": (None, [_P, C.c_int64, _D, _D, _I64]),
            "or_brute_locate_batch": (None, [_P, C.c_int64, _D, _D, _I64, _I64]),
            "or_trace_batch": (C.c_int32, [_P, C.c_int64, _D, _D, _D, C.c_double, C.c_int64, _D, _I64, _I32,
                                           _I64, _I32, _D]),
            "or_interact_batch": (C.c_int32, [_P, C.c_int64, _D, _D, _D, C.c_double, _D, C.c_int64, _I64, _D,
                                              _I64, _I32]),
            "or_brute_sequence": (C.c_int64, [_P, _D, _D, C.c_double, C.c_double, _I32, _D, _D, C.c_int64]),
            "or_quad_poly": (C.c_double, [_D, C.c_int, C.c_double, C.c_double, C.c_int]),
            "or_tau_true_batch": (None, [C.POINTER(_Model), C.c_int64, _D, _D, _D, C.c_double, C.c_double, _D]),
            "or_sample_density": (None, [_P, C.c_int64, _D, _I64, _D]),
            "or_splitmix_output": (C.c_uint64, [C.c_uint64, C.c_uint64]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _ptr(a: Optional[np.ndarray], ctype):
    if a is None:
        return C.cast(None, C.POINTER(ctype))
    return a.ctypes.data_as(C.POINTER(ctype))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class ModelRef:
    """Keeps a model's ctypes record and the arrays it points to alive."""

    def __init__(self, model):
        self.table = _f64(model.table.reshape(-1)) if model.table is not None and model.table.size else \
            np.zeros(1, np.float64)
        m = _Model()
        m.kind = int(model.kind)
        m.n_table = int(model.table.shape[0]) if model.table is not None else 0
        for j, v in enumerate(np.asarray(model.params, np.float64)[:8]):
            m.p[j] = float(v)
        m.table = _ptr(self.table, C.c_double)
        m.m_tot = float(model.m_tot)
        for a in range(3):
            m.lo[a] = float(model.domain_lo[a])
            m.hi[a] = float(model.domain_hi[a])
        self.c = m


def _params(bp) -> _Params:
    p = _Params()
    p.kind = int(bp.kind)
    p.use_delta = int(bool(bp.use_delta))
    p.use_tau = int(bool(bp.use_tau))
    p.use_q = int(bool(bp.use_q))
    p.delta_max = float(bp.delta_max)
    p.tau_max = float(bp.tau_max)
    p.q_max = float(bp.q_max)
    p.kappa = float(bp.kappa)
    p.max_level = int(bp.max_level)
    p.n_ran = int(bp.n_ran)
    p.seed = int(bp.seed) & ((1 << 64) - 1)
    p.max_nodes = int(getattr(bp, "max_nodes", 0) or 0)
    p.split_axis = int(getattr(bp, "split_axis", 0) or 0)
    p.split_plane = int(getattr(bp, "split_plane", 0) or 0)
    return p


def splitmix_output(key: int, j: int) -> int:
    return int(_load().or_splitmix_output(C.c_uint64(key), C.c_uint64(j)))


def rho_true(model, pts: np.ndarray) -> np.ndarray:
    lib = _load()
    pts = _f64(pts).reshape(-1, 3)
    out = np.empty(pts.shape[0], np.float64)
    mr = ModelRef(model)
    lib.or_rho_true_batch(C.byref(mr.c), pts.shape[0], _ptr(pts, C.c_double), _ptr(out, C.c_double))
    return out


def node_stats(model, bp, lvl, idx) -> np.ndarray:
    """[subdivide, rho_mean, mass, delta, tau_node, q] of the node with per-axis levels/positions."""
    lib = _load()
    l = np.ascontiguousarray(lvl, np.int32)
    i = np.ascontiguousarray(idx, np.int64)
    out = np.empty(6, np.float64)
    mr = ModelRef(model)
    p = _params(bp)
    lib.or_node_stats(C.byref(mr.c), C.byref(p), _ptr(l, C.c_int32), _ptr(i, C.c_int64), _ptr(out, C.c_double))
    return out


@dataclass
class Tree:
    """The oracle's node list (arrays copied out of C) plus its live C handle."""

    kind: int
    lvl: np.ndarray       # [n,3]
    idx: np.ndarray       # [n,3]
    child: np.ndarray     # [n]
    leaf: np.ndarray      # [n]
    lo: np.ndarray        # [n,3]
    hi: np.ndarray        # [n,3]
    rho: np.ndarray       # [n]
    mass: np.ndarray      # [n]
    delta: np.ndarray
    taun: np.ndarray
    q: np.ndarray
    leaf_node: np.ndarray  # [n_leaves]
    handle: C.c_void_p

    @property
    def n_nodes(self) -> int:
        return int(self.child.shape[0])

    @property
    def n_leaves(self) -> int:
        return int(self.leaf_node.shape[0])

    @property
    def leaf_lo(self):
        return self.lo[self.leaf_node]

    @property
    def leaf_hi(self):
        return self.hi[self.leaf_node]

    @property
    def leaf_rho(self):
        return self.rho[self.leaf_node]

    def __del__(self):
        try:
            if self.handle:
                _load().or_tree_free(self.handle)
                self.handle = None
        except Exception:
            pass


def _export(h, kind) -> Tree:
    lib = _load()
    n = int(lib.or_tree_n_nodes(h))
    nl = int(lib.or_tree_n_leaves(h))
    lvl = np.empty((n, 3), np.int32)
    idx = np.empty((n, 3), np.int64)
    child = np.empty(n, np.int32)
    leaf = np.empty(n, np.int32)
    lo = np.empty((n, 3), np.float64)
    hi = np.empty((n, 3), np.float64)
    rho = np.empty(n, np.float64)
    mass = np.empty(n, np.float64)
    delta = np.empty(n, np.float64)
    taun = np.empty(n, np.float64)
    q = np.empty(n, np.float64)
    ln = np.empty(nl, np.int64)
    lib.or_tree_export(h, _ptr(lvl, C.c_int32), _ptr(idx, C.c_int64), _ptr(child, C.c_int32),
                       _ptr(leaf, C.c_int32), _ptr(lo, C.c_double), _ptr(hi, C.c_double), _ptr(rho, C.c_double),
                       _ptr(mass, C.c_double), _ptr(delta, C.c_double), _ptr(taun, C.c_double),
                       _ptr(q, C.c_double), _ptr(ln, C.c_int64))
    return Tree(kind, lvl, idx, child, leaf, lo, hi, rho, mass, delta, taun, q, ln, h)


def build_tree(model, bp, max_nodes: int = 0) -> Tree:
    """Node-list construction (Sect. 2.2, 4.1, 4.2) in the oracle."""
    lib = _load()
    mr = ModelRef(model)
    p = _params(bp)
    p.max_nodes = int(max_nodes)
    h = _P()
    rc = lib.or_build(C.byref(mr.c), C.byref(p), C.byref(h))
    if rc != 0:
        raise RuntimeError(f"oracle build failed ({rc})")
    return _export(h, int(bp.kind))


def tau_max_recipe(model, bp, fraction: float = 0.9) -> float:
    """The tau_max recipe of Sect. 4.1 in the oracle: build with the mass criterion only, sort the
    leaves' optical depths (Eq. 2) ascending, take the one at 0-based position floor(fraction * N)."""
    b = dataclasses.replace(bp, use_tau=False, use_q=False)
    t = build_tree(model, b)
    taus = np.sort(t.taun[t.child < 0])
    n = taus.shape[0]
    return float(taus[min(int(math.floor(fraction * n)), n - 1)])


def wrap_tree(kind: int, node_lo, node_hi, child, leaf, leaf_rho) -> Tree:
    """Let the oracle trace an externally built tree (node boxes [n,3], links, leaf ids, densities)."""
    lib = _load()
    lo = _f64(node_lo).reshape(-1, 3)
    hi = _f64(node_hi).reshape(-1, 3)
    ch = np.ascontiguousarray(child, np.int32)
    lf = np.ascontiguousarray(leaf, np.int32)
    rho = _f64(leaf_rho)
    h = _P()
    rc = lib.or_tree_wrap(int(kind), lo.shape[0], _ptr(lo, C.c_double), _ptr(hi, C.c_double),
                          _ptr(ch, C.c_int32), _ptr(lf, C.c_int32), rho.shape[0], _ptr(rho, C.c_double),
                          C.byref(h))
    if rc != 0:
        raise RuntimeError(f"oracle wrap failed ({rc})")
    return _export(h, int(kind))


def locate(tree: Tree, p, k=None) -> np.ndarray:
    lib = _load()
    p = _f64(p).reshape(-1, 3)
    k = np.zeros_like(p) if k is None else _f64(k).reshape(-1, 3)
    out = np.empty(p.shape[0], np.int64)
    lib.or_locate_batch(tree.handle, p.shape[0], _ptr(p, C.c_double), _ptr(k, C.c_double), _ptr(out, C.c_int64))
    return out


def brute_locate(tree: Tree, p, k=None):
    lib = _load()
    p = _f64(p).reshape(-1, 3)
    k = np.zeros_like(p) if k is None else _f64(k).reshape(-1, 3)
    out = np.empty(p.shape[0], np.int64)
    hits = np.empty(p.shape[0], np.int64)
    lib.or_brute_locate_batch(tree.handle, p.shape[0], _ptr(p, C.c_double), _ptr(k, C.c_double),
                              _ptr(out, C.c_int64), _ptr(hits, C.c_int64))
    return out, hits


def default_max_steps(n_leaves: int) -> int:
    return 4 * int(n_leaves) + 64


def _threads(threads: Optional[int]) -> int:
    if threads is None or threads <= 0:
        return max(1, os.cpu_count() or 1)
    return int(threads)


def interact(tree: Tree, o, k, tau_int, smax=None, kappa: float = 1.0, max_steps: Optional[int] = None,
             threads: Optional[int] = None) -> dict:
    """Interaction-point search in the oracle: for each path, the leaf in which the accumulated
    optical depth first reaches tau_int (-1 when the path ends first), the path parameter t of the
    interaction inside it (or of the path end), the recorded segments walked, and the status."""
    lib = _load()
    o = _f64(o).reshape(-1, 3)
    k = _f64(k).reshape(-1, 3)
    ti = _f64(tau_int).reshape(-1)
    n = o.shape[0]
    sm = None if smax is None else _f64(smax).reshape(-1)
    ms = default_max_steps(tree.n_leaves) if max_steps is None else int(max_steps)
    cell = np.empty(n, np.int64)
    t = np.empty(n, np.float64)
    nc = np.empty(n, np.int64)
    st = np.empty(n, np.int32)
    nt = min(_threads(threads), max(1, n // 256))
    chunks = np.linspace(0, n, nt + 1).astype(np.int64)

    def run(c):
        a, b = int(chunks[c]), int(chunks[c + 1])
        if b <= a:
            return
        lib.or_interact_batch(tree.handle, b - a, _ptr(o[a:], C.c_double), _ptr(k[a:], C.c_double),
                              _ptr(None if sm is None else sm[a:], C.c_double), float(kappa),
                              _ptr(ti[a:], C.c_double), ms, _ptr(cell[a:], C.c_int64), _ptr(t[a:], C.c_double),
                              _ptr(nc[a:], C.c_int64), _ptr(st[a:], C.c_int32))

    if nt == 1:
        run(0)
    else:
        with _cf.ThreadPoolExecutor(nt) as ex:
            list(ex.map(run, range(nt)))
    return dict(cell=cell, t=t, ncross=nc, status=st)


def trace(tree: Tree, o, k, smax=None, kappa: float = 1.0, emit: bool = False, max_steps: Optional[int] = None,
          threads: Optional[int] = None) -> dict:
    """Path calculation in the oracle (top-down relocation after every step).

    Returns tau, ncross, status and, with ``emit``, the CSR arrays
    seg_off [n+1], seg_cell, seg_ds.  Rays are split across ``threads``
    host threads (the C routine releases the GIL).
    """
    lib = _load()
    o = _f64(o).reshape(-1, 3)
    k = _f64(k).reshape(-1, 3)
    n = o.shape[0]
    sm = None if smax is None else _f64(smax).reshape(-1)
    ms = default_max_steps(tree.n_leaves) if max_steps is None else int(max_steps)
    tau = np.empty(n, np.float64)
    nc = np.empty(n, np.int64)
    st = np.empty(n, np.int32)
    nt = min(_threads(threads), max(1, n // 256))
    chunks = np.linspace(0, n, nt + 1).astype(np.int64)

    def run(c, seg_off=None, seg_cell=None, seg_ds=None):
        a, b = int(chunks[c]), int(chunks[c + 1])
        if b <= a:
            return
        so = None if seg_off is None else seg_off[a:b + 1]
        lib.or_trace_batch(tree.handle, b - a, _ptr(o[a:], C.c_double), _ptr(k[a:], C.c_double),
                           _ptr(None if sm is None else sm[a:], C.c_double), float(kappa), ms,
                           _ptr(tau[a:], C.c_double), _ptr(nc[a:], C.c_int64), _ptr(st[a:], C.c_int32),
                           _ptr(so, C.c_int64), _ptr(seg_cell, C.c_int32), _ptr(seg_ds, C.c_double))

    def par(fn, *args):
        if nt == 1:
            fn(0, *args)
            return
        with _cf.ThreadPoolExecutor(nt) as ex:
            list(ex.map(lambda c: fn(c, *args), range(nt)))

    par(run)
    out = dict(tau=tau, ncross=nc, status=st)
    if emit:
        seg_off = np.zeros(n + 1, np.int64)
        np.cumsum(nc, out=seg_off[1:])
        S = int(seg_off[-1])
        seg_cell = np.empty(max(S, 1), np.int32)
        seg_ds = np.empty(max(S, 1), np.float64)
        par(run, seg_off, seg_cell, seg_ds)
        out.update(seg_off=seg_off, seg_cell=seg_cell[:S], seg_ds=seg_ds[:S])
    return out


def brute_sequence(tree: Tree, o, k, t0: float, t1: float, cap: int = 1 << 16):
    lib = _load()
    o = _f64(o).reshape(3)
    k = _f64(k).reshape(3)
    cells = np.empty(cap, np.int32)
    tin = np.empty(cap, np.float64)
    ds = np.empty(cap, np.float64)
    n = lib.or_brute_sequence(tree.handle, _ptr(o, C.c_double), _ptr(k, C.c_double), float(t0), float(t1),
                              _ptr(cells, C.c_int32), _ptr(tin, C.c_double), _ptr(ds, C.c_double), cap)
    if n < 0:
        raise RuntimeError("brute_sequence capacity exceeded")
    return cells[:n].copy(), tin[:n].copy(), ds[:n].copy()


def quad_poly(coeffs, a: float, b: float, adaptive: bool = True) -> float:
    c = _f64(coeffs)
    return float(_load().or_quad_poly(_ptr(c, C.c_double), c.shape[0], float(a), float(b), int(adaptive)))


def tau_true(model, o, k, L, kappa: float = 1.0, rtol: float = 1e-11, threads: Optional[int] = None):
    """kappa * integral of rho_t along each path (adaptive Gauss-Kronrod with breakpoints)."""
    lib = _load()
    o = _f64(o).reshape(-1, 3)
    k = _f64(k).reshape(-1, 3)
    L = _f64(L).reshape(-1)
    n = o.shape[0]
    out = np.empty(n, np.float64)
    mr = ModelRef(model)
    nt = min(_threads(threads), max(1, n // 64))
    chunks = np.linspace(0, n, nt + 1).astype(np.int64)

    def run(c):
        a, b = int(chunks[c]), int(chunks[c + 1])
        if b > a:
            lib.or_tau_true_batch(C.byref(mr.c), b - a, _ptr(o[a:], C.c_double), _ptr(k[a:], C.c_double),
                                  _ptr(L[a:], C.c_double), float(kappa), float(rtol), _ptr(out[a:], C.c_double))

    if nt == 1:
        run(0)
    else:
        with _cf.ThreadPoolExecutor(nt) as ex:
            list(ex.map(run, range(nt)))
    return out


def sample_density(tree: Tree, pts):
    lib = _load()
    pts = _f64(pts).reshape(-1, 3)
    cell = np.empty(pts.shape[0], np.int64)
    rho = np.empty(pts.shape[0], np.float64)
    lib.or_sample_density(tree.handle, pts.shape[0], _ptr(pts, C.c_double), _ptr(cell, C.c_int64),
                          _ptr(rho, C.c_double))
    return cell, rho


def population_std(x) -> float:
    """Two-pass population standard deviation (the Delta-rho / Delta-tau statistic, Sect. 3.2)."""
    x = np.asarray(x, np.float64)
    if x.size == 0:
        return 0.0
    mu = x.sum() / x.size
    return float(np.sqrt(((x - mu) ** 2).sum() / x.size))


def adjoint(tree_n_leaves: int, seg_off, seg_cell, seg_ds, w, kappa: float = 1.0) -> np.ndarray:
    """d(sum_r w_r tau_r)/d(rho_c) = kappa * sum over segments in cell c of w_r ds, in FP64."""
    seg_off = np.asarray(seg_off, np.int64)
    counts = np.diff(seg_off)
    wr = np.repeat(np.asarray(w, np.float64), counts)
    g = np.zeros(tree_n_leaves, np.float64)
    np.add.at(g, np.asarray(seg_cell, np.int64), kappa * wr * np.asarray(seg_ds, np.float64))
    return g
