"""GB300 path calculation through octree and k-d tree dust grids.

A thin ctypes binding over the C ABI in ``include/hgrt.h`` (library
``_build/libhgrt.so``).  Functions keep the C names without the ``hg_``
prefix; they only marshal arguments: every step of the path (location,
exit-wall tests, neighbor search, sums, emission, adjoint, metrics) runs in
the library's CUDA kernels.  Device arrays are ``torch`` CUDA tensors and
every call runs on the current torch stream.  Importing the package fails
if the library has not been built (``build_lib.build()``) -- there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhgrt.so")

OCTREE = 0
KDTREE = 1
FP64 = 0
FP32K = 1
RAY_STEPLIMIT = 1
RAY_LOST = 2
RAY_BADINPUT = 4
RAY_OVERFLOW = 8
NOALLOC_MAX_RAYS = 262144  # HG_NOALLOC_MAX_RAYS

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"libhgrt.so not found at {LIB_PATH}; build it with "
        "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
_lib = C.CDLL(LIB_PATH)


class HgError(RuntimeError):
    pass


# ----------------------------------------------------------------------------- C structures (mirror hgrt.h)

class _Model(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_table", C.c_int32), ("p", C.c_double * 8),
                ("table", C.POINTER(C.c_double)), ("m_tot", C.c_double),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3)]


class _BuildParams(C.Structure):
    _fields_ = [("kind", C.c_int32), ("use_delta", C.c_int32), ("use_tau", C.c_int32), ("use_q", C.c_int32),
                ("delta_max", C.c_double), ("tau_max", C.c_double), ("q_max", C.c_double),
                ("kappa", C.c_double), ("max_level", C.c_int32), ("n_ran", C.c_int32),
                ("seed", C.c_uint64), ("max_nodes", C.c_int64), ("split_axis", C.c_int32),
                ("split_plane", C.c_int32)]


class _Desc(C.Structure):
    _fields_ = [("kind", C.c_int32), ("reserved", C.c_int32), ("n_nodes", C.c_int64), ("n_leaves", C.c_int64),
                ("node_lo", C.POINTER(C.c_double)), ("node_hi", C.POINTER(C.c_double)),
                ("child_first", C.POINTER(C.c_int32)), ("node_leaf", C.POINTER(C.c_int32)),
                ("leaf_rho", C.POINTER(C.c_double)), ("nbr_off", C.POINTER(C.c_int64)),
                ("nbr_id", C.POINTER(C.c_int32))]


class _HostNodes(C.Structure):
    _fields_ = [("level", C.POINTER(C.c_int32)), ("index", C.POINTER(C.c_int64)),
                ("mass", C.POINTER(C.c_double)), ("delta", C.POINTER(C.c_double)),
                ("tau", C.POINTER(C.c_double)), ("q", C.POINTER(C.c_double))]


class _GridInfo(C.Structure):
    _fields_ = [("kind", C.c_int32), ("max_depth", C.c_int32), ("n_nodes", C.c_int64), ("n_leaves", C.c_int64),
                ("n_tail", C.c_int64), ("device_bytes", C.c_int64), ("long_walls", C.c_int64),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3), ("nav", C.c_int32), ("reserved", C.c_int32)]


NAV_NEIGHBOR_LISTS = 0  # HG_NAV_NEIGHBOR_LISTS
NAV_ROPES = 1           # HG_NAV_ROPES


class TraceOpts(C.Structure):
    """hg_trace_opts: precision, threads per block, shared-memory tree nodes, schedule, register budget,
    path splitting, step limit."""
    _fields_ = [("precision", C.c_int32), ("block", C.c_int32), ("smem_nodes", C.c_int32),
                ("schedule", C.c_int32), ("min_blocks", C.c_int32), ("split", C.c_int32),
                ("max_steps", C.c_int64)]


SPLIT_AUTO, SPLIT_OFF, SPLIT_FORCE = 0, 1, 2
_SPLIT = {"auto": SPLIT_AUTO, "off": SPLIT_OFF, "force": SPLIT_FORCE, 0: 0, 1: 1, 2: 2}


_V = C.c_void_p
_I64 = C.c_int64
_S = C.c_int  # hg_status
_SIGS = {
    "hg_build_grid": (_S, [C.POINTER(_Model), C.POINTER(_BuildParams), C.c_int32, C.POINTER(_V)]),
    "hg_build_grid_gpu": (_S, [C.POINTER(_Model), C.POINTER(_BuildParams), _V, C.POINTER(_V)]),
    "hg_tau_max_recipe": (_S, [C.POINTER(_Model), C.POINTER(_BuildParams), C.c_double, C.c_int32,
                               C.POINTER(C.c_double)]),
    "hg_host_grid_desc": (_S, [_V, C.POINTER(_Desc)]),
    "hg_host_grid_nodes": (_S, [_V, C.POINTER(_HostNodes)]),
    "hg_free_host_grid": (None, [_V]),
    "hg_load_grid": (_S, [C.POINTER(_Desc), C.c_int32, C.POINTER(_V)]),
    "hg_build_ropes": (_S, [C.POINTER(_Desc), C.c_int32, C.POINTER(C.c_int32)]),
    "hg_load_grid_ropes": (_S, [C.POINTER(_Desc), C.POINTER(C.c_int32), C.c_int32, C.POINTER(_V)]),
    "hg_free_grid": (None, [_V]),
    "hg_grid_get_info": (_S, [_V, C.POINTER(_GridInfo)]),
    "hg_trace_rays": (_S, [_V, _I64, _V, _V, _V, C.c_double, C.POINTER(TraceOpts), _V, _V, _V, _V]),
    "hg_trace_rays_noalloc": (_S, [_V, _I64, _V, _V, _V, C.c_double, C.POINTER(TraceOpts), _V, _V, _V, _V]),
    "hg_trace_rays_rho": (_S, [_V, _I64, _V, _V, _V, C.c_double, _V, C.POINTER(TraceOpts), _V, _V, _V, _V]),
    "hg_scan_offsets": (_S, [_I64, _V, _V, _V]),
    "hg_trace_fill": (_S, [_V, _I64, _V, _V, _V, C.POINTER(TraceOpts), _V, _V, _V, _I64, _V, _V]),
    "hg_sample_density": (_S, [_V, _I64, _V, _V, _V, _V]),
    "hg_tau_gradient": (_S, [_V, _I64, _V, _V, _V, C.c_double, _V, C.c_int32, _V, C.POINTER(TraceOpts), _V]),
    "hg_find_interactions": (_S, [_V, _I64, _V, _V, _V, C.c_double, _V, C.POINTER(TraceOpts), _V, _V, _V, _V,
                                  _V]),
    "hg_rays_prepare": (_S, [_V, _I64, _V, _V, _V, C.POINTER(TraceOpts), C.POINTER(_V), _V]),
    "hg_rays_trace": (_S, [_V, C.c_double, _V, C.c_int32, _V, _V, _V, _V]),
    "hg_rays_trace_gradient": (_S, [_V, C.c_double, _V, C.c_int32, _V, _V, _V, _V, C.c_int32, _V, _V]),
    "hg_rays_trace_stage": (_S, [_V, C.c_double, _V, C.c_int32, _V, _V, _V, _V, C.c_int32, _V, C.c_int32, _V]),
    "hg_rays_emit_staged": (_S, [_V, _V, _V, _V, _I64, _V, _V]),
    "hg_rays_emit_staged_gradient": (_S, [_V, _V, _V, _V, _I64, _V, C.c_double, _V, C.c_int32, _V, _V]),
    "hg_rays_fill": (_S, [_V, C.c_int32, _V, _V, _V, _I64, _V, _V]),
    "hg_rays_gradient": (_S, [_V, C.c_double, _V, C.c_int32, _V, _V]),
    "hg_rays_free": (None, [_V, _V]),
    "hg_reduce_status": (_S, [_I64, _V, _V, _V]),
    "hg_status_from_bits": (_S, [C.c_uint32]),
    "hg_load_model": (_S, [C.POINTER(_Model), C.POINTER(_V)]),
    "hg_free_model": (None, [_V]),
    "hg_model_density": (_S, [_V, _I64, _V, _V, _V]),
    "hg_model_tau": (_S, [_V, _I64, _V, _V, _V, C.c_double, C.c_double, _V, _V]),
    "hg_diff_stats": (_S, [_I64, _V, _V, _V, _V]),
    "hg_sum_i32": (_S, [_I64, _V, _V, _V]),
    "hg_batch_create": (_S, [C.c_int32, C.POINTER(_V), C.POINTER(_I64), C.c_int32, C.POINTER(_V)]),
    "hg_batch_free": (None, [_V]),
    "hg_batch_trace": (_S, [_V, _V, _V, _V, C.c_double, C.POINTER(TraceOpts), _V, _V, _V, _V]),
    "hg_autotune": (_S, [_V, _I64, _V, _V, C.c_int32, C.POINTER(TraceOpts), C.POINTER(C.c_float), _V]),
    "hg_status_str": (C.c_char_p, [_S]),
    "hg_last_error": (C.c_char_p, []),
    "hg_version": (C.c_int32, []),
    "hg_launch_count": (C.c_int64, []),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


def _check(status: int, what: str):
    if status != 0:
        msg = _lib.hg_last_error().decode(errors="replace")
        name = _lib.hg_status_str(status).decode()
        raise HgError(f"{what}: {name} ({status}): {msg}")


def launch_count() -> int:
    """Kernel launches this library has issued in this process."""
    return int(_lib.hg_launch_count())


# ----------------------------------------------------------------------------- helpers

def _torch():
    import torch
    return torch


def _stream():
    torch = _torch()
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(t, dtype=None, shape=None, name="array"):
    """Device pointer of a contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return C.c_void_p(t.data_ptr())


def _np_ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _model_struct(model):
    """hg_model from a parameter record with kind, params, table, m_tot, domain_lo, domain_hi."""
    table = np.ascontiguousarray(np.asarray(model.table, np.float64).reshape(-1))
    if table.size == 0:
        table = np.zeros(1, np.float64)
    m = _Model()
    m.kind = int(model.kind)
    m.n_table = int(np.asarray(model.table).shape[0]) if np.asarray(model.table).size else 0
    for j, v in enumerate(np.asarray(model.params, np.float64)[:8]):
        m.p[j] = float(v)
    m.table = _np_ptr(table, C.c_double)
    m.m_tot = float(model.m_tot)
    for a in range(3):
        m.lo[a] = float(model.domain_lo[a])
        m.hi[a] = float(model.domain_hi[a])
    return m, table


def _opts(precision="fp64", block=0, smem_nodes=-1, schedule=0, max_steps=0, min_blocks=0,
          split="auto") -> TraceOpts:
    """Launch options.  split: "auto" (cut long paths into segments when the queue is work-ordered),
    "off", or "force" (cut every path of more than 3 estimated crossings; for testing)."""
    o = TraceOpts()
    o.precision = {"fp64": FP64, "fp32k": FP32K, FP64: FP64, FP32K: FP32K}[precision]
    o.block = int(block)
    o.smem_nodes = int(smem_nodes)
    o.schedule = int(schedule)
    o.min_blocks = int(min_blocks)
    o.split = _SPLIT[split]
    o.max_steps = int(max_steps)
    return o


# ----------------------------------------------------------------------------- grid construction

class HostGrid:
    """A grid built on the host by hg_build_grid; numpy views of its arrays."""

    def __init__(self, handle):
        self._h = C.c_void_p(handle) if not isinstance(handle, C.c_void_p) else handle
        d = _Desc()
        _check(_lib.hg_host_grid_desc(self._h, C.byref(d)), "hg_host_grid_desc")
        nd = _HostNodes()
        _check(_lib.hg_host_grid_nodes(self._h, C.byref(nd)), "hg_host_grid_nodes")
        self.kind = int(d.kind)
        self.n_nodes = int(d.n_nodes)
        self.n_leaves = int(d.n_leaves)
        n, nl = self.n_nodes, self.n_leaves
        v = np.ctypeslib.as_array
        self.node_lo = v(d.node_lo, (n, 3))
        self.node_hi = v(d.node_hi, (n, 3))
        self.child_first = v(d.child_first, (n,))
        self.node_leaf = v(d.node_leaf, (n,))
        self.leaf_rho = v(d.leaf_rho, (nl,))
        self.nbr_off = v(d.nbr_off, (6 * nl + 1,))
        n_nbr = int(self.nbr_off[-1])
        self.nbr_id = v(d.nbr_id, (n_nbr,)) if n_nbr > 0 else np.zeros(0, np.int32)
        self.level = v(nd.level, (n, 3))
        self.index = v(nd.index, (n, 3))
        self.mass = v(nd.mass, (n,))
        self.delta = v(nd.delta, (n,))
        self.tau = v(nd.tau, (n,))
        self.q = v(nd.q, (n,))

    @property
    def leaf_node(self):
        return np.nonzero(self.child_first < 0)[0]

    def desc(self) -> "GridDesc":
        return GridDesc(self.kind, self.node_lo, self.node_hi, self.child_first, self.node_leaf, self.leaf_rho,
                        self.nbr_off, self.nbr_id, _owner=self)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _lib.hg_free_host_grid(h)
            self._h = None


def _build_params(params):
    p = _BuildParams()
    p.kind = int(params.kind)
    p.use_delta = int(bool(params.use_delta))
    p.use_tau = int(bool(params.use_tau))
    p.use_q = int(bool(params.use_q))
    p.delta_max = float(params.delta_max)
    p.tau_max = float(params.tau_max)
    p.q_max = float(params.q_max)
    p.kappa = float(params.kappa)
    p.max_level = int(params.max_level)
    p.n_ran = int(params.n_ran)
    p.seed = int(params.seed) & ((1 << 64) - 1)
    p.max_nodes = int(getattr(params, "max_nodes", 0) or 0)
    p.split_axis = int(getattr(params, "split_axis", 0) or 0)
    p.split_plane = int(getattr(params, "split_plane", 0) or 0)
    return p


def build_grid(model, params, threads: int = 0) -> HostGrid:
    """Host tree construction (hg_build_grid): node list, criteria of Eq. 1-3, neighbor lists."""
    m, _keep = _model_struct(model)
    p = _build_params(params)
    h = C.c_void_p()
    _check(_lib.hg_build_grid(C.byref(m), C.byref(p), int(threads), C.byref(h)), "hg_build_grid")
    return HostGrid(h)


def build_grid_gpu(model, params) -> HostGrid:
    """hg_build_grid_gpu: the node list with its Monte Carlo node evaluation on the current GPU
    (one thread per node, a level per launch) and the neighbor lists (one thread per leaf wall)."""
    m, _keep = _model_struct(model)
    p = _build_params(params)
    h = C.c_void_p()
    _check(_lib.hg_build_grid_gpu(C.byref(m), C.byref(p), _stream(), C.byref(h)), "hg_build_grid_gpu")
    return HostGrid(h)


def tau_max_recipe(model, params, fraction: float = 0.9, threads: int = 0) -> float:
    """The tau_max recipe of Sect. 4.1 (hg_tau_max_recipe): the leaf optical depth at position
    floor(fraction * N) of the sorted list of a grid built with the mass criterion only."""
    m, _keep = _model_struct(model)
    p = _build_params(params)
    out = C.c_double()
    _check(_lib.hg_tau_max_recipe(C.byref(m), C.byref(p), float(fraction), int(threads), C.byref(out)),
           "hg_tau_max_recipe")
    return float(out.value)


@dataclass
class GridDesc:
    """hg_grid_desc as numpy arrays (node boxes [n,3], links, leaf densities, neighbor CSR)."""

    kind: int
    node_lo: np.ndarray
    node_hi: np.ndarray
    child_first: np.ndarray
    node_leaf: np.ndarray
    leaf_rho: np.ndarray
    nbr_off: np.ndarray
    nbr_id: np.ndarray
    _owner: object = None

    def struct(self):
        keep = [np.ascontiguousarray(self.node_lo, np.float64), np.ascontiguousarray(self.node_hi, np.float64),
                np.ascontiguousarray(self.child_first, np.int32), np.ascontiguousarray(self.node_leaf, np.int32),
                np.ascontiguousarray(self.leaf_rho, np.float64), np.ascontiguousarray(self.nbr_off, np.int64),
                np.ascontiguousarray(self.nbr_id, np.int32)]
        if keep[6].size == 0:
            keep[6] = np.zeros(1, np.int32)
        d = _Desc()
        d.kind = int(self.kind)
        d.n_nodes = keep[0].shape[0]
        d.n_leaves = keep[4].shape[0]
        d.node_lo = _np_ptr(keep[0], C.c_double)
        d.node_hi = _np_ptr(keep[1], C.c_double)
        d.child_first = _np_ptr(keep[2], C.c_int32)
        d.node_leaf = _np_ptr(keep[3], C.c_int32)
        d.leaf_rho = _np_ptr(keep[4], C.c_double)
        d.nbr_off = _np_ptr(keep[5], C.c_int64)
        d.nbr_id = _np_ptr(keep[6], C.c_int32)
        return d, keep


class Grid:
    """A grid resident in HBM (hg_load_grid)."""

    def __init__(self, handle):
        self._h = handle
        info = _GridInfo()
        _check(_lib.hg_grid_get_info(self._h, C.byref(info)), "hg_grid_get_info")
        self.kind = int(info.kind)
        self.max_depth = int(info.max_depth)
        self.n_nodes = int(info.n_nodes)
        self.n_leaves = int(info.n_leaves)
        self.n_tail = int(info.n_tail)
        self.device_bytes = int(info.device_bytes)
        self.long_walls = int(info.long_walls)
        self.lo = tuple(info.lo)
        self.hi = tuple(info.hi)
        self.nav = int(info.nav)

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h:
            _lib.hg_free_grid(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def load_grid(desc, validate: bool = True, nav: str = "lists", ropes=None) -> Grid:
    """Upload a grid (a HostGrid or GridDesc) to the current CUDA device.  nav="lists": the next leaf
    from the neighbor lists (hg_load_grid); nav="ropes": from ropes (hg_load_grid_ropes), given as an
    int32 [n_leaves, 6] array or built by the library when None."""
    if isinstance(desc, HostGrid):
        desc = desc.desc()
    d, _keep = desc.struct()
    h = C.c_void_p()
    if nav == "lists":
        _check(_lib.hg_load_grid(C.byref(d), int(bool(validate)), C.byref(h)), "hg_load_grid")
    elif nav == "ropes":
        rp = None
        if ropes is not None:
            ropes = np.ascontiguousarray(ropes, np.int32)
            if ropes.size != 6 * d.n_leaves:
                raise ValueError("ropes needs 6 entries per leaf")
            rp = _np_ptr(ropes, C.c_int32)
        _check(_lib.hg_load_grid_ropes(C.byref(d), rp, int(bool(validate)), C.byref(h)), "hg_load_grid_ropes")
    else:
        raise ValueError("nav must be 'lists' or 'ropes'")
    return Grid(h)


def build_ropes(desc, threads: int = 0) -> np.ndarray:
    """hg_build_ropes: per leaf and wall (-x,+x,-y,+y,-z,+z) the leaf id, -1 on the domain boundary, or
    -2 - node for an internal node; int32 [n_leaves, 6]."""
    if isinstance(desc, HostGrid):
        desc = desc.desc()
    d, _keep = desc.struct()
    out = np.empty((d.n_leaves, 6), np.int32)
    _check(_lib.hg_build_ropes(C.byref(d), int(threads), _np_ptr(out, C.c_int32)), "hg_build_ropes")
    return out


# ----------------------------------------------------------------------------- path calculation

def _rays(o, d, s_max):
    torch = _torch()
    n = int(o.shape[0])
    po = _dptr(o, torch.float64, (n, 3), "o")
    pd = _dptr(d, torch.float64, (n, 3), "d")
    ps = _dptr(s_max, torch.float64, (n,), "s_max")
    return n, po, pd, ps


def trace_rays(grid: Grid, o, d, s_max=None, kappa: float = 1.0, precision="fp64", out=None, status: bool = True,
               **opt):
    """tau, ncross (and per-ray status) for every ray (hg_trace_rays)."""
    torch = _torch()
    n, po, pd, ps = _rays(o, d, s_max)
    op = _opts(precision, **opt)
    tdt = torch.float64 if op.precision == FP64 else torch.float32
    if out is None:
        tau = torch.empty(n, dtype=tdt, device=o.device)
        nc = torch.empty(n, dtype=torch.int32, device=o.device)
        st = torch.empty(n, dtype=torch.uint8, device=o.device) if status else None
    else:
        tau, nc, st = out
    _check(_lib.hg_trace_rays(grid.handle, n, po, pd, ps, float(kappa), C.byref(op), _dptr(tau, tdt, (n,), "tau"),
                              _dptr(nc, torch.int32, (n,), "ncross"), _dptr(st, torch.uint8, (n,), "status"),
                              _stream()), "hg_trace_rays")
    return tau, nc, st


def trace_rays_noalloc(grid: Grid, o, d, s_max=None, kappa: float = 1.0, precision="fp64", out=None,
                       status: bool = True, **opt):
    """hg_trace_rays_noalloc: as trace_rays, with the library's fixed scratch instead of
    the allocator (for callers that cannot allocate device memory while they trace;
    at most NOALLOC_MAX_RAYS rays per call, calls must not overlap on the GPU)."""
    torch = _torch()
    n, po, pd, ps = _rays(o, d, s_max)
    op = _opts(precision, **opt)
    tdt = torch.float64 if op.precision == FP64 else torch.float32
    if out is None:
        tau = torch.empty(n, dtype=tdt, device=o.device)
        nc = torch.empty(n, dtype=torch.int32, device=o.device)
        st = torch.empty(n, dtype=torch.uint8, device=o.device) if status else None
    else:
        tau, nc, st = out
    _check(_lib.hg_trace_rays_noalloc(grid.handle, n, po, pd, ps, float(kappa), C.byref(op),
                                      _dptr(tau, tdt, (n,), "tau"), _dptr(nc, torch.int32, (n,), "ncross"),
                                      _dptr(st, torch.uint8, (n,), "status"), _stream()), "hg_trace_rays_noalloc")
    return tau, nc, st


def trace_rays_rho(grid: Grid, o, d, rho, s_max=None, kappa: float = 1.0, precision="fp64", **opt):
    """tau with the leaf densities taken from ``rho`` (f64 [n_leaves])."""
    torch = _torch()
    n, po, pd, ps = _rays(o, d, s_max)
    op = _opts(precision, **opt)
    tdt = torch.float64 if op.precision == FP64 else torch.float32
    tau = torch.empty(n, dtype=tdt, device=o.device)
    nc = torch.empty(n, dtype=torch.int32, device=o.device)
    _check(_lib.hg_trace_rays_rho(grid.handle, n, po, pd, ps, float(kappa),
                                  _dptr(rho, torch.float64, (grid.n_leaves,), "rho"), C.byref(op), _dptr(tau),
                                  _dptr(nc), None, _stream()), "hg_trace_rays_rho")
    return tau, nc


def find_interactions(grid: Grid, o, d, tau_int, s_max=None, kappa: float = 1.0, out=None, **opt):
    """Interaction points (hg_find_interactions): for each path the leaf where the accumulated optical
    depth reaches tau_int (-1 if it ends first), the path parameter t there (or of the path end), the
    segments walked and the status."""
    torch = _torch()
    n, po, pd, ps = _rays(o, d, s_max)
    op = _opts("fp64", **opt)
    if out is None:
        cell = torch.empty(n, dtype=torch.int32, device=o.device)
        t = torch.empty(n, dtype=torch.float64, device=o.device)
        nc = torch.empty(n, dtype=torch.int32, device=o.device)
        st = torch.empty(n, dtype=torch.uint8, device=o.device)
    else:
        cell, t, nc, st = out
    _check(_lib.hg_find_interactions(grid.handle, n, po, pd, ps, float(kappa),
                                     _dptr(tau_int, torch.float64, (n,), "tau_int"), C.byref(op),
                                     _dptr(cell, torch.int32, (n,), "cell"), _dptr(t, torch.float64, (n,), "t"),
                                     _dptr(nc, torch.int32, (n,), "ncross"), _dptr(st, torch.uint8, (n,), "status"),
                                     _stream()), "hg_find_interactions")
    return cell, t, nc, st


def scan_offsets(counts):
    """Exclusive scan of int32 counts into int64 offsets [n+1] (hg_scan_offsets)."""
    torch = _torch()
    n = int(counts.shape[0])
    off = torch.empty(n + 1, dtype=torch.int64, device=counts.device)
    _check(_lib.hg_scan_offsets(n, _dptr(counts, torch.int32, (n,), "counts"), _dptr(off), _stream()),
           "hg_scan_offsets")
    return off


def trace_fill(grid: Grid, o, d, seg_off, s_max=None, precision="fp64", capacity: Optional[int] = None,
               status=None, **opt):
    """Segment emission pass (hg_trace_fill) given the offsets of the counting pass."""
    torch = _torch()
    n, po, pd, ps = _rays(o, d, s_max)
    op = _opts(precision, **opt)
    if capacity is None:
        capacity = int(seg_off[-1].item())
    cell = torch.empty(max(capacity, 1), dtype=torch.int32, device=o.device)
    ds = torch.empty(max(capacity, 1), dtype=torch.float64 if op.precision == FP64 else torch.float32,
                     device=o.device)
    _check(_lib.hg_trace_fill(grid.handle, n, po, pd, ps, C.byref(op), _dptr(seg_off, torch.int64, (n + 1,)),
                              _dptr(cell), _dptr(ds), int(capacity),
                              _dptr(status, torch.uint8, (n,), "status"), _stream()), "hg_trace_fill")
    return cell[:capacity], ds[:capacity]


def trace_emit(grid: Grid, o, d, s_max=None, kappa: float = 1.0, precision="fp64", **opt):
    """Counting pass + scan + emission: tau, ncross, status, seg_off, seg_cell, seg_ds."""
    tau, nc, st = trace_rays(grid, o, d, s_max, kappa, precision, **opt)
    off = scan_offsets(nc)
    cell, ds = trace_fill(grid, o, d, off, s_max, precision, status=st, **opt)
    return dict(tau=tau, ncross=nc, status=st, seg_off=off, seg_cell=cell, seg_ds=ds)


def sample_density(grid: Grid, pts):
    """Grid density rho_g and containing leaf at points (hg_sample_density)."""
    torch = _torch()
    n = int(pts.shape[0])
    cell = torch.empty(n, dtype=torch.int32, device=pts.device)
    rho = torch.empty(n, dtype=torch.float64, device=pts.device)
    _check(_lib.hg_sample_density(grid.handle, n, _dptr(pts, torch.float64, (n, 3), "pts"), _dptr(cell),
                                  _dptr(rho), _stream()), "hg_sample_density")
    return cell, rho


def tau_gradient(grid: Grid, o, d, w, s_max=None, kappa: float = 1.0, grad=None, grad_precision="fp32", **opt):
    """Accumulate d(sum_r w_r tau_r)/d(rho) into ``grad`` (hg_tau_gradient); returns grad."""
    torch = _torch()
    n, po, pd, ps = _rays(o, d, s_max)
    gp = {"fp64": 0, "fp32": 1}[grad_precision]
    gdt = torch.float64 if gp == 0 else torch.float32
    if grad is None:
        grad = torch.zeros(grid.n_leaves, dtype=gdt, device=o.device)
    op = _opts("fp64", **opt)
    _check(_lib.hg_tau_gradient(grid.handle, n, po, pd, ps, float(kappa), _dptr(w, torch.float32, (n,), "w"), gp,
                                _dptr(grad, gdt, (grid.n_leaves,), "grad"), C.byref(op), _stream()),
           "hg_tau_gradient")
    return grad


class Rays:
    """Prepared rays (hg_rays_prepare): one setup -- 1/d, clip, first leaf, work-ordered queue and
    path segments -- shared by the optical-depth, emission and adjoint walks of the same rays.
    The tensors o, d (and s_max) are kept referenced and must not change while the object lives."""

    def __init__(self, grid: Grid, o, d, s_max=None, **opt):
        n, po, pd, ps = _rays(o, d, s_max)
        self.grid, self.n, self._keep = grid, n, (o, d, s_max)
        self.device = o.device
        op = _opts("fp64", **opt)
        h = C.c_void_p()
        _check(_lib.hg_rays_prepare(grid.handle, n, po, pd, ps, C.byref(op), C.byref(h), _stream()),
               "hg_rays_prepare")
        self._h = h

    def trace(self, kappa: float = 1.0, precision="fp64", rho=None, out=None, status: bool = True):
        """tau, ncross, status (hg_rays_trace)."""
        torch = _torch()
        n = self.n
        prec = {"fp64": FP64, "fp32k": FP32K}[precision]
        tdt = torch.float64 if prec == FP64 else torch.float32
        if out is None:
            tau = torch.empty(n, dtype=tdt, device=self.device)
            nc = torch.empty(n, dtype=torch.int32, device=self.device)
            st = torch.empty(n, dtype=torch.uint8, device=self.device) if status else None
        else:
            tau, nc, st = out
        pr = None if rho is None else _dptr(rho, torch.float64, (self.grid.n_leaves,), "rho")
        _check(_lib.hg_rays_trace(self._h, float(kappa), pr, prec, _dptr(tau, tdt, (n,), "tau"),
                                  _dptr(nc, torch.int32, (n,), "ncross"), _dptr(st, torch.uint8, (n,), "status"),
                                  _stream()), "hg_rays_trace")
        return tau, nc, st

    def trace_gradient(self, w, kappa: float = 1.0, precision="fp64", rho=None, grad=None, grad_precision="fp32",
                       out=None, status: bool = True):
        """tau, ncross, status and the accumulated gradient in one walk (hg_rays_trace_gradient)."""
        torch = _torch()
        n = self.n
        prec = {"fp64": FP64, "fp32k": FP32K}[precision]
        tdt = torch.float64 if prec == FP64 else torch.float32
        gp = {"fp64": 0, "fp32": 1}[grad_precision]
        gdt = torch.float64 if gp == 0 else torch.float32
        if out is None:
            tau = torch.empty(n, dtype=tdt, device=self.device)
            nc = torch.empty(n, dtype=torch.int32, device=self.device)
            st = torch.empty(n, dtype=torch.uint8, device=self.device) if status else None
        else:
            tau, nc, st = out
        if grad is None:
            grad = torch.zeros(self.grid.n_leaves, dtype=gdt, device=self.device)
        pr = None if rho is None else _dptr(rho, torch.float64, (self.grid.n_leaves,), "rho")
        _check(_lib.hg_rays_trace_gradient(self._h, float(kappa), pr, prec, _dptr(tau, tdt, (n,), "tau"),
                                           _dptr(nc, torch.int32, (n,), "ncross"),
                                           _dptr(st, torch.uint8, (n,), "status"),
                                           _dptr(w, torch.float32, (n,), "w"), gp,
                                           _dptr(grad, gdt, (self.grid.n_leaves,), "grad"), _stream()),
               "hg_rays_trace_gradient")
        return tau, nc, st, grad

    def trace_stage(self, kappa: float = 1.0, precision="fp64", w=None, rho=None, grad=None, grad_precision="fp32",
                    out=None, status: bool = True, stage_per_ray: int = 0):
        """hg_rays_trace_stage: tau, ncross, status (and, with w, the accumulated gradient) while
        staging the emitted cells for emit_staged.  Returns (tau, nc, st, grad or None)."""
        torch = _torch()
        n = self.n
        prec = {"fp64": FP64, "fp32k": FP32K}[precision]
        tdt = torch.float64 if prec == FP64 else torch.float32
        gp = {"fp64": 0, "fp32": 1}[grad_precision]
        gdt = torch.float64 if gp == 0 else torch.float32
        if out is None:
            tau = torch.empty(n, dtype=tdt, device=self.device)
            nc = torch.empty(n, dtype=torch.int32, device=self.device)
            st = torch.empty(n, dtype=torch.uint8, device=self.device) if status else None
        else:
            tau, nc, st = out
        pw = pg = None
        if w is not None:
            if grad is None:
                grad = torch.zeros(self.grid.n_leaves, dtype=gdt, device=self.device)
            pw = _dptr(w, torch.float32, (n,), "w")
            pg = _dptr(grad, gdt, (self.grid.n_leaves,), "grad")
        pr = None if rho is None else _dptr(rho, torch.float64, (self.grid.n_leaves,), "rho")
        _check(_lib.hg_rays_trace_stage(self._h, float(kappa), pr, prec, _dptr(tau, tdt, (n,), "tau"),
                                        _dptr(nc, torch.int32, (n,), "ncross"), _dptr(st, torch.uint8, (n,), "status"),
                                        pw, gp, pg, int(stage_per_ray), _stream()), "hg_rays_trace_stage")
        self._stage_prec = prec
        return tau, nc, st, (grad if w is not None else None)

    def emit_staged(self, seg_off, capacity: Optional[int] = None, status=None, out=None):
        """hg_rays_emit_staged: the staged cells and lengths copied to their CSR slots."""
        torch = _torch()
        n = self.n
        ddt = torch.float64 if getattr(self, "_stage_prec", FP64) == FP64 else torch.float32
        if capacity is None:
            capacity = int(seg_off[-1].item())
        if out is None:
            cell = torch.empty(max(capacity, 1), dtype=torch.int32, device=self.device)
            ds = torch.empty(max(capacity, 1), dtype=ddt, device=self.device)
        else:
            cell, ds = out
        _check(_lib.hg_rays_emit_staged(self._h, _dptr(seg_off, torch.int64, (n + 1,)), _dptr(cell), _dptr(ds, ddt),
                                        int(capacity), _dptr(status, torch.uint8, (n,), "status"), _stream()),
               "hg_rays_emit_staged")
        return cell[:capacity], ds[:capacity]

    def emit_staged_gradient(self, seg_off, w, kappa: float = 1.0, grad=None, grad_precision="fp32",
                             capacity: Optional[int] = None, status=None, out=None):
        """hg_rays_emit_staged_gradient: the staged emission copied to its CSR slots while the adjoint
        (kappa w ds per staged crossing) accumulates into grad.  Returns (cell, ds, grad)."""
        torch = _torch()
        n = self.n
        ddt = torch.float64 if getattr(self, "_stage_prec", FP64) == FP64 else torch.float32
        gp = {"fp64": 0, "fp32": 1}[grad_precision]
        gdt = torch.float64 if gp == 0 else torch.float32
        if capacity is None:
            capacity = int(seg_off[-1].item())
        if out is None:
            cell = torch.empty(max(capacity, 1), dtype=torch.int32, device=self.device)
            ds = torch.empty(max(capacity, 1), dtype=ddt, device=self.device)
        else:
            cell, ds = out
        if grad is None:
            grad = torch.zeros(self.grid.n_leaves, dtype=gdt, device=self.device)
        _check(_lib.hg_rays_emit_staged_gradient(
            self._h, _dptr(seg_off, torch.int64, (n + 1,)), _dptr(cell), _dptr(ds, ddt), int(capacity),
            _dptr(status, torch.uint8, (n,), "status"), float(kappa), _dptr(w, torch.float32, (n,), "w"), gp,
            _dptr(grad, gdt, (self.grid.n_leaves,), "grad"), _stream()), "hg_rays_emit_staged_gradient")
        return cell[:capacity], ds[:capacity], grad

    def emit_single_pass(self, kappa: float = 1.0, precision="fp64", w=None, grad=None, grad_precision="fp32",
                         stage_per_ray: int = 0, adjoint: str = "copy"):
        """Optical depth (and gradient) with the emission in one walk plus a copy:
        tau, ncross, status, seg_off, seg_cell, seg_ds (and grad).  With w, adjoint="copy" scatters
        the gradient from the staged lengths during the copy; "walk" scatters it inside the walk."""
        if adjoint not in ("copy", "walk"):
            raise ValueError("adjoint must be 'copy' or 'walk'")
        in_walk = w is not None and adjoint == "walk"
        tau, nc, st, g = self.trace_stage(kappa, precision, w=w if in_walk else None, grad=grad,
                                          grad_precision=grad_precision, stage_per_ray=stage_per_ray)
        off = scan_offsets(nc)
        if w is None or in_walk:
            cell, ds = self.emit_staged(off, status=st)
        else:
            cell, ds, g = self.emit_staged_gradient(off, w, kappa=kappa, grad=grad, grad_precision=grad_precision,
                                                    status=st)
        return dict(tau=tau, ncross=nc, status=st, seg_off=off, seg_cell=cell, seg_ds=ds, grad=g)

    def fill(self, seg_off, precision="fp64", capacity: Optional[int] = None, status=None, out=None):
        """Emitted cells and lengths (hg_rays_fill) at the offsets of a trace of these rays."""
        torch = _torch()
        n = self.n
        prec = {"fp64": FP64, "fp32k": FP32K}[precision]
        ddt = torch.float64 if prec == FP64 else torch.float32
        if capacity is None:
            capacity = int(seg_off[-1].item())
        if out is None:
            cell = torch.empty(max(capacity, 1), dtype=torch.int32, device=self.device)
            ds = torch.empty(max(capacity, 1), dtype=ddt, device=self.device)
        else:
            cell, ds = out
        _check(_lib.hg_rays_fill(self._h, prec, _dptr(seg_off, torch.int64, (n + 1,)), _dptr(cell),
                                 _dptr(ds, ddt), int(capacity), _dptr(status, torch.uint8, (n,), "status"),
                                 _stream()), "hg_rays_fill")
        return cell[:capacity], ds[:capacity]

    def emit(self, kappa: float = 1.0, precision="fp64"):
        """Counting pass + scan + emission on these rays: tau, ncross, status, seg_off, seg_cell, seg_ds."""
        tau, nc, st = self.trace(kappa, precision)
        off = scan_offsets(nc)
        cell, ds = self.fill(off, precision, status=st)
        return dict(tau=tau, ncross=nc, status=st, seg_off=off, seg_cell=cell, seg_ds=ds)

    def gradient(self, w, kappa: float = 1.0, grad=None, grad_precision="fp32"):
        """Accumulate d(sum_r w_r tau_r)/d(rho) into ``grad`` (hg_rays_gradient); returns grad."""
        torch = _torch()
        gp = {"fp64": 0, "fp32": 1}[grad_precision]
        gdt = torch.float64 if gp == 0 else torch.float32
        if grad is None:
            grad = torch.zeros(self.grid.n_leaves, dtype=gdt, device=self.device)
        _check(_lib.hg_rays_gradient(self._h, float(kappa), _dptr(w, torch.float32, (self.n,), "w"), gp,
                                     _dptr(grad, gdt, (self.grid.n_leaves,), "grad"), _stream()),
               "hg_rays_gradient")
        return grad

    def free(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.hg_rays_free(self._h, _stream())
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def prepare_rays(grid: Grid, o, d, s_max=None, **opt) -> Rays:
    return Rays(grid, o, d, s_max, **opt)


def reduce_status(status):
    """OR of all per-ray status bits (device uint32 tensor [1])."""
    torch = _torch()
    n = int(status.shape[0])
    out = torch.empty(1, dtype=torch.int32, device=status.device)
    _check(_lib.hg_reduce_status(n, _dptr(status, torch.uint8, (n,)), _dptr(out), _stream()), "hg_reduce_status")
    return out


def status_from_bits(bits: int) -> int:
    return int(_lib.hg_status_from_bits(int(bits) & 0xFFFFFFFF))


def sum_i32(x):
    torch = _torch()
    n = int(x.shape[0])
    out = torch.empty(1, dtype=torch.int64, device=x.device)
    _check(_lib.hg_sum_i32(n, _dptr(x, torch.int32, (n,)), _dptr(out), _stream()), "hg_sum_i32")
    return out


# ----------------------------------------------------------------------------- quality metrics

class DModel:
    """A density model uploaded for rho_t / tau_t on the device (hg_load_model)."""

    def __init__(self, model):
        m, _keep = _model_struct(model)
        h = C.c_void_p()
        _check(_lib.hg_load_model(C.byref(m), C.byref(h)), "hg_load_model")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _lib.hg_free_model(h)
            self._h = None


def load_model(model) -> DModel:
    return DModel(model)


def model_density(dm: DModel, pts):
    torch = _torch()
    n = int(pts.shape[0])
    rho = torch.empty(n, dtype=torch.float64, device=pts.device)
    _check(_lib.hg_model_density(dm._h, n, _dptr(pts, torch.float64, (n, 3)), _dptr(rho), _stream()),
           "hg_model_density")
    return rho


def model_tau(dm: DModel, o, d, length, kappa: float = 1.0, rtol: float = 1e-11):
    torch = _torch()
    n, po, pd, pl = _rays(o, d, length)
    tau = torch.empty(n, dtype=torch.float64, device=o.device)
    _check(_lib.hg_model_tau(dm._h, n, po, pd, pl, float(kappa), float(rtol), _dptr(tau), _stream()),
           "hg_model_tau")
    return tau


def diff_stats(a, b):
    """Device f64[3] = (n, mean, population std) of a - b (hg_diff_stats)."""
    torch = _torch()
    n = int(a.shape[0])
    out = torch.empty(3, dtype=torch.float64, device=a.device)
    _check(_lib.hg_diff_stats(n, _dptr(a, torch.float64, (n,)), _dptr(b, torch.float64, (n,)), _dptr(out),
                              _stream()), "hg_diff_stats")
    return out


# ----------------------------------------------------------------------------- batching and tuning

class Batch:
    """Many grids traced in one persistent launch (hg_batch_create / hg_batch_trace)."""

    def __init__(self, grids: Sequence[Grid], ray_begin: Sequence[int]):
        self.grids = list(grids)  # keep the grids alive as long as the batch
        arr = (C.c_void_p * len(grids))(*[g.handle.value if isinstance(g.handle, C.c_void_p) else g.handle
                                          for g in grids])
        rb = np.ascontiguousarray(np.asarray(ray_begin, np.int64))
        if rb.shape[0] != len(grids) + 1:
            raise ValueError("ray_begin needs n_grids + 1 entries")
        self.ray_begin = rb
        h = C.c_void_p()
        _check(_lib.hg_batch_create(len(grids), C.cast(arr, C.POINTER(C.c_void_p)), _np_ptr(rb, C.c_int64), 0,
                                    C.byref(h)), "hg_batch_create")
        self._h = h
        self.n_rays = int(rb[-1])

    def trace(self, o, d, s_max=None, kappa: float = 1.0, precision="fp64", out=None, status: bool = True, **opt):
        torch = _torch()
        n, po, pd, ps = _rays(o, d, s_max)
        if n != self.n_rays:
            raise ValueError(f"batch holds {self.n_rays} rays, got {n}")
        op = _opts(precision, **opt)
        tdt = torch.float64 if op.precision == FP64 else torch.float32
        if out is None:
            tau = torch.empty(n, dtype=tdt, device=o.device)
            nc = torch.empty(n, dtype=torch.int32, device=o.device)
            st = torch.empty(n, dtype=torch.uint8, device=o.device) if status else None
        else:
            tau, nc, st = out
        _check(_lib.hg_batch_trace(self._h, po, pd, ps, float(kappa), C.byref(op), _dptr(tau, tdt, (n,)),
                                   _dptr(nc, torch.int32, (n,)), _dptr(st, torch.uint8, (n,)), _stream()),
               "hg_batch_trace")
        return tau, nc, st

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _lib.hg_batch_free(h)
            self._h = None


def autotune(grid: Grid, o, d, precision="fp64"):
    """Sweep launch shapes on these rays; the winner becomes the grid's default. Returns (opts dict, ms)."""
    n, po, pd, _ = _rays(o, d, None)
    best = TraceOpts()
    ms = C.c_float()
    p = {"fp64": FP64, "fp32k": FP32K}[precision]
    _check(_lib.hg_autotune(grid.handle, n, po, pd, p, C.byref(best), C.byref(ms), _stream()), "hg_autotune")
    return dict(block=best.block, smem_nodes=best.smem_nodes, schedule=best.schedule,
                min_blocks=best.min_blocks), float(ms.value)


# ----------------------------------------------------------------------------- autograd

class TauFn:
    """torch.autograd.Function for rho -> tau (linear in rho).

    forward: hg_trace_rays_rho (FP64); backward: the adjoint kernel
    hg_tau_gradient, an atomic scatter of kappa * w_r * ds into each crossed
    leaf (FP64 atomics for double gradients).
    """

    _fn = None

    @classmethod
    def apply(cls, rho, grid: Grid, o, d, s_max=None, kappa: float = 1.0):
        if cls._fn is None:
            torch = _torch()

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(ctx, rho_, grid_, o_, d_, s_max_, kappa_):
                    ctx.grid, ctx.kappa = grid_, kappa_
                    ctx.save_for_backward(o_, d_, *([] if s_max_ is None else [s_max_]))
                    ctx.has_smax = s_max_ is not None
                    tau, _ = trace_rays_rho(grid_, o_, d_, rho_.contiguous(), s_max_, kappa_)
                    return tau

                @staticmethod
                def backward(ctx, g):
                    saved = ctx.saved_tensors
                    o_, d_ = saved[0], saved[1]
                    s_ = saved[2] if ctx.has_smax else None
                    w = g.detach().to(torch.float32).contiguous()
                    grad = tau_gradient(ctx.grid, o_, d_, w, s_, ctx.kappa, grad_precision="fp64")
                    return grad, None, None, None, None, None

            cls._fn = _F
        return cls._fn.apply(rho, grid, o, d, s_max, kappa)
