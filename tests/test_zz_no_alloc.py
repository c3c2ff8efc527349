"""The allocation-free tracing entry point (hg_trace_rays_noalloc).

Callers that cannot allocate device memory while they trace (a stream
capture that forbids allocation, a real-time loop, a fixed memory budget)
use this entry point; it must give what hg_trace_rays gives.  Two calls in a
row, with different rays, check that nothing left in the library's fixed
scratch array from one call leaks into the next; a call at exactly the
array's ray limit uses its last start record; and the stream-ordered pool's
high-water mark and the device's free memory show that a call takes no
memory.  This file is collected last so that a run stopping at the first
failure has run every other test.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _np(t):
    return t.detach().cpu().numpy()


def _hg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_0705_gb300 as hg
    return hg


def _same(hg, grid, O, K, S, kappa, precision, ref=None):
    if ref is None:
        ref = hg.trace_rays(grid, O, K, S, kappa=kappa, precision=precision)
    tau, nc, st = hg.trace_rays_noalloc(grid, O, K, S, kappa=kappa, precision=precision)
    torch.cuda.synchronize()
    # counts and statuses are exact; tau equal up to the grouping of additions when hg_trace_rays cuts
    # long paths into segments (this entry point walks every path whole)
    np.testing.assert_array_equal(_np(nc), _np(ref[1]))
    np.testing.assert_array_equal(_np(st), _np(ref[2]))
    rt = _np(ref[0]).astype(np.float64)
    rtol = 1e-6 if precision == "fp64" else 1e-5
    assert (np.abs(_np(tau).astype(np.float64) - rt) <= rtol * np.abs(rt)).all()
    assert int(_np(nc).sum()) > 0


def test_noalloc_matches_trace_rays_on_two_calls_in_a_row():
    hg = _hg()
    model, bp, n_rays, seed = synth.workload_disk_small()
    bp.kind = synth.TREE_KD
    grid = hg.load_grid(hg.build_grid(model, bp))
    o, k = synth.emission_rays(seed, 30000)
    a, d, L = synth.endpoint_paths(seed + 1, 12345)
    calls = [dict(o=o, k=k, smax=None, kappa=1.0, precision="fp64"),
             dict(o=a, k=d, smax=L, kappa=2.0, precision="fp32k")]
    for c in calls:
        O = torch.tensor(c["o"], device="cuda")
        K = torch.tensor(c["k"], device="cuda")
        S = None if c["smax"] is None else torch.tensor(c["smax"], device="cuda")
        _same(hg, grid, O, K, S, c["kappa"], c["precision"])


def test_noalloc_at_exactly_its_ray_limit():
    # the largest accepted batch fills the fixed array to its last start record
    hg = _hg()
    model, bp, n_rays, seed = synth.workload_disk_small()
    grid = hg.load_grid(hg.build_grid(model, bp))
    n = hg.NOALLOC_MAX_RAYS
    o, k = synth.emission_rays(seed + 7, n)
    O, K = torch.tensor(o, device="cuda"), torch.tensor(k, device="cuda")
    _same(hg, grid, O, K, None, 1.0, "fp64")
    # the last rays alone, traced after the full batch, still agree
    _same(hg, grid, O[-1000:].contiguous(), K[-1000:].contiguous(), None, 1.0, "fp64")


class _Pool:
    """Used-memory high-water mark of the device's current stream-ordered pool (the pool the library's
    other entry points draw their scratch from), read through the CUDA driver API."""

    USED_MEM_CURRENT, USED_MEM_HIGH = 7, 8

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuCtxGetDevice(ctypes.byref(dev)) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetMemPool(ctypes.byref(self.pool), dev) == 0

    def _get(self, attr):
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return int(v.value)

    def reset_high(self):
        z = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH, ctypes.byref(z)) == 0
        return self._get(self.USED_MEM_CURRENT)

    def high(self):
        return self._get(self.USED_MEM_HIGH)


def test_noalloc_call_takes_no_device_memory():
    # after a warm-up call (which loads the kernels), a call through the allocation-free entry point leaves
    # the pool's high-water mark and the device's free memory where they were; hg_trace_rays on the same
    # rays does raise the mark, which shows that the check sees the scratch the other entry points take
    hg = _hg()
    model, bp, n_rays, seed = synth.workload_disk_small()
    grid = hg.load_grid(hg.build_grid(model, bp))
    o, k = synth.emission_rays(seed + 9, 50000)
    O, K = torch.tensor(o, device="cuda"), torch.tensor(k, device="cuda")
    out = (torch.empty(O.shape[0], dtype=torch.float64, device="cuda"),
           torch.empty(O.shape[0], dtype=torch.int32, device="cuda"),
           torch.empty(O.shape[0], dtype=torch.uint8, device="cuda"))
    hg.trace_rays_noalloc(grid, O, K, out=out)
    torch.cuda.synchronize()
    pool = _Pool()
    used = pool.reset_high()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        hg.trace_rays_noalloc(grid, O, K, out=out)
    torch.cuda.synchronize()
    assert pool.high() == used
    assert torch.cuda.mem_get_info()[0] == free0
    used = pool.reset_high()
    hg.trace_rays(grid, O, K, out=out)
    torch.cuda.synchronize()
    assert pool.high() >= used + 48 * O.shape[0]


def test_noalloc_rejects_more_rays_than_its_scratch_holds():
    hg = _hg()
    model, bp, n_rays, seed = synth.workload_disk_small()
    grid = hg.load_grid(hg.build_grid(model, bp))
    n = hg.NOALLOC_MAX_RAYS + 1
    O = torch.zeros(n, 3, dtype=torch.float64, device="cuda")
    with pytest.raises(hg.HgError, match="exceed the fixed scratch"):
        hg.trace_rays_noalloc(grid, O, O)
