"""The allocation-free tracing entry point (hg_trace_rays_noalloc).

Callers that cannot allocate device memory while they trace (a stream
capture that forbids allocation, a real-time loop, a fixed memory budget)
use this entry point; it must give what hg_trace_rays gives.  Two calls in a
row, with different rays, check that nothing left in the library's fixed
scratch array from one call leaks into the next.  This file is collected
last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _np(t):
    return t.detach().cpu().numpy()


def test_noalloc_matches_trace_rays_on_two_calls_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_0705_gb300 as hg
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
        ref_tau, ref_nc, ref_st = hg.trace_rays(grid, O, K, S, kappa=c["kappa"], precision=c["precision"])
        tau, nc, st = hg.trace_rays_noalloc(grid, O, K, S, kappa=c["kappa"], precision=c["precision"])
        torch.cuda.synchronize()
        np.testing.assert_array_equal(_np(nc), _np(ref_nc))
        np.testing.assert_array_equal(_np(st), _np(ref_st))
        rt = _np(ref_tau).astype(np.float64)
        rtol = 1e-6 if c["precision"] == "fp64" else 1e-5
        assert (np.abs(_np(tau).astype(np.float64) - rt) <= rtol * np.abs(rt)).all()
        assert int(_np(nc).sum()) > 0


def test_noalloc_rejects_more_rays_than_its_scratch_holds():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_0705_gb300 as hg
    model, bp, n_rays, seed = synth.workload_disk_small()
    grid = hg.load_grid(hg.build_grid(model, bp))
    n = hg.NOALLOC_MAX_RAYS + 1
    O = torch.zeros(n, 3, dtype=torch.float64, device="cuda")
    with pytest.raises(hg.HgError, match="exceed the fixed scratch"):
        hg.trace_rays_noalloc(grid, O, O)
