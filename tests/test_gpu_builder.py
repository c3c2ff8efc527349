"""The tree construction on the GPU (hg_build_grid_gpu) against the oracle's builder:
bit-identical node lists and statistics for models without exponentials (constant, dyadic
lattice, torus without clumps), and for the disk and clump models the same node lists with
statistics within a few ulps (CUDA's exp against the host libm's), at the test sizes and at the
full disk workload.  Its neighbor lists, found on the device, equal the host builder's (which the
CPU tests pin by wall tiling and symmetry)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
hg = pytest.importorskip("paper_1311_0705_gb300")

pytestmark = pytest.mark.gpu


def _same_structure(H, T):
    assert H.n_nodes == T.n_nodes and H.n_leaves == T.n_leaves
    np.testing.assert_array_equal(H.level, T.lvl)
    np.testing.assert_array_equal(H.index, T.idx)
    np.testing.assert_array_equal(H.node_lo, T.lo)
    np.testing.assert_array_equal(H.node_hi, T.hi)
    np.testing.assert_array_equal(H.child_first, T.child)
    np.testing.assert_array_equal(H.node_leaf, T.leaf)


def _same_lists(H, Hh):
    np.testing.assert_array_equal(H.nbr_off, Hh.nbr_off)
    np.testing.assert_array_equal(H.nbr_id, Hh.nbr_id)


def _same_stats(H, T, exact):
    pairs = ((H.leaf_rho, T.leaf_rho), (H.mass, T.mass), (H.tau, T.taun))
    if exact:
        for a, b in pairs:
            np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(H.q, T.q)
        return
    # a draw's exp may differ by an ulp: sums of positive draws stay within a few ulps relative;
    # q = (max - min) / max within a few ulps of 1 absolute
    for a, b in pairs:
        np.testing.assert_allclose(a, b, rtol=1e-13, atol=0)
    np.testing.assert_allclose(H.q, T.q, rtol=0, atol=1e-15)


EXACT = [
    ("dyadic-oct", lambda: synth.make_dyadic(3, level=2), dict(kind=0, delta_max=1e-3, max_level=4)),
    ("dyadic-kd", lambda: synth.make_dyadic(4, level=3), dict(kind=1, delta_max=2e-3, use_q=True, q_max=0.5,
                                                              max_level=5)),
    ("const-tau", lambda: synth.make_const(2.0), dict(kind=1, use_delta=False, use_tau=True, tau_max=0.9,
                                                      max_level=6)),
    ("torus-smooth-oct", lambda: synth.make_torus(13, n_clumps=0), dict(kind=0, delta_max=1e-3, use_q=True,
                                                                        q_max=0.5, max_level=5)),
    ("dyadic-kd-grad", lambda: synth.make_dyadic(4, level=3), dict(kind=1, delta_max=2e-3, use_q=True, q_max=0.5,
                                                                   max_level=5, split_axis=1)),
]
WITH_EXP = [
    ("disk-oct", lambda: synth.make_disk(), dict(kind=0, delta_max=1e-4, max_level=6)),
    ("disk-kd", lambda: synth.make_disk(), dict(kind=1, delta_max=5e-5, max_level=6)),
    ("torus-kd-all", lambda: synth.make_torus(11, n_clumps=60), dict(kind=1, delta_max=1e-3, use_tau=True,
                                                                     tau_max=2.0, use_q=True, q_max=0.9,
                                                                     max_level=5)),
    ("disk-kd-grad", lambda: synth.make_disk(), dict(kind=1, delta_max=5e-5, max_level=6, split_axis=1)),
]


@pytest.mark.parametrize("name,mk,kw", EXACT, ids=[c[0] for c in EXACT])
def test_device_builder_bit_exact_without_exp(name, mk, kw):
    model = mk()
    bp = synth.BuildParams(seed=synth.BASE_SEED + 19, **kw)
    H = hg.build_grid_gpu(model, bp)
    T = oracle.build_tree(model, bp)
    _same_structure(H, T)
    _same_stats(H, T, exact=True)
    _same_lists(H, hg.build_grid(model, bp, threads=4))


@pytest.mark.parametrize("name,mk,kw", WITH_EXP, ids=[c[0] for c in WITH_EXP])
def test_device_builder_with_exp_models(name, mk, kw):
    model = mk()
    bp = synth.BuildParams(seed=synth.BASE_SEED + 19, **kw)
    H = hg.build_grid_gpu(model, bp)
    T = oracle.build_tree(model, bp)
    _same_structure(H, T)
    _same_stats(H, T, exact=False)
    _same_lists(H, hg.build_grid(model, bp, threads=4))


@pytest.mark.parametrize("kind", [0, 1], ids=["octree", "kd"])
def test_device_builder_full_disk_workload(kind):
    # the disk-1e6 grids (mass 1e-6, max level 12): 3.3e6 octree / 1.4e6 k-d leaves
    model, bp, _, _ = synth.workload_disk_1e6(kind)
    H = hg.build_grid_gpu(model, bp)
    T = oracle.build_tree(model, bp)
    _same_structure(H, T)
    _same_stats(H, T, exact=False)
    _same_lists(H, hg.build_grid(model, bp))


def test_device_builder_grid_traces_like_host_grid():
    # a grid from the device builder loads and walks like the host builder's (same cells and lengths)
    model = synth.make_torus(11, n_clumps=60)
    bp = synth.BuildParams(kind=1, delta_max=1e-3, use_tau=True, tau_max=2.0, use_q=True, q_max=0.9, max_level=5)
    gd = hg.load_grid(hg.build_grid_gpu(model, bp))
    gh = hg.load_grid(hg.build_grid(model, bp))
    o, k = synth.emission_rays(31, 3000)
    O, K = torch.tensor(o, device="cuda"), torch.tensor(k, device="cuda")
    a = hg.prepare_rays(gd, O, K).emit_single_pass()
    b = hg.prepare_rays(gh, O, K).emit_single_pass()
    for key in ("ncross", "seg_off", "seg_cell", "seg_ds"):
        np.testing.assert_array_equal(a[key].cpu().numpy(), b[key].cpu().numpy())


def test_device_builder_rejects_bad_parameters():
    model = synth.make_disk()
    for kw in (dict(n_ran=0), dict(max_level=21), dict(kind=5)):
        bp = synth.BuildParams(**{**dict(kind=0, delta_max=1e-3, max_level=3), **kw})
        with pytest.raises(hg.HgError):
            hg.build_grid_gpu(model, bp)
