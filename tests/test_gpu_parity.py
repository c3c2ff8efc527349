"""GPU path calculation against the FP64 oracle, element by element.

Cell sequences and crossing counts must match bit for bit; FP64 optical
depths within 1e-6 relative (identical operation order makes them equal in
practice); FP32-Kahan optical depths within 1e-5 relative of the oracle's
FP64 value.  Every call goes through the C ABI (``paper_1311_0705_gb300``).
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TAU_RTOL_FP64 = 1e-6
TAU_RTOL_FP32K = 1e-5


@pytest.fixture(scope="module")
def hg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1311_0705_gb300 as m
    return m


def _cuda(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _np(t):
    return t.detach().cpu().numpy()


def _check_tau(got, ref, rtol):
    got = np.asarray(got, np.float64)
    err = np.abs(got - ref)
    assert (err <= rtol * np.abs(ref) + 1e-300).all(), float((err / np.maximum(np.abs(ref), 1e-300)).max())


def _compare(hg, grid, tree, o, k, smax=None, kappa=1.0, precision="fp64", max_steps=None, **opt):
    ms = oracle.default_max_steps(tree.n_leaves) if max_steps is None else max_steps
    ref = oracle.trace(tree, o, k, smax=smax, kappa=kappa, emit=True, max_steps=ms)
    O, K = _cuda(o), _cuda(k)
    S = None if smax is None else _cuda(smax)
    out = hg.trace_emit(grid, O, K, S, kappa=kappa, precision=precision, max_steps=ms, **opt)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(_np(out["ncross"]), ref["ncross"])
    np.testing.assert_array_equal(_np(out["status"]), ref["status"])
    np.testing.assert_array_equal(_np(out["seg_off"]), ref["seg_off"])
    np.testing.assert_array_equal(_np(out["seg_cell"]), ref["seg_cell"])
    if precision == "fp64":
        np.testing.assert_array_equal(_np(out["seg_ds"]), ref["seg_ds"])
        _check_tau(_np(out["tau"]), ref["tau"], TAU_RTOL_FP64)
    else:
        np.testing.assert_array_equal(_np(out["seg_ds"]), ref["seg_ds"].astype(np.float32))
        _check_tau(_np(out["tau"]), ref["tau"], TAU_RTOL_FP32K)
    return ref, out


# ----------------------------------------------------------------------------- grids

@pytest.fixture(scope="module")
def disk_grids(hg):
    model, bp, n_rays, seed = synth.workload_disk_small()
    out = {}
    for kind in (synth.TREE_OCTREE, synth.TREE_KD):
        bp.kind = kind
        H = hg.build_grid(model, bp)
        T = oracle.build_tree(model, bp)
        np.testing.assert_array_equal(H.child_first, T.child)
        np.testing.assert_array_equal(H.leaf_rho, T.leaf_rho)
        out[kind] = (hg.load_grid(H), T, H)
    o, k = synth.emission_rays(seed, n_rays)
    return model, out, o, k


@pytest.mark.parametrize("shape", [dict(), dict(split="force"), dict(schedule=1, smem_nodes=0)],
                         ids=["auto", "forced-split", "static-nosmem"])
def test_gradient_axis_kd_sequences_bit_exact(hg, shape):
    # a k-d tree split on the axis of the strongest density gradient (Sect. 2.2): nodes no longer cycle
    # through x, y, z, so the descent, neighbor lists and segment planner meet uneven refinement
    model, bp, n_rays, seed = synth.workload_disk_small()
    bp.kind, bp.split_axis, bp.delta_max = synth.TREE_KD, 1, 5e-5
    H = hg.build_grid(model, bp)
    T = oracle.build_tree(model, bp)
    np.testing.assert_array_equal(H.child_first, T.child)
    assert (T.lvl.max(axis=0) == bp.max_level).all()
    o, k = synth.emission_rays(seed + 7, 4000)
    ref, _ = _compare(hg, hg.load_grid(H), T, o, k, **shape)
    assert ref["ncross"].sum() > 4000 * 5


SPLIT_VARIANTS = [(synth.TREE_OCTREE, synth.PLANE_BARYCENTRE, 0, 1e-4), (synth.TREE_KD, synth.PLANE_EQUAL_MASS, 0, 5e-5),
                  (synth.TREE_KD, synth.PLANE_EQUAL_DENSITY, 0, 5e-5), (synth.TREE_KD, synth.PLANE_EQUAL_MASS, 1, 5e-5)]
SPLIT_IDS = ["octree-barycentre", "kd-equal-mass", "kd-equal-density", "kd-gradient-equal-mass"]


def _wall_rays(tree, seed, n):
    """Rays starting on the tree's own (non-dyadic) leaf walls, edges and corners, half of them along
    axis-aligned or in-plane directions (zero components), the rest isotropic."""
    rng = np.random.default_rng(seed)
    leaves = rng.integers(0, tree.n_leaves, n)
    lo, hi = tree.leaf_lo[leaves], tree.leaf_hi[leaves]
    p = lo + rng.random((n, 3)) * (hi - lo)
    pick = rng.random((n, 3))
    p = np.where(pick < 0.35, lo, np.where(pick < 0.7, hi, p))
    k = synth.isotropic_dirs(rng, n)
    m = rng.random(n) < 0.5
    kd = rng.choice([-1.0, -0.0, 0.0, 1.0, 0.6, -0.8], size=(n, 3))
    bad = np.all(kd == 0, axis=1)
    kd[bad, 0] = 1.0
    k[m] = kd[m]
    return p, k


@pytest.mark.parametrize("kind,plane,axis,dmax", SPLIT_VARIANTS, ids=SPLIT_IDS)
@pytest.mark.parametrize("shape", [dict(), dict(split="force"), dict(schedule=1, smem_nodes=0)],
                         ids=["auto", "forced-split", "static-nosmem"])
def test_split_location_variants_sequences_bit_exact(hg, kind, plane, axis, dmax, shape):
    # barycentric octrees and equal-mass / equal-mean-density k-d trees (Sect. 2.2): node boxes with FP64
    # planes that are no dyadic lattice points, walked through their FP64-keyed leaf records; cell
    # sequences, lengths, counts and statuses bit-exact against the oracle, tau within 1e-6 (FP64) / 1e-5
    model, bp, n_rays, seed = synth.workload_disk_small()
    bp.kind, bp.split_plane, bp.split_axis, bp.delta_max = kind, plane, axis, dmax
    H = hg.build_grid(model, bp)
    T = oracle.build_tree(model, bp)
    np.testing.assert_array_equal(H.child_first, T.child)
    np.testing.assert_array_equal(H.node_lo, T.lo)
    np.testing.assert_array_equal(H.node_hi, T.hi)
    grid = hg.load_grid(H, validate=True)
    o, k = synth.emission_rays(seed + 11, 4000)
    ref, _ = _compare(hg, grid, T, o, k, **shape)
    assert ref["ncross"].sum() > 4000 * 5
    _compare(hg, grid, T, o, k, precision="fp32k", **shape)
    a, d, L = synth.endpoint_paths(seed + 12, 2000)
    _compare(hg, grid, T, a, d, smax=L, kappa=1.7, **shape)
    wo, wk = _wall_rays(T, seed + 13, 3000)
    _compare(hg, grid, T, wo, wk, **shape)


SHAPES = [dict(), dict(schedule=1), dict(schedule=2, block=128, smem_nodes=0), dict(schedule=3, block=256, smem_nodes=64),
          dict(schedule=1, block=64, smem_nodes=100000), dict(min_blocks=4), dict(min_blocks=4, schedule=1, block=96)]


@pytest.mark.parametrize("kind", [0, 1], ids=["octree", "kd"])
@pytest.mark.parametrize("shape", SHAPES, ids=[str(s) for s in SHAPES])
def test_small_disk_sequences_bit_exact(hg, disk_grids, kind, shape):
    model, grids, o, k = disk_grids
    grid, tree, _ = grids[kind]
    _compare(hg, grid, tree, o, k, **shape)


@pytest.mark.parametrize("kind", [0, 1], ids=["octree", "kd"])
def test_fp32k_sequence_and_tau_bound(hg, disk_grids, kind):
    model, grids, o, k = disk_grids
    grid, tree, _ = grids[kind]
    _compare(hg, grid, tree, o, k, precision="fp32k")


@pytest.mark.parametrize("kind", [0, 1], ids=["octree", "kd"])
def test_path_ends_kappa_and_ragged_counts(hg, disk_grids, kind):
    model, grids, _, _ = disk_grids
    grid, tree, _ = grids[kind]
    a, k, L = synth.endpoint_paths(77, 3001)
    _compare(hg, grid, tree, a, k, smax=L, kappa=2.5)
    _compare(hg, grid, tree, a, k, smax=L * 0.37, kappa=0.5, precision="fp32k")


def test_outside_origins_misses_and_bad_inputs(hg, disk_grids):
    model, grids, _, _ = disk_grids
    grid, tree, _ = grids[0]
    rng = np.random.default_rng(3)
    o = rng.uniform(-3, 3, size=(2000, 3))
    k = synth.isotropic_dirs(rng, 2000)
    k[:10] = 0.0
    k[10:20, 1] = np.nan
    o[20:30, 0] = np.inf
    k[30:40] = [[-0.0, 0.0, 1.0]] * 10
    ref, _ = _compare(hg, grid, tree, o, k)
    assert (ref["status"][:30] == oracle.RAY_BADINPUT).all()
    assert (ref["ncross"] == 0).any() and (ref["ncross"] > 0).any()


@pytest.mark.parametrize("kind", [0, 1], ids=["octree", "kd"])
def test_degenerate_rays_on_uniform_grid(hg, kind):
    model = synth.make_const(1.5)
    bp = synth.BuildParams(kind=kind, delta_max=-1.0, max_level=3)
    grid = hg.load_grid(hg.build_grid(model, bp))
    tree = oracle.build_tree(model, bp)
    o, k = synth.degenerate_rays(levels=3, n_random=2000, seed=kind + 5)
    _compare(hg, grid, tree, o, k)
    _compare(hg, grid, tree, o, k, smem_nodes=0, schedule=1)


@pytest.mark.parametrize("kind", [0, 1], ids=["octree", "kd"])
def test_degenerate_rays_on_adaptive_grid(hg, kind):
    # lattice-aligned rays through a refined grid exercise edge/corner exits and list scans
    model = synth.make_torus(21, n_clumps=20)
    bp = synth.BuildParams(kind=kind, delta_max=1e-3, use_q=True, q_max=0.9, max_level=5)
    grid = hg.load_grid(hg.build_grid(model, bp))
    tree = oracle.build_tree(model, bp)
    o, k = synth.degenerate_rays(levels=5, n_random=3000, seed=kind + 9)
    _compare(hg, grid, tree, o, k)
    o2, k2 = synth.emission_rays(kind + 100, 5000)
    _compare(hg, grid, tree, o2, k2)


def test_step_limit_reported_like_oracle(hg, disk_grids):
    model, grids, o, k = disk_grids
    grid, tree, _ = grids[1]
    ref, out = _compare(hg, grid, tree, o[:3000], k[:3000], max_steps=7)
    assert (ref["status"] == oracle.RAY_STEPLIMIT).any()


def test_empty_and_single_ray(hg, disk_grids):
    model, grids, o, k = disk_grids
    grid, tree, _ = grids[0]
    tau, nc, st = hg.trace_rays(grid, _cuda(np.zeros((0, 3))), _cuda(np.zeros((0, 3))))
    assert tau.numel() == 0
    _compare(hg, grid, tree, o[:1], k[:1])


# ----------------------------------------------------------------------------- scan, reductions

@pytest.mark.parametrize("n", [0, 1, 5, 8191, 8192, 8193, 100003, 2_500_001])
def test_scan_offsets(hg, n):
    c = np.random.default_rng(n).integers(0, 200, size=n).astype(np.int32)
    off = _np(hg.scan_offsets(_cuda(c, torch.int32)))
    ref = np.zeros(n + 1, np.int64)
    np.cumsum(c, out=ref[1:])
    np.testing.assert_array_equal(off, ref)


def test_status_and_sum_reductions(hg):
    s = np.zeros(100000, np.uint8)
    s[5] = 1
    s[99999] = 4
    assert int(_np(hg.reduce_status(_cuda(s, torch.uint8)))[0]) == 5
    x = np.random.default_rng(1).integers(0, 1000, size=123457).astype(np.int32)
    assert int(_np(hg.sum_i32(_cuda(x, torch.int32)))[0]) == int(x.sum())


# ----------------------------------------------------------------------------- density and metrics

@pytest.mark.parametrize("kind", [0, 1], ids=["octree", "kd"])
def test_sample_density(hg, disk_grids, kind):
    model, grids, _, _ = disk_grids
    grid, tree, _ = grids[kind]
    pts = synth.sample_points(31, 50000)
    pts[:64] = np.array([[-1, -1, -1], [1, 1, 1], [0, 0, 0], [1, 0, 0]] * 16, np.float64)
    pts[64:70] = [[2, 0, 0], [0, -1.5, 0], [0, 0, 1.0000001], [-1, -1, -1], [0.5, 0.25, -0.125], [1, 1, -1]]
    ref_c, ref_r = oracle.sample_density(tree, pts)
    c, r = hg.sample_density(grid, _cuda(pts))
    np.testing.assert_array_equal(_np(c), ref_c)
    np.testing.assert_array_equal(_np(r), ref_r)


@pytest.mark.parametrize("mk", [lambda: synth.make_disk(), lambda: synth.make_torus(4, n_clumps=200),
                                lambda: synth.make_dyadic(2, level=2), lambda: synth.make_const(3.0)],
                         ids=["disk", "torus", "dyadic", "const"])
def test_model_density_and_tau(hg, mk):
    model = mk()
    dm = hg.load_model(model)
    pts = synth.sample_points(8, 20000)
    rt = _np(hg.model_density(dm, _cuda(pts)))
    np.testing.assert_allclose(rt, oracle.rho_true(model, pts), rtol=1e-14, atol=0)
    a, k, L = synth.endpoint_paths(9, 500)
    tt = _np(hg.model_tau(dm, _cuda(a), _cuda(k), _cuda(L), kappa=1.3))
    np.testing.assert_allclose(tt, oracle.tau_true(model, a, k, L, kappa=1.3), rtol=1e-9, atol=1e-12)


def test_delta_metrics_match_oracle(hg, disk_grids):
    model, grids, _, _ = disk_grids
    dm = hg.load_model(model)
    for kind in (0, 1):
        grid, tree, _ = grids[kind]
        pts = synth.sample_points(12, 100000)
        c, rg = hg.sample_density(grid, _cuda(pts))
        rt = hg.model_density(dm, _cuda(pts))
        st = _np(hg.diff_stats(rt, rg))
        _, org = oracle.sample_density(tree, pts)
        ort = oracle.rho_true(model, pts)
        assert st[0] == 100000
        assert st[2] == pytest.approx(oracle.population_std(ort - org), rel=1e-9)
        a, k, L = synth.endpoint_paths(13, 3000)
        tg, _, _ = hg.trace_rays(grid, _cuda(a), _cuda(k), _cuda(L))
        tt = hg.model_tau(dm, _cuda(a), _cuda(k), _cuda(L))
        st2 = _np(hg.diff_stats(tt, tg))
        ot = oracle.tau_true(model, a, k, L)
        og = oracle.trace(tree, a, k, smax=L)["tau"]
        assert st2[2] == pytest.approx(oracle.population_std(ot - og), rel=1e-7)
        assert st2[1] == pytest.approx((ot - og).mean(), rel=1e-6, abs=1e-12)


# ----------------------------------------------------------------------------- adjoint

@pytest.mark.parametrize("kind", [0, 1], ids=["octree", "kd"])
def test_adjoint_against_oracle_accumulation(hg, disk_grids, kind):
    model, grids, o, k = disk_grids
    grid, tree, _ = grids[kind]
    w = synth.adjoint_weights(5, o.shape[0])
    kappa = 1.7
    ref = oracle.trace(tree, o, k, kappa=kappa, emit=True)
    g64_ref = oracle.adjoint(tree.n_leaves, ref["seg_off"], ref["seg_cell"], ref["seg_ds"], w.astype(np.float64),
                             kappa)
    g64 = _np(hg.tau_gradient(grid, _cuda(o), _cuda(k), _cuda(w, torch.float32), kappa=kappa, grad_precision="fp64"))
    np.testing.assert_allclose(g64, g64_ref, rtol=1e-12, atol=1e-300)
    g32 = _np(hg.tau_gradient(grid, _cuda(o), _cuda(k), _cuda(w, torch.float32), kappa=kappa,
                              grad_precision="fp32")).astype(np.float64)
    # per-cell bound: gamma_n * sum |terms| with n = contributions + 1 (cast of each term)
    counts = np.bincount(ref["seg_cell"], minlength=tree.n_leaves).astype(np.float64)
    u = 2.0 ** -24
    gam = (counts + 1) * u / (1 - (counts + 1) * u)
    assert (np.abs(g32 - g64_ref) <= gam * np.abs(g64_ref) + 1e-30).all()


# ----------------------------------------------------------------------------- path segments

def _launches(hg, fn):
    n0 = hg.launch_count()
    out = fn()
    torch.cuda.synchronize()
    return out, hg.launch_count() - n0


@pytest.mark.parametrize("precision", ["fp64", "fp32k"])
@pytest.mark.parametrize("kind", [0, 1], ids=["octree", "kd"])
def test_forced_path_segments_match_oracle(hg, disk_grids, kind, precision):
    # every path of more than 3 estimated crossings is cut into up to 16 segments walked apart
    model, grids, o, k = disk_grids
    grid, tree, _ = grids[kind]
    O, K = _cuda(o), _cuda(k)
    ref = oracle.trace(tree, o, k, kappa=1.3)
    (tau, nc, st), n = _launches(hg, lambda: hg.trace_rays(grid, O, K, kappa=1.3, precision=precision,
                                                            split="force"))
    assert n == 5  # setup, queue order, split planner, walk, combine
    np.testing.assert_array_equal(_np(nc), ref["ncross"])
    np.testing.assert_array_equal(_np(st), ref["status"])
    _check_tau(_np(tau), ref["tau"], TAU_RTOL_FP64 if precision == "fp64" else TAU_RTOL_FP32K)
    (whole, nc1, _), n1 = _launches(hg, lambda: hg.trace_rays(grid, O, K, kappa=1.3, precision=precision,
                                                               split="off", schedule=3))
    assert n1 == 3
    np.testing.assert_array_equal(_np(nc1), ref["ncross"])
    if precision == "fp64":
        # the same segments, summed in groups: a few ulps apart, and some rays do differ
        _check_tau(_np(tau), _np(whole), 1e-13)
        assert (_np(tau) != _np(whole)).any()


@pytest.mark.parametrize("kind", [0, 1], ids=["octree", "kd"])
def test_forced_segments_with_path_ends(hg, disk_grids, kind):
    model, grids, _, _ = disk_grids
    grid, tree, _ = grids[kind]
    a, k, L = synth.endpoint_paths(78, 3001)
    for frac, prec in ((1.0, "fp64"), (0.37, "fp32k"), (0.9, "fp64")):
        smax = L * frac
        ref = oracle.trace(tree, a, k, smax=smax, kappa=2.5)
        tau, nc, st = hg.trace_rays(grid, _cuda(a), _cuda(k), _cuda(smax), kappa=2.5, precision=prec,
                                    split="force")
        np.testing.assert_array_equal(_np(nc), ref["ncross"])
        np.testing.assert_array_equal(_np(st), ref["status"])
        _check_tau(_np(tau), ref["tau"], TAU_RTOL_FP64 if prec == "fp64" else TAU_RTOL_FP32K)


@pytest.mark.parametrize("kind", [0, 1], ids=["octree", "kd"])
def test_forced_segments_degenerate_rays(hg, kind):
    # rays along planes, edges and through corners of a dyadic grid: cuts are only placed deep inside leaves
    model = synth.make_dyadic(7, level=2)
    bp = synth.BuildParams(kind=kind, delta_max=1e-3, max_level=4)
    grid = hg.load_grid(hg.build_grid(model, bp))
    tree = oracle.build_tree(model, bp)
    o, k = synth.degenerate_rays(levels=4, n_random=3000, seed=kind + 11)
    ref = oracle.trace(tree, o, k)
    tau, nc, st = hg.trace_rays(grid, _cuda(o), _cuda(k), split="force")
    np.testing.assert_array_equal(_np(nc), ref["ncross"])
    np.testing.assert_array_equal(_np(st), ref["status"])
    _check_tau(_np(tau), ref["tau"], TAU_RTOL_FP64)


@pytest.mark.parametrize("kind", [0, 1], ids=["octree", "kd"])
def test_forced_segments_adjoint(hg, disk_grids, kind):
    model, grids, o, k = disk_grids
    grid, tree, _ = grids[kind]
    w = synth.adjoint_weights(9, o.shape[0])
    ref = oracle.trace(tree, o, k, emit=True)
    g_ref = oracle.adjoint(tree.n_leaves, ref["seg_off"], ref["seg_cell"], ref["seg_ds"], w.astype(np.float64), 0.8)
    g, n = _launches(hg, lambda: hg.tau_gradient(grid, _cuda(o), _cuda(k), _cuda(w, torch.float32), kappa=0.8,
                                                 grad_precision="fp64", split="force"))
    assert n == 6  # setup, queue order, split planner, walk, combine, gradient slots to leaf order
    np.testing.assert_allclose(_np(g), g_ref, rtol=1e-12, atol=1e-300)


def _same_emission(out, ref, precision):
    np.testing.assert_array_equal(_np(out["ncross"]), ref["ncross"])
    np.testing.assert_array_equal(_np(out["status"]), ref["status"])
    np.testing.assert_array_equal(_np(out["seg_off"]), ref["seg_off"])
    np.testing.assert_array_equal(_np(out["seg_cell"]), ref["seg_cell"])
    if precision == "fp64":
        np.testing.assert_array_equal(_np(out["seg_ds"]), ref["seg_ds"])
        _check_tau(_np(out["tau"]), ref["tau"], TAU_RTOL_FP64)
    else:
        np.testing.assert_array_equal(_np(out["seg_ds"]), ref["seg_ds"].astype(np.float32))
        _check_tau(_np(out["tau"]), ref["tau"], TAU_RTOL_FP32K)


@pytest.mark.parametrize("split", ["force", "auto", "off"])
@pytest.mark.parametrize("kind", [0, 1], ids=["octree", "kd"])
def test_prepared_rays_emission_bit_exact(hg, disk_grids, kind, split):
    # segments emit their cells at offsets from the segment counts of the trace: the whole
    # sequences and lengths must come out bit for bit as the oracle's
    model, grids, o, k = disk_grids
    grid, tree, _ = grids[kind]
    ref = oracle.trace(tree, o, k, kappa=0.7, emit=True)
    R, n = _launches(hg, lambda: hg.prepare_rays(grid, _cuda(o), _cuda(k), split=split, schedule=3))
    assert n == (2 if split == "off" else 3)  # setup, queue order (, split planner)
    for prec in ("fp64", "fp32k"):
        _same_emission(R.emit(kappa=0.7, precision=prec), ref, prec)
    R.free()


@pytest.mark.parametrize("kind", [0, 1], ids=["octree", "kd"])
def test_prepared_rays_path_ends_and_gradient(hg, disk_grids, kind):
    model, grids, _, _ = disk_grids
    grid, tree, _ = grids[kind]
    a, k, L = synth.endpoint_paths(79, 4001)
    smax = 0.8 * L
    ref = oracle.trace(tree, a, k, smax=smax, kappa=1.9, emit=True)
    R = hg.prepare_rays(grid, _cuda(a), _cuda(k), _cuda(smax), split="force")
    _same_emission(R.emit(kappa=1.9), ref, "fp64")
    w = synth.adjoint_weights(13, a.shape[0])
    g_ref = oracle.adjoint(tree.n_leaves, ref["seg_off"], ref["seg_cell"], ref["seg_ds"], w.astype(np.float64), 1.9)
    g, n = _launches(hg, lambda: R.gradient(_cuda(w, torch.float32), kappa=1.9, grad_precision="fp64"))
    assert n == 3  # walk, combine, gradient slots to leaf order
    np.testing.assert_allclose(_np(g), g_ref, rtol=1e-12, atol=1e-300)
    # a second trace with other densities reuses the plan
    rho = torch.full((tree.n_leaves,), 2.0, dtype=torch.float64, device="cuda")
    tau2, nc2, _ = R.trace(kappa=1.0, rho=rho)
    np.testing.assert_array_equal(_np(nc2), ref["ncross"])
    seg_len = np.add.reduceat(ref["seg_ds"], ref["seg_off"][:-1][ref["ncross"] > 0]) if ref["seg_ds"].size else []
    got = _np(tau2)[ref["ncross"] > 0]
    np.testing.assert_allclose(got, 2.0 * np.asarray(seg_len), rtol=1e-12)


@pytest.mark.parametrize("split", ["force", "off"])
@pytest.mark.parametrize("kind", [0, 1], ids=["octree", "kd"])
def test_fused_trace_and_gradient(hg, disk_grids, kind, split):
    # optical depth, counts and the adjoint scatter in one walk, then an emission fill on the same plan
    model, grids, o, k = disk_grids
    grid, tree, _ = grids[kind]
    w = synth.adjoint_weights(17, o.shape[0])
    ref = oracle.trace(tree, o, k, kappa=1.2, emit=True)
    g_ref = oracle.adjoint(tree.n_leaves, ref["seg_off"], ref["seg_cell"], ref["seg_ds"], w.astype(np.float64), 1.2)
    R = hg.prepare_rays(grid, _cuda(o), _cuda(k), split=split, schedule=3)
    W = _cuda(w, torch.float32)
    (tau, nc, st, g64), n = _launches(hg, lambda: R.trace_gradient(W, kappa=1.2, grad_precision="fp64"))
    assert n == (3 if split == "force" else 2)  # walk (, combine), gradient slots to leaf order
    np.testing.assert_array_equal(_np(nc), ref["ncross"])
    np.testing.assert_array_equal(_np(st), ref["status"])
    _check_tau(_np(tau), ref["tau"], TAU_RTOL_FP64)
    np.testing.assert_allclose(_np(g64), g_ref, rtol=1e-12, atol=1e-300)
    tau32, nc32, _, g32 = R.trace_gradient(W, kappa=1.2, precision="fp32k", grad_precision="fp32")
    np.testing.assert_array_equal(_np(nc32), ref["ncross"])
    _check_tau(_np(tau32), ref["tau"], TAU_RTOL_FP32K)
    counts = np.bincount(ref["seg_cell"], minlength=tree.n_leaves).astype(np.float64)
    u = 2.0 ** -24
    gam = (counts + 1) * u / (1 - (counts + 1) * u)
    assert (np.abs(_np(g32).astype(np.float64) - g_ref) <= gam * np.abs(g_ref) + 1e-30).all()
    off = hg.scan_offsets(nc32)
    cell, ds = R.fill(off)
    np.testing.assert_array_equal(_np(cell), ref["seg_cell"])
    np.testing.assert_array_equal(_np(ds), ref["seg_ds"])
    R.free()


@pytest.mark.parametrize("split", ["force", "auto", "off"])
@pytest.mark.parametrize("kind", [0, 1], ids=["octree", "kd"])
def test_single_pass_emission_bit_exact(hg, disk_grids, kind, split):
    # the trace stages every emitted cell; a copy puts them at the scanned offsets: the whole
    # sequences and lengths must be the oracle's, with or without the gradient, scattered in the
    # walk or in the copy (from the staged lengths: FP32 ones after an FP32-Kahan trace)
    model, grids, o, k = disk_grids
    grid, tree, _ = grids[kind]
    w = synth.adjoint_weights(23, o.shape[0])  # in [0, 1): every adjoint term is >= 0
    ref = oracle.trace(tree, o, k, kappa=0.9, emit=True)
    g_ref = oracle.adjoint(tree.n_leaves, ref["seg_off"], ref["seg_cell"], ref["seg_ds"], w.astype(np.float64), 0.9)
    R = hg.prepare_rays(grid, _cuda(o), _cuda(k), split=split, schedule=3)
    W = _cuda(w, torch.float32)
    for prec, with_w, adj in (("fp64", True, "walk"), ("fp64", True, "copy"), ("fp32k", False, "copy"),
                              ("fp64", False, "copy"), ("fp32k", True, "walk"), ("fp32k", True, "copy")):
        out = R.emit_single_pass(kappa=0.9, precision=prec, w=W if with_w else None, grad_precision="fp64",
                                 adjoint=adj)
        _same_emission(out, ref, prec)
        if with_w:
            # FP64 lengths: the oracle's terms, summed in another order; FP32 staged lengths: each
            # term within 2^-24 relative, so the (non-negative) sum within 2^-23
            rtol = 2.0 ** -23 if (prec == "fp32k" and adj == "copy") else 1e-12
            np.testing.assert_allclose(_np(out["grad"]), g_ref, rtol=rtol, atol=1e-300)
    R.free()


@pytest.mark.parametrize("kind", [0, 1], ids=["octree", "kd"])
def test_copy_adjoint_ignores_capacity_and_overflow(hg, disk_grids, kind):
    # the adjoint scattered during the copy covers every crossing: when the emission capacity
    # drops entries (their rays flagged HG_RAY_OVERFLOW), and when the staging pool overflowed
    # (a fill walk and a gradient walk take over)
    model, grids, o, k = disk_grids
    grid, tree, _ = grids[kind]
    a, kk, L = synth.endpoint_paths(82, 3001)
    w = synth.adjoint_weights(24, a.shape[0])
    ref = oracle.trace(tree, a, kk, smax=L, kappa=1.3, emit=True)
    g_ref = oracle.adjoint(tree.n_leaves, ref["seg_off"], ref["seg_cell"], ref["seg_ds"], w.astype(np.float64), 1.3)
    R = hg.prepare_rays(grid, _cuda(a), _cuda(kk), _cuda(L), split="force")
    W = _cuda(w, torch.float32)
    counts = np.bincount(ref["seg_cell"], minlength=tree.n_leaves).astype(np.float64)
    u = 2.0 ** -24
    gam32 = (counts + 1) * u / (1 - (counts + 1) * u)  # FP32 terms and FP32 running sums
    for gp in ("fp64", "fp32"):
        tau, nc, st, _ = R.trace_stage(kappa=1.3)
        off = hg.scan_offsets(nc)
        total = int(off[-1].item())
        cap = total // 2
        cell, ds, g = R.emit_staged_gradient(off, W, kappa=1.3, grad_precision=gp, capacity=cap, status=st)
        if gp == "fp64":
            np.testing.assert_allclose(_np(g), g_ref, rtol=1e-12, atol=1e-300)
        else:
            assert (np.abs(_np(g).astype(np.float64) - g_ref) <= gam32 * g_ref + 1e-30).all()
        so = ref["seg_off"]
        cut = (so[1:] > cap) & (so[1:] > so[:-1])  # rays with an entry at or beyond the capacity
        np.testing.assert_array_equal((_np(st) & hg.RAY_OVERFLOW) != 0, cut)
        np.testing.assert_array_equal(_np(cell)[:cap], ref["seg_cell"][:cap])
        np.testing.assert_array_equal(_np(ds)[:cap], ref["seg_ds"][:cap])
        assert cut.any() and not cut.all()
    tau, nc, st, _ = R.trace_stage(kappa=1.3, stage_per_ray=-3)  # pool of 3 chunks: overflows
    off = hg.scan_offsets(nc)
    cell, ds, g = R.emit_staged_gradient(off, W, kappa=1.3, grad_precision="fp64", status=st)
    np.testing.assert_array_equal(_np(cell), ref["seg_cell"])
    np.testing.assert_array_equal(_np(ds), ref["seg_ds"])
    np.testing.assert_array_equal(_np(st), ref["status"])
    np.testing.assert_allclose(_np(g), g_ref, rtol=1e-12, atol=1e-300)
    R.free()


@pytest.mark.parametrize("kind", [0, 1], ids=["octree", "kd"])
def test_single_pass_emission_pool_overflow_falls_back(hg, disk_grids, kind):
    # a pool of 3 chunks cannot hold the crossings: the copy is skipped and the fill walk emits
    model, grids, o, k = disk_grids
    grid, tree, _ = grids[kind]
    a, kk, L = synth.endpoint_paths(81, 3001)
    ref = oracle.trace(tree, a, kk, smax=L, emit=True)
    R = hg.prepare_rays(grid, _cuda(a), _cuda(kk), _cuda(L), split="force")
    out = R.emit_single_pass(stage_per_ray=-3)
    _same_emission(out, ref, "fp64")
    out2 = R.emit_single_pass()  # the default pool holds them
    _same_emission(out2, ref, "fp64")
    R.free()


def test_prepared_fill_needs_a_trace_when_paths_are_split(hg, disk_grids):
    model, grids, o, k = disk_grids
    grid, tree, _ = grids[0]
    R = hg.prepare_rays(grid, _cuda(o), _cuda(k), split="force")
    off = torch.zeros(o.shape[0] + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(hg.HgError, match="hg_rays_trace"):
        R.fill(off, capacity=0)
    R.free()
    R2 = hg.prepare_rays(grid, _cuda(o[:0]), _cuda(k[:0]))
    tau, nc, st = R2.trace()
    assert tau.numel() == 0
    R2.free()


def test_step_limit_turns_splitting_off(hg, disk_grids):
    model, grids, o, k = disk_grids
    grid, tree, _ = grids[0]
    _, n = _launches(hg, lambda: hg.trace_rays(grid, _cuda(o), _cuda(k), split="force", max_steps=7))
    assert n == 3


def test_taufn_autograd_and_finite_differences(hg, disk_grids):
    model, grids, o, k = disk_grids
    grid, tree, H = grids[1]
    O, K = _cuda(o[:2000]), _cuda(k[:2000])
    rho = torch.tensor(H.leaf_rho, dtype=torch.float64, device="cuda", requires_grad=True)
    w = torch.tensor(synth.adjoint_weights(6, 2000), device="cuda").to(torch.float64)
    tau = hg.TauFn.apply(rho, grid, O, K, None, 1.1)
    tau_plain, _, _ = hg.trace_rays(grid, O, K, kappa=1.1)
    np.testing.assert_array_equal(_np(tau), _np(tau_plain))
    (w * tau).sum().backward()
    g = _np(rho.grad)
    rng = np.random.default_rng(0)
    hit = np.nonzero(g)[0]
    cells = np.concatenate([rng.choice(hit, 50, replace=False), rng.integers(0, grid.n_leaves, 50)])
    base = rho.detach().clone()
    for c in cells:
        h = 1e-3 * max(1.0, float(base[c]))
        vals = []
        for sgn in (1, -1):
            r = base.clone()
            r[c] += sgn * h
            t, _ = hg.trace_rays_rho(grid, O, K, r, kappa=1.1)
            vals.append(float((w * t).sum()))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert fd == pytest.approx(g[c], rel=1e-6, abs=1e-10)


# ----------------------------------------------------------------------------- interaction points

def _same_interactions(hg, grid, tree, o, k, ti, smax=None, kappa=1.0, **opt):
    ref = oracle.interact(tree, o, k, ti, smax=smax, kappa=kappa)
    cell, t, nc, st = hg.find_interactions(grid, _cuda(o), _cuda(k), _cuda(ti), None if smax is None else _cuda(smax),
                                           kappa=kappa, **opt)
    np.testing.assert_array_equal(_np(cell), ref["cell"])
    np.testing.assert_array_equal(_np(nc), ref["ncross"])
    np.testing.assert_array_equal(_np(st), ref["status"])
    np.testing.assert_array_equal(_np(t), ref["t"])  # the same FP64 operations in the same order
    return ref


# the default launch shape of the search is 3 blocks per SM (80 registers); min_blocks=4 runs the 64-register build
@pytest.mark.parametrize("shape", [dict(), dict(schedule=1), dict(schedule=2, block=128), dict(min_blocks=4)],
                         ids=["auto", "s1", "s2", "occ4"])
@pytest.mark.parametrize("kind", [0, 1], ids=["octree", "kd"])
def test_interaction_points_match_oracle(hg, disk_grids, kind, shape):
    model, grids, o, k = disk_grids
    grid, tree, _ = grids[kind]
    u = np.random.default_rng(31).uniform(size=o.shape[0])
    ti = -np.log(u) * 0.2  # a mix of interactions and escapes
    ti[:5] = 0.0
    ti[5:10] = -1.0
    ti[10:15] = np.inf
    ref = _same_interactions(hg, grid, tree, o, k, ti, kappa=1.1, **shape)
    assert (ref["cell"] >= 0).any() and (ref["cell"] < 0).any()


@pytest.mark.parametrize("kind", [0, 1], ids=["octree", "kd"])
def test_interaction_points_path_ends_and_bad_inputs(hg, disk_grids, kind):
    model, grids, _, _ = disk_grids
    grid, tree, _ = grids[kind]
    a, k, L = synth.endpoint_paths(83, 3001)
    ti = np.random.default_rng(4).exponential(0.05, 3001)
    ti[:7] = np.nan
    _same_interactions(hg, grid, tree, a, k, ti, smax=0.6 * L, kappa=2.0)
    rng = np.random.default_rng(8)
    o = rng.uniform(-3, 3, size=(2000, 3))
    kk = synth.isotropic_dirs(rng, 2000)
    kk[:10] = 0.0
    _same_interactions(hg, grid, tree, o, kk, rng.exponential(0.1, 2000))


# ----------------------------------------------------------------------------- long neighbor lists
# A wall with more than 16 neighbors keeps only its list head and its rope node on the device: a path whose exit
# point misses the head is located top-down from the rope node (the leaf found there tested like a listed
# neighbor, the root searched when it fails).  The clumpy torus makes such walls at small sizes.

LONG_LIST_GRIDS = [(synth.TREE_OCTREE, 3e-4, 6), (synth.TREE_KD, 1e-4, 8)]


def _long_wall_rays(H, tree, seed, per_wall=40):
    """Rays from inside each leaf that has a long wall to points of that wall: uniform on the face, on the
    corners of its neighbors, and on the face's own edges and corners."""
    cnt = np.diff(H.nbr_off)
    idx = np.nonzero(cnt > 16)[0]
    rng = np.random.default_rng(seed)
    o, k = [], []
    for i in idx:
        a, w = int(i // 6), int(i % 6)
        ax = w // 2
        lo, hi = tree.leaf_lo[a], tree.leaf_hi[a]
        nb = H.nbr_id[H.nbr_off[i]:H.nbr_off[i + 1]]
        for j in range(per_wall):
            p = lo + rng.random(3) * (hi - lo)
            q = lo + rng.random(3) * (hi - lo)
            if j % 4 == 1:  # a corner of a listed neighbor
                c = int(nb[rng.integers(0, nb.size)])
                q = np.where(rng.random(3) < 0.5, tree.leaf_lo[c], tree.leaf_hi[c])
            elif j % 4 == 2:  # the face's own edges and corners
                q = np.where(rng.random(3) < 0.5, lo, hi)
            q[ax] = hi[ax] if w % 2 else lo[ax]
            d = q - p
            n = np.linalg.norm(d)
            if n == 0.0:
                continue
            o.append(p)
            k.append(d / n)
    return np.array(o), np.array(k)


@pytest.mark.parametrize("kind,dmax,level", LONG_LIST_GRIDS, ids=["octree", "kd"])
def test_long_lists_search_from_the_rope_node(hg, kind, dmax, level):
    model = synth.workload_torus_1e7()[0]
    bp = synth.BuildParams(kind=kind, delta_max=dmax, max_level=level, seed=synth.BASE_SEED)
    H = hg.build_grid(model, bp)
    G = hg.load_grid(H, validate=True)
    assert G.long_walls > 0
    tree = oracle.wrap_tree(H.kind, H.node_lo, H.node_hi, H.child_first, H.node_leaf, H.leaf_rho)
    o, k = _long_wall_rays(H, tree, 90 + kind)
    assert o.shape[0] > 400
    for shape in (dict(), dict(split="force"), dict(schedule=1, smem_nodes=0)):
        _compare(hg, G, tree, o, k, **shape)
    _compare(hg, G, tree, o, k, precision="fp32k")
    e, d = synth.emission_rays(91 + kind, 20000)
    _compare(hg, G, tree, e, d)
    ref = oracle.interact(tree, o, k, np.random.default_rng(kind).exponential(0.5, o.shape[0]), kappa=3.0)
    cell, t, nc, st = hg.find_interactions(G, _cuda(o), _cuda(k),
                                           _cuda(np.random.default_rng(kind).exponential(0.5, o.shape[0])),
                                           kappa=3.0)
    np.testing.assert_array_equal(_np(cell), ref["cell"])
    np.testing.assert_array_equal(_np(t), ref["t"])
    np.testing.assert_array_equal(_np(nc), ref["ncross"])


# ----------------------------------------------------------------------------- ropes
# The rope walk (hg_load_grid_ropes): the next leaf from the exit wall's rope, located below the rope's node
# when that is not a leaf, instead of from the neighbor list.  Same contract, so the same oracle.

@pytest.fixture(scope="module")
def rope_grids(hg, disk_grids):
    model, grids, o, k = disk_grids
    out = {}
    for kind in (0, 1):
        _, tree, H = grids[kind]
        G = hg.load_grid(H, validate=True, nav="ropes")
        assert G.nav == hg.NAV_ROPES and G.n_tail == 1
        out[kind] = (G, tree, H)
    return out


ROPE_SHAPES = [dict(), dict(schedule=1, smem_nodes=0), dict(split="force"), dict(schedule=2, block=128),
               dict(min_blocks=4)]


@pytest.mark.parametrize("kind", [0, 1], ids=["octree", "kd"])
@pytest.mark.parametrize("shape", ROPE_SHAPES, ids=[str(s) for s in ROPE_SHAPES])
def test_rope_walk_sequences_bit_exact(hg, disk_grids, rope_grids, kind, shape):
    model, grids, o, k = disk_grids
    G, tree, H = rope_grids[kind]
    ref, _ = _compare(hg, G, tree, o, k, **shape)
    assert ref["ncross"].sum() > 0
    _compare(hg, G, tree, o, k, precision="fp32k", **shape)


@pytest.mark.parametrize("kind", [0, 1], ids=["octree", "kd"])
def test_rope_walk_path_ends_degenerate_rays_and_interactions(hg, rope_grids, kind):
    G, tree, H = rope_grids[kind]
    a, d, L = synth.endpoint_paths(78, 3001)
    _compare(hg, G, tree, a, d, smax=L, kappa=2.5)
    wo, wk = _wall_rays(tree, 79 + kind, 4000)
    _compare(hg, G, tree, wo, wk)
    _compare(hg, G, tree, wo, wk, split="force")
    o, k = synth.emission_rays(80, 3000)
    ti = np.random.default_rng(kind).exponential(2.0, 3000)
    _same_interactions(hg, G, tree, o, k, ti, kappa=3.0)


@pytest.mark.parametrize("kind", [0, 1], ids=["octree", "kd"])
def test_rope_walk_degenerate_rays_on_adaptive_grid(hg, kind):
    model = synth.make_torus(21, n_clumps=20)
    bp = synth.BuildParams(kind=kind, delta_max=1e-3, use_q=True, q_max=0.9, max_level=5)
    H = hg.build_grid(model, bp)
    grid = hg.load_grid(H, nav="ropes", ropes=hg.build_ropes(H))
    tree = oracle.build_tree(model, bp)
    o, k = synth.degenerate_rays(levels=5, n_random=3000, seed=kind + 9)
    _compare(hg, grid, tree, o, k)
    _compare(hg, grid, tree, o, k, split="force", smem_nodes=0)


@pytest.mark.parametrize("kind", [0, 1], ids=["octree", "kd"])
def test_rope_walk_emission_and_adjoint(hg, disk_grids, rope_grids, kind):
    model, grids, o, k = disk_grids
    G, tree, H = rope_grids[kind]
    w = synth.adjoint_weights(81, o.shape[0])
    ref = oracle.trace(tree, o, k, emit=True)
    gr = oracle.adjoint(tree.n_leaves, ref["seg_off"], ref["seg_cell"], ref["seg_ds"], w.astype(np.float64))
    O, K, W = _cuda(o), _cuda(k), _cuda(w, torch.float32)
    R = hg.prepare_rays(G, O, K, split="force")
    sp = R.emit_single_pass(w=W, grad_precision="fp64")
    torch.cuda.synchronize()
    np.testing.assert_array_equal(_np(sp["seg_off"]), ref["seg_off"])
    np.testing.assert_array_equal(_np(sp["seg_cell"]), ref["seg_cell"])
    np.testing.assert_array_equal(_np(sp["seg_ds"]), ref["seg_ds"])
    np.testing.assert_allclose(_np(sp["grad"]), gr, rtol=1e-12, atol=0)
    R.free()
    g = hg.tau_gradient(G, O, K, W, grad_precision="fp64")
    np.testing.assert_allclose(_np(g), gr, rtol=1e-12, atol=0)


@pytest.mark.parametrize("kind,plane,axis,dmax", SPLIT_VARIANTS, ids=SPLIT_IDS)
def test_rope_walk_on_split_location_variants(hg, kind, plane, axis, dmax):
    model, bp, n_rays, seed = synth.workload_disk_small()
    bp.kind, bp.split_plane, bp.split_axis, bp.delta_max = kind, plane, axis, dmax
    H = hg.build_grid(model, bp)
    T = oracle.build_tree(model, bp)
    G = hg.load_grid(H, validate=True, nav="ropes")
    o, k = synth.emission_rays(seed + 21, 4000)
    _compare(hg, G, T, o, k)
    wo, wk = _wall_rays(T, seed + 22, 3000)
    _compare(hg, G, T, wo, wk, split="force")


@pytest.mark.parametrize("kind", [0, 1], ids=["octree", "kd"])
def test_rope_walk_through_the_allocation_free_entry_point(hg, disk_grids, rope_grids, kind):
    # the allocation-free optical-depth pass walks rope grids with the same kernels
    model, grids, o, k = disk_grids
    G, tree, H = rope_grids[kind]
    ref = oracle.trace(tree, o, k, kappa=1.3)
    tau, nc, st = hg.trace_rays_noalloc(G, _cuda(o), _cuda(k), kappa=1.3)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(_np(nc), ref["ncross"])
    np.testing.assert_array_equal(_np(st), ref["status"])
    _check_tau(_np(tau), ref["tau"], TAU_RTOL_FP64)


def test_rope_and_list_grids_in_one_batch_match_oracle(hg):
    grids, trees, begins = _uneven_batch(hg, ropes=True)
    assert {g.nav for g in grids} == {hg.NAV_NEIGHBOR_LISTS, hg.NAV_ROPES}
    n = begins[-1]
    o, k = synth.emission_rays(synth.config_seed(4) + 15, n)
    b = hg.Batch(grids, begins)
    O, K = _cuda(o), _cuda(k)
    for prec, rtol in (("fp64", TAU_RTOL_FP64), ("fp32k", TAU_RTOL_FP32K)):
        tau, nc, st = b.trace(O, K, kappa=1.4, precision=prec)
        torch.cuda.synchronize()
        for i, t in enumerate(trees):
            s = slice(begins[i], begins[i + 1])
            ref = oracle.trace(t, o[s], k[s], kappa=1.4)
            np.testing.assert_array_equal(_np(nc[s]), ref["ncross"])
            np.testing.assert_array_equal(_np(st[s]), ref["status"])
            _check_tau(_np(tau[s]), ref["tau"], rtol)


# ----------------------------------------------------------------------------- batching and tuning

def test_batch_matches_single_grid_launches(hg):
    specs = synth.batch_specs(n_grids=6, rays_lo=1e3, rays_hi=2e4, leaves_lo=2e3, leaves_hi=3e4)
    grids, os_, ks, begins = [], [], [], [0]
    for i, sp in enumerate(specs):
        bp = synth.BuildParams(kind=sp["kind"], delta_max=1.0 / sp["target_leaves"], max_level=7, seed=sp["seed"])
        grids.append(hg.load_grid(hg.build_grid(sp["model"], bp)))
        o, k = synth.emission_rays(sp["seed"], sp["n_rays"])
        os_.append(o)
        ks.append(k)
        begins.append(begins[-1] + sp["n_rays"])
    O = _cuda(np.concatenate(os_))
    K = _cuda(np.concatenate(ks))
    b = hg.Batch(grids, begins)
    for prec in ("fp64", "fp32k"):
        tau, nc, st = b.trace(O, K, kappa=1.4, precision=prec)
        for i, g in enumerate(grids):
            s = slice(begins[i], begins[i + 1])
            t1, n1, s1 = hg.trace_rays(g, O[s].contiguous(), K[s].contiguous(), kappa=1.4, precision=prec,
                                       split="off")
            np.testing.assert_array_equal(_np(tau[s]), _np(t1))
            np.testing.assert_array_equal(_np(nc[s]), _np(n1))
            np.testing.assert_array_equal(_np(st[s]), _np(s1))


def _uneven_batch(hg, ropes=False):
    """Seven grids of uneven size for the batched launch: octree and k-d tree of each of the disk,
    the clump-free ring and the ring with clumps (seeded parameters), one more disk octree, and one
    grid that gets no rays; ray counts from 0 to ~2e4.  ropes: every other grid loaded for the rope
    walk."""
    rng = np.random.default_rng(synth.config_seed(4) + 101)
    specs = []
    for kind in (synth.TREE_OCTREE, synth.TREE_KD):
        for mk in ("disk", "ring", "clumps"):
            specs.append((kind, mk))
    specs.append((synth.TREE_OCTREE, "disk"))
    grids, trees, begins = [], [], [0]
    n_rays = [int(x) for x in np.exp(rng.uniform(np.log(800), np.log(20000), len(specs)))]
    n_rays[3] = 0
    for (kind, mk), nr in zip(specs, n_rays):
        sub = int(rng.integers(0, 2 ** 31))
        if mk == "disk":
            model = synth.make_disk(h_R=float(rng.uniform(0.15, 0.35)), h_z=float(rng.uniform(0.02, 0.08)))
        elif mk == "ring":
            model = synth.make_torus(sub, n_clumps=0, R0=float(rng.uniform(0.4, 0.6)), r_tube=0.15,
                                     tau_eq=float(rng.uniform(1.0, 10.0)))
        else:
            model = synth.make_torus(sub, n_clumps=int(rng.integers(50, 300)), R0=0.5, r_tube=0.2,
                                     tau_eq=float(rng.uniform(1.0, 10.0)))
        target = float(np.exp(rng.uniform(np.log(2e3), np.log(4e4))))
        bp = synth.BuildParams(kind=kind, delta_max=1.0 / target, max_level=7, seed=sub)
        H = hg.build_grid(model, bp)
        grids.append(hg.load_grid(H, nav="ropes" if ropes and len(grids) % 2 else "lists"))
        trees.append(oracle.wrap_tree(H.kind, H.node_lo, H.node_hi, H.child_first, H.node_leaf, H.leaf_rho))
        begins.append(begins[-1] + nr)
    return grids, trees, begins


def test_batch_matches_oracle_on_uneven_grids(hg):
    # the batched persistent launch against the oracle, grid by grid: counts and statuses bit-exact, tau
    # within 1e-6 (FP64) and 1e-5 (FP32-Kahan) of the oracle's FP64 sums; once from inside the domain to
    # its exit, once along paths with both ends drawn in the domain (s_max)
    grids, trees, begins = _uneven_batch(hg)
    leaves = [g.n_leaves for g in grids]
    assert max(leaves) > 4 * min(leaves)
    n = begins[-1]
    o, k = synth.emission_rays(synth.config_seed(4) + 5, n)
    a, d, L = synth.endpoint_paths(synth.config_seed(4) + 6, n)
    b = hg.Batch(grids, begins)
    for rays in ((o, k, None), (a, d, L)):
        O, K = _cuda(rays[0]), _cuda(rays[1])
        S = None if rays[2] is None else _cuda(rays[2])
        refs = [oracle.trace(t, rays[0][begins[i]:begins[i + 1]], rays[1][begins[i]:begins[i + 1]],
                             smax=None if rays[2] is None else rays[2][begins[i]:begins[i + 1]], kappa=1.4)
                for i, t in enumerate(trees)]
        for prec, rtol in (("fp64", TAU_RTOL_FP64), ("fp32k", TAU_RTOL_FP32K)):
            tau, nc, st = b.trace(O, K, S, kappa=1.4, precision=prec)
            torch.cuda.synchronize()
            for i, ref in enumerate(refs):
                s = slice(begins[i], begins[i + 1])
                np.testing.assert_array_equal(_np(nc[s]), ref["ncross"])
                np.testing.assert_array_equal(_np(st[s]), ref["status"])
                _check_tau(_np(tau[s]), ref["tau"], rtol)
            assert int(_np(nc).sum()) > 0


def test_batch_graph_capture_replay(hg):
    specs = synth.batch_specs(n_grids=3, rays_lo=1e3, rays_hi=5e3, leaves_lo=2e3, leaves_hi=1e4)
    grids, os_, ks, begins = [], [], [], [0]
    for sp in specs:
        bp = synth.BuildParams(kind=sp["kind"], delta_max=1.0 / sp["target_leaves"], max_level=7, seed=sp["seed"])
        grids.append(hg.load_grid(hg.build_grid(sp["model"], bp)))
        o, k = synth.emission_rays(sp["seed"], sp["n_rays"])
        os_.append(o)
        ks.append(k)
        begins.append(begins[-1] + sp["n_rays"])
    O = _cuda(np.concatenate(os_))
    K = _cuda(np.concatenate(ks))
    b = hg.Batch(grids, begins)
    ref = [_np(x) for x in b.trace(O, K)]
    out = (torch.empty(b.n_rays, dtype=torch.float64, device="cuda"),
           torch.empty(b.n_rays, dtype=torch.int32, device="cuda"),
           torch.empty(b.n_rays, dtype=torch.uint8, device="cuda"))
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.trace(O, K, out=out)
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        b.trace(O, K, out=out)
    for t in out:
        t.zero_()
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    for r, x in zip(ref, out):
        np.testing.assert_array_equal(r, _np(x))


def test_autotune_keeps_results(hg, disk_grids):
    model, grids, o, k = disk_grids
    grid, tree, _ = grids[1]
    O, K = _cuda(o), _cuda(k)
    before = hg.trace_rays(grid, O, K)
    cfg, ms = hg.autotune(grid, O, K)
    assert cfg["block"] in (128, 256) and cfg["schedule"] in (1, 2, 3) and cfg["min_blocks"] in (3, 4) and ms > 0
    after = hg.trace_rays(grid, O, K)
    # counts are exact; tau may differ in the grouping of additions when the tuned schedule splits paths
    np.testing.assert_array_equal(_np(before[1]), _np(after[1]))
    _check_tau(_np(after[0]), _np(before[0]), 1e-13)


# ----------------------------------------------------------------------------- full-size disk grids

@pytest.fixture(scope="module")
def disk_1e6(hg):
    out = {}
    for kind in (0, 1):
        model, bp, n_rays, seed = synth.workload_disk_1e6(kind)
        H = hg.build_grid(model, bp)
        T = oracle.build_tree(model, bp)
        np.testing.assert_array_equal(H.child_first, T.child)
        np.testing.assert_array_equal(H.leaf_rho, T.leaf_rho)
        out[kind] = (hg.load_grid(H), T)
        out[kind + 2] = (hg.load_grid(H, nav="ropes"), T)
    o, k = synth.emission_rays(seed, n_rays)
    return model, out, o, k


@pytest.mark.parametrize("nav", ["lists", "ropes"])
@pytest.mark.parametrize("kind", [0, 1], ids=["octree", "kd"])
def test_disk_1e6_leaves_1e6_rays(hg, disk_1e6, kind, nav):
    model, grids, o, k = disk_1e6
    grid, tree = grids[kind + (2 if nav == "ropes" else 0)]
    O, K = _cuda(o), _cuda(k)
    ref = oracle.trace(tree, o, k)
    for prec in ("fp64", "fp32k"):
        tau, nc, st = hg.trace_rays(grid, O, K, precision=prec)
        np.testing.assert_array_equal(_np(nc), ref["ncross"])
        np.testing.assert_array_equal(_np(st), ref["status"])
        _check_tau(_np(tau), ref["tau"], TAU_RTOL_FP64 if prec == "fp64" else TAU_RTOL_FP32K)
    # full sequences on a sample of rays, traced in the same launch shape as the benchmark
    sel = np.random.default_rng(kind).choice(o.shape[0], 20000, replace=False)
    _compare(hg, grid, tree, o[sel], k[sel])


def test_single_leaf_grid(hg):
    model = synth.make_const(2.0)
    bp = synth.BuildParams(kind=1, delta_max=2.0, max_level=3)
    grid = hg.load_grid(hg.build_grid(model, bp))
    tree = oracle.build_tree(model, bp)
    assert tree.n_leaves == 1
    o, k = synth.emission_rays(4, 500)
    _compare(hg, grid, tree, o, k)


# ----------------------------------------------------------------------------- full-size torus + clumps grid
# (1e7-leaf class): builder decisions sampled against the
# oracle's node evaluation, and sampled ray sequences against the oracle walk on the same grid


@pytest.fixture(scope="module")
def torus_full(hg):
    model, bp, n_rays, seed = synth.workload_torus_1e7()
    H = hg.build_grid(model, bp)
    return model, bp, H, seed


def test_torus_full_size_builder_decisions_sampled(hg, torus_full):
    model, bp, H, seed = torus_full
    assert 9e6 < H.n_leaves < 1.1e7
    rng = np.random.default_rng(1)
    leaves = H.leaf_node[rng.choice(H.n_leaves, 300, replace=False)]
    parent = np.full(H.n_nodes, -1, np.int64)
    internal = np.nonzero(H.child_first >= 0)[0]
    nch = 2
    for c in range(nch):
        parent[H.child_first[internal] + c] = internal
    for nd in leaves:
        st = oracle.node_stats(model, bp, H.level[nd], H.index[nd])
        assert st[0] == 0.0                      # the oracle would not split this leaf either
        assert st[1] == H.leaf_rho[H.node_leaf[nd]]  # same Monte Carlo density, bit for bit
        p = parent[nd]
        sp = oracle.node_stats(model, bp, H.level[p], H.index[p])
        assert sp[0] == 1.0                      # and it would split the parent


@pytest.fixture(scope="module")
def torus_tree(torus_full):
    model, bp, H, seed = torus_full
    return oracle.wrap_tree(H.kind, H.node_lo, H.node_hi, H.child_first, H.node_leaf, H.leaf_rho)


def test_torus_full_size_1e6_rays_match_oracle(hg, torus_full, torus_tree):
    # the full grid, 1e6 rays: crossing counts and statuses bit-exact against the oracle, tau within 1e-6
    # (FP64) and 1e-5 (FP32-Kahan with the FP64 wall test) of the oracle's FP64 tau, in the launch shape the
    # benchmark uses (work-ordered queue, automatic path segments); full cell sequences on a sample
    model, bp, H, seed = torus_full
    grid = hg.load_grid(H)
    o, k = synth.emission_rays(seed, 1_000_000)
    ref = oracle.trace(torus_tree, o, k)
    O, K = _cuda(o), _cuda(k)
    for prec, rtol in (("fp64", TAU_RTOL_FP64), ("fp32k", TAU_RTOL_FP32K)):
        tau, nc, st = hg.trace_rays(grid, O, K, precision=prec)
        np.testing.assert_array_equal(_np(nc), ref["ncross"])
        np.testing.assert_array_equal(_np(st), ref["status"])
        _check_tau(_np(tau), ref["tau"], rtol)
    assert ref["ncross"].mean() > 20
    sel = np.random.default_rng(3).choice(o.shape[0], 20000, replace=False)
    _compare(hg, grid, torus_tree, o[sel], k[sel])
    _compare(hg, grid, torus_tree, o[sel], k[sel], precision="fp32k")


def test_torus_full_size_gradient(hg, torus_full, torus_tree):
    # the adjoint at full size (1e7 rays, the full k-d grid): FP64 and FP32 reductions on the GPU against
    # the oracle's FP64 accumulation of its own emitted segments (in ten 1e6-ray chunks): FP64 within
    # 2 (n_c + 10) u per cell (all terms positive, only the order differs: n_c atomic additions against n_c
    # additions plus ten chunk sums), FP32 within gamma_{n_c + 1}; and central differences on 100 cells
    model, bp, H, seed = torus_full
    grid = hg.load_grid(H)
    n = 10_000_000
    o, k = synth.emission_rays(seed, n)
    w = synth.adjoint_weights(seed + 3, n)
    O, K, W = _cuda(o), _cuda(k), _cuda(w, torch.float32)
    g64 = _np(hg.tau_gradient(grid, O, K, W, grad_precision="fp64"))
    g32 = _np(hg.tau_gradient(grid, O, K, W, grad_precision="fp32")).astype(np.float64)
    g_ref = np.zeros(H.n_leaves, np.float64)
    counts = np.zeros(H.n_leaves, np.int64)
    chunk = 1_000_000
    for a in range(0, n, chunk):
        r = oracle.trace(torus_tree, o[a:a + chunk], k[a:a + chunk], emit=True)
        g_ref += oracle.adjoint(H.n_leaves, r["seg_off"], r["seg_cell"], r["seg_ds"],
                                w[a:a + chunk].astype(np.float64))
        counts += np.bincount(r["seg_cell"], minlength=H.n_leaves)
        del r
    err64 = np.abs(g64 - g_ref)
    assert (err64 <= 2.3e-16 * (counts + 10) * g_ref + 1e-300).all(), float((err64 / np.maximum(g_ref, 1e-300)).max())
    u = 2.0 ** -24
    gam = (counts + 1) * u / (1 - (counts + 1) * u)
    err32 = np.abs(g32 - g_ref)
    assert (err32 <= gam * g_ref + 1e-30).all()
    hit = np.nonzero(g_ref > 0)[0]
    assert hit.size > 100_000
    assert float(np.median(err32[hit] / g_ref[hit])) < 1e-6
    assert (g64[counts == 0] == 0).all() and (g32[counts == 0] == 0).all()
    # central differences: tau is linear in rho, and rays that miss the cell give identical bits both ways
    rng = np.random.default_rng(5)
    pw = g_ref[hit] / g_ref[hit].sum()
    cells = np.concatenate([rng.choice(hit, 50, replace=False), rng.choice(hit, 50, replace=False, p=pw)])
    rho = torch.tensor(H.leaf_rho, dtype=torch.float64, device="cuda")
    Wd = W.double()
    for c in cells:
        h = 1e-3 * max(1.0, float(rho[c]))
        rp, rm = rho.clone(), rho.clone()
        rp[c] += h
        rm[c] -= h
        tp, _ = hg.trace_rays_rho(grid, O, K, rp)
        tm, _ = hg.trace_rays_rho(grid, O, K, rm)
        fd = float((Wd * (tp - tm)).sum()) / (2 * h)
        assert fd == pytest.approx(g_ref[c], rel=1e-6)
