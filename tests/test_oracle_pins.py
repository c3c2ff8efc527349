"""Pins of the FP64 oracle against closed forms, invariants and brute force.

Nothing here compares the oracle with itself: each check uses a value the
mathematics fixes (exact integrals, exact volumes, leaf counts of uniform
refinement), a published generator output, or a brute-force search that
shares no logic with the oracle's descent and walk.
"""
import dataclasses
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------------------- generator and quadrature

def test_splitmix64_published_outputs():
    vals = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if l.startswith("0x")]
    for j, v in enumerate(vals):
        assert oracle.splitmix_output(0, j) == v


@pytest.mark.parametrize("deg", list(range(0, 23)))
def test_gk15_exact_for_polynomials(deg):
    # a 15-point Kronrod rule integrates polynomials up to degree 22 exactly
    c = np.zeros(deg + 1)
    c[deg] = 1.0
    a, b = -0.3, 1.7
    exact = (b ** (deg + 1) - a ** (deg + 1)) / (deg + 1)
    got = oracle.quad_poly(c, a, b, adaptive=False)
    assert got == pytest.approx(exact, rel=1e-13, abs=1e-14)


def test_gk15_not_exact_beyond_degree_22():
    c = np.zeros(31)
    c[30] = 1.0
    exact = 2.0 / 31.0
    assert abs(oracle.quad_poly(c, -1.0, 1.0, adaptive=False) - exact) > 1e-8
    # the adaptive driver refines until the embedded Gauss estimate agrees
    assert oracle.quad_poly(c, -1.0, 1.0, adaptive=True) == pytest.approx(exact, rel=1e-12)


# ----------------------------------------------------------------------------- model densities

def test_disk_density_closed_form():
    m = synth.make_disk()
    pts = np.array([[0, 0, 0], [0.25, 0, 0.03], [0.0, -0.5, -0.06], [0.6, 0.8, 0.0]], np.float64)
    exp = [1.0, math.exp(-2.0), math.exp(-4.0), math.exp(-4.0)]
    np.testing.assert_allclose(oracle.rho_true(m, pts), exp, rtol=1e-15)


def test_torus_density_hard_edge_and_clump_peak():
    m = synth.make_torus(1, n_clumps=0)
    rho0 = m.params[2]
    assert rho0 == pytest.approx(25.0)
    got = oracle.rho_true(m, np.array([[0.5, 0, 0], [0, 0.5, 0.19], [0.0, 0.0, 0.0], [0.71, 0, 0], [0.5, 0, 0.21]]))
    np.testing.assert_array_equal(got, [rho0, rho0, 0.0, 0.0, 0.0])
    mc = synth.make_torus(2, n_clumps=1)
    c = mc.table[0]
    # clump peak: tube plus amplitude A; outside the 5-sigma sphere only the tube remains
    assert oracle.rho_true(mc, c[None, :3])[0] == pytest.approx(mc.params[2] + c[4], rel=1e-15)
    off = c[:3] + np.array([5.01 * c[3], 0, 0])
    inside_tube = (math.hypot(off[0], off[1]) - 0.5) ** 2 + off[2] ** 2 < 0.04
    assert oracle.rho_true(mc, off[None])[0] == (mc.params[2] if inside_tube else 0.0)


def test_clump_mass_normalisation():
    # the truncated Gaussian amplitude makes each clump hold its nominal mass
    frac = synth.clump_truncated_fraction()
    from scipy.integrate import quad
    s = 0.01
    A = 1.0 / ((2 * math.pi) ** 1.5 * s ** 3 * frac)
    radial, _ = quad(lambda r: 4 * math.pi * r * r * A * math.exp(-0.5 * r * r / (s * s)), 0, 5 * s,
                     epsabs=0, epsrel=1e-13)
    assert radial == pytest.approx(1.0, rel=1e-12)


# ----------------------------------------------------------------------------- tree construction

def _bp(**kw):
    return synth.BuildParams(**kw)


@pytest.mark.parametrize("L", [1, 2, 3])
def test_uniform_refinement_counts_and_octree_kd_equivalence(L):
    m = synth.make_const(1.0)
    to = oracle.build_tree(m, _bp(kind=synth.TREE_OCTREE, delta_max=-1.0, max_level=L))
    tk = oracle.build_tree(m, _bp(kind=synth.TREE_KD, delta_max=-1.0, max_level=L))
    assert to.n_leaves == 8 ** L
    assert tk.n_leaves == 2 ** (3 * L)
    # one octree level equals three k-d levels (Sect. 2.1): identical leaf boxes
    ko = sorted(map(tuple, np.hstack([to.leaf_lo, to.leaf_hi])))
    kk = sorted(map(tuple, np.hstack([tk.leaf_lo, tk.leaf_hi])))
    assert ko == kk


def _layered(axis, level=2, low=1.0, high=10.0):
    """Piecewise-constant model that varies along one axis only: `low` below the domain's middle on
    that axis, `high` above (a dyadic lattice, x fastest in the table)."""
    n = 1 << level
    zz, yy, xx = np.indices((n, n, n))
    upper = (xx, yy, zz)[axis] >= n // 2
    vals = np.where(upper, high, low).astype(np.float64).reshape(-1)
    lo, hi = np.full(3, -1.0), np.full(3, 1.0)
    return synth.Model(synth.MODEL_DYADIC, np.array([float(level)], np.float64), vals.reshape(-1, 1),
                       float(vals.sum()) * float(np.prod((hi - lo) / n)), lo, hi, "layered")


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_gradient_axis_splits_across_the_density_jump(axis):
    # density constant on each side of the plane through the middle of `axis` (Sect. 2.2, the
    # orientation of the strongest gradient): the root is halved on that axis; the cyclic rule
    # halves it on x whatever the density
    m = _layered(axis)
    tg = oracle.build_tree(m, _bp(kind=synth.TREE_KD, delta_max=0.1, max_level=3, split_axis=1))
    tc = oracle.build_tree(m, _bp(kind=synth.TREE_KD, delta_max=0.1, max_level=3, split_axis=0))
    want = [0, 0, 0]
    want[axis] = 1
    assert tg.lvl[tg.child[0]].tolist() == want
    assert tc.lvl[tc.child[0]].tolist() == [1, 0, 0]
    # each half is uniform: no positive gradient below the root, so the halves split cyclically
    c = tg.child[0]
    for h in (c, c + 1):
        if tg.child[h] >= 0:
            depth = int(tg.lvl[h].sum())
            grand = tg.lvl[tg.child[h]] - tg.lvl[h]
            assert grand.tolist() == [1 if a == depth % 3 else 0 for a in range(3)] or tg.lvl[h][depth % 3] >= 3


def test_gradient_axis_on_uniform_density_is_the_cyclic_tree():
    m = synth.make_const(2.0)
    kw = dict(kind=synth.TREE_KD, use_delta=False, use_tau=True, tau_max=0.9, max_level=4)
    tg = oracle.build_tree(m, _bp(split_axis=1, **kw))
    tc = oracle.build_tree(m, _bp(split_axis=0, **kw))
    np.testing.assert_array_equal(tg.lvl, tc.lvl)
    np.testing.assert_array_equal(tg.idx, tc.idx)
    np.testing.assert_array_equal(tg.child, tc.child)


def test_gradient_axis_halves_no_axis_beyond_max_level():
    # always subdivide, max level 1: every axis is halved exactly once, so the leaves are the 2x2x2
    # lattice although the density only varies along y
    m = _layered(1, level=1)
    t = oracle.build_tree(m, _bp(kind=synth.TREE_KD, delta_max=-1.0, max_level=1, split_axis=1))
    assert t.n_leaves == 8
    assert t.lvl.max(axis=0).tolist() == [1, 1, 1]
    boxes = sorted(map(tuple, np.hstack([t.leaf_lo, t.leaf_hi])))
    lattice = sorted((x, y, z, x + 1.0, y + 1.0, z + 1.0) for x in (-1.0, 0.0) for y in (-1.0, 0.0)
                     for z in (-1.0, 0.0))
    assert boxes == lattice


def test_mass_criterion_exact_on_uniform_model():
    # uniform density: delta = V/V_dom exactly, so delta_max = 1/64 stops at 64 leaves
    m = synth.make_const(3.0)
    to = oracle.build_tree(m, _bp(kind=synth.TREE_OCTREE, delta_max=1.0 / 64, max_level=10))
    tk = oracle.build_tree(m, _bp(kind=synth.TREE_KD, delta_max=1.0 / 64, max_level=10))
    assert to.n_leaves == 64 and tk.n_leaves == 64
    to2 = oracle.build_tree(m, _bp(kind=synth.TREE_OCTREE, delta_max=1.0 / 64 * 0.999, max_level=10))
    assert to2.n_leaves == 512


def test_node_optical_depth_closed_form():
    # Eq. 2 for a cube of side s with uniform rho: tau = kappa rho sqrt(3) s
    rho0, kappa = 2.0, 1.5
    m = synth.make_const(rho0)
    for L in range(0, 5):
        st = oracle.node_stats(m, _bp(kind=synth.TREE_OCTREE, kappa=kappa, max_level=10), [L, L, L], [0, 0, 0])
        s = 2.0 / 2 ** L
        assert st[4] == pytest.approx(kappa * rho0 * math.sqrt(3.0) * s, rel=1e-15)
    # box a x b x c
    st = oracle.node_stats(m, _bp(kind=synth.TREE_KD, kappa=kappa, max_level=10), [1, 0, 0], [1, 0, 0])
    a, b, c = 1.0, 2.0, 2.0
    assert st[4] == pytest.approx(kappa * rho0 * a * b * c * math.sqrt(a * a + b * b + c * c) / (a * b * c),
                                  rel=1e-15)


def test_tau_criterion_uniform_count():
    # tau_node = kappa rho sqrt(3) s <= tau_max stops refinement: s = 2 / 2^L
    rho0 = 1.0
    m = synth.make_const(rho0)
    tau_max = 0.5
    L = math.ceil(math.log2(2 * math.sqrt(3.0) / tau_max))
    t = oracle.build_tree(m, _bp(kind=synth.TREE_OCTREE, use_delta=False, use_tau=True, tau_max=tau_max,
                                 max_level=10))
    assert t.n_leaves == 8 ** L


def _quantile_lattice_model():
    # a level-2 lattice (64 cells of side 0.5) whose sorted values are 1 x 56, 2, 4, 8 x 6, placed by a
    # fixed permutation; powers of two make every leaf's Monte Carlo mean exact (Eq. 1)
    vals = np.array([1.0] * 56 + [2.0, 4.0] + [8.0] * 6)
    vals = vals[np.random.default_rng(11).permutation(64)]
    lo, hi = np.full(3, -1.0), np.full(3, 1.0)
    return synth.Model(synth.MODEL_DYADIC, np.array([2.0]), vals.reshape(-1, 1), float(vals.sum()) * 0.125,
                       lo, hi, "quantile lattice")


@pytest.mark.parametrize("kind", [synth.TREE_OCTREE, synth.TREE_KD])
def test_tau_max_recipe_known_quantile(kind):
    # Sect. 4.1: tau_max is the leaf optical depth at sorted position floor(0.9 N).  With no effective mass
    # threshold every node splits down to max level 2, giving the 64 lattice cells as leaves (k-d: depth 6);
    # each leaf's Eq. 2 depth is kappa v sqrt(3) s with s = 1/2.  N = 64, so position floor(57.6) = 57 holds
    # v = 4; positions 56 and 58 hold 2 and 8, so an off-by-one, a ceiling or rounding fails.
    m = _quantile_lattice_model()
    kappa = 1.5
    bp = _bp(kind=kind, delta_max=1e-12, max_level=2, kappa=kappa, use_tau=True, tau_max=1e9)
    t = oracle.build_tree(m, dataclasses.replace(bp, use_tau=False))
    assert t.n_leaves == 64
    unit = kappa * math.sqrt(3.0) * 0.5
    # fraction -> value at position floor(fraction * 64) (clamped to 63)
    for frac, v in ((0.9, 4.0), (0.89, 2.0), (0.875, 2.0), (0.92, 8.0), (0.0, 1.0), (1.0, 8.0), (0.5, 1.0)):
        assert oracle.tau_max_recipe(m, bp, fraction=frac) == pytest.approx(v * unit, rel=4e-16), frac


def test_density_dispersion_limits():
    claims = json.load(open(os.path.join(GOLDEN, "paper_claims.json")))["q_limits"]
    m = synth.make_const(1.0)
    st = oracle.node_stats(m, _bp(kind=synth.TREE_OCTREE, max_level=10), [2, 2, 2], [1, 2, 3])
    assert st[5] == claims["uniform"]
    mt = synth.make_torus(3, n_clumps=0)
    # the level-3 node [0.25, 0.5] x [0, 0.25] x [0, 0.25] straddles the inner tube edge at R = 0.3
    st = oracle.node_stats(mt, _bp(kind=synth.TREE_OCTREE, max_level=10), [3, 3, 3], [5, 4, 4])
    assert st[5] == claims["hard_edge"]
    # a node fully inside the tube has q = 0, one fully outside has rho_max = 0 and q = 0
    st = oracle.node_stats(mt, _bp(kind=synth.TREE_OCTREE, max_level=10), [5, 5, 5], [23, 16, 16])
    assert st[5] == 0.0 and st[1] == pytest.approx(mt.params[2])
    st = oracle.node_stats(mt, _bp(kind=synth.TREE_OCTREE, max_level=10), [3, 3, 3], [0, 0, 0])
    assert st[5] == 0.0 and st[1] == 0.0


def test_q_criterion_refines_hard_edge_to_max_level():
    mt = synth.make_torus(3, n_clumps=0)
    t = oracle.build_tree(mt, _bp(kind=synth.TREE_OCTREE, use_delta=False, use_q=True, q_max=0.99, max_level=5))
    edge = t.q[t.leaf_node] > 0.99
    assert edge.any()
    # every leaf that still straddles the edge sits at the maximum level
    assert (t.lvl[t.leaf_node][edge] == 5).all()


def test_node_list_order_and_geometry(disk_small):
    model, bp, t, _ = disk_small
    depth = t.lvl[:, 0]
    assert (np.diff(depth) >= 0).all()  # breadth-first: children appended at the end
    internal = np.where(t.child >= 0)[0]
    assert (np.diff(t.child[internal]) == 8).all()
    assert (t.leaf[t.leaf_node] == np.arange(t.n_leaves)).all()
    assert (np.diff(t.leaf_node) > 0).all()
    # leaf volumes sum to the domain volume exactly (dyadic boxes)
    vol = np.prod(t.leaf_hi - t.leaf_lo, axis=1)
    assert math.fsum(vol) == 8.0
    # children tile their parent
    for n in internal[:200]:
        f = t.child[n]
        ch = slice(f, f + 8)
        assert math.fsum(np.prod(t.hi[ch] - t.lo[ch], axis=1)) == np.prod(t.hi[n] - t.lo[n])


def test_leaf_masses_sum_to_total_mass(disk_small):
    model, bp, t, _ = disk_small
    total = t.mass[t.leaf_node].sum()
    assert total == pytest.approx(model.m_tot, rel=5e-3)
    # exact on the uniform and piecewise-constant models
    m = synth.make_const(2.0)
    tu = oracle.build_tree(m, _bp(kind=synth.TREE_KD, delta_max=1e-3, max_level=6))
    assert tu.mass[tu.leaf_node].sum() == pytest.approx(m.m_tot, rel=1e-14)
    md = synth.make_dyadic(5, level=2)
    td = oracle.build_tree(md, _bp(kind=synth.TREE_OCTREE, delta_max=-1.0, max_level=3))
    assert td.mass[td.leaf_node].sum() == pytest.approx(md.m_tot, rel=1e-12)


def test_disk_total_mass_independent_quadrature():
    # the synthetic-input module's total mass vs a separate 2-D tensor Gauss-Legendre sum over quadrants
    m = synth.make_disk()
    h, hz = m.params[1], m.params[2]
    x, w = np.polynomial.legendre.leggauss(400)
    # split [0,1] into pieces graded toward 0 to follow the cusp at R = 0
    edges = np.concatenate([[0.0], np.geomspace(1e-6, 1.0, 40)])
    xs, ws = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        xs.append(0.5 * (b - a) * x + 0.5 * (a + b))
        ws.append(0.5 * (b - a) * w)
    xs = np.concatenate(xs)
    ws = np.concatenate(ws)
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    W = np.outer(ws, ws)
    radial = 4.0 * np.sum(W * np.exp(-np.sqrt(X * X + Y * Y) / h))
    mz = 2 * hz * (1 - math.exp(-1 / hz))
    assert radial * mz == pytest.approx(m.m_tot, rel=1e-7)


def test_kd_about_half_the_leaves_of_octree_sanity(disk_small):
    # loose sanity only (Sect. 3.3 prose): the k-d tree needs fewer leaves at equal delta_max
    model, bp, to, _ = disk_small
    tk = oracle.build_tree(model, _bp(kind=synth.TREE_KD, delta_max=bp.delta_max, max_level=bp.max_level,
                                      seed=bp.seed))
    ratio = tk.n_leaves / to.n_leaves
    assert 0.2 < ratio < 0.9


def test_octree_and_kd_nodes_share_samples():
    # a node's Monte Carlo samples depend on its box only, so an octree node and the
    # k-d node with the same box get identical statistics
    m = synth.make_disk()
    for l, i in [([2, 2, 2], [1, 2, 3]), ([4, 4, 4], [7, 8, 9])]:
        so = oracle.node_stats(m, _bp(kind=synth.TREE_OCTREE, max_level=12), l, i)
        sk = oracle.node_stats(m, _bp(kind=synth.TREE_KD, max_level=12), l, i)
        np.testing.assert_array_equal(so[1:], sk[1:])


# ----------------------------------------------------------------------------- point location

def _lattice_points(rng, n, L):
    ticks = np.array([-1 + 2 * j / 2 ** L for j in range(2 ** L + 1)])
    p = rng.uniform(-1, 1, size=(n, 3))
    mask = rng.random((n, 3)) < 0.6
    p = np.where(mask, ticks[rng.integers(0, len(ticks), size=(n, 3))], p)
    k = rng.choice([-1.0, -0.0, 0.0, 1.0, 0.3, -0.7], size=(n, 3))
    return p, k


def test_locate_matches_brute_force(disk_small):
    model, bp, t, _ = disk_small
    rng = np.random.default_rng(11)
    p = rng.uniform(-1, 1, size=(3000, 3))
    k = synth.isotropic_dirs(rng, 3000)
    pl, kl = _lattice_points(rng, 3000, 6)
    P = np.vstack([p, pl])
    K = np.vstack([k, kl])
    got = oracle.locate(t, P, K)
    ref, hits = oracle.brute_locate(t, P, K)
    inside = hits == 1
    # every point of the closed domain lies in exactly one leaf, unless it sits on a
    # lower domain face with a direction leaving the domain
    leaving = np.any(((P == -1.0) & (K < 0)) | ((P == 1.0) & (K > 0)), axis=1)
    assert (hits <= 1).all()
    assert (inside == ~leaving).all()
    np.testing.assert_array_equal(got[inside], ref[inside])
    assert (got[~inside] == -1).all()


def test_sample_density_matches_leaf_values(disk_small):
    model, bp, t, _ = disk_small
    pts = synth.sample_points(3, 2000)
    cell, rho = oracle.sample_density(t, pts)
    ref, hits = oracle.brute_locate(t, pts, np.zeros_like(pts))
    np.testing.assert_array_equal(cell, ref)
    np.testing.assert_array_equal(rho, t.leaf_rho[ref])


# ----------------------------------------------------------------------------- path calculation

def _exact_chord(o, k):
    """Chord of the ray o + t k (t >= 0) through [-1,1]^3 in exact rational arithmetic."""
    t0, t1 = Fraction(0), None
    for a in range(3):
        oa, ka = Fraction(float(o[a])), Fraction(float(k[a]))
        if ka == 0:
            continue
        ta, tb = (Fraction(-1) - oa) / ka, (Fraction(1) - oa) / ka
        lo, hi = min(ta, tb), max(ta, tb)
        t0 = max(t0, lo)
        t1 = hi if t1 is None else min(t1, hi)
    return max(Fraction(0), t1 - t0)


def test_brute_force_sequences(disk_small):
    model, bp, t, seed = disk_small
    o, k = synth.emission_rays(99, 150)
    r = oracle.trace(t, o, k, emit=True, threads=1)
    for i in range(o.shape[0]):
        a, b = r["seg_off"][i], r["seg_off"][i + 1]
        cells, tin, ds = oracle.brute_sequence(t, o[i], k[i], 0.0, float(_exact_chord(o[i], k[i])) * 2)
        keep = ds > 0
        np.testing.assert_array_equal(r["seg_cell"][a:b], cells[keep])
        np.testing.assert_allclose(r["seg_ds"][a:b], ds[keep], rtol=1e-12, atol=1e-15)


def test_uniform_density_tau_closed_form():
    rho0, kappa = 2.5, 1.5
    m = synth.make_const(rho0)
    t = oracle.build_tree(m, _bp(kind=synth.TREE_KD, delta_max=1.0 / 200, max_level=8))
    o, k = synth.emission_rays(5, 400)
    r = oracle.trace(t, o, k, kappa=kappa)
    for i in range(400):
        chord = float(_exact_chord(o[i], k[i]))
        assert r["tau"][i] == pytest.approx(kappa * rho0 * chord, rel=1e-13)


def test_segment_lengths_sum_to_chord(disk_small):
    model, bp, t, seed = disk_small
    o, k = synth.emission_rays(seed, 500)
    r = oracle.trace(t, o, k, emit=True)
    sums = np.add.reduceat(r["seg_ds"], r["seg_off"][:-1]) if r["seg_ds"].size else np.zeros(500)
    for i in range(500):
        assert sums[i] == pytest.approx(float(_exact_chord(o[i], k[i])), rel=1e-12)
    assert (r["status"] == 0).all()


def test_outside_origins_and_path_end():
    m = synth.make_const(1.0)
    t = oracle.build_tree(m, _bp(kind=synth.TREE_OCTREE, delta_max=-1.0, max_level=2))
    o = np.array([[-3.0, 0.1, 0.2], [-3.0, 5.0, 0.2], [0.1, 0.2, 0.3], [2.0, 0.0, 0.0]])
    k = np.array([[1.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0], [1.0, 0.0, 0.0]])
    r = oracle.trace(t, o, k, emit=True)
    assert r["tau"][0] == pytest.approx(2.0, rel=1e-15)  # enters at x=-1, leaves at x=1
    assert r["ncross"][0] == 4
    assert r["ncross"][1] == 0 and r["tau"][1] == 0.0  # misses
    assert r["tau"][2] == pytest.approx(0.7, rel=1e-15)
    assert r["ncross"][3] == 0  # behind the box
    # path end inside a cell
    r2 = oracle.trace(t, o[:1], k[:1], smax=np.array([2.3]))
    assert r2["tau"][0] == pytest.approx(0.3, rel=1e-13)


def test_degenerate_rays_are_complete():
    # rays inside split planes, through edges and corners: sum ds still equals the chord
    m = synth.make_const(1.0)
    for kind in (synth.TREE_OCTREE, synth.TREE_KD):
        t = oracle.build_tree(m, _bp(kind=kind, delta_max=-1.0, max_level=3))
        o, k = synth.degenerate_rays(levels=3, n_random=300)
        r = oracle.trace(t, o, k, emit=True)
        assert (r["status"] == 0).all()
        for i in range(o.shape[0]):
            a, b = r["seg_off"][i], r["seg_off"][i + 1]
            assert r["seg_ds"][a:b].sum() == pytest.approx(float(_exact_chord(o[i], k[i])), rel=1e-13, abs=1e-15)
            # consecutive cells are distinct leaves
            c = r["seg_cell"][a:b]
            assert (c[1:] != c[:-1]).all()


# ----------------------------------------------------------------------------- quality metrics

def test_tau_true_closed_forms():
    m = synth.make_disk()
    h, hz = m.params[1], m.params[2]
    o = np.array([[0, 0, -1.0], [-1.0, 0, 0]])
    k = np.array([[0, 0, 1.0], [1.0, 0, 0]])
    got = oracle.tau_true(m, o, k, np.array([2.0, 2.0]))
    assert got[0] == pytest.approx(2 * hz * (1 - math.exp(-1 / hz)), rel=1e-10)
    assert got[1] == pytest.approx(2 * h * (1 - math.exp(-1 / h)), rel=1e-10)
    mt = synth.make_torus(4, n_clumps=0)
    rho0, R0, r = mt.params[2], mt.params[0], mt.params[1]
    for z in [0.0, 0.1, 0.19]:
        got = oracle.tau_true(mt, np.array([[-1.0, 0, z]]), np.array([[1.0, 0, 0]]), np.array([2.0]))[0]
        assert got == pytest.approx(rho0 * 4 * math.sqrt(r * r - z * z), rel=1e-9)
    mc = synth.make_torus(6, n_clumps=1, tau_eq=1e-300)
    c = mc.table[0]
    got = oracle.tau_true(mc, np.array([[-1.0, c[1], c[2]]]), np.array([[1.0, 0, 0]]), np.array([2.0]))[0]
    from scipy.special import erf
    s = c[3]
    assert got == pytest.approx(c[4] * s * math.sqrt(2 * math.pi) * erf(5 / math.sqrt(2)), rel=1e-9)


def test_delta_metrics_vanish_when_grid_represents_model():
    md = synth.make_dyadic(9, level=2)
    t = oracle.build_tree(md, _bp(kind=synth.TREE_KD, delta_max=-1.0, max_level=3))
    pts = synth.sample_points(4, 5000)
    _, rg = oracle.sample_density(t, pts)
    rt = oracle.rho_true(md, pts)
    assert oracle.population_std(rt - rg) < 1e-13 * rt.max()
    a, k, L = synth.endpoint_paths(8, 300)
    tg = oracle.trace(t, a, k, smax=L)["tau"]
    tt = oracle.tau_true(md, a, k, L)
    assert oracle.population_std(tt - tg) < 1e-10 * tt.max()


def test_population_std_two_pass():
    x = 1e8 + np.array([4.0, 7.0, 13.0, 16.0])
    assert oracle.population_std(x) == pytest.approx(math.sqrt(22.5), rel=1e-12)


# ----------------------------------------------------------------------------- adjoint

def test_adjoint_matches_central_differences(disk_small):
    model, bp, t, seed = disk_small
    o, k = synth.emission_rays(seed + 1, 300)
    w = synth.adjoint_weights(seed, 300).astype(np.float64)
    kappa = 1.3
    r = oracle.trace(t, o, k, kappa=kappa, emit=True)
    g = oracle.adjoint(t.n_leaves, r["seg_off"], r["seg_cell"], r["seg_ds"], w, kappa)
    rng = np.random.default_rng(0)
    cells = np.concatenate([rng.choice(np.nonzero(g)[0], 5, replace=False), rng.integers(0, t.n_leaves, 3)])
    base = t.leaf_rho.copy()
    node_lo, node_hi = t.lo, t.hi
    for c in cells:
        hstep = 1e-3 * max(1.0, abs(base[c]))
        vals = []
        for sgn in (+1, -1):
            rho = base.copy()
            rho[c] += sgn * hstep
            tw = oracle.wrap_tree(t.kind, node_lo, node_hi, t.child, t.leaf, rho)
            vals.append(np.dot(w, oracle.trace(tw, o, k, kappa=kappa)["tau"]))
        fd = (vals[0] - vals[1]) / (2 * hstep)
        assert fd == pytest.approx(g[c], rel=1e-7, abs=1e-9)


# ----------------------------------------------------------------------------- interaction points

def test_interaction_uniform_closed_form():
    # uniform rho0: the interaction lies at t = tau_int / (kappa rho0) along a unit direction, in the leaf
    # containing that point (brute force); paths too short end at the exact chord without interaction
    rho0, kappa = 2.5, 1.5
    m = synth.make_const(rho0)
    t = oracle.build_tree(m, _bp(kind=synth.TREE_KD, delta_max=1.0 / 200, max_level=8))
    n = 400
    o, k = synth.emission_rays(6, n)
    chord = np.array([float(_exact_chord(o[i], k[i])) for i in range(n)])
    f = np.random.default_rng(2).uniform(0.02, 1.5, n)
    ti = f * kappa * rho0 * chord
    r = oracle.interact(t, o, k, ti, kappa=kappa)
    assert (r["status"] == 0).all()
    inside = f < 1 - 1e-9
    np.testing.assert_allclose(r["t"][inside], ti[inside] / (kappa * rho0), rtol=1e-12)
    pts = o[inside] + k[inside] * r["t"][inside][:, None]
    ref, hits = oracle.brute_locate(t, pts, k[inside])
    assert (hits == 1).all()
    np.testing.assert_array_equal(r["cell"][inside], ref)
    out = f > 1 + 1e-9
    assert (r["cell"][out] == -1).all()
    np.testing.assert_allclose(r["t"][out], chord[out], rtol=1e-12)


def test_interaction_matches_prefix_sums_of_the_path(disk_small):
    # disk grid: the walk stops in the first emitted segment at which kappa * (running sum of rho*ds, left
    # to right) reaches tau_int; the solved t lies in that leaf's slab interval and reproduces tau_int
    model, bp, t, seed = disk_small
    n = 300
    o, k = synth.emission_rays(seed + 7, n)
    kappa = 1.3
    r = oracle.trace(t, o, k, kappa=kappa, emit=True)
    ti = np.random.default_rng(9).uniform(0.0, 1.2, n) * r["tau"]
    q = oracle.interact(t, o, k, ti, kappa=kappa)
    assert (q["status"] == 0).all()
    for i in range(n):
        a, b = r["seg_off"][i], r["seg_off"][i + 1]
        cells, ds = r["seg_cell"][a:b], r["seg_ds"][a:b]
        rho = t.leaf_rho[cells]
        S = np.cumsum(rho * ds)
        hit = np.nonzero(kappa * S >= ti[i])[0]
        if hit.size == 0:
            assert q["cell"][i] == -1 and q["ncross"][i] == b - a
            continue
        j = int(hit[0])
        assert q["cell"][i] == cells[j] and q["ncross"][i] == j + 1
        bc, tin, bds = oracle.brute_sequence(t, o[i], k[i], 0.0, 2 * float(_exact_chord(o[i], k[i])))
        m = np.nonzero(bc == cells[j])[0][0]
        t_in, t_out = tin[m], tin[m] + bds[m]
        assert t_in - 1e-12 <= q["t"][i] <= t_out + 1e-12
        S_before = S[j - 1] if j else 0.0
        assert kappa * (S_before + rho[j] * (q["t"][i] - t_in)) == pytest.approx(ti[i], rel=1e-9, abs=1e-12)


def test_interaction_nonpositive_and_nan_tau(disk_small):
    model, bp, t, seed = disk_small
    n = 20
    o, k = synth.emission_rays(seed + 8, n)
    r = oracle.trace(t, o, k, emit=True)
    q = oracle.interact(t, o, k, np.full(n, -1.0))
    np.testing.assert_array_equal(q["cell"], r["seg_cell"][r["seg_off"][:-1]])
    assert (q["t"] == 0.0).all() and (q["ncross"] == 1).all()
    q2 = oracle.interact(t, o, k, np.full(n, np.nan))
    assert (q2["status"] == oracle.RAY_BADINPUT).all() and (q2["cell"] == -1).all()


# ----------------------------------------------------------------------------- split locations (Sect. 2.2)
# Non-dyadic planes: the barycentric octree and the equal-mass and equal-mean-density k-d trees.  The root's
# planes are pinned against positions the model fixes analytically (the estimates come from n_ran draws,
# hence the tolerances, about 5 standard deviations at 4000 draws); deeper trees against exact tiling,
# brute-force location, brute-force sequences and the uniform-density closed form.

def _slabs_x(values):
    """Piecewise-constant model varying along x only: len(values) = 2^L slabs of equal width."""
    n = len(values)
    L = int(round(math.log2(n)))
    zz, yy, xx = np.indices((n, n, n))
    vals = np.asarray(values, np.float64)[xx].reshape(-1)
    lo, hi = np.full(3, -1.0), np.full(3, 1.0)
    return synth.Model(synth.MODEL_DYADIC, np.array([float(L)]), vals.reshape(-1, 1),
                       float(vals.sum()) * float(np.prod((hi - lo) / n)), lo, hi, "slabs")


def _root_planes(model, kind, plane, n_ran=4000):
    t = oracle.build_tree(model, _bp(kind=kind, delta_max=1e-12, max_level=1, n_ran=n_ran, split_plane=plane))
    c0 = t.child[0]
    assert c0 > 0
    return t.hi[c0]  # the lower child's upper corner holds the cut positions


def test_barycentric_octree_root_at_centre_of_mass():
    # rho = 1 for x < 0 and 3 for x >= 0: centre of mass ((1)(-1/2) + (3)(1/2)) / 4 = 1/4 on x, 0 on y and z
    c = _root_planes(_slabs_x([1.0, 3.0]), synth.TREE_OCTREE, synth.PLANE_BARYCENTRE)
    assert c[0] == pytest.approx(0.25, abs=0.05)
    assert abs(c[1]) < 0.05 and abs(c[2]) < 0.05
    # uniform density: the centre of mass is the geometric centre
    c = _root_planes(synth.make_const(1.0), synth.TREE_OCTREE, synth.PLANE_BARYCENTRE)
    assert np.abs(c).max() < 0.06


def test_equal_mass_kd_root_halves_the_mass():
    # rho = 1 for x < 0, 3 for x >= 0: total mass 4 (per unit y-z area / 4), half reached at 1 + 3c = 2, c = 1/3
    c = _root_planes(_slabs_x([1.0, 3.0]), synth.TREE_KD, synth.PLANE_EQUAL_MASS)
    assert c[0] == pytest.approx(1.0 / 3.0, abs=0.05)
    assert c[1] == 1.0 and c[2] == 1.0   # the cyclic root cuts x only
    # rho = 3 below 0, 1 above: mirror image, c = -1/3
    c = _root_planes(_slabs_x([3.0, 1.0]), synth.TREE_KD, synth.PLANE_EQUAL_MASS)
    assert c[0] == pytest.approx(-1.0 / 3.0, abs=0.05)
    # uniform density: the median of the draws
    c = _root_planes(synth.make_const(1.0), synth.TREE_KD, synth.PLANE_EQUAL_MASS)
    assert abs(c[0]) < 0.06


def test_equal_mean_density_kd_root():
    # slabs of width 1/2 on x with rho 1, 1, 7, 1: left mean (1 + 7c) / (1 + c) equals right mean
    # (4 - 7c) / (1 - c) only at c = 1/3 (left mean below the right one before it, above after it)
    c = _root_planes(_slabs_x([1.0, 1.0, 7.0, 1.0]), synth.TREE_KD, synth.PLANE_EQUAL_DENSITY)
    assert c[0] == pytest.approx(1.0 / 3.0, abs=0.05)
    # uniform density (rho = 1, so every mean is exactly 1): all planes tie and the middle draw pair wins
    c = _root_planes(synth.make_const(1.0), synth.TREE_KD, synth.PLANE_EQUAL_DENSITY)
    assert abs(c[0]) < 0.06


SPLIT_VARIANTS = [(synth.TREE_OCTREE, synth.PLANE_BARYCENTRE, 0), (synth.TREE_KD, synth.PLANE_EQUAL_MASS, 0),
                  (synth.TREE_KD, synth.PLANE_EQUAL_DENSITY, 0), (synth.TREE_KD, synth.PLANE_EQUAL_MASS, 1)]
SPLIT_IDS = ["octree-barycentre", "kd-equal-mass", "kd-equal-density", "kd-gradient-equal-mass"]


def _variant_tree(kind, plane, axis, model=None, delta_max=2e-3, max_level=5):
    model = synth.make_disk() if model is None else model
    return oracle.build_tree(model, _bp(kind=kind, delta_max=delta_max, max_level=max_level, split_plane=plane,
                                        split_axis=axis))


@pytest.mark.parametrize("kind,plane,axis", SPLIT_VARIANTS, ids=SPLIT_IDS)
def test_split_variant_children_tile_their_parents(kind, plane, axis):
    t = _variant_tree(kind, plane, axis)
    assert t.n_leaves > 200
    nch = 8 if kind == synth.TREE_OCTREE else 2
    off_lattice = 0
    for nd in np.nonzero(t.child >= 0)[0]:
        c0 = t.child[nd]
        lo, hi = t.lo[nd], t.hi[nd]
        cut = t.hi[c0]
        for j in range(nch):
            clo, chi = t.lo[c0 + j], t.hi[c0 + j]
            for a in range(3):
                split = (kind == synth.TREE_OCTREE) or cut[a] != hi[a]
                if not split:
                    assert clo[a] == lo[a] and chi[a] == hi[a]
                    continue
                assert lo[a] < cut[a] < hi[a]
                up = ((j >> a) & 1) if kind == synth.TREE_OCTREE else j
                assert (clo[a], chi[a]) == ((cut[a], hi[a]) if up else (lo[a], cut[a]))
                off_lattice += cut[a] != 0.5 * (lo[a] + hi[a])
    assert off_lattice > 0  # the planes really are not the geometric centres
    # k-d depth limit and per-axis level limit
    assert t.lvl.max() <= 5 if kind == synth.TREE_OCTREE else t.lvl.sum(axis=1).max() <= 15


def _plane_points(t, rng, n):
    """Points on the tree's own (non-dyadic) leaf walls, edges and corners, with awkward directions."""
    leaves = rng.integers(0, t.n_leaves, n)
    lo, hi = t.leaf_lo[leaves], t.leaf_hi[leaves]
    p = lo + rng.random((n, 3)) * (hi - lo)
    pick = rng.random((n, 3))
    p = np.where(pick < 0.3, lo, np.where(pick < 0.6, hi, p))
    k = rng.choice([-1.0, -0.0, 0.0, 1.0, 0.3, -0.7], size=(n, 3))
    return p, k


@pytest.mark.parametrize("kind,plane,axis", SPLIT_VARIANTS, ids=SPLIT_IDS)
def test_split_variant_locate_matches_brute_force(kind, plane, axis):
    t = _variant_tree(kind, plane, axis)
    rng = np.random.default_rng(21)
    p = rng.uniform(-1, 1, size=(2000, 3))
    k = synth.isotropic_dirs(rng, 2000)
    pl, kl = _plane_points(t, rng, 3000)
    P, K = np.vstack([p, pl]), np.vstack([k, kl])
    got = oracle.locate(t, P, K)
    ref, hits = oracle.brute_locate(t, P, K)
    inside = hits == 1
    leaving = np.any(((P == -1.0) & (K < 0)) | ((P == 1.0) & (K > 0)), axis=1)
    assert (hits <= 1).all()
    assert (inside == ~leaving).all()
    np.testing.assert_array_equal(got[inside], ref[inside])


@pytest.mark.parametrize("kind,plane,axis", SPLIT_VARIANTS, ids=SPLIT_IDS)
def test_split_variant_sequences_match_brute_force(kind, plane, axis):
    t = _variant_tree(kind, plane, axis)
    o, k = synth.emission_rays(31, 120)
    r = oracle.trace(t, o, k, emit=True, threads=1)
    for i in range(o.shape[0]):
        a, b = r["seg_off"][i], r["seg_off"][i + 1]
        chord = float(_exact_chord(o[i], k[i]))
        cells, tin, ds = oracle.brute_sequence(t, o[i], k[i], 0.0, chord * 2)
        keep = ds > 0
        np.testing.assert_array_equal(r["seg_cell"][a:b], cells[keep])
        np.testing.assert_allclose(r["seg_ds"][a:b], ds[keep], rtol=1e-12, atol=1e-15)
        assert r["seg_ds"][a:b].sum() == pytest.approx(chord, rel=1e-12)


@pytest.mark.parametrize("kind,plane", [(synth.TREE_OCTREE, synth.PLANE_BARYCENTRE),
                                        (synth.TREE_KD, synth.PLANE_EQUAL_MASS),
                                        (synth.TREE_KD, synth.PLANE_EQUAL_DENSITY)])
def test_split_variant_uniform_density_tau_closed_form(kind, plane):
    # uniform rho: the draw-driven planes are not the centres, yet every leaf carries rho0 exactly, so
    # tau = kappa rho0 chord on every ray
    rho0, kappa = 2.5, 1.5
    t = _variant_tree(kind, plane, 0, model=synth.make_const(rho0), delta_max=1.0 / 300, max_level=6)
    assert t.n_leaves >= 300
    o, k = synth.emission_rays(6, 300)
    r = oracle.trace(t, o, k, kappa=kappa)
    for i in range(300):
        assert r["tau"][i] == pytest.approx(kappa * rho0 * float(_exact_chord(o[i], k[i])), rel=1e-13)


def test_split_location_rejected_for_the_wrong_tree():
    with pytest.raises(RuntimeError):
        oracle.build_tree(synth.make_disk(), _bp(kind=synth.TREE_OCTREE, split_plane=synth.PLANE_EQUAL_MASS))
    with pytest.raises(RuntimeError):
        oracle.build_tree(synth.make_disk(), _bp(kind=synth.TREE_KD, split_plane=synth.PLANE_BARYCENTRE))
