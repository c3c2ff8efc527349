"""Host-side checks of the library (no GPU): exported C ABI, tree builder
against the oracle's node list, neighbor-list invariants, and rejection of
malformed grid descriptions by hg_load_grid's validation."""
import math
import os
import re

import numpy as np
import pytest

import oracle
import synth

hg = pytest.importorskip("paper_1311_0705_gb300")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    import ctypes
    hdr = open(os.path.join(ROOT, "include", "hgrt.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    names = set(re.findall(r"\b(hg_[a-z0-9_]+)\s*\(", hdr))
    assert len(names) >= 25
    lib = ctypes.CDLL(hg.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    # the binding wraps every declared function
    assert names <= set(hg.EXPORTED), sorted(names - set(hg.EXPORTED))


def test_status_strings_and_bits():
    assert hg._lib.hg_status_str(0) == b"ok"
    assert hg.status_from_bits(0) == 0
    assert hg.status_from_bits(hg.RAY_LOST | hg.RAY_STEPLIMIT) == 6
    assert hg.status_from_bits(hg.RAY_STEPLIMIT) == 5


def _same_tree(H, T):
    assert H.n_nodes == T.n_nodes and H.n_leaves == T.n_leaves
    np.testing.assert_array_equal(H.node_lo, T.lo)
    np.testing.assert_array_equal(H.node_hi, T.hi)
    np.testing.assert_array_equal(H.child_first, T.child)
    np.testing.assert_array_equal(H.node_leaf, T.leaf)
    np.testing.assert_array_equal(H.leaf_rho, T.leaf_rho)
    np.testing.assert_array_equal(H.mass, T.mass)
    np.testing.assert_array_equal(H.q, T.q)
    np.testing.assert_array_equal(H.tau, T.taun)
    np.testing.assert_array_equal(H.level, T.lvl)
    np.testing.assert_array_equal(H.index, T.idx)


CASES = [
    ("disk-oct", lambda: synth.make_disk(), dict(kind=0, delta_max=1e-4, max_level=6)),
    ("disk-kd", lambda: synth.make_disk(), dict(kind=1, delta_max=5e-5, max_level=6)),
    ("torus-kd-all", lambda: synth.make_torus(11, n_clumps=60), dict(kind=1, delta_max=1e-3, use_tau=True,
                                                                     tau_max=2.0, use_q=True, q_max=0.9,
                                                                     max_level=5)),
    ("torus-oct-q", lambda: synth.make_torus(12, n_clumps=30), dict(kind=0, delta_max=1e-2, use_q=True,
                                                                    q_max=0.99, max_level=4)),
    ("dyadic-oct", lambda: synth.make_dyadic(3, level=2), dict(kind=0, delta_max=1e-3, max_level=4)),
    ("const-tau", lambda: synth.make_const(2.0), dict(kind=1, use_delta=False, use_tau=True, tau_max=0.9,
                                                      max_level=6)),
    # k-d trees split on the axis of the strongest density gradient (Sect. 2.2)
    ("disk-kd-grad", lambda: synth.make_disk(), dict(kind=1, delta_max=5e-5, max_level=6, split_axis=1)),
    ("torus-kd-grad", lambda: synth.make_torus(11, n_clumps=60), dict(kind=1, delta_max=1e-3, use_tau=True,
                                                                      tau_max=2.0, use_q=True, q_max=0.9,
                                                                      max_level=5, split_axis=1)),
    ("dyadic-kd-grad", lambda: synth.make_dyadic(4, level=3), dict(kind=1, delta_max=2e-3, use_q=True,
                                                                   q_max=0.5, max_level=5, split_axis=1)),
    # split locations other than the centre (Sect. 2.2): explicit FP64 boxes
    ("disk-oct-bary", lambda: synth.make_disk(), dict(kind=0, delta_max=1e-4, max_level=6, split_plane=1)),
    ("disk-kd-mass", lambda: synth.make_disk(), dict(kind=1, delta_max=5e-5, max_level=6, split_plane=2)),
    ("disk-kd-dens", lambda: synth.make_disk(), dict(kind=1, delta_max=5e-5, max_level=6, split_plane=3)),
    ("torus-kd-mass-grad", lambda: synth.make_torus(11, n_clumps=60), dict(kind=1, delta_max=1e-3, use_tau=True,
                                                                           tau_max=2.0, use_q=True, q_max=0.9,
                                                                           max_level=5, split_axis=1,
                                                                           split_plane=2)),
    ("torus-oct-bary-q", lambda: synth.make_torus(12, n_clumps=30), dict(kind=0, delta_max=1e-2, use_q=True,
                                                                         q_max=0.99, max_level=4, split_plane=1)),
    ("dyadic-kd-dens", lambda: synth.make_dyadic(3, level=2), dict(kind=1, delta_max=1e-3, max_level=4,
                                                                   split_plane=3)),
]


@pytest.mark.parametrize("name,mk,kw", CASES, ids=[c[0] for c in CASES])
def test_builder_matches_oracle_bit_exact(name, mk, kw):
    model = mk()
    bp = synth.BuildParams(seed=synth.BASE_SEED + 17, **kw)
    H = hg.build_grid(model, bp, threads=4)
    T = oracle.build_tree(model, bp)
    _same_tree(H, T)


def test_builder_independent_of_thread_count():
    model = synth.make_torus(5, n_clumps=40)
    bp = synth.BuildParams(kind=1, delta_max=2e-3, use_q=True, q_max=0.9, max_level=5)
    a = hg.build_grid(model, bp, threads=1)
    b = hg.build_grid(model, bp, threads=7)
    np.testing.assert_array_equal(a.child_first, b.child_first)
    np.testing.assert_array_equal(a.leaf_rho, b.leaf_rho)
    np.testing.assert_array_equal(a.nbr_off, b.nbr_off)
    np.testing.assert_array_equal(a.nbr_id, b.nbr_id)


def _leaf_boxes(H):
    ln = H.leaf_node
    return H.node_lo[ln], H.node_hi[ln]


@pytest.mark.parametrize("kind,split_axis,split_plane", [(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 0, 1), (1, 0, 2),
                                                          (1, 0, 3)],
                         ids=["octree", "kd", "kd-gradient", "octree-bary", "kd-mass", "kd-dens"])
def test_neighbor_lists_tile_walls_and_are_symmetric(kind, split_axis, split_plane):
    model = synth.make_disk()
    H = hg.build_grid(model, synth.BuildParams(kind=kind, delta_max=3e-4, max_level=6, split_axis=split_axis,
                                               split_plane=split_plane))
    lo, hi = _leaf_boxes(H)
    dlo, dhi = H.node_lo[0], H.node_hi[0]
    pairs = set()
    for i in range(H.n_leaves):
        for w in range(6):
            a, s = w // 2, w % 2
            ids = H.nbr_id[H.nbr_off[6 * i + w]:H.nbr_off[6 * i + w + 1]]
            plane = hi[i, a] if s else lo[i, a]
            on_boundary = plane == (dhi[a] if s else dlo[a])
            assert on_boundary == (ids.size == 0)
            if ids.size == 0:
                continue
            t = [b for b in range(3) if b != a]
            ov = np.ones(ids.size)
            for b in t:
                ov *= np.minimum(hi[i, b], hi[ids, b]) - np.maximum(lo[i, b], lo[ids, b])
            assert (ov > 0).all()
            # adjacent across the wall, sorted by decreasing overlap, tiling the wall
            np.testing.assert_array_equal(lo[ids, a] if s else hi[ids, a], plane)
            assert (np.diff(ov) <= 0).all()
            area = (hi[i, t[0]] - lo[i, t[0]]) * (hi[i, t[1]] - lo[i, t[1]])
            assert ov.sum() == pytest.approx(area, rel=1e-15 if split_plane == 0 else 1e-12)
            for j in ids:
                pairs.add((i, w, int(j)))
    for (i, w, j) in pairs:
        assert (j, w ^ 1, i) in pairs


def _desc(H):
    d = H.desc()
    return hg.GridDesc(d.kind, d.node_lo.copy(), d.node_hi.copy(), d.child_first.copy(), d.node_leaf.copy(),
                       d.leaf_rho.copy(), d.nbr_off.copy(), d.nbr_id.copy())


@pytest.fixture(scope="module")
def small_host():
    return hg.build_grid(synth.make_disk(), synth.BuildParams(kind=1, delta_max=2e-3, max_level=4))


def _corrupt(desc, what):
    if what == "cycle":
        desc.child_first[desc.child_first > 0][0:1] = 0
        idx = np.nonzero(desc.child_first > 0)[0][0]
        desc.child_first[idx] = 0
    elif what == "nbr_range":
        desc.nbr_id[3] = 10 ** 8
    elif what == "nbr_not_adjacent":
        k = np.nonzero(np.diff(desc.nbr_off) > 0)[0][5]
        e = desc.nbr_off[k]
        desc.nbr_id[e] = (desc.nbr_id[e] + 7) % desc.leaf_rho.shape[0]
    elif what == "not_tiling":
        k = np.nonzero(np.diff(desc.nbr_off) >= 2)[0][0]
        desc.nbr_off[k + 1] -= 1
    elif what == "leaf_order":
        lv = np.nonzero(desc.node_leaf >= 0)[0]
        desc.node_leaf[lv[0]], desc.node_leaf[lv[1]] = desc.node_leaf[lv[1]], desc.node_leaf[lv[0]]
    elif what == "child_box":
        c = desc.child_first[0]
        desc.node_hi[c, 0] += 1e-3
    elif what == "nan_rho":
        desc.leaf_rho[2] = np.nan
    return desc


@pytest.mark.parametrize("what", ["cycle", "nbr_range", "nbr_not_adjacent", "not_tiling", "leaf_order",
                                  "child_box", "nan_rho"])
def test_load_grid_rejects_corrupt_descriptions(small_host, what):
    # validation runs on the host before any device work: no GPU needed
    desc = _corrupt(_desc(small_host), what)
    with pytest.raises(hg.HgError, match="grid description invalid"):
        hg.load_grid(desc, validate=True)


def test_builder_rejects_split_plane_of_the_other_tree_kind():
    with pytest.raises(hg.HgError, match="split_plane"):
        hg.build_grid(synth.make_disk(), synth.BuildParams(kind=0, split_plane=2))
    with pytest.raises(hg.HgError, match="split_plane"):
        hg.build_grid(synth.make_disk(), synth.BuildParams(kind=1, split_plane=1))
    with pytest.raises(hg.HgError, match="split_plane"):
        hg.build_grid(synth.make_disk(), synth.BuildParams(kind=1, split_plane=4))


def test_builder_rejects_bad_split_axis():
    with pytest.raises(hg.HgError, match="split_axis"):
        hg.build_grid(synth.make_disk(), synth.BuildParams(kind=1, delta_max=1e-3, max_level=3, split_axis=2))


def test_builder_rejects_bad_parameters():
    with pytest.raises(hg.HgError):
        hg.build_grid(synth.make_disk(), synth.BuildParams(kind=0, max_level=25))
    with pytest.raises(hg.HgError):
        hg.build_grid(synth.make_disk(), synth.BuildParams(kind=0, n_ran=0))
    bp = synth.BuildParams(kind=0, delta_max=-1.0, max_level=5)
    bp.max_nodes = 100
    with pytest.raises(hg.HgError, match="capacity"):
        hg.build_grid(synth.make_const(), bp)


def test_single_leaf_grid_has_no_neighbor_entries():
    # a root that no criterion splits (here delta = 1 <= delta_max) stays the only leaf; the same
    # happens when all of a root's Monte Carlo samples miss a thin structure (Eq. 1 gives M = 0)
    bp = synth.BuildParams(kind=0, delta_max=2.0, max_level=4)
    H = hg.build_grid(synth.make_const(1.0), bp)
    assert H.n_leaves == 1 and H.nbr_id.size == 0 and (H.nbr_off == 0).all()


@pytest.mark.parametrize("kind", [0, 1])
def test_tau_max_recipe_matches_oracle(kind):
    # Sect. 4.1: tau_max = the leaf optical depth at position floor(0.9 N) of a mass-criterion-only grid
    model = synth.make_torus(13, n_clumps=40)
    bp = synth.BuildParams(kind=kind, delta_max=2e-3, use_tau=True, tau_max=123.0, use_q=True, max_level=5)
    for frac in (0.9, 0.5, 1.0, 0.0):
        got = hg.tau_max_recipe(model, bp, fraction=frac, threads=3)
        assert got == oracle.tau_max_recipe(model, bp, fraction=frac)
    tm = hg.tau_max_recipe(model, bp)
    H = hg.build_grid(model, synth.BuildParams(kind=kind, delta_max=2e-3, max_level=5))
    taus = H.tau[H.leaf_node]
    # at most 10 % of the leaves lie above it, and only ties keep the count below 10 % - 1
    above = int((taus > tm).sum())
    assert above <= int(0.1 * H.n_leaves) + 1 and (taus >= tm).sum() >= H.n_leaves - int(0.9 * H.n_leaves)
    with pytest.raises(hg.HgError):
        hg.tau_max_recipe(model, bp, fraction=1.5)


@pytest.mark.parametrize("kind", [0, 1])
def test_tau_max_recipe_known_quantile_matches_oracle(kind):
    # the lattice whose Sect. 4.1 quantile the oracle pins (sorted cell values 1 x 56, 2, 4, 8 x 6):
    # the library's recipe gives the same optical depth at every fraction
    vals = np.array([1.0] * 56 + [2.0, 4.0] + [8.0] * 6)[np.random.default_rng(11).permutation(64)]
    m = synth.Model(synth.MODEL_DYADIC, np.array([2.0]), vals.reshape(-1, 1), float(vals.sum()) * 0.125,
                    np.full(3, -1.0), np.full(3, 1.0), "quantile lattice")
    bp = synth.BuildParams(kind=kind, delta_max=1e-12, max_level=2, kappa=1.5)
    for frac in (0.9, 0.89, 0.92, 0.0, 1.0):
        assert hg.tau_max_recipe(m, bp, fraction=frac, threads=2) == oracle.tau_max_recipe(m, bp, fraction=frac)
    assert hg.tau_max_recipe(m, bp) == pytest.approx(4.0 * 1.5 * math.sqrt(3.0) * 0.5, rel=4e-16)


# ----------------------------------------------------------------------------- ropes

def _depths(H):
    d = np.zeros(H.n_nodes, np.int64)
    nch = 8 if H.kind == 0 else 2
    for nd in range(H.n_nodes):
        c = H.child_first[nd]
        if c >= 0:
            d[c:c + nch] = d[nd] + 1
    return d


@pytest.mark.parametrize("kind,split_plane", [(0, 0), (1, 0), (0, 1), (1, 2)],
                         ids=["octree", "kd", "octree-bary", "kd-mass"])
def test_ropes_are_the_deepest_covering_nodes(kind, split_plane):
    # brute force over every node: the nodes across a leaf wall that cover its whole face are nested, and the
    # rope is the deepest of them; the leaves below it that touch the face are exactly the wall's neighbor list
    H = hg.build_grid(synth.make_disk(), synth.BuildParams(kind=kind, delta_max=2e-3, max_level=5,
                                                           split_plane=split_plane))
    assert 300 < H.n_leaves < 3000
    R = hg.build_ropes(H, threads=3)
    np.testing.assert_array_equal(R, hg.build_ropes(H, threads=1))
    lo, hi = H.node_lo, H.node_hi
    depth = _depths(H)
    dlo, dhi = lo[0], hi[0]
    n_internal = 0
    for i in range(H.n_leaves):
        ln = H.leaf_node[i]
        for w in range(6):
            a, s = w // 2, w % 2
            P = hi[ln, a] if s else lo[ln, a]
            r = R[i, w]
            if P == (dhi[a] if s else dlo[a]):
                assert r == -1
                continue
            across = (lo[:, a] <= P) & (P < hi[:, a]) if s else (lo[:, a] < P) & (P <= hi[:, a])
            cover = across.copy()
            for b in range(3):
                if b != a:
                    cover &= (lo[:, b] <= lo[ln, b]) & (hi[ln, b] <= hi[:, b])
            nodes = np.nonzero(cover)[0]
            deepest = nodes[np.argmax(depth[nodes])]
            assert (depth[nodes] == depth[deepest]).sum() == 1
            node = H.leaf_node[r] if r >= 0 else -2 - r
            assert node == deepest
            n_internal += r <= -2
            # the rope's node touches the wall from the far side
            assert (lo[node, a] if s else hi[node, a]) == P
            # leaves below it touching the face = the neighbor list
            below = set()
            stack = [node]
            while stack:
                nd = stack.pop()
                if H.child_first[nd] < 0:
                    j = H.node_leaf[nd]
                    ok = (lo[nd, a] == P) if s else (hi[nd, a] == P)
                    for b in range(3):
                        if b != a:
                            ok = ok and min(hi[nd, b], hi[ln, b]) > max(lo[nd, b], lo[ln, b])
                    if ok:
                        below.add(int(j))
                else:
                    stack.extend(range(H.child_first[nd], H.child_first[nd] + (8 if kind == 0 else 2)))
            lst = set(H.nbr_id[H.nbr_off[6 * i + w]:H.nbr_off[6 * i + w + 1]].tolist())
            assert below == lst
    assert n_internal > 0


def test_build_ropes_rejects_bad_leaf_ids():
    H = hg.build_grid(synth.make_disk(), synth.BuildParams(kind=1, delta_max=2e-3, max_level=4))
    d = _desc(H)
    d.node_leaf[d.node_leaf >= 0] = 0
    with pytest.raises(hg.HgError):
        hg.build_ropes(d)
