// Host tree construction (Sect. 2.2, 4.1, 4.2) and neighbor lists (Sect. 2.3).
//
// The node list of Sect. 2.2 is built breadth first: the paper's single
// loop over a list that appends children at its end visits nodes level by
// level, so each level is evaluated in parallel and its children appended
// in parent order afterwards, which yields the same list.  Every node's
// Monte Carlo samples (Eq. 1) come from a SplitMix64 counter stream keyed
// by the node's box, so the result does not depend on the thread count.
//
// Neighbor lists are found per leaf wall by a descent over the tree in
// exact integer lattice coordinates and sorted by decreasing overlap area
// (ties by ascending leaf id).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <memory>
#include <thread>

#include "hg_internal.h"
#include "gbuild.h"
#include "model_eval.h"

namespace {

template <class F>
void parallel_for(int64_t n, int threads, F &&fn) {
    if (n <= 0) return;
    if (threads <= 1 || n < 64) {
        fn(0, n);
        return;
    }
    std::atomic<int64_t> next{0};
    const int64_t chunk = std::max<int64_t>(16, n / (threads * 16));
    std::vector<std::thread> pool;
    for (int t = 0; t < threads; t++)
        pool.emplace_back([&]() {
            for (;;) {
                int64_t a = next.fetch_add(chunk);
                if (a >= n) break;
                fn(a, std::min(n, a + chunk));
            }
        });
    for (auto &th : pool) th.join();
}

// Density model with a uniform spatial index over the clumps.  The sum
// visits a point's candidate clumps in ascending order and applies the
// same cut-off test as a plain loop over all clumps, so the value is the
// same double.
struct HostModel {
    hg_model m{};
    std::vector<double> table;
    int G = 0;
    std::vector<int32_t> cell_off, cell_ids;

    void init(const hg_model &src) {
        m = src;
        size_t per = (src.kind == HG_MODEL_TORUS) ? 5 : 1;
        table.assign(src.table, src.table + (size_t)std::max(0, src.n_table) * per);
        m.table = table.data();
        if (src.kind == HG_MODEL_TORUS && src.n_table > 0) build_index();
    }

    void build_index() {
        G = 48;
        const int64_t nc = (int64_t)G * G * G;
        std::vector<std::vector<int32_t>> lists((size_t)nc);
        double ext[3];
        for (int a = 0; a < 3; a++) ext[a] = m.hi[a] - m.lo[a];
        for (int32_t j = 0; j < m.n_table; j++) {
            const double *c = &table[5 * (size_t)j];
            double rad = 5.0 * c[3] * (1.0 + 1e-9) + 1e-12;
            int lo[3], hi[3];
            for (int a = 0; a < 3; a++) {
                lo[a] = std::max(0, (int)std::floor((c[a] - rad - m.lo[a]) / ext[a] * G) - 1);
                hi[a] = std::min(G - 1, (int)std::floor((c[a] + rad - m.lo[a]) / ext[a] * G) + 1);
            }
            for (int z = lo[2]; z <= hi[2]; z++)
                for (int y = lo[1]; y <= hi[1]; y++)
                    for (int x = lo[0]; x <= hi[0]; x++) {
                        // conservative sphere-box test (cell grown by a relative margin)
                        int ix[3] = {x, y, z};
                        double d2 = 0.0;
                        for (int a = 0; a < 3; a++) {
                            double b0 = m.lo[a] + ext[a] * ((double)ix[a] / G) - 1e-9 * ext[a];
                            double b1 = m.lo[a] + ext[a] * ((double)(ix[a] + 1) / G) + 1e-9 * ext[a];
                            double v = c[a] < b0 ? b0 - c[a] : (c[a] > b1 ? c[a] - b1 : 0.0);
                            d2 += v * v;
                        }
                        if (d2 <= rad * rad) lists[(size_t)x + G * ((size_t)y + G * z)].push_back(j);
                    }
        }
        cell_off.assign((size_t)nc + 1, 0);
        for (int64_t c = 0; c < nc; c++) cell_off[c + 1] = cell_off[c] + (int32_t)lists[c].size();
        cell_ids.resize((size_t)cell_off[nc]);
        for (int64_t c = 0; c < nc; c++) std::copy(lists[c].begin(), lists[c].end(), cell_ids.begin() + cell_off[c]);
    }

    // the model as the node evaluation reads it (pointers into this object)
    hg::ModelView view() const {
        hg::ModelView v;
        v.kind = m.kind;
        v.n_table = m.n_table;
        for (int j = 0; j < 8; j++) v.p[j] = m.p[j];
        for (int a = 0; a < 3; a++) {
            v.lo[a] = m.lo[a];
            v.hi[a] = m.hi[a];
        }
        v.m_tot = m.m_tot;
        v.table = table.data();
        v.G = G;
        v.cell_off = cell_off.empty() ? nullptr : cell_off.data();
        v.cell_ids = cell_ids.empty() ? nullptr : cell_ids.data();
        return v;
    }

};

// Split planes at a location other than the centre (Sect. 2.2), from a
// node's n draws (see hg_build_params in hgrt.h for the definitions).
double box_centre(double lo, double hi) { return lo + 0.5 * (hi - lo); }

// Octree: the three planes through the draws' centre of mass.
void barycentre_planes(const hg::Draw *d, int32_t n, const double *lo, const double *hi, double *c) {
    double S = 0.0, Sx[3] = {0.0, 0.0, 0.0};
    for (int32_t s = 0; s < n; s++) {
        S += d[s].r;
        for (int a = 0; a < 3; a++) Sx[a] += d[s].r * d[s].x[a];
    }
    for (int a = 0; a < 3; a++) {
        double v = (S > 0.0) ? Sx[a] / S : box_centre(lo[a], hi[a]);
        c[a] = (lo[a] < v && v < hi[a]) ? v : box_centre(lo[a], hi[a]);
    }
}

// k-d tree: the equal-mass or equal-mean-density plane on axis a.  Reorders d.
double kd_plane(int mode, hg::Draw *d, int32_t n, int a, double lo, double hi, std::vector<double> &right) {
    const double centre = box_centre(lo, hi);
    if (n < 2) return centre;
    std::sort(d, d + n, [a](const hg::Draw &p, const hg::Draw &q) {
        return p.x[a] < q.x[a] || (p.x[a] == q.x[a] && p.s < q.s);
    });
    int32_t j = -1;
    if (mode == HG_PLANE_EQUAL_MASS) {
        double total = 0.0;
        for (int32_t k = 0; k < n; k++) total += d[k].r;
        if (!(total > 0.0)) return centre;
        double run = 0.0;
        for (int32_t k = 0; k < n; k++) {
            run += d[k].r;
            if (2.0 * run >= total) {
                j = k;
                break;
            }
        }
        if (j == n - 1) j = n - 2;
        if (j < 0 || !(d[j].x[a] < d[j + 1].x[a])) return centre;
    } else {
        // right[k]: the density sum of draws k+1 .. n-1, added right to left
        right.assign((size_t)n, 0.0);
        double r = 0.0;
        for (int32_t k = n - 1; k >= 1; k--) {
            r += d[k].r;
            right[(size_t)k - 1] = r;
        }
        double left = 0.0, best = 0.0;
        int32_t best_mid = 0;
        for (int32_t k = 0; k <= n - 2; k++) {
            left += d[k].r;
            if (!(d[k].x[a] < d[k + 1].x[a])) continue;
            const double diff = std::fabs(left / (double)(k + 1) - right[(size_t)k] / (double)(n - 1 - k));
            const int32_t mid = std::abs(2 * k - (n - 2));
            if (j < 0 || diff < best || (diff == best && mid < best_mid)) {
                j = k;
                best = diff;
                best_mid = mid;
            }
        }
        if (j < 0) return centre;
    }
    const double v = d[j].x[a] + 0.5 * (d[j + 1].x[a] - d[j].x[a]);
    return (lo < v && v < hi) ? v : centre;
}

// Where a node that the criteria subdivide is cut (planes[3]); clears
// st.sub when the box has no room for a plane strictly inside on a cut axis.
void place_planes(const hg_build_params &P, const double *lo, const double *hi, hg::Draw *d,
                  std::vector<double> &scratch, hg::NodeStats &st, double *planes) {
    for (int a = 0; a < 3; a++) planes[a] = box_centre(lo[a], hi[a]);
    if (st.sub) {
        if (P.kind == HG_OCTREE)
            barycentre_planes(d, P.n_ran, lo, hi, planes);
        else
            planes[st.axis] = kd_plane(P.split_plane, d, P.n_ran, st.axis, lo[st.axis], hi[st.axis], scratch);
    }
    for (int a = 0; a < 3; a++) {
        if (P.kind == HG_KDTREE && a != st.axis) continue;
        if (!(lo[a] < planes[a] && planes[a] < hi[a])) st.sub = 0;
    }
}

}  // namespace

struct hg_host_grid {
    int32_t kind = 0;
    std::vector<int32_t> lvl;   // [3n]
    std::vector<int64_t> idx;   // [3n]
    std::vector<int32_t> child; // [n]
    std::vector<int32_t> leaf;  // [n]
    std::vector<double> lo, hi; // [3n]
    std::vector<double> rho, mass, delta, tau, q;  // [n]
    std::vector<double> leaf_rho;
    std::vector<int64_t> leaf_node;
    std::vector<int64_t> nbr_off;
    std::vector<int32_t> nbr_id;
};

namespace {

// Neighbor lists from the FP64 boxes, for trees whose planes are not dyadic:
// the same descent as below, with exact comparisons of the stored bounds;
// overlap areas (the sort key) are products of FP64 differences.
void build_neighbors_fp64(hg_host_grid &G, int threads) {
    const int64_t nl = (int64_t)G.leaf_node.size();
    const double *dlo = &G.lo[0], *dhi = &G.hi[0];  // the root's box
    const int nch = (G.kind == HG_OCTREE) ? 8 : 2;
    auto walk = [&](int64_t ln, int w, std::vector<int64_t> &stack, auto &&fn) {
        const int a = w >> 1, s = w & 1;
        const double *L = &G.lo[3 * ln], *H = &G.hi[3 * ln];
        const double P = s ? H[a] : L[a];
        if ((s && P == dhi[a]) || (!s && P == dlo[a])) return;
        stack.clear();
        stack.push_back(0);
        while (!stack.empty()) {
            const int64_t nd = stack.back();
            stack.pop_back();
            const double *nlo = &G.lo[3 * nd], *nhi = &G.hi[3 * nd];
            const bool across = s ? (nlo[a] <= P && P < nhi[a]) : (nlo[a] < P && P <= nhi[a]);
            if (!across) continue;
            double area = 1.0;
            bool ok = true;
            for (int b = 0; b < 3; b++) {
                if (b == a) continue;
                const double hi_b = std::min(nhi[b], H[b]), lo_b = std::max(nlo[b], L[b]);
                if (!(hi_b > lo_b)) {
                    ok = false;
                    break;
                }
                area *= hi_b - lo_b;
            }
            if (!ok) continue;
            if (G.child[nd] < 0) {
                fn(G.leaf[nd], area);
            } else {
                for (int c = nch - 1; c >= 0; c--) stack.push_back(G.child[nd] + c);
            }
        }
    };
    std::vector<int64_t> counts((size_t)nl * 6, 0);
    parallel_for(nl, threads, [&](int64_t a0, int64_t a1) {
        std::vector<int64_t> stack;
        for (int64_t i = a0; i < a1; i++)
            for (int w = 0; w < 6; w++) {
                int64_t c = 0;
                walk(G.leaf_node[i], w, stack, [&](int32_t, double) { c++; });
                counts[6 * i + w] = c;
            }
    });
    G.nbr_off.assign((size_t)nl * 6 + 1, 0);
    for (int64_t j = 0; j < nl * 6; j++) G.nbr_off[j + 1] = G.nbr_off[j] + counts[j];
    G.nbr_id.assign((size_t)G.nbr_off[nl * 6], 0);
    parallel_for(nl, threads, [&](int64_t a0, int64_t a1) {
        std::vector<int64_t> stack;
        std::vector<std::pair<double, int32_t>> buf;
        for (int64_t i = a0; i < a1; i++)
            for (int w = 0; w < 6; w++) {
                buf.clear();
                walk(G.leaf_node[i], w, stack, [&](int32_t id, double area) { buf.emplace_back(-area, id); });
                std::sort(buf.begin(), buf.end());
                const int64_t o = G.nbr_off[6 * i + w];
                for (size_t e = 0; e < buf.size(); e++) G.nbr_id[o + e] = buf[e].second;
            }
    });
}

// Neighbor lists in lattice units of the finest per-axis level.
void build_neighbors(hg_host_grid &G, int threads) {
    const int64_t n = (int64_t)G.child.size();
    const int64_t nl = (int64_t)G.leaf_node.size();
    int32_t Lm = 0;
    for (int32_t v : G.lvl) Lm = std::max(Lm, v);
    const int64_t top = (int64_t)1 << Lm;
    auto ibox = [&](int64_t nd, int a, int64_t &lo, int64_t &hi) {
        int32_t l = G.lvl[3 * nd + a];
        lo = G.idx[3 * nd + a] << (Lm - l);
        hi = (G.idx[3 * nd + a] + 1) << (Lm - l);
    };
    const int nch = (G.kind == HG_OCTREE) ? 8 : 2;
    // visit every leaf across wall w of leaf node ln; fn(leaf id, area)
    auto walk = [&](int64_t ln, int w, std::vector<int64_t> &stack, auto &&fn) {
        const int a = w >> 1, s = w & 1;
        int64_t L[3], H[3];
        for (int b = 0; b < 3; b++) ibox(ln, b, L[b], H[b]);
        const int64_t P = s ? H[a] : L[a];
        if ((s && P == top) || (!s && P == 0)) return;
        stack.clear();
        stack.push_back(0);
        while (!stack.empty()) {
            int64_t nd = stack.back();
            stack.pop_back();
            int64_t nlo[3], nhi[3];
            for (int b = 0; b < 3; b++) ibox(nd, b, nlo[b], nhi[b]);
            bool across = s ? (nlo[a] <= P && P < nhi[a]) : (nlo[a] < P && P <= nhi[a]);
            if (!across) continue;
            int64_t area = 1;
            bool ok = true;
            for (int b = 0; b < 3; b++) {
                if (b == a) continue;
                int64_t ov = std::min(nhi[b], H[b]) - std::max(nlo[b], L[b]);
                if (ov <= 0) { ok = false; break; }
                area *= ov;
            }
            if (!ok) continue;
            if (G.child[nd] < 0) {
                fn(G.leaf[nd], area);
            } else {
                for (int c = nch - 1; c >= 0; c--) stack.push_back(G.child[nd] + c);
            }
        }
    };
    std::vector<int64_t> counts((size_t)nl * 6, 0);
    parallel_for(nl, threads, [&](int64_t a0, int64_t a1) {
        std::vector<int64_t> stack;
        for (int64_t i = a0; i < a1; i++)
            for (int w = 0; w < 6; w++) {
                int64_t c = 0;
                walk(G.leaf_node[i], w, stack, [&](int32_t, int64_t) { c++; });
                counts[6 * i + w] = c;
            }
    });
    G.nbr_off.assign((size_t)nl * 6 + 1, 0);
    for (int64_t j = 0; j < nl * 6; j++) G.nbr_off[j + 1] = G.nbr_off[j] + counts[j];
    G.nbr_id.assign((size_t)G.nbr_off[nl * 6], 0);
    parallel_for(nl, threads, [&](int64_t a0, int64_t a1) {
        std::vector<int64_t> stack;
        std::vector<std::pair<int64_t, int32_t>> buf;
        for (int64_t i = a0; i < a1; i++)
            for (int w = 0; w < 6; w++) {
                buf.clear();
                walk(G.leaf_node[i], w, stack, [&](int32_t id, int64_t area) { buf.emplace_back(-area, id); });
                std::sort(buf.begin(), buf.end());
                int64_t o = G.nbr_off[6 * i + w];
                for (size_t e = 0; e < buf.size(); e++) G.nbr_id[o + e] = buf[e].second;
            }
    });
    (void)n;
}

}  // namespace

namespace {

hg_status check_build_args(const char *name, const hg_model *model, const hg_build_params *params, void *out) {
    if (!model || !params || !out) {
        hg::set_error("%s: null argument", name);
        return HG_EINVAL;
    }
    const hg_build_params &P = *params;
    if (P.kind != HG_OCTREE && P.kind != HG_KDTREE) { hg::set_error("bad tree kind %d", P.kind); return HG_EINVAL; }
    if (P.n_ran < 1 || P.max_level < 0 || P.max_level > 20) {
        hg::set_error("%s: n_ran must be >= 1 and max_level in 0..20", name);
        return HG_EINVAL;
    }
    if (P.split_axis != HG_AXIS_CYCLIC && P.split_axis != HG_AXIS_GRADIENT) {
        hg::set_error("%s: split_axis must be HG_AXIS_CYCLIC or HG_AXIS_GRADIENT", name);
        return HG_EINVAL;
    }
    const bool plane_ok = P.split_plane == HG_PLANE_CENTRE ||
                          (P.kind == HG_OCTREE && P.split_plane == HG_PLANE_BARYCENTRE) ||
                          (P.kind == HG_KDTREE &&
                           (P.split_plane == HG_PLANE_EQUAL_MASS || P.split_plane == HG_PLANE_EQUAL_DENSITY));
    if (!plane_ok) {
        hg::set_error("%s: split_plane %d is not a location for this kind of tree", name, P.split_plane);
        return HG_EINVAL;
    }
    if (!(model->m_tot > 0.0)) { hg::set_error("%s: m_tot must be > 0", name); return HG_EINVAL; }
    if (model->kind < HG_MODEL_CONST || model->kind > HG_MODEL_DYADIC) {
        hg::set_error("%s: bad model kind %d", name, model->kind);
        return HG_EINVAL;
    }
    if ((model->kind == HG_MODEL_TORUS || model->kind == HG_MODEL_DYADIC) && model->n_table > 0 && !model->table) {
        hg::set_error("%s: model table missing", name);
        return HG_EINVAL;
    }
    for (int a = 0; a < 3; a++)
        if (!(model->hi[a] > model->lo[a])) { hg::set_error("%s: empty domain", name); return HG_EINVAL; }
    return HG_OK;
}

// The node list, level by level: eval(begin, end, st) evaluates nodes
// [begin, end) (their levels and indices are in G), then the nodes to
// subdivide get their children appended in parent order.  Leaves are
// numbered in node order (the caller builds the neighbor lists).
// With split planes other than the centre, eval also fills planes (3 per
// node of the level) and each child's box is cut from its parent's there.
template <class Eval>
hg_status build_levels(const HostModel &M, const hg_build_params &P, hg_host_grid &G, Eval &&eval) {
    const hg::ModelView V = M.view();
    auto push = [&](const int32_t *l, const int64_t *i, const double *lo, const double *hi) {
        for (int a = 0; a < 3; a++) {
            G.lvl.push_back(l[a]);
            G.idx.push_back(i[a]);
            G.lo.push_back(lo ? lo[a] : hg::model_bound(V, a, i[a], l[a]));
            G.hi.push_back(hi ? hi[a] : hg::model_bound(V, a, i[a] + 1, l[a]));
        }
        G.child.push_back(-1);
        G.leaf.push_back(-1);
    };
    const bool centre = (P.split_plane == HG_PLANE_CENTRE);
    std::vector<double> planes;
    G.kind = P.kind;
    int32_t l0[3] = {0, 0, 0};
    int64_t i0[3] = {0, 0, 0};
    push(l0, i0, nullptr, nullptr);
    int64_t begin = 0;
    std::vector<hg::NodeStats> st;
    while (begin < (int64_t)G.child.size()) {
        const int64_t end = (int64_t)G.child.size();
        st.assign((size_t)(end - begin), hg::NodeStats{});
        if (!centre) planes.assign((size_t)(end - begin) * 3, 0.0);
        hg_status hs = eval(begin, end, st, planes);
        if (hs != HG_OK) return hs;
        for (int64_t j = 0; j < end - begin; j++) {
            G.rho.push_back(st[j].rho);
            G.mass.push_back(st[j].mass);
            G.delta.push_back(st[j].delta);
            G.tau.push_back(st[j].tau);
            G.q.push_back(st[j].q);
        }
        for (int64_t nd = begin; nd < end; nd++) {
            if (!st[nd - begin].sub) continue;
            const int nch = (P.kind == HG_OCTREE) ? 8 : 2;
            if (P.max_nodes > 0 && (int64_t)G.child.size() + nch > P.max_nodes) {
                hg::set_error("hg_build_grid: more than max_nodes=%lld nodes", (long long)P.max_nodes);
                return HG_EOVERFLOW;
            }
            if ((int64_t)G.child.size() + nch > INT32_MAX) {
                hg::set_error("hg_build_grid: node count exceeds int32 ids");
                return HG_EOVERFLOW;
            }
            G.child[nd] = (int32_t)G.child.size();
            int32_t l[3] = {G.lvl[3 * nd], G.lvl[3 * nd + 1], G.lvl[3 * nd + 2]};
            int64_t i[3] = {G.idx[3 * nd], G.idx[3 * nd + 1], G.idx[3 * nd + 2]};
            const int axis = st[nd - begin].axis;  // k-d: the split axis (octree: -1)
            const double plo[3] = {G.lo[3 * nd], G.lo[3 * nd + 1], G.lo[3 * nd + 2]};
            const double phi[3] = {G.hi[3 * nd], G.hi[3 * nd + 1], G.hi[3 * nd + 2]};
            for (int c = 0; c < nch; c++) {
                int32_t lc[3] = {l[0], l[1], l[2]};
                int64_t ic[3] = {i[0], i[1], i[2]};
                double clo[3] = {plo[0], plo[1], plo[2]}, chi[3] = {phi[0], phi[1], phi[2]};
                for (int a = 0; a < 3; a++) {
                    if (axis >= 0 && a != axis) continue;
                    const int up = (axis < 0) ? ((c >> a) & 1) : c;
                    lc[a] = l[a] + 1;
                    ic[a] = 2 * i[a] + up;
                    if (!centre) (up ? clo[a] : chi[a]) = planes[3 * (size_t)(nd - begin) + a];
                }
                if (centre)
                    push(lc, ic, nullptr, nullptr);
                else
                    push(lc, ic, clo, chi);
            }
        }
        begin = end;
    }
    const int64_t n = (int64_t)G.child.size();
    for (int64_t nd = 0; nd < n; nd++)
        if (G.child[nd] < 0) {
            G.leaf[nd] = (int32_t)G.leaf_node.size();
            G.leaf_node.push_back(nd);
            G.leaf_rho.push_back(G.rho[nd]);
        }
    return HG_OK;
}

int host_threads(int32_t n_threads) {
    return n_threads > 0 ? n_threads : (int)std::max(1u, std::thread::hardware_concurrency());
}

}  // namespace

extern "C" hg_status hg_build_grid(const hg_model *model, const hg_build_params *params, int32_t n_threads,
                                   hg_host_grid **out) {
    hg_status hs = check_build_args("hg_build_grid", model, params, out);
    if (hs != HG_OK) return hs;
    *out = nullptr;
    const hg_build_params P = *params;
    const int threads = host_threads(n_threads);
    std::unique_ptr<hg_host_grid> G(new hg_host_grid());
    HostModel M;
    try {
        M.init(*model);
        const hg::ModelView V = M.view();
        const bool centre = (P.split_plane == HG_PLANE_CENTRE);
        hs = build_levels(M, P, *G, [&](int64_t begin, int64_t end, std::vector<hg::NodeStats> &st,
                                        std::vector<double> &planes) {
            parallel_for(end - begin, threads, [&](int64_t a0, int64_t a1) {
                std::vector<hg::Draw> draws(centre ? 0 : (size_t)P.n_ran);
                std::vector<double> scratch;
                for (int64_t j = a0; j < a1; j++) {
                    const int64_t nd = begin + j;
                    const int32_t *l = &G->lvl[3 * nd];
                    const int64_t *i = &G->idx[3 * nd];
                    const int32_t depth = (P.kind == HG_OCTREE) ? l[0] : l[0] + l[1] + l[2];
                    if (centre) {
                        st[j] = hg::eval_node_stats(V, P, l, i, depth);
                    } else {
                        const double *lo = &G->lo[3 * nd], *hi = &G->hi[3 * nd];
                        st[j] = hg::eval_node_stats(V, P, l, i, depth, lo, hi, draws.data());
                        place_planes(P, lo, hi, draws.data(), scratch, st[j], &planes[3 * (size_t)j]);
                    }
                }
            });
            return HG_OK;
        });
        if (hs == HG_OK) {
            if (centre)
                build_neighbors(*G, threads);
            else
                build_neighbors_fp64(*G, threads);
        }
    } catch (const std::bad_alloc &) {
        hg::set_error("hg_build_grid: out of host memory");
        return HG_ENOMEM;
    }
    if (hs != HG_OK) return hs;
    *out = G.release();
    return HG_OK;
}

extern "C" hg_status hg_build_grid_gpu(const hg_model *model, const hg_build_params *params, hg_stream stream,
                                       hg_host_grid **out) {
    hg_status hs = check_build_args("hg_build_grid_gpu", model, params, out);
    if (hs != HG_OK) return hs;
    if (params->split_plane != HG_PLANE_CENTRE) {
        hg::set_error("hg_build_grid_gpu: split planes other than the centre are built by hg_build_grid only");
        return HG_EINVAL;
    }
    *out = nullptr;
    const hg_build_params P = *params;
    std::unique_ptr<hg_host_grid> G(new hg_host_grid());
    try {
        HostModel M;
        M.init(*model);
        hg::GpuTree T;
        hs = hg::gpu_build_tree(M.view(), P, stream, T);
        if (hs != HG_OK) return hs;
        G->kind = P.kind;
        G->lvl = std::move(T.lvl);
        G->idx = std::move(T.idx);
        G->child = std::move(T.child);
        G->leaf = std::move(T.leaf);
        G->lo = std::move(T.lo);
        G->hi = std::move(T.hi);
        G->rho = std::move(T.rho);
        G->mass = std::move(T.mass);
        G->delta = std::move(T.delta);
        G->tau = std::move(T.tau);
        G->q = std::move(T.q);
        G->leaf_rho = std::move(T.leaf_rho);
        G->leaf_node = std::move(T.leaf_node);
        G->nbr_off = std::move(T.nbr_off);
        G->nbr_id = std::move(T.nbr_id);
    } catch (const std::bad_alloc &) {
        hg::set_error("hg_build_grid_gpu: out of host memory");
        return HG_ENOMEM;
    }
    *out = G.release();
    return HG_OK;
}

// The tau_max recipe of Sect. 4.1: build with the mass criterion only, sort
// the leaves' optical depths (Eq. 2, as the builder computes them) in
// ascending order and take the one at position floor(fraction * N_leaves)
// (0-based, at most N_leaves - 1); the paper uses fraction 0.9.
extern "C" hg_status hg_tau_max_recipe(const hg_model *model, const hg_build_params *params, double fraction,
                                       int32_t n_threads, double *tau_max) {
    if (!params || !tau_max || !(fraction >= 0.0 && fraction <= 1.0)) {
        hg::set_error("hg_tau_max_recipe: bad arguments (fraction must lie in [0, 1])");
        return HG_EINVAL;
    }
    hg_build_params p = *params;
    p.use_tau = 0;
    p.use_q = 0;
    hg_host_grid *G = nullptr;
    hg_status st = hg_build_grid(model, &p, n_threads, &G);
    if (st != HG_OK) return st;
    try {
        std::vector<double> t;
        t.reserve(G->leaf_node.size());
        for (const int64_t nd : G->leaf_node) t.push_back(G->tau[nd]);
        std::sort(t.begin(), t.end());
        const int64_t N = (int64_t)t.size();
        const int64_t i = std::min<int64_t>((int64_t)std::floor(fraction * (double)N), N - 1);
        *tau_max = t[(size_t)i];
    } catch (const std::bad_alloc &) {
        delete G;
        hg::set_error("hg_tau_max_recipe: out of host memory");
        return HG_ENOMEM;
    }
    delete G;
    return HG_OK;
}

extern "C" hg_status hg_host_grid_desc(const hg_host_grid *g, hg_grid_desc *out) {
    if (!g || !out) { hg::set_error("hg_host_grid_desc: null argument"); return HG_EINVAL; }
    out->kind = g->kind;
    out->reserved = 0;
    out->n_nodes = (int64_t)g->child.size();
    out->n_leaves = (int64_t)g->leaf_node.size();
    out->node_lo = g->lo.data();
    out->node_hi = g->hi.data();
    out->child_first = g->child.data();
    out->node_leaf = g->leaf.data();
    out->leaf_rho = g->leaf_rho.data();
    out->nbr_off = g->nbr_off.data();
    out->nbr_id = g->nbr_id.data();
    return HG_OK;
}

extern "C" hg_status hg_host_grid_nodes(const hg_host_grid *g, hg_host_nodes *out) {
    if (!g || !out) { hg::set_error("hg_host_grid_nodes: null argument"); return HG_EINVAL; }
    out->level = g->lvl.data();
    out->index = g->idx.data();
    out->mass = g->mass.data();
    out->delta = g->delta.data();
    out->tau = g->tau.data();
    out->q = g->q.data();
    return HG_OK;
}

extern "C" void hg_free_host_grid(hg_host_grid *g) { delete g; }
