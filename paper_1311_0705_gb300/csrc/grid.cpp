// Grid upload (hg_load_grid): validation of a grid description, derivation
// of the packed leaf records and descent nodes, and the copy to HBM.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <system_error>
#include <memory>
#include <thread>
#include <vector>

#include "hg_internal.h"

namespace {

constexpr int kScanLimit = 16;  // neighbor lists longer than this are searched top-down

hg_status cuda_fail(cudaError_t e, const char *what) {
    hg::set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? HG_ENOMEM : HG_ECUDA;
}

hg_status validate(const hg_grid_desc &D, bool check_lists) {
    const int64_t n = D.n_nodes, nl = D.n_leaves;
    const int nch = (D.kind == HG_OCTREE) ? 8 : 2;
    std::vector<int32_t> parent((size_t)n, -1);
    int64_t next_leaf = 0;
    for (int64_t i = 0; i < n; i++) {
        const double *lo = D.node_lo + 3 * i, *hi = D.node_hi + 3 * i;
        for (int a = 0; a < 3; a++)
            if (!(std::isfinite(lo[a]) && std::isfinite(hi[a]) && lo[a] < hi[a])) {
                hg::set_error("node %lld has an empty or non-finite box", (long long)i);
                return HG_EFORMAT;
            }
        const int32_t c = D.child_first[i];
        if (c < 0) {
            if (D.node_leaf[i] != next_leaf) {
                hg::set_error("node %lld: leaf ids must follow list order", (long long)i);
                return HG_EFORMAT;
            }
            next_leaf++;
            continue;
        }
        if (D.node_leaf[i] != -1) {
            hg::set_error("internal node %lld carries a leaf id", (long long)i);
            return HG_EFORMAT;
        }
        if (c <= i || (int64_t)c + nch > n) {
            hg::set_error("node %lld: child index %d out of order or range", (long long)i, c);
            return HG_EFORMAT;
        }
        for (int j = 0; j < nch; j++) {
            if (parent[c + j] != -1) {
                hg::set_error("node %d has two parents", c + j);
                return HG_EFORMAT;
            }
            parent[c + j] = (int32_t)i;
        }
        // children tile the parent
        const double *c0hi = D.node_hi + 3 * (int64_t)c;
        if (D.kind == HG_OCTREE) {
            for (int j = 0; j < 8; j++) {
                const double *clo = D.node_lo + 3 * ((int64_t)c + j), *chi = D.node_hi + 3 * ((int64_t)c + j);
                for (int a = 0; a < 3; a++) {
                    double s = c0hi[a];
                    bool up = (j >> a) & 1;
                    double elo = up ? s : lo[a], ehi = up ? hi[a] : s;
                    if (clo[a] != elo || chi[a] != ehi || !(lo[a] < s && s < hi[a])) {
                        hg::set_error("octree children of node %lld do not tile it", (long long)i);
                        return HG_EFORMAT;
                    }
                }
            }
        } else {
            int ax = -1;
            for (int a = 0; a < 3; a++)
                if (c0hi[a] != hi[a]) ax = (ax == -1) ? a : 3;
            if (ax < 0 || ax > 2) {
                hg::set_error("k-d node %lld: children must split exactly one axis", (long long)i);
                return HG_EFORMAT;
            }
            const double s = c0hi[ax];
            for (int j = 0; j < 2; j++) {
                const double *clo = D.node_lo + 3 * ((int64_t)c + j), *chi = D.node_hi + 3 * ((int64_t)c + j);
                for (int a = 0; a < 3; a++) {
                    double elo = lo[a], ehi = hi[a];
                    if (a == ax) {
                        elo = j ? s : lo[a];
                        ehi = j ? hi[a] : s;
                    }
                    if (clo[a] != elo || chi[a] != ehi || !(lo[ax] < s && s < hi[ax])) {
                        hg::set_error("k-d children of node %lld do not tile it", (long long)i);
                        return HG_EFORMAT;
                    }
                }
            }
        }
    }
    if (next_leaf != nl) {
        hg::set_error("leaf count %lld does not match n_leaves %lld", (long long)next_leaf, (long long)nl);
        return HG_EFORMAT;
    }
    for (int64_t i = 1; i < n; i++)
        if (parent[i] < 0) {
            hg::set_error("node %lld is unreachable", (long long)i);
            return HG_EFORMAT;
        }
    std::vector<int64_t> leaf_node((size_t)nl);
    for (int64_t i = 0; i < n; i++)
        if (D.node_leaf[i] >= 0) leaf_node[D.node_leaf[i]] = i;
    for (int64_t j = 0; j < nl; j++)
        if (!std::isfinite(D.leaf_rho[j])) {
            hg::set_error("leaf %lld has a non-finite density", (long long)j);
            return HG_EFORMAT;
        }
    if (!check_lists) return HG_OK;
    // neighbor lists: adjacency, positive overlap, tiling, order
    if (D.nbr_off[0] != 0) { hg::set_error("nbr_off[0] must be 0"); return HG_EFORMAT; }
    const double *dlo = D.node_lo, *dhi = D.node_hi;
    for (int64_t i = 0; i < nl; i++) {
        const double *lo = D.node_lo + 3 * leaf_node[i], *hi = D.node_hi + 3 * leaf_node[i];
        for (int w = 0; w < 6; w++) {
            const int a = w >> 1, s = w & 1;
            const int64_t b0 = D.nbr_off[6 * i + w], b1 = D.nbr_off[6 * i + w + 1];
            if (b1 < b0) { hg::set_error("nbr_off not monotone at leaf %lld", (long long)i); return HG_EFORMAT; }
            const double plane = s ? hi[a] : lo[a];
            const bool boundary = s ? (plane == dhi[a]) : (plane == dlo[a]);
            if (boundary != (b1 == b0)) {
                hg::set_error("leaf %lld wall %d: list must be empty exactly on the domain boundary", (long long)i, w);
                return HG_EFORMAT;
            }
            const int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
            const double wall_area = (hi[t1] - lo[t1]) * (hi[t2] - lo[t2]);
            double sum = 0.0, prev = INFINITY;
            for (int64_t e = b0; e < b1; e++) {
                const int32_t j = D.nbr_id[e];
                if (j < 0 || j >= nl) { hg::set_error("neighbor id %d out of range", j); return HG_EFORMAT; }
                const double *jlo = D.node_lo + 3 * leaf_node[j], *jhi = D.node_hi + 3 * leaf_node[j];
                if ((s ? jlo[a] : jhi[a]) != plane) {
                    hg::set_error("leaf %lld wall %d: neighbor %d is not adjacent", (long long)i, w, j);
                    return HG_EFORMAT;
                }
                double o1 = std::min(hi[t1], jhi[t1]) - std::max(lo[t1], jlo[t1]);
                double o2 = std::min(hi[t2], jhi[t2]) - std::max(lo[t2], jlo[t2]);
                if (!(o1 > 0.0 && o2 > 0.0)) {
                    hg::set_error("leaf %lld wall %d: neighbor %d has no overlap", (long long)i, w, j);
                    return HG_EFORMAT;
                }
                double area = o1 * o2;
                if (area > prev * (1.0 + 1e-12)) {
                    hg::set_error("leaf %lld wall %d: list not sorted by decreasing overlap", (long long)i, w);
                    return HG_EFORMAT;
                }
                prev = area;
                sum += area;
            }
            if (b1 > b0 && std::fabs(sum - wall_area) > 1e-9 * wall_area) {
                hg::set_error("leaf %lld wall %d: neighbors do not tile the wall", (long long)i, w);
                return HG_EFORMAT;
            }
        }
    }
    return HG_OK;
}

// Does node nd lie across leaf wall (a, s) at plane P -- on the far side of
// it, touching it -- and cover the wall's face [flo, fhi] on the two other
// axes?
bool rope_covers(const hg_grid_desc &D, int64_t nd, int a, int s, double P, const double *flo, const double *fhi) {
    const double *lo = D.node_lo + 3 * nd, *hi = D.node_hi + 3 * nd;
    const bool across = s ? (lo[a] <= P && P < hi[a]) : (lo[a] < P && P <= hi[a]);
    if (!across) return false;
    for (int b = 0; b < 3; b++)
        if (b != a && !(lo[b] <= flo[b] && fhi[b] <= hi[b])) return false;
    return true;
}

// The rope of wall w of the leaf node ln: the deepest node across the wall
// that covers the whole face, found by a descent from the root that goes on
// while exactly one child covers it.  Encoded as the leaf id (>= 0), -1 on
// the domain boundary, or -2 - node for an internal node.
int32_t rope_of(const hg_grid_desc &D, int64_t ln, int w) {
    const int a = w >> 1, s = w & 1;
    const double *flo = D.node_lo + 3 * ln, *fhi = D.node_hi + 3 * ln;
    const double P = s ? fhi[a] : flo[a];
    if (P == (s ? D.node_hi[a] : D.node_lo[a])) return -1;
    const int nch = (D.kind == HG_OCTREE) ? 8 : 2;
    int64_t nd = 0;
    for (;;) {
        const int32_t c = D.child_first[nd];
        if (c < 0) return D.node_leaf[nd];
        int64_t next = -1;
        int hits = 0;
        for (int j = 0; j < nch; j++)
            if (rope_covers(D, (int64_t)c + j, a, s, P, flo, fhi)) {
                next = (int64_t)c + j;
                hits++;
            }
        if (hits != 1) return (int32_t)(-2 - nd);
        nd = next;
    }
}

// Every rope target must lie across its wall and cover the face (then a
// descent from it reaches the leaf holding any exit point of the face);
// exactly the walls on the domain boundary have none.
hg_status validate_ropes(const hg_grid_desc &D, const std::vector<int64_t> &leaf_node, const int32_t *ropes) {
    const int64_t nl = D.n_leaves, n = D.n_nodes;
    for (int64_t i = 0; i < nl; i++) {
        const int64_t ln = leaf_node[(size_t)i];
        const double *flo = D.node_lo + 3 * ln, *fhi = D.node_hi + 3 * ln;
        for (int w = 0; w < 6; w++) {
            const int a = w >> 1, s = w & 1;
            const double P = s ? fhi[a] : flo[a];
            const bool boundary = P == (s ? D.node_hi[a] : D.node_lo[a]);
            const int32_t r = ropes[6 * i + w];
            int64_t nd = -1;
            if (r >= 0 && r < nl) nd = leaf_node[(size_t)r];
            if (r <= -2 && -2 - (int64_t)r < n) nd = -2 - (int64_t)r;
            if (boundary ? (r != -1) : (nd < 0 || !rope_covers(D, nd, a, s, P, flo, fhi))) {
                hg::set_error("leaf %lld wall %d: rope %d does not cover the wall", (long long)i, w, r);
                return HG_EFORMAT;
            }
        }
    }
    return HG_OK;
}

hg_status load_grid_impl(const hg_grid_desc *desc, const int32_t *ropes, int32_t validate_flag, hg_grid **out);

}  // namespace

extern "C" hg_status hg_build_ropes(const hg_grid_desc *desc, int32_t n_threads, int32_t *ropes) {
    if (!desc || !ropes || desc->n_leaves < 1 || desc->n_nodes < 1 || !desc->node_lo || !desc->node_hi ||
        !desc->child_first || !desc->node_leaf || (desc->kind != HG_OCTREE && desc->kind != HG_KDTREE)) {
        hg::set_error("hg_build_ropes: incomplete description or no output");
        return HG_EINVAL;
    }
    const hg_grid_desc D = *desc;
    try {
        std::vector<int64_t> leaf_node((size_t)D.n_leaves, -1);
        const int nch = (D.kind == HG_OCTREE) ? 8 : 2;
        for (int64_t i = 0; i < D.n_nodes; i++) {
            const int32_t l = D.node_leaf[i], c = D.child_first[i];
            if (l >= D.n_leaves || (l >= 0) == (c >= 0) || (c >= 0 && (c <= i || (int64_t)c + nch > D.n_nodes))) {
                hg::set_error("hg_build_ropes: bad leaf id or child link at node %lld", (long long)i);
                return HG_EFORMAT;
            }
            if (l >= 0) leaf_node[(size_t)l] = i;
        }
        for (int64_t i = 0; i < D.n_leaves; i++)
            if (leaf_node[(size_t)i] < 0) {
                hg::set_error("hg_build_ropes: leaf %lld has no node", (long long)i);
                return HG_EFORMAT;
            }
        const int threads = n_threads > 0 ? n_threads : (int)std::max(1u, std::thread::hardware_concurrency());
        std::atomic<int64_t> next{0};
        const int64_t chunk = 4096;
        auto work = [&]() {
            for (;;) {
                const int64_t a0 = next.fetch_add(chunk);
                if (a0 >= D.n_leaves) break;
                const int64_t a1 = std::min(D.n_leaves, a0 + chunk);
                for (int64_t i = a0; i < a1; i++)
                    for (int w = 0; w < 6; w++) ropes[6 * i + w] = rope_of(D, leaf_node[(size_t)i], w);
            }
        };
        if (threads <= 1 || D.n_leaves < 2 * chunk) {
            work();
        } else {
            std::vector<std::thread> pool;
            for (int t = 0; t < threads; t++) pool.emplace_back(work);
            for (auto &th : pool) th.join();
        }
    } catch (const std::bad_alloc &) {
        hg::set_error("hg_build_ropes: out of host memory");
        return HG_ENOMEM;
    } catch (const std::system_error &) {
        hg::set_error("hg_build_ropes: could not start threads");
        return HG_EINVAL;
    }
    return HG_OK;
}

extern "C" hg_status hg_load_grid(const hg_grid_desc *desc, int32_t validate_flag, hg_grid **out) {
    return load_grid_impl(desc, nullptr, validate_flag, out);
}

extern "C" hg_status hg_load_grid_ropes(const hg_grid_desc *desc, const int32_t *ropes, int32_t validate_flag,
                                        hg_grid **out) {
    if (!desc || !out) { hg::set_error("hg_load_grid_ropes: null argument"); return HG_EINVAL; }
    std::vector<int32_t> own;
    if (!ropes) {
        try {
            own.resize((size_t)std::max<int64_t>(desc->n_leaves, 1) * 6);
        } catch (const std::bad_alloc &) {
            hg::set_error("hg_load_grid_ropes: out of host memory");
            return HG_ENOMEM;
        }
        hg_status st = hg_build_ropes(desc, 0, own.data());
        if (st != HG_OK) return st;
        ropes = own.data();
    }
    return load_grid_impl(desc, ropes, validate_flag, out);
}

namespace {

// Upload a grid; with ropes (host [6 n_leaves]) each leaf record's wall
// slots hold the ropes instead of the neighbor-list heads, and no list
// tails are stored.
hg_status load_grid_impl(const hg_grid_desc *desc, const int32_t *ropes, int32_t validate_flag, hg_grid **out) {
    if (!desc || !out) { hg::set_error("hg_load_grid: null argument"); return HG_EINVAL; }
    *out = nullptr;
    const hg_grid_desc D = *desc;
    if ((D.kind != HG_OCTREE && D.kind != HG_KDTREE) || D.n_nodes < 1 || D.n_leaves < 1 || !D.node_lo ||
        !D.node_hi || !D.child_first || !D.node_leaf || !D.leaf_rho ||
        (!ropes && (!D.nbr_off || (!D.nbr_id && D.nbr_off[6 * D.n_leaves] > 0)))) {
        hg::set_error("hg_load_grid: incomplete description");
        return HG_EINVAL;
    }
    if (D.n_leaves > INT32_MAX || D.n_nodes > INT32_MAX) {
        hg::set_error("hg_load_grid: ids must fit in int32");
        return HG_EINVAL;
    }
    if (validate_flag) {
        hg_status st = validate(D, !ropes);
        if (st != HG_OK) return st;
        if (ropes) {
            std::vector<int64_t> ln((size_t)D.n_leaves);
            for (int64_t i = 0; i < D.n_nodes; i++)
                if (D.node_leaf[i] >= 0) ln[(size_t)D.node_leaf[i]] = i;
            if ((st = validate_ropes(D, ln, ropes)) != HG_OK) return st;
        }
    }
    const int64_t n = D.n_nodes, nl = D.n_leaves;
    std::unique_ptr<hg_grid> g(new hg_grid());
    try {
        // node depths for the descent limit
        std::vector<int32_t> depth((size_t)n, 0);
        int32_t max_depth = 0;
        const int nch = (D.kind == HG_OCTREE) ? 8 : 2;
        for (int64_t i = 0; i < n; i++)
            if (D.child_first[i] >= 0)
                for (int j = 0; j < nch; j++) {
                    depth[D.child_first[i] + j] = depth[i] + 1;
                    max_depth = std::max(max_depth, depth[i] + 1);
                }
        // descent nodes
        std::vector<unsigned char> nodes;
        if (D.kind == HG_KDTREE) {
            nodes.resize((size_t)n * sizeof(hg::KdNode));
            hg::KdNode *K = reinterpret_cast<hg::KdNode *>(nodes.data());
            for (int64_t i = 0; i < n; i++) {
                const int32_t c = D.child_first[i];
                K[i].child = c;
                if (c < 0) {
                    K[i].split = 0;
                    K[i].info = D.node_leaf[i];
                } else {
                    int ax = 0;
                    while (ax < 2 && D.node_hi[3 * (int64_t)c + ax] == D.node_hi[3 * i + ax]) ax++;
                    K[i].split = hg::host_okey(D.node_hi[3 * (int64_t)c + ax]);
                    K[i].info = ax;
                }
            }
        } else {
            nodes.resize((size_t)n * sizeof(hg::OctNode));
            hg::OctNode *O = reinterpret_cast<hg::OctNode *>(nodes.data());
            for (int64_t i = 0; i < n; i++) {
                const int32_t c = D.child_first[i];
                O[i].child = c;
                O[i].leaf = D.node_leaf[i];
                for (int a = 0; a < 3; a++) O[i].s[a] = (c < 0) ? 0 : hg::host_okey(D.node_hi[3 * (int64_t)c + a]);
            }
        }
        // leaf records and neighbor-list tails
        std::vector<int64_t> leaf_node((size_t)nl);
        for (int64_t i = 0; i < n; i++)
            if (D.node_leaf[i] >= 0) leaf_node[D.node_leaf[i]] = i;
        std::vector<hg::LeafRec> rec((size_t)nl);
        std::vector<int32_t> tail;
        int64_t long_walls = 0;
        // A list too long to scan keeps one tail entry instead: the wall's rope node (the deepest
        // node across the wall that covers the whole face), where the top-down search for the exit
        // point can start instead of the root.
        std::vector<int32_t> wall_ropes;
        if (!ropes) {
            bool any_long = false;
            for (int64_t i = 0; i < 6 * nl && !any_long; i++) any_long = D.nbr_off[i + 1] - D.nbr_off[i] > kScanLimit;
            if (any_long) {
                wall_ropes.resize((size_t)(6 * nl));
                hg_status st = hg_build_ropes(desc, 0, wall_ropes.data());
                if (st != HG_OK) return st;
            }
        }
        const double *dhi = D.node_hi;
        for (int64_t i = 0; i < nl; i++) {
            hg::LeafRec &R = rec[i];
            std::memset(&R, 0, sizeof(R));
            const int64_t nd = leaf_node[i];
            for (int a = 0; a < 3; a++) {
                R.lo[a] = hg::host_okey(D.node_lo[3 * nd + a]);
                R.hi[a] = hg::host_okey(D.node_hi[3 * nd + a]);
                if (D.node_hi[3 * nd + a] == dhi[a]) R.flags |= (uint8_t)(1u << a);
            }
            R.rho = D.leaf_rho[i];
            R.rho32 = (float)D.leaf_rho[i];
            if (tail.size() > UINT32_MAX) {
                hg::set_error("hg_load_grid: neighbor tails exceed 2^32 entries");
                return HG_EOVERFLOW;
            }
            R.nbr_base = (uint32_t)tail.size();
            if (ropes) {
                for (int w = 0; w < 6; w++) {
                    R.first[w] = ropes[6 * i + w];
                    R.cnt[w] = 0;
                }
                continue;
            }
            for (int w = 0; w < 6; w++) {
                const int64_t b0 = D.nbr_off[6 * i + w], b1 = D.nbr_off[6 * i + w + 1];
                const int64_t cnt = b1 - b0;
                R.first[w] = cnt > 0 ? D.nbr_id[b0] : -1;
                R.cnt[w] = (uint8_t)std::min<int64_t>(cnt, 255);
                if (cnt >= 2 && cnt <= kScanLimit) {
                    for (int64_t e = b0 + 1; e < b1; e++) tail.push_back(D.nbr_id[e]);
                } else if (cnt > kScanLimit) {
                    const int32_t r = wall_ropes[(size_t)(6 * i + w)];
                    tail.push_back(r <= -2 ? -2 - r : -1);  // an internal node; -1: search from the root
                    long_walls++;
                }
            }
        }
        if (tail.empty()) tail.push_back(-1);
        // expected crossings per unit length on a coarse lattice (work estimate)
        std::vector<float> work((size_t)hg::kWorkN * hg::kWorkN * hg::kWorkN, 0.0f);
        {
            const int N = hg::kWorkN;
            double ext[3], cvol = 1.0;
            for (int a = 0; a < 3; a++) {
                ext[a] = D.node_hi[a] - D.node_lo[a];
                cvol *= ext[a] / N;
            }
            std::vector<double> acc(work.size(), 0.0);
            for (int64_t i = 0; i < nl; i++) {
                const double *lo = D.node_lo + 3 * leaf_node[i], *hi = D.node_hi + 3 * leaf_node[i];
                const double a = hi[0] - lo[0], b = hi[1] - lo[1], c = hi[2] - lo[2];
                const double rate = (a * b + b * c + c * a) / (2.0 * a * b * c);
                int c0[3], c1[3];
                for (int ax = 0; ax < 3; ax++) {
                    c0[ax] = std::max(0, std::min(N - 1, (int)std::floor((lo[ax] - D.node_lo[ax]) / ext[ax] * N)));
                    c1[ax] = std::max(0, std::min(N - 1, (int)std::ceil((hi[ax] - D.node_lo[ax]) / ext[ax] * N) - 1));
                }
                for (int z = c0[2]; z <= c1[2]; z++)
                    for (int y = c0[1]; y <= c1[1]; y++)
                        for (int x = c0[0]; x <= c1[0]; x++) {
                            const int cc[3] = {x, y, z};
                            double ov = 1.0;
                            for (int ax = 0; ax < 3; ax++) {
                                const double l = D.node_lo[ax] + ext[ax] * cc[ax] / N;
                                const double h = D.node_lo[ax] + ext[ax] * (cc[ax] + 1) / N;
                                ov *= std::max(0.0, std::min(h, hi[ax]) - std::max(l, lo[ax]));
                            }
                            acc[(size_t)x + N * ((size_t)y + N * z)] += ov * rate;
                        }
            }
            for (size_t j = 0; j < work.size(); j++) work[j] = (float)(acc[j] / cvol);
        }

        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return cuda_fail(e, "hg_load_grid: no CUDA device");
        g->device = dev;
        auto upload = [&](void **dst, const void *src, size_t bytes) -> cudaError_t {
            cudaError_t r = cudaMalloc(dst, bytes);
            if (r != cudaSuccess) return r;
            return cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
        };
        if ((e = upload(&g->d_rec, rec.data(), rec.size() * sizeof(hg::LeafRec))) != cudaSuccess ||
            (e = upload(&g->d_tail, tail.data(), tail.size() * sizeof(int32_t))) != cudaSuccess ||
            (e = upload(&g->d_nodes, nodes.data(), nodes.size())) != cudaSuccess ||
            (e = upload(&g->d_work, work.data(), work.size() * sizeof(float))) != cudaSuccess) {
            hg_status st = cuda_fail(e, "hg_load_grid: upload");
            hg_free_grid(g.release());
            return st;
        }
        hg::DevGrid &G = g->d;
        G.rec = static_cast<const hg::LeafRec *>(g->d_rec);
        G.tail = static_cast<const int32_t *>(g->d_tail);
        G.nodes = g->d_nodes;
        G.work = static_cast<const float *>(g->d_work);
        G.work_n = hg::kWorkN;
        for (int a = 0; a < 3; a++) {
            G.dlo[a] = D.node_lo[a];
            G.dhi[a] = D.node_hi[a];
            G.klo[a] = hg::host_okey(G.dlo[a]);
            G.khi[a] = hg::host_okey(G.dhi[a]);
        }
        G.n_leaves = nl;
        G.n_nodes = n;
        G.kind = D.kind;
        G.max_depth = max_depth;
        G.scan_limit = kScanLimit;
        G.nav = ropes ? HG_NAV_ROPES : HG_NAV_NEIGHBOR_LISTS;
        G.pad = 0;
        hg_grid_info &I = g->info;
        I.kind = D.kind;
        I.max_depth = max_depth;
        I.n_nodes = n;
        I.n_leaves = nl;
        I.n_tail = (int64_t)tail.size();
        I.device_bytes = (int64_t)(rec.size() * sizeof(hg::LeafRec) + tail.size() * 4 + nodes.size() +
                                   work.size() * sizeof(float));
        I.long_walls = long_walls;
        I.nav = ropes ? HG_NAV_ROPES : HG_NAV_NEIGHBOR_LISTS;
        I.reserved = 0;
        for (int a = 0; a < 3; a++) {
            I.lo[a] = G.dlo[a];
            I.hi[a] = G.dhi[a];
        }
    } catch (const std::bad_alloc &) {
        hg::set_error("hg_load_grid: out of host memory");
        return HG_ENOMEM;
    }
    *out = g.release();
    return HG_OK;
}

}  // namespace

extern "C" void hg_free_grid(hg_grid *g) {
    if (!g) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != g->device) cudaSetDevice(g->device);
    if (g->d_rec) cudaFree(g->d_rec);
    if (g->d_tail) cudaFree(g->d_tail);
    if (g->d_nodes) cudaFree(g->d_nodes);
    if (g->d_work) cudaFree(g->d_work);
    if (cur != g->device) cudaSetDevice(cur);
    delete g;
}

extern "C" hg_status hg_grid_get_info(const hg_grid *g, hg_grid_info *out) {
    if (!g || !out) { hg::set_error("hg_grid_get_info: null argument"); return HG_EINVAL; }
    *out = g->info;
    return HG_OK;
}
