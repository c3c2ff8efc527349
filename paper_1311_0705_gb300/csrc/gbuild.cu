// Tree construction on the device (Sect. 2.2, 2.3, 4.1, 4.2).  The node list
// grows a level at a time as in the host builder: the Monte Carlo evaluation
// of a level's nodes -- n_ran density draws per node for the mass fraction
// (Eq. 1), optical depth (Eq. 2) and density dispersion (Eq. 3) criteria --
// one thread per node; a scan of the child counts; the children of the
// nodes to subdivide appended in parent order.  Then the leaves are numbered
// in node order, the bounds computed, and the neighbor lists found (one
// thread per leaf wall).  The arithmetic is the host builder's
// (model_eval.h, compiled with -fmad=false like the host's
// -ffp-contract=off), so the draws, bounds, sums and decisions match it
// except where CUDA's exp rounds differently from the host's libm (disk and
// clump models).  Everything stays on the device until one copy at the end.
#include <cuda_runtime.h>

#include <algorithm>

#include "hg_internal.h"
#include "gbuild.h"
#include "model_eval.h"

namespace hg {
hg_status cuda_err(cudaError_t e, const char *what);
int sm_count();

__global__ void __launch_bounds__(256) build_eval_kernel(const ModelView M, const hg_build_params P, int64_t n,
                                                         const int32_t *__restrict__ lvl,
                                                         const int64_t *__restrict__ idx, NodeStats *out) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t l[3] = {lvl[3 * j], lvl[3 * j + 1], lvl[3 * j + 2]};
        const int64_t i[3] = {idx[3 * j], idx[3 * j + 1], idx[3 * j + 2]};
        const int32_t depth = (P.kind == HG_OCTREE) ? l[0] : l[0] + l[1] + l[2];
        out[j] = eval_node_stats(M, P, l, i, depth);
    }
}

static cudaError_t upload(void **dst, const void *src, size_t bytes, cudaStream_t s) {
    cudaError_t e = cudaMalloc(dst, std::max<size_t>(bytes, 16));
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, s);
    return e;
}

// ---------------------------------------------------------------- neighbor lists
// In integer lattice units of the finest per-axis level Lm: a node at level
// l with index i spans [i 2^(Lm-l), (i+1) 2^(Lm-l)) on that axis, so walls
// and overlaps are compared exactly.
struct NbrTree {
    int32_t kind, Lm;
    const int32_t *lvl;
    const int64_t *idx;
    const int32_t *child;
    const int32_t *leaf;
    const int64_t *leaf_node;
};

// Octree: at most 7 siblings wait per level (depth <= 20); k-d: one per level
// (depth <= 60).  A walk that would need more reports it instead.
constexpr int kNbrStack = 192;

__device__ __forceinline__ void nbr_box(const NbrTree &T, int64_t nd, int b, int64_t &lo, int64_t &hi) {
    const int32_t l = T.lvl[3 * nd + b];
    const int64_t i = T.idx[3 * nd + b];
    lo = i << (T.Lm - l);
    hi = (i + 1) << (T.Lm - l);
}

// Visit every leaf across wall w (axis w / 2, upper side when w is odd) of
// leaf node ln that overlaps the wall with positive area: a depth-first
// descent from the root through the nodes that straddle the wall plane and
// overlap the wall.  fn(leaf id, area).  Returns false if the stack would
// overflow.
template <class F>
__device__ bool nbr_walk(const NbrTree &T, int64_t ln, int w, F &&fn) {
    const int a = w >> 1, s = w & 1;
    int64_t L[3], H[3];
    for (int b = 0; b < 3; b++) nbr_box(T, ln, b, L[b], H[b]);
    const int64_t P = s ? H[a] : L[a];
    if ((s && P == ((int64_t)1 << T.Lm)) || (!s && P == 0)) return true;  // a wall of the domain
    const int nch = (T.kind == HG_OCTREE) ? 8 : 2;
    int32_t stack[kNbrStack];
    int sp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const int32_t nd = stack[--sp];
        int64_t nlo[3], nhi[3];
        for (int b = 0; b < 3; b++) nbr_box(T, nd, b, nlo[b], nhi[b]);
        const bool across = s ? (nlo[a] <= P && P < nhi[a]) : (nlo[a] < P && P <= nhi[a]);
        if (!across) continue;
        int64_t area = 1;
        bool ok = true;
        for (int b = 0; b < 3; b++) {
            if (b == a) continue;
            const int64_t ov = (nhi[b] < H[b] ? nhi[b] : H[b]) - (nlo[b] > L[b] ? nlo[b] : L[b]);
            if (ov <= 0) {
                ok = false;
                break;
            }
            area *= ov;
        }
        if (!ok) continue;
        const int32_t c = T.child[nd];
        if (c < 0) {
            fn(T.leaf[nd], area);
        } else {
            if (sp + nch > kNbrStack) return false;
            for (int k = nch - 1; k >= 0; k--) stack[sp++] = c + k;
        }
    }
    return true;
}

__global__ void __launch_bounds__(256) nbr_count_kernel(const NbrTree T, int64_t nl, int32_t *counts,
                                                        uint32_t *err) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 6 * nl; t += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = 0;
        if (!nbr_walk(T, T.leaf_node[t / 6], (int)(t % 6), [&](int32_t, int64_t) { c++; })) atomicOr(err, 1u);
        counts[t] = c;
    }
}

// Each wall's list written at its offset, then sorted in place by
// decreasing area, ties by ascending id.
__global__ void __launch_bounds__(256) nbr_fill_kernel(const NbrTree T, int64_t nl, const int64_t *__restrict__ off,
                                                       int32_t *ids, int64_t *areas, uint32_t *err) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 6 * nl; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = off[t], e = off[t + 1];
        int64_t k = b;
        const bool ok = nbr_walk(T, T.leaf_node[t / 6], (int)(t % 6), [&](int32_t id, int64_t area) {
            if (k < e) {
                ids[k] = id;
                areas[k] = area;
            }
            k++;
        });
        if (!ok || k != e) {
            atomicOr(err, 2u);
            continue;
        }
        // Shell sort (Ciura's gaps), so that the few long lists beside strongly refined regions
        // stay cheap; the keys (area, id) are distinct within a list
        const int64_t len = e - b;
        const int gaps[8] = {701, 301, 132, 57, 23, 10, 4, 1};
        for (int gi = 0; gi < 8; gi++) {
            const int64_t gap = gaps[gi];
            if (gap >= len) continue;
            for (int64_t x = b + gap; x < e; x++) {
                const int32_t id = ids[x];
                const int64_t ar = areas[x];
                int64_t y = x;
                while (y - gap >= b && (areas[y - gap] < ar || (areas[y - gap] == ar && ids[y - gap] > id))) {
                    ids[y] = ids[y - gap];
                    areas[y] = areas[y - gap];
                    y -= gap;
                }
                ids[y] = id;
                areas[y] = ar;
            }
        }
    }
}

// The neighbor lists of a node list held on the device: count, scan, fill
// and sort, then copied to the host.
static hg_status device_neighbors(const NbrTree &T, int64_t nl, cudaStream_t s, std::vector<int64_t> &nbr_off,
                                  std::vector<int32_t> &nbr_id) {
    int32_t *d_cnt = nullptr, *d_ids = nullptr;
    int64_t *d_off = nullptr, *d_area = nullptr;
    uint32_t *d_err = nullptr;
    hg_status hs = HG_OK;
    int64_t total = 0;
    uint32_t err = 0;
    const int64_t nw = 6 * nl;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nw + 255) / 256, (int64_t)sm_count() * 16));
    cudaError_t e = cudaMalloc((void **)&d_cnt, (size_t)std::max<int64_t>(nw, 1) * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc((void **)&d_off, (size_t)(nw + 1) * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc((void **)&d_err, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess && nw > 0) {
        nbr_count_kernel<<<blocks, 256, 0, s>>>(T, nl, d_cnt, d_err);
        note_launches(1);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        hs = cuda_err(e, "device neighbor lists: count");
    else
        hs = hg_scan_offsets(nw, d_cnt, d_off, s);
    if (hs == HG_OK) {
        e = cudaMemcpyAsync(&total, d_off + nw, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaMalloc((void **)&d_ids, (size_t)std::max<int64_t>(total, 1) * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMalloc((void **)&d_area, (size_t)std::max<int64_t>(total, 1) * sizeof(int64_t));
        if (e == cudaSuccess && nw > 0) {
            nbr_fill_kernel<<<blocks, 256, 0, s>>>(T, nl, d_off, d_ids, d_area, d_err);
            note_launches(1);
            e = cudaGetLastError();
        }
        try {
            nbr_off.assign((size_t)nw + 1, 0);
            nbr_id.assign((size_t)total, 0);
        } catch (const std::bad_alloc &) {
            set_error("device neighbor lists: out of host memory");
            hs = HG_ENOMEM;
        }
        if (hs == HG_OK && e == cudaSuccess)
            e = cudaMemcpyAsync(nbr_off.data(), d_off, (size_t)(nw + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (hs == HG_OK && e == cudaSuccess && total > 0)
            e = cudaMemcpyAsync(nbr_id.data(), d_ids, (size_t)total * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (hs == HG_OK && e == cudaSuccess)
            e = cudaMemcpyAsync(&err, d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (hs == HG_OK && e != cudaSuccess) hs = cuda_err(e, "device neighbor lists: fill");
        if (hs == HG_OK && err) {
            set_error("device neighbor lists: descent stack exceeded or list mismatch (flags %u)", err);
            hs = HG_EOVERFLOW;
        }
    }
    cudaStreamSynchronize(s);
    cudaFree(d_cnt);
    cudaFree(d_off);
    cudaFree(d_err);
    cudaFree(d_ids);
    cudaFree(d_area);
    return hs;
}

// ---------------------------------------------------------------- the level loop
__global__ void __launch_bounds__(256) child_count_kernel(int64_t begin, int64_t m, const NodeStats *__restrict__ st,
                                                          int nch, int32_t *cnt) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
        cnt[j] = st[begin + j].sub ? nch : 0;
}

// Children of the level's nodes to subdivide, in parent order from `end`:
// octree child c at (2 i_a + bit a of c) on every axis; k-d child c at
// 2 i + c on the node's split axis.
__global__ void __launch_bounds__(256) append_kernel(int32_t kind, int64_t begin, int64_t end, int64_t m,
                                                     const NodeStats *__restrict__ st, const int64_t *__restrict__ off,
                                                     int32_t *lvl, int64_t *idx, int32_t *child) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t nd = begin + j;
        if (!st[nd].sub) {
            child[nd] = -1;
            continue;
        }
        const int64_t first = end + off[j];
        child[nd] = (int32_t)first;
        const int32_t l[3] = {lvl[3 * nd], lvl[3 * nd + 1], lvl[3 * nd + 2]};
        const int64_t i[3] = {idx[3 * nd], idx[3 * nd + 1], idx[3 * nd + 2]};
        if (kind == HG_OCTREE) {
            for (int c = 0; c < 8; c++)
                for (int a = 0; a < 3; a++) {
                    lvl[3 * (first + c) + a] = l[a] + 1;
                    idx[3 * (first + c) + a] = 2 * i[a] + ((c >> a) & 1);
                }
        } else {
            const int axis = st[nd].axis;
            for (int c = 0; c < 2; c++)
                for (int a = 0; a < 3; a++) {
                    lvl[3 * (first + c) + a] = a == axis ? l[a] + 1 : l[a];
                    idx[3 * (first + c) + a] = a == axis ? 2 * i[a] + c : i[a];
                }
        }
    }
}

__global__ void __launch_bounds__(256) leaf_flag_kernel(int64_t n, const int32_t *__restrict__ child, int32_t *flag) {
    for (int64_t nd = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; nd < n; nd += (int64_t)gridDim.x * blockDim.x)
        flag[nd] = child[nd] < 0 ? 1 : 0;
}

// Leaf ids in node order, the nodes' bounds, and the statistics split per field.
__global__ void __launch_bounds__(256) finish_kernel(const ModelView M, int64_t n, const int32_t *__restrict__ lvl,
                                                     const int64_t *__restrict__ idx, const int32_t *__restrict__ child,
                                                     const int64_t *__restrict__ loff, const NodeStats *__restrict__ st,
                                                     int32_t *leaf, int64_t *leaf_node, double *leaf_rho, double *lo,
                                                     double *hi, double *rho, double *mass, double *delta, double *tau,
                                                     double *q) {
    for (int64_t nd = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; nd < n; nd += (int64_t)gridDim.x * blockDim.x) {
        const NodeStats S = st[nd];
        if (child[nd] < 0) {
            const int64_t li = loff[nd];
            leaf[nd] = (int32_t)li;
            leaf_node[li] = nd;
            leaf_rho[li] = S.rho;
        } else {
            leaf[nd] = -1;
        }
        for (int a = 0; a < 3; a++) {
            lo[3 * nd + a] = model_bound(M, a, idx[3 * nd + a], lvl[3 * nd + a]);
            hi[3 * nd + a] = model_bound(M, a, idx[3 * nd + a] + 1, lvl[3 * nd + a]);
        }
        rho[nd] = S.rho;
        mass[nd] = S.mass;
        delta[nd] = S.delta;
        tau[nd] = S.tau;
        q[nd] = S.q;
    }
}

namespace {

// Device buffers of the build, released together.
struct BuildBufs {
    std::vector<void *> ptrs;
    ~BuildBufs() {
        for (void *p : ptrs) cudaFree(p);
    }
    template <class T>
    cudaError_t alloc(T **p, int64_t count) {
        *p = nullptr;
        cudaError_t e = cudaMalloc((void **)p, (size_t)std::max<int64_t>(count, 1) * sizeof(T));
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
    void release(void *p) {
        for (auto &q : ptrs)
            if (q == p) {
                cudaFree(q);
                q = nullptr;
            }
    }
};

template <class T>
cudaError_t grow(BuildBufs &B, T **p, int64_t used, int64_t cap, cudaStream_t s) {
    T *q = nullptr;
    cudaError_t e = B.alloc(&q, cap);
    if (e == cudaSuccess && used > 0) e = cudaMemcpyAsync(q, *p, (size_t)used * sizeof(T), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
        B.release(*p);
        *p = q;
    }
    return e;
}

template <class T>
cudaError_t fetch(std::vector<T> &v, const T *d, int64_t count, cudaStream_t s) {
    v.resize((size_t)count);
    return count > 0 ? cudaMemcpyAsync(v.data(), d, (size_t)count * sizeof(T), cudaMemcpyDeviceToHost, s)
                     : cudaSuccess;
}

}  // namespace

hg_status gpu_build_tree(const ModelView &hm, const hg_build_params &P, hg_stream stream, GpuTree &out) {
    cudaStream_t s = (cudaStream_t)stream;
    BuildBufs B;
    // the model on the device
    ModelView dv = hm;
    double *d_table = nullptr;
    int32_t *d_coff = nullptr, *d_cids = nullptr;
    const size_t per = (hm.kind == HG_MODEL_TORUS) ? 5 : 1;
    const int64_t ntab = hm.n_table > 0 ? (int64_t)hm.n_table * (int64_t)per : 0;
    cudaError_t e = B.alloc(&d_table, ntab);
    if (e == cudaSuccess && ntab > 0)
        e = cudaMemcpyAsync(d_table, hm.table, (size_t)ntab * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && hm.G > 0) {
        const int64_t ncell = (int64_t)hm.G * hm.G * hm.G;
        e = B.alloc(&d_coff, ncell + 1);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d_coff, hm.cell_off, (size_t)(ncell + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = B.alloc(&d_cids, (int64_t)hm.cell_off[ncell]);
        if (e == cudaSuccess && hm.cell_off[ncell] > 0)
            e = cudaMemcpyAsync(d_cids, hm.cell_ids, (size_t)hm.cell_off[ncell] * sizeof(int32_t),
                                cudaMemcpyHostToDevice, s);
    }
    if (e != cudaSuccess) return cuda_err(e, "device builder: model upload");
    dv.table = d_table;
    dv.cell_off = d_coff;
    dv.cell_ids = d_cids;
    // the node list: root first
    int64_t cap = 1 << 16;
    int32_t *d_lvl = nullptr, *d_child = nullptr, *d_cnt = nullptr;
    int64_t *d_idx = nullptr, *d_off = nullptr;
    NodeStats *d_st = nullptr;
    e = B.alloc(&d_lvl, 3 * cap);
    if (e == cudaSuccess) e = B.alloc(&d_idx, 3 * cap);
    if (e == cudaSuccess) e = B.alloc(&d_child, cap);
    if (e == cudaSuccess) e = B.alloc(&d_st, cap);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_lvl, 0, 3 * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_idx, 0, 3 * sizeof(int64_t), s);
    if (e != cudaSuccess) return cuda_err(e, "device builder: node list");
    const int nch = (P.kind == HG_OCTREE) ? 8 : 2;
    int64_t begin = 0, end = 1, scan_cap = 0;
    while (begin < end) {
        const int64_t m = end - begin;
        const unsigned blocks = (unsigned)std::min<int64_t>((m + 255) / 256, (int64_t)sm_count() * 16);
        build_eval_kernel<<<blocks, 256, 0, s>>>(dv, P, m, d_lvl + 3 * begin, d_idx + 3 * begin, d_st + begin);
        note_launches(1);
        if (m > scan_cap) {
            B.release(d_cnt);
            B.release(d_off);
            scan_cap = std::max<int64_t>(m, 2 * scan_cap);
            e = B.alloc(&d_cnt, scan_cap);
            if (e == cudaSuccess) e = B.alloc(&d_off, scan_cap + 1);
            if (e != cudaSuccess) return cuda_err(e, "device builder: scan buffers");
        }
        child_count_kernel<<<blocks, 256, 0, s>>>(begin, m, d_st, nch, d_cnt);
        note_launches(1);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_err(e, "device builder: node evaluation");
        hg_status hs = hg_scan_offsets(m, d_cnt, d_off, stream);
        if (hs != HG_OK) return hs;
        int64_t added = 0;
        e = cudaMemcpyAsync(&added, d_off + m, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_err(e, "device builder: level");
        if (P.max_nodes > 0 && end + added > P.max_nodes) {
            set_error("hg_build_grid: more than max_nodes=%lld nodes", (long long)P.max_nodes);
            return HG_EOVERFLOW;
        }
        if (end + added > INT32_MAX) {
            set_error("hg_build_grid: node count exceeds int32 ids");
            return HG_EOVERFLOW;
        }
        if (end + added > cap) {
            const int64_t nc = std::max<int64_t>(end + added, 2 * cap);
            e = grow(B, &d_lvl, 3 * end, 3 * nc, s);
            if (e == cudaSuccess) e = grow(B, &d_idx, 3 * end, 3 * nc, s);
            if (e == cudaSuccess) e = grow(B, &d_child, end, nc, s);
            if (e == cudaSuccess) e = grow(B, &d_st, end, nc, s);
            if (e != cudaSuccess) return cuda_err(e, "device builder: node list growth");
            cap = nc;
        }
        append_kernel<<<blocks, 256, 0, s>>>(P.kind, begin, end, m, d_st, d_off, d_lvl, d_idx, d_child);
        note_launches(1);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_err(e, "device builder: children");
        begin = end;
        end += added;
    }
    // leaves, bounds, statistics
    const int64_t n = end;
    int32_t *d_flag = nullptr, *d_leaf = nullptr;
    int64_t *d_loff = nullptr, *d_ln = nullptr;
    double *d_lrho = nullptr, *d_lo = nullptr, *d_hi = nullptr, *d_f = nullptr;
    e = B.alloc(&d_flag, n);
    if (e == cudaSuccess) e = B.alloc(&d_loff, n + 1);
    if (e == cudaSuccess) e = B.alloc(&d_leaf, n);
    if (e != cudaSuccess) return cuda_err(e, "device builder: leaves");
    const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 16));
    leaf_flag_kernel<<<nb, 256, 0, s>>>(n, d_child, d_flag);
    note_launches(1);
    hg_status hs = hg_scan_offsets(n, d_flag, d_loff, stream);
    if (hs != HG_OK) return hs;
    int64_t nl = 0;
    e = cudaMemcpyAsync(&nl, d_loff + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = B.alloc(&d_ln, nl);
    if (e == cudaSuccess) e = B.alloc(&d_lrho, nl);
    if (e == cudaSuccess) e = B.alloc(&d_lo, 3 * n);
    if (e == cudaSuccess) e = B.alloc(&d_hi, 3 * n);
    if (e == cudaSuccess) e = B.alloc(&d_f, 5 * n);
    if (e != cudaSuccess) return cuda_err(e, "device builder: outputs");
    finish_kernel<<<nb, 256, 0, s>>>(dv, n, d_lvl, d_idx, d_child, d_loff, d_st, d_leaf, d_ln, d_lrho, d_lo, d_hi,
                                     d_f, d_f + n, d_f + 2 * n, d_f + 3 * n, d_f + 4 * n);
    note_launches(1);
    e = cudaGetLastError();
    try {
        if (e == cudaSuccess) e = fetch(out.lvl, d_lvl, 3 * n, s);
        if (e == cudaSuccess) e = fetch(out.idx, d_idx, 3 * n, s);
        if (e == cudaSuccess) e = fetch(out.child, d_child, n, s);
        if (e == cudaSuccess) e = fetch(out.leaf, (const int32_t *)d_leaf, n, s);
        if (e == cudaSuccess) e = fetch(out.leaf_node, (const int64_t *)d_ln, nl, s);
        if (e == cudaSuccess) e = fetch(out.leaf_rho, (const double *)d_lrho, nl, s);
        if (e == cudaSuccess) e = fetch(out.lo, (const double *)d_lo, 3 * n, s);
        if (e == cudaSuccess) e = fetch(out.hi, (const double *)d_hi, 3 * n, s);
        if (e == cudaSuccess) e = fetch(out.rho, (const double *)d_f, n, s);
        if (e == cudaSuccess) e = fetch(out.mass, (const double *)d_f + n, n, s);
        if (e == cudaSuccess) e = fetch(out.delta, (const double *)d_f + 2 * n, n, s);
        if (e == cudaSuccess) e = fetch(out.tau, (const double *)d_f + 3 * n, n, s);
        if (e == cudaSuccess) e = fetch(out.q, (const double *)d_f + 4 * n, n, s);
    } catch (const std::bad_alloc &) {
        set_error("device builder: out of host memory");
        return HG_ENOMEM;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_err(e, "device builder: results");
    int32_t Lm = 0;
    for (int32_t v : out.lvl) Lm = std::max(Lm, v);
    const NbrTree T{P.kind, Lm, d_lvl, d_idx, d_child, d_leaf, d_ln};
    return device_neighbors(T, nl, s, out.nbr_off, out.nbr_id);
}

}  // namespace hg
