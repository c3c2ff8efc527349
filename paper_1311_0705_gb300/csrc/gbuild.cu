// Tree construction on the device (Sect. 2.2, 4.1, 4.2): the Monte Carlo
// evaluation of the nodes -- n_ran density draws per node for the mass
// fraction (Eq. 1), optical depth (Eq. 2) and density dispersion (Eq. 3)
// criteria -- one thread per node, a level of the breadth-first node list
// per launch.  The arithmetic is the host builder's (model_eval.h, compiled
// with -fmad=false like the host's -ffp-contract=off), so the draws, bounds,
// sums and decisions match it except where CUDA's exp rounds differently
// from the host's libm (disk and clump models).  The host appends the
// children of the nodes to subdivide; the neighbor lists of the finished
// node list are found on the device too (one thread per leaf wall).
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

struct GpuNodeEval {
    ModelView dv;  // the model with device pointers
    cudaStream_t s = nullptr;
    void *d_table = nullptr, *d_off = nullptr, *d_ids = nullptr;
    int32_t *d_lvl = nullptr;
    int64_t *d_idx = nullptr;
    NodeStats *d_out = nullptr;
    int64_t cap = 0;  // nodes the level buffers hold
};

static cudaError_t upload(void **dst, const void *src, size_t bytes, cudaStream_t s) {
    cudaError_t e = cudaMalloc(dst, std::max<size_t>(bytes, 16));
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyHostToDevice, s);
    return e;
}

hg_status gpu_eval_create(const ModelView &hm, hg_stream stream, GpuNodeEval **out) {
    *out = nullptr;
    GpuNodeEval *E = new GpuNodeEval();
    E->s = (cudaStream_t)stream;
    E->dv = hm;
    const size_t per = (hm.kind == HG_MODEL_TORUS) ? 5 : 1;
    const size_t ntab = hm.n_table > 0 ? (size_t)hm.n_table * per : 0;
    cudaError_t e = upload(&E->d_table, hm.table, ntab * sizeof(double), E->s);
    if (e == cudaSuccess && hm.G > 0) {
        const size_t ncell = (size_t)hm.G * hm.G * hm.G;
        e = upload(&E->d_off, hm.cell_off, (ncell + 1) * sizeof(int32_t), E->s);
        if (e == cudaSuccess) e = upload(&E->d_ids, hm.cell_ids, (size_t)hm.cell_off[ncell] * sizeof(int32_t), E->s);
    }
    if (e != cudaSuccess) {
        gpu_eval_free(E);
        return cuda_err(e, "device builder: model upload");
    }
    E->dv.table = static_cast<const double *>(E->d_table);
    E->dv.cell_off = static_cast<const int32_t *>(E->d_off);
    E->dv.cell_ids = static_cast<const int32_t *>(E->d_ids);
    *out = E;
    return HG_OK;
}

hg_status gpu_eval_level(GpuNodeEval *E, const hg_build_params &P, int64_t n, const int32_t *lvl, const int64_t *idx,
                         NodeStats *out) {
    if (n <= 0) return HG_OK;
    cudaError_t e = cudaSuccess;
    if (n > E->cap) {
        cudaFree(E->d_lvl);
        cudaFree(E->d_idx);
        cudaFree(E->d_out);
        E->d_lvl = nullptr;
        E->d_idx = nullptr;
        E->d_out = nullptr;
        E->cap = 0;
        const int64_t cap = std::max<int64_t>(n, 1 << 16);
        e = cudaMalloc((void **)&E->d_lvl, (size_t)cap * 3 * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMalloc((void **)&E->d_idx, (size_t)cap * 3 * sizeof(int64_t));
        if (e == cudaSuccess) e = cudaMalloc((void **)&E->d_out, (size_t)cap * sizeof(NodeStats));
        if (e != cudaSuccess) return cuda_err(e, "device builder: level buffers");
        E->cap = cap;
    }
    e = cudaMemcpyAsync(E->d_lvl, lvl, (size_t)n * 3 * sizeof(int32_t), cudaMemcpyHostToDevice, E->s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(E->d_idx, idx, (size_t)n * 3 * sizeof(int64_t), cudaMemcpyHostToDevice, E->s);
    if (e != cudaSuccess) return cuda_err(e, "device builder: level upload");
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 16);
    build_eval_kernel<<<(unsigned)blocks, 256, 0, E->s>>>(E->dv, P, n, E->d_lvl, E->d_idx, E->d_out);
    note_launches(1);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, E->d_out, (size_t)n * sizeof(NodeStats), cudaMemcpyDeviceToHost, E->s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(E->s);
    return e == cudaSuccess ? HG_OK : cuda_err(e, "device builder: node evaluation");
}

void gpu_eval_free(GpuNodeEval *E) {
    if (!E) return;
    if (E->s) cudaStreamSynchronize(E->s);
    cudaFree(E->d_table);
    cudaFree(E->d_off);
    cudaFree(E->d_ids);
    cudaFree(E->d_lvl);
    cudaFree(E->d_idx);
    cudaFree(E->d_out);
    delete E;
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

hg_status gpu_build_neighbors(int32_t kind, int64_t n, int64_t nl, const int32_t *lvl, const int64_t *idx,
                              const int32_t *child, const int32_t *leaf, const int64_t *leaf_node, hg_stream stream,
                              std::vector<int64_t> &nbr_off, std::vector<int32_t> &nbr_id) {
    cudaStream_t s = (cudaStream_t)stream;
    int32_t Lm = 0;
    for (int64_t j = 0; j < 3 * n; j++) Lm = std::max(Lm, lvl[j]);
    void *d_lvl = nullptr, *d_idx = nullptr, *d_child = nullptr, *d_leaf = nullptr, *d_ln = nullptr;
    int32_t *d_cnt = nullptr, *d_ids = nullptr;
    int64_t *d_off = nullptr, *d_area = nullptr;
    uint32_t *d_err = nullptr;
    hg_status hs = HG_OK;
    int64_t total = 0;
    uint32_t err = 0;
    const int64_t nw = 6 * nl;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nw + 255) / 256, (int64_t)sm_count() * 16));
    cudaError_t e = upload(&d_lvl, lvl, (size_t)n * 3 * sizeof(int32_t), s);
    if (e == cudaSuccess) e = upload(&d_idx, idx, (size_t)n * 3 * sizeof(int64_t), s);
    if (e == cudaSuccess) e = upload(&d_child, child, (size_t)n * sizeof(int32_t), s);
    if (e == cudaSuccess) e = upload(&d_leaf, leaf, (size_t)n * sizeof(int32_t), s);
    if (e == cudaSuccess) e = upload(&d_ln, leaf_node, (size_t)nl * sizeof(int64_t), s);
    if (e == cudaSuccess) e = cudaMalloc((void **)&d_cnt, (size_t)std::max<int64_t>(nw, 1) * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc((void **)&d_off, (size_t)(nw + 1) * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc((void **)&d_err, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(uint32_t), s);
    NbrTree T{kind, Lm, static_cast<const int32_t *>(d_lvl), static_cast<const int64_t *>(d_idx),
              static_cast<const int32_t *>(d_child), static_cast<const int32_t *>(d_leaf),
              static_cast<const int64_t *>(d_ln)};
    if (e == cudaSuccess && nw > 0) {
        nbr_count_kernel<<<blocks, 256, 0, s>>>(T, nl, d_cnt, d_err);
        note_launches(1);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        hs = cuda_err(e, "device neighbor lists: count");
    } else {
        hs = hg_scan_offsets(nw, d_cnt, d_off, stream);
    }
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
    cudaFree(d_lvl);
    cudaFree(d_idx);
    cudaFree(d_child);
    cudaFree(d_leaf);
    cudaFree(d_ln);
    cudaFree(d_cnt);
    cudaFree(d_off);
    cudaFree(d_err);
    cudaFree(d_ids);
    cudaFree(d_area);
    return hs;
}

}  // namespace hg
