// Batched launch over many grids and the launch-shape autotuner.
//
// The rays of all grids form one queue, ordered so that the grids with the
// most rays come first; persistent threads take queue positions through a
// warp-aggregated atomic counter, map a position to (grid, ray) with a
// binary search over the per-grid queue offsets held in shared memory, and
// walk it with the same per-crossing loop as the single-grid kernel.  One
// launch covers the whole batch, so it can be captured in a CUDA graph.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "hg_internal.h"
#include "walk.cuh"

namespace cg = cooperative_groups;

namespace hg {
hg_status cuda_err(cudaError_t e, const char *what);
int sm_count();

constexpr int kMaxBatch = 1024;

struct BatchEntry {
    DevGrid G;
    int64_t ray0;
    int64_t max_steps;
};

struct BatchArgs {
    const BatchEntry *E;
    const int64_t *qbeg;  // [n_grids+1] queue offsets in processing order
    const int32_t *perm;  // [n_grids] grid at each queue slot
    int n_grids;
    int64_t total;
    const double *o;
    const double *d;
    const double *smax;
    double kappa;
    void *tau;
    int32_t *ncross;
    uint8_t *status;
    int64_t max_steps;  // 0: per grid 4 n_leaves + 64
    unsigned long long *counter;
    RayStart *starts;   // [total] start records, indexed by ray
};

// Queue position -> slot (grid in processing order) by binary search.
__device__ __forceinline__ int queue_slot(const int64_t *s_qbeg, int n_grids, int64_t q) {
    int lo = 0, hi = n_grids - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_qbeg[mid] <= q)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Setup pass over the whole batch (checks, 1/d, clip, first leaf).
__global__ void __launch_bounds__(256) batch_setup_kernel(const BatchArgs A) {
    __shared__ int64_t s_qbeg[kMaxBatch + 1];
    __shared__ int32_t s_perm[kMaxBatch];
    for (int i = threadIdx.x; i <= A.n_grids; i += blockDim.x) s_qbeg[i] = A.qbeg[i];
    for (int i = threadIdx.x; i < A.n_grids; i += blockDim.x) s_perm[i] = A.perm[i];
    __syncthreads();
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < A.total; q += (int64_t)gridDim.x * blockDim.x) {
        const int slot = queue_slot(s_qbeg, A.n_grids, q);
        const BatchEntry *E = A.E + s_perm[slot];
        const int64_t ray = E->ray0 + (q - s_qbeg[slot]);
        A.starts[ray] = ray_setup<2>(E->G, nullptr, 0, A.o, A.d, A.smax, ray);
    }
}

// Rays of the whole batch: queue positions from a warp-aggregated atomic
// counter, mapped to (grid, ray) through the queue offsets in shared memory.
struct BatchRays {
    static constexpr bool kSegments = false;
    const BatchArgs *A;
    const int64_t *s_qbeg;
    const int32_t *s_perm;
    __device__ __forceinline__ bool next(int64_t &ray, const DevGrid *&g, int32_t &ms) {
        cg::coalesced_group grp = cg::coalesced_threads();
        unsigned long long base = 0;
        if (grp.thread_rank() == 0) base = atomicAdd(A->counter, (unsigned long long)grp.size());
        base = grp.shfl(base, 0);
        const int64_t q = (int64_t)(base + grp.thread_rank());
        if (q >= A->total) return false;
        const int slot = queue_slot(s_qbeg, A->n_grids, q);
        const BatchEntry *E = A->E + s_perm[slot];
        ray = E->ray0 + (q - s_qbeg[slot]);
        g = &E->G;
        const int64_t m = A->max_steps > 0 ? A->max_steps : E->max_steps;
        ms = (int32_t)(m < 0x7fffffff ? m : 0x7fffffff);
        return true;
    }
};

// NAV: 0 every grid holds neighbor lists, 1 every grid ropes, 2 a mix (read per grid).
template <int PREC, int NAV>
__global__ void __launch_bounds__(256) batch_kernel(const BatchArgs A) {
    __shared__ int64_t s_qbeg[kMaxBatch + 1];
    __shared__ int32_t s_perm[kMaxBatch];
    __shared__ double s_geo[9 * 256];  // the walking threads' ray geometry (blocks of at most 256)
    for (int i = threadIdx.x; i <= A.n_grids; i += blockDim.x) s_qbeg[i] = A.qbeg[i];
    for (int i = threadIdx.x; i < A.n_grids; i += blockDim.x) s_perm[i] = A.perm[i];
    __syncthreads();
    BatchRays src{&A, s_qbeg, s_perm};
    WalkIO io{};
    io.o = A.o;
    io.d = A.d;
    io.smax = A.smax;
    io.starts = A.starts;
    io.kappa = A.kappa;
    io.tau = A.tau;
    io.ncross = A.ncross;
    io.status = A.status;
    walk_loop<2, MODE_TAU, PREC, NAV>(src, io, nullptr, 0, s_geo);
}

}  // namespace hg

struct hg_batch {
    int n_grids = 0;
    int64_t total = 0;
    hg::BatchEntry *d_entries = nullptr;
    int64_t *d_qbeg = nullptr;
    int32_t *d_perm = nullptr;
    unsigned long long *d_counter = nullptr;
    int device = 0;
    int nav = 0;  // 0 all grids with neighbor lists, 1 all with ropes, 2 mixed
};

using namespace hg;

extern "C" hg_status hg_batch_create(int32_t n_grids, const hg_grid *const *grids, const int64_t *ray_begin,
                                     int32_t chunk, hg_batch **out) {
    (void)chunk;
    if (!out || !grids || !ray_begin || n_grids < 1 || n_grids > kMaxBatch) {
        set_error("hg_batch_create: need 1..%d grids, grid pointers and ray offsets", kMaxBatch);
        return HG_EINVAL;
    }
    *out = nullptr;
    if (ray_begin[0] != 0) {
        set_error("hg_batch_create: ray_begin[0] must be 0");
        return HG_EINVAL;
    }
    std::vector<BatchEntry> ent((size_t)n_grids);
    std::vector<int64_t> cnt((size_t)n_grids);
    for (int i = 0; i < n_grids; i++) {
        if (!grids[i] || ray_begin[i + 1] < ray_begin[i]) {
            set_error("hg_batch_create: bad grid %d or ray range", i);
            return HG_EINVAL;
        }
        ent[i].G = grids[i]->d;
        ent[i].G.nodes = grids[i]->d.nodes;
        ent[i].ray0 = ray_begin[i];
        ent[i].max_steps = 4 * grids[i]->d.n_leaves + 64;
        cnt[i] = ray_begin[i + 1] - ray_begin[i];
    }
    // largest ray counts first, so that the long queues start early
    std::vector<int32_t> perm((size_t)n_grids);
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) { return cnt[a] > cnt[b]; });
    std::vector<int64_t> qbeg((size_t)n_grids + 1, 0);
    for (int s = 0; s < n_grids; s++) qbeg[s + 1] = qbeg[s] + cnt[perm[s]];
    hg_batch *b = new hg_batch();
    b->n_grids = n_grids;
    int n_ropes = 0;
    for (int i = 0; i < n_grids; i++) n_ropes += grids[i]->d.nav == HG_NAV_ROPES ? 1 : 0;
    b->nav = n_ropes == 0 ? 0 : (n_ropes == n_grids ? 1 : 2);
    b->total = qbeg[n_grids];
    cudaGetDevice(&b->device);
    cudaError_t e = cudaMalloc(&b->d_entries, ent.size() * sizeof(BatchEntry));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_qbeg, qbeg.size() * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_perm, perm.size() * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemcpy(b->d_entries, ent.data(), ent.size() * sizeof(BatchEntry), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_qbeg, qbeg.data(), qbeg.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_perm, perm.data(), perm.size() * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        hg_batch_free(b);
        return cuda_err(e, "hg_batch_create");
    }
    *out = b;
    return HG_OK;
}

extern "C" void hg_batch_free(hg_batch *b) {
    if (!b) return;
    cudaFree(b->d_entries);
    cudaFree(b->d_qbeg);
    cudaFree(b->d_perm);
    cudaFree(b->d_counter);
    delete b;
}

extern "C" hg_status hg_batch_trace(hg_batch *b, const double *o, const double *d, const double *s_max,
                                    double kappa, const hg_trace_opts *opts, void *tau, int32_t *ncross,
                                    uint8_t *ray_status, hg_stream stream) {
    if (!b || (b->total > 0 && (!o || !d || !tau || !ncross))) {
        set_error("hg_batch_trace: bad arguments");
        return HG_EINVAL;
    }
    const int prec = opts ? opts->precision : HG_FP64;
    if (prec != HG_FP64 && prec != HG_FP32K) {
        set_error("hg_batch_trace: bad precision");
        return HG_EINVAL;
    }
    if (b->total == 0) return HG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    BatchArgs A{};
    A.E = b->d_entries;
    A.qbeg = b->d_qbeg;
    A.perm = b->d_perm;
    A.n_grids = b->n_grids;
    A.total = b->total;
    A.o = o;
    A.d = d;
    A.smax = s_max;
    A.kappa = kappa;
    A.tau = tau;
    A.ncross = ncross;
    A.status = ray_status;
    A.max_steps = opts ? opts->max_steps : 0;
    A.counter = b->d_counter;
    const int block = (opts && opts->block > 0) ? opts->block : 256;
    if (block < 32 || block > 256 || block % 32) {
        set_error("hg_batch_trace: block must be a multiple of 32 in 32..256");
        return HG_EINVAL;
    }
    using BatchFn = void (*)(const BatchArgs);
    static const BatchFn kernels[2][3] = {{&batch_kernel<HG_FP64, 0>, &batch_kernel<HG_FP64, 1>, &batch_kernel<HG_FP64, 2>},
                                          {&batch_kernel<HG_FP32K, 0>, &batch_kernel<HG_FP32K, 1>,
                                           &batch_kernel<HG_FP32K, 2>}};
    const BatchFn kern = kernels[prec == HG_FP64 ? 0 : 1][b->nav];
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, 0);
    if (e != cudaSuccess) return cuda_err(e, "batch occupancy");
    int64_t blocks = (int64_t)std::max(1, per_sm) * sm_count();
    blocks = std::min<int64_t>(blocks, (b->total + block - 1) / block);
    RayStart *starts = nullptr;
    e = cudaMallocAsync((void **)&starts, (size_t)b->total * sizeof(RayStart), s);
    if (e != cudaSuccess) return cuda_err(e, "batch start scratch");
    A.starts = starts;
    e = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) {
        cudaFreeAsync(starts, s);
        return cuda_err(e, "batch counter reset");
    }
    const int64_t sblocks = std::min<int64_t>((b->total + 255) / 256, (int64_t)sm_count() * 8);
    batch_setup_kernel<<<(unsigned)sblocks, 256, 0, s>>>(A);
    kern<<<(unsigned)blocks, block, 0, s>>>(A);
    note_launches(2);
    e = cudaGetLastError();
    cudaFreeAsync(starts, s);
    return e == cudaSuccess ? HG_OK : cuda_err(e, "batch launch");
}

// ------------------------------------------------------------------ autotuner

extern "C" hg_status hg_autotune(hg_grid *g, int64_t n, const double *o, const double *d, int32_t precision,
                                 hg_trace_opts *best, float *best_ms, hg_stream stream) {
    if (!g || n <= 0 || !o || !d || (precision != HG_FP64 && precision != HG_FP32K)) {
        set_error("hg_autotune: bad arguments");
        return HG_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    void *tau = nullptr;
    int32_t *nc = nullptr;
    cudaError_t e = cudaMallocAsync(&tau, (size_t)n * 8, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&nc, (size_t)n * 4, s);
    if (e != cudaSuccess) return cuda_err(e, "hg_autotune scratch");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int node_bytes = g->d.kind == HG_KDTREE ? 16 : 32;
    const int blocks[] = {128, 256};
    const int smem_kb[] = {0, 8, 32, 64};
    hg_trace_opts win{};
    float win_ms = 1e30f;
    hg_status st = HG_OK;
    for (int sched = 1; sched <= 3 && st == HG_OK; sched++)
        for (int occ = 3; occ <= 4; occ++)
            for (int bl : blocks)
                for (int kb : smem_kb) {
                    hg_trace_opts op{};
                    op.precision = precision;
                    op.block = bl;
                    op.smem_nodes = (int)std::min<int64_t>(g->d.n_nodes, (int64_t)kb * 1024 / node_bytes);
                    op.schedule = sched;
                    op.min_blocks = occ;
                    st = hg_trace_rays(g, n, o, d, nullptr, 1.0, &op, tau, nc, nullptr, stream);
                    if (st == HG_EINVAL) {  // shape does not fit: skip it
                        st = HG_OK;
                        continue;
                    }
                    if (st != HG_OK) break;
                    float best_here = 1e30f;
                    for (int rep = 0; rep < 3; rep++) {
                        cudaEventRecord(e0, s);
                        st = hg_trace_rays(g, n, o, d, nullptr, 1.0, &op, tau, nc, nullptr, stream);
                        cudaEventRecord(e1, s);
                        cudaEventSynchronize(e1);
                        float ms = 0.f;
                        cudaEventElapsedTime(&ms, e0, e1);
                        best_here = std::min(best_here, ms);
                    }
                    if (best_here < win_ms) {
                        win_ms = best_here;
                        win = op;
                    }
                }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(tau, s);
    cudaFreeAsync(nc, s);
    cudaStreamSynchronize(s);
    if (st != HG_OK) return st;
    TuneEntry &T = g->tuned[precision];
    T.valid = 1;
    T.block = win.block;
    T.smem_nodes = win.smem_nodes;
    T.schedule = win.schedule;
    T.min_blocks = win.min_blocks;
    if (best) *best = win;
    if (best_ms) *best_ms = win_ms;
    return HG_OK;
}
