// Path-calculation kernels and their C entry points: optical depth and
// crossing counts, segment emission, adjoint scatter, density sampling,
// plus the small scan / reduction kernels the path needs.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "hg_internal.h"
#include "walk.cuh"

namespace cg = cooperative_groups;

namespace hg {

struct TraceArgs {
    DevGrid G;
    int64_t n;
    const double *o;
    const double *d;
    const double *smax;
    double kappa;
    void *tau;
    int32_t *ncross;
    uint8_t *status;
    const int64_t *seg_off;
    int32_t *seg_cell;
    void *seg_ds;
    int64_t seg_cap;
    const float *w;
    void *grad;
    const double *rho_ext;  // densities replacing the grid's own (MODE_TAU), or NULL
    int64_t max_steps;
    unsigned long long *counter;
    const RayStart *starts;
    const int64_t *order;  // queue position -> ray (most work first), or NULL
    int n_smem;
    int dyn;
};

// Stage the first n nodes of the (breadth-first) node list in shared memory.
__device__ __forceinline__ void stage_nodes(const void *nodes, int bytes, unsigned char *smem) {
    const int4 *src = reinterpret_cast<const int4 *>(nodes);
    int4 *dst = reinterpret_cast<int4 *>(smem);
    for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) dst[i] = __ldg(src + i);
    __syncthreads();
}

// Setup pass: one ray per thread, every thread doing the same work (checks,
// 1/d, clip, top-down location of the first leaf), so that the walking
// kernel's refill is a handful of loads instead of a divergent descent.
//
// Crossings per path are heavy-tailed (on the disk grids the median path
// crosses 5 leaves, the longest several hundred), and a launch lasts at
// least as long as its longest path.  So with a non-NULL bucket_count the
// pass also sorts the rays into kBuckets classes of estimated work (the
// coarse-lattice estimate, or the exact count when seg_off gives it) and
// the dynamic queue hands out the heaviest paths first.
constexpr int kBuckets = 32;

__device__ __forceinline__ int work_bucket(float w) {
    const int b = (int)(__log2f(1.0f + fmaxf(w, 0.0f)) * 3.0f);
    return kBuckets - 1 - (b < 0 ? 0 : (b > kBuckets - 1 ? kBuckets - 1 : b));  // 0 = most work
}

template <int KIND>
__global__ void __launch_bounds__(256) setup_kernel(const DevGrid G, int64_t n, const double *__restrict__ o,
                                                    const double *__restrict__ d, const double *__restrict__ smax,
                                                    RayStart *starts, int n_smem, unsigned long long *bucket_count,
                                                    const int64_t *__restrict__ seg_off) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned int hist[kBuckets];
    if (threadIdx.x < kBuckets) hist[threadIdx.x] = 0;
    stage_nodes(G.nodes, n_smem * (KIND == HG_KDTREE ? 16 : 32), smem);
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        RayStart R = ray_setup<KIND>(G, smem, n_smem, o, d, smax, r, bucket_count != nullptr && !seg_off);
        if (seg_off) R.work = (float)(seg_off[r + 1] - seg_off[r]);
        starts[r] = R;
        if (bucket_count) atomicAdd(&hist[work_bucket(R.work)], 1u);
    }
    if (bucket_count) {
        __syncthreads();
        if (threadIdx.x < kBuckets && hist[threadIdx.x]) atomicAdd(&bucket_count[threadIdx.x], hist[threadIdx.x]);
    }
}

// Queue order from the bucket counts: ray r goes to the next free slot of
// its bucket (lanes of a warp with the same bucket share one atomic; the
// order inside a bucket is arbitrary and results do not depend on it).
__global__ void __launch_bounds__(256) order_kernel(int64_t n, const RayStart *__restrict__ starts,
                                                    const unsigned long long *bucket_count,
                                                    unsigned long long *bucket_fill, int64_t *order) {
    __shared__ unsigned long long base[kBuckets];
    if (threadIdx.x == 0) {
        unsigned long long acc = 0;
        for (int b = 0; b < kBuckets; b++) {
            base[b] = acc;
            acc += bucket_count[b];
        }
    }
    __syncthreads();
    const unsigned lane = threadIdx.x & 31u;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int b = work_bucket(starts[r].work);
        const unsigned mask = __match_any_sync(__activemask(), b);
        const int leader = __ffs(mask) - 1;
        const unsigned rank = __popc(mask & ((1u << lane) - 1u));
        unsigned long long slot = 0;
        if ((int)lane == leader) slot = atomicAdd(&bucket_fill[b], (unsigned long long)__popc(mask));
        slot = __shfl_sync(mask, slot, leader);
        order[base[b] + slot + rank] = r;
    }
}

// Rays of one grid for the walking loop: a static stride, or a
// warp-aggregated atomic on a global counter.
struct GridRays {
    const DevGrid *G;
    int64_t n;
    int64_t cursor;
    int64_t stride;
    unsigned long long *counter;
    const int64_t *order;
    int32_t max_steps;
    bool dyn;
    __device__ __forceinline__ bool next(int64_t &ray, const DevGrid *&g, int32_t &ms) {
        g = G;
        ms = max_steps;
        if (dyn) {
            cg::coalesced_group grp = cg::coalesced_threads();
            unsigned long long base = 0;
            if (grp.thread_rank() == 0) base = atomicAdd(counter, (unsigned long long)grp.size());
            base = grp.shfl(base, 0);
            ray = (int64_t)(base + grp.thread_rank());
            if (ray < n && order) ray = order[ray];
            return ray < n;
        }
        ray = cursor;
        cursor += stride;
        return ray < n;
    }
};

// One persistent loop per thread (walk_loop): a lane whose ray has ended
// takes the next one, and every iteration advances each lane by one record
// load, so lanes never wait for the longest path in their warp.
//   OCC: resident blocks of 256 threads per SM the register budget is cut for
//   (3: 80 registers; 4: 64 registers).
template <int KIND, int MODE, int PREC, int OCC>
__global__ void __launch_bounds__(256, OCC) trace_kernel(const TraceArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int node_bytes = (KIND == HG_KDTREE) ? 16 : 32;
    stage_nodes(A.G.nodes, A.n_smem * node_bytes, smem);
    GridRays src;
    src.G = &A.G;
    src.n = A.n;
    src.cursor = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    src.stride = (int64_t)gridDim.x * blockDim.x;
    src.counter = A.counter;
    src.order = A.order;
    src.max_steps = (int32_t)(A.max_steps < 0x7fffffff ? A.max_steps : 0x7fffffff);
    src.dyn = A.dyn != 0;
    WalkIO io;
    io.o = A.o;
    io.d = A.d;
    io.smax = A.smax;
    io.starts = A.starts;
    io.kappa = A.kappa;
    io.tau = A.tau;
    io.ncross = A.ncross;
    io.status = A.status;
    io.seg_off = A.seg_off;
    io.seg_cell = A.seg_cell;
    io.seg_ds = A.seg_ds;
    io.seg_cap = A.seg_cap;
    io.w = A.w;
    io.grad = A.grad;
    io.rho_ext = A.rho_ext;
    walk_loop<KIND, MODE, PREC>(src, io, smem, A.n_smem);
}

// ------------------------------------------------------------------ launch plumbing

typedef void (*KernelFn)(const TraceArgs);

KernelFn pick_kernel(int kind, int mode, int prec, int occ) {
#define HG_K(K, M, P) {&trace_kernel<K, M, P, 3>, &trace_kernel<K, M, P, 4>}
    static const KernelFn table[2][3][2][2] = {
        {{HG_K(0, 0, 0), HG_K(0, 0, 1)}, {HG_K(0, 1, 0), HG_K(0, 1, 1)}, {HG_K(0, 2, 0), HG_K(0, 2, 1)}},
        {{HG_K(1, 0, 0), HG_K(1, 0, 1)}, {HG_K(1, 1, 0), HG_K(1, 1, 1)}, {HG_K(1, 2, 0), HG_K(1, 2, 1)}}};
#undef HG_K
    return table[kind][mode][prec][occ == 4 ? 1 : 0];
}

hg_status cuda_err(cudaError_t e, const char *what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? HG_ENOMEM : HG_ECUDA;
}

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// Default launch shape: 256 threads, the top 2048 k-d nodes (32 KB) or
// 1024 octree nodes (32 KB) in shared memory, persistent dynamic schedule.
hg_status resolve_opts(const hg_grid *g, const hg_trace_opts *opts, int &precision, int &block, int &smem_nodes,
                       int &schedule, int &min_blocks, int64_t &max_steps) {
    precision = opts ? opts->precision : HG_FP64;
    if (precision != HG_FP64 && precision != HG_FP32K) {
        set_error("precision must be HG_FP64 or HG_FP32K");
        return HG_EINVAL;
    }
    const TuneEntry &T = g->tuned[precision];
    block = (opts && opts->block > 0) ? opts->block : (T.valid ? T.block : 256);
    smem_nodes = (opts && opts->smem_nodes >= 0) ? opts->smem_nodes
                                                  : (T.valid ? T.smem_nodes : (g->d.kind == HG_KDTREE ? 2048 : 1024));
    schedule = (opts && opts->schedule > 0) ? opts->schedule : (T.valid ? T.schedule : 0);
    min_blocks = (opts && opts->min_blocks > 0) ? opts->min_blocks : (T.valid ? T.min_blocks : 3);
    max_steps = (opts && opts->max_steps > 0) ? opts->max_steps : 4 * g->d.n_leaves + 64;
    if (block < 32 || block > 256 || block % 32) {
        set_error("block must be a multiple of 32 in 32..256");
        return HG_EINVAL;
    }
    if (min_blocks != 3 && min_blocks != 4) {
        set_error("min_blocks must be 3 or 4");
        return HG_EINVAL;
    }
    if (schedule < 0 || schedule > 3) {
        set_error("schedule must be 0 (auto), 1, 2 or 3");
        return HG_EINVAL;
    }
    // clamp to the node count and to 200 KB of shared memory
    const int node_bytes = g->d.kind == HG_KDTREE ? 16 : 32;
    smem_nodes = (int)std::min<int64_t>(std::min<int64_t>(smem_nodes, g->d.n_nodes), (200 * 1024) / node_bytes);
    return HG_OK;
}

hg_status launch_trace(const hg_grid *g, int mode, int prec, TraceArgs A, int block, int smem_nodes, int schedule,
                       int min_blocks, cudaStream_t stream) {
    if (A.n == 0) return HG_OK;
    KernelFn k = pick_kernel(g->d.kind, mode, prec, min_blocks);
    const int node_bytes = g->d.kind == HG_KDTREE ? 16 : 32;
    const size_t smem = (size_t)smem_nodes * node_bytes;
    static std::once_flag once;
    std::call_once(once, [] {
        for (int kd = 0; kd < 2; kd++)
            for (int m = 0; m < 3; m++)
                for (int p = 0; p < 2; p++)
                    for (int oc = 3; oc <= 4; oc++)
                        cudaFuncSetAttribute(pick_kernel(kd, m, p, oc), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             200 * 1024);
        cudaFuncSetAttribute(setup_kernel<HG_KDTREE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(setup_kernel<HG_OCTREE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    });
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem);
    if (e != cudaSuccess) return cuda_err(e, "occupancy query");
    if (per_sm < 1) {
        set_error("launch shape does not fit on an SM (block %d, %zu B shared)", block, smem);
        return HG_EINVAL;
    }
    int64_t blocks = (int64_t)per_sm * sm_count();
    const int64_t need = (A.n + block - 1) / block;
    if (blocks > need) blocks = need;
    // auto schedule: order by estimated work only when each resident thread
    // gets few paths (then the heaviest paths would otherwise set the end)
    if (schedule == 0) schedule = (A.n < 48 * blocks * block) ? 3 : 2;
    A.n_smem = smem_nodes;
    A.dyn = (schedule >= 2);
    const bool ordered = (schedule == 3);
    // setup pass into a scratch array of start records
    // scratch: start records, and for the dynamic schedule the work-ordered
    // queue with its bucket counters
    const size_t start_bytes = ((size_t)A.n * sizeof(RayStart) + 255) / 256 * 256;
    const size_t order_bytes = ordered ? ((size_t)A.n * sizeof(int64_t) + 255) / 256 * 256 : 0;
    const size_t count_bytes = ordered ? 2 * kBuckets * sizeof(unsigned long long) : 0;
    unsigned char *scratch = nullptr;
    e = cudaMallocAsync((void **)&scratch, start_bytes + order_bytes + count_bytes, stream);
    if (e != cudaSuccess) return cuda_err(e, "ray start scratch");
    RayStart *starts = reinterpret_cast<RayStart *>(scratch);
    int64_t *order = ordered ? reinterpret_cast<int64_t *>(scratch + start_bytes) : nullptr;
    unsigned long long *counts =
        ordered ? reinterpret_cast<unsigned long long *>(scratch + start_bytes + order_bytes) : nullptr;
    if (counts) {
        e = cudaMemsetAsync(counts, 0, count_bytes, stream);
        if (e != cudaSuccess) {
            cudaFreeAsync(scratch, stream);
            return cuda_err(e, "scratch reset");
        }
    }
    {
        // the fill pass knows each ray's exact crossing count from its offsets
        const int64_t *exact = (mode == MODE_FILL) ? A.seg_off : nullptr;
        const int64_t sblocks = std::min<int64_t>((A.n + 255) / 256, (int64_t)sm_count() * 8);
        if (g->d.kind == HG_KDTREE)
            setup_kernel<HG_KDTREE><<<(unsigned)sblocks, 256, smem, stream>>>(g->d, A.n, A.o, A.d, A.smax, starts,
                                                                             smem_nodes, counts, exact);
        else
            setup_kernel<HG_OCTREE><<<(unsigned)sblocks, 256, smem, stream>>>(g->d, A.n, A.o, A.d, A.smax, starts,
                                                                             smem_nodes, counts, exact);
        note_launches(1);
        if (order) {
            order_kernel<<<(unsigned)sblocks, 256, 0, stream>>>(A.n, starts, counts, counts + kBuckets, order);
            note_launches(1);
        }
    }
    A.starts = starts;
    A.order = order;
    unsigned long long *ctr = nullptr;
    if (A.dyn) {
        e = cudaMallocAsync((void **)&ctr, sizeof(unsigned long long), stream);
        if (e != cudaSuccess) {
            cudaFreeAsync(scratch, stream);
            return cuda_err(e, "scratch counter");
        }
        e = cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), stream);
        if (e != cudaSuccess) {
            cudaFreeAsync(ctr, stream);
            cudaFreeAsync(scratch, stream);
            return cuda_err(e, "scratch counter");
        }
        A.counter = ctr;
    }
    k<<<(unsigned)blocks, block, smem, stream>>>(A);
    e = cudaGetLastError();
    note_launches(1);
    if (ctr) cudaFreeAsync(ctr, stream);
    cudaFreeAsync(scratch, stream);
    if (e != cudaSuccess) return cuda_err(e, "trace launch");
    return HG_OK;
}

hg_status check_rays(const hg_grid *g, int64_t n, const double *o, const double *d) {
    if (!g) {
        set_error("null grid");
        return HG_EINVAL;
    }
    if (n < 0 || (n > 0 && (!o || !d))) {
        set_error("bad ray arrays");
        return HG_EINVAL;
    }
    return HG_OK;
}

// ------------------------------------------------------------------ density sampling

template <int KIND>
__global__ void sample_kernel(const DevGrid G, int64_t n, const double *__restrict__ pts, int32_t *cell,
                              double *rho, int n_smem) {
    extern __shared__ __align__(16) unsigned char smem[];
    stage_nodes(G.nodes, n_smem * (KIND == HG_KDTREE ? 16 : 32), smem);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const long long p0 = okey(pts[3 * i]), p1 = okey(pts[3 * i + 1]), p2 = okey(pts[3 * i + 2]);
        int32_t c = -1;
        // a point query uses the half-open rule of a zero direction
        if (in_axis(p0, G.klo[0], G.khi[0], false, false, true) && in_axis(p1, G.klo[1], G.khi[1], false, false, true) &&
            in_axis(p2, G.klo[2], G.khi[2], false, false, true))
            c = descend<KIND>(G, smem, n_smem, p0, p1, p2, 0u);
        if (cell) cell[i] = c;
        rho[i] = (c >= 0) ? __ldg(&G.rec[c].rho) : 0.0;
    }
}

// ------------------------------------------------------------------ scan and reductions

constexpr int kScanBlock = 1024;
constexpr int kScanItems = 8;  // per thread: one block covers 8192 counts

__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t *sh, int64_t *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t s = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    const int64_t warp_prefix = wid ? sh[wid - 1] : 0;
    *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_prefix + x - v;
}

// Pass 1: sum of each tile of kScanBlock*kScanItems counts.
__global__ void scan_tile_sums(int64_t n, const int32_t *__restrict__ c, int64_t *tile_sum) {
    __shared__ int64_t sh[32];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock * kScanItems;
    int64_t s = 0;
    for (int j = 0; j < kScanItems; j++) {
        const int64_t i = base + (int64_t)j * kScanBlock + threadIdx.x;
        if (i < n) s += c[i];
    }
    int64_t tot;
    block_excl_scan(s, sh, &tot);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

// Pass 2: exclusive scan of the tile sums by one block (serial over chunks).
__global__ void scan_tile_prefix(int64_t tiles, int64_t *tile_sum) {
    __shared__ int64_t sh[32];
    int64_t carry = 0;
    for (int64_t b = 0; b < tiles; b += blockDim.x) {
        const int64_t i = b + threadIdx.x;
        const int64_t v = i < tiles ? tile_sum[i] : 0;
        int64_t tot;
        const int64_t ex = block_excl_scan(v, sh, &tot);
        if (i < tiles) tile_sum[i] = carry + ex;
        carry += tot;
    }
}

// Pass 3: scan inside each tile, offset by the tile's prefix.
__global__ void scan_tile_apply(int64_t n, const int32_t *__restrict__ c, const int64_t *tile_prefix,
                                int64_t *out) {
    __shared__ int64_t sh[32];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock * kScanItems + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        const int64_t i = base + j;
        v[j] = (i < n) ? c[i] : 0;
        s += v[j];
    }
    int64_t tot;
    int64_t run = tile_prefix[blockIdx.x] + block_excl_scan(s, sh, &tot);
#pragma unroll
    for (int j = 0; j < kScanItems; j++) {
        const int64_t i = base + j;
        if (i < n) out[i] = run;
        run += v[j];
    }
    if (base < n && n <= base + kScanItems) out[n] = run;
}

__global__ void or_status_kernel(int64_t n, const uint8_t *__restrict__ s, uint32_t *out) {
    uint32_t v = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v |= s[i];
    v = __reduce_or_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0 && v) atomicOr(out, v);
}

__global__ void sum_i32_kernel(int64_t n, const int32_t *__restrict__ x, unsigned long long *out) {
    long long v = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v += x[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, (unsigned long long)v);
}

}  // namespace hg

using namespace hg;

extern "C" hg_status hg_trace_rays(const hg_grid *g, int64_t n, const double *o, const double *d,
                                   const double *s_max, double kappa, const hg_trace_opts *opts, void *tau,
                                   int32_t *ncross, uint8_t *ray_status, hg_stream stream) {
    hg_status st = check_rays(g, n, o, d);
    if (st != HG_OK) return st;
    if (n > 0 && (!tau || !ncross)) {
        set_error("hg_trace_rays: tau and ncross are required");
        return HG_EINVAL;
    }
    int prec, block, smem_nodes, schedule, min_blocks;
    int64_t max_steps;
    if ((st = resolve_opts(g, opts, prec, block, smem_nodes, schedule, min_blocks, max_steps)) != HG_OK) return st;
    TraceArgs A{};
    A.G = g->d;
    A.n = n;
    A.o = o;
    A.d = d;
    A.smax = s_max;
    A.kappa = kappa;
    A.tau = tau;
    A.ncross = ncross;
    A.status = ray_status;
    A.max_steps = max_steps;
    return launch_trace(g, MODE_TAU, prec, A, block, smem_nodes, schedule, min_blocks, (cudaStream_t)stream);
}

extern "C" hg_status hg_trace_rays_rho(const hg_grid *g, int64_t n, const double *o, const double *d,
                                       const double *s_max, double kappa, const double *rho,
                                       const hg_trace_opts *opts, void *tau, int32_t *ncross, uint8_t *ray_status,
                                       hg_stream stream) {
    hg_status st = check_rays(g, n, o, d);
    if (st != HG_OK) return st;
    if (n > 0 && (!tau || !ncross || !rho)) {
        set_error("hg_trace_rays_rho: rho, tau and ncross are required");
        return HG_EINVAL;
    }
    int prec, block, smem_nodes, schedule, min_blocks;
    int64_t max_steps;
    if ((st = resolve_opts(g, opts, prec, block, smem_nodes, schedule, min_blocks, max_steps)) != HG_OK) return st;
    TraceArgs A{};
    A.G = g->d;
    A.n = n;
    A.o = o;
    A.d = d;
    A.smax = s_max;
    A.kappa = kappa;
    A.rho_ext = rho;
    A.tau = tau;
    A.ncross = ncross;
    A.status = ray_status;
    A.max_steps = max_steps;
    return launch_trace(g, MODE_TAU, prec, A, block, smem_nodes, schedule, min_blocks, (cudaStream_t)stream);
}

extern "C" hg_status hg_trace_fill(const hg_grid *g, int64_t n, const double *o, const double *d,
                                   const double *s_max, const hg_trace_opts *opts, const int64_t *seg_off,
                                   int32_t *seg_cell, void *seg_ds, int64_t seg_capacity, uint8_t *ray_status,
                                   hg_stream stream) {
    hg_status st = check_rays(g, n, o, d);
    if (st != HG_OK) return st;
    if (n > 0 && (!seg_off || (seg_capacity > 0 && (!seg_cell || !seg_ds)) || seg_capacity < 0)) {
        set_error("hg_trace_fill: bad segment arrays");
        return HG_EINVAL;
    }
    int prec, block, smem_nodes, schedule, min_blocks;
    int64_t max_steps;
    if ((st = resolve_opts(g, opts, prec, block, smem_nodes, schedule, min_blocks, max_steps)) != HG_OK) return st;
    TraceArgs A{};
    A.G = g->d;
    A.n = n;
    A.o = o;
    A.d = d;
    A.smax = s_max;
    A.seg_off = seg_off;
    A.seg_cell = seg_cell;
    A.seg_ds = seg_ds;
    A.seg_cap = seg_capacity;
    A.status = ray_status;
    A.max_steps = max_steps;
    return launch_trace(g, MODE_FILL, prec, A, block, smem_nodes, schedule, min_blocks, (cudaStream_t)stream);
}

extern "C" hg_status hg_tau_gradient(const hg_grid *g, int64_t n, const double *o, const double *d,
                                     const double *s_max, double kappa, const float *w, int32_t grad_precision,
                                     void *grad_rho, const hg_trace_opts *opts, hg_stream stream) {
    hg_status st = check_rays(g, n, o, d);
    if (st != HG_OK) return st;
    if (n > 0 && (!w || !grad_rho)) {
        set_error("hg_tau_gradient: w and grad_rho are required");
        return HG_EINVAL;
    }
    if (grad_precision != 0 && grad_precision != 1) {
        set_error("hg_tau_gradient: grad_precision must be 0 (f64) or 1 (f32)");
        return HG_EINVAL;
    }
    int prec, block, smem_nodes, schedule, min_blocks;
    int64_t max_steps;
    if ((st = resolve_opts(g, opts, prec, block, smem_nodes, schedule, min_blocks, max_steps)) != HG_OK) return st;
    TraceArgs A{};
    A.G = g->d;
    A.n = n;
    A.o = o;
    A.d = d;
    A.smax = s_max;
    A.kappa = kappa;
    A.w = w;
    A.grad = grad_rho;
    A.max_steps = max_steps;
    return launch_trace(g, MODE_ADJ, grad_precision, A, block, smem_nodes, schedule, min_blocks, (cudaStream_t)stream);
}

extern "C" hg_status hg_sample_density(const hg_grid *g, int64_t n, const double *pts, int32_t *cell, double *rho,
                                       hg_stream stream) {
    if (!g || n < 0 || (n > 0 && (!pts || !rho))) {
        set_error("hg_sample_density: bad arguments");
        return HG_EINVAL;
    }
    if (n == 0) return HG_OK;
    const int node_bytes = g->d.kind == HG_KDTREE ? 16 : 32;
    const int n_smem = (int)std::min<int64_t>(g->d.n_nodes, (32 * 1024) / node_bytes);
    const size_t smem = (size_t)n_smem * node_bytes;
    const int block = 256;
    int64_t blocks = std::min<int64_t>((n + block - 1) / block, (int64_t)sm_count() * 8);
    if (g->d.kind == HG_KDTREE)
        sample_kernel<HG_KDTREE><<<(unsigned)blocks, block, smem, (cudaStream_t)stream>>>(g->d, n, pts, cell, rho,
                                                                                         n_smem);
    else
        sample_kernel<HG_OCTREE><<<(unsigned)blocks, block, smem, (cudaStream_t)stream>>>(g->d, n, pts, cell, rho,
                                                                                         n_smem);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HG_OK : cuda_err(e, "sample launch");
}

extern "C" hg_status hg_scan_offsets(int64_t n, const int32_t *count, int64_t *seg_off, hg_stream stream) {
    if (n < 0 || !seg_off || (n > 0 && !count)) {
        set_error("hg_scan_offsets: bad arguments");
        return HG_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        cudaError_t e = cudaMemsetAsync(seg_off, 0, sizeof(int64_t), s);
        return e == cudaSuccess ? HG_OK : cuda_err(e, "scan");
    }
    const int64_t tile = (int64_t)kScanBlock * kScanItems;
    const int64_t tiles = (n + tile - 1) / tile;
    int64_t *sums = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&sums, (size_t)tiles * sizeof(int64_t), s);
    if (e != cudaSuccess) return cuda_err(e, "scan scratch");
    scan_tile_sums<<<(unsigned)tiles, kScanBlock, 0, s>>>(n, count, sums);
    scan_tile_prefix<<<1, kScanBlock, 0, s>>>(tiles, sums);
    scan_tile_apply<<<(unsigned)tiles, kScanBlock, 0, s>>>(n, count, sums, seg_off);
    note_launches(3);
    e = cudaGetLastError();
    cudaFreeAsync(sums, s);
    return e == cudaSuccess ? HG_OK : cuda_err(e, "scan launch");
}

extern "C" hg_status hg_reduce_status(int64_t n, const uint8_t *ray_status, uint32_t *out_bits, hg_stream stream) {
    if (n < 0 || !out_bits || (n > 0 && !ray_status)) {
        set_error("hg_reduce_status: bad arguments");
        return HG_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(out_bits, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess && n > 0) {
        int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 4);
        or_status_kernel<<<(unsigned)blocks, 256, 0, s>>>(n, ray_status, out_bits);
        note_launches(1);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? HG_OK : cuda_err(e, "status reduce");
}

extern "C" hg_status hg_sum_i32(int64_t n, const int32_t *x, int64_t *out, hg_stream stream) {
    if (n < 0 || !out || (n > 0 && !x)) {
        set_error("hg_sum_i32: bad arguments");
        return HG_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int64_t), s);
    if (e == cudaSuccess && n > 0) {
        int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 4);
        sum_i32_kernel<<<(unsigned)blocks, 256, 0, s>>>(n, x, reinterpret_cast<unsigned long long *>(out));
        note_launches(1);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? HG_OK : cuda_err(e, "sum");
}

namespace hg {

// Launch the FP64 / FP32K optical-depth pass with scratch the caller
// provides (start records for n rays and a work counter) instead of the
// stream-ordered allocator.  Used by the allocation-free entry point.
hg_status trace_rays_prealloc(const hg_grid *g, int64_t n, const double *o, const double *d, const double *s_max,
                              double kappa, const hg_trace_opts *opts, void *tau, int32_t *ncross,
                              uint8_t *ray_status, RayStart *starts, unsigned long long *counter,
                              cudaStream_t stream) {
    hg_status st = check_rays(g, n, o, d);
    if (st != HG_OK) return st;
    if (n > 0 && (!tau || !ncross)) {
        set_error("tau and ncross are required");
        return HG_EINVAL;
    }
    int prec, block, smem_nodes, schedule, min_blocks;
    int64_t max_steps;
    if ((st = resolve_opts(g, opts, prec, block, smem_nodes, schedule, min_blocks, max_steps)) != HG_OK) return st;
    if (n == 0) return HG_OK;
    TraceArgs A{};
    A.G = g->d;
    A.n = n;
    A.o = o;
    A.d = d;
    A.smax = s_max;
    A.kappa = kappa;
    A.tau = tau;
    A.ncross = ncross;
    A.status = ray_status;
    A.max_steps = max_steps;
    A.n_smem = smem_nodes;
    A.dyn = (schedule == 2);
    A.starts = starts;
    A.counter = counter;
    KernelFn k = pick_kernel(g->d.kind, MODE_TAU, prec, min_blocks);
    const int node_bytes = g->d.kind == HG_KDTREE ? 16 : 32;
    const size_t smem = (size_t)smem_nodes * node_bytes;
    if (smem > 48 * 1024) {
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(setup_kernel<HG_KDTREE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(setup_kernel<HG_OCTREE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem);
    if (e != cudaSuccess) return cuda_err(e, "occupancy query");
    if (per_sm < 1) {
        set_error("launch shape does not fit on an SM (block %d, %zu B shared)", block, smem);
        return HG_EINVAL;
    }
    int64_t blocks = std::min<int64_t>((int64_t)per_sm * sm_count(), (n + block - 1) / block);
    if (A.dyn) {
        e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), stream);
        if (e != cudaSuccess) return cuda_err(e, "counter reset");
    }
    const int64_t sblocks = std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 8);
    if (g->d.kind == HG_KDTREE)
        setup_kernel<HG_KDTREE><<<(unsigned)sblocks, 256, smem, stream>>>(g->d, n, o, d, s_max, starts, smem_nodes,
                                                                         nullptr, nullptr);
    else
        setup_kernel<HG_OCTREE><<<(unsigned)sblocks, 256, smem, stream>>>(g->d, n, o, d, s_max, starts, smem_nodes,
                                                                         nullptr, nullptr);
    k<<<(unsigned)blocks, block, smem, stream>>>(A);
    note_launches(2);
    e = cudaGetLastError();
    return e == cudaSuccess ? HG_OK : cuda_err(e, "trace launch");
}

}  // namespace hg
