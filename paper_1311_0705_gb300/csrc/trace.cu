// Path-calculation kernels and their C entry points: optical depth and
// crossing counts, segment emission, adjoint scatter, density sampling,
// plus the small scan / reduction kernels the path needs.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <new>

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
    uint32_t gmul, gmask;   // gradient slot of leaf c: (c * gmul) & gmask; gmul 0: slot c
    const double *rho_ext;  // densities replacing the grid's own (MODE_TAU), or NULL
    int64_t max_steps;
    unsigned long long *counter;
    const RayStart *starts;
    const int64_t *order;  // queue position -> ray (most work first), or NULL
    int n_smem;
    int dyn;
    // path segments of split rays (queue positions before the rays), or NULL
    const unsigned long long *n_seg;
    int64_t n_seg_cap;
    const SegStart *segs;
    double *part_acc;
    int32_t *part_nc;
    int32_t *part_last;
    uint8_t *part_st;
    const int64_t *seg_base;  // emission offset of each path segment (fill walks)
    // emission staging (MODE_*_STAGE)
    void *stg_ent;
    uint32_t *stg_next;
    uint32_t stg_nchunks;
    unsigned long long *stg_ctr;
    uint32_t *stg_start_ray;
    uint32_t *stg_start_seg;
    uint32_t *stg_overflow;
    const uint32_t *run_if;  // when non-NULL, the walk runs only if *run_if != 0
    // interaction points (MODE_INTERACT)
    const double *tau_int;
    int32_t *int_cell;
    double *int_t;
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

// With a non-NULL work_total the pass also adds up the rays' estimated work
// (each rounded up to an integer, so the total does not depend on the order
// of the additions); the split planner sizes path segments from it.
template <int KIND>
__global__ void __launch_bounds__(256) setup_kernel(const DevGrid G, int64_t n, const double *__restrict__ o,
                                                    const double *__restrict__ d, const double *__restrict__ smax,
                                                    RayStart *starts, int n_smem, unsigned long long *bucket_count,
                                                    const int64_t *__restrict__ seg_off,
                                                    unsigned long long *work_total, float *work) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned int hist[kBuckets];
    if (threadIdx.x < kBuckets) hist[threadIdx.x] = 0;
    const int node_bytes = n_smem * (KIND == HG_KDTREE ? 16 : 32);
    // the work lattice follows the staged nodes when the pass estimates work
    const bool estimate = bucket_count != nullptr && !seg_off;
    float *lat = (estimate && G.work) ? reinterpret_cast<float *>(smem + node_bytes) : nullptr;
    if (lat) stage_lattice(G, lat);
    stage_nodes(G.nodes, node_bytes, smem);
    unsigned long long wsum = 0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        RayStart R = ray_setup<KIND>(G, smem, n_smem, o, d, smax, r, estimate, lat);
        if (seg_off) R.work = (float)(seg_off[r + 1] - seg_off[r]);
        starts[r] = R;
        if (work) work[r] = R.work;
        if (bucket_count) atomicAdd(&hist[work_bucket(R.work)], 1u);
        wsum += (unsigned long long)ceilf(fmaxf(R.work, 0.0f));
    }
    if (work_total) {
        for (int off = 16; off > 0; off >>= 1) wsum += __shfl_down_sync(0xffffffffu, wsum, off);
        if ((threadIdx.x & 31) == 0 && wsum) atomicAdd(work_total, wsum);
    }
    if (bucket_count) {
        __syncthreads();
        if (threadIdx.x < kBuckets && hist[threadIdx.x]) atomicAdd(&bucket_count[threadIdx.x], hist[threadIdx.x]);
    }
}

// ------------------------------------------------------------------ path segments
//
// A launch lasts at least as long as its longest path, walked leaf after
// leaf by one thread.  With few rays per resident thread the planner cuts
// each long path into segments of about W estimated crossings that
// separate threads walk, so the cell sequence stays that of the whole
// path:
//   * a cut is a time t_c at which the point o + d t_c lies deep inside a
//     leaf L: at least 2^-18 times the problem's scale from every face of L
//     (the planner works in single precision, whose rounding is ~2^-22 of
//     that scale, and the walk's double-precision rounding ~2^-50);
//   * the walk of the whole path is then certainly in L at t_c: it entered
//     L before t_c and leaves it at t_out(L) > t_c, the smallest of L's
//     wall times in the contract's arithmetic;
//   * the segment before the cut stops after the leaf whose exit time
//     passes t_c -- that is L, and it records L's segment with the entry
//     time of the whole path's walk;
//   * the segment after the cut starts in L at time t_c, does not record L,
//     and leaves it at t_out(L) > t_c (so the exit time is not raised to the
//     entry time): the same exit wall, exit point and next leaf as the whole
//     path's walk, which it follows from there on.
// The combine pass checks that each segment stopped in the leaf the next one
// starts in (HG_RAY_LOST otherwise) and adds the partial results in path
// order.  tau differs from the left-to-right sum of the whole path only by
// the grouping of the additions.

constexpr int kMaxSegs = 16;

struct SplitRec {
    int64_t ray;
    int32_t first;  // its segments are first .. first+count-1, in path order
    int32_t count;
};

// Plan the segments of the rays whose estimated work w exceeds
// max(64, A), A = total / T the mean work per thread of the walking launch
// (only those can outlast the launch's bulk when the heaviest go first),
// into K = min(16, ceil(w / W)) pieces of equal estimated work,
// W = max(32, A / 2).  Forced: every ray of more than 3 estimated crossings,
// W = 2.  One warp per ray, over the heavy end of the work-ordered queue:
// the lanes sample the work lattice at 32 points of the path and sum them
// (a warp prefix sum), lane j places cut j where the sum reaches (j + 1) / K
// of the total (descent and depth test), and the accepted cuts are those of
// increasing t_c in distinct leaves, in path order.  Segment slots are
// taken with one atomic per ray; their count is bounded (sum over split
// rays of ceil(w/W) <= total/W + total/max(64, A) <= 3 T, or 16 n when
// forced), so seg_cap is never reached -- if it were, the ray would stay
// whole and the slots taken would be marked empty.
constexpr int kPlanWarps = 8;  // warps per 256-thread block

template <int KIND>
__global__ void __launch_bounds__(256) split_kernel(const DevGrid G, int64_t n, const double *__restrict__ o,
                                                    const double *__restrict__ d, const double *__restrict__ smax,
                                                    RayStart *starts, int n_smem, const unsigned long long *work_total,
                                                    const unsigned long long *bucket_count,
                                                    const int64_t *__restrict__ order, int64_t threads, int force,
                                                    SegStart *segs, int64_t seg_cap, unsigned long long *seg_count,
                                                    SplitRec *list, unsigned long long *split_count) {
    __shared__ int32_t s_leaf[kPlanWarps][kMaxSegs];
    __shared__ long long s_key[kPlanWarps][kMaxSegs];
    __shared__ long long s_ncand;
    __shared__ __align__(16) float lat[kWorkN * kWorkN * kWorkN];
    if (!G.work || G.work_n <= 0) return;
    stage_lattice(G, lat);
    const float A = (float)*work_total / (float)threads;
    const float W = force ? 2.0f : fmaxf(32.0f, 0.5f * A);
    const float thr = force ? 3.0f : fmaxf(64.0f, A);
    if (threadIdx.x == 0) {
        // the queue is sorted by work bucket: candidates are the buckets up to that of the threshold
        const int bt = work_bucket(thr);
        long long c = 0;
        for (int b = 0; b <= bt; b++) c += (long long)bucket_count[b];
        s_ncand = c;
    }
    __syncthreads();
    const long long ncand = s_ncand;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    float dom = 0.0f;
#pragma unroll
    for (int a = 0; a < 3; a++) dom = fmaxf(dom, fmaxf(fabsf((float)G.dlo[a]), fabsf((float)G.dhi[a])));
    for (int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib; q < ncand; q += nwarps) {
        const int64_t r = order[q];
        const RayStart R = starts[r];
        if (R.cur < 0 || !(R.work > thr)) continue;  // uniform over the warp
        const int K = (int)fminf((float)kMaxSegs, ceilf(R.work / W));
        const float of[3] = {(float)o[3 * r], (float)o[3 * r + 1], (float)o[3 * r + 2]};
        const float kf[3] = {(float)d[3 * r], (float)d[3 * r + 1], (float)d[3 * r + 2]};
        const uint32_t sg = R.sg & 0x3fu;
        // the walked interval as the setup's march took it: entry time to the domain exit or s_max
        const float ts = (float)kdouble(R.ktstart);
        const float tend = R.t1;
        // cuts stay clear of both ends of the path
        const float lo_t = ts + (tend - ts) * 0x1p-10f, hi_t = tend - (tend - ts) * 0x1p-10f;
        // cut time of this lane: where the estimated work reaches (lane + 1) / K of the total.  The
        // estimate comes from 32 samples of the work lattice, lane i at the middle of the i-th of 32
        // equal pieces of the walked interval; a warp prefix sum gives the work up to each piece's
        // end, and a search over it the piece where the target falls (linear inside the piece).
        // Coarser than a cell-by-cell march, which cost each warp ~1000 instructions per long path;
        // the cuts only balance work.
        const float dt = (tend - ts) * (1.0f / 32.0f);
        float rate = 0.0f;
        {
            const int N = G.work_n;
            const float tm = ts + ((float)lane + 0.5f) * dt;
            int ci[3];
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const float lo = (float)G.dlo[a];
                const float p = (of[a] + kf[a] * tm - lo) * ((float)N / ((float)G.dhi[a] - lo));
                const int c = (int)floorf(p);
                ci[a] = c < 0 ? 0 : (c > N - 1 ? N - 1 : c);
            }
            rate = lat[ci[0] + N * (ci[1] + N * ci[2])];
        }
        float e = rate * dt;  // inclusive prefix sum over the pieces
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const float v = __shfl_up_sync(0xffffffffu, e, off);
            if (lane >= off) e += v;
        }
        const float E = __shfl_sync(0xffffffffu, e, 31);
        const float target = E * (float)(lane + 1) / (float)K;
        int pos = 0;  // first piece whose prefix reaches the target
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
            const float v = __shfl_sync(0xffffffffu, e, pos + step - 1);
            if (v < target) pos += step;
        }
        const float e_before = __shfl_sync(0xffffffffu, e, pos > 0 ? pos - 1 : 0);
        const float r_pos = __shfl_sync(0xffffffffu, rate, pos);
        const bool found = E > 0.0f && r_pos > 0.0f;
        const float tc = found ? ts + (float)pos * dt + (target - (pos > 0 ? e_before : 0.0f)) / r_pos : 0.0f;
        // the leaf containing o + d t_c, and whether the point lies deep inside it
        bool ok = false;
        int32_t Lid = -1;
        if (lane < K - 1 && found && tc > lo_t && tc < hi_t) {
            long long q3[3], qm[3], qp[3];
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const float x = of[a] + kf[a] * tc;
                const float m = (fabsf(of[a]) + fabsf(kf[a] * tc) + dom) * 0x1p-18f;
                q3[a] = f32_key(x);
                qm[a] = f32_key(x - m);
                qp[a] = f32_key(x + m);
            }
            if (in_axis(q3[0], G.klo[0], G.khi[0], dpos(sg, 0), dneg(sg, 0), true) &&
                in_axis(q3[1], G.klo[1], G.khi[1], dpos(sg, 1), dneg(sg, 1), true) &&
                in_axis(q3[2], G.klo[2], G.khi[2], dpos(sg, 2), dneg(sg, 2), true))
                Lid = descend<KIND>(G, nullptr, 0, q3[0], q3[1], q3[2], sg);
            if (Lid >= 0) {
                Leaf L;
                load_leaf(G.rec, Lid, L);
                ok = true;
#pragma unroll
                for (int a = 0; a < 3; a++) ok = ok && qm[a] >= L.lo(a) && qp[a] <= L.hi(a);
            }
        }
        // accept cuts in path order: increasing t_c, a leaf different from the previous cut's
        int ncut = 0;
        float tprev = ts;
        int32_t prev_leaf = R.cur;
        for (int j = 0; j < K - 1; j++) {
            const bool okj = __shfl_sync(0xffffffffu, ok, j);
            const float tj = __shfl_sync(0xffffffffu, tc, j);
            const int32_t Lj = __shfl_sync(0xffffffffu, Lid, j);
            if (okj && tj > tprev && Lj != prev_leaf) {
                if (lane == j) {
                    s_leaf[wib][ncut] = Lid;
                    s_key[wib][ncut] = f32_key(tc);
                }
                ncut++;
                tprev = tj;
                prev_leaf = Lj;
            }
        }
        __syncwarp();
        if (ncut == 0) continue;
        const int nseg = ncut + 1;
        unsigned long long first = 0;
        if (lane == 0) first = atomicAdd(seg_count, (unsigned long long)nseg);
        first = __shfl_sync(0xffffffffu, first, 0);
        if (first + (unsigned long long)nseg > (unsigned long long)seg_cap) {
            for (unsigned long long s = first + lane; s < (unsigned long long)seg_cap; s += 32) {
                SegStart E;
                E.ktstart = 0;
                E.ktstop = KEY_INF;
                E.ray = r;
                E.cur = -1;
                E.sg = 0;
                segs[s] = E;
            }
            continue;
        }
        if (lane < nseg) {
            SegStart E;
            E.ktstart = lane == 0 ? R.ktstart : s_key[wib][lane - 1];
            E.ktstop = lane < ncut ? s_key[wib][lane] : KEY_INF;
            E.ray = r;
            E.cur = lane == 0 ? R.cur : s_leaf[wib][lane - 1];
            E.sg = sg | (lane == 0 ? 0u : SG_SKIP_FIRST);
            segs[first + lane] = E;
        }
        if (lane == 0) {
            const unsigned long long i = atomicAdd(split_count, 1ULL);
            SplitRec rec;
            rec.ray = r;
            rec.first = (int32_t)first;
            rec.count = nseg;
            list[i] = rec;
            starts[r].sg = R.sg | SG_SPLIT;
        }
        __syncwarp();
    }
}

// Where each path segment writes its emitted cells: after the crossings of
// the ray's earlier segments (their counts from an optical-depth walk over
// the same plan).
__global__ void __launch_bounds__(256) seg_base_kernel(const SplitRec *__restrict__ list,
                                                       const unsigned long long *split_count,
                                                       const int64_t *__restrict__ seg_off,
                                                       const int32_t *__restrict__ part_nc, int64_t *seg_base) {
    const int64_t m = (int64_t)*split_count;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const SplitRec rec = list[i];
        int64_t b = seg_off[rec.ray];
        for (int j = 0; j < rec.count; j++) {
            seg_base[rec.first + j] = b;
            b += part_nc[rec.first + j];
        }
    }
}

// Results of the split rays from their segments' partial results.
template <int MODE, int PREC>
__global__ void __launch_bounds__(256) combine_kernel(const SplitRec *__restrict__ list,
                                                      const unsigned long long *split_count,
                                                      const SegStart *__restrict__ segs,
                                                      const double *__restrict__ part_acc,
                                                      const int32_t *__restrict__ part_nc,
                                                      const int32_t *__restrict__ part_last,
                                                      const uint8_t *__restrict__ part_st, double kappa, void *tau,
                                                      int32_t *ncross, uint8_t *status) {
    const int64_t m = (int64_t)*split_count;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const SplitRec rec = list[i];
        double acc = 0.0;
        int32_t nc = 0;
        uint32_t st = 0;
        for (int j = 0; j < rec.count; j++) {
            const int64_t s = rec.first + j;
            if (MODE == MODE_TAU) {
                acc += part_acc[s];
                nc += part_nc[s];
            }
            st |= part_st[s];
            if (j + 1 < rec.count && part_last[s] != segs[s + 1].cur) st |= HG_RAY_LOST;
        }
        if (MODE == MODE_TAU) {
            if (PREC == HG_FP64)
                static_cast<double *>(tau)[rec.ray] = kappa * acc;
            else
                static_cast<float *>(tau)[rec.ray] = (float)acc;
            ncross[rec.ray] = nc;
        }
        if (MODE == MODE_FILL) {
            if (status && st) status[rec.ray] |= (uint8_t)st;
        } else if (status) {
            status[rec.ray] = (uint8_t)st;
        }
    }
}

// Queue order from the bucket counts: ray r goes to the next free slot of
// its bucket.  Each block ranks a chunk of rays in shared memory and takes
// one global slot range per bucket; the order inside a bucket is arbitrary
// and results do not depend on it.
__global__ void __launch_bounds__(256) order_kernel(int64_t n, const float *__restrict__ work,
                                                    const unsigned long long *bucket_count,
                                                    unsigned long long *bucket_fill, int64_t *order) {
    __shared__ unsigned long long base[kBuckets];
    __shared__ unsigned long long gbase[kBuckets];
    __shared__ unsigned int hist[kBuckets];
    if (threadIdx.x == 0) {
        unsigned long long acc = 0;
        for (int b = 0; b < kBuckets; b++) {
            base[b] = acc;
            acc += bucket_count[b];
        }
    }
    for (int64_t c0 = (int64_t)blockIdx.x * blockDim.x; c0 < n; c0 += (int64_t)gridDim.x * blockDim.x) {
        if (threadIdx.x < kBuckets) hist[threadIdx.x] = 0;
        __syncthreads();
        const int64_t r = c0 + threadIdx.x;
        int b = 0;
        unsigned rank = 0;
        if (r < n) {
            b = work_bucket(work[r]);
            rank = atomicAdd(&hist[b], 1u);
        }
        __syncthreads();
        if (threadIdx.x < kBuckets && hist[threadIdx.x])
            gbase[threadIdx.x] = atomicAdd(&bucket_fill[threadIdx.x], (unsigned long long)hist[threadIdx.x]);
        __syncthreads();
        if (r < n) order[base[b] + gbase[b] + rank] = r;
        __syncthreads();
    }
}

// Rays of one grid for the walking loop: a static stride, or a
// warp-aggregated atomic on a global counter.
struct GridRays {
    static constexpr bool kSegments = true;
    const DevGrid *G;
    int64_t n;
    int64_t cursor;
    int64_t stride;
    unsigned long long *counter;
    const int64_t *order;
    int64_t n_seg;  // queue positions 0 .. n_seg-1 are path segments (items n + s)
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
            int64_t pos = (int64_t)(base + grp.thread_rank());
            if (pos < n_seg) {
                ray = n + pos;
                return true;
            }
            pos -= n_seg;
            ray = (pos < n && order) ? order[pos] : pos;
            return pos < n;
        }
        ray = cursor;
        cursor += stride;
        return ray < n;
    }
};

// Dynamic shared memory of a walking launch: the top tree nodes, then the
// threads' geometry slots (9 doubles per thread) at a 16-byte boundary.
__host__ __device__ __forceinline__ size_t geo_offset(size_t node_bytes) { return (node_bytes + 15) / 16 * 16; }
__host__ __device__ __forceinline__ size_t walk_smem(size_t node_bytes, int block) {
    return geo_offset(node_bytes) + (size_t)block * 9 * sizeof(double);
}

// One persistent loop per thread (walk_loop): a lane whose ray has ended
// takes the next one, and every iteration advances each lane by one record
// load, so lanes never wait for the longest path in their warp.
//   OCC: resident blocks of 256 threads per SM the register budget is cut for
//   (3: 80 registers; 4: 64 registers).
//   NAV: 0 the grid's records hold neighbor-list heads, 1 ropes.
template <int KIND, int MODE, int PREC, int OCC, int NAV>
__global__ void __launch_bounds__(256, OCC) trace_kernel(const TraceArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    if (A.run_if && *A.run_if == 0u) return;  // a fallback walk with nothing to do
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
    src.n_seg = 0;
    if (A.n_seg && src.dyn) {
        const unsigned long long c = *A.n_seg;
        src.n_seg = (int64_t)(c < (unsigned long long)A.n_seg_cap ? c : (unsigned long long)A.n_seg_cap);
    }
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
    if (A.gmul) {
        io.gmul = A.gmul;
        io.gmask = A.gmask;
    }
    io.rho_ext = A.rho_ext;
    io.n_rays = A.n;
    io.segs = A.segs;
    io.part_acc = A.part_acc;
    io.part_nc = A.part_nc;
    io.part_last = A.part_last;
    io.part_st = A.part_st;
    io.seg_base = A.seg_base;
    io.stg_ent = A.stg_ent;
    io.stg_next = A.stg_next;
    io.stg_nchunks = A.stg_nchunks;
    io.stg_ctr = A.stg_ctr;
    io.stg_start_ray = A.stg_start_ray;
    io.stg_start_seg = A.stg_start_seg;
    io.stg_overflow = A.stg_overflow;
    io.tau_int = A.tau_int;
    io.int_cell = A.int_cell;
    io.int_t = A.int_t;
    walk_loop<KIND, MODE, PREC, NAV>(src, io, smem, A.n_smem,
                                     reinterpret_cast<double *>(smem + geo_offset(A.n_smem * node_bytes)));
}

// ------------------------------------------------------------------ launch plumbing

typedef void (*KernelFn)(const TraceArgs);

// Walking kernels by [navigation][kind][mode][prec][occupancy]; prec runs
// 0..1, and 0..3 for MODE_TAUADJ and MODE_TAUADJ_STAGE (optical depth and
// gradient precisions).  Rope grids get their own instantiations, so that the
// neighbor-list walk carries no code for ropes.
constexpr int kModes = 7;
inline int mode_precs(int m) {
    return (m == MODE_TAUADJ || m == MODE_TAUADJ_STAGE) ? 4 : (m == MODE_INTERACT ? 1 : 2);
}
KernelFn pick_kernel(int kind, int mode, int prec, int occ, int nav) {
#define HG_K(N, K, M, P) {&trace_kernel<K, M, P, 3, N>, &trace_kernel<K, M, P, 4, N>}
#define HG_M(N, K, M) {HG_K(N, K, M, 0), HG_K(N, K, M, 1), {nullptr, nullptr}, {nullptr, nullptr}}
#define HG_MA(N, K, M) {HG_K(N, K, M, 0), HG_K(N, K, M, 1), HG_K(N, K, M, 2), HG_K(N, K, M, 3)}
#define HG_M1(N, K, M) {HG_K(N, K, M, 0), {nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}}
#define HG_KIND(N, K) {HG_M(N, K, 0), HG_M(N, K, 1), HG_M(N, K, 2), HG_MA(N, K, 3), HG_M(N, K, 4), HG_MA(N, K, 5), \
                       HG_M1(N, K, 6)}
    static const KernelFn table[2][2][kModes][4][2] = {{HG_KIND(0, 0), HG_KIND(0, 1)}, {HG_KIND(1, 0), HG_KIND(1, 1)}};
#undef HG_KIND
#undef HG_M1
#undef HG_MA
#undef HG_M
#undef HG_K
    return table[nav == HG_NAV_ROPES ? 1 : 0][kind][mode][prec][occ == 4 ? 1 : 0];
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

// Default launch shape of the walks: 256 threads, 4 blocks per SM (64
// registers: the ray geometry sits in shared memory), the top 64 tree nodes
// in shared memory -- the walk descends only after edge and corner exits
// and list misses, and every byte of shared memory is taken from the L1
// that serves its record gathers -- persistent dynamic schedule.  The setup
// pass, which descends for every ray, stages the top 8 KB of the tree
// (setup_nodes): its deep levels come through L1 as well, and with 32 KB of
// nodes (and the 16 KB work lattice) per block the k-d preparation of 1e6
// rays took 0.52 ms against 0.29 ms.
constexpr int kWalkNodes = 64;
int setup_nodes(const hg_grid *g) {
    const int node_bytes = g->d.kind == HG_KDTREE ? 16 : 32;
    return (int)std::min<int64_t>(g->d.n_nodes, (8 * 1024) / node_bytes);
}

hg_status resolve_opts(const hg_grid *g, const hg_trace_opts *opts, int &precision, int &block, int &smem_nodes,
                       int &schedule, int &min_blocks, int64_t &max_steps, int &split) {
    precision = opts ? opts->precision : HG_FP64;
    if (precision != HG_FP64 && precision != HG_FP32K) {
        set_error("precision must be HG_FP64 or HG_FP32K");
        return HG_EINVAL;
    }
    const TuneEntry &T = g->tuned[precision];
    block = (opts && opts->block > 0) ? opts->block : (T.valid ? T.block : 256);
    smem_nodes = (opts && opts->smem_nodes >= 0) ? opts->smem_nodes : (T.valid ? T.smem_nodes : kWalkNodes);
    schedule = (opts && opts->schedule > 0) ? opts->schedule : (T.valid ? T.schedule : 0);
    min_blocks = (opts && opts->min_blocks > 0) ? opts->min_blocks : (T.valid ? T.min_blocks : 4);
    max_steps = (opts && opts->max_steps > 0) ? opts->max_steps : 4 * g->d.n_leaves + 64;
    split = opts ? opts->split : HG_SPLIT_AUTO;
    if (split < HG_SPLIT_AUTO || split > HG_SPLIT_FORCE) {
        set_error("split must be HG_SPLIT_AUTO, HG_SPLIT_OFF or HG_SPLIT_FORCE");
        return HG_EINVAL;
    }
    // a step limit below the default could end a whole path but not its segments
    if (max_steps < 4 * g->d.n_leaves + 64) split = HG_SPLIT_OFF;
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

constexpr int kLatticeBytes = kWorkN * kWorkN * kWorkN * (int)sizeof(float);
constexpr int kWalkSmemMax = 200 * 1024 + 256 * 9 * (int)sizeof(double);
constexpr int kSetupSmemMax = 200 * 1024 + kLatticeBytes;

void set_smem_limits() {
    static std::once_flag once;
    std::call_once(once, [] {
        for (int nav = 0; nav < 2; nav++)
            for (int kd = 0; kd < 2; kd++)
                for (int m = 0; m < kModes; m++)
                    for (int p = 0; p < mode_precs(m); p++)
                        for (int oc = 3; oc <= 4; oc++)
                            cudaFuncSetAttribute(pick_kernel(kd, m, p, oc, nav),
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kWalkSmemMax);
        // the setup pass also stages the work lattice after the nodes
        cudaFuncSetAttribute(setup_kernel<HG_KDTREE>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSetupSmemMax);
        cudaFuncSetAttribute(setup_kernel<HG_OCTREE>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSetupSmemMax);
    });
}

// Resident blocks of a walking kernel for a launch shape.
hg_status walk_blocks(KernelFn k, int block, size_t smem, int64_t n, int64_t &blocks) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, smem);
    if (e != cudaSuccess) return cuda_err(e, "occupancy query");
    if (per_sm < 1) {
        set_error("launch shape does not fit on an SM (block %d, %zu B shared)", block, smem);
        return HG_EINVAL;
    }
    blocks = std::min<int64_t>((int64_t)per_sm * sm_count(), (n + block - 1) / block);
    return HG_OK;
}

}  // namespace hg

// Setup, queue order and path segments of one ray batch on one grid: what
// every walk over these rays shares.  Owns one stream-ordered scratch
// allocation.
struct hg_rays {
    const hg_grid *g = nullptr;
    int64_t n = 0;
    const double *o = nullptr, *d = nullptr, *smax = nullptr;
    int block = 256, smem_nodes = 0, min_blocks = 3;
    int64_t max_steps = 0, threads = 0;
    bool dyn = false, ordered = false, splitting = false;
    bool traced = false;  // an optical-depth walk recorded the segments' crossing counts
    size_t smem = 0;       // top tree nodes (the setup pass)
    size_t walk_smem = 0;  // top tree nodes and the threads' ray geometry (the walks)
    unsigned char *scratch = nullptr;
    hg::RayStart *starts = nullptr;
    int64_t *order = nullptr;
    float *work = nullptr;
    unsigned long long *counts = nullptr, *work_total = nullptr, *seg_count = nullptr, *split_count = nullptr,
                       *queue = nullptr;
    hg::SegStart *segs = nullptr;
    double *part_acc = nullptr;
    int32_t *part_nc = nullptr, *part_last = nullptr;
    uint8_t *part_st = nullptr;
    int64_t *seg_base = nullptr;
    hg::SplitRec *list = nullptr;
    int64_t seg_cap = 0;
    // emission staging, allocated by the first staged trace
    unsigned char *stg = nullptr;
    size_t stg_bytes = 0;
    void *stg_ent = nullptr;
    uint32_t *stg_next = nullptr, *stg_start_ray = nullptr, *stg_start_seg = nullptr, *stg_overflow = nullptr;
    unsigned long long *stg_ctr = nullptr;
    uint32_t stg_nchunks = 0;
    int stg_prec = -1;    // precision of the staged lengths; -1: nothing staged
    // gradient scratch: 2^k slots >= n_leaves, leaf c accumulated at slot (c * gscr_mul) & gscr_mask
    void *gscr = nullptr;
    size_t gscr_bytes = 0;
    uint32_t gscr_mul = 0, gscr_mask = 0;
};

namespace hg {

// Build a plan: scratch, setup pass, and for the ordered schedule the
// work-ordered queue and (when allowed) the path segments.
//   exact: per-ray crossing offsets that order the queue exactly, or NULL.
hg_status make_plan(hg_rays &P, const hg_grid *g, int64_t n, const double *o, const double *d, const double *smax,
                    int block, int smem_nodes, int schedule, int min_blocks, int64_t max_steps, bool allow_split,
                    int split, const int64_t *exact, cudaStream_t stream) {
    set_smem_limits();
    P.g = g;
    P.n = n;
    P.o = o;
    P.d = d;
    P.smax = smax;
    P.block = block;
    P.smem_nodes = smem_nodes;
    P.min_blocks = min_blocks;
    P.max_steps = max_steps;
    const int node_bytes = g->d.kind == HG_KDTREE ? 16 : 32;
    P.smem = (size_t)smem_nodes * node_bytes;
    P.walk_smem = walk_smem(P.smem, block);
    int64_t blocks = 0;
    const KernelFn k0 = pick_kernel(g->d.kind, MODE_TAU, HG_FP64, min_blocks, g->d.nav);
    hg_status hs = walk_blocks(k0, block, P.walk_smem, n, blocks);
    if (hs != HG_OK) return hs;
    P.threads = blocks * block;
    // auto schedule: order by estimated work only when each resident thread
    // gets few paths (then the heaviest paths would otherwise set the end)
    if (schedule == 0) schedule = (n < 48 * P.threads) ? 3 : 2;
    P.dyn = (schedule >= 2);
    P.ordered = (schedule == 3);
    P.splitting = P.ordered && allow_split && split != HG_SPLIT_OFF && g->d.work;
    if (P.splitting) {  // segments add queue items: the walks run every resident thread
        hs = walk_blocks(k0, block, P.walk_smem, INT64_MAX / 2, blocks);
        if (hs != HG_OK) return hs;
        P.threads = blocks * block;
    }
    P.seg_cap = P.splitting ? std::min<int64_t>((split == HG_SPLIT_FORCE ? 16 * n : 3 * P.threads) + 1024, 16 * n)
                            : 0;
    // scratch: start records; the queue counter; for the ordered schedule the
    // queue, work estimates and counters (bucket counts and fills, work
    // total, segment and split-ray counts); for splitting the segment
    // records, partial results, emission offsets and the list of split rays
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t start_bytes = al((size_t)n * sizeof(RayStart));
    const size_t order_bytes = P.ordered ? al((size_t)n * sizeof(int64_t)) : 0;
    const size_t work_bytes = P.ordered ? al((size_t)n * sizeof(float)) : 0;
    const size_t count_bytes = al((2 * kBuckets + 4) * sizeof(unsigned long long));
    const size_t seg_bytes = al((size_t)P.seg_cap * sizeof(SegStart));
    const size_t acc_bytes = al((size_t)P.seg_cap * sizeof(double));
    const size_t i32_bytes = al((size_t)P.seg_cap * sizeof(int32_t));
    const size_t u8_bytes = al((size_t)P.seg_cap);
    const size_t base_bytes = al((size_t)P.seg_cap * sizeof(int64_t));
    const size_t list_bytes = al((size_t)(P.seg_cap / 2) * sizeof(SplitRec));
    const size_t total_bytes = start_bytes + order_bytes + work_bytes + count_bytes + seg_bytes + acc_bytes +
                               2 * i32_bytes + u8_bytes + base_bytes + list_bytes;
    cudaError_t e = cudaMallocAsync((void **)&P.scratch, total_bytes, stream);
    if (e != cudaSuccess) {
        P.scratch = nullptr;
        return cuda_err(e, "ray plan scratch");
    }
    size_t off = 0;
    auto take = [&](size_t b) {
        unsigned char *q = b ? P.scratch + off : nullptr;
        off += b;
        return q;
    };
    P.starts = reinterpret_cast<RayStart *>(take(start_bytes));
    P.order = reinterpret_cast<int64_t *>(take(order_bytes));
    P.work = reinterpret_cast<float *>(take(work_bytes));
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(take(count_bytes));
    P.segs = reinterpret_cast<SegStart *>(take(seg_bytes));
    P.part_acc = reinterpret_cast<double *>(take(acc_bytes));
    P.part_nc = reinterpret_cast<int32_t *>(take(i32_bytes));
    P.part_last = reinterpret_cast<int32_t *>(take(i32_bytes));
    P.part_st = reinterpret_cast<uint8_t *>(take(u8_bytes));
    P.seg_base = reinterpret_cast<int64_t *>(take(base_bytes));
    P.list = reinterpret_cast<SplitRec *>(take(list_bytes));
    P.counts = P.ordered ? cnt : nullptr;
    P.work_total = cnt + 2 * kBuckets;
    P.seg_count = cnt + 2 * kBuckets + 1;
    P.split_count = cnt + 2 * kBuckets + 2;
    P.queue = cnt + 2 * kBuckets + 3;
    e = cudaMemsetAsync(cnt, 0, count_bytes, stream);
    if (e != cudaSuccess) return cuda_err(e, "scratch reset");
    const int64_t sblocks = std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 8);
    const int snodes = setup_nodes(g);
    const size_t setup_smem = (size_t)snodes * node_bytes + ((P.ordered && !exact && g->d.work) ? kLatticeBytes : 0);
    if (g->d.kind == HG_KDTREE)
        setup_kernel<HG_KDTREE><<<(unsigned)sblocks, 256, setup_smem, stream>>>(
            g->d, n, o, d, smax, P.starts, snodes, P.counts, exact, P.ordered ? P.work_total : nullptr, P.work);
    else
        setup_kernel<HG_OCTREE><<<(unsigned)sblocks, 256, setup_smem, stream>>>(
            g->d, n, o, d, smax, P.starts, snodes, P.counts, exact, P.ordered ? P.work_total : nullptr, P.work);
    note_launches(1);
    if (P.ordered) {
        order_kernel<<<(unsigned)sblocks, 256, 0, stream>>>(n, P.work, P.counts, P.counts + kBuckets, P.order);
        note_launches(1);
    }
    if (P.splitting) {
        const int force = split == HG_SPLIT_FORCE ? 1 : 0;
        // one warp per candidate ray: as many blocks as are resident at once
        const unsigned pblocks = (unsigned)sm_count() * 4;
        if (g->d.kind == HG_KDTREE)
            split_kernel<HG_KDTREE><<<pblocks, 256, 0, stream>>>(
                g->d, n, o, d, smax, P.starts, smem_nodes, P.work_total, P.counts, P.order, P.threads, force, P.segs,
                P.seg_cap, P.seg_count, P.list, P.split_count);
        else
            split_kernel<HG_OCTREE><<<pblocks, 256, 0, stream>>>(
                g->d, n, o, d, smax, P.starts, smem_nodes, P.work_total, P.counts, P.order, P.threads, force, P.segs,
                P.seg_cap, P.seg_count, P.list, P.split_count);
        note_launches(1);
    }
    e = cudaGetLastError();
    return e == cudaSuccess ? HG_OK : cuda_err(e, "ray plan");
}

void free_plan(hg_rays &P, cudaStream_t stream) {
    if (P.scratch) cudaFreeAsync(P.scratch, stream);
    P.scratch = nullptr;
    if (P.stg) cudaFreeAsync(P.stg, stream);
    P.stg = nullptr;
    P.stg_bytes = 0;
    if (P.gscr) cudaFreeAsync(P.gscr, stream);
    P.gscr = nullptr;
    P.gscr_bytes = 0;
}

// The gradient walks and the copy of a plan scatter into a zeroed scratch
// of 2^k slots (2^k >= n_leaves), leaf c at slot (c * mul) mod 2^k with mul
// odd near 0.618 * 2^k: a bijection that puts consecutive leaf ids (which
// the builder gives to spatially close leaves) about 0.618 * 2^k slots
// apart.  Rays crossing a dense region then spread their atomic adds over
// many L2 lines instead of queueing on the few that hold its leaves.
// grad_scratch_begin allocates and zeroes it and points A at it;
// grad_scratch_end adds slot (c * mul) mod 2^k to grad[c] for every leaf.
hg_status grad_scratch_begin(hg_rays &P, int gp, TraceArgs &A, cudaStream_t stream) {
    const int64_t nl = std::max<int64_t>(P.g->d.n_leaves, 1);
    int k = 0;
    while (((int64_t)1 << k) < nl) k++;
    const size_t bytes = ((size_t)1 << k) * (gp == 0 ? sizeof(double) : sizeof(float));
    if (bytes > P.gscr_bytes) {
        if (P.gscr) cudaFreeAsync(P.gscr, stream);
        P.gscr = nullptr;
        P.gscr_bytes = 0;
        cudaError_t e = cudaMallocAsync(&P.gscr, bytes, stream);
        if (e != cudaSuccess) {
            P.gscr = nullptr;
            return cuda_err(e, "gradient scratch");
        }
        P.gscr_bytes = bytes;
    }
    cudaError_t e = cudaMemsetAsync(P.gscr, 0, bytes, stream);
    if (e != cudaSuccess) return cuda_err(e, "gradient scratch reset");
    P.gscr_mask = (uint32_t)(((uint64_t)1 << k) - 1);
    P.gscr_mul = (uint32_t)(0.6180339887498949 * (double)((uint64_t)1 << k)) | 1u;
    A.grad = P.gscr;
    A.gmul = P.gscr_mul;
    A.gmask = P.gscr_mask;
    return HG_OK;
}

template <typename T>
__global__ void __launch_bounds__(256) grad_unhash_kernel(int64_t n, const T *__restrict__ scr, uint32_t mul,
                                                          uint32_t mask, T *grad) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x)
        grad[c] += scr[((uint32_t)c * mul) & mask];
}

hg_status grad_scratch_end(hg_rays &P, int gp, void *grad, cudaStream_t stream) {
    const int64_t n = P.g->d.n_leaves;
    if (n <= 0) return HG_OK;
    const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 8);
    if (gp == 0)
        grad_unhash_kernel<double><<<blocks, 256, 0, stream>>>(n, static_cast<const double *>(P.gscr), P.gscr_mul,
                                                              P.gscr_mask, static_cast<double *>(grad));
    else
        grad_unhash_kernel<float><<<blocks, 256, 0, stream>>>(n, static_cast<const float *>(P.gscr), P.gscr_mul,
                                                             P.gscr_mask, static_cast<float *>(grad));
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HG_OK : cuda_err(e, "gradient unhash");
}

// Size the staging pool: per_ray entries per ray plus one chunk per walking
// thread (each thread's last chunk is partly filled), at most 2^31 entries;
// per_ray < 0: exactly -per_ray chunks.
hg_status make_staging(hg_rays &P, int prec, int64_t per_ray, cudaStream_t stream) {
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    int64_t entries = per_ray < 0 ? -per_ray * (int64_t)kStageChunk
                                  : P.n * per_ray + (P.threads + 1) * (int64_t)kStageChunk;
    entries = std::min<int64_t>(entries, (int64_t)0x7fffffff - kStageChunk);
    const int64_t nchunks = entries / kStageChunk;
    entries = nchunks * kStageChunk;
    const size_t esz = prec == HG_FP64 ? 16 : 8;  // see stage_put
    const size_t b_ent = al((size_t)entries * esz);
    const size_t b_next = al((size_t)nchunks * sizeof(uint32_t)), b_sr = al((size_t)P.n * sizeof(uint32_t));
    const size_t b_ss = al((size_t)std::max<int64_t>(P.seg_cap, 1) * sizeof(uint32_t)), b_ctr = 256;
    const size_t total = b_ent + b_next + b_sr + b_ss + b_ctr;
    if (total > P.stg_bytes) {
        if (P.stg) cudaFreeAsync(P.stg, stream);
        P.stg = nullptr;
        P.stg_bytes = 0;
        cudaError_t e = cudaMallocAsync((void **)&P.stg, total, stream);
        if (e != cudaSuccess) {
            P.stg = nullptr;
            return cuda_err(e, "emission staging");
        }
        P.stg_bytes = total;
    }
    unsigned char *q = P.stg;
    P.stg_ent = q;
    q += b_ent;
    P.stg_next = reinterpret_cast<uint32_t *>(q);
    q += b_next;
    P.stg_start_ray = reinterpret_cast<uint32_t *>(q);
    q += b_sr;
    P.stg_start_seg = reinterpret_cast<uint32_t *>(q);
    q += b_ss;
    P.stg_ctr = reinterpret_cast<unsigned long long *>(q);
    P.stg_overflow = reinterpret_cast<uint32_t *>(q + 8);
    P.stg_nchunks = (uint32_t)nchunks;
    cudaError_t e = cudaMemsetAsync(q, 0, 16, stream);
    return e == cudaSuccess ? HG_OK : cuda_err(e, "staging reset");
}

// Copy cnt staged entries starting at entry e (following the walking
// thread's chunk chain) to the emission arrays at b, G lanes together (lane
// g of the group, G a power of two dividing 32): each chunk piece is read
// and written by consecutive lanes.  Entries at or beyond cap are dropped
// (returns false then, on every lane of the group).
// GP >= 0: also scatter the adjoint, grad[slot(cell)] += wk * ds (wk = kappa
// w of the ray; GP 0 FP64, 1 FP32 gradient; slot(c) = (c * gmul) & gmask),
// for every entry, dropped or not.
template <int G, int GP, typename DS>
__device__ __forceinline__ bool copy_staged_group(uint32_t e, int64_t cnt, int64_t b, const void *__restrict__ ent,
                                                  const uint32_t *__restrict__ next, int32_t *out_cell, DS *out_ds,
                                                  int64_t cap, int g, double wk, void *grad, uint32_t gmul,
                                                  uint32_t gmask, unsigned long long keep) {
    bool fit = true;
    while (cnt > 0) {
        const int64_t piece = std::min<int64_t>(cnt, (int64_t)(kStageChunk - (e & (kStageChunk - 1u))));
        for (int64_t k = g; k < piece; k += G) {
            int32_t c;
            DS l;
            stage_get(ent, (int64_t)e + k, c, l);
            if (b + k < cap) {
                out_cell[b + k] = c;
                out_ds[b + k] = l;
            } else {
                fit = false;
            }
            const uint32_t slot = ((uint32_t)c * gmul) & gmask;
            if (GP == 0) {
                red_add_keep(static_cast<double *>(grad) + slot, wk * (double)l, keep);
            } else if (GP == 1) {
                red_add_keep(static_cast<float *>(grad) + slot, __double2float_rn(wk * (double)l), keep);
            }
        }
        cnt -= piece;
        b += piece;
        if (cnt > 0) e = next[e >> kStageShift] << kStageShift;
    }
    return fit;
}

// Emission from the staging pool: each ray's crossings (or its segments',
// in path order with the counts of the staged walk) copied to its CSR slot,
// the entries of 32 consecutive unsplit rays spread over a warp's lanes and a
// warp per split ray; with GP >= 0 the same pass scatters the adjoint (kappa w
// of the ray times each length).
// Does nothing when the pool overflowed (the walks that follow then do the
// emission and the adjoint).
template <int GP, typename DS>
__global__ void __launch_bounds__(256) gather_kernel(int64_t n, const RayStart *__restrict__ starts,
                                                     const int64_t *__restrict__ seg_off,
                                                     const uint32_t *__restrict__ start_ray,
                                                     const SplitRec *__restrict__ list,
                                                     const unsigned long long *split_count,
                                                     const uint32_t *__restrict__ start_seg,
                                                     const int32_t *__restrict__ part_nc,
                                                     const void *__restrict__ ent,
                                                     const uint32_t *__restrict__ next, const uint32_t *overflow,
                                                     int32_t *out_cell, DS *out_ds, int64_t cap, uint8_t *status,
                                                     double kappa, const float *__restrict__ w, void *grad,
                                                     uint32_t gmul, uint32_t gmask) {
    if (*overflow) return;
    const unsigned long long keep = GP >= 0 ? l2_evict_last_policy() : 0ULL;
    const int lane = threadIdx.x & 31;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t w0 = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    // unsplit rays: a warp takes 32 consecutive rays and spreads their entries over its lanes, entry e of
    // the window going to lane e mod 32 (a lane finds its ray by a binary search over the window's
    // exclusive prefix of counts), so that short rays leave no lane idle and the CSR writes of
    // consecutive entries are consecutive
    for (int64_t r0 = w0 * 32; r0 < n; r0 += nw * 32) {
        const int64_t r = r0 + lane;
        int64_t cnt = 0, b = 0;
        uint32_t first = 0;
        double wk = 0.0;
        if (r < n && !(starts[r].sg & SG_SPLIT)) {
            b = seg_off[r];
            cnt = seg_off[r + 1] - b;
            if (cnt > 0) {
                first = start_ray[r];
                if (GP >= 0) wk = kappa * (double)__ldg(w + r);
                if (status && b + cnt > cap) status[r] |= HG_RAY_OVERFLOW;
            }
        }
        int64_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int64_t excl = incl - cnt;
        const int64_t total = __shfl_sync(0xffffffffu, incl, 31);
        for (int64_t base = 0; base < total; base += 32) {
            const int64_t e = base + lane;
            // the largest window lane j with excl_j <= e owns entry e (lanes without entries share the
            // next lane's prefix, so they are never the largest)
            int j = 0;
#pragma unroll
            for (int step = 16; step >= 1; step >>= 1) {
                const int64_t ex = __shfl_sync(0xffffffffu, excl, j + step);
                if (ex <= e) j += step;
            }
            const int64_t exj = __shfl_sync(0xffffffffu, excl, j);
            const int64_t bj = __shfl_sync(0xffffffffu, b, j);
            const uint32_t fj = __shfl_sync(0xffffffffu, first, j);
            const double wkj = GP >= 0 ? __shfl_sync(0xffffffffu, wk, j) : 0.0;
            if (e >= total) continue;
            const int64_t k = e - exj;
            // the walking thread appended the ray in its chunk chain: entries are contiguous up to the
            // end of the first chunk, then continue in the chained chunks
            int64_t pos = (int64_t)fj + k;
            const int64_t avail = (int64_t)(kStageChunk - (fj & (kStageChunk - 1u)));
            if (k >= avail) {
                int64_t rest = k - avail;
                uint32_t c = next[fj >> kStageShift];
                while (rest >= (int64_t)kStageChunk) {
                    c = next[c];
                    rest -= kStageChunk;
                }
                pos = ((int64_t)c << kStageShift) + rest;
            }
            int32_t cc;
            DS l;
            stage_get(ent, pos, cc, l);
            if (bj + k < cap) {
                out_cell[bj + k] = cc;
                out_ds[bj + k] = l;
            }
            const uint32_t slot = ((uint32_t)cc * gmul) & gmask;
            if (GP == 0) {
                red_add_keep(static_cast<double *>(grad) + slot, wkj * (double)l, keep);
            } else if (GP == 1) {
                red_add_keep(static_cast<float *>(grad) + slot, __double2float_rn(wkj * (double)l), keep);
            }
        }
    }
    // split rays: one warp each, segments in path order
    const int64_t m = split_count ? (int64_t)*split_count : 0;
    for (int64_t i = w0; i < m; i += nw) {
        const SplitRec rec = list[i];
        int64_t b = seg_off[rec.ray];
        const double wk = GP >= 0 ? kappa * (double)__ldg(w + rec.ray) : 0.0;
        bool fit = true;
        for (int j = 0; j < rec.count; j++) {
            const int64_t cnt = part_nc[rec.first + j];
            if (cnt > 0)
                fit = copy_staged_group<32, GP>(start_seg[rec.first + j], cnt, b, ent, next, out_cell, out_ds, cap,
                                                lane, wk, grad, gmul, gmask, keep) &&
                      fit;
            b += cnt;
        }
        if (!__all_sync(0xffffffffu, fit) && status && lane == 0) status[rec.ray] |= HG_RAY_OVERFLOW;
    }
}

// One walk over a plan.  A carries the outputs of the mode (and kappa, w,
// rho_ext); the plan supplies rays, start records, queue and segments.
hg_status walk_plan(hg_rays &P, int mode, int prec, TraceArgs A, cudaStream_t stream) {
    if (P.n == 0) return HG_OK;
    const hg_grid *g = P.g;
    KernelFn k = pick_kernel(g->d.kind, mode, prec, P.min_blocks, g->d.nav);
    int64_t blocks = 0;
    hg_status hs = walk_blocks(k, P.block, P.walk_smem, P.splitting ? INT64_MAX / 2 : P.n, blocks);
    if (hs != HG_OK) return hs;
    A.G = g->d;
    A.n = P.n;
    A.o = P.o;
    A.d = P.d;
    A.smax = P.smax;
    A.max_steps = P.max_steps;
    A.n_smem = P.smem_nodes;
    A.dyn = P.dyn ? 1 : 0;
    A.starts = P.starts;
    A.order = P.order;
    A.counter = P.queue;
    if (P.splitting) {
        A.n_seg = P.seg_count;
        A.n_seg_cap = P.seg_cap;
        A.segs = P.segs;
        A.part_acc = P.part_acc;
        A.part_nc = P.part_nc;
        A.part_last = P.part_last;
        A.part_st = P.part_st;
        A.seg_base = P.seg_base;
    }
    if (mode == MODE_TAU_STAGE || mode == MODE_TAUADJ_STAGE) {
        A.stg_ent = P.stg_ent;
        A.stg_next = P.stg_next;
        A.stg_nchunks = P.stg_nchunks;
        A.stg_ctr = P.stg_ctr;
        A.stg_start_ray = P.stg_start_ray;
        A.stg_start_seg = P.stg_start_seg;
        A.stg_overflow = P.stg_overflow;
    }
    cudaError_t e = cudaMemsetAsync(P.queue, 0, sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return cuda_err(e, "queue reset");
    const unsigned cblocks =
        (unsigned)std::max<int64_t>(1, std::min<int64_t>((P.seg_cap / 2 + 255) / 256, (int64_t)sm_count() * 4));
    if (P.splitting && mode == MODE_FILL) {
        seg_base_kernel<<<cblocks, 256, 0, stream>>>(P.list, P.split_count, A.seg_off, P.part_nc, P.seg_base);
        note_launches(1);
    }
    k<<<(unsigned)blocks, P.block, P.walk_smem, stream>>>(A);
    note_launches(1);
    e = cudaGetLastError();
    if (e == cudaSuccess && P.splitting) {
        if (mode == MODE_TAU || mode == MODE_TAUADJ || mode == MODE_TAU_STAGE || mode == MODE_TAUADJ_STAGE) {
            if ((prec & 1) == HG_FP64)
                combine_kernel<MODE_TAU, HG_FP64><<<cblocks, 256, 0, stream>>>(
                    P.list, P.split_count, P.segs, P.part_acc, P.part_nc, P.part_last, P.part_st, A.kappa, A.tau,
                    A.ncross, A.status);
            else
                combine_kernel<MODE_TAU, HG_FP32K><<<cblocks, 256, 0, stream>>>(
                    P.list, P.split_count, P.segs, P.part_acc, P.part_nc, P.part_last, P.part_st, A.kappa, A.tau,
                    A.ncross, A.status);
        } else if (mode == MODE_FILL) {
            combine_kernel<MODE_FILL, 0><<<cblocks, 256, 0, stream>>>(P.list, P.split_count, P.segs, P.part_acc,
                                                                    P.part_nc, P.part_last, P.part_st, A.kappa,
                                                                    nullptr, nullptr, A.status);
        } else {
            combine_kernel<MODE_ADJ, 0><<<cblocks, 256, 0, stream>>>(P.list, P.split_count, P.segs, P.part_acc,
                                                                   P.part_nc, P.part_last, P.part_st, A.kappa,
                                                                   nullptr, nullptr, A.status);
        }
        note_launches(1);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_err(e, "trace launch");
    if (mode == MODE_TAU || mode == MODE_TAUADJ || mode == MODE_TAU_STAGE || mode == MODE_TAUADJ_STAGE)
        P.traced = true;
    return HG_OK;
}

// A one-shot walk: plan, walk, free.  Long paths are cut only in the modes
// whose per-ray results add up (a one-shot fill has no segment counts).
hg_status launch_trace(const hg_grid *g, int mode, int prec, TraceArgs A, int block, int smem_nodes, int schedule,
                       int min_blocks, int split, cudaStream_t stream) {
    if (A.n == 0) return HG_OK;
    hg_rays P;
    hg_status hs = make_plan(P, g, A.n, A.o, A.d, A.smax, block, smem_nodes, schedule, min_blocks, A.max_steps,
                             mode == MODE_TAU || mode == MODE_ADJ, split, mode == MODE_FILL ? A.seg_off : nullptr,
                             stream);
    if (mode == MODE_ADJ) {  // through the hashed gradient slots (prec: the gradient's precision)
        void *grad = A.grad;
        if (hs == HG_OK) hs = grad_scratch_begin(P, prec, A, stream);
        if (hs == HG_OK) hs = walk_plan(P, mode, prec, A, stream);
        if (hs == HG_OK) hs = grad_scratch_end(P, prec, grad, stream);
    } else if (hs == HG_OK) {
        hs = walk_plan(P, mode, prec, A, stream);
    }
    free_plan(P, stream);
    return hs;
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
    int prec, block, smem_nodes, schedule, min_blocks, split;
    int64_t max_steps;
    if ((st = resolve_opts(g, opts, prec, block, smem_nodes, schedule, min_blocks, max_steps, split)) != HG_OK) return st;
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
    return launch_trace(g, MODE_TAU, prec, A, block, smem_nodes, schedule, min_blocks, split, (cudaStream_t)stream);
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
    int prec, block, smem_nodes, schedule, min_blocks, split;
    int64_t max_steps;
    if ((st = resolve_opts(g, opts, prec, block, smem_nodes, schedule, min_blocks, max_steps, split)) != HG_OK) return st;
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
    return launch_trace(g, MODE_TAU, prec, A, block, smem_nodes, schedule, min_blocks, split, (cudaStream_t)stream);
}

extern "C" hg_status hg_find_interactions(const hg_grid *g, int64_t n, const double *o, const double *d,
                                          const double *s_max, double kappa, const double *tau_int,
                                          const hg_trace_opts *opts, int32_t *cell, double *t, int32_t *ncross,
                                          uint8_t *ray_status, hg_stream stream) {
    hg_status st = check_rays(g, n, o, d);
    if (st != HG_OK) return st;
    if (n > 0 && (!tau_int || !cell || !t || !ncross)) {
        set_error("hg_find_interactions: tau_int, cell, t and ncross are required");
        return HG_EINVAL;
    }
    int prec, block, smem_nodes, schedule, min_blocks, split;
    int64_t max_steps;
    if ((st = resolve_opts(g, opts, prec, block, smem_nodes, schedule, min_blocks, max_steps, split)) != HG_OK) return st;
    // The search keeps the drawn depth and the interaction state beside the walk's own: cut to 64
    // registers it spills, and at 80 (3 blocks/SM) it runs about a tenth faster on the disk grids.
    if (!(opts && opts->min_blocks > 0)) min_blocks = 3;
    TraceArgs A{};
    A.G = g->d;
    A.n = n;
    A.o = o;
    A.d = d;
    A.smax = s_max;
    A.kappa = kappa;
    A.tau_int = tau_int;
    A.int_cell = cell;
    A.int_t = t;
    A.ncross = ncross;
    A.status = ray_status;
    A.max_steps = max_steps;
    // FP64 only, and never cut into segments (where a path stops depends on all that precedes)
    return launch_trace(g, MODE_INTERACT, HG_FP64, A, block, smem_nodes, schedule, min_blocks, HG_SPLIT_OFF,
                        (cudaStream_t)stream);
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
    int prec, block, smem_nodes, schedule, min_blocks, split;
    int64_t max_steps;
    if ((st = resolve_opts(g, opts, prec, block, smem_nodes, schedule, min_blocks, max_steps, split)) != HG_OK) return st;
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
    return launch_trace(g, MODE_FILL, prec, A, block, smem_nodes, schedule, min_blocks, split, (cudaStream_t)stream);
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
    int prec, block, smem_nodes, schedule, min_blocks, split;
    int64_t max_steps;
    if ((st = resolve_opts(g, opts, prec, block, smem_nodes, schedule, min_blocks, max_steps, split)) != HG_OK) return st;
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
    return launch_trace(g, MODE_ADJ, grad_precision, A, block, smem_nodes, schedule, min_blocks, split,
                        (cudaStream_t)stream);
}

// ------------------------------------------------------------------ prepared rays

extern "C" hg_status hg_rays_prepare(const hg_grid *g, int64_t n, const double *o, const double *d,
                                     const double *s_max, const hg_trace_opts *opts, hg_rays **out,
                                     hg_stream stream) {
    if (!out) {
        set_error("hg_rays_prepare: out is required");
        return HG_EINVAL;
    }
    *out = nullptr;
    hg_status st = check_rays(g, n, o, d);
    if (st != HG_OK) return st;
    int prec, block, smem_nodes, schedule, min_blocks, split;
    int64_t max_steps;
    if ((st = resolve_opts(g, opts, prec, block, smem_nodes, schedule, min_blocks, max_steps, split)) != HG_OK) return st;
    hg_rays *r = new (std::nothrow) hg_rays;
    if (!r) {
        set_error("hg_rays_prepare: out of host memory");
        return HG_ENOMEM;
    }
    if (n > 0) {
        st = make_plan(*r, g, n, o, d, s_max, block, smem_nodes, schedule, min_blocks, max_steps, true, split, nullptr,
                       (cudaStream_t)stream);
        if (st != HG_OK) {
            free_plan(*r, (cudaStream_t)stream);
            delete r;
            return st;
        }
    }
    r->g = g;
    r->n = n;
    *out = r;
    return HG_OK;
}

extern "C" hg_status hg_rays_trace(hg_rays *r, double kappa, const double *rho, int32_t precision, void *tau,
                                   int32_t *ncross, uint8_t *ray_status, hg_stream stream) {
    if (!r) {
        set_error("hg_rays_trace: null rays");
        return HG_EINVAL;
    }
    if (precision != HG_FP64 && precision != HG_FP32K) {
        set_error("precision must be HG_FP64 or HG_FP32K");
        return HG_EINVAL;
    }
    if (r->n > 0 && (!tau || !ncross)) {
        set_error("hg_rays_trace: tau and ncross are required");
        return HG_EINVAL;
    }
    TraceArgs A{};
    A.kappa = kappa;
    A.tau = tau;
    A.ncross = ncross;
    A.status = ray_status;
    A.rho_ext = rho;
    return walk_plan(*r, MODE_TAU, precision, A, (cudaStream_t)stream);
}

extern "C" hg_status hg_rays_trace_gradient(hg_rays *r, double kappa, const double *rho, int32_t precision,
                                            void *tau, int32_t *ncross, uint8_t *ray_status, const float *w,
                                            int32_t grad_precision, void *grad_rho, hg_stream stream) {
    if (!r) {
        set_error("hg_rays_trace_gradient: null rays");
        return HG_EINVAL;
    }
    if (precision != HG_FP64 && precision != HG_FP32K) {
        set_error("precision must be HG_FP64 or HG_FP32K");
        return HG_EINVAL;
    }
    if (grad_precision != 0 && grad_precision != 1) {
        set_error("hg_rays_trace_gradient: grad_precision must be 0 (f64) or 1 (f32)");
        return HG_EINVAL;
    }
    if (r->n > 0 && (!tau || !ncross || !w || !grad_rho)) {
        set_error("hg_rays_trace_gradient: tau, ncross, w and grad_rho are required");
        return HG_EINVAL;
    }
    if (r->n == 0) return HG_OK;
    TraceArgs A{};
    A.kappa = kappa;
    A.tau = tau;
    A.ncross = ncross;
    A.status = ray_status;
    A.rho_ext = rho;
    A.w = w;
    hg_status st = grad_scratch_begin(*r, grad_precision, A, (cudaStream_t)stream);
    if (st == HG_OK) st = walk_plan(*r, MODE_TAUADJ, precision | (grad_precision << 1), A, (cudaStream_t)stream);
    if (st == HG_OK) st = grad_scratch_end(*r, grad_precision, grad_rho, (cudaStream_t)stream);
    return st;
}

extern "C" hg_status hg_rays_trace_stage(hg_rays *r, double kappa, const double *rho, int32_t precision, void *tau,
                                         int32_t *ncross, uint8_t *ray_status, const float *w, int32_t grad_precision,
                                         void *grad_rho, int32_t stage_per_ray, hg_stream stream) {
    if (!r) {
        set_error("hg_rays_trace_stage: null rays");
        return HG_EINVAL;
    }
    if (precision != HG_FP64 && precision != HG_FP32K) {
        set_error("precision must be HG_FP64 or HG_FP32K");
        return HG_EINVAL;
    }
    if (w && grad_precision != 0 && grad_precision != 1) {
        set_error("hg_rays_trace_stage: grad_precision must be 0 (f64) or 1 (f32)");
        return HG_EINVAL;
    }
    if (r->n > 0 && (!tau || !ncross || (w && !grad_rho))) {
        set_error("hg_rays_trace_stage: tau and ncross (and grad_rho with w) are required");
        return HG_EINVAL;
    }
    if (r->n == 0) {
        r->stg_prec = precision;
        return HG_OK;
    }
    hg_status st = make_staging(*r, precision, stage_per_ray ? stage_per_ray : 64, (cudaStream_t)stream);
    if (st != HG_OK) return st;
    TraceArgs A{};
    A.kappa = kappa;
    A.tau = tau;
    A.ncross = ncross;
    A.status = ray_status;
    A.rho_ext = rho;
    A.w = w;
    if (w) {
        st = grad_scratch_begin(*r, grad_precision, A, (cudaStream_t)stream);
        if (st == HG_OK)
            st = walk_plan(*r, MODE_TAUADJ_STAGE, precision | (grad_precision << 1), A, (cudaStream_t)stream);
        if (st == HG_OK) st = grad_scratch_end(*r, grad_precision, grad_rho, (cudaStream_t)stream);
    } else {
        st = walk_plan(*r, MODE_TAU_STAGE, precision, A, (cudaStream_t)stream);
    }
    r->stg_prec = (st == HG_OK) ? precision : -1;
    return st;
}

// hg_rays_emit_staged (gp < 0) and hg_rays_emit_staged_gradient (gp 0: FP64
// gradient, 1: FP32).
static hg_status emit_staged(const char *name, hg_rays *r, const int64_t *seg_off, int32_t *seg_cell, void *seg_ds,
                             int64_t seg_capacity, uint8_t *ray_status, double kappa, const float *w, int gp,
                             void *grad, cudaStream_t s) {
    if (!r) {
        set_error("%s: null rays", name);
        return HG_EINVAL;
    }
    if (r->stg_prec < 0) {
        set_error("%s: call hg_rays_trace_stage on these rays first", name);
        return HG_EINVAL;
    }
    if (r->n > 0 && (!seg_off || (seg_capacity > 0 && (!seg_cell || !seg_ds)) || seg_capacity < 0)) {
        set_error("%s: bad segment arrays", name);
        return HG_EINVAL;
    }
    if (gp >= 0 && r->n > 0 && (!w || !grad)) {
        set_error("%s: w and grad_rho are required", name);
        return HG_EINVAL;
    }
    if (r->n == 0) return HG_OK;
    TraceArgs B{};  // the adjoint: the copy's scatter, or the fallback gradient walk
    B.kappa = kappa;
    B.w = w;
    B.run_if = r->stg_overflow;  // statuses stay those of the staged trace and the fill
    if (gp >= 0) {
        hg_status st = grad_scratch_begin(*r, gp, B, s);
        if (st != HG_OK) return st;
    }
    const int64_t gblocks = std::min<int64_t>((r->n * 8 + 255) / 256, (int64_t)sm_count() * 8);
    const unsigned long long *sc = r->splitting ? r->split_count : nullptr;
#define HG_GATHER(GP, DS)                                                                                          \
    gather_kernel<GP, DS><<<(unsigned)gblocks, 256, 0, s>>>(                                                     \
        r->n, r->starts, seg_off, r->stg_start_ray, r->list, sc, r->stg_start_seg, r->part_nc, r->stg_ent,      \
        r->stg_next, r->stg_overflow, seg_cell, static_cast<DS *>(seg_ds), seg_capacity, ray_status, kappa, w,  \
        B.grad, B.gmul, B.gmask)
    if (r->stg_prec == HG_FP64) {
        if (gp < 0)
            HG_GATHER(-1, double);
        else if (gp == 0)
            HG_GATHER(0, double);
        else
            HG_GATHER(1, double);
    } else {
        if (gp < 0)
            HG_GATHER(-1, float);
        else if (gp == 0)
            HG_GATHER(0, float);
        else
            HG_GATHER(1, float);
    }
#undef HG_GATHER
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(e, "gather launch");
    // the fill walk (and the adjoint walk) run only when the staging pool overflowed
    TraceArgs A{};
    A.seg_off = seg_off;
    A.seg_cell = seg_cell;
    A.seg_ds = seg_ds;
    A.seg_cap = seg_capacity;
    A.status = ray_status;
    A.run_if = r->stg_overflow;
    hg_status st = walk_plan(*r, MODE_FILL, r->stg_prec, A, s);
    if (st != HG_OK || gp < 0) return st;
    st = walk_plan(*r, MODE_ADJ, gp, B, s);
    if (st == HG_OK) st = grad_scratch_end(*r, gp, grad, s);
    return st;
}

extern "C" hg_status hg_rays_emit_staged(hg_rays *r, const int64_t *seg_off, int32_t *seg_cell, void *seg_ds,
                                         int64_t seg_capacity, uint8_t *ray_status, hg_stream stream) {
    return emit_staged("hg_rays_emit_staged", r, seg_off, seg_cell, seg_ds, seg_capacity, ray_status, 0.0, nullptr,
                       -1, nullptr, (cudaStream_t)stream);
}

extern "C" hg_status hg_rays_emit_staged_gradient(hg_rays *r, const int64_t *seg_off, int32_t *seg_cell,
                                                  void *seg_ds, int64_t seg_capacity, uint8_t *ray_status,
                                                  double kappa, const float *w, int32_t grad_precision,
                                                  void *grad_rho, hg_stream stream) {
    if (grad_precision != 0 && grad_precision != 1) {
        set_error("hg_rays_emit_staged_gradient: grad_precision must be 0 (f64) or 1 (f32)");
        return HG_EINVAL;
    }
    return emit_staged("hg_rays_emit_staged_gradient", r, seg_off, seg_cell, seg_ds, seg_capacity, ray_status, kappa,
                       w, grad_precision, grad_rho, (cudaStream_t)stream);
}

extern "C" hg_status hg_rays_fill(hg_rays *r, int32_t precision, const int64_t *seg_off, int32_t *seg_cell,
                                  void *seg_ds, int64_t seg_capacity, uint8_t *ray_status, hg_stream stream) {
    if (!r) {
        set_error("hg_rays_fill: null rays");
        return HG_EINVAL;
    }
    if (precision != HG_FP64 && precision != HG_FP32K) {
        set_error("precision must be HG_FP64 or HG_FP32K");
        return HG_EINVAL;
    }
    if (r->n > 0 && (!seg_off || (seg_capacity > 0 && (!seg_cell || !seg_ds)) || seg_capacity < 0)) {
        set_error("hg_rays_fill: bad segment arrays");
        return HG_EINVAL;
    }
    if (r->splitting && !r->traced) {
        set_error("hg_rays_fill: these rays are walked as path segments; call hg_rays_trace on them first");
        return HG_EINVAL;
    }
    TraceArgs A{};
    A.seg_off = seg_off;
    A.seg_cell = seg_cell;
    A.seg_ds = seg_ds;
    A.seg_cap = seg_capacity;
    A.status = ray_status;
    return walk_plan(*r, MODE_FILL, precision, A, (cudaStream_t)stream);
}

extern "C" hg_status hg_rays_gradient(hg_rays *r, double kappa, const float *w, int32_t grad_precision,
                                      void *grad_rho, hg_stream stream) {
    if (!r) {
        set_error("hg_rays_gradient: null rays");
        return HG_EINVAL;
    }
    if (r->n > 0 && (!w || !grad_rho)) {
        set_error("hg_rays_gradient: w and grad_rho are required");
        return HG_EINVAL;
    }
    if (grad_precision != 0 && grad_precision != 1) {
        set_error("hg_rays_gradient: grad_precision must be 0 (f64) or 1 (f32)");
        return HG_EINVAL;
    }
    if (r->n == 0) return HG_OK;
    TraceArgs A{};
    A.kappa = kappa;
    A.w = w;
    hg_status st = grad_scratch_begin(*r, grad_precision, A, (cudaStream_t)stream);
    if (st == HG_OK) st = walk_plan(*r, MODE_ADJ, grad_precision, A, (cudaStream_t)stream);
    if (st == HG_OK) st = grad_scratch_end(*r, grad_precision, grad_rho, (cudaStream_t)stream);
    return st;
}

extern "C" void hg_rays_free(hg_rays *r, hg_stream stream) {
    if (!r) return;
    free_plan(*r, (cudaStream_t)stream);
    delete r;
}

extern "C" hg_status hg_sample_density(const hg_grid *g, int64_t n, const double *pts, int32_t *cell, double *rho,
                                       hg_stream stream) {
    if (!g || n < 0 || (n > 0 && (!pts || !rho))) {
        set_error("hg_sample_density: bad arguments");
        return HG_EINVAL;
    }
    if (n == 0) return HG_OK;
    const int node_bytes = g->d.kind == HG_KDTREE ? 16 : 32;
    const int n_smem = (int)std::min<int64_t>(g->d.n_nodes, (8 * 1024) / node_bytes);
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
    int prec, block, smem_nodes, schedule, min_blocks, split;
    int64_t max_steps;
    if ((st = resolve_opts(g, opts, prec, block, smem_nodes, schedule, min_blocks, max_steps, split)) != HG_OK) return st;
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
    KernelFn k = pick_kernel(g->d.kind, MODE_TAU, prec, min_blocks, g->d.nav);
    const int node_bytes = g->d.kind == HG_KDTREE ? 16 : 32;
    const size_t smem = (size_t)smem_nodes * node_bytes;
    const size_t wsmem = walk_smem(smem, block);
    cudaError_t e = cudaSuccess;
    if (wsmem > 48 * 1024) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kWalkSmemMax);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(setup_kernel<HG_KDTREE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(setup_kernel<HG_OCTREE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return cuda_err(e, "shared-memory limit of the allocation-free walk");
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, block, wsmem);
    if (e != cudaSuccess) return cuda_err(e, "occupancy query");
    if (per_sm < 1) {
        set_error("launch shape does not fit on an SM (block %d, %zu B shared)", block, wsmem);
        return HG_EINVAL;
    }
    int64_t blocks = std::min<int64_t>((int64_t)per_sm * sm_count(), (n + block - 1) / block);
    if (A.dyn) {
        e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), stream);
        if (e != cudaSuccess) return cuda_err(e, "counter reset");
    }
    const int64_t sblocks = std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 8);
    const int snodes = setup_nodes(g);
    const size_t ssmem = (size_t)snodes * node_bytes;
    if (g->d.kind == HG_KDTREE)
        setup_kernel<HG_KDTREE><<<(unsigned)sblocks, 256, ssmem, stream>>>(g->d, n, o, d, s_max, starts, snodes,
                                                                          nullptr, nullptr, nullptr, nullptr);
    else
        setup_kernel<HG_OCTREE><<<(unsigned)sblocks, 256, ssmem, stream>>>(g->d, n, o, d, s_max, starts, snodes,
                                                                          nullptr, nullptr, nullptr, nullptr);
    k<<<(unsigned)blocks, block, wsmem, stream>>>(A);
    note_launches(2);
    e = cudaGetLastError();
    return e == cudaSuccess ? HG_OK : cuda_err(e, "trace launch");
}

}  // namespace hg
