// Device-side path calculation through an octree or k-d tree grid
// (Sect. 2.3): top-down location of the first leaf, then one exit-wall test
// per crossed leaf and the next leaf from that wall's neighbor list.
//
// GB300 runs FP64 add, multiply and compare at about 1/64 of its FP32 rate
// (and 1/16 of its 64-bit integer compare rate), so every comparison of two
// FP64 values is made on order-preserving 64-bit integer keys of those
// values (see okey), which gives exactly the IEEE result (-0 and +0 share a
// key), and only the arithmetic of the contract stays in FP64: the time to
// a wall ahead, the exit point, the segment length and the running sum.
// Leaf bounds and descent split planes are stored as keys; a wall needed in
// arithmetic is turned back into its double by the inverse map.
//
// Every translation unit including this file is compiled with -fmad=false,
// so each FP64 multiply and add below is rounded separately, as the
// arithmetic contract in hgrt.h states; the contract's fused operations (the
// point o + k t on a path and the running sum of rho ds) are explicit
// __fma_rn calls.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>

#include <cstddef>

#include "hg_internal.h"

namespace hg {

// Order-preserving key of a non-NaN double: a < b  <=>  okey(a) < okey(b),
// a == b <=> okey(a) == okey(b) (so -0.0 and +0.0 both map to 0).
__device__ __forceinline__ long long okey(double x) {
    const long long b = __double_as_longlong(x);
    const long long k = b ^ ((b >> 63) & 0x7fffffffffffffffLL);
    return k == -1LL ? 0LL : k;
}
// Inverse of okey (the double with that key; +0.0 for key 0).
__device__ __forceinline__ double kdouble(long long k) {
    return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}
constexpr long long KEY_INF = 0x7ff0000000000000LL;  // okey(+inf)

template <class T>
__device__ __forceinline__ T sel3(int a, T v0, T v1, T v2) {
    return a == 0 ? v0 : (a == 1 ? v1 : v2);
}
__device__ __forceinline__ int32_t sel6(int w, int32_t v0, int32_t v1, int32_t v2, int32_t v3, int32_t v4,
                                        int32_t v5) {
    int32_t r = v0;
    r = (w == 1) ? v1 : r;
    r = (w == 2) ? v2 : r;
    r = (w == 3) ? v3 : r;
    r = (w == 4) ? v4 : r;
    r = (w == 5) ? v5 : r;
    return r;
}

// One leaf record held in registers (bounds as keys).
struct Leaf {
    long long lo0, lo1, lo2, hi0, hi1, hi2;
    double rho;
    float rho32;
    uint32_t base;
    int32_t f0, f1, f2, f3, f4, f5;
    uint32_t c03, c45;

    __device__ __forceinline__ int32_t first(int w) const { return sel6(w, f0, f1, f2, f3, f4, f5); }
    __device__ __forceinline__ int cnt(int w) const {
        return w < 4 ? (int)((c03 >> (8 * w)) & 255u) : (int)((c45 >> (8 * (w - 4))) & 255u);
    }
    __device__ __forceinline__ uint32_t flags() const { return (c45 >> 16) & 255u; }
    __device__ __forceinline__ long long lo(int a) const { return sel3(a, lo0, lo1, lo2); }
    __device__ __forceinline__ long long hi(int a) const { return sel3(a, hi0, hi1, hi2); }
};

// Fetch a whole 96-byte record with three 32-byte read-only loads, one per
// sector (256-bit global loads; the record is 32-byte aligned).  Six 16-byte
// loads asked L1 for every sector twice, and both halves of a missing sector
// went on to L2; the plain optical-depth walk is 3-5 % faster this way.
__device__ __forceinline__ void load_leaf(const LeafRec *__restrict__ R, int32_t id, Leaf &L) {
    const unsigned long long *q = reinterpret_cast<const unsigned long long *>(R + id);
    unsigned long long a0, a1, a2, a3, b0, b1, b2, b3;
    uint32_t e0, e1, e2, e3, e4, e5, e6, e7;
    asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];" : "=l"(a0), "=l"(a1), "=l"(a2), "=l"(a3) : "l"(q));
    asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];" : "=l"(b0), "=l"(b1), "=l"(b2), "=l"(b3) : "l"(q + 4));
    asm("ld.global.nc.v8.u32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(e0), "=r"(e1), "=r"(e2), "=r"(e3), "=r"(e4), "=r"(e5), "=r"(e6), "=r"(e7)
        : "l"(q + 8));
    L.lo0 = (long long)a0;
    L.lo1 = (long long)a1;
    L.lo2 = (long long)a2;
    L.hi0 = (long long)a3;
    L.hi1 = (long long)b0;
    L.hi2 = (long long)b1;
    L.rho = __longlong_as_double((long long)b2);
    L.rho32 = __uint_as_float((uint32_t)(b3 & 0xffffffffULL));
    L.base = (uint32_t)(b3 >> 32);
    L.f0 = (int32_t)e0;
    L.f1 = (int32_t)e1;
    L.f2 = (int32_t)e2;
    L.f3 = (int32_t)e3;
    L.f4 = (int32_t)e4;
    L.f5 = (int32_t)e5;
    L.c03 = e6;
    L.c45 = e7;
}

// Direction signs of a ray: bit a = d_a > 0, bit 3+a = d_a < 0 (neither:
// d_a is a signed zero).
__device__ __forceinline__ bool dpos(uint32_t s, int a) { return (s >> a) & 1u; }
__device__ __forceinline__ bool dneg(uint32_t s, int a) { return (s >> (3 + a)) & 1u; }

// Direction-aware containment on one axis (keys): l < p < h, or p == l with
// d >= 0, or p == h with d < 0, or p == h on the domain's upper face with d == 0.
__device__ __forceinline__ bool in_axis(long long p, long long l, long long h, bool pos, bool neg, bool upper_face) {
    return (l < p && p < h) || (p == l && !neg) || (p == h && (neg || (!pos && upper_face)));
}

// Top-down descent (Sect. 2.3) on keys, from the root or from node start (a
// rope's node).  The first n_smem nodes of the list (the top levels, since
// the list is breadth first) come from shared memory.
// KIND: HG_OCTREE, HG_KDTREE, or 2 = decided at run time from G.kind.
template <int KIND>
__device__ __forceinline__ int32_t descend(const DevGrid &G, const unsigned char *snodes, int n_smem, long long p0,
                                           long long p1, long long p2, uint32_t sg, int32_t start = 0) {
    const bool kd = (KIND == 2) ? (G.kind == HG_KDTREE) : (KIND == HG_KDTREE);
    int32_t nd = start;
    for (int it = 0; it <= G.max_depth; it++) {
        if (kd) {
            longlong2 v;
            if (nd < n_smem)
                v = reinterpret_cast<const longlong2 *>(snodes)[nd];
            else
                v = __ldg(reinterpret_cast<const longlong2 *>(G.nodes) + nd);
            const int32_t child = (int32_t)(uint32_t)((unsigned long long)v.y & 0xffffffffULL);
            const int32_t info = (int32_t)(uint32_t)((unsigned long long)v.y >> 32);
            if (child < 0) return info;
            const long long pa = sel3(info, p0, p1, p2);
            const bool up = (pa > v.x) || (pa == v.x && !dneg(sg, info));
            nd = child + (up ? 1 : 0);
        } else {
            longlong2 v0, v1;
            if (nd < n_smem) {
                v0 = reinterpret_cast<const longlong2 *>(snodes)[2 * nd];
                v1 = reinterpret_cast<const longlong2 *>(snodes)[2 * nd + 1];
            } else {
                v0 = __ldg(reinterpret_cast<const longlong2 *>(G.nodes) + 2 * nd);
                v1 = __ldg(reinterpret_cast<const longlong2 *>(G.nodes) + 2 * nd + 1);
            }
            const int32_t child = (int32_t)(uint32_t)((unsigned long long)v1.y & 0xffffffffULL);
            const int32_t leaf = (int32_t)(uint32_t)((unsigned long long)v1.y >> 32);
            if (child < 0) return leaf;
            const int ci = ((p0 > v0.x) || (p0 == v0.x && !dneg(sg, 0)) ? 1 : 0) |
                           ((p1 > v0.y) || (p1 == v0.y && !dneg(sg, 1)) ? 2 : 0) |
                           ((p2 > v1.x) || (p2 == v1.x && !dneg(sg, 2)) ? 4 : 0);
            nd = child + ci;
        }
    }
    return -1;
}

// Per-ray walking state.  The ray's geometry -- origin o, direction k and
// 1/k per axis -- sits in shared memory, in slots of the walking thread
// (slot q of thread t at g[q * gs] with g = base + t, gs = threads per block,
// so that a warp's accesses fall on consecutive words): it is read a few
// times per crossing, and keeping its 18 registers out of the register file
// lets four 256-thread blocks share an SM without spilling.
struct RayState {
    double *g;   // this thread's first geometry slot
    int gs;      // slot stride
    __device__ __forceinline__ double o(int a) const { return g[a * gs]; }
    __device__ __forceinline__ double k(int a) const { return g[(3 + a) * gs]; }
    __device__ __forceinline__ double ik(int a) const { return g[(6 + a) * gs]; }
    __device__ __forceinline__ void set_geometry(const double *oo, const double *kk, double i0, double i1,
                                                 double i2) {
#pragma unroll
        for (int a = 0; a < 3; a++) {
            g[a * gs] = (oo[a] == 0.0) ? 0.0 : oo[a];  // a signed-zero origin walks like +0
            g[(3 + a) * gs] = kk[a];
        }
        g[6 * gs] = i0;
        g[7 * gs] = i1;
        g[8 * gs] = i2;
    }
    long long ktend;   // key of the path end (KEY_INF: walk to the domain exit)
    long long ktstop;  // a path segment ends after the leaf whose exit time passes this (KEY_INF: none)
    long long ktcur;   // key of the current time
    uint32_t sg;      // direction sign bits
    int32_t cur;
    int32_t steps;
};

enum { WALK_GO = 0, WALK_END = 1, WALK_SKIP = 2 };

// Flag bits above the six direction-sign bits of a ray's sg word.
constexpr uint32_t SG_SKIP_FIRST = 1u << 6;  // a path segment: its first leaf belongs to the segment before
constexpr uint32_t SG_SPLIT = 1u << 7;       // the ray is walked as path segments (start record only)

// Start state of a ray, written by the setup pass and read when a walking
// thread takes the ray: 48 bytes, three 16-byte loads.
struct alignas(16) RayStart {
    double ik0, ik1, ik2;  // 1/d per axis (0 where d_a == 0)
    long long ktstart;     // key of the entry time
    int32_t cur;           // first leaf, or -1 when the ray does not walk
    uint32_t sg;           // direction sign bits | status bits << 8
    float work;            // estimated number of crossings (orders the queue)
    float t1;              // end of the estimate's march (domain exit or s_max, single precision)
};
static_assert(sizeof(RayStart) == 48 && offsetof(RayStart, ktstart) == 24 && offsetof(RayStart, cur) == 32 &&
                  offsetof(RayStart, sg) == 36,
              "ray_resume reads the start record as two double2 and one int4");

// Start record of one segment of a long path (written by the split planner):
// the leaf it starts in and the time it enters it, and the time after which
// it stops.  32 bytes, two 16-byte loads; 1/d comes from the ray's RayStart.
struct alignas(16) SegStart {
    long long ktstart;  // key of the entry time into the first leaf
    long long ktstop;   // stop after the leaf whose exit time passes this (KEY_INF: walk to the end)
    int64_t ray;
    int32_t cur;        // first leaf
    uint32_t sg;        // direction sign bits | SG_SKIP_FIRST
};
static_assert(sizeof(SegStart) == 32 && offsetof(SegStart, ray) == 16,
              "seg_resume reads the segment record as two longlong2");

// Key (okey) of the double equal to the FP32 value with bits fb; subnormal
// FP32 values map to zero's key.  Integer operations only.
__device__ __forceinline__ long long f32_key(float f) {
    const uint32_t fb = __float_as_uint(f);
    const uint32_t e = (fb >> 23) & 0xffu;
    if (e == 0u) return 0LL;
    const unsigned long long mag = e == 0xffu ? 0x7ff0000000000000ULL
                                               : ((unsigned long long)(e + 896u) << 52) |
                                                     ((unsigned long long)(fb & 0x7fffffu) << 29);
    return (fb >> 31) ? -(long long)mag : (long long)mag;
}

// Copy the work lattice (kWorkN^3 floats) into shared memory at lat.
__device__ __forceinline__ void stage_lattice(const DevGrid &G, float *lat) {
    const int4 *src = reinterpret_cast<const int4 *>(G.work);
    int4 *dst = reinterpret_cast<int4 *>(lat);
    for (int i = threadIdx.x; i < kWorkN * kWorkN * kWorkN / 4; i += blockDim.x) dst[i] = __ldg(src + i);
}

// March of the path o + t k, t in [t0, t1], through the coarse work
// lattice (expected crossings per unit length, G.work, or its copy in
// shared memory lat): a 3-D DDA (Amanatides & Woo, 1987) in single
// precision.  Calls f(t, tn, rate, e)
// for every lattice cell the path crosses, [t, tn] being the part inside
// it and e the work before it; returns the total work.  It only orders and
// cuts the work; it never affects a result.
template <class F>
__device__ __forceinline__ float work_march(const DevGrid &G, const float *lat, const float *o, const float *k,
                                            float t0, float t1, F &&f) {
    const int N = G.work_n;
    if (!G.work || N <= 0 || !(t1 > t0)) return 0.0f;
    float tmax[3], tdel[3];
    int c[3], step[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float lo = (float)G.dlo[a];
        const float sc = (float)N / ((float)G.dhi[a] - lo);
        const float ka = k[a] * sc;  // lattice units per unit t
        const float p = (o[a] + k[a] * t0 - lo) * sc;
        int ci = (int)floorf(p);
        ci = ci < 0 ? 0 : (ci > N - 1 ? N - 1 : ci);
        c[a] = ci;
        if (ka > 0.0f) {
            tdel[a] = 1.0f / ka;
            tmax[a] = t0 + ((float)(ci + 1) - p) * tdel[a];
            step[a] = 1;
        } else if (ka < 0.0f) {
            tdel[a] = -1.0f / ka;
            tmax[a] = t0 + (p - (float)ci) * tdel[a];
            step[a] = -1;
        } else {
            tdel[a] = 0.0f;
            tmax[a] = CUDART_INF_F;
            step[a] = 0;
        }
    }
    float t = t0;
    float e = 0.0f;
    for (int it = 0; it < 3 * N + 3; it++) {
        const int ax = (tmax[0] <= tmax[1]) ? (tmax[0] <= tmax[2] ? 0 : 2) : (tmax[1] <= tmax[2] ? 1 : 2);
        float tn = fminf(tmax[ax], t1);
        if (tn < t) tn = t;
        const float rate = lat[c[0] + N * (c[1] + N * c[2])];
        f(t, tn, rate, e);
        e += rate * (tn - t);
        t = tn;
        if (!(tmax[ax] < t1)) break;
        c[ax] += step[ax];
        if (c[ax] < 0 || c[ax] >= N) break;
        tmax[ax] += tdel[ax];
    }
    return e;
}

// Bit tests on doubles (integer operations: the FP64 pipe is scarce).
__device__ __forceinline__ bool dfinite(double x) { return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff; }
__device__ __forceinline__ bool dzero(double x) { return (__double_as_longlong(x) << 1) == 0; }
__device__ __forceinline__ bool dgt0(double x) { return __double_as_longlong(x) > 0; }  // x > 0 (x not NaN)
__device__ __forceinline__ bool dlt0(double x) { return __double_as_longlong(x) < 0 && !dzero(x); }

// Set up a ray (the first-cell location of Sect. 2.3): checks, 1/d, clip
// against the domain, top-down descent to the first leaf.  Runs once per
// ray in its own pass.  An origin strictly inside the domain (every
// emission path) needs no clip: the contract's entry time is then 0 and
// the start point the origin itself.
template <int KIND>
__device__ __forceinline__ RayStart ray_setup(const DevGrid &G, const unsigned char *snodes, int n_smem,
                                              const double *__restrict__ o, const double *__restrict__ d,
                                              const double *__restrict__ smax, int64_t r, bool estimate = false,
                                              const float *lat = nullptr) {
    RayStart R;
    R.ik0 = R.ik1 = R.ik2 = 0.0;
    R.ktstart = 0;
    R.cur = -1;
    R.sg = 0;
    R.work = 0.0f;
    R.t1 = 0.0f;
    double oo[3] = {o[3 * r], o[3 * r + 1], o[3 * r + 2]};
    const double kk[3] = {d[3 * r], d[3 * r + 1], d[3 * r + 2]};
    const double tend = smax ? smax[r] : CUDART_INF;
    const bool tend_nan = !dfinite(tend) && (__double_as_longlong(tend) << 12) != 0;
    if (!(dfinite(oo[0]) && dfinite(oo[1]) && dfinite(oo[2]) && dfinite(kk[0]) && dfinite(kk[1]) &&
          dfinite(kk[2])) ||
        (dzero(kk[0]) && dzero(kk[1]) && dzero(kk[2])) || tend_nan) {
        R.sg = HG_RAY_BADINPUT << 8;
        return R;
    }
    // a signed-zero origin coordinate gives the same comparisons and sums as +0
#pragma unroll
    for (int a = 0; a < 3; a++)
        if (dzero(oo[a])) oo[a] = 0.0;
    double ik[3];
    uint32_t sg = 0;
    long long ko[3];
    bool inside = true;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        ik[a] = dzero(kk[a]) ? 0.0 : 1.0 / kk[a];
        sg |= (dgt0(kk[a]) ? 1u : 0u) << a;
        sg |= (dlt0(kk[a]) ? 1u : 0u) << (3 + a);
        ko[a] = okey(oo[a]);
        inside = inside && G.klo[a] < ko[a] && ko[a] < G.khi[a];
    }
    double ts = 0.0;
    long long p[3] = {ko[0], ko[1], ko[2]};
    float t1f;
    if (inside) {
        // entry time 0; the path is empty only when s_max <= 0
        if (!(okey(tend) > 0)) return R;
        float tout = CUDART_INF_F;
#pragma unroll
        for (int a = 0; a < 3; a++)
            if (!dzero(kk[a]))
                tout = fminf(tout, ((dgt0(kk[a]) ? (float)G.dhi[a] : (float)G.dlo[a]) - (float)oo[a]) / (float)kk[a]);
        t1f = fminf(tout, (float)tend);
    } else {
        double tout = CUDART_INF;
        int entry = -1;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            if (dzero(kk[a])) {
                if (ko[a] < G.klo[a] || ko[a] > G.khi[a]) return R;
                continue;
            }
            const double tn = ((dgt0(kk[a]) ? G.dlo[a] : G.dhi[a]) - oo[a]) * ik[a];
            const double tf = ((dgt0(kk[a]) ? G.dhi[a] : G.dlo[a]) - oo[a]) * ik[a];
            if (tn > ts) {
                ts = tn;
                entry = a;
            }
            if (tf < tout) tout = tf;
        }
        if (!(ts < tout) || !(ts < tend)) return R;
        if (entry >= 0) {
#pragma unroll
            for (int a = 0; a < 3; a++) {
                double v;
                if (a == entry) {
                    v = dgt0(kk[a]) ? G.dlo[a] : G.dhi[a];
                } else {
                    v = __fma_rn(kk[a], ts, oo[a]);
                    if (v < G.dlo[a]) v = G.dlo[a];
                    if (v > G.dhi[a]) v = G.dhi[a];
                }
                p[a] = okey(v);
            }
        }
#pragma unroll
        for (int a = 0; a < 3; a++)
            if (!in_axis(p[a], G.klo[a], G.khi[a], dpos(sg, a), dneg(sg, a), true)) return R;
        t1f = (float)(tend < tout ? tend : tout);
    }
    const int32_t c = descend<KIND>(G, snodes, n_smem, p[0], p[1], p[2], sg);
    if (c < 0) {
        R.sg = HG_RAY_LOST << 8;
        return R;
    }
    R.ik0 = ik[0];
    R.ik1 = ik[1];
    R.ik2 = ik[2];
    R.ktstart = okey(ts);
    R.cur = c;
    R.sg = sg;
    R.t1 = t1f;
    if (estimate) {
        const float of[3] = {(float)oo[0], (float)oo[1], (float)oo[2]};
        const float kf[3] = {(float)kk[0], (float)kk[1], (float)kk[2]};
        R.work = work_march(G, lat ? lat : G.work, of, kf, (float)ts, t1f, [](float, float, float, float) {});
    }
    return R;
}

// Take a ray for walking from its start record.  Returns WALK_GO with S
// filled (S.cur = first leaf, not loaded yet), or WALK_END with the setup
// status in *st.
template <bool SEGS>
__device__ __forceinline__ int ray_resume(const double *__restrict__ o, const double *__restrict__ d,
                                          const double *__restrict__ smax, const RayStart *__restrict__ starts,
                                          int64_t r, RayState &S, uint32_t *st) {
    const double2 *q = reinterpret_cast<const double2 *>(starts + r);
    const double2 a = __ldg(q), b = __ldg(q + 1);
    const int4 c = __ldg(reinterpret_cast<const int4 *>(q + 2));
    // c = {cur, sg | status << 8, pad, pad}
    *st = (uint32_t)c.y >> 8;
    if (c.x < 0) return WALK_END;
    if (SEGS && ((uint32_t)c.y & SG_SPLIT)) return WALK_SKIP;  // its segments do the work
    S.ktcur = __double_as_longlong(b.y);
    S.cur = c.x;
    S.sg = (uint32_t)c.y & 0xffu;
    const double oo[3] = {o[3 * r], o[3 * r + 1], o[3 * r + 2]};
    const double kk[3] = {d[3 * r], d[3 * r + 1], d[3 * r + 2]};
    S.set_geometry(oo, kk, a.x, a.y, b.x);
    S.ktend = smax ? okey(smax[r]) : KEY_INF;
    if (SEGS) S.ktstop = KEY_INF;
    S.steps = 0;
    return WALK_GO;
}

// Take a path segment for walking: its start leaf and entry time from the
// segment record, 1/d from the ray's start record.  *ray = the ray it is part
// of.  Returns WALK_END for an empty record (no start leaf).
__device__ __forceinline__ int seg_resume(const double *__restrict__ o, const double *__restrict__ d,
                                           const double *__restrict__ smax, const RayStart *__restrict__ starts,
                                           const SegStart *__restrict__ segs, int64_t s, RayState &S,
                                           int64_t *ray) {
    const longlong2 *q = reinterpret_cast<const longlong2 *>(segs + s);
    const longlong2 a = __ldg(q), b = __ldg(q + 1);
    const int64_t r = b.x;
    *ray = r;
    S.ktcur = a.x;
    S.ktstop = a.y;
    S.cur = (int32_t)(uint32_t)((unsigned long long)b.y & 0xffffffffULL);
    S.sg = (uint32_t)((unsigned long long)b.y >> 32);
    if (S.cur < 0) return WALK_END;
    const double2 *p = reinterpret_cast<const double2 *>(starts + r);
    const double2 i01 = __ldg(p), i2 = __ldg(p + 1);
    const double oo[3] = {o[3 * r], o[3 * r + 1], o[3 * r + 2]};
    const double kk[3] = {d[3 * r], d[3 * r + 1], d[3 * r + 2]};
    S.set_geometry(oo, kk, i01.x, i01.y, i2.x);
    S.ktend = smax ? okey(smax[r]) : KEY_INF;
    S.steps = 0;
    return WALK_GO;
}

// Key of the time to the wall ahead on one axis (KEY_INF when d_a == 0:
// that axis never exits).
__device__ __forceinline__ long long wall_time(bool pos, bool neg, long long lo, long long hi, double o, double ik) {
    if (!(pos || neg)) return KEY_INF;
    return okey((kdouble(pos ? hi : lo) - o) * ik);
}

// Exit-wall test of the current leaf (the step the paper calls the most
// important, Sect. 2.3).  Sets *ds (0: nothing to record) and *ax (-1 when
// the path ends inside the leaf).  Returns WALK_END when the walk stops
// after this leaf's segment (the path ends, leaves the domain, or a path
// segment reaches its stop time), WALK_GO when the next leaf follows.
template <bool SEGS>
__device__ __forceinline__ int ray_exit(int32_t max_steps, RayState &S, const Leaf &L, double *ds, bool *rec,
                                        int *ax_out, double *tex_out, uint32_t *st) {
    *ds = 0.0;
    *rec = false;
    *ax_out = -1;
    if (S.steps >= max_steps) {
        *st = HG_RAY_STEPLIMIT;
        return WALK_END;
    }
    S.steps++;
    const uint32_t sg = S.sg;
    const long long ct0 = wall_time(dpos(sg, 0), dneg(sg, 0), L.lo0, L.hi0, S.o(0), S.ik(0));
    const long long ct1 = wall_time(dpos(sg, 1), dneg(sg, 1), L.lo1, L.hi1, S.o(1), S.ik(1));
    const long long ct2 = wall_time(dpos(sg, 2), dneg(sg, 2), L.lo2, L.hi2, S.o(2), S.ik(2));
    // smallest time, ties to the lower axis; the path end only when strictly smaller
    long long kt = KEY_INF;
    int ax = -1;
    if (ct0 < kt) { kt = ct0; ax = 0; }
    if (ct1 < kt) { kt = ct1; ax = 1; }
    if (ct2 < kt) { kt = ct2; ax = 2; }
    if (S.ktend < kt) { kt = S.ktend; ax = -1; }
    if (kt < S.ktcur) kt = S.ktcur;
    const double tex = kdouble(kt);
    *ds = tex - kdouble(S.ktcur);
    *rec = kt != S.ktcur;  // ds != 0 (equal keys are equal times)
    S.ktcur = kt;
    *ax_out = ax;
    *tex_out = tex;
    if (ax < 0 || (SEGS && kt > S.ktstop)) return WALK_END;
    if (L.first(2 * ax + (dpos(sg, ax) ? 1 : 0)) == -1) return WALK_END;  // exit wall on the domain boundary
    return WALK_GO;
}

// The next record to load and how to treat it.
enum { CAND_ENTER = 0, CAND_TEST = 1, CAND_ROPE = 2 };
struct Cand {
    int32_t id;     // record to load next (CAND_ROPE: the rope's internal node to search below)
    int32_t mode;   // CAND_ENTER: known to contain the exit point; CAND_TEST: a listed neighbor (or a leaf a rope
                    // leads to); CAND_ROPE: no record to load, locate the exit point below node id
    int32_t ax;     // exit axis
    int32_t e;      // next tail entry to try
    int32_t ntail;  // tail entries of the exit wall's list (-1: not read yet)
    uint32_t off;   // where they start (KEEP: the left leaf's nbr_base until they are read)
    int32_t prev;   // the leaf being left
    uint32_t c03, c45;  // KEEP: the left leaf's list lengths, so that a missed head re-reads no record
    long long p1, p2;  // keys of the exit point on the two other axes (b1 < b2)
};

// After an exit through axis ax at time tex: the exit point (the wall on
// the exit axis, o + d t clamped to the leaf on the others) and the first
// neighbor to test, the head of the exit wall's list stored in the leaf --
// or, on a grid loaded with ropes, the wall's rope: a leaf to test, or
// (C.id <= -2) the internal node -2 - C.id to search below (cand_rope).
// KEEP (the interaction search, which has registers to spare at 3 blocks per
// SM): keep the left leaf's list lengths and tail base in the candidate.
template <int NAV, bool KEEP>
__device__ __forceinline__ void cand_first(const RayState &S, const Leaf &L, int ax, double tex, Cand &C) {
    const uint32_t sg = S.sg;
    const int w = 2 * ax + (dpos(sg, ax) ? 1 : 0);
    const int b1 = (ax == 0) ? 1 : 0;
    const int b2 = (ax == 2) ? 1 : 2;
    const double ob1 = S.o(b1), kb1 = S.k(b1);
    const double ob2 = S.o(b2), kb2 = S.k(b2);
    long long p1 = okey(__fma_rn(kb1, tex, ob1));
    long long p2 = okey(__fma_rn(kb2, tex, ob2));
    const long long l1 = L.lo(b1), h1 = L.hi(b1), l2 = L.lo(b2), h2 = L.hi(b2);
    if (p1 < l1) p1 = l1;
    if (p1 > h1) p1 = h1;
    if (p2 < l2) p2 = l2;
    if (p2 > h2) p2 = h2;
    const int32_t f = L.first(w);
    if (NAV == 0) {
        C.id = f;
        C.mode = CAND_TEST;
    } else {
        C.id = f < -1 ? -2 - f : f;
        C.mode = f < -1 ? CAND_ROPE : CAND_TEST;
    }
    C.ax = ax;
    C.e = 0;
    C.ntail = -1;
    C.prev = S.cur;
    if (KEEP) {
        C.off = L.base;
        C.c03 = L.c03;
        C.c45 = L.c45;
    }
    C.p1 = p1;
    C.p2 = p2;
}

// Does the freshly loaded listed neighbor L contain the exit point?  (The
// direction-aware rule on the two other axes; on the exit axis every listed
// neighbor starts at the wall.)
__device__ __forceinline__ bool cand_contains(uint32_t sg, const Leaf &L, const Cand &C) {
    const int b1 = (C.ax == 0) ? 1 : 0;
    const int b2 = (C.ax == 2) ? 1 : 2;
    return in_axis(C.p1, L.lo(b1), L.hi(b1), dpos(sg, b1), dneg(sg, b1), (L.flags() >> b1) & 1u) &&
           in_axis(C.p2, L.lo(b2), L.hi(b2), dpos(sg, b2), dneg(sg, b2), (L.flags() >> b2) & 1u);
}

// Where the rest of the exit wall's list is: read from the leaf being left
// (only needed when the head does not contain the exit point).  A list
// longer than scan_limit keeps a single tail entry, the wall's rope node:
// then C.ntail = -2 and C.off points at it.
template <bool KEEP>
__device__ __forceinline__ void cand_tail_info(const DevGrid &G, uint32_t sg, Cand &C) {
    const int w = 2 * C.ax + (dpos(sg, C.ax) ? 1 : 0);
    uint32_t c03, c45, off;
    if (KEEP) {
        c03 = C.c03;
        c45 = C.c45;
        off = C.off;
    } else {
        const unsigned char *rec = reinterpret_cast<const unsigned char *>(G.rec + C.prev);
        const double2 d = __ldg(reinterpret_cast<const double2 *>(rec + 48));
        const int4 f = __ldg(reinterpret_cast<const int4 *>(rec + 80));
        c03 = (uint32_t)f.z;
        c45 = (uint32_t)f.w;
        off = (uint32_t)((unsigned long long)__double_as_longlong(d.y) >> 32);
    }
    int cw = 0;
    for (int v = 0; v <= w; v++) {
        const int c = v < 4 ? (int)((c03 >> (8 * v)) & 255u) : (int)((c45 >> (8 * (v - 4))) & 255u);
        if (v == w) {
            cw = c;
        } else if (c >= 2) {
            off += c <= G.scan_limit ? (uint32_t)(c - 1) : 1u;
        }
    }
    C.off = off;
    C.ntail = (cw >= 2 && cw <= G.scan_limit) ? cw - 1 : (cw > G.scan_limit ? -2 : 0);
}

// No listed neighbor contains the exit point: an exit point on the domain
// surface with the direction pointing out ends the path (returns true);
// otherwise the caller locates the point top-down.
__device__ __forceinline__ bool cand_leaves_domain(const DevGrid &G, uint32_t sg, const Cand &C) {
    const int b1 = (C.ax == 0) ? 1 : 0;
    const int b2 = (C.ax == 2) ? 1 : 2;
    return !in_axis(C.p1, G.klo[b1], G.khi[b1], dpos(sg, b1), dneg(sg, b1), true) ||
           !in_axis(C.p2, G.klo[b2], G.khi[b2], dpos(sg, b2), dneg(sg, b2), true);
}

// Top-down location of the exit point: the wall on the exit axis (the near
// bound of the listed neighbor L) and the clamped point on the others, from
// the root or from node start.
template <int KIND>
__device__ __forceinline__ int32_t cand_descend(const DevGrid &G, const unsigned char *snodes, int n_smem,
                                                uint32_t sg, const Leaf &L, const Cand &C, int32_t start = 0) {
    const int ax = C.ax;
    const long long wall = dpos(sg, ax) ? L.lo(ax) : L.hi(ax);
    const int b1 = (ax == 0) ? 1 : 0;
    const long long q0 = (ax == 0) ? wall : (b1 == 0 ? C.p1 : C.p2);
    const long long q1 = (ax == 1) ? wall : (b1 == 1 ? C.p1 : C.p2);
    const long long q2 = (ax == 2) ? wall : C.p2;
    return descend<KIND>(G, snodes, n_smem, q0, q1, q2, sg, start);
}

// Rope walk: the leaf below the rope's internal node C.id that holds the
// exit point (on the exit axis the far wall of the leaf being left, whose
// bounds there are lo, hi; the clamped point on the others).  The caller then
// tests that leaf like a listed neighbor.
template <int KIND>
__device__ __forceinline__ int32_t rope_descend(const DevGrid &G, const unsigned char *snodes, int n_smem, uint32_t sg,
                                             long long lo, long long hi, const Cand &C) {
    const int ax = C.ax;
    const long long wall = dpos(sg, ax) ? hi : lo;
    const int b1 = (ax == 0) ? 1 : 0;
    const long long q0 = (ax == 0) ? wall : (b1 == 0 ? C.p1 : C.p2);
    const long long q1 = (ax == 1) ? wall : (b1 == 1 ? C.p1 : C.p2);
    const long long q2 = (ax == 2) ? wall : C.p2;
    return descend<KIND>(G, snodes, n_smem, q0, q1, q2, sg, C.id);
}

// Gradient scatter: a relaxed device-scope reduction (as atomicAdd without a
// result), with an L2 evict-last policy so that the gradient lines stay in
// L2 while the leaf-record gathers stream through it.
__device__ __forceinline__ unsigned long long l2_evict_last_policy() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void red_add_keep(float *a, float v, unsigned long long pol) {
    asm volatile("red.relaxed.gpu.global.add.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(a), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void red_add_keep(double *a, double v, unsigned long long pol) {
    asm volatile("red.relaxed.gpu.global.add.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(a), "d"(v), "l"(pol) : "memory");
}

// Outputs and inputs of one walking launch.
// MODE_TAUADJ: the optical depth and the adjoint scatter in one walk.
// MODE_TAU_STAGE, MODE_TAUADJ_STAGE: the same, also staging every emitted
// (cell, ds) for a gather into the emission arrays once the counts are known.
// MODE_INTERACT: the walk stops where the accumulated optical depth reaches a
// drawn tau_int (the interaction point of the Monte Carlo loop).
enum {
    MODE_TAU = 0,
    MODE_FILL = 1,
    MODE_ADJ = 2,
    MODE_TAUADJ = 3,
    MODE_TAU_STAGE = 4,
    MODE_TAUADJ_STAGE = 5,
    MODE_INTERACT = 6
};

// Emission staging: a pool of chunks of kStageChunk entries (cell, ds);
// each walking thread appends the crossings of the rays and segments it
// walks to its own chain of chunks, taking a new chunk from a global
// counter when one fills.  Entry positions are stored shifted by one chunk
// (position p is entry p - kStageChunk) so that 0 means "no chunk yet".
// An entry keeps its cell beside its length, written with one vector store:
// 16 bytes {ds, cell, unused} after an FP64 walk, 8 bytes {ds, cell} after
// an FP32-Kahan one.  A thread's stores then complete a 32-byte sector
// every two (FP64) or four crossings; with separate cell and length arrays
// a sector of cells took eight, and sectors that L2 evicted half-written
// reached DRAM twice.
constexpr int kStageShift = 7;
constexpr uint32_t kStageChunk = 1u << kStageShift;
__device__ __forceinline__ void stage_put(void *ent, uint32_t e, int32_t c, double ds) {
    reinterpret_cast<int4 *>(ent)[e] = make_int4(__double2loint(ds), __double2hiint(ds), c, 0);
}
__device__ __forceinline__ void stage_put(void *ent, uint32_t e, int32_t c, float ds) {
    reinterpret_cast<int2 *>(ent)[e] = make_int2(__float_as_int(ds), c);
}
__device__ __forceinline__ void stage_get(const void *ent, int64_t e, int32_t &c, double &ds) {
    const int4 v = __ldg(reinterpret_cast<const int4 *>(ent) + e);
    ds = __hiloint2double(v.y, v.x);
    c = v.z;
}
__device__ __forceinline__ void stage_get(const void *ent, int64_t e, int32_t &c, float &ds) {
    const int2 v = __ldg(reinterpret_cast<const int2 *>(ent) + e);
    ds = __int_as_float(v.x);
    c = v.y;
}
struct WalkIO {
    const double *o;
    const double *d;
    const double *smax;
    const RayStart *starts;
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
    // gradient slot of leaf c: (c * gmul) mod 2^32 masked by gmask (identity by default); an odd
    // multiplier scatters spatially close leaves over distinct L2 lines, so that the atomic adds of
    // the many rays crossing a dense region do not queue on a few lines
    uint32_t gmul = 1u, gmask = 0xffffffffu;
    const double *rho_ext;  // densities replacing the grid's own (MODE_TAU), or NULL
    // interaction points (MODE_INTERACT): drawn optical depths in, leaf and path parameter out
    const double *tau_int = nullptr;
    int32_t *int_cell = nullptr;
    double *int_t = nullptr;
    // Path segments: queue items n_rays + s are segment s of a split ray.
    // Each writes its partial results at index s; a combine pass sums them.
    int64_t n_rays = 0x7fffffffffffffffLL;
    const SegStart *segs = nullptr;
    double *part_acc = nullptr;    // partial sum of rho*ds (FP64) or the Kahan sum (FP32K)
    int32_t *part_nc = nullptr;    // partial crossing count
    int32_t *part_last = nullptr;  // leaf the segment stopped in
    uint8_t *part_st = nullptr;    // partial status bits
    const int64_t *seg_base = nullptr;  // emission offset of each segment (MODE_FILL)
    // staging (MODE_*_STAGE)
    void *stg_ent = nullptr;             // staged entries (FP64 or HG_FP32K layout, see stage_put)
    uint32_t *stg_next = nullptr;        // chunk -> next chunk of the same thread
    uint32_t stg_nchunks = 0;
    unsigned long long *stg_ctr = nullptr;
    uint32_t *stg_start_ray = nullptr;   // first entry of each unsplit ray
    uint32_t *stg_start_seg = nullptr;   // first entry of each path segment
    uint32_t *stg_overflow = nullptr;    // set when the pool ran out
};

// The walking loop of one thread.  Each iteration loads exactly one leaf
// record -- the first leaf of a new ray, a listed neighbor to test (the
// head, or the next tail entry after a miss), or the leaf a top-down
// search found -- so a lane that missed the list head costs its warp one
// more iteration instead of a chain of dependent loads inside one.
// Src hands out rays: bool next(int64_t &ray, const DevGrid *&G, int32_t &max_steps);
// when Src::kSegments, an item ray >= io.n_rays is path segment
// ray - io.n_rays of a split ray (otherwise that code is compiled out).
//   PREC (MODE_TAU/MODE_FILL): HG_FP64 or HG_FP32K.
//   PREC (MODE_ADJ): 0 = FP64 gradient atomics, 1 = FP32.
//   PREC (MODE_TAUADJ): bit 0 the optical depth's (HG_FP32K), bit 1 the gradient's (FP32).
//   NAV: 0 the grids hold neighbor lists, 1 ropes, 2 either (read per grid).
// geo: shared memory for the geometry slots, 9 doubles per thread of the block.
template <int KIND, int MODE, int PREC, int NAV, class Src>
__device__ __forceinline__ void walk_loop(Src &src, const WalkIO &io, const unsigned char *snodes, int n_smem,
                                          double *geo) {
    constexpr bool SEGS = Src::kSegments;
    constexpr bool STAGE = (MODE == MODE_TAU_STAGE || MODE == MODE_TAUADJ_STAGE);
    constexpr bool INTER = (MODE == MODE_INTERACT);
    constexpr bool TAU = (MODE == MODE_TAU || MODE == MODE_TAUADJ || STAGE);
    constexpr bool ADJ = (MODE == MODE_ADJ || MODE == MODE_TAUADJ || MODE == MODE_TAUADJ_STAGE);
    constexpr bool TWO = (MODE == MODE_TAUADJ || MODE == MODE_TAUADJ_STAGE);
    constexpr int TPREC = TWO ? (PREC & 1) : (ADJ ? HG_FP64 : PREC);  // HG_FP64 or HG_FP32K
    constexpr int GPREC = TWO ? ((PREC >> 1) & 1) : PREC;             // 0 FP64, 1 FP32 gradient
    const DevGrid *Gp = nullptr;
    int64_t ray = 0;
    int32_t max_steps = 0;
    RayState S;
    S.g = geo + threadIdx.x;
    S.gs = (int)blockDim.x;
    Leaf L;
    Cand C;
    double acc = 0.0;     // FP64 sum of rho*ds
    float acc32 = 0.0f;   // FP32 Kahan sum
    float comp32 = 0.0f;  // Kahan compensation
    int32_t nc = 0;
    int64_t seg_base = 0;
    double wk = 0.0;  // kappa * w for the adjoint
    uint32_t st = 0;
    bool have = false;
    uint32_t sp = 0;  // staging: next entry position (shifted; 0 = no chunk)
    double tint = 0.0, it = 0.0;  // interaction: drawn optical depth; interaction time
    int32_t icell = -1;           // interaction leaf, -1 while none
    bool walked = false;          // the path has a first leaf (its end time is the current time)
    const float kappa32 = (float)io.kappa;
    const unsigned long long keep = ADJ ? l2_evict_last_policy() : 0ULL;
    for (;;) {
        if (!have) {
            if (!src.next(ray, Gp, max_steps)) break;
            acc = 0.0;
            acc32 = 0.0f;
            comp32 = 0.0f;
            nc = 0;
            have = true;
            int64_t r = ray;
            int rs = WALK_GO;
            st = 0;
            if (SEGS && ray >= io.n_rays)
                rs = seg_resume(io.o, io.d, io.smax, io.starts, io.segs, ray - io.n_rays, S, &r);
            else
                rs = ray_resume<SEGS>(io.o, io.d, io.smax, io.starts, ray, S, &st);
            if (rs == WALK_SKIP) {
                have = false;
                continue;
            }
            if (MODE == MODE_FILL) seg_base = (SEGS && ray >= io.n_rays) ? io.seg_base[ray - io.n_rays] : io.seg_off[r];
            if (ADJ) wk = io.kappa * (double)io.w[r];
            if (INTER) {
                tint = io.tau_int[r];
                icell = -1;
                it = 0.0;
                walked = (rs == WALK_GO);
                if (((unsigned long long)__double_as_longlong(tint) << 1) > 0xffe0000000000000ULL) {  // NaN
                    st = HG_RAY_BADINPUT;
                    walked = false;
                    rs = WALK_END;
                }
            }
            if (rs == WALK_END) goto finish;
            C.id = S.cur;
            C.mode = CAND_ENTER;
        }
        {
            const DevGrid &G = *Gp;
            load_leaf(G.rec, C.id, L);
            if (C.mode == CAND_TEST && !cand_contains(S.sg, L, C)) {
                if (C.ntail == -1) cand_tail_info<INTER>(G, S.sg, C);
                if (C.e < C.ntail) {
                    C.id = __ldg(G.tail + C.off + C.e);
                    C.e++;
                    continue;
                }
                if (cand_leaves_domain(G, S.sg, C)) goto finish;
                // edge or corner exit, or a long list: locate the exit point top-down -- for a long list
                // first below the wall's rope node, the leaf found there then tested like a listed
                // neighbor (a point on the face's edge may belong outside the node); else from the root
                int32_t start = 0;
                if (C.ntail == -2) {
                    start = __ldg(G.tail + C.off);
                    C.ntail = 0;
                    if (start < 0) start = 0;
                }
                const int32_t j = cand_descend<KIND>(G, snodes, n_smem, S.sg, L, C, start);
                if (j < 0) {
                    st = HG_RAY_LOST;
                    goto finish;
                }
                C.id = j;
                C.mode = start > 0 ? CAND_TEST : CAND_ENTER;
                continue;
            }
            S.cur = C.id;
            double ds, tex;
            bool rec;
            int ax;
            const long long kin = S.ktcur;  // entry time into this leaf
            const int r = ray_exit<SEGS>(max_steps, S, L, &ds, &rec, &ax, &tex, &st);
            const bool skip = SEGS && (S.sg & SG_SKIP_FIRST) != 0;  // the segment before records this leaf
            if (SEGS) S.sg &= ~SG_SKIP_FIRST;
            if (rec && !skip) {
                if (INTER) {
                    // stop in the first segment after which kappa * S reaches tau_int; inside it tau grows
                    // linearly: t = t_in + (tau_int - kappa S_before) / (kappa rho), at most the exit time
                    const double rho = L.rho;
                    const double s_new = __fma_rn(rho, ds, acc);
                    if (io.kappa * s_new >= tint) {
                        const double a = tint - io.kappa * acc;
                        const double b = io.kappa * rho;
                        const double tin = kdouble(kin);
                        double t = tin;
                        if (a > 0.0 && b > 0.0) t = tin + a / b;
                        if (t > tex) t = tex;
                        icell = S.cur;
                        it = t;
                        nc++;
                        goto finish;
                    }
                    acc = s_new;
                }
                if (TAU) {
                    if (TPREC == HG_FP64) {
                        const double rho = io.rho_ext ? __ldg(io.rho_ext + S.cur) : L.rho;
                        acc = __fma_rn(rho, ds, acc);
                    } else {
                        const float rho32 = io.rho_ext ? __double2float_rn(__ldg(io.rho_ext + S.cur)) : L.rho32;
                        const float kr32 = __fmul_rn(kappa32, rho32);
                        const float y = __fsub_rn(__fmul_rn(kr32, __double2float_rn(ds)), comp32);
                        const float t = __fadd_rn(acc32, y);
                        comp32 = __fsub_rn(__fsub_rn(t, acc32), y);
                        acc32 = t;
                    }
                }
                if (MODE == MODE_FILL) {
                    const int64_t idx = seg_base + nc;
                    if (idx >= io.seg_cap) {
                        st |= HG_RAY_OVERFLOW;
                        goto finish;
                    }
                    io.seg_cell[idx] = S.cur;
                    if (PREC == HG_FP64)
                        static_cast<double *>(io.seg_ds)[idx] = ds;
                    else
                        static_cast<float *>(io.seg_ds)[idx] = __double2float_rn(ds);
                }
                if (STAGE && sp != 0xffffffffu) {
                    if ((sp & (kStageChunk - 1u)) == 0u) {
                        const uint32_t c = (uint32_t)atomicAdd(io.stg_ctr, 1ULL);
                        if (c >= io.stg_nchunks) {
                            sp = 0xffffffffu;  // pool exhausted: the emission falls back to a fill walk
                            *io.stg_overflow = 1u;
                        } else {
                            if (sp != 0u) io.stg_next[((sp - 1u) >> kStageShift) - 1u] = c;
                            sp = (c + 1u) << kStageShift;
                        }
                    }
                    if (sp != 0xffffffffu) {
                        const uint32_t e = sp - kStageChunk;
                        if (nc == 0) {
                            if (SEGS && ray >= io.n_rays)
                                io.stg_start_seg[ray - io.n_rays] = e;
                            else
                                io.stg_start_ray[ray] = e;
                        }
                        if (TPREC == HG_FP64)
                            stage_put(io.stg_ent, e, S.cur, ds);
                        else
                            stage_put(io.stg_ent, e, S.cur, __double2float_rn(ds));
                        sp++;
                    }
                }
                if (ADJ) {
                    const double v = wk * ds;
                    const uint32_t slot = ((uint32_t)S.cur * io.gmul) & io.gmask;
                    if (GPREC == 0)
                        red_add_keep(static_cast<double *>(io.grad) + slot, v, keep);
                    else
                        red_add_keep(static_cast<float *>(io.grad) + slot, __double2float_rn(v), keep);
                }
                nc++;
            }
            if (r == WALK_GO) {
                if (NAV == 0 || (NAV == 2 && G.nav == HG_NAV_NEIGHBOR_LISTS))
                    cand_first<0, INTER>(S, L, ax, tex, C);
                else
                    cand_first<1, INTER>(S, L, ax, tex, C);
                if (NAV != 0 && C.mode == CAND_ROPE) {  // a rope to an internal node: the exit point's leaf below it
                    C.id = rope_descend<KIND>(G, snodes, n_smem, S.sg, L.lo(ax), L.hi(ax), C);
                    C.mode = CAND_TEST;
                    if (C.id < 0) {
                        st = HG_RAY_LOST;
                        goto finish;
                    }
                }
                continue;
            }
        }
    finish:
        if (SEGS && ray >= io.n_rays) {
            const int64_t sidx = ray - io.n_rays;
            if (TAU) {
                io.part_acc[sidx] = (TPREC == HG_FP64) ? acc : (double)acc32;
                io.part_nc[sidx] = nc;
            }
            io.part_last[sidx] = S.cur;
            io.part_st[sidx] = (uint8_t)st;
        } else if (INTER) {
            io.int_cell[ray] = icell;
            io.int_t[ray] = (icell >= 0) ? it : (walked ? kdouble(S.ktcur) : 0.0);
            io.ncross[ray] = nc;
            if (io.status) io.status[ray] = (uint8_t)st;
        } else if (TAU) {
            if (TPREC == HG_FP64)
                static_cast<double *>(io.tau)[ray] = io.kappa * acc;
            else
                static_cast<float *>(io.tau)[ray] = acc32;
            io.ncross[ray] = nc;
            if (io.status) io.status[ray] = (uint8_t)st;
        } else if (MODE == MODE_FILL) {
            if (io.status && st) io.status[ray] |= (uint8_t)st;
        } else {
            if (io.status) io.status[ray] = (uint8_t)st;
        }
        have = false;
    }
}

}  // namespace hg
