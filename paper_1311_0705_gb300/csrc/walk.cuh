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
// arithmetic contract in hgrt.h states.
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

// Fetch a whole 96-byte record with six 16-byte read-only loads.
__device__ __forceinline__ void load_leaf(const LeafRec *__restrict__ R, int32_t id, Leaf &L) {
    const longlong2 *q = reinterpret_cast<const longlong2 *>(R + id);
    const longlong2 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2);
    const double2 d = __ldg(reinterpret_cast<const double2 *>(q + 3));
    const int4 *qi = reinterpret_cast<const int4 *>(R + id) + 4;
    const int4 e = __ldg(qi), f = __ldg(qi + 1);
    L.lo0 = a.x;
    L.lo1 = a.y;
    L.lo2 = b.x;
    L.hi0 = b.y;
    L.hi1 = c.x;
    L.hi2 = c.y;
    L.rho = d.x;
    const unsigned long long bits = (unsigned long long)__double_as_longlong(d.y);
    L.rho32 = __uint_as_float((uint32_t)(bits & 0xffffffffULL));
    L.base = (uint32_t)(bits >> 32);
    L.f0 = e.x;
    L.f1 = e.y;
    L.f2 = e.z;
    L.f3 = e.w;
    L.f4 = f.x;
    L.f5 = f.y;
    L.c03 = (uint32_t)f.z;
    L.c45 = (uint32_t)f.w;
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

// Top-down descent (Sect. 2.3) on keys.  The first n_smem nodes of the list
// (the top levels, since the list is breadth first) come from shared memory.
// KIND: HG_OCTREE, HG_KDTREE, or 2 = decided at run time from G.kind.
template <int KIND>
__device__ __forceinline__ int32_t descend(const DevGrid &G, const unsigned char *snodes, int n_smem, long long p0,
                                           long long p1, long long p2, uint32_t sg) {
    const bool kd = (KIND == 2) ? (G.kind == HG_KDTREE) : (KIND == HG_KDTREE);
    int32_t nd = 0;
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

// Per-ray walking state.
struct RayState {
    double o0, o1, o2, k0, k1, k2, ik0, ik1, ik2;
    long long ktend;  // key of the path end (KEY_INF: walk to the domain exit)
    long long ktcur;  // key of the current time
    uint32_t sg;      // direction sign bits
    int32_t cur;
    int32_t steps;
};

enum { WALK_GO = 0, WALK_END = 1 };

// Start state of a ray, written by the setup pass and read when a walking
// thread takes the ray: 48 bytes, three 16-byte loads.
struct alignas(16) RayStart {
    double ik0, ik1, ik2;  // 1/d per axis (0 where d_a == 0)
    long long ktstart;     // key of the entry time
    int32_t cur;           // first leaf, or -1 when the ray does not walk
    uint32_t sg;           // direction sign bits | status bits << 8
    int64_t pad;
};
static_assert(sizeof(RayStart) == 48 && offsetof(RayStart, ktstart) == 24 && offsetof(RayStart, cur) == 32 &&
                  offsetof(RayStart, sg) == 36,
              "ray_resume reads the start record as two double2 and one int4");

// Set up a ray (the first-cell location of Sect. 2.3): checks, 1/d, clip
// against the domain, top-down descent to the first leaf.  Runs once per
// ray in its own pass, so it keeps plain FP64 compares.
template <int KIND>
__device__ __forceinline__ RayStart ray_setup(const DevGrid &G, const unsigned char *snodes, int n_smem,
                                              const double *__restrict__ o, const double *__restrict__ d,
                                              const double *__restrict__ smax, int64_t r) {
    RayStart R;
    R.ik0 = R.ik1 = R.ik2 = 0.0;
    R.ktstart = 0;
    R.cur = -1;
    R.sg = 0;
    R.pad = 0;
    double oo[3] = {o[3 * r], o[3 * r + 1], o[3 * r + 2]};
    const double kk[3] = {d[3 * r], d[3 * r + 1], d[3 * r + 2]};
    const double tend = smax ? smax[r] : CUDART_INF;
    if (!(isfinite(oo[0]) && isfinite(oo[1]) && isfinite(oo[2]) && isfinite(kk[0]) && isfinite(kk[1]) &&
          isfinite(kk[2])) ||
        (kk[0] == 0.0 && kk[1] == 0.0 && kk[2] == 0.0) || isnan(tend)) {
        R.sg = HG_RAY_BADINPUT << 8;
        return R;
    }
    // a signed-zero origin coordinate gives the same comparisons and sums as +0
#pragma unroll
    for (int a = 0; a < 3; a++)
        if (oo[a] == 0.0) oo[a] = 0.0;
    double ik[3];
    uint32_t sg = 0;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        ik[a] = (kk[a] != 0.0) ? 1.0 / kk[a] : 0.0;
        sg |= (kk[a] > 0.0 ? 1u : 0u) << a;
        sg |= (kk[a] < 0.0 ? 1u : 0u) << (3 + a);
    }
    double ts = 0.0, tout = CUDART_INF;
    int entry = -1;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        if (kk[a] == 0.0) {
            if (oo[a] < G.dlo[a] || oo[a] > G.dhi[a]) return R;
            continue;
        }
        const double tn = ((kk[a] > 0.0 ? G.dlo[a] : G.dhi[a]) - oo[a]) * ik[a];
        const double tf = ((kk[a] > 0.0 ? G.dhi[a] : G.dlo[a]) - oo[a]) * ik[a];
        if (tn > ts) {
            ts = tn;
            entry = a;
        }
        if (tf < tout) tout = tf;
    }
    if (!(ts < tout) || !(ts < tend)) return R;
    long long p[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        double v;
        if (entry < 0) {
            v = oo[a];
        } else if (a == entry) {
            v = (kk[a] > 0.0) ? G.dlo[a] : G.dhi[a];
        } else {
            v = oo[a] + kk[a] * ts;
            if (v < G.dlo[a]) v = G.dlo[a];
            if (v > G.dhi[a]) v = G.dhi[a];
        }
        p[a] = okey(v);
    }
#pragma unroll
    for (int a = 0; a < 3; a++)
        if (!in_axis(p[a], G.klo[a], G.khi[a], dpos(sg, a), dneg(sg, a), true)) return R;
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
    return R;
}

// Take a ray for walking from its start record.  Returns WALK_GO with S and
// L filled, or WALK_END with the setup status in *st.
__device__ __forceinline__ int ray_resume(const DevGrid &G, const double *__restrict__ o,
                                          const double *__restrict__ d, const double *__restrict__ smax,
                                          const RayStart *__restrict__ starts, int64_t r, RayState &S, Leaf &L,
                                          uint32_t *st) {
    const double2 *q = reinterpret_cast<const double2 *>(starts + r);
    const double2 a = __ldg(q), b = __ldg(q + 1);
    const int4 c = __ldg(reinterpret_cast<const int4 *>(q + 2));
    // c = {cur, sg | status << 8, pad, pad}
    *st = (uint32_t)c.y >> 8;
    if (c.x < 0) return WALK_END;
    S.ik0 = a.x;
    S.ik1 = a.y;
    S.ik2 = b.x;
    S.ktcur = __double_as_longlong(b.y);
    S.cur = c.x;
    S.sg = (uint32_t)c.y & 0xffu;
    double o0 = o[3 * r], o1 = o[3 * r + 1], o2 = o[3 * r + 2];
    S.o0 = (o0 == 0.0) ? 0.0 : o0;
    S.o1 = (o1 == 0.0) ? 0.0 : o1;
    S.o2 = (o2 == 0.0) ? 0.0 : o2;
    S.k0 = d[3 * r];
    S.k1 = d[3 * r + 1];
    S.k2 = d[3 * r + 2];
    S.ktend = smax ? okey(smax[r]) : KEY_INF;
    S.steps = 0;
    load_leaf(G.rec, S.cur, L);
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
// after this leaf's segment, WALK_GO when ray_advance should follow.
__device__ __forceinline__ int ray_exit(int32_t max_steps, RayState &S, const Leaf &L, double *ds, int *ax_out,
                                        double *tex_out, uint32_t *st) {
    *ds = 0.0;
    *ax_out = -1;
    if (S.steps >= max_steps) {
        *st = HG_RAY_STEPLIMIT;
        return WALK_END;
    }
    S.steps++;
    const uint32_t sg = S.sg;
    const long long ct0 = wall_time(dpos(sg, 0), dneg(sg, 0), L.lo0, L.hi0, S.o0, S.ik0);
    const long long ct1 = wall_time(dpos(sg, 1), dneg(sg, 1), L.lo1, L.hi1, S.o1, S.ik1);
    const long long ct2 = wall_time(dpos(sg, 2), dneg(sg, 2), L.lo2, L.hi2, S.o2, S.ik2);
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
    S.ktcur = kt;
    *ax_out = ax;
    *tex_out = tex;
    if (ax < 0) return WALK_END;
    if (L.first(2 * ax + (dpos(sg, ax) ? 1 : 0)) < 0) return WALK_END;  // exit wall on the domain boundary
    return WALK_GO;
}

// Move to the leaf beyond the exit wall: the wall's neighbor list (head
// stored in the leaf), then a top-down search for edge and corner exits
// and long lists.  Returns WALK_GO, or WALK_END when the exit point lies on
// the domain surface with the direction pointing out (or the ray is lost).
template <int KIND>
__device__ __forceinline__ int ray_advance(const DevGrid &G, const unsigned char *snodes, int n_smem, RayState &S,
                                           Leaf &L, int ax, double tex, uint32_t *st) {
    const uint32_t sg = S.sg;
    const bool pax = dpos(sg, ax);
    const int w = 2 * ax + (pax ? 1 : 0);
    const int32_t nxt = L.first(w);
    // exit point: the wall on the exit axis, o + d t clamped to the leaf on the others
    const int b1 = (ax == 0) ? 1 : 0;
    const int b2 = (ax == 2) ? 1 : 2;
    const long long wall = pax ? L.hi(ax) : L.lo(ax);
    long long p1, p2;
    {
        const double ob1 = sel3(b1, S.o0, S.o1, S.o2), kb1 = sel3(b1, S.k0, S.k1, S.k2);
        const double ob2 = sel3(b2, S.o0, S.o1, S.o2), kb2 = sel3(b2, S.k0, S.k1, S.k2);
        p1 = okey(ob1 + kb1 * tex);
        p2 = okey(ob2 + kb2 * tex);
        const long long l1 = L.lo(b1), h1 = L.hi(b1), l2 = L.lo(b2), h2 = L.hi(b2);
        if (p1 < l1) p1 = l1;
        if (p1 > h1) p1 = h1;
        if (p2 < l2) p2 = l2;
        if (p2 > h2) p2 = h2;
    }
    const bool pos1 = dpos(sg, b1), neg1 = dneg(sg, b1), pos2 = dpos(sg, b2), neg2 = dneg(sg, b2);
    // an exit point on the domain surface with the direction pointing out ends the path
    if (!in_axis(p1, G.klo[b1], G.khi[b1], pos1, neg1, true) || !in_axis(p2, G.klo[b2], G.khi[b2], pos2, neg2, true))
        return WALK_END;
    // neighbor-list search.  What is still needed from the current leaf is
    // taken out first; each candidate is then loaded straight into L.
    const int cw = L.cnt(w);
    uint32_t off = L.base;
    for (int v = 0; v < w; v++) {
        const int c = L.cnt(v);
        if (c >= 2 && c <= G.scan_limit) off += (uint32_t)(c - 1);
    }
    const uint32_t ub1 = 1u << b1, ub2 = 1u << b2;
    load_leaf(G.rec, nxt, L);  // the list head is stored in the leaf itself
    if (in_axis(p1, L.lo(b1), L.hi(b1), pos1, neg1, L.flags() & ub1) &&
        in_axis(p2, L.lo(b2), L.hi(b2), pos2, neg2, L.flags() & ub2)) {
        S.cur = nxt;
        return WALK_GO;
    }
    if (cw >= 2 && cw <= G.scan_limit) {
        for (int e = 0; e < cw - 1; e++) {
            const int32_t j = __ldg(G.tail + off + e);
            load_leaf(G.rec, j, L);
            if (in_axis(p1, L.lo(b1), L.hi(b1), pos1, neg1, L.flags() & ub1) &&
                in_axis(p2, L.lo(b2), L.hi(b2), pos2, neg2, L.flags() & ub2)) {
                S.cur = j;
                return WALK_GO;
            }
        }
    }
    // edge or corner exit, or a long list: locate the exit point top-down
    const long long q0 = (ax == 0) ? wall : (b1 == 0 ? p1 : p2);
    const long long q1 = (ax == 1) ? wall : (b1 == 1 ? p1 : p2);
    const long long q2 = (ax == 2) ? wall : p2;
    const int32_t j = descend<KIND>(G, snodes, n_smem, q0, q1, q2, sg);
    if (j < 0) {
        *st = HG_RAY_LOST;
        return WALK_END;
    }
    S.cur = j;
    load_leaf(G.rec, j, L);
    return WALK_GO;
}

}  // namespace hg
