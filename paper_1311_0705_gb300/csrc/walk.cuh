// Device-side path calculation through an octree or k-d tree grid
// (Sect. 2.3): top-down location of the first leaf, then one exit-wall test
// per crossed leaf and the next leaf from that wall's neighbor list.
//
// Every translation unit including this file is compiled with -fmad=false,
// so each FP64 multiply and add below is rounded separately, as the
// arithmetic contract in hgrt.h states.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>

#include "hg_internal.h"

namespace hg {

__device__ __forceinline__ double sel3(int a, double v0, double v1, double v2) {
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

// One leaf record held in registers.
struct Leaf {
    double lo0, lo1, lo2, hi0, hi1, hi2;
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
    __device__ __forceinline__ double lo(int a) const { return sel3(a, lo0, lo1, lo2); }
    __device__ __forceinline__ double hi(int a) const { return sel3(a, hi0, hi1, hi2); }
};

// Fetch a whole 96-byte record with six 16-byte read-only loads.
__device__ __forceinline__ void load_leaf(const LeafRec *__restrict__ R, int32_t id, Leaf &L) {
    const double2 *q = reinterpret_cast<const double2 *>(R + id);
    const double2 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2), d = __ldg(q + 3);
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

// Direction-aware containment on one axis: l < p < h, or p == l with k >= 0,
// or p == h with k < 0, or p == h on the domain's upper face with k == 0.
__device__ __forceinline__ bool in_axis(double p, double l, double h, double k, bool upper_face) {
    return (l < p && p < h) || (p == l && k >= 0.0) || (p == h && (k < 0.0 || (k == 0.0 && upper_face)));
}

__device__ __forceinline__ bool in_domain(const DevGrid &G, double p0, double p1, double p2, double k0, double k1,
                                          double k2) {
    return in_axis(p0, G.dlo[0], G.dhi[0], k0, true) && in_axis(p1, G.dlo[1], G.dhi[1], k1, true) &&
           in_axis(p2, G.dlo[2], G.dhi[2], k2, true);
}

// Top-down descent (Sect. 2.3).  The first n_smem nodes of the list (the top
// levels, since the list is breadth first) are read from shared memory.
// KIND: HG_OCTREE, HG_KDTREE, or 2 = decided at run time from G.kind.
template <int KIND>
__device__ __forceinline__ int32_t descend(const DevGrid &G, const unsigned char *snodes, int n_smem, double p0,
                                           double p1, double p2, double k0, double k1, double k2) {
    const bool kd = (KIND == 2) ? (G.kind == HG_KDTREE) : (KIND == HG_KDTREE);
    int32_t nd = 0;
    for (int it = 0; it <= G.max_depth; it++) {
        if (kd) {
            double2 v;
            if (nd < n_smem)
                v = reinterpret_cast<const double2 *>(snodes)[nd];
            else
                v = __ldg(reinterpret_cast<const double2 *>(G.nodes) + nd);
            const unsigned long long bits = (unsigned long long)__double_as_longlong(v.y);
            const int32_t child = (int32_t)(uint32_t)(bits & 0xffffffffULL);
            const int32_t info = (int32_t)(uint32_t)(bits >> 32);
            if (child < 0) return info;
            const double pa = sel3(info, p0, p1, p2), ka = sel3(info, k0, k1, k2);
            const bool up = (pa > v.x) || (pa == v.x && ka >= 0.0);
            nd = child + (up ? 1 : 0);
        } else {
            double2 v0, v1;
            if (nd < n_smem) {
                v0 = reinterpret_cast<const double2 *>(snodes)[2 * nd];
                v1 = reinterpret_cast<const double2 *>(snodes)[2 * nd + 1];
            } else {
                v0 = __ldg(reinterpret_cast<const double2 *>(G.nodes) + 2 * nd);
                v1 = __ldg(reinterpret_cast<const double2 *>(G.nodes) + 2 * nd + 1);
            }
            const unsigned long long bits = (unsigned long long)__double_as_longlong(v1.y);
            const int32_t child = (int32_t)(uint32_t)(bits & 0xffffffffULL);
            const int32_t leaf = (int32_t)(uint32_t)(bits >> 32);
            if (child < 0) return leaf;
            const int ci = ((p0 > v0.x) || (p0 == v0.x && k0 >= 0.0) ? 1 : 0) |
                           ((p1 > v0.y) || (p1 == v0.y && k1 >= 0.0) ? 2 : 0) |
                           ((p2 > v1.x) || (p2 == v1.x && k2 >= 0.0) ? 4 : 0);
            nd = child + ci;
        }
    }
    return -1;
}

// Per-ray walking state.
struct RayState {
    double o0, o1, o2, k0, k1, k2, ik0, ik1, ik2;
    double tend, tcur;
    int32_t cur;
    int32_t steps;
};

enum { WALK_GO = 0, WALK_END = 1 };

// Set up a ray: checks, clip against the domain, first leaf.  Returns
// WALK_GO with S.cur and L filled, or WALK_END (status in *st).
template <int KIND>
__device__ __forceinline__ int ray_init(const DevGrid &G, const unsigned char *snodes, int n_smem,
                                        const double *__restrict__ o, const double *__restrict__ d,
                                        const double *__restrict__ smax, int64_t r, RayState &S, Leaf &L,
                                        uint32_t *st) {
    *st = 0;
    S.o0 = o[3 * r];
    S.o1 = o[3 * r + 1];
    S.o2 = o[3 * r + 2];
    S.k0 = d[3 * r];
    S.k1 = d[3 * r + 1];
    S.k2 = d[3 * r + 2];
    S.tend = smax ? smax[r] : CUDART_INF;
    if (!(isfinite(S.o0) && isfinite(S.o1) && isfinite(S.o2) && isfinite(S.k0) && isfinite(S.k1) &&
          isfinite(S.k2)) ||
        (S.k0 == 0.0 && S.k1 == 0.0 && S.k2 == 0.0) || isnan(S.tend)) {
        *st = HG_RAY_BADINPUT;
        return WALK_END;
    }
    S.ik0 = (S.k0 != 0.0) ? 1.0 / S.k0 : 0.0;
    S.ik1 = (S.k1 != 0.0) ? 1.0 / S.k1 : 0.0;
    S.ik2 = (S.k2 != 0.0) ? 1.0 / S.k2 : 0.0;
    double ts = 0.0, tout = CUDART_INF;
    int entry = -1;
    const double oo[3] = {S.o0, S.o1, S.o2}, kk[3] = {S.k0, S.k1, S.k2}, ik[3] = {S.ik0, S.ik1, S.ik2};
#pragma unroll
    for (int a = 0; a < 3; a++) {
        if (kk[a] == 0.0) {
            if (oo[a] < G.dlo[a] || oo[a] > G.dhi[a]) return WALK_END;
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
    if (!(ts < tout) || !(ts < S.tend)) return WALK_END;
    double p[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        if (entry < 0) {
            p[a] = oo[a];
        } else if (a == entry) {
            p[a] = (kk[a] > 0.0) ? G.dlo[a] : G.dhi[a];
        } else {
            double v = oo[a] + kk[a] * ts;
            if (v < G.dlo[a]) v = G.dlo[a];
            if (v > G.dhi[a]) v = G.dhi[a];
            p[a] = v;
        }
    }
    if (!in_domain(G, p[0], p[1], p[2], S.k0, S.k1, S.k2)) return WALK_END;
    const int32_t c = descend<KIND>(G, snodes, n_smem, p[0], p[1], p[2], S.k0, S.k1, S.k2);
    if (c < 0) {
        *st = HG_RAY_LOST;
        return WALK_END;
    }
    S.cur = c;
    S.tcur = ts;
    S.steps = 0;
    load_leaf(G.rec, c, L);
    return WALK_GO;
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
    double tex = CUDART_INF;
    int ax = -1;
    if (S.k0 != 0.0) {
        const double t = ((S.k0 > 0.0 ? L.hi0 : L.lo0) - S.o0) * S.ik0;
        if (t < tex) { tex = t; ax = 0; }
    }
    if (S.k1 != 0.0) {
        const double t = ((S.k1 > 0.0 ? L.hi1 : L.lo1) - S.o1) * S.ik1;
        if (t < tex) { tex = t; ax = 1; }
    }
    if (S.k2 != 0.0) {
        const double t = ((S.k2 > 0.0 ? L.hi2 : L.lo2) - S.o2) * S.ik2;
        if (t < tex) { tex = t; ax = 2; }
    }
    if (S.tend < tex) {
        tex = S.tend;
        ax = -1;
    }
    if (tex < S.tcur) tex = S.tcur;
    *ds = tex - S.tcur;
    S.tcur = tex;
    *ax_out = ax;
    *tex_out = tex;
    if (ax < 0) return WALK_END;
    const double kax = sel3(ax, S.k0, S.k1, S.k2);
    if (L.first(2 * ax + (kax > 0.0 ? 1 : 0)) < 0) return WALK_END;  // exit wall on the domain boundary
    return WALK_GO;
}

// Move to the leaf beyond the exit wall: the wall's neighbor list (head
// stored in the leaf), then a top-down search for edge and corner exits
// and long lists.  Returns WALK_GO, or WALK_END when the exit point lies on
// the domain surface with the direction pointing out (or the ray is lost).
template <int KIND>
__device__ __forceinline__ int ray_advance(const DevGrid &G, const unsigned char *snodes, int n_smem, RayState &S,
                                           Leaf &L, int ax, double tex, uint32_t *st) {
    const double kax = sel3(ax, S.k0, S.k1, S.k2);
    const int w = 2 * ax + (kax > 0.0 ? 1 : 0);
    const int32_t nxt = L.first(w);
    // exit point: the wall on the exit axis, clamped o + k t on the others
    const int b1 = (ax == 0) ? 1 : 0;
    const int b2 = (ax == 2) ? 1 : 2;
    const double wall = kax > 0.0 ? L.hi(ax) : L.lo(ax);
    const double ob1 = sel3(b1, S.o0, S.o1, S.o2), kb1 = sel3(b1, S.k0, S.k1, S.k2);
    const double ob2 = sel3(b2, S.o0, S.o1, S.o2), kb2 = sel3(b2, S.k0, S.k1, S.k2);
    double p1 = ob1 + kb1 * tex;
    double p2 = ob2 + kb2 * tex;
    {
        const double l1 = L.lo(b1), h1 = L.hi(b1), l2 = L.lo(b2), h2 = L.hi(b2);
        if (p1 < l1) p1 = l1;
        if (p1 > h1) p1 = h1;
        if (p2 < l2) p2 = l2;
        if (p2 > h2) p2 = h2;
    }
    // an exit point on the domain surface with the direction pointing out ends the path
    if (!in_axis(p1, G.dlo[b1], G.dhi[b1], kb1, true) || !in_axis(p2, G.dlo[b2], G.dhi[b2], kb2, true))
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
    if (in_axis(p1, L.lo(b1), L.hi(b1), kb1, L.flags() & ub1) && in_axis(p2, L.lo(b2), L.hi(b2), kb2, L.flags() & ub2)) {
        S.cur = nxt;
        return WALK_GO;
    }
    if (cw >= 2 && cw <= G.scan_limit) {
        for (int e = 0; e < cw - 1; e++) {
            const int32_t j = __ldg(G.tail + off + e);
            load_leaf(G.rec, j, L);
            if (in_axis(p1, L.lo(b1), L.hi(b1), kb1, L.flags() & ub1) &&
                in_axis(p2, L.lo(b2), L.hi(b2), kb2, L.flags() & ub2)) {
                S.cur = j;
                return WALK_GO;
            }
        }
    }
    // edge or corner exit, or a long list: locate the exit point top-down
    const double q0 = (ax == 0) ? wall : (b1 == 0 ? p1 : p2);
    const double q1 = (ax == 1) ? wall : (b1 == 1 ? p1 : p2);
    const double q2 = (ax == 2) ? wall : p2;
    const int32_t j = descend<KIND>(G, snodes, n_smem, q0, q1, q2, S.k0, S.k1, S.k2);
    if (j < 0) {
        *st = HG_RAY_LOST;
        return WALK_END;
    }
    S.cur = j;
    load_leaf(G.rec, j, L);
    return WALK_GO;
}

}  // namespace hg
