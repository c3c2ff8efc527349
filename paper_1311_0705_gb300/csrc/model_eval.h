// Node evaluation of the tree construction (Sect. 2.2, 4.1, 4.2), shared by
// the host builder (build.cpp) and the device builder (gbuild.cu) so that
// both take every decision with the same arithmetic: the analytic density
// models, the node bounds, the counter-based Monte Carlo draws and the three
// subdivision criteria (mass fraction Eq. 1, optical depth Eq. 2, density
// dispersion Eq. 3).  Compiled as plain C++ on the host and as
// __host__ __device__ code by nvcc; the only operations that may round
// differently between the two are the exponentials of the disk and clump
// models (the host's libm against CUDA's exp).
#pragma once

#include <cmath>
#include <cstdint>

#include "hgrt.h"

#ifdef __CUDACC__
#define HG_HD __host__ __device__ __forceinline__
#else
#define HG_HD inline
#endif

namespace hg {

constexpr uint64_t kGamma = 0x9e3779b97f4a7c15ULL;

// SplitMix64 output function (Steele, Lea & Flood 2014).
HG_HD uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// Stream key of a node: the seed and the node's box (levels and indices).
HG_HD uint64_t box_key(uint64_t seed, const int32_t *l, const int64_t *i) {
    uint64_t lv = (uint64_t)l[0] | ((uint64_t)l[1] << 8) | ((uint64_t)l[2] << 16);
    uint64_t k = mix64(seed + kGamma * (1ULL + lv));
    k = mix64(k + kGamma * (1ULL + (uint64_t)i[0]));
    k = mix64(k + kGamma * (1ULL + (uint64_t)i[1]));
    return mix64(k + kGamma * (1ULL + (uint64_t)i[2]));
}

// Draw j of a stream: 53 random bits as a double in [0, 1).
HG_HD double unit_draw(uint64_t key, uint64_t j) { return (double)(mix64(key + kGamma * (j + 1ULL)) >> 11) * 0x1.0p-53; }

// A density model as the builders read it (pointers to host or device
// memory, whichever side evaluates).  G > 0: the clumps of the torus model
// are indexed on a G^3 lattice over the domain, cell c listing (ascending)
// the clumps that can reach it: cell_ids[cell_off[c] .. cell_off[c + 1]).
struct ModelView {
    int32_t kind = 0;
    int32_t n_table = 0;
    double p[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    double m_tot = 0.0;
    const double *table = nullptr;
    int32_t G = 0;
    const int32_t *cell_off = nullptr;
    const int32_t *cell_ids = nullptr;
};

HG_HD double model_rho(const ModelView &m, double x, double y, double z) {
    switch (m.kind) {
    case HG_MODEL_CONST:
        return m.p[0];
    case HG_MODEL_DISK: {
        double R = sqrt(x * x + y * y);
        double e = -(R / m.p[1]) - (fabs(z) / m.p[2]);
        return m.p[0] * exp(e);
    }
    case HG_MODEL_TORUS: {
        double s = sqrt(x * x + y * y) - m.p[0];
        double v = (s * s + z * z < m.p[1] * m.p[1]) ? m.p[2] : 0.0;
        if (m.n_table <= 0) return v;
        double pos[3] = {x, y, z};
        int ix[3];
        for (int a = 0; a < 3; a++) {
            int q = (int)floor((pos[a] - m.lo[a]) / (m.hi[a] - m.lo[a]) * m.G);
            ix[a] = q < 0 ? 0 : (q >= m.G ? m.G - 1 : q);
        }
        int64_t c = (int64_t)ix[0] + (int64_t)m.G * ((int64_t)ix[1] + (int64_t)m.G * ix[2]);
        for (int32_t e = m.cell_off[c]; e < m.cell_off[c + 1]; e++) {
            const double *cl = m.table + 5 * (int64_t)m.cell_ids[e];
            double dx = x - cl[0], dy = y - cl[1], dz = z - cl[2];
            double r2 = dx * dx + dy * dy + dz * dz;
            double s2 = cl[3] * cl[3];
            if (r2 < 25.0 * s2) v += cl[4] * exp(-0.5 * (r2 / s2));
        }
        return v;
    }
    case HG_MODEL_DYADIC: {
        int L = (int)m.p[0];
        int64_t n = (int64_t)1 << L;
        double pos[3] = {x, y, z};
        int64_t ix[3];
        for (int a = 0; a < 3; a++) {
            double f = (pos[a] - m.lo[a]) / (m.hi[a] - m.lo[a]) * (double)n;
            int64_t q = (int64_t)floor(f);
            ix[a] = q < 0 ? 0 : (q > n - 1 ? n - 1 : q);
        }
        return m.table[ix[0] + n * (ix[1] + n * ix[2])];
    }
    }
    return 0.0;
}

// lo + (hi - lo) i / 2^l on axis a, the top end being hi itself.
HG_HD double model_bound(const ModelView &m, int a, int64_t i, int32_t l) {
    if (i == ((int64_t)1 << l)) return m.hi[a];
    return m.lo[a] + (m.hi[a] - m.lo[a]) * ldexp((double)i, -l);
}

struct NodeStats {
    double rho, mass, delta, tau, q;
    int32_t sub;
    int32_t axis;  // k-d trees: the axis a subdivision splits (octrees: -1)
};

// One Monte Carlo draw of a node (position, density, draw number), kept by
// the host builder to place non-centre split planes.
struct Draw {
    double x[3];
    double r;
    int32_t s;
};

// The node with levels l and indices i (depth: its depth in the tree):
// n_ran draws of its box give rho = mean density, M = V rho, delta = M /
// M_tot (Eq. 1), tau = kappa M sqrt(a^2 + b^2 + c^2) / (abc) (Eq. 2) and
// q = (rho_max - rho_min) / rho_max over the draws (Eq. 3); it is
// subdivided when any enabled criterion exceeds its threshold, unless it is
// at the maximum level.  A k-d node splits on the cyclic axis, or with
// HG_AXIS_GRADIENT on the axis of the largest positive
// g_a = |m_hi - m_lo| / (hi_a - lo_a), m_lo / m_hi the mean densities of the
// draws below / at or above the node's midpoint on axis a (ties to the lower
// axis), among the axes halved fewer than max_level times; when none has a
// positive g_a, the first of those in cyclic order.
//
// box_lo / box_hi: the node's box when it is not the dyadic lattice cell of
// (l, i) (trees with non-centre split planes), else NULL.  draws: NULL, or
// room for n_ran draws, which are then recorded.
HG_HD NodeStats eval_node_stats(const ModelView &M, const hg_build_params &P, const int32_t *l, const int64_t *i,
                                int32_t depth, const double *box_lo = nullptr, const double *box_hi = nullptr,
                                Draw *draws = nullptr) {
    double lo[3], hi[3];
    for (int a = 0; a < 3; a++) {
        lo[a] = box_lo ? box_lo[a] : model_bound(M, a, i[a], l[a]);
        hi[a] = box_hi ? box_hi[a] : model_bound(M, a, i[a] + 1, l[a]);
    }
    const uint64_t key = box_key(P.seed, l, i);
    const bool grad = (P.kind == HG_KDTREE && P.split_axis == HG_AXIS_GRADIENT);
    double mid[3] = {0.0, 0.0, 0.0}, s_lo[3] = {0.0, 0.0, 0.0}, s_hi[3] = {0.0, 0.0, 0.0};
    int32_t n_lo[3] = {0, 0, 0};
    if (grad)
        for (int a = 0; a < 3; a++)
            mid[a] = (P.split_plane == HG_PLANE_CENTRE) ? model_bound(M, a, 2 * i[a] + 1, l[a] + 1)
                                                        : lo[a] + 0.5 * (hi[a] - lo[a]);
    double S = 0.0, rmin = 0.0, rmax = 0.0;
    for (int32_t s = 0; s < P.n_ran; s++) {
        double x = lo[0] + unit_draw(key, 3ULL * s) * (hi[0] - lo[0]);
        double y = lo[1] + unit_draw(key, 3ULL * s + 1) * (hi[1] - lo[1]);
        double z = lo[2] + unit_draw(key, 3ULL * s + 2) * (hi[2] - lo[2]);
        double r = model_rho(M, x, y, z);
        if (draws) {
            draws[s].x[0] = x;
            draws[s].x[1] = y;
            draws[s].x[2] = z;
            draws[s].r = r;
            draws[s].s = s;
        }
        S += r;
        if (s == 0 || r < rmin) rmin = r;
        if (s == 0 || r > rmax) rmax = r;
        if (grad) {
            const double pos[3] = {x, y, z};
            for (int a = 0; a < 3; a++) {
                if (pos[a] < mid[a]) {
                    s_lo[a] += r;
                    n_lo[a]++;
                } else {
                    s_hi[a] += r;
                }
            }
        }
    }
    NodeStats st;
    double a = hi[0] - lo[0], b = hi[1] - lo[1], c = hi[2] - lo[2];
    double V = a * b * c;
    st.rho = S / (double)P.n_ran;
    st.mass = V * st.rho;
    st.delta = st.mass / M.m_tot;
    st.tau = P.kappa * st.mass * sqrt(a * a + b * b + c * c) / (a * b * c);
    st.q = (rmax > 0.0) ? (rmax - rmin) / rmax : 0.0;
    bool at_max = (P.kind == HG_OCTREE) ? (l[0] >= P.max_level) : (depth >= 3 * P.max_level);
    bool sub = (P.use_delta && st.delta > P.delta_max) || (P.use_tau && st.tau > P.tau_max) ||
               (P.use_q && st.q > P.q_max);
    st.sub = (sub && !at_max) ? 1 : 0;
    st.axis = -1;
    if (P.kind == HG_KDTREE) {
        const int cyc = (l[0] + l[1] + l[2]) % 3;
        st.axis = cyc;
        if (grad) {
            // every axis is halved at most max_level times (so the depth stays <= 3 max_level): the
            // first such axis in cyclic order, unless an eligible axis has a positive gradient
            for (int k = 0; k < 3; k++)
                if (l[(cyc + k) % 3] < P.max_level) {
                    st.axis = (cyc + k) % 3;
                    break;
                }
            double best = 0.0;
            for (int ax = 0; ax < 3; ax++) {
                const int32_t n_hi = P.n_ran - n_lo[ax];
                if (l[ax] >= P.max_level || n_lo[ax] == 0 || n_hi == 0) continue;
                const double g = fabs(s_hi[ax] / (double)n_hi - s_lo[ax] / (double)n_lo[ax]) / (hi[ax] - lo[ax]);
                if (g > best) {
                    best = g;
                    st.axis = ax;
                }
            }
        }
    }
    return st;
}

}  // namespace hg
