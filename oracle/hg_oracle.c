/*
 * hg_oracle.c -- plain FP64 CPU oracle for octree / k-d tree path calculation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this file's library; the product path
 * never does.  It shares no source, header or helper with the CUDA library.
 *
 * What it computes, each part following the paper (Saftly, Baes & Camps,
 * "Hierarchical octree and k-d tree grids for 3D radiative transfer"):
 *
 *   - the test-model densities rho_t(x) (Sect. 3.1 stand-ins), one plain loop
 *     over all clumps, no spatial index;
 *   - tree construction as one loop over a node list that starts with the
 *     root, children appended at the end, leaves = nodes never subdivided
 *     (Sect. 2.2), with the Monte Carlo node mass of Eq. 1, the mass
 *     fraction criterion delta > delta_max (Sect. 2.2 and 4.1), the node
 *     optical depth of Eq. 2 against tau_max (Sect. 4.1) and the density
 *     dispersion q of Eq. 3 against q_max (Sect. 4.2); octree nodes split
 *     into 8 at the geometric centre or at the barycentre of their draws,
 *     k-d nodes on the cyclic axis x, y, z, x, ... or on the axis of the
 *     strongest density gradient estimated from the node's draws, at the
 *     geometric centre, at the plane that gives both halves equal Monte
 *     Carlo mass, or at the plane that gives them equal mean density
 *     (Sect. 2.2's orientation and location options);
 *   - top-down point location from the root (Sect. 2.3);
 *   - the path calculation: the ordered list of leaves whose interior a
 *     straight path crosses, with segment lengths, and the optical depth
 *     tau = kappa * sum rho ds (Sect. 2.3, 3.2).  The next cell after each
 *     exit is found by top-down relocation from the root after every step
 *     (the traditional method the paper contrasts with neighbor lists,
 *     Sect. 2.3), never by neighbor lists;
 *   - the interaction-point search: the same walk stopped in the leaf where
 *     the accumulated optical depth first reaches a drawn tau_int, with the
 *     time inside it from the linear growth of tau across the leaf (the step
 *     that follows the path in the Monte Carlo loop, Sect. 2.3);
 *   - brute-force references: point location by a linear scan over all
 *     leaves, and the crossed-cell list from every leaf's slab interval;
 *   - the true optical depth along a path by adaptive Gauss-Kronrod
 *     quadrature of rho_t with breakpoints at the model's kinks and edges
 *     (Sect. 3.2, Delta-tau metric).
 *
 * Arithmetic contract (all IEEE binary64, round to nearest, compiled with
 * -ffp-contract=off so that only the explicit fma() calls fuse):
 *   invk_a = 1/k_a for k_a != 0 (a signed zero counts as zero);
 *   in leaf [lo, hi] the wall ahead on axis a is hi_a if k_a > 0 else lo_a,
 *   t_a = (wall_a - o_a) * invk_a; the exit is the smallest t_a, ties to the
 *   lowest axis, the path end wins only when strictly smaller, and the
 *   exit time is raised to the current time if rounding put it behind;
 *   ds = t_exit - t_cur, segments with ds == 0 are skipped;
 *   the point at time t on axis b is fma(k_b, t, o_b) (one rounding); the
 *   exit point is p_a = wall_a on the exit axis and the point at t_exit on
 *   the others, clamped to the leaf's [lo_b, hi_b];
 *   a point p belongs to box [l, h] for direction k iff on every axis
 *   l < p < h, or p == l and k >= 0, or p == h and k < 0 (the domain's
 *   upper face also accepts k == 0); descent takes the upper child iff
 *   p > c or (p == c and k >= 0);
 *   S = fma(rho, ds, S) over the segments, left to right; tau = kappa * S.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OCTREE 0
#define OR_KD 1

#define OR_MODEL_CONST 0
#define OR_MODEL_DISK 1
#define OR_MODEL_TORUS 2
#define OR_MODEL_DYADIC 3

#define OR_RAY_STEPLIMIT 1
#define OR_RAY_LOST 2
#define OR_RAY_BADINPUT 4
#define OR_RAY_OVERFLOW 8

typedef struct {
    int32_t kind;
    int32_t n_table;
    double p[8];
    const double *table; /* torus: [n][5] cx, cy, cz, sigma, A; dyadic: [8^L] */
    double m_tot;
    double lo[3], hi[3];
} or_model;

typedef struct {
    int32_t kind;
    int32_t use_delta, use_tau, use_q;
    double delta_max, tau_max, q_max, kappa;
    int32_t max_level, n_ran;
    uint64_t seed;
    int64_t max_nodes;
    int32_t split_axis; /* k-d: 0 cyclic, 1 strongest density gradient */
    int32_t split_plane; /* 0 geometric centre; octree 1 barycentre; k-d 2 equal mass, 3 equal mean density */
} or_params;

typedef struct {
    int32_t kind;
    int64_t n_nodes, n_leaves, cap;
    int32_t *lvl;     /* [3n] per-axis subdivision level */
    int64_t *idx;     /* [3n] per-axis integer position at that level */
    int32_t *child;   /* [n] first child in the list, -1 for a leaf */
    int32_t *leaf;    /* [n] leaf id, -1 for an internal node */
    double *lo, *hi;  /* [3n] node boxes, node-major */
    double *rho;      /* [n] mean sampled density of the node */
    double *mass;     /* [n] Monte Carlo mass (Eq. 1) */
    double *delta, *taun, *q; /* [n] criterion values */
    int64_t *leaf_node; /* [n_leaves] */
} or_tree;

/* ------------------------------------------------------------------ SplitMix64
 * Steele, Lea & Flood (2014), "Fast splittable pseudorandom number
 * generators": state advances by the golden-ratio increment, each output is
 * the state passed through the 64-bit finaliser below.  Used as a counter
 * generator: output j of the stream with key K is mix(K + (j+1)*GAMMA). */
#define OR_GAMMA 0x9e3779b97f4a7c15ULL

static uint64_t or_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static uint64_t or_node_key(uint64_t seed, const int32_t l[3], const int64_t i[3])
{
    uint64_t k = seed;
    uint64_t lv = (uint64_t)l[0] | ((uint64_t)l[1] << 8) | ((uint64_t)l[2] << 16);
    k = or_mix64(k + OR_GAMMA * (1ULL + lv));
    k = or_mix64(k + OR_GAMMA * (1ULL + (uint64_t)i[0]));
    k = or_mix64(k + OR_GAMMA * (1ULL + (uint64_t)i[1]));
    k = or_mix64(k + OR_GAMMA * (1ULL + (uint64_t)i[2]));
    return k;
}

static double or_uniform(uint64_t key, uint64_t j)
{
    return (double)(or_mix64(key + OR_GAMMA * (j + 1ULL)) >> 11) * 0x1.0p-53;
}

uint64_t or_splitmix_output(uint64_t key, uint64_t j) { return or_mix64(key + OR_GAMMA * (j + 1ULL)); }

/* ------------------------------------------------------------------ models */

double or_rho_true(const or_model *m, double x, double y, double z)
{
    switch (m->kind) {
    case OR_MODEL_CONST:
        return m->p[0];
    case OR_MODEL_DISK: {
        double R = sqrt(x * x + y * y);
        double e = -(R / m->p[1]) - (fabs(z) / m->p[2]);
        return m->p[0] * exp(e);
    }
    case OR_MODEL_TORUS: {
        double s = sqrt(x * x + y * y) - m->p[0];
        double v = (s * s + z * z < m->p[1] * m->p[1]) ? m->p[2] : 0.0;
        for (int32_t j = 0; j < m->n_table; j++) {
            const double *c = m->table + 5 * (int64_t)j;
            double dx = x - c[0], dy = y - c[1], dz = z - c[2];
            double r2 = dx * dx + dy * dy + dz * dz;
            double s2 = c[3] * c[3];
            if (r2 < 25.0 * s2) v += c[4] * exp(-0.5 * (r2 / s2));
        }
        return v;
    }
    case OR_MODEL_DYADIC: {
        int L = (int)m->p[0];
        int64_t n = (int64_t)1 << L;
        double pos[3] = {x, y, z};
        int64_t ix[3];
        for (int a = 0; a < 3; a++) {
            double f = (pos[a] - m->lo[a]) / (m->hi[a] - m->lo[a]) * (double)n;
            int64_t q = (int64_t)floor(f);
            if (q < 0) q = 0;
            if (q > n - 1) q = n - 1;
            ix[a] = q;
        }
        return m->table[ix[0] + n * (ix[1] + n * ix[2])];
    }
    }
    return 0.0;
}

void or_rho_true_batch(const or_model *m, int64_t n, const double *pts, double *out)
{
    for (int64_t i = 0; i < n; i++) out[i] = or_rho_true(m, pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
}

/* ------------------------------------------------------------------ tree construction */

/* Bound at integer position i of level l on axis a: the dyadic point
 * lo + (hi - lo) * i / 2^l, with the top end taken as hi itself. */
static double or_bound(const or_model *m, int a, int64_t i, int32_t l)
{
    if (i == ((int64_t)1 << l)) return m->hi[a];
    return m->lo[a] + (m->hi[a] - m->lo[a]) * ldexp((double)i, -l);
}

typedef struct {
    double rho_mean, mass, delta, tau, q;
    int subdivide;
    int axis;        /* k-d: the axis a subdivision splits */
    double plane[3]; /* where the planes cut: octree all three axes, k-d the split axis */
} or_stats;

#define OR_PLANE_CENTRE 0
#define OR_PLANE_BARYCENTRE 1
#define OR_PLANE_EQUAL_MASS 2
#define OR_PLANE_EQUAL_DENSITY 3

/* One Monte Carlo draw of a node: its position and density. */
typedef struct {
    double x[3];
    double r;
    int32_t s; /* draw number */
} or_draw;

static int or_draw_axis; /* axis the comparison below orders by (set before each qsort) */

static int or_cmp_draw(const void *pa, const void *pb)
{
    const or_draw *a = (const or_draw *)pa, *b = (const or_draw *)pb;
    double u = a->x[or_draw_axis], v = b->x[or_draw_axis];
    if (u < v) return -1;
    if (u > v) return 1;
    return (a->s > b->s) - (a->s < b->s);
}

/* The geometric centre of [lo, hi] on one axis of a node whose box is not a
 * dyadic lattice cell. */
static double or_centre(double lo, double hi) { return lo + 0.5 * (hi - lo); }

/* Barycentric octree subdivision (Sect. 2.2, after the earlier octree paper):
 * the three planes pass through the node's centre of mass, estimated from
 * its draws as sum(rho x) / sum(rho), both sums in draw order.  An axis whose
 * estimate is undefined (no mass) or not strictly inside the node is cut at
 * the geometric centre. */
static void or_barycentre(const or_draw *d, int32_t n, const double lo[3], const double hi[3], double c[3])
{
    double S = 0.0, Sx[3] = {0.0, 0.0, 0.0};
    for (int32_t s = 0; s < n; s++) {
        S += d[s].r;
        for (int a = 0; a < 3; a++) Sx[a] += d[s].r * d[s].x[a];
    }
    for (int a = 0; a < 3; a++) {
        double v = (S > 0.0) ? Sx[a] / S : or_centre(lo[a], hi[a]);
        if (!(lo[a] < v && v < hi[a])) v = or_centre(lo[a], hi[a]);
        c[a] = v;
    }
}

/* k-d split location on axis a (Sect. 2.2).  The draws are ordered by their
 * coordinate on a (ties by draw number); a plane between consecutive draws
 * j and j+1 sits at x_j + (x_{j+1} - x_j) / 2.
 *   equal mass: the first j at which the running sum of densities, left to
 *     right, reaches half the total (2 C_j >= C_total), but never the last
 *     draw -- the two sides then carry as equal Monte Carlo masses as the
 *     draws allow;
 *   equal mean density: the j minimising |C_j / (j+1) - R_j / (n-1-j)|, the
 *     mean draw density left of the plane against right of it (R_j summed
 *     right to left), over the j whose two draws differ in position; ties
 *     go to the j nearest the middle (smallest |2j - (n-2)|), then the
 *     smaller j.
 * No usable draw pair, no mass (equal mass), or a plane not strictly inside
 * the node: the geometric centre. */
static double or_kd_plane(int mode, or_draw *d, int32_t n, int a, double lo, double hi)
{
    double fallback = or_centre(lo, hi);
    if (n < 2) return fallback;
    or_draw_axis = a;
    qsort(d, (size_t)n, sizeof(or_draw), or_cmp_draw);
    int32_t best = -1;
    if (mode == OR_PLANE_EQUAL_MASS) {
        double total = 0.0;
        for (int32_t j = 0; j < n; j++) total += d[j].r;
        if (!(total > 0.0)) return fallback;
        double c = 0.0;
        for (int32_t j = 0; j < n; j++) {
            c += d[j].r;
            if (2.0 * c >= total) { best = j; break; }
        }
        if (best == n - 1) best = n - 2;
        if (best < 0 || !(d[best].x[a] < d[best + 1].x[a])) return fallback;
    } else {
        double *right = malloc((size_t)n * sizeof(double));
        if (!right) return fallback;
        double r = 0.0;
        for (int32_t j = n - 1; j >= 1; j--) {
            r += d[j].r;
            right[j - 1] = r; /* sum of draws j .. n-1: the right side of plane j-1 */
        }
        double c = 0.0, best_d = 0.0;
        int32_t best_mid = 0;
        for (int32_t j = 0; j <= n - 2; j++) {
            c += d[j].r;
            if (!(d[j].x[a] < d[j + 1].x[a])) continue;
            double diff = fabs(c / (double)(j + 1) - right[j] / (double)(n - 1 - j));
            int32_t mid = abs(2 * j - (n - 2));
            if (best < 0 || diff < best_d || (diff == best_d && mid < best_mid)) {
                best = j;
                best_d = diff;
                best_mid = mid;
            }
        }
        free(right);
        if (best < 0) return fallback;
    }
    double v = d[best].x[a] + 0.5 * (d[best + 1].x[a] - d[best].x[a]);
    return (lo < v && v < hi) ? v : fallback;
}


/* The k-d split axis.  Cyclic: x, y, z, x, ... by depth (Sect. 2.2).
 * Gradient (the paper's alternative orientation, Sect. 2.2): the axis with
 * the strongest density gradient in the node, read from its draws: on axis
 * a, m_lo and m_hi are the mean densities of the draws below and at or
 * above the node's midpoint, g_a = |m_hi - m_lo| / (width on a), 0 when a
 * half holds no draw.  Only axes halved fewer than max_level times compete
 * (no axis finer than the octree-equivalent level); the largest positive
 * g_a wins, the lower axis on ties; if none is positive, the first
 * competing axis counting cyclically from depth mod 3. */
static int or_split_axis(const or_params *P, const int32_t l[3], int32_t depth, const double g[3],
                         const int has_both[3])
{
    int first = depth % 3;
    if (P->split_axis == 0) return first;
    int ax = first;
    for (int k = 0; k < 3; k++) {
        int b = (first + k) % 3;
        if (l[b] < P->max_level) { ax = b; break; }
    }
    double best = 0.0;
    for (int b = 0; b < 3; b++) {
        if (l[b] >= P->max_level || !has_both[b]) continue;
        if (g[b] > best) { best = g[b]; ax = b; }
    }
    return ax;
}

/* Sample a node (box [lo, hi], per-axis levels l and positions i, which key
 * its draws), evaluate Eq. 1-3 and the stopping criteria, and for a node to
 * subdivide the split axis (k-d) and plane position(s). */
static or_stats or_node_eval(const or_model *m, const or_params *P, const int32_t l[3], const int64_t i[3],
                             int32_t depth, const double lo[3], const double hi[3])
{
    or_stats st;
    uint64_t key = or_node_key(P->seed, l, i);
    double S = 0.0, rmin = 0.0, rmax = 0.0;
    /* per axis: the sums of the draws' densities below and at or above the midpoint */
    double half_mid[3], sum_below[3] = {0.0, 0.0, 0.0}, sum_above[3] = {0.0, 0.0, 0.0};
    int32_t cnt_below[3] = {0, 0, 0};
    for (int a = 0; a < 3; a++)
        half_mid[a] = (P->split_plane == OR_PLANE_CENTRE) ? or_bound(m, a, 2 * i[a] + 1, l[a] + 1)
                                                          : or_centre(lo[a], hi[a]);
    or_draw *draws = NULL;
    if (P->split_plane != OR_PLANE_CENTRE) draws = malloc((size_t)P->n_ran * sizeof(or_draw));
    for (int32_t s = 0; s < P->n_ran; s++) {
        double x = lo[0] + or_uniform(key, 3ULL * s) * (hi[0] - lo[0]);
        double y = lo[1] + or_uniform(key, 3ULL * s + 1) * (hi[1] - lo[1]);
        double z = lo[2] + or_uniform(key, 3ULL * s + 2) * (hi[2] - lo[2]);
        double r = or_rho_true(m, x, y, z);
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
        double xyz[3] = {x, y, z};
        for (int a = 0; a < 3; a++) {
            if (xyz[a] < half_mid[a]) { sum_below[a] += r; cnt_below[a]++; }
            else sum_above[a] += r;
        }
    }
    double a = hi[0] - lo[0], b = hi[1] - lo[1], c = hi[2] - lo[2];
    double V = a * b * c;
    st.rho_mean = S / (double)P->n_ran;
    st.mass = V * st.rho_mean;                                      /* Eq. 1 */
    st.delta = st.mass / m->m_tot;                                  /* Sect. 2.2 */
    st.tau = P->kappa * st.mass * sqrt(a * a + b * b + c * c) / (a * b * c); /* Eq. 2 */
    st.q = (rmax > 0.0) ? (rmax - rmin) / rmax : 0.0;               /* Eq. 3 */
    int at_max = (P->kind == OR_OCTREE) ? (l[0] >= P->max_level) : (depth >= 3 * P->max_level);
    int sub = 0;
    if (P->use_delta && st.delta > P->delta_max) sub = 1;
    if (P->use_tau && st.tau > P->tau_max) sub = 1;
    if (P->use_q && st.q > P->q_max) sub = 1;
    st.subdivide = at_max ? 0 : sub;
    double g[3];
    int has_both[3];
    for (int a = 0; a < 3; a++) {
        int32_t above = P->n_ran - cnt_below[a];
        has_both[a] = cnt_below[a] > 0 && above > 0;
        g[a] = has_both[a] ? fabs(sum_above[a] / (double)above - sum_below[a] / (double)cnt_below[a]) / (hi[a] - lo[a])
                           : 0.0;
    }
    st.axis = (P->kind == OR_OCTREE) ? -1 : or_split_axis(P, l, depth, g, has_both);
    for (int a = 0; a < 3; a++) st.plane[a] = or_bound(m, a, 2 * i[a] + 1, l[a] + 1);
    if (P->split_plane != OR_PLANE_CENTRE) {
        for (int a = 0; a < 3; a++) st.plane[a] = or_centre(lo[a], hi[a]);
        if (draws && st.subdivide) {
            if (P->kind == OR_OCTREE)
                or_barycentre(draws, P->n_ran, lo, hi, st.plane);
            else
                st.plane[st.axis] = or_kd_plane(P->split_plane, draws, P->n_ran, st.axis, lo[st.axis], hi[st.axis]);
        }
        /* a box too thin to hold a plane strictly inside on a cut axis stays a leaf */
        for (int a = 0; a < 3; a++) {
            if (P->kind == OR_KD && a != st.axis) continue;
            if (!(lo[a] < st.plane[a] && st.plane[a] < hi[a])) st.subdivide = 0;
        }
    }
    free(draws);
    return st;
}

/* Exposed for sampled checks of large grids: evaluate one node by its
 * per-axis levels and positions.  out = {subdivide, rho, mass, delta, tau, q}. */
void or_node_stats(const or_model *m, const or_params *P, const int32_t *l, const int64_t *i, double *out)
{
    int32_t depth = l[0] + l[1] + l[2];
    if (P->kind == OR_OCTREE) depth = l[0];
    double lo[3], hi[3];
    for (int a = 0; a < 3; a++) {
        lo[a] = or_bound(m, a, i[a], l[a]);
        hi[a] = or_bound(m, a, i[a] + 1, l[a]);
    }
    or_stats st = or_node_eval(m, P, l, i, depth, lo, hi);
    out[0] = st.subdivide;
    out[1] = st.rho_mean;
    out[2] = st.mass;
    out[3] = st.delta;
    out[4] = st.tau;
    out[5] = st.q;
}

static int or_tree_reserve(or_tree *T, int64_t need)
{
    if (need <= T->cap) return 0;
    int64_t cap = T->cap ? T->cap : 1024;
    while (cap < need) cap *= 2;
#define OR_GROW(ptr, per)                                                         \
    do {                                                                          \
        void *np_ = realloc((ptr), (size_t)cap * (per) * sizeof(*(ptr)));          \
        if (!np_) return -1;                                                      \
        (ptr) = np_;                                                              \
    } while (0)
    OR_GROW(T->lvl, 3);
    OR_GROW(T->idx, 3);
    OR_GROW(T->child, 1);
    OR_GROW(T->leaf, 1);
    OR_GROW(T->lo, 3);
    OR_GROW(T->hi, 3);
    OR_GROW(T->rho, 1);
    OR_GROW(T->mass, 1);
    OR_GROW(T->delta, 1);
    OR_GROW(T->taun, 1);
    OR_GROW(T->q, 1);
#undef OR_GROW
    T->cap = cap;
    return 0;
}

/* Append a node: per-axis levels and positions, and its box (NULL: the
 * dyadic lattice cell those give). */
static void or_push(or_tree *T, const or_model *m, const int32_t l[3], const int64_t i[3], const double *lo,
                    const double *hi)
{
    int64_t n = T->n_nodes++;
    for (int a = 0; a < 3; a++) {
        T->lvl[3 * n + a] = l[a];
        T->idx[3 * n + a] = i[a];
        T->lo[3 * n + a] = lo ? lo[a] : or_bound(m, a, i[a], l[a]);
        T->hi[3 * n + a] = hi ? hi[a] : or_bound(m, a, i[a] + 1, l[a]);
    }
    T->child[n] = -1;
    T->leaf[n] = -1;
}

void or_tree_free(or_tree *T)
{
    if (!T) return;
    free(T->lvl); free(T->idx); free(T->child); free(T->leaf); free(T->lo); free(T->hi);
    free(T->rho); free(T->mass); free(T->delta); free(T->taun); free(T->q); free(T->leaf_node);
    free(T);
}

/* Build the node list.  Returns 0 on success, -1 on allocation failure,
 * -2 when max_nodes would be exceeded, -3 on bad parameters. */
int or_build(const or_model *m, const or_params *P, or_tree **out)
{
    *out = NULL;
    if (P->n_ran < 1 || !(m->m_tot > 0.0) || P->max_level < 0 || P->max_level > 20) return -3;
    if (P->split_plane < 0 || P->split_plane > 3) return -3;
    if (P->kind == OR_OCTREE && P->split_plane > OR_PLANE_BARYCENTRE) return -3;
    if (P->kind == OR_KD && P->split_plane == OR_PLANE_BARYCENTRE) return -3;
    or_tree *T = calloc(1, sizeof(or_tree));
    if (!T) return -1;
    T->kind = P->kind;
    if (or_tree_reserve(T, 1)) { or_tree_free(T); return -1; }
    int32_t l0[3] = {0, 0, 0};
    int64_t i0[3] = {0, 0, 0};
    or_push(T, m, l0, i0, NULL, NULL);
    for (int64_t n = 0; n < T->n_nodes; n++) {
        int32_t l[3] = {T->lvl[3 * n], T->lvl[3 * n + 1], T->lvl[3 * n + 2]};
        int64_t i[3] = {T->idx[3 * n], T->idx[3 * n + 1], T->idx[3 * n + 2]};
        double lo[3] = {T->lo[3 * n], T->lo[3 * n + 1], T->lo[3 * n + 2]};
        double hi[3] = {T->hi[3 * n], T->hi[3 * n + 1], T->hi[3 * n + 2]};
        int32_t depth = (T->kind == OR_OCTREE) ? l[0] : l[0] + l[1] + l[2];
        or_stats st = or_node_eval(m, P, l, i, depth, lo, hi);
        T->rho[n] = st.rho_mean;
        T->mass[n] = st.mass;
        T->delta[n] = st.delta;
        T->taun[n] = st.tau;
        T->q[n] = st.q;
        if (!st.subdivide) continue;
        int nch = (T->kind == OR_OCTREE) ? 8 : 2;
        if (P->max_nodes > 0 && T->n_nodes + nch > P->max_nodes) { or_tree_free(T); return -2; }
        if (or_tree_reserve(T, T->n_nodes + nch)) { or_tree_free(T); return -1; }
        T->child[n] = (int32_t)T->n_nodes;
        for (int c = 0; c < nch; c++) {
            int32_t lc[3] = {l[0], l[1], l[2]};
            int64_t ic[3] = {i[0], i[1], i[2]};
            double clo[3] = {lo[0], lo[1], lo[2]}, chi[3] = {hi[0], hi[1], hi[2]};
            for (int a = 0; a < 3; a++) {
                if (T->kind == OR_KD && a != st.axis) continue;
                int up = (T->kind == OR_OCTREE) ? ((c >> a) & 1) : c;
                lc[a] = l[a] + 1;
                ic[a] = 2 * i[a] + up;
                if (up)
                    clo[a] = st.plane[a];
                else
                    chi[a] = st.plane[a];
            }
            /* centre planes: the child's dyadic cell (the same values, from its levels and positions) */
            if (P->split_plane == OR_PLANE_CENTRE)
                or_push(T, m, lc, ic, NULL, NULL);
            else
                or_push(T, m, lc, ic, clo, chi);
        }
    }
    /* leaves in list order */
    int64_t nl = 0;
    for (int64_t n = 0; n < T->n_nodes; n++)
        if (T->child[n] < 0) nl++;
    T->leaf_node = malloc((size_t)(nl ? nl : 1) * sizeof(int64_t));
    if (!T->leaf_node) { or_tree_free(T); return -1; }
    nl = 0;
    for (int64_t n = 0; n < T->n_nodes; n++)
        if (T->child[n] < 0) { T->leaf[n] = (int32_t)nl; T->leaf_node[nl++] = n; }
    T->n_leaves = nl;
    *out = T;
    return 0;
}

/* Wrap an externally built tree (node boxes node-major, first-child links,
 * leaf ids and leaf densities) so that the traversal below can run on it. */
int or_tree_wrap(int32_t kind, int64_t n_nodes, const double *lo, const double *hi, const int32_t *child,
                 const int32_t *leaf, int64_t n_leaves, const double *leaf_rho, or_tree **out)
{
    *out = NULL;
    or_tree *T = calloc(1, sizeof(or_tree));
    if (!T) return -1;
    T->kind = kind;
    if (or_tree_reserve(T, n_nodes)) { or_tree_free(T); return -1; }
    T->n_nodes = n_nodes;
    T->n_leaves = n_leaves;
    memcpy(T->lo, lo, (size_t)n_nodes * 3 * sizeof(double));
    memcpy(T->hi, hi, (size_t)n_nodes * 3 * sizeof(double));
    memcpy(T->child, child, (size_t)n_nodes * sizeof(int32_t));
    memcpy(T->leaf, leaf, (size_t)n_nodes * sizeof(int32_t));
    memset(T->lvl, 0, (size_t)n_nodes * 3 * sizeof(int32_t));
    memset(T->idx, 0, (size_t)n_nodes * 3 * sizeof(int64_t));
    T->leaf_node = malloc((size_t)(n_leaves ? n_leaves : 1) * sizeof(int64_t));
    if (!T->leaf_node) { or_tree_free(T); return -1; }
    for (int64_t n = 0; n < n_nodes; n++) {
        T->rho[n] = 0.0;
        if (leaf[n] >= 0) {
            if (leaf[n] >= n_leaves) { or_tree_free(T); return -3; }
            T->leaf_node[leaf[n]] = n;
            T->rho[n] = leaf_rho[leaf[n]];
        }
    }
    *out = T;
    return 0;
}

int64_t or_tree_n_nodes(const or_tree *T) { return T->n_nodes; }
int64_t or_tree_n_leaves(const or_tree *T) { return T->n_leaves; }

/* Copy the tree out: node arrays [n_nodes] (boxes [3n]) and leaf arrays [n_leaves]. */
void or_tree_export(const or_tree *T, int32_t *lvl, int64_t *idx, int32_t *child, int32_t *leaf, double *lo,
                    double *hi, double *rho, double *mass, double *delta, double *taun, double *q,
                    int64_t *leaf_node)
{
    int64_t n = T->n_nodes;
    if (lvl) memcpy(lvl, T->lvl, (size_t)n * 3 * sizeof(int32_t));
    if (idx) memcpy(idx, T->idx, (size_t)n * 3 * sizeof(int64_t));
    if (child) memcpy(child, T->child, (size_t)n * sizeof(int32_t));
    if (leaf) memcpy(leaf, T->leaf, (size_t)n * sizeof(int32_t));
    if (lo) memcpy(lo, T->lo, (size_t)n * 3 * sizeof(double));
    if (hi) memcpy(hi, T->hi, (size_t)n * 3 * sizeof(double));
    if (rho) memcpy(rho, T->rho, (size_t)n * sizeof(double));
    if (mass) memcpy(mass, T->mass, (size_t)n * sizeof(double));
    if (delta) memcpy(delta, T->delta, (size_t)n * sizeof(double));
    if (taun) memcpy(taun, T->taun, (size_t)n * sizeof(double));
    if (q) memcpy(q, T->q, (size_t)n * sizeof(double));
    if (leaf_node) memcpy(leaf_node, T->leaf_node, (size_t)T->n_leaves * sizeof(int64_t));
}

/* ------------------------------------------------------------------ point location */

static int or_in_box(const double *l, const double *h, const double *p, const double *k, const double *dlo,
                     const double *dhi)
{
    for (int a = 0; a < 3; a++) {
        int ok = (l[a] < p[a] && p[a] < h[a]) || (p[a] == l[a] && k[a] >= 0.0) || (p[a] == h[a] && k[a] < 0.0) ||
                 (p[a] == h[a] && k[a] == 0.0 && h[a] == dhi[a]);
        (void)dlo;
        if (!ok) return 0;
    }
    return 1;
}

/* Top-down descent from the root (Sect. 2.3).  Returns the leaf id or -1. */
int64_t or_locate(const or_tree *T, const double *p, const double *k)
{
    const double *dlo = T->lo, *dhi = T->hi;
    if (!or_in_box(dlo, dhi, p, k, dlo, dhi)) return -1;
    int64_t n = 0;
    while (T->child[n] >= 0) {
        int64_t f = T->child[n];
        if (T->kind == OR_KD) {
            int a = 0;
            while (a < 3 && T->hi[3 * f + a] == T->hi[3 * n + a]) a++;
            if (a == 3) return -1; /* malformed */
            double c = T->hi[3 * f + a];
            int up = (p[a] > c) || (p[a] == c && k[a] >= 0.0);
            n = f + up;
        } else {
            int ci = 0;
            for (int a = 0; a < 3; a++) {
                double c = T->hi[3 * f + a];
                int up = (p[a] > c) || (p[a] == c && k[a] >= 0.0);
                ci |= up << a;
            }
            n = f + ci;
        }
    }
    return T->leaf[n];
}

/* Linear scan over all leaves with the same containment rule; returns the
 * number of leaves that contain p and the last one found in *which. */
int64_t or_brute_locate(const or_tree *T, const double *p, const double *k, int64_t *which)
{
    int64_t hits = 0;
    *which = -1;
    for (int64_t j = 0; j < T->n_leaves; j++) {
        int64_t n = T->leaf_node[j];
        if (or_in_box(T->lo + 3 * n, T->hi + 3 * n, p, k, T->lo, T->hi)) {
            hits++;
            *which = j;
        }
    }
    return hits;
}

void or_locate_batch(const or_tree *T, int64_t n, const double *p, const double *k, int64_t *out)
{
    for (int64_t i = 0; i < n; i++) out[i] = or_locate(T, p + 3 * i, k + 3 * i);
}

void or_brute_locate_batch(const or_tree *T, int64_t n, const double *p, const double *k, int64_t *out,
                           int64_t *hits)
{
    for (int64_t i = 0; i < n; i++) hits[i] = or_brute_locate(T, p + 3 * i, k + 3 * i, out + i);
}

/* ------------------------------------------------------------------ path calculation */

/* Trace one path.  seg_cell/seg_ds may be NULL (no emission); cap is their
 * capacity.  Returns the ray status bits; *ncross = emitted segments,
 * *S = sum rho*ds. */
static int or_trace_one(const or_tree *T, const double *o, const double *k, int has_smax, double smax,
                        int64_t max_steps, int64_t *ncross, double *S, int32_t *seg_cell, double *seg_ds,
                        int64_t cap)
{
    *ncross = 0;
    *S = 0.0;
    for (int a = 0; a < 3; a++)
        if (!isfinite(o[a]) || !isfinite(k[a])) return OR_RAY_BADINPUT;
    if (k[0] == 0.0 && k[1] == 0.0 && k[2] == 0.0) return OR_RAY_BADINPUT;
    if (has_smax && isnan(smax)) return OR_RAY_BADINPUT;
    const double *dlo = T->lo, *dhi = T->hi;
    double invk[3];
    for (int a = 0; a < 3; a++) invk[a] = (k[a] != 0.0) ? 1.0 / k[a] : 0.0;

    /* clip against the domain box */
    double t_start = 0.0, t_out = INFINITY;
    int entry = -1;
    for (int a = 0; a < 3; a++) {
        if (k[a] == 0.0) {
            if (o[a] < dlo[a] || o[a] > dhi[a]) return 0;
            continue;
        }
        double tn = ((k[a] > 0.0 ? dlo[a] : dhi[a]) - o[a]) * invk[a];
        double tf = ((k[a] > 0.0 ? dhi[a] : dlo[a]) - o[a]) * invk[a];
        if (tn > t_start) { t_start = tn; entry = a; }
        if (tf < t_out) t_out = tf;
    }
    if (!(t_start < t_out)) return 0;
    if (has_smax && !(t_start < smax)) return 0;
    double p[3];
    if (entry < 0) {
        p[0] = o[0]; p[1] = o[1]; p[2] = o[2];
    } else {
        for (int a = 0; a < 3; a++) {
            if (a == entry) { p[a] = (k[a] > 0.0) ? dlo[a] : dhi[a]; continue; }
            double v = fma(k[a], t_start, o[a]);
            if (v < dlo[a]) v = dlo[a];
            if (v > dhi[a]) v = dhi[a];
            p[a] = v;
        }
    }
    int64_t cur = or_locate(T, p, k);
    if (cur < 0) return 0; /* leaves the domain at its entry point */

    double t_cur = t_start;
    int64_t steps = 0;
    for (;;) {
        if (steps >= max_steps) return OR_RAY_STEPLIMIT;
        steps++;
        int64_t nd = T->leaf_node[cur];
        const double *lo = T->lo + 3 * nd, *hi = T->hi + 3 * nd;
        double t_ex = INFINITY;
        int ax = -1;
        for (int a = 0; a < 3; a++) {
            if (k[a] == 0.0) continue;
            double w = (k[a] > 0.0) ? hi[a] : lo[a];
            double t = (w - o[a]) * invk[a];
            if (t < t_ex) { t_ex = t; ax = a; }
        }
        if (has_smax && smax < t_ex) { t_ex = smax; ax = -1; }
        if (t_ex < t_cur) t_ex = t_cur;
        double ds = t_ex - t_cur;
        if (ds != 0.0) {
            if (seg_cell) {
                if (*ncross >= cap) return OR_RAY_OVERFLOW;
                seg_cell[*ncross] = (int32_t)cur;
                seg_ds[*ncross] = ds;
            }
            *S = fma(T->rho[nd], ds, *S);
            (*ncross)++;
        }
        t_cur = t_ex;
        if (ax < 0) return 0;
        double wall = (k[ax] > 0.0) ? hi[ax] : lo[ax];
        if (wall == ((k[ax] > 0.0) ? dhi[ax] : dlo[ax])) return 0; /* leaves the domain */
        for (int b = 0; b < 3; b++) {
            if (b == ax) { p[b] = wall; continue; }
            double v = fma(k[b], t_ex, o[b]);
            if (v < lo[b]) v = lo[b];
            if (v > hi[b]) v = hi[b];
            p[b] = v;
        }
        /* an exit point on the domain surface with the direction pointing
         * out (edge or corner exits) ends the path */
        if (!or_in_box(dlo, dhi, p, k, dlo, dhi)) return 0;
        int64_t nxt = or_locate(T, p, k);
        if (nxt < 0) return OR_RAY_LOST;
        cur = nxt;
    }
}

/* Trace a batch.  smax may be NULL (walk to the domain exit).  With seg_off
 * non-NULL, segments are written at seg_off[i] .. and seg_off[i+1] bounds
 * the capacity of ray i.  Returns the OR of all ray statuses. */
int32_t or_trace_batch(const or_tree *T, int64_t n, const double *o, const double *k, const double *smax,
                       double kappa, int64_t max_steps, double *tau, int64_t *ncross, int32_t *status,
                       const int64_t *seg_off, int32_t *seg_cell, double *seg_ds)
{
    int32_t all = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t nc = 0;
        double S = 0.0;
        int32_t *sc = NULL;
        double *sd = NULL;
        int64_t cap = 0;
        if (seg_off) {
            sc = seg_cell + seg_off[i];
            sd = seg_ds + seg_off[i];
            cap = seg_off[i + 1] - seg_off[i];
        }
        int st = or_trace_one(T, o + 3 * i, k + 3 * i, smax != NULL, smax ? smax[i] : 0.0, max_steps, &nc, &S,
                              sc, sd, cap);
        tau[i] = kappa * S;
        ncross[i] = nc;
        if (status) status[i] = st;
        all |= st;
    }
    return all;
}

/* Interaction-point search (the step after the path in the Monte Carlo loop,
 * Sect. 2.3): walk as or_trace_one, accumulating S = sum rho*ds left to
 * right, and stop in the first recorded segment after which kappa*S >= tau_int.
 * Inside that leaf (entered at t_cur, left at t_exit) the interaction time
 * solves kappa*S_before + kappa*rho*(t - t_cur) = tau_int:
 *   a = tau_int - kappa*S_before; b = kappa*rho;
 *   t = t_cur + a/b when a > 0 and b > 0, else t_cur; t = min(t, t_exit).
 * *cell = the leaf id, *t = that time, *ncross = recorded segments up to and
 * including it.  A path that ends (domain exit, s_max) first gives
 * *cell = -1 and *t = its end time. */
static int or_interact_one(const or_tree *T, const double *o, const double *k, int has_smax, double smax,
                           double kappa, double tau_int, int64_t max_steps, int64_t *cell, double *t_out,
                           int64_t *ncross)
{
    *cell = -1;
    *t_out = 0.0;
    *ncross = 0;
    for (int a = 0; a < 3; a++)
        if (!isfinite(o[a]) || !isfinite(k[a])) return OR_RAY_BADINPUT;
    if (k[0] == 0.0 && k[1] == 0.0 && k[2] == 0.0) return OR_RAY_BADINPUT;
    if (has_smax && isnan(smax)) return OR_RAY_BADINPUT;
    if (isnan(tau_int)) return OR_RAY_BADINPUT;
    const double *dlo = T->lo, *dhi = T->hi;
    double invk[3];
    for (int a = 0; a < 3; a++) invk[a] = (k[a] != 0.0) ? 1.0 / k[a] : 0.0;
    double t_start = 0.0, t_out_dom = INFINITY;
    int entry = -1;
    for (int a = 0; a < 3; a++) {
        if (k[a] == 0.0) {
            if (o[a] < dlo[a] || o[a] > dhi[a]) return 0;
            continue;
        }
        double tn = ((k[a] > 0.0 ? dlo[a] : dhi[a]) - o[a]) * invk[a];
        double tf = ((k[a] > 0.0 ? dhi[a] : dlo[a]) - o[a]) * invk[a];
        if (tn > t_start) { t_start = tn; entry = a; }
        if (tf < t_out_dom) t_out_dom = tf;
    }
    if (!(t_start < t_out_dom)) return 0;
    if (has_smax && !(t_start < smax)) return 0;
    double p[3];
    if (entry < 0) {
        p[0] = o[0]; p[1] = o[1]; p[2] = o[2];
    } else {
        for (int a = 0; a < 3; a++) {
            if (a == entry) { p[a] = (k[a] > 0.0) ? dlo[a] : dhi[a]; continue; }
            double v = fma(k[a], t_start, o[a]);
            if (v < dlo[a]) v = dlo[a];
            if (v > dhi[a]) v = dhi[a];
            p[a] = v;
        }
    }
    int64_t cur = or_locate(T, p, k);
    if (cur < 0) return 0;
    double t_cur = t_start, S = 0.0;
    int64_t steps = 0;
    for (;;) {
        if (steps >= max_steps) { *t_out = t_cur; return OR_RAY_STEPLIMIT; }
        steps++;
        int64_t nd = T->leaf_node[cur];
        const double *lo = T->lo + 3 * nd, *hi = T->hi + 3 * nd;
        double t_ex = INFINITY;
        int ax = -1;
        for (int a = 0; a < 3; a++) {
            if (k[a] == 0.0) continue;
            double w = (k[a] > 0.0) ? hi[a] : lo[a];
            double t = (w - o[a]) * invk[a];
            if (t < t_ex) { t_ex = t; ax = a; }
        }
        if (has_smax && smax < t_ex) { t_ex = smax; ax = -1; }
        if (t_ex < t_cur) t_ex = t_cur;
        double ds = t_ex - t_cur;
        if (ds != 0.0) {
            const double rho = T->rho[nd];
            const double S_new = fma(rho, ds, S);
            (*ncross)++;
            if (kappa * S_new >= tau_int) {
                const double a = tau_int - kappa * S;
                const double b = kappa * rho;
                double t = t_cur;
                if (a > 0.0 && b > 0.0) t = t_cur + a / b;
                if (t > t_ex) t = t_ex;
                *cell = cur;
                *t_out = t;
                return 0;
            }
            S = S_new;
        }
        t_cur = t_ex;
        *t_out = t_cur;
        if (ax < 0) return 0;
        double wall = (k[ax] > 0.0) ? hi[ax] : lo[ax];
        if (wall == ((k[ax] > 0.0) ? dhi[ax] : dlo[ax])) return 0;
        for (int b = 0; b < 3; b++) {
            if (b == ax) { p[b] = wall; continue; }
            double v = fma(k[b], t_ex, o[b]);
            if (v < lo[b]) v = lo[b];
            if (v > hi[b]) v = hi[b];
            p[b] = v;
        }
        if (!or_in_box(dlo, dhi, p, k, dlo, dhi)) return 0;
        int64_t nxt = or_locate(T, p, k);
        if (nxt < 0) return OR_RAY_LOST;
        cur = nxt;
    }
}

int32_t or_interact_batch(const or_tree *T, int64_t n, const double *o, const double *k, const double *smax,
                          double kappa, const double *tau_int, int64_t max_steps, int64_t *cell, double *t,
                          int64_t *ncross, int32_t *status)
{
    int32_t all = 0;
    for (int64_t i = 0; i < n; i++) {
        int st = or_interact_one(T, o + 3 * i, k + 3 * i, smax != NULL, smax ? smax[i] : 0.0, kappa, tau_int[i],
                                 max_steps, cell + i, t + i, ncross + i);
        if (status) status[i] = st;
        all |= st;
    }
    return all;
}

/* Brute-force crossed-cell list: every leaf's slab interval intersected with
 * the path [t0, t1]; intervals of positive length are kept and sorted by
 * entry time.  Meant for rays in general position with no zero direction
 * component.  Returns the number of cells (<= cap), or -1 on overflow. */
int64_t or_brute_sequence(const or_tree *T, const double *o, const double *k, double t0, double t1,
                          int32_t *cells, double *tin_out, double *ds_out, int64_t cap)
{
    int64_t cnt = 0;
    for (int64_t j = 0; j < T->n_leaves; j++) {
        int64_t nd = T->leaf_node[j];
        const double *lo = T->lo + 3 * nd, *hi = T->hi + 3 * nd;
        double tin = t0, tout = t1;
        for (int a = 0; a < 3; a++) {
            double inv = 1.0 / k[a];
            double ta = (lo[a] - o[a]) * inv, tb = (hi[a] - o[a]) * inv;
            double n1 = ta < tb ? ta : tb, f1 = ta < tb ? tb : ta;
            if (n1 > tin) tin = n1;
            if (f1 < tout) tout = f1;
        }
        if (tout > tin) {
            if (cnt >= cap) return -1;
            cells[cnt] = (int32_t)j;
            tin_out[cnt] = tin;
            ds_out[cnt] = tout - tin;
            cnt++;
        }
    }
    /* insertion sort by entry time (short lists) */
    for (int64_t a = 1; a < cnt; a++) {
        int32_t c = cells[a];
        double ti = tin_out[a], d = ds_out[a];
        int64_t b = a - 1;
        while (b >= 0 && tin_out[b] > ti) {
            cells[b + 1] = cells[b];
            tin_out[b + 1] = tin_out[b];
            ds_out[b + 1] = ds_out[b];
            b--;
        }
        cells[b + 1] = c;
        tin_out[b + 1] = ti;
        ds_out[b + 1] = d;
    }
    return cnt;
}

/* ------------------------------------------------------------------ true optical depth */

/* 15-point Kronrod rule with its embedded 7-point Gauss rule on [-1, 1]
 * (abscissae x_j and weights; the Gauss points are the odd-indexed Kronrod
 * abscissae). */
static const double or_xgk[8] = {
    0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
    0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
    0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
    0.207784955007898467600689403773245, 0.000000000000000000000000000000000};
static const double or_wgk[8] = {
    0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
    0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
    0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
    0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
static const double or_wg[4] = {
    0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
    0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

typedef double (*or_fn)(const void *ctx, double t);

static void or_gk15(or_fn f, const void *ctx, double a, double b, double *res, double *err)
{
    double c = 0.5 * (a + b), h = 0.5 * (b - a);
    double fc = f(ctx, c);
    double rk = fc * or_wgk[7], rg = fc * or_wg[3];
    for (int j = 0; j < 7; j++) {
        double x = h * or_xgk[j];
        double f1 = f(ctx, c - x), f2 = f(ctx, c + x);
        rk += or_wgk[j] * (f1 + f2);
        if (j & 1) rg += or_wg[j / 2] * (f1 + f2);
    }
    *res = rk * h;
    *err = fabs((rk - rg) * h);
}

static double or_adapt(or_fn f, const void *ctx, double a, double b, double rtol, int depth)
{
    double r, e;
    or_gk15(f, ctx, a, b, &r, &e);
    if (depth >= 60 || e <= rtol * fabs(r) || e < 1e-300 || !(b > a)) return r;
    double c = 0.5 * (a + b);
    return or_adapt(f, ctx, a, c, rtol, depth + 1) + or_adapt(f, ctx, c, b, rtol, depth + 1);
}

/* Integrate a polynomial sum c_j t^j adaptively (pins the quadrature rule). */
typedef struct { const double *c; int n; } or_poly;
static double or_poly_eval(const void *ctx, double t)
{
    const or_poly *P = ctx;
    double v = 0.0;
    for (int j = P->n - 1; j >= 0; j--) v = v * t + P->c[j];
    return v;
}
double or_quad_poly(const double *c, int n, double a, double b, int adaptive)
{
    or_poly P = {c, n};
    if (adaptive) return or_adapt(or_poly_eval, &P, a, b, 1e-13, 0);
    double r, e;
    or_gk15(or_poly_eval, &P, a, b, &r, &e);
    return r;
}

typedef struct { const or_model *m; const double *o, *k; } or_ray_ctx;
static double or_ray_rho(const void *ctx, double t)
{
    const or_ray_ctx *R = ctx;
    return or_rho_true(R->m, R->o[0] + R->k[0] * t, R->o[1] + R->k[1] * t, R->o[2] + R->k[2] * t);
}

static void or_add_bp(double *bp, int *nb, int cap, double t, double t1)
{
    if (t > 0.0 && t < t1 && *nb < cap) bp[(*nb)++] = t;
}

static double or_horner(const double *c, int deg, double t)
{
    double v = c[deg];
    for (int j = deg - 1; j >= 0; j--) v = v * t + c[j];
    return v;
}

/* Real roots of the polynomial sum c_j t^j (degree deg <= 4) inside (a, b):
 * roots of the derivative split (a, b) into monotone pieces, each bisected. */
static int or_poly_roots(const double *c, int deg, double a, double b, double *roots)
{
    while (deg > 0 && c[deg] == 0.0) deg--;
    if (deg == 0) return 0;
    if (deg == 1) {
        double t = -c[0] / c[1];
        if (t > a && t < b) { roots[0] = t; return 1; }
        return 0;
    }
    double dc[4];
    for (int j = 1; j <= deg; j++) dc[j - 1] = j * c[j];
    double crit[4];
    int nc = or_poly_roots(dc, deg - 1, a, b, crit);
    double edges[6];
    int ne = 0;
    edges[ne++] = a;
    for (int j = 0; j < nc; j++) edges[ne++] = crit[j];
    edges[ne++] = b;
    int nr = 0;
    for (int j = 0; j + 1 < ne; j++) {
        double lo = edges[j], hi = edges[j + 1];
        double flo = or_horner(c, deg, lo), fhi = or_horner(c, deg, hi);
        if (flo == 0.0) { if (lo > a) roots[nr++] = lo; continue; }
        if ((flo < 0.0) == (fhi < 0.0)) continue;
        for (int it = 0; it < 200 && hi - lo > 0.0; it++) {
            double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            double fm = or_horner(c, deg, mid);
            if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; } else hi = mid;
        }
        roots[nr++] = 0.5 * (lo + hi);
    }
    return nr;
}

static int or_cmp_double(const void *x, const void *y)
{
    double a = *(const double *)x, b = *(const double *)y;
    return (a > b) - (a < b);
}

/* True optical depth kappa * integral_0^L rho_t(o + k t) dt.  Breakpoints:
 * disk -- the plane z = 0 and the closest approach to the z axis; torus --
 * the tube surface (quartic roots) and for every clump its truncation
 * sphere and closest approach; dyadic -- every lattice plane. */
double or_tau_true(const or_model *m, const double *o, const double *k, double L, double kappa, double rtol)
{
    enum { CAP = 8192 };
    double *bp = malloc(sizeof(double) * CAP);
    int nb = 0;
    bp[nb++] = 0.0;
    if (m->kind == OR_MODEL_DISK) {
        if (k[2] != 0.0) or_add_bp(bp, &nb, CAP, -o[2] / k[2], L);
        double kk = k[0] * k[0] + k[1] * k[1];
        if (kk > 0.0) or_add_bp(bp, &nb, CAP, -(o[0] * k[0] + o[1] * k[1]) / kk, L);
    } else if (m->kind == OR_MODEL_TORUS) {
        double R = m->p[0], r = m->p[1];
        double A = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        double B = 2.0 * (o[0] * k[0] + o[1] * k[1] + o[2] * k[2]);
        double C = o[0] * o[0] + o[1] * o[1] + o[2] * o[2] + R * R - r * r;
        double D = k[0] * k[0] + k[1] * k[1];
        double E = 2.0 * (o[0] * k[0] + o[1] * k[1]);
        double F = o[0] * o[0] + o[1] * o[1];
        double c[5] = {C * C - 4.0 * R * R * F, 2.0 * B * C - 4.0 * R * R * E, B * B + 2.0 * A * C - 4.0 * R * R * D,
                       2.0 * A * B, A * A};
        double roots[4];
        int nr = or_poly_roots(c, 4, 0.0, L, roots);
        for (int j = 0; j < nr; j++) or_add_bp(bp, &nb, CAP, roots[j], L);
        for (int32_t j = 0; j < m->n_table; j++) {
            const double *cl = m->table + 5 * (int64_t)j;
            double w[3] = {o[0] - cl[0], o[1] - cl[1], o[2] - cl[2]};
            double b2 = w[0] * k[0] + w[1] * k[1] + w[2] * k[2];
            double cc = w[0] * w[0] + w[1] * w[1] + w[2] * w[2] - 25.0 * cl[3] * cl[3];
            double disc = b2 * b2 - A * cc;
            if (disc <= 0.0) continue;
            double sq = sqrt(disc);
            or_add_bp(bp, &nb, CAP, (-b2 - sq) / A, L);
            or_add_bp(bp, &nb, CAP, (-b2 + sq) / A, L);
            or_add_bp(bp, &nb, CAP, -b2 / A, L);
        }
    } else if (m->kind == OR_MODEL_DYADIC) {
        int64_t n = (int64_t)1 << (int)m->p[0];
        for (int a = 0; a < 3; a++) {
            if (k[a] == 0.0) continue;
            for (int64_t j = 1; j < n; j++) {
                double pl = m->lo[a] + (m->hi[a] - m->lo[a]) * ((double)j / (double)n);
                or_add_bp(bp, &nb, CAP, (pl - o[a]) / k[a], L);
            }
        }
    }
    bp[nb++] = L;
    qsort(bp, (size_t)nb, sizeof(double), or_cmp_double);
    or_ray_ctx ctx = {m, o, k};
    double tot = 0.0;
    for (int j = 0; j + 1 < nb; j++)
        if (bp[j + 1] > bp[j]) tot += or_adapt(or_ray_rho, &ctx, bp[j], bp[j + 1], rtol, 0);
    free(bp);
    return kappa * tot;
}

void or_tau_true_batch(const or_model *m, int64_t n, const double *o, const double *k, const double *L,
                       double kappa, double rtol, double *out)
{
    for (int64_t i = 0; i < n; i++) out[i] = or_tau_true(m, o + 3 * i, k + 3 * i, L[i], kappa, rtol);
}

/* Grid density at points: top-down location, then the leaf's density
 * (Sect. 3.2, Delta-rho metric).  cell = -1 and rho = 0 outside. */
void or_sample_density(const or_tree *T, int64_t n, const double *pts, int64_t *cell, double *rho)
{
    const double kpos[3] = {0.0, 0.0, 0.0};
    for (int64_t i = 0; i < n; i++) {
        int64_t c = or_locate(T, pts + 3 * i, kpos);
        cell[i] = c;
        rho[i] = (c >= 0) ? T->rho[T->leaf_node[c]] : 0.0;
    }
}
