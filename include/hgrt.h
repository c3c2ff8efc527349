/*
 * hgrt.h -- C ABI of the GB300 path-calculation library for octree and k-d
 * tree dust grids (Saftly, Baes & Camps, "Hierarchical octree and k-d tree
 * grids for 3D radiative transfer simulations").
 *
 * Conventions shared by every entry point
 *   - Pointers marked "dev" are CUDA device pointers, "host" are host
 *     pointers.  The caller owns every buffer it passes; the library owns
 *     only what it allocates behind an opaque handle (hg_host_grid, hg_grid,
 *     hg_dmodel, hg_batch) and frees it in the matching hg_free_* call.
 *   - Calls that take a stream are asynchronous on that stream (NULL means
 *     the legacy default stream).  Argument, allocation and launch errors
 *     are returned synchronously as hg_status; a kernel fault surfaces on
 *     the caller's next synchronisation.  Scratch memory these calls need
 *     is taken from the CUDA stream-ordered allocator on the same stream
 *     and released on it before the call returns.
 *   - Per-ray problems never abort a launch: they are reported as bit
 *     flags (HG_RAY_*) in the optional per-ray status array.
 *   - hg_last_error() returns a message for the calling thread's last
 *     failed call.
 *   - Arrays of 3-vectors are row-major [n][3] doubles (x, y, z per row).
 *   - A loaded grid is immutable and may be used from several streams at
 *     once.
 */
#ifndef HGRT_H
#define HGRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum hg_status {
    HG_OK = 0,
    HG_EINVAL = 1,      /* bad argument */
    HG_ENOMEM = 2,      /* host or device allocation failed */
    HG_ECUDA = 3,       /* a CUDA runtime call failed */
    HG_EOVERFLOW = 4,   /* output capacity too small */
    HG_ESTEPLIMIT = 5,  /* some ray hit its step limit */
    HG_ELOST = 6,       /* some ray found no next cell */
    HG_EFORMAT = 7,     /* grid description failed validation */
    HG_EBADINPUT = 8,   /* some ray had a non-finite or zero direction */
    HG_ENOTFOUND = 9    /* missing CUDA device or symbol */
} hg_status;

/* per-ray status bits */
#define HG_RAY_STEPLIMIT 1u /* the walk stopped at max_steps */
#define HG_RAY_LOST 2u      /* no leaf contained an exit point inside the domain */
#define HG_RAY_BADINPUT 4u  /* non-finite origin/direction/length or zero direction */
#define HG_RAY_OVERFLOW 8u  /* emission capacity exceeded; segments truncated */

#define HG_OCTREE 0
#define HG_KDTREE 1

#define HG_MODEL_CONST 0  /* rho = p[0] */
#define HG_MODEL_DISK 1   /* rho = p[0] exp(-R/p[1] - |z|/p[2]), R = sqrt(x^2+y^2) */
#define HG_MODEL_TORUS 2  /* rho0 = p[2] inside (sqrt(x^2+y^2)-p[0])^2 + z^2 < p[1]^2, plus clumps */
#define HG_MODEL_DYADIC 3 /* piecewise constant on a 2^p[0] lattice, values in table */

#define HG_FP64 0   /* wall test, segment lengths and tau in FP64 */
#define HG_FP32K 1  /* wall test in FP64; segment lengths and densities cast to FP32,
                       tau summed in FP32 with Kahan compensation */

typedef void *hg_stream; /* a cudaStream_t */

/* ------------------------------------------------------------------------ density models
 * Stand-ins for the paper's test models (Sect. 3.1): an exponential disk,
 * a ring torus with a hard edge plus truncated Gaussian clumps, a uniform
 * medium and a piecewise-constant lattice.
 *   torus table: n_table rows of (cx, cy, cz, sigma, A); clump j adds
 *     A exp(-0.5 r^2/sigma^2) where r^2 < 25 sigma^2, summed in row order.
 *   dyadic table: 8^L values, index ix + n (iy + n iz), n = 2^L.
 * m_tot is the total mass inside [lo, hi] used by the mass criterion. */
typedef struct hg_model {
    int32_t kind;
    int32_t n_table;
    double p[8];
    const double *table; /* host */
    double m_tot;
    double lo[3], hi[3]; /* domain box */
} hg_model;

/* ------------------------------------------------------------------------ tree construction
 * Subdivision-stopping criteria of Sect. 2.2 and 4: a node is subdivided
 * when any enabled test fires (and it is above the maximum level):
 *   mass fraction   delta = M / m_tot > delta_max      (Sect. 2.2, Eq. 1)
 *   optical depth   kappa M sqrt(a^2+b^2+c^2)/(abc) > tau_max   (Eq. 2)
 *   dispersion      q = (rho_max - rho_min)/rho_max > q_max     (Eq. 3)
 * M = V * mean of rho_t at n_ran positions drawn uniformly in the node
 * (Eq. 1) with SplitMix64 keyed by the node's box, so that a node's samples
 * do not depend on the build order.  max_level counts octree levels; a k-d
 * tree may be 3*max_level splits deep (Sect. 2.1).
 * k-d split orientation (Sect. 2.2): HG_AXIS_CYCLIC, the axes in turn x, y,
 * z, x, ...; or HG_AXIS_GRADIENT, the axis of the strongest density
 * gradient in the node, estimated from its n_ran draws: on each axis a the
 * draws below and above the node's midpoint give mean densities m_lo, m_hi,
 * and g_a = |m_hi - m_lo| / (hi_a - lo_a) (0 when a half has no draw);
 * among the axes halved fewer than max_level times (so that no axis is
 * refined beyond the octree-equivalent level and the depth stays at most
 * 3*max_level) the largest positive g_a wins, ties to the lower axis; when
 * none is positive, the first of those axes in cyclic order from the
 * node's depth mod 3.
 * Split location (Sect. 2.2), from the node's n_ran draws (positions x_s,
 * densities r_s, s = 0..n_ran-1):
 *   HG_PLANE_CENTRE: the geometric centre (the dyadic midpoint);
 *   HG_PLANE_BARYCENTRE (octrees): the three planes through the centre of
 *     mass sum(r_s x_s) / sum(r_s), sums in draw order;
 *   HG_PLANE_EQUAL_MASS (k-d trees): with the draws ordered by their
 *     coordinate on the split axis (ties by s), the plane between draws j
 *     and j+1 for the first j whose running density sum C_j (left to right)
 *     satisfies 2 C_j >= C_total, but at most n_ran-2;
 *   HG_PLANE_EQUAL_DENSITY (k-d trees): the plane between draws j and j+1
 *     minimising |C_j/(j+1) - R_j/(n_ran-1-j)| (R_j the sum right of the
 *     plane, added right to left) over the j whose draws differ in
 *     position; ties to the smallest |2j - (n_ran-2)|, then the smaller j.
 * A plane between draws sits at x_j + (x_{j+1} - x_j)/2.  Without mass (or
 * usable draws), or when that value is not strictly inside the node, the
 * node's centre lo + (hi - lo)/2 is used; a node too thin to hold any plane
 * strictly inside stays a leaf.  With a location other than the centre the
 * gradient orientation compares the draws below and above lo + (hi - lo)/2.
 * Such trees have FP64 node boxes that are no dyadic lattice cells; their
 * neighbor lists are found and sorted with FP64 box arithmetic.  The level
 * and index outputs still count the halvings per axis (they key the draws). */
#define HG_AXIS_CYCLIC 0
#define HG_AXIS_GRADIENT 1
#define HG_PLANE_CENTRE 0
#define HG_PLANE_BARYCENTRE 1
#define HG_PLANE_EQUAL_MASS 2
#define HG_PLANE_EQUAL_DENSITY 3
typedef struct hg_build_params {
    int32_t kind; /* HG_OCTREE or HG_KDTREE */
    int32_t use_delta, use_tau, use_q;
    double delta_max, tau_max, q_max, kappa;
    int32_t max_level; /* 0..20 */
    int32_t n_ran;     /* >= 1 */
    uint64_t seed;
    int64_t max_nodes; /* 0 = unlimited; otherwise the build fails with HG_EOVERFLOW beyond it */
    int32_t split_axis;  /* k-d trees: HG_AXIS_CYCLIC or HG_AXIS_GRADIENT; ignored for octrees */
    int32_t split_plane; /* HG_PLANE_CENTRE; octrees also HG_PLANE_BARYCENTRE; k-d trees also
                            HG_PLANE_EQUAL_MASS or HG_PLANE_EQUAL_DENSITY (host builder only) */
} hg_build_params;

/* Flat description of a grid: the node list of Sect. 2.2 (root first,
 * children contiguous: 8 for an octree in x-fastest order, 2 for a k-d
 * tree, lower child first), leaf densities, and the six neighbor lists per
 * leaf of Sect. 2.3 (walls -x,+x,-y,+y,-z,+z; each list sorted by
 * decreasing overlap area, ties by ascending leaf id).  All host pointers,
 * read only during the call that receives them. */
typedef struct hg_grid_desc {
    int32_t kind;
    int32_t reserved;
    int64_t n_nodes;
    int64_t n_leaves;
    const double *node_lo;       /* [n_nodes][3] */
    const double *node_hi;       /* [n_nodes][3] */
    const int32_t *child_first;  /* [n_nodes], -1 for a leaf */
    const int32_t *node_leaf;    /* [n_nodes], leaf id or -1; leaf ids follow list order */
    const double *leaf_rho;      /* [n_leaves] */
    const int64_t *nbr_off;      /* [6*n_leaves+1], list of wall w of leaf i = nbr_off[6i+w] .. nbr_off[6i+w+1] */
    const int32_t *nbr_id;       /* [nbr_off[6*n_leaves]]; may be NULL when that is 0 (a single leaf) */
} hg_grid_desc;

/* Extra per-node builder output (host arrays owned by the hg_host_grid). */
typedef struct hg_host_nodes {
    const int32_t *level;  /* [n_nodes][3] per-axis subdivision level */
    const int64_t *index;  /* [n_nodes][3] per-axis integer position at that level */
    const double *mass;    /* [n_nodes] Eq. 1 */
    const double *delta;   /* [n_nodes] M / m_tot */
    const double *tau;     /* [n_nodes] Eq. 2 */
    const double *q;       /* [n_nodes] Eq. 3 */
} hg_host_nodes;

typedef struct hg_host_grid hg_host_grid;

/* Build a tree on the host with n_threads threads (<= 0: all cores).
 * Deterministic: the result does not depend on n_threads. */
hg_status hg_build_grid(const hg_model *model, const hg_build_params *params, int32_t n_threads,
                        hg_host_grid **out);
/* hg_build_grid on the current GPU: every level of the breadth-first node
 * list (Sect. 2.2) has its nodes' n_ran Monte Carlo draws, mass, optical
 * depth and dispersion (Eq. 1-3) computed by one device thread per node,
 * with the host builder's draws and arithmetic, and its children appended
 * by a scan; the neighbor lists (Sect. 2.3) are found by one device thread
 * per leaf wall.  All on `stream`, one copy to the host at the end.  Same
 * tree, statistics and lists as
 * hg_build_grid except that CUDA's exp may round differently from the
 * host's libm in the disk and clump models (a statistic then differs in its
 * last bits, and a node whose criterion lies that close to its threshold
 * may be decided the other way).  Synchronous: returns when the grid is
 * built.  Device memory used: the model table and clump index, about 150
 * bytes per node and 36 per leaf, then 12 per neighbor-list entry. */
hg_status hg_build_grid_gpu(const hg_model *model, const hg_build_params *params, hg_stream stream,
                            hg_host_grid **out);
/* The tau_max recipe of Sect. 4.1: build with params' mass criterion only
 * (use_tau and use_q ignored), sort the leaves' optical depths (Eq. 2) in
 * ascending order and return in *tau_max the one at 0-based position
 * floor(fraction * N_leaves) (at most N_leaves - 1); the paper takes
 * fraction = 0.9.  Build then with the mass criterion and this tau_max. */
hg_status hg_tau_max_recipe(const hg_model *model, const hg_build_params *params, double fraction,
                            int32_t n_threads, double *tau_max);
/* View the built grid as a description (pointers stay valid until hg_free_host_grid). */
hg_status hg_host_grid_desc(const hg_host_grid *g, hg_grid_desc *out);
hg_status hg_host_grid_nodes(const hg_host_grid *g, hg_host_nodes *out);
void hg_free_host_grid(hg_host_grid *g);

/* ------------------------------------------------------------------------ device grid */
typedef struct hg_grid hg_grid;

typedef struct hg_grid_info {
    int32_t kind;
    int32_t max_depth;      /* deepest node in the node list (k-d splits or octree levels) */
    int64_t n_nodes, n_leaves;
    int64_t n_tail;         /* stored neighbor entries beyond each wall's first */
    int64_t device_bytes;   /* HBM held by the grid */
    int64_t long_walls;     /* walls whose list is longer than the scan limit (searched top-down from the
                               wall's rope node, the deepest node across the wall covering it) */
    double lo[3], hi[3];
    int32_t nav;            /* HG_NAV_NEIGHBOR_LISTS or HG_NAV_ROPES: how the next leaf is found */
    int32_t reserved;
} hg_grid_info;

#define HG_NAV_NEIGHBOR_LISTS 0
#define HG_NAV_ROPES 1

/* Upload a grid: the node list of Sect. 2.2 and the six per-leaf neighbor
 * lists of Sect. 2.3 (built once with the grid, sorted by decreasing overlap
 * area) become 96-byte leaf records holding each wall's list head, the list
 * tails and the descent nodes of the top-down search (Sect. 2.3), in device
 * memory owned by the returned handle until hg_free_grid.  desc and the
 * arrays it points to are host memory, read during the call only.  With
 * validate != 0 the description is checked first
 * (links in range, children tiling their parent, leaf ids, every neighbor
 * list adjacent to its wall and tiling it); a failure returns HG_EFORMAT.
 * Needs a current CUDA device. */
hg_status hg_load_grid(const hg_grid_desc *desc, int32_t validate, hg_grid **out);
void hg_free_grid(hg_grid *g);
hg_status hg_grid_get_info(const hg_grid *g, hg_grid_info *out);

/* Ropes: the alternative to neighbor lists from the ray-shooting literature
 * that Sect. 1 and 2.3 set the paper's method against (stackless k-d
 * traversal, one link per leaf wall).  The rope of a leaf wall is the
 * deepest node lying across the wall (on its far side, touching it) whose
 * box covers the wall's whole face; it is found by a descent from the root
 * that continues while exactly one child covers the face.  A path leaving a
 * leaf through that wall goes to the rope's node and, when that is not a
 * leaf, locates its exit point top-down below it instead of from the root;
 * an exit point the rope's leaf does not hold (edge and corner exits) is
 * located from the root, as with neighbor lists.  Results are those of the
 * neighbor-list walk: the next leaf is the one the contract defines.
 * hg_build_ropes writes ropes[6 i + w] for leaf i, wall w (-x,+x,-y,+y,-z,
 * +z): the leaf id (>= 0), -1 on the domain boundary, or -2 - node for an
 * internal node.  desc: host arrays (the neighbor lists are not read);
 * ropes: host int32[6 n_leaves], caller-owned; n_threads <= 0: all cores.
 * HG_EFORMAT for leaf ids that do not match the node list. */
hg_status hg_build_ropes(const hg_grid_desc *desc, int32_t n_threads, int32_t *ropes);
/* hg_load_grid for the rope walk: each leaf record's six wall slots hold
 * ropes (from hg_build_ropes; NULL: built here with all cores) instead of
 * the neighbor-list heads, and no list tails are stored (the description's
 * neighbor lists may be NULL).  Every walk of the library then follows
 * ropes on this grid.  With validate != 0 the node list is checked as by
 * hg_load_grid and every rope must lie across its wall and cover its face
 * (HG_EFORMAT otherwise). */
hg_status hg_load_grid_ropes(const hg_grid_desc *desc, const int32_t *ropes, int32_t validate, hg_grid **out);

/* ------------------------------------------------------------------------ path calculation
 * A path is x(t) = o + t d for t in [t_start, t_end]: t_start = 0 for an
 * origin inside the domain, else the entry time of the slab test; t_end is
 * the domain exit, or s_max if given and smaller.  The result is the
 * ordered list of leaves whose interior the path crosses with the length
 * ds inside each, and tau = kappa * sum rho_leaf ds (Sect. 2.3, 3.2).  The
 * first leaf comes from a top-down descent; every later one from the exit
 * wall's neighbor list (Sect. 2.3), the list's first entry being stored in
 * the leaf itself, with a top-down descent when no listed neighbor
 * contains the exit point (edge and corner exits) or the list is long (for
 * a long list the descent starts at the deepest node across the wall that
 * covers the whole wall, and falls back to the root if the leaf found there
 * does not hold the exit point).
 *
 * FP64 arithmetic as in this contract (fma: one rounding; every other
 * multiply and add rounded on its own):
 *   invk_a = 1/d_a (d_a == +-0: axis a never exits);
 *   t_a = (wall_a - o_a) * invk_a for the wall ahead on each axis; exit at
 *   the smallest, ties to the lower axis; t_end wins only when smaller;
 *   exit times are never below the current time; ds = t_exit - t_cur and
 *   segments with ds == 0 are skipped (not emitted, not counted);
 *   exit point p_a = wall_a, p_b = fma(d_b, t_exit, o_b) clamped to the
 *   leaf (the entry point of an outside origin likewise);
 *   p lies in box [l, h] iff per axis l < p < h, p == l with d >= 0, or
 *   p == h with d < 0 (the domain's upper face also with d == 0);
 *   FP64 tau = kappa * S, S = fma(rho, ds, S) over the segments left to
 *   right.
 * Directions are used as given (not normalised); s_max is in the same t. */
typedef struct hg_trace_opts {
    int32_t precision;   /* HG_FP64 or HG_FP32K */
    int32_t block;       /* threads per block (32..256, multiple of 32); 0 = tuned or default */
    int32_t smem_nodes;  /* top tree nodes the walks stage in shared memory (clamped to 200 KB); -1 = tuned or
                            default (64: the walk descends only after edge and corner exits and list misses, and
                            shared memory is taken from the L1 that serves its record gathers).  The setup pass
                            (first leaf of every ray) always stages the top 8 KB */
    int32_t schedule;    /* 0 = tuned or automatic; 1 = static ray stride; 2 = dynamic queue (warp-aggregated
                            counter) in input order; 3 = dynamic queue, rays with the most estimated
                            crossings first (automatic when there are fewer than 48 rays per
                            resident thread) */
    int32_t min_blocks;  /* 0 = tuned or default (4; 3 for hg_find_interactions, whose walk needs more
                            than 64 registers); 3 or 4 resident 256-thread blocks per SM the kernel's
                            register budget is cut for (80 or 64 registers; each walking thread also keeps
                            its ray's origin, direction and 1/d in 72 bytes of shared memory) */
    int32_t split;       /* HG_SPLIT_AUTO (0), HG_SPLIT_OFF or HG_SPLIT_FORCE; see below */
    int64_t max_steps;   /* per-ray step limit; 0 = 4 * n_leaves + 64 */
} hg_trace_opts;

/* Path segments.  With schedule 3 (work-ordered queue), in hg_trace_rays,
 * hg_trace_rays_rho and hg_tau_gradient, a path whose estimated crossings
 * exceed max(64, A) is cut into at most 16 segments of about max(32, A/2)
 * that separate threads walk (A = estimated total / the launch's threads;
 * HG_SPLIT_FORCE: every path of more than 3, in pieces of 2, for testing).  Cuts lie at the middle of a leaf the path crosses,
 * deep inside it, so every segment follows the whole path's cell sequence:
 * crossing counts, statuses, emitted cells and gradients are those of the
 * unsplit walk; tau is the sum of the segments' partial sums, which differs
 * from the left-to-right sum only in the grouping of the additions (a few
 * ulps).  A segment that does not end in the leaf where the next one starts
 * would set HG_RAY_LOST; the placement rule makes that impossible.  A
 * max_steps below the default turns splitting off. */
#define HG_SPLIT_AUTO 0
#define HG_SPLIT_OFF 1
#define HG_SPLIT_FORCE 2

/* tau: dev f64[n] (HG_FP64) or f32[n] (HG_FP32K).  ncross: dev i32[n],
 * number of segments with ds > 0.  ray_status: dev u8[n] or NULL.
 * o, d: dev f64[n][3]; s_max: dev f64[n] or NULL. */
hg_status hg_trace_rays(const hg_grid *g, int64_t n, const double *o, const double *d, const double *s_max,
                        double kappa, const hg_trace_opts *opts, void *tau, int32_t *ncross,
                        uint8_t *ray_status, hg_stream stream);

/* As hg_trace_rays, with the leaf densities read from rho (dev f64[n_leaves])
 * instead of the grid's own: tau is linear in rho, and this is the forward
 * pass whose adjoint is hg_tau_gradient. */
hg_status hg_trace_rays_rho(const hg_grid *g, int64_t n, const double *o, const double *d, const double *s_max,
                            double kappa, const double *rho, const hg_trace_opts *opts, void *tau,
                            int32_t *ncross, uint8_t *ray_status, hg_stream stream);

/* Allocation-free optical-depth pass (the paper has no counterpart: this is
 * an interface of this library only).  Some callers cannot allocate device
 * memory at the time they trace -- code running inside a stream capture
 * whose owner forbids allocation nodes, real-time loops that must never
 * enter an allocator, hosts that give the library a fixed memory budget.
 * This call takes the arguments of hg_trace_rays and gives the same crossing
 * counts and statuses; tau is the same sum, equal up to the grouping of the
 * additions where hg_trace_rays cuts a long path into segments (a few ulps).
 * It walks every path whole, each thread taking rays at a static stride,
 * whatever opts.schedule and opts.split ask for (they are accepted and
 * checked, then ignored).  Its scratch -- one 48-byte start record per ray
 * and a work counter -- comes from a fixed array compiled into the library;
 * it calls no cudaMalloc, cudaFree or other allocator.
 *   - n must not exceed HG_NOALLOC_MAX_RAYS; a larger n returns HG_EINVAL
 *     before anything is launched (split the batch, or use hg_trace_rays).
 *   - Every GPU that loads the library holds the array (about 12.6 MB)
 *     until the process exits.
 *   - The first call on a device looks the array's device address up
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - Every call uses the same array and leaves its contents behind; calls
 *     whose work overlaps on the GPU (other streams, other host threads)
 *     race and give wrong results, so serialise them. */
#define HG_NOALLOC_MAX_RAYS 262144
hg_status hg_trace_rays_noalloc(const hg_grid *g, int64_t n, const double *o, const double *d,
                                const double *s_max, double kappa, const hg_trace_opts *opts, void *tau,
                                int32_t *ncross, uint8_t *ray_status, hg_stream stream);

/* Exclusive scan: seg_off[0] = 0, seg_off[i+1] = seg_off[i] + count[i]
 * (dev i32[n] -> dev i64[n+1]). */
hg_status hg_scan_offsets(int64_t n, const int32_t *count, int64_t *seg_off, hg_stream stream);

/* Emission pass (Sect. 2.3 "ordered list of dust cells"): writes ray i's
 * segments to seg_cell[seg_off[i] ..] (dev i32, leaf ids) and seg_ds (dev
 * f64, or f32 under HG_FP32K) in path order.  seg_off comes from
 * hg_scan_offsets over the ncross of hg_trace_rays with the same inputs;
 * entries at or beyond seg_capacity are not written and flag the ray
 * HG_RAY_OVERFLOW. */
hg_status hg_trace_fill(const hg_grid *g, int64_t n, const double *o, const double *d, const double *s_max,
                        const hg_trace_opts *opts, const int64_t *seg_off, int32_t *seg_cell, void *seg_ds,
                        int64_t seg_capacity, uint8_t *ray_status, hg_stream stream);

/* Interaction-point search (the step that follows the path in the Monte
 * Carlo loop of Sect. 2.3): each path is walked as in hg_trace_rays, in FP64,
 * and stops in the first recorded segment after which kappa * S >= tau_int[i]
 * (S the contract's running sum fma(rho, ds, S)).  Inside that leaf, entered at t_in
 * and left at t_exit, the interaction time solves the linear growth of tau:
 *   a = tau_int - kappa*S_before, b = kappa*rho,
 *   t = t_in + a/b when a > 0 and b > 0, else t_in;  t = min(t, t_exit).
 * Outputs: cell[i] the leaf (-1 when the path ends first), t[i] the
 * interaction time (else the path's end time, 0 for a path that misses the
 * grid), ncross[i] the recorded segments walked including the interaction
 * leaf, ray_status[i] as for hg_trace_rays (HG_RAY_BADINPUT also for a NaN
 * tau_int).  tau_int dev f64[n] (the caller draws -ln u); cell dev i32[n],
 * t dev f64[n], ncross dev i32[n].  Paths are never split into segments
 * here (where one stops depends on everything before). */
hg_status hg_find_interactions(const hg_grid *g, int64_t n, const double *o, const double *d, const double *s_max,
                               double kappa, const double *tau_int, const hg_trace_opts *opts, int32_t *cell,
                               double *t, int32_t *ncross, uint8_t *ray_status, hg_stream stream);

/* Grid density at points (Sect. 3.2, rho_g): top-down location with the
 * half-open rule above for a zero direction; cell = -1 and rho = 0 for
 * points outside the domain.  pts dev f64[n][3], cell dev i32[n] (or
 * NULL), rho dev f64[n]. */
hg_status hg_sample_density(const hg_grid *g, int64_t n, const double *pts, int32_t *cell, double *rho,
                            hg_stream stream);

/* Adjoint of tau with respect to the leaf densities.  Sect. 3.2 defines the
 * optical depth along a path as kappa times the integral of the density,
 * which on a grid is tau_r = kappa sum over the path's segments of
 * rho_cell ds (Sect. 2.3); tau is therefore linear in the leaf densities and
 * this is its exact derivative: for L = sum_r w_r tau_r,
 * grad_rho[c] += kappa * sum over segments s of ray r inside c of w_r ds_s.
 * w dev f32[n]; grad_rho dev f32[n_leaves] (grad_precision 1, FP32 atomics)
 * or f64[n_leaves] (grad_precision 0, FP64 atomics), ACCUMULATED. */
hg_status hg_tau_gradient(const hg_grid *g, int64_t n, const double *o, const double *d, const double *s_max,
                          double kappa, const float *w, int32_t grad_precision, void *grad_rho,
                          const hg_trace_opts *opts, hg_stream stream);

/* ------------------------------------------------------------------------ prepared rays
 * The optical-depth, emission and adjoint walks of one ray batch (Sect. 2.3
 * for each) share their setup: 1/d, clip, first leaf, the work-ordered queue
 * and the path segments.  hg_rays_prepare does that once; the walks below
 * then reuse it.  The rays' arrays (o, d, s_max) are read by every walk and
 * must stay unchanged until hg_rays_free.  Launch options (block,
 * smem_nodes, schedule, min_blocks, split, max_steps) are fixed at
 * preparation; the precision of each walk is given per call.  With path
 * segments (see hg_trace_opts.split), hg_rays_fill writes each segment's
 * cells after the crossings of the ray's earlier segments, which the last
 * hg_rays_trace on the same rays counted, so a fill needs a trace first
 * (HG_EINVAL otherwise); results are those of the one-shot calls. */
typedef struct hg_rays hg_rays;

/* Prepare n rays (o, d dev f64[n][3]; s_max dev f64[n] or NULL) on grid g.
 * *out receives a handle owning device scratch (stream-ordered on stream). */
hg_status hg_rays_prepare(const hg_grid *g, int64_t n, const double *o, const double *d, const double *s_max,
                          const hg_trace_opts *opts, hg_rays **out, hg_stream stream);
/* As hg_trace_rays (rho: dev f64[n_leaves] replacing the grid's densities,
 * or NULL).  Records the segments' crossing counts for hg_rays_fill. */
hg_status hg_rays_trace(hg_rays *r, double kappa, const double *rho, int32_t precision, void *tau,
                        int32_t *ncross, uint8_t *ray_status, hg_stream stream);
/* hg_rays_trace and hg_rays_gradient in one walk: tau, ncross and status,
 * and grad_rho += d(sum_r w_r tau_r)/d(rho) (ACCUMULATED), from the same
 * segments. */
hg_status hg_rays_trace_gradient(hg_rays *r, double kappa, const double *rho, int32_t precision, void *tau,
                                 int32_t *ncross, uint8_t *ray_status, const float *w, int32_t grad_precision,
                                 void *grad_rho, hg_stream stream);
/* Single-pass emission.  hg_rays_trace_stage is hg_rays_trace (w NULL) or
 * hg_rays_trace_gradient (w non-NULL) that also stages every emitted (cell,
 * ds) in a pool owned by the handle: about stage_per_ray entries per ray
 * (0 = 64) plus one 128-entry chunk per walking thread, 16 bytes per entry
 * after an FP64 trace and 8 after an HG_FP32K one, kept until
 * hg_rays_free.  hg_rays_emit_staged then copies each ray's crossings to
 * seg_cell / seg_ds at seg_off (hg_scan_offsets over the staged ncross) --
 * the same arrays hg_rays_fill writes, without a second walk.  When the pool
 * was too small, the copy is skipped and a fill walk (launched either way,
 * returning at once otherwise) does the emission: results never depend on
 * the pool size.  stage_per_ray < 0 makes the pool exactly -stage_per_ray
 * chunks (to exercise that fallback).  ds precision is the staged trace's. */
hg_status hg_rays_trace_stage(hg_rays *r, double kappa, const double *rho, int32_t precision, void *tau,
                              int32_t *ncross, uint8_t *ray_status, const float *w, int32_t grad_precision,
                              void *grad_rho, int32_t stage_per_ray, hg_stream stream);
hg_status hg_rays_emit_staged(hg_rays *r, const int64_t *seg_off, int32_t *seg_cell, void *seg_ds,
                              int64_t seg_capacity, uint8_t *ray_status, hg_stream stream);
/* hg_rays_emit_staged that also accumulates the adjoint of the optical depth
 * (for L = sum_i w_i tau_i, as hg_tau_gradient): grad_rho[c] += kappa w_i ds
 * for every staged crossing of ray i through leaf c -- what hg_rays_gradient
 * adds, taken from the staged lengths in the same pass as the copy instead
 * of a walk (ds as staged: FP32 after an HG_FP32K trace).  Meant after
 * hg_rays_trace_stage with w NULL (with w, the walk has already added the
 * gradient once).  grad_precision 0:
 * grad_rho is double[n_leaves], 1: float[n_leaves]; w is float[n] of device
 * memory; the gradient does not depend on seg_capacity.  When the pool
 * overflowed, a fill walk and a gradient walk do the work instead.  The
 * order of the atomic additions is unspecified. */
hg_status hg_rays_emit_staged_gradient(hg_rays *r, const int64_t *seg_off, int32_t *seg_cell, void *seg_ds,
                                       int64_t seg_capacity, uint8_t *ray_status, double kappa, const float *w,
                                       int32_t grad_precision, void *grad_rho, hg_stream stream);
/* As hg_trace_fill; seg_off from hg_scan_offsets over the ncross of
 * hg_rays_trace (or hg_rays_trace_gradient) on the same rays. */
hg_status hg_rays_fill(hg_rays *r, int32_t precision, const int64_t *seg_off, int32_t *seg_cell, void *seg_ds,
                       int64_t seg_capacity, uint8_t *ray_status, hg_stream stream);
/* As hg_tau_gradient (grad_rho ACCUMULATED). */
hg_status hg_rays_gradient(hg_rays *r, double kappa, const float *w, int32_t grad_precision, void *grad_rho,
                           hg_stream stream);
/* Release the handle; its scratch is freed in order on stream (the stream of
 * its last walk).  NULL is ignored. */
void hg_rays_free(hg_rays *r, hg_stream stream);

/* OR of the per-ray status bits into *out_bits (dev u32, overwritten). */
hg_status hg_reduce_status(int64_t n, const uint8_t *ray_status, uint32_t *out_bits, hg_stream stream);
/* Map OR-ed ray bits to one call-level status (host). */
hg_status hg_status_from_bits(uint32_t bits);

/* ------------------------------------------------------------------------ grid-quality metrics (Sect. 3.2) */
typedef struct hg_dmodel hg_dmodel;

/* Upload a density model for the true density rho_t and true optical depth. */
hg_status hg_load_model(const hg_model *model, hg_dmodel **out);
void hg_free_model(hg_dmodel *m);
/* rho_t at points: pts dev f64[n][3] -> rho dev f64[n]. */
hg_status hg_model_density(const hg_dmodel *m, int64_t n, const double *pts, double *rho, hg_stream stream);
/* tau_t = kappa * integral_0^len rho_t(o + t d) dt by adaptive 15-point
 * Gauss-Kronrod quadrature with breakpoints at the model's kinks and edges,
 * local relative tolerance rtol.  Directions must be unit vectors. */
hg_status hg_model_tau(const hg_dmodel *m, int64_t n, const double *o, const double *d, const double *len,
                       double kappa, double rtol, double *tau, hg_stream stream);
/* Statistics of x = a - b (dev f64[n] each): out dev f64[3] = {n, mean, population std},
 * two passes in FP64 (Delta-rho and Delta-tau are the std of rho_t - rho_g and tau_t - tau_g). */
hg_status hg_diff_stats(int64_t n, const double *a, const double *b, double *out, hg_stream stream);
/* Sum of ncross (dev i32[n]) into *out (dev i64): <N_cross> = *out / n (Sect. 3.2). */
hg_status hg_sum_i32(int64_t n, const int32_t *x, int64_t *out, hg_stream stream);

/* ------------------------------------------------------------------------ batched launch
 * The paper traces paths through one grid at a time (Sect. 2.3); this
 * batched form is this library's own: the optical-depth pass of
 * hg_trace_rays (same contract and results, whole paths, never split) over
 * many grids of uneven size, each with its own ray range, traced in one
 * persistent launch: ray chunks of every grid form one work list that
 * resident blocks drain through an atomic counter, larger grids first.
 * ray_begin (host i64[n_grids+1]) splits the concatenated ray and output
 * arrays by grid.  The batch holds a device table of the grids (which
 * must outlive it) and a reusable work counter; hg_batch_trace may be
 * captured into a CUDA graph once and replayed. */
typedef struct hg_batch hg_batch;
hg_status hg_batch_create(int32_t n_grids, const hg_grid *const *grids, const int64_t *ray_begin,
                          int32_t chunk, hg_batch **out);
void hg_batch_free(hg_batch *b);
hg_status hg_batch_trace(hg_batch *b, const double *o, const double *d, const double *s_max, double kappa,
                         const hg_trace_opts *opts, void *tau, int32_t *ncross, uint8_t *ray_status,
                         hg_stream stream);

/* ------------------------------------------------------------------------ autotuner
 * Time candidate launch configurations (threads per block, shared-memory
 * tree nodes, schedule) on a sample of n rays with CUDA events, keep the
 * fastest for this grid and precision (used when opts fields are 0 / -1),
 * and return it in *best.  Synchronises the stream. */
hg_status hg_autotune(hg_grid *g, int64_t n, const double *o, const double *d, int32_t precision,
                      hg_trace_opts *best, float *best_ms, hg_stream stream);

/* ------------------------------------------------------------------------ misc */
const char *hg_status_str(hg_status s);
const char *hg_last_error(void);
int32_t hg_version(void);
/* Number of kernel launches this library issued in the calling process. */
int64_t hg_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* HGRT_H */
