// Internal declarations shared by the library's translation units.
#pragma once

#include <atomic>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "hgrt.h"

namespace hg {

void set_error(const char *fmt, ...);

// Order-preserving integer key of a non-NaN double (host side of the map
// the kernels use): a < b <=> key(a) < key(b), and -0.0 maps like +0.0.
inline long long host_okey(double x) {
    long long b;
    std::memcpy(&b, &x, 8);
    const long long k = b ^ ((b >> 63) & 0x7fffffffffffffffLL);
    return k == -1LL ? 0LL : k;
}
void note_launches(int64_t n);

// Leaf record in HBM: 96 bytes = three 32-byte sectors, so a step that
// enters a leaf fetches exactly three sectors.
//   sector 0: lo.x lo.y lo.z hi.x
//   sector 1: hi.y hi.z rho rho32 nbr_base
//   sector 2: first[6] cnt[6] flags pad
// Bounds are stored as order-preserving integer keys of their FP64 values
// (the sign bit kept, the other bits flipped for negative values, -0 stored
// as +0), so that the kernels compare them with integer instructions.
// first[w] is the head of wall w's neighbor list (the largest overlap,
// Sect. 2.3), -1 when the wall lies on the domain boundary.  cnt[w] is the
// list length, saturated at 255; lists of length 2..scan_limit keep
// entries 1.. in the tail array starting at nbr_base, walls in order.
// flags bit a: hi on axis a equals the domain's upper bound.
struct alignas(32) LeafRec {
    int64_t lo[3];
    int64_t hi[3];
    double rho;
    float rho32;
    uint32_t nbr_base;
    int32_t first[6];
    uint8_t cnt[6];
    uint8_t flags;
    uint8_t pad;
};
static_assert(sizeof(LeafRec) == 96, "leaf record must be three sectors");

// Descent nodes: k-d 16 B, octree 32 B.  Split planes are stored as keys
// like the leaf bounds.  child = first child index in the node list
// (children contiguous) or -1 for a leaf; info/leaf = leaf id for a leaf,
// split axis for an internal k-d node.
struct alignas(16) KdNode {
    int64_t split;
    int32_t child;
    int32_t info;
};
struct alignas(16) OctNode {
    int64_t s[3];
    int32_t child;
    int32_t leaf;
};
static_assert(sizeof(KdNode) == 16 && sizeof(OctNode) == 32, "node sizes");

// What a kernel needs to walk one grid (passed by value).
struct DevGrid {
    const LeafRec *rec;
    const int32_t *tail;
    const void *nodes;
    const float *work;         // [work_n^3] expected crossings per unit length on a coarse lattice
    double dlo[3], dhi[3];
    long long klo[3], khi[3];  // keys of the domain bounds
    int64_t n_leaves;
    int64_t n_nodes;
    int32_t kind;
    int32_t max_depth;
    int32_t scan_limit;
    int32_t work_n;
    int32_t nav;  // HG_NAV_NEIGHBOR_LISTS or HG_NAV_ROPES: what the records' wall slots hold
    int32_t pad;
};

// Coarse lattice of the expected number of leaf crossings per unit path
// length (volume average of S/(4V) over the leaves, Cauchy's mean chord),
// used only to order rays by their estimated work.
constexpr int kWorkN = 16;

struct TuneEntry {
    int valid = 0;
    int block = 0;
    int smem_nodes = 0;
    int schedule = 0;
    int min_blocks = 0;
};

}  // namespace hg

struct hg_grid {
    hg::DevGrid d;
    hg_grid_info info;
    void *d_rec = nullptr;
    void *d_tail = nullptr;
    void *d_nodes = nullptr;
    void *d_work = nullptr;
    int device = 0;
    hg::TuneEntry tuned[2];
};

namespace hg {
// implemented in trace.cu
hg_status resolve_opts(const hg_grid *g, const hg_trace_opts *opts, int &precision, int &block, int &smem_nodes,
                       int &schedule, int &min_blocks, int64_t &max_steps, int &split);
}  // namespace hg
