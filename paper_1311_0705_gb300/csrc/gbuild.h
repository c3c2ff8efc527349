// The tree construction on the device (gbuild.cu), called by the builder in
// build.cpp.
#pragma once

#include <cstdint>
#include <vector>

#include "hgrt.h"

namespace hg {
struct ModelView;

// A node list as the host builder stores it (per node: levels and indices
// [3], bounds [3], first child or -1, leaf id or -1, statistics; per leaf:
// its node and density; neighbor lists in CSR over the 6 walls of each leaf).
struct GpuTree {
    std::vector<int32_t> lvl, child, leaf, nbr_id;
    std::vector<int64_t> idx, leaf_node, nbr_off;
    std::vector<double> lo, hi, rho, mass, delta, tau, q, leaf_rho;
};

// The whole construction on the device: per level of the breadth-first node
// list, the Monte Carlo node evaluation (one thread per node), a scan of the
// child counts and the children appended in parent order; then the leaf
// numbering, the bounds and the neighbor lists; one copy to the host at the
// end.  The same node list as the host builder's level loop.
hg_status gpu_build_tree(const ModelView &host_model, const hg_build_params &P, hg_stream stream, GpuTree &out);

}  // namespace hg
