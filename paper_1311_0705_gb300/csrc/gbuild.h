// The tree construction's device parts (gbuild.cu), called by the builder in
// build.cpp: the Monte Carlo node evaluation of one level of the node list,
// and the neighbor lists of a finished node list (host arrays in and out).
#pragma once

#include <cstdint>
#include <vector>

#include "hgrt.h"

namespace hg {
struct ModelView;
struct NodeStats;
struct GpuNodeEval;
hg_status gpu_eval_create(const ModelView &host_model, hg_stream stream, GpuNodeEval **out);
hg_status gpu_eval_level(GpuNodeEval *E, const hg_build_params &P, int64_t n, const int32_t *lvl, const int64_t *idx,
                         NodeStats *out);
void gpu_eval_free(GpuNodeEval *E);

// Neighbor lists of every leaf wall (walls -x, +x, -y, +y, -z, +z), as the
// host builder defines them: the leaves across the wall overlapping it with
// positive area, sorted by decreasing overlap area, ties by ascending leaf
// id.  lvl, idx: [3 n_nodes]; child, leaf: [n_nodes]; leaf_node: [n_leaves].
hg_status gpu_build_neighbors(int32_t kind, int64_t n_nodes, int64_t n_leaves, const int32_t *lvl,
                              const int64_t *idx, const int32_t *child, const int32_t *leaf, const int64_t *leaf_node,
                              hg_stream stream, std::vector<int64_t> &nbr_off, std::vector<int32_t> &nbr_id);
}  // namespace hg
