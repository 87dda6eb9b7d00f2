// Host reference executor and helpers shared by the debug entry points.
#pragma once
#include <cstdint>
#include <vector>

#include "hlu_internal.h"

namespace hlu {

// alpha: the launch scalar of TF_ALPHA tasks and PF_ALPHA pieces
template <class T>
int host_execute(const Schedule& S, T* arena, int32_t* ranks, int32_t* piv, double eps,
                 uint64_t order_seed, int32_t* cap_hits, int64_t limit = -1, double alpha = 0.0);

// Trees from the exported flat layout (clusters: nc x 12, blocks: nb x 8), with
// the leaf ranges filled in.
void trees_from_export(int32_t nc, const int32_t* cl, int32_t nb, const int32_t* bl,
                       std::vector<Cluster>& C, std::vector<Block>& B);
}  // namespace hlu
