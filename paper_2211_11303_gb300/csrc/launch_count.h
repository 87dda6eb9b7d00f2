// Count of this library's own kernel launches (process-wide), read through
// hlu_launch_count().  Library kernels (e.g. sorts and scans from CUDA's
// bundled templates) are not counted.
#pragma once
#include <atomic>
#include <cstdint>

namespace hlu {
extern std::atomic<int64_t> g_launches;
inline void note_launch(int64_t n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace hlu
