// Device memory accounting and the caller-settable allocator (devmem.h).
#include "devmem.h"

#include <mutex>
#include <new>
#include <unordered_map>

#include "../../include/hlu.h"

namespace hlu {
namespace {

struct Alloc {
  hlu_alloc_fn alloc = nullptr;  // null: cudaMalloc / cudaFree
  hlu_free_fn free = nullptr;
  void* ctx = nullptr;
};
struct Live {
  size_t bytes;
  Alloc by;  // the allocator that returned the block frees it
};

std::mutex g_mu;
Alloc g_alloc;
int64_t g_in_use = 0;
int64_t g_limit = 0;  // 0: no limit
std::unordered_map<void*, Live> g_live;

}  // namespace

cudaError_t dev_alloc(void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 1;
  Alloc a;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_limit > 0 && g_in_use + (int64_t)bytes > g_limit) return cudaErrorMemoryAllocation;
    a = g_alloc;
  }
  void* q = nullptr;
  if (a.alloc) {
    q = a.alloc(bytes, a.ctx);
    if (!q) return cudaErrorMemoryAllocation;
  } else {
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) return e;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  g_live[q] = Live{bytes, a};
  g_in_use += (int64_t)bytes;
  *p = q;
  return cudaSuccess;
}

static cudaError_t free_impl(void* p, bool whole_device, cudaStream_t s) {
  if (!p) return cudaSuccess;
  Live l{0, Alloc()};
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_live.find(p);
    if (it == g_live.end()) return cudaFree(p);  // not ours: plain CUDA memory
    l = it->second;
    g_in_use -= (int64_t)l.bytes;
    g_live.erase(it);
  }
  if (l.by.free) {
    // the caller's allocator may hand the block out again at once: no kernel
    // of this library may still use it
    cudaError_t e = whole_device ? cudaDeviceSynchronize() : cudaStreamSynchronize(s);
    l.by.free(p, l.bytes, l.by.ctx);
    return e;
  }
  return cudaFree(p);
}

cudaError_t dev_free(void* p) { return free_impl(p, true, nullptr); }
cudaError_t dev_free_on(void* p, cudaStream_t s) { return free_impl(p, false, s); }

int64_t dev_bytes_in_use() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_in_use;
}

bool dev_custom_allocator() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_alloc.alloc != nullptr;
}

char* ThrustAlloc::allocate(std::ptrdiff_t n) {
  void* p = nullptr;
  if (dev_alloc(&p, (size_t)n) != cudaSuccess) throw std::bad_alloc();
  return static_cast<char*>(p);
}
void ThrustAlloc::deallocate(char* p, size_t) { dev_free(p); }

}  // namespace hlu

extern "C" {

int hlu_set_allocator(hlu_alloc_fn alloc, hlu_free_fn free, void* ctx) {
  if ((alloc == nullptr) != (free == nullptr)) return HLU_ERR_ARG;
  std::lock_guard<std::mutex> lk(hlu::g_mu);
  hlu::g_alloc.alloc = alloc;
  hlu::g_alloc.free = free;
  hlu::g_alloc.ctx = ctx;
  return HLU_OK;
}

int hlu_set_device_memory_limit(int64_t bytes) {
  if (bytes < 0) return HLU_ERR_ARG;
  std::lock_guard<std::mutex> lk(hlu::g_mu);
  hlu::g_limit = bytes;
  return HLU_OK;
}

int64_t hlu_device_bytes_in_use(void) { return hlu::dev_bytes_in_use(); }

}  // extern "C"
