// Device memory of the library: every allocation of handles, factors,
// workspaces and build temporaries goes through dev_alloc / dev_free, which
// call the allocator set by hlu_set_allocator (default cudaMalloc/cudaFree),
// keep a count of the bytes in use, and refuse an allocation that would take
// that count past the limit set by hlu_set_device_memory_limit.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace hlu {

cudaError_t dev_alloc(void** p, size_t bytes);  // cudaErrorMemoryAllocation when refused
cudaError_t dev_free(void* p);                  // NULL is a no-op
// dev_free for a block that only work queued on stream s used: a
// caller-supplied allocator gets it back once s has drained (cudaFree
// itself waits for the whole device)
cudaError_t dev_free_on(void* p, cudaStream_t s);
int64_t dev_bytes_in_use();
bool dev_custom_allocator();

template <class T>
inline cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_alloc(reinterpret_cast<void**>(p), bytes);
}

// Allocator for thrust's temporary storage (thrust::cuda::par(a).on(s)).
struct ThrustAlloc {
  typedef char value_type;
  char* allocate(std::ptrdiff_t n);  // throws std::bad_alloc when refused
  void deallocate(char* p, size_t n);
};

}  // namespace hlu
