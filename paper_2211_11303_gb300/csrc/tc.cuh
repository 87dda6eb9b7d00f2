// Fifth-generation tensor core (tcgen05) helpers for sm_103a: tensor-memory
// allocation, shared-memory matrix descriptors, TF32 MMA with the
// accumulator in tensor memory, completion through an mbarrier, and the
// tensor-memory load of the accumulator.  Inline PTX only; used by the task
// executor's tile products (exec.cu).
//
// Operand layout (both operands K-major, no swizzle): a "core matrix" is 8
// rows x 16 bytes (4 TF32 values of one row), stored as 128 contiguous bytes,
// row r at byte 16 r.  In a staged K-chunk of 32 values, core matrix (row
// group i, K group j) sits at byte i * kTcSBO + j * kTcLBO: the descriptor's
// leading-dimension offset is the step between K groups, its stride offset
// the step between 8-row groups.
#pragma once
#include <cstdint>

namespace hlu {
namespace tc {

constexpr uint32_t kTcLBO = 128;   // bytes between core matrices along K
constexpr uint32_t kTcSBO = 1024;  // bytes between 8-row groups (8 K groups x 128 B)
constexpr int kTcChunkK = 32;      // K values staged per chunk (4 MMAs of K = 8)
constexpr int kTcCols = 128;       // tensor-memory columns held per CTA (fp32 accumulator N = 128)
constexpr uint32_t kTcOperandBytes = 128 * kTcChunkK * 4;  // one staged operand: 128 rows x 32 K
constexpr uint32_t kTcStageBytes = 2 * kTcOperandBytes;    // A and B

// byte offset of element (row, k) of a staged K-major operand chunk
__device__ __forceinline__ uint32_t tc_offset(int row, int k) {
  return (uint32_t)(row >> 3) * kTcSBO + (uint32_t)(k >> 2) * kTcLBO + (uint32_t)(row & 7) * 16u +
         (uint32_t)(k & 3) * 4u;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory descriptor: start address, LBO and SBO in 16-byte units,
// the fixed version field (bit 46), no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((kTcLBO >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((kTcSBO >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor of kind::tf32: D in FP32, A and B TF32, both
// K-major, M = 128, N = 128.
constexpr uint32_t kIdescTf32 = (1u << 4)              // D format: F32
                                | (2u << 7)            // A format: TF32
                                | (2u << 10)           // B format: TF32
                                | ((128u >> 3) << 17)  // N / 8
                                | ((128u >> 4) << 24); // M / 16

// round to the nearest TF32 value (kept in a 32-bit register)
__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// --- tensor memory ---------------------------------------------------------
// all 32 lanes of one warp; the allocated address is written to *dst (shared)
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes made visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// D[taddr] (+)= A * B^T for one K = 8 step; one thread issues
__device__ __forceinline__ void mma_tf32(uint32_t taddr, uint64_t adesc, uint64_t bdesc, bool accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(taddr),
      "l"(adesc), "l"(bdesc), "r"(kIdescTf32), "r"((uint32_t)accumulate)
      : "memory");
}
// the mbarrier at `bar` receives one arrival when every MMA issued so far by
// this thread has completed
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// --- mbarrier ----------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// --- tensor memory -> registers ------------------------------------------------
// 32 lanes x 32 consecutive 32-bit columns: thread t of the warp receives lane
// (taddr lane + t), columns taddr col .. +31.  The warp must own the lane
// quarter (warp index mod 4).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace tc
}  // namespace hlu
