// vct_tc.cuh -- 5th-generation tensor-core (tcgen05) building blocks shared by
// the surrogate's kernels: the canonical K-major shared-memory layout and its
// matrix descriptor, the kind::f16 instruction descriptor, MMA issue and commit,
// bounded mbarrier waits, TMEM loads and stores, and the fences that hand
// shared memory to the tensor cores.
//
// MMAs are issued by a whole converged warp: every lane runs the issue code and
// the lane chosen by elect.sync (the same lane for the warp's lifetime) carries
// the predicate that issues each tcgen05.mma and tcgen05.commit.  Issued this
// way an M = 128, N = 16 MMA with A in tensor memory costs about 13 cycles of
// issue, against about 50 from one thread of a diverged warp (measured on
// GB300 with a burst of 64 MMAs and clock64); for N = 256 both are bound by the
// tensor core's 128 cycles.
//
// Operands in shared memory use the canonical K-major layout without swizzle:
// element (r, k) of an R x K operand sits at (r/8)(16 K) + (k/8) 128 + (r%8) 16
// + (k%8) 2 bytes, i.e. 8 x 16-byte core matrices, contiguous along K.
#pragma once
#include <cstdint>

namespace vct {
namespace {

// Waits: each try_wait may suspend the thread up to kSuspendNs until the phase
// completes (so waiting warps do not spin on the issue slots), at most
// kWaitLimit of them (about two seconds in all).
constexpr long kWaitLimit = 1L << 11;
constexpr uint32_t kSuspendNs = 1000000;

__device__ __forceinline__ uint32_t cm_off(int r, int k, int K) {
  return (uint32_t)((r >> 3) * (K * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, int K) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((128u >> 4) & 0x3FFF) << 16;                // K-direction core-matrix step
  d |= (uint64_t)(((uint32_t)(K * 16) >> 4) & 0x3FFF) << 32;  // 8-row group step
  d |= (uint64_t)1 << 46;                                      // descriptor version
  return d;                                                    // no swizzle, base offset 0
}

// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// 1 in the lane elect.sync chooses, 0 elsewhere (all 32 lanes must execute it)
__device__ __forceinline__ uint32_t elect_one() {
  uint32_t pred = 0;
  asm volatile("{\n .reg .pred P;\n elect.sync _|P, 0xffffffff;\n selp.u32 %0, 1, 0, P;\n}\n" : "=r"(pred));
  return pred;
}

// D (+)= A B^T, issued by the lanes whose `issue` is nonzero
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t da, uint64_t db, uint32_t idesc,
                                    uint32_t accumulate, uint32_t issue) {
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.b32 p, %4, 0;\n setp.ne.b32 q, %5, 0;\n"
      " @q tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(accumulate), "r"(issue));
}

// The same with the A operand in tensor memory (rows = lanes, BF16 pairs per column).
__device__ __forceinline__ void mma_ta(uint32_t d_tmem, uint32_t a_tmem, uint64_t db, uint32_t idesc,
                                       uint32_t accumulate, uint32_t issue) {
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.b32 p, %4, 0;\n setp.ne.b32 q, %5, 0;\n"
      " @q tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(db), "r"(idesc), "r"(accumulate), "r"(issue));
}

// The mbarrier's arrive once every MMA the issuing lane has issued is complete.
__device__ __forceinline__ void commit(uint32_t bar, uint32_t issue) {
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.b32 q, %1, 0;\n"
      " @q tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(bar),
      "r"(issue));
}

// Bounded wait of a whole warp for an mbarrier phase; every lane polls (and so
// acquires), the warp agrees on the outcome.  A wait that runs out, or finds
// the CTA's abort flag set, returns false and sets the flag for everyone.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t phase, volatile int *abort) {
  uint32_t done = 0;
  for (long it = 0; it < kWaitLimit && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase), "r"(kSuspendNs));
    if (!done && *abort) break;
  }
  const bool ok = __all_sync(0xffffffffu, done != 0);
  if (!ok) *abort = 1;
  asm volatile("tcgen05.fence::after_thread_sync;");
  return ok;
}

// The same without the suspend hint, for short waits (a few MMAs): every lane
// polls with plain try_wait (which returns after a brief system-dependent
// time), at most kSpinLimit times.
constexpr long kSpinLimit = 1L << 22;
__device__ __forceinline__ bool warp_wait_spin(uint32_t bar, uint32_t phase, volatile int *abort) {
  uint32_t done = 0;
  for (long it = 0; it < kSpinLimit && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase));
    if (!done && *abort) break;
  }
  const bool ok = __all_sync(0xffffffffu, done != 0);
  if (!ok) *abort = 1;
  asm volatile("tcgen05.fence::after_thread_sync;");
  return ok;
}

// A warp hands its part of a buffer on: its shared-memory writes become
// visible to the tensor cores' proxy, its TMEM reads and writes are complete,
// then lane 0 arrives on the mbarrier (count = the number of epilogue warps).
__device__ __forceinline__ void warp_arrive(uint32_t bar) {
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncwarp();
  if ((threadIdx.x & 31) == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t r[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n"
      "tcgen05.wait::st.sync.aligned;\n" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
      "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]));
}

// Loads and stores that do not wait: issue several, then one tcgen05.wait.
// wait_ld passes the loaded registers through an empty asm after the wait, so
// that no use of them is scheduled before it.
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t r[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld32(uint32_t r[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) asm volatile("" : "+r"(r[j]));
}

__device__ __forceinline__ void tmem_st16_nowait(uint32_t taddr, const uint32_t r[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n"
      ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
      : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Make this thread's shared-memory writes visible to the tensor cores, then
// meet at the block barrier.
__device__ __forceinline__ void publish_smem() {
  asm volatile("tcgen05.fence::before_thread_sync;");
  asm volatile("fence.proxy.async.shared::cta;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
}

}  // namespace
}  // namespace vct
