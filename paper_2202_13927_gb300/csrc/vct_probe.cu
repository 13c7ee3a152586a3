// vct_probe.cu -- throughput probes that measure the roofline denominators of
// this GPU: FP32 FMA, FP64 FMA, INT32 multiply-add (low and high half), MUFU
// (lg2), packed FP32 FMA (two lanes' worth per instruction, fma.rn.f32x2),
// unsigned-integer-to-float conversion and 32 x 32 -> 64-bit multiply rates.
// Each thread runs eight independent dependency chains so that latency does
// not limit the rate; the result is stored so nothing is optimised away.
#include "vct_internal.cuh"

namespace vct {
namespace {

constexpr int kChains = 8;

__global__ void probe_ffma(int iters, float seed, float *sink) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + threadIdx.x * 1e-7f + c;
  const float m = 0.9999999f, b = 1e-7f;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], m, b);
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 12345.678f) sink[0] = s;
}

__global__ void probe_dfma(int iters, double seed, double *sink) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + threadIdx.x * 1e-7 + c;
  const double m = 0.9999999, b = 1e-7;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], m, b);
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 12345.678) sink[0] = s;
}

__global__ void probe_imad(int iters, uint32_t seed, uint32_t *sink) {
  uint32_t a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + threadIdx.x + 977u * c;
  const uint32_t b = 0x7F4A7C15u;
  // a quadratic recurrence: an affine one could be collapsed by the compiler
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = a[c] * a[c] + b;
  uint32_t s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s ^= a[c];
  if (s == 0x12345678u) sink[0] = s;
}

// the high half of a 32 x 32 multiply, as Philox uses it
__global__ void probe_imad_hi(int iters, uint32_t seed, uint32_t *sink) {
  uint32_t a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + threadIdx.x + 977u * c;
  const uint32_t b = 0x7F4A7C15u;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = __umulhi(a[c], a[c]) + b;
  uint32_t s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s ^= a[c];
  if (s == 0x12345678u) sink[0] = s;
}

__global__ void probe_mufu(int iters, float seed, float *sink) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + threadIdx.x * 1e-3f + c;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = __log2f(a[c] + 2.0f);
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  if (s == 12345.678f) sink[0] = s;
}

// Both halves of a 32 x 32 multiply in one widening multiply (mul.wide.u32),
// as Philox's first product of a round uses it, plus an add of the halves.
__global__ void probe_imad_wide(int iters, uint32_t seed, uint32_t *sink) {
  uint32_t a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + threadIdx.x + 977u * c;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      unsigned long long p;
      asm("mul.wide.u32 %0, %1, %2;" : "=l"(p) : "r"(a[c]), "r"(a[c]));
      a[c] = (uint32_t)(p >> 32) + (uint32_t)p;
    }
  uint32_t s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s ^= a[c];
  if (s == 0x12345678u) sink[0] = s;
}

// Packed FP32 FMA: one instruction does two FMAs on a pair of registers.
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

__global__ void probe_ffma2(int iters, float seed, float *sink) {
  unsigned long long a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c)
    a[c] = ((unsigned long long)__float_as_uint(seed + c) << 32) | __float_as_uint(seed + threadIdx.x * 1e-7f);
  const unsigned long long m = ((unsigned long long)__float_as_uint(0.9999999f) << 32) | __float_as_uint(0.9999999f);
  const unsigned long long b = ((unsigned long long)__float_as_uint(1e-7f) << 32) | __float_as_uint(1e-7f);
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = ffma2(a[c], m, b);
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += __uint_as_float((uint32_t)a[c]) + __uint_as_float((uint32_t)(a[c] >> 32));
  if (s == 12345.678f) sink[0] = s;
}

// Unsigned integer to float conversion (round toward zero), as Box-Muller's
// uniforms use it; the integer chain keeps the conversions independent.
__global__ void probe_i2f(int iters, uint32_t seed, float *sink) {
  uint32_t a[kChains];
  float f[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    a[c] = seed + threadIdx.x + 977u * c;
    f[c] = 0.0f;
  }
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      f[c] = __uint2float_rz(a[c] ^ (uint32_t)i);
      a[c] += __float_as_uint(f[c]);
    }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += f[c];
  if (s == 12345.678f) sink[0] = s;
}

}  // namespace
}  // namespace vct

extern "C" vct_status vct_probe(int32_t kind, int32_t iters, float *ms_out, double *ops_out,
                                void *cuda_stream) {
  if (kind < 0 || kind > 7 || iters < 1 || !ms_out || !ops_out)
    return vct::record_error(VCT_ERR_ARG, "vct_probe: kind 0..7, iters >= 1, outputs required");
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256, blocks = sms * 8;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  void *sink = nullptr;
  cudaError_t e = cudaMallocAsync(&sink, 64, st);
  cudaEvent_t a, b;
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e != cudaSuccess) return vct::record_error(VCT_ERR_CUDA, "vct_probe: setup failed");
  for (int rep = 0; rep < 2; ++rep) {  // the first run warms up
    cudaEventRecord(a, st);
    switch (kind) {
      case 0: vct::probe_ffma<<<blocks, threads, 0, st>>>(iters, 1.0f, (float *)sink); break;
      case 1: vct::probe_dfma<<<blocks, threads, 0, st>>>(iters, 1.0, (double *)sink); break;
      case 2: vct::probe_imad<<<blocks, threads, 0, st>>>(iters, 7u, (uint32_t *)sink); break;
      case 4: vct::probe_imad_hi<<<blocks, threads, 0, st>>>(iters, 7u, (uint32_t *)sink); break;
      case 5: vct::probe_ffma2<<<blocks, threads, 0, st>>>(iters, 1.0f, (float *)sink); break;
      case 6: vct::probe_i2f<<<blocks, threads, 0, st>>>(iters, 7u, (float *)sink); break;
      case 7: vct::probe_imad_wide<<<blocks, threads, 0, st>>>(iters, 7u, (uint32_t *)sink); break;
      default: vct::probe_mufu<<<blocks, threads, 0, st>>>(iters, 1.0f, (float *)sink); break;
    }
    cudaEventRecord(b, st);
  }
  e = cudaEventSynchronize(b);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFreeAsync(sink, st);
  if (e != cudaSuccess) return vct::record_error(VCT_ERR_CUDA, "vct_probe: run failed");
  *ms_out = ms;
  // lane operations: two FMAs per packed instruction (kind 5), one otherwise
  *ops_out = (double)blocks * threads * (double)iters * vct::kChains * (kind == 5 ? 2.0 : 1.0);
  return VCT_OK;
}
