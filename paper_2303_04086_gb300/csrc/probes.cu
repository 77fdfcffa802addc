// Microbenchmarks for the roofline denominators not covered by the measured
// HBM copy and BF16 GEMM figures: L2 streaming read, L2 random 8-byte reads
// (the access pattern of the PSH gather once its tables are cached) and the
// packed FP32 FMA rate of the SIMT MLP.  Each loop is bounded by its
// arguments; nothing waits on anything.
#include <cuda_runtime.h>

#include <cstdint>

#include "inolf_internal.h"

namespace inolf {
namespace {

constexpr uint32_t kProbeBytes = 32u << 20;  // L2-resident on a 129 MB L2
constexpr int kProbeThreads = 256;
constexpr uint32_t kSinkMagic = 0x9e3779b9u;

__global__ void __launch_bounds__(kProbeThreads) k_probe_l2_read(const uint4* __restrict__ buf, uint32_t n16,
                                                                 int reps, uint32_t* sink) {
  uint32_t acc = 0;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (int r = 0; r < reps; ++r) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n16; i += 4 * stride) {
      const uint4 a = __ldcg(buf + i), b = __ldcg(buf + i + stride), c = __ldcg(buf + i + 2 * stride),
                  d = __ldcg(buf + i + 3 * stride);
      acc ^= (a.x ^ a.w) + (b.y ^ b.z) + (c.x ^ c.y) + (d.z ^ d.w);
    }
    for (; i < n16; i += stride) {
      const uint4 a = __ldcg(buf + i);
      acc ^= a.x ^ a.y ^ a.z ^ a.w;
    }
  }
  if (acc == kSinkMagic) sink[0] = acc;  // keeps the loads
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_l2_gather(const uint2* __restrict__ buf, uint32_t mask,
                                                                   int iters, uint32_t* sink) {
  uint32_t x = (blockIdx.x * blockDim.x + threadIdx.x) * 0x9E3779B1u + 0x7F4A7C15u;
  uint32_t acc = 0;
  for (int it = 0; it < iters; ++it) {
    uint32_t idx[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {  // xorshift32 (Marsaglia 2003)
      x ^= x << 13;
      x ^= x >> 17;
      x ^= x << 5;
      idx[q] = x & mask;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint2 v = __ldcg(buf + idx[q]);
      acc += v.x ^ v.y;
    }
  }
  if (acc == kSinkMagic) sink[0] = acc;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_fma(float* out, int iters, float a, float b) {
  // 8 independent packed chains c = c * a + b (two FP32 lanes each)
  uint64_t c[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float v = (float)(threadIdx.x + q);
    c[q] = ((uint64_t)__float_as_uint(v + 0.5f) << 32) | __float_as_uint(v);
  }
  const uint64_t av = ((uint64_t)__float_as_uint(a) << 32) | __float_as_uint(a);
  const uint64_t bv = ((uint64_t)__float_as_uint(b) << 32) | __float_as_uint(b);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < 8; ++q) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(c[q]) : "l"(av), "l"(bv));
  }
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < 8; ++q) s += __uint_as_float((uint32_t)c[q]) + __uint_as_float((uint32_t)(c[q] >> 32));
  if (s == -1.0f) out[0] = s;  // keeps the chains
}

// Device time of one launch of `launch` (after one untimed launch).
template <class F>
float time_launch(cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, F&& launch) {
  launch();
  cudaEventRecord(e0, st);
  launch();
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  return ms;
}

}  // namespace
}  // namespace inolf

extern "C" inolf_status inolf_probe_peaks(inolf_peaks* out, void* stream) {
  using namespace inolf;
  clear_error();
  if (!out) return fail(INOLF_E_INVALID, "inolf_probe_peaks: out is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
    return fail(INOLF_E_CUDA, "inolf_probe_peaks: no device");
  void* buf = nullptr;
  uint32_t* sink = nullptr;
  if (cudaMalloc(&buf, kProbeBytes) != cudaSuccess) return fail(INOLF_E_CUDA, "inolf_probe_peaks: cudaMalloc failed");
  if (cudaMalloc(&sink, 64) != cudaSuccess) {
    cudaFree(buf);
    return fail(INOLF_E_CUDA, "inolf_probe_peaks: cudaMalloc failed");
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaMemsetAsync(buf, 0x5a, kProbeBytes, st);
  const unsigned grid = (unsigned)sms * 8u;
  const uint32_t n16 = kProbeBytes / 16u;
  const int reps = 64;
  const float ms_read = time_launch(st, e0, e1, [&] {
    k_probe_l2_read<<<grid, kProbeThreads, 0, st>>>((const uint4*)buf, n16, reps, sink);
  });
  const int iters = 256;
  const uint32_t mask = kProbeBytes / 8u - 1u;  // power of two
  const float ms_gather = time_launch(st, e0, e1, [&] {
    k_probe_l2_gather<<<grid, kProbeThreads, 0, st>>>((const uint2*)buf, mask, iters, sink);
  });
  const int fiters = 4096;
  const float ms_fma = time_launch(st, e0, e1, [&] {
    k_probe_fma<<<grid, kProbeThreads, 0, st>>>((float*)sink, fiters, 0.999f, 1e-3f);
  });
  const cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  cudaFree(buf);
  if (err != cudaSuccess || !(ms_read > 0.f) || !(ms_gather > 0.f) || !(ms_fma > 0.f))
    return fail(INOLF_E_CUDA, "inolf_probe_peaks: a probe launch failed");
  const double threads = (double)grid * kProbeThreads;
  out->l2_read_gbs = (double)kProbeBytes * reps / (ms_read * 1e-3) / 1e9;
  out->l2_gather_gsps = threads * iters * 8.0 / (ms_gather * 1e-3) / 1e9;
  out->fp32_tflops = threads * fiters * 8.0 * 2.0 * 2.0 / (ms_fma * 1e-3) / 1e12;
  return INOLF_OK;
}
