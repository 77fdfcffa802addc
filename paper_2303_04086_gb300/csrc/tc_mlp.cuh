// Layers 1-3 of the MLP F_s on the tensor cores for 2 x 128 rows whose A1
// operand rows are already in shared memory (shared by the render and serve
// kernels).  256 threads; thread tid owns row tid & 127 of tile tid >> 7.
// sB3 holds W3 as a 16-row operand (rows 4..15 zero: N = 16 is the smallest
// N of an M = 128 MMA), K-major like W2.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "kernels_common.cuh"
#include "tc_ptx.cuh"

namespace inolf {

static constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s: the MMAs of a tile take microseconds

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ uint16_t pack_fp8(float a, float b) {
  return (uint16_t)__nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
}
__device__ __forceinline__ float round_bf16(float a) { return __bfloat162float(__float2bfloat16_rn(a)); }
__device__ __forceinline__ float round_fp8(float a) {
  __half_raw h = __nv_cvt_fp8_to_halfraw(__nv_cvt_float_to_fp8(a, __NV_SATFINITE, __NV_E4M3), __NV_E4M3);
  return __half2float(__half(h));
}

// stores the pair (a, b) of input column k (even) of row `row`
template <bool kFP8>
__device__ __forceinline__ void store_pair(uint8_t* A, uint32_t row, uint32_t k, uint32_t chunks, float a, float b,
                                           float inv_scale) {
  if (kFP8) {
    const uint32_t off = tc::core_off(row, k >> 4, chunks) + (k & 15u);
    *reinterpret_cast<uint16_t*>(A + off) = pack_fp8(a * inv_scale, b * inv_scale);
  } else {
    const uint32_t off = tc::core_off(row, k >> 3, chunks) + (k & 7u) * 2u;
    *reinterpret_cast<uint32_t*>(A + off) = pack_bf16(a, b);
  }
}

// Writes one row of an A operand tile as consecutive column pairs from column
// 0 on, storing each 16-byte chunk (8 BF16 or 16 FP8 values) when it is
// complete: one 16-byte store per chunk instead of one store per pair, and a
// warp's stores fill whole core matrices (no shared-memory bank conflicts).
template <bool kFP8>
struct RowWriter {
  uint8_t* A;
  uint32_t row, chunks, n;  // n = pairs pushed so far
  uint32_t w0, w1, w2, w3;
  float inv_s;

  __device__ __forceinline__ RowWriter(uint8_t* A_, uint32_t row_, uint32_t chunks_, float inv_s_)
      : A(A_), row(row_), chunks(chunks_), n(0), w0(0), w1(0), w2(0), w3(0), inv_s(inv_s_) {}

  __device__ __forceinline__ void push(float a, float b) {
    if (kFP8) {  // 2-byte pairs shift through the 16-byte chunk
      const uint32_t v = pack_fp8(a * inv_s, b * inv_s);
      w0 = (w0 >> 16) | (w1 << 16);
      w1 = (w1 >> 16) | (w2 << 16);
      w2 = (w2 >> 16) | (w3 << 16);
      w3 = (w3 >> 16) | (v << 16);
      if ((++n & 7u) == 0) flush((n >> 3) - 1u);
    } else {
      w0 = w1;
      w1 = w2;
      w2 = w3;
      w3 = pack_bf16(a, b);
      if ((++n & 3u) == 0) flush((n >> 2) - 1u);
    }
  }
  // two consecutive pairs at once; the count of pairs pushed so far must be
  // even (the words then hold whole 32-bit column groups, so no shifting)
  __device__ __forceinline__ void push2(float a0, float b0, float a1, float b1) {
    if (kFP8) {
      const uint32_t v =
          (uint32_t)pack_fp8(a0 * inv_s, b0 * inv_s) | ((uint32_t)pack_fp8(a1 * inv_s, b1 * inv_s) << 16);
      w0 = w1;
      w1 = w2;
      w2 = w3;
      w3 = v;
      n += 2;
      if ((n & 7u) == 0) flush((n >> 3) - 1u);
    } else {
      w0 = w2;
      w1 = w3;
      w2 = pack_bf16(a0, b0);
      w3 = pack_bf16(a1, b1);
      n += 2;
      if ((n & 3u) == 0) flush((n >> 2) - 1u);
    }
  }
  __device__ __forceinline__ void flush(uint32_t c) {
    *reinterpret_cast<uint4*>(A + tc::core_off(row, c, chunks)) = make_uint4(w0, w1, w2, w3);
  }
  // zero pairs up to column K (a multiple of the chunk width).  FP8 rows pad
  // whole chunks (K rounds up to 32 columns): the open chunk is completed
  // pair by pair, the chunks after it are stored as zeros at once.
  __device__ __forceinline__ void pad_to(uint32_t K) {
    if constexpr (kFP8) {
      while ((n & 7u) != 0u) push(0.f, 0.f);
      for (; 2u * n < K; n += 8u) {
        w0 = w1 = w2 = w3 = 0u;
        flush(n >> 3);
      }
    } else {
      while (2u * n < K) push(0.f, 0.f);
    }
  }
};

// Precision-dependent scales (FP8: per-tensor, amax / 448; BF16: unit).
// A layer's accumulator dequantises with mul = s_in s_w and the next layer's
// input quantises with 1 / s_next; both are positive, so ReLU commutes with
// them and the two multiplications fold into one (q1, q2).  The last layer's
// input scale sh2 is applied once to the 4 dot products instead of to each of
// the 64 inputs.
struct TcScales {
  float inv_sx, q1, q2, o3;
  __device__ static TcScales make(bool fp8, const float act[3], const float w[3]) {
    TcScales s;
    s.inv_sx = fp8 ? 1.0f / act[0] : 1.0f;
    s.q1 = fp8 ? (act[0] * w[0]) / act[1] : 1.0f;
    s.q2 = fp8 ? (act[1] * w[1]) / act[2] : 1.0f;
    s.o3 = fp8 ? act[2] * w[2] : 1.0f;  // dequantises the last layer's accumulator
    return s;
  }
};

// Steps after the A1 rows are written: D1 = A1 W1^T (tcgen05, TMEM), ReLU and
// quantisation into A2 (in place of A1), D2 = A2 W2^T, ReLU and quantisation
// into A3 (in place of A2), D3 = A3 W3^T (N = 16, the 4 outputs in columns
// 0..3) and sigmoid.  Every thread of the CTA must call it; `out` receives
// the thread's row.  Returns false (uniformly) when an MMA completion wait ran
// out.
template <bool kFP8>
__device__ __forceinline__ bool tc_mlp_run(uint8_t* sA, const uint8_t* sB1, const uint8_t* sB2, const uint8_t* sB3,
                                           uint32_t K1, uint32_t tmem, uint64_t* bar, uint32_t& phase,
                                           const TcScales& sc, float4& out) {
  constexpr uint32_t ES = kFP8 ? 1u : 2u;
  constexpr uint32_t KSTEP_CHUNKS = 2;  // one MMA consumes 32 bytes of K per row
  constexpr uint32_t tile_bytes = 128u * 64u * ES;
  const uint32_t chunks1 = K1 * ES / 16u, chunks2 = 64u * ES / 16u;
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t t = (uint32_t)tid >> 7, row = (uint32_t)tid & 127u;
  uint8_t* A = sA + t * tile_bytes;
  const uint32_t lane_base = ((uint32_t)(warp & 3) * 32u) << 16;
  const uint32_t fmt = kFP8 ? 0u : 1u;
  const uint32_t id = tc::idesc(128, 64, fmt), id3 = tc::idesc(128, 16, fmt);
  // D (+)= A B^T for both tiles (thread 0), committed to `bar`, then waited for
  auto mma = [&](const uint8_t* sB, uint32_t chunks, uint32_t idesc) -> bool {
    if (tid == 0) {
      tc::fence_after();
      for (uint32_t tt = 0; tt < 2; ++tt) {
        const uint32_t a0 = tc::smem_u32(sA + tt * tile_bytes), b0 = tc::smem_u32(sB);
        for (uint32_t s = 0; s < chunks / KSTEP_CHUNKS; ++s) {
          const uint64_t ad = tc::desc_kmajor(a0 + s * 256u, 128u, chunks * 128u);
          const uint64_t bd = tc::desc_kmajor(b0 + s * 256u, 128u, chunks * 128u);
          if (kFP8) tc::mma_fp8(tmem + tt * 64u, ad, bd, idesc, s > 0);
          else tc::mma_bf16(tmem + tt * 64u, ad, bd, idesc, s > 0);
        }
      }
      tc::mma_commit(bar);
    }
    const bool ok = tc::mbar_wait(bar, phase, kWaitLimitNs);
    phase ^= 1u;
    if (__syncthreads_or(!ok)) return false;
    tc::fence_after();
    return true;
  };
  // this thread's TMEM row (64 columns) -> ReLU (FP8: times `scale`, then
  // quantised) -> the next layer's A operand row, in place
  auto next_input = [&](float scale) {
#pragma unroll 1
    for (uint32_t c = 0; c < 4; ++c) {
      float v[16];
      tc::tmem_ld16(tmem + lane_base + t * 64u + c * 16u, v);
      if (kFP8) {
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float a0 = fmaxf(v[4 * q + 0] * scale, 0.f);
          const float a1 = fmaxf(v[4 * q + 1] * scale, 0.f);
          const float a2 = fmaxf(v[4 * q + 2] * scale, 0.f);
          const float a3 = fmaxf(v[4 * q + 3] * scale, 0.f);
          w[q] = (uint32_t)pack_fp8(a0, a1) | ((uint32_t)pack_fp8(a2, a3) << 16);
        }
        *reinterpret_cast<uint4*>(A + tc::core_off(row, c, chunks2)) = make_uint4(w[0], w[1], w[2], w[3]);
      } else {
        uint32_t w[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) w[q] = pack_bf16(fmaxf(v[2 * q], 0.f), fmaxf(v[2 * q + 1], 0.f));
        *reinterpret_cast<uint4*>(A + tc::core_off(row, 2 * c, chunks2)) = make_uint4(w[0], w[1], w[2], w[3]);
        *reinterpret_cast<uint4*>(A + tc::core_off(row, 2 * c + 1, chunks2)) = make_uint4(w[4], w[5], w[6], w[7]);
      }
    }
    tc::fence_before();
    tc::fence_async_smem();
    __syncthreads();
  };
  tc::fence_async_smem();
  __syncthreads();
  if (!mma(sB1, chunks1, id)) return false;  // D1 = A1 W1^T
  next_input(sc.q1);                         // A2
  if (!mma(sB2, chunks2, id)) return false;  // D2 = A2 W2^T
  next_input(sc.q2);                         // A3
  if (!mma(sB3, chunks2, id3)) return false; // D3 = A3 W3^T (columns 0..3)
  float v[16];
  tc::tmem_ld16(tmem + lane_base + t * 64u, v);
  out = make_float4(sigmoidf_(v[0] * sc.o3), sigmoidf_(v[1] * sc.o3), sigmoidf_(v[2] * sc.o3),
                    sigmoidf_(v[3] * sc.o3));
  tc::fence_before();
  __syncthreads();
  return true;
}

}  // namespace inolf
