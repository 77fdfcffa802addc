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

// Operand kinds of the tensor-core MLP: BF16 (kind::f16), FP8 e4m3
// (kind::f8f6f4) and FP32, whose products run on the tensor cores as split
// TF32 (kind::tf32, three products per K step; see tc_mlp_run_tf32).
enum : int { kOpBF16 = 0, kOpFP8 = 1, kOpF32 = 2 };

// Bytes per operand element of each kind.
template <int kOp>
__host__ __device__ constexpr uint32_t op_bytes() {
  return kOp == kOpFP8 ? 1u : (kOp == kOpF32 ? 4u : 2u);
}

// x rounded to the nearest TF32 value (10 explicit mantissa bits, ties away
// from zero: the magnitude's bit 12 is added before the low 13 bits are
// cleared), for finite x.  The host packs the weights with the same integer
// steps, so host and device splits agree bit for bit.
__host__ __device__ __forceinline__ uint32_t tf32_rna_bits(uint32_t u) { return (u + 0x1000u) & 0xFFFFE000u; }

// stores the pair (a, b) of input column k (even) of row `row`
template <int kOp>
__device__ __forceinline__ void store_pair(uint8_t* A, uint32_t row, uint32_t k, uint32_t chunks, float a, float b,
                                           float inv_scale) {
  if (kOp == kOpFP8) {
    const uint32_t off = tc::core_off(row, k >> 4, chunks) + (k & 15u);
    *reinterpret_cast<uint16_t*>(A + off) = pack_fp8(a * inv_scale, b * inv_scale);
  } else if (kOp == kOpF32) {
    const uint32_t off = tc::core_off(row, k >> 2, chunks) + (k & 3u) * 4u;
    *reinterpret_cast<float2*>(A + off) = make_float2(a, b);
  } else {
    const uint32_t off = tc::core_off(row, k >> 3, chunks) + (k & 7u) * 2u;
    *reinterpret_cast<uint32_t*>(A + off) = pack_bf16(a, b);
  }
}

// Writes one row of an A operand tile as consecutive column pairs from column
// 0 on, storing each 16-byte chunk (8 BF16, 16 FP8 or 4 FP32 values) when it
// is complete: one 16-byte store per chunk instead of one store per pair, and
// a warp's stores fill whole core matrices (no shared-memory bank conflicts).
template <int kOp>
struct RowWriter {
  static constexpr bool kFP8 = kOp == kOpFP8, kF32 = kOp == kOpF32;
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
    } else if (kF32) {  // 8-byte pairs, two per chunk
      w0 = w2;
      w1 = w3;
      w2 = __float_as_uint(a);
      w3 = __float_as_uint(b);
      if ((++n & 1u) == 0) flush((n >> 1) - 1u);
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
    } else if (kF32) {  // exactly one chunk
      w0 = __float_as_uint(a0);
      w1 = __float_as_uint(b0);
      w2 = __float_as_uint(a1);
      w3 = __float_as_uint(b1);
      n += 2;
      flush((n >> 1) - 1u);
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

// FP32 operands on the tensor cores as split TF32: every FP32 value x is
// held as hi = tf32(x) and lo = tf32(x - hi) (x - hi is exact in FP32), and
// each product A W^T as A_lo W_hi^T + A_hi W_lo^T + A_hi W_hi^T (kind::tf32,
// FP32 accumulation in tensor memory); the dropped A_lo W_lo^T and the
// roundings of the lo parts are below 2^-21 of each product, so the layers
// keep FP32-level accuracy (the published 3xTF32 scheme).
__device__ __forceinline__ void split_tf32(uint4 v, uint4& hi, uint4& lo) {
  hi.x = tf32_rna_bits(v.x);
  hi.y = tf32_rna_bits(v.y);
  hi.z = tf32_rna_bits(v.z);
  hi.w = tf32_rna_bits(v.w);
  lo.x = tf32_rna_bits(__float_as_uint(__uint_as_float(v.x) - __uint_as_float(hi.x)));
  lo.y = tf32_rna_bits(__float_as_uint(__uint_as_float(v.y) - __uint_as_float(hi.y)));
  lo.z = tf32_rna_bits(__float_as_uint(__uint_as_float(v.z) - __uint_as_float(hi.z)));
  lo.w = tf32_rna_bits(__float_as_uint(__uint_as_float(v.w) - __uint_as_float(hi.w)));
}

// Barrier of the 128 threads of pipeline `id - 1` (named barrier `id`).
__device__ __forceinline__ void pipe_sync(uint32_t id) { asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory"); }
// The same barrier, returning whether `v` held in any of its threads.
__device__ __forceinline__ bool pipe_or(uint32_t id, bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, %2, 128, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(id)
      : "memory");
  return r != 0;
}

// One pipeline of 128 threads (4 warps; thread i owns row i & 127 of its
// tile and tensor-memory lane (warp & 3) * 32 + lane): the three layers of
// one 128-row tile whose raw FP32 A1 rows (K1 columns, K1 a multiple of 8)
// sit in Ah.  Ah / Al: the tile's hi and lo buffers, 128 rows x 64 columns
// each.  sB: [W1 hi | W1 lo | W2 hi | W2 lo | W3 hi | W3 lo], W1 64 x K1, W2
// 64 x 64, W3 16 x 64 (rows 4..15 zero), each K-major in 8-row x 16-byte
// core matrices.  tmem: the pipeline's 64 accumulator columns; `lead` (the
// pipeline's first thread) issues its MMAs and commits them to `bar`; `bid`
// is its named barrier.  after_last_mma() runs in every thread of the
// pipeline once the last layer's MMAs have completed: Ah and Al are free
// from then on (the caller starts the next tile's copy there).  Returns
// false (uniformly in the pipeline) when an MMA completion wait ran out.
template <class AfterLastMma>
__device__ __forceinline__ bool tc_mlp_run_tf32(uint8_t* Ah, uint8_t* Al, const uint8_t* sB, uint32_t K1,
                                                uint32_t tmem, bool lead, uint32_t bid, uint64_t* bar,
                                                uint32_t& phase, float4& out, AfterLastMma&& after_last_mma) {
  const uint32_t chunks1 = K1 / 4u, chunks2 = 16u;
  const uint8_t* sB1h = sB;
  const uint8_t* sB1l = sB1h + 64u * K1 * 4u;
  const uint8_t* sB2h = sB1l + 64u * K1 * 4u;
  const uint8_t* sB2l = sB2h + 64u * 64u * 4u;
  const uint8_t* sB3h = sB2l + 64u * 64u * 4u;
  const uint8_t* sB3l = sB3h + 16u * 64u * 4u;
  const int warp = threadIdx.x >> 5;
  const uint32_t row = (uint32_t)threadIdx.x & 127u;
  const uint32_t lane_base = ((uint32_t)(warp & 3) * 32u) << 16;
  const uint32_t id = tc::idesc(128, 64, 2u), id3 = tc::idesc(128, 16, 2u);
  // D = A W^T, three products per K step of 8, committed to `bar`, waited for
  auto mma = [&](const uint8_t* Bh, const uint8_t* Bl, uint32_t chunks, uint32_t idesc) -> bool {
    if (lead) {
      tc::fence_after();
      const uint32_t ah = tc::smem_u32(Ah), al = tc::smem_u32(Al);
      const uint32_t bh = tc::smem_u32(Bh), bl = tc::smem_u32(Bl);
      for (uint32_t s = 0; s < chunks / 2u; ++s) {
        const uint64_t adh = tc::desc_kmajor(ah + s * 256u, 128u, chunks * 128u);
        const uint64_t adl = tc::desc_kmajor(al + s * 256u, 128u, chunks * 128u);
        const uint64_t bdh = tc::desc_kmajor(bh + s * 256u, 128u, chunks * 128u);
        const uint64_t bdl = tc::desc_kmajor(bl + s * 256u, 128u, chunks * 128u);
        tc::mma_tf32(tmem, adl, bdh, idesc, s > 0);  // the small products first
        tc::mma_tf32(tmem, adh, bdl, idesc, 1u);
        tc::mma_tf32(tmem, adh, bdh, idesc, 1u);
      }
      tc::mma_commit(bar);
    }
    const bool ok = tc::mbar_wait(bar, phase, kWaitLimitNs);
    phase ^= 1u;
    if (pipe_or(bid, !ok)) return false;
    tc::fence_after();
    return true;
  };
  // this thread's TMEM row (64 columns) -> ReLU -> hi / lo parts of the next
  // layer's A operand row, in place
  auto next_input = [&]() {
    float v[64];
    tc::tmem_ld64(tmem + lane_base, v);  // the whole row, one load and one wait
#pragma unroll
    for (uint32_t q = 0; q < 16; ++q) {
      const uint4 x = make_uint4(__float_as_uint(fmaxf(v[4 * q], 0.f)), __float_as_uint(fmaxf(v[4 * q + 1], 0.f)),
                                 __float_as_uint(fmaxf(v[4 * q + 2], 0.f)), __float_as_uint(fmaxf(v[4 * q + 3], 0.f)));
      uint4 hi, lo;
      split_tf32(x, hi, lo);
      const uint32_t off = tc::core_off(row, q, chunks2);
      *reinterpret_cast<uint4*>(Ah + off) = hi;
      *reinterpret_cast<uint4*>(Al + off) = lo;
    }
    tc::fence_before();
    tc::fence_async_smem();
    pipe_sync(bid);
  };
  // layer-1 input: split this thread's raw FP32 row in place (chunks1 is even)
#pragma unroll 2
  for (uint32_t c = 0; c < chunks1; ++c) {
    const uint32_t off = tc::core_off(row, c, chunks1);
    uint4 hi, lo;
    split_tf32(*reinterpret_cast<const uint4*>(Ah + off), hi, lo);
    *reinterpret_cast<uint4*>(Ah + off) = hi;
    *reinterpret_cast<uint4*>(Al + off) = lo;
  }
  tc::fence_async_smem();
  pipe_sync(bid);
  if (!mma(sB1h, sB1l, chunks1, id)) return false;  // D1 = A1 W1^T
  next_input();                                      // A2
  if (!mma(sB2h, sB2l, chunks2, id)) return false;  // D2 = A2 W2^T
  next_input();                                      // A3
  if (!mma(sB3h, sB3l, chunks2, id3)) return false; // D3 = A3 W3^T (columns 0..3)
  after_last_mma();
  float v[16];
  tc::tmem_ld16(tmem + lane_base, v);
  out = make_float4(sigmoidf_(v[0]), sigmoidf_(v[1]), sigmoidf_(v[2]), sigmoidf_(v[3]));
  tc::fence_before();
  pipe_sync(bid);
  return true;
}

}  // namespace inolf
