// Tensor-core shade: the corner-bundle gather followed by the MLP F_s (Eq. 3)
// on the 5th-generation tensor cores, with BF16 or FP8-e4m3 operands, or FP32
// operands as split TF32, and FP32 accumulation in tensor memory.  With
// operand tiles in the render workspace the shade runs as k_encode_tc
// (gather + encode into the tiles) and k_mlp_tc / k_mlp_tf32 (the MLP over
// bulk-copied tiles); without them BF16 / FP8 run as the fused k_shade_tc.
//
// k_shade_tc: one CTA = 256 threads = two tiles of 128 hit rays.  Per tile pair:
//   1. every thread gathers its ray's encoding (Sec. 4.1: 16 corner features
//      of the PSH levels, trilinear) and SH view encoding, quantises it and
//      writes its row of the A operand (K-major, 8x16-byte core matrices);
//   2. one thread issues D1 = A1 W1^T (M = 128, N = 64) for both tiles into
//      tensor memory (64 FP32 columns per tile) and commits to an mbarrier;
//   3. each warp reads its 32 rows of D1 (tcgen05.ld), applies ReLU and the
//      quantisation of the next layer's input and writes A2 in place of A1;
//   4. D2 = A2 W2^T on the tensor cores;
//   5. each warp reads its rows of D2, applies ReLU and the last layer's
//      quantisation and writes A3 in place of A2;
//   6. D3 = A3 W3^T on the tensor cores with W3 padded to 16 rows (the
//      smallest N of an M = 128 MMA); each thread reads the 4 outputs of its
//      row and writes sigmoid(.) as RGBA.
// The weights of all three layers are staged once per CTA into shared memory
// by one bulk (TMA) copy from a blob laid out on the host in the operand
// format.  Every mbarrier wait is bounded by a global-timer limit; on expiry
// the CTA flags an error in the workspace header, frees its tensor memory and
// returns.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "inolf_internal.h"
#include "kernels_common.cuh"
#include "tc_ptx.cuh"
#include "tc_mlp.cuh"

namespace inolf {

static constexpr int kTcThreads = 256;
static constexpr uint32_t kTmemCols = 128;  // 2 tiles x 64 FP32 columns
static constexpr int kW3Rows = 16;          // W3 padded to the smallest N of an M = 128 MMA

// Encodes hit h into its operand row (Sec. 4.1): the trilinear PSH features
// of every level, then the SH view encoding and, for density-cube objects,
// alpha_c; zero-padded to K1 columns.  Returns the hit's ray index.
// rec: the hit record (ray, t bits) of hit h, loaded by the caller.
template <int kOp>
__device__ __forceinline__ int64_t encode_rec(const Params& p, uint2 rec, uint32_t h, uint32_t K1,
                                              RowWriter<kOp>& rw) {
  float o[3], d[3], x[3];
  ray_of(p, rec.x, o, d);
  hit_unit_coords(p, o, d, __uint_as_float(rec.y), x);
  // levels in pairs: the Phi load of the next level in flight, no state copies
  LevelFetchB fa, fb;
  fetch_bundle_phi(p.lv[0], x, fa);
  for (int l = 0; l < p.L; l += 2) {
    float e0, e1, g0, g1;
    if (l + 1 < p.L) fetch_bundle_phi(p.lv[l + 1], x, fb);
    finish_bundle(p.lv[l], p.fp16, fa, e0, e1);
    if (l + 1 >= p.L) {
      rw.push(e0, e1);
      break;
    }
    if (l + 2 < p.L) fetch_bundle_phi(p.lv[l + 2], x, fa);
    finish_bundle(p.lv[l + 1], p.fp16, fb, g0, g1);
    rw.push2(e0, e1, g0, g1);  // levels l, l + 1: columns 4 (l / 2) .. + 3
  }
  float sh[16];
  sh16(p, d, sh);
  if ((p.L & 1) == 0) {
#pragma unroll
    for (int i = 0; i < 4; ++i) rw.push2(sh[4 * i], sh[4 * i + 1], sh[4 * i + 2], sh[4 * i + 3]);
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) rw.push(sh[2 * i], sh[2 * i + 1]);
  }
  if (p.variant) rw.push(p.hit_alpha[h], 0.f);  // alpha_c, the last input of F_s (Eq. 5)
  rw.pad_to(K1);
  return rec.x;
}

template <int kOp>
__device__ __forceinline__ int64_t encode_hit(const Params& p, uint32_t h, uint32_t K1, RowWriter<kOp>& rw) {
  return encode_rec<kOp>(p, p.hits[h], h, K1, rw);
}

// Writes the shaded colour of hit h (ray `ray`); density-cube objects add
// the diffuse colour read at the hit point, c = c_d + tint c_s (Eq. 7).
__device__ __forceinline__ void store_rgba(const Params& p, uint32_t h, int64_t ray, float4 rgba) {
  if (p.variant) {
    const uint2 rec = p.hits[h];
    float o[3], d[3], x[3];
    ray_of(p, ray, o, d);
    hit_unit_coords(p, o, d, __uint_as_float(rec.y), x);
    const float4 dc = cube_diffuse(p.cub, x);
    rgba = make_float4(fmaf(dc.w, rgba.x, dc.x), fmaf(dc.w, rgba.y, dc.y), fmaf(dc.w, rgba.z, dc.z), rgba.w);
  }
  p.rgba[p.ray_base + ray] = rgba;
}

template <bool kFP8>
__global__ void __launch_bounds__(kTcThreads, 4) k_shade_tc(const __grid_constant__ Params p) {
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr uint32_t ES = kFP8 ? 1u : 2u;  // operand element bytes
  const uint32_t K1 = (uint32_t)p.tc_k1;
  const uint32_t chunks1 = K1 * ES / 16u;
  const uint32_t wbytes = p.tc_wbytes;
  uint8_t* sB1 = smem;
  uint8_t* sB2 = smem + 64u * K1 * ES;
  const uint8_t* sB3 = sB2 + 64u * 64u * ES;  // W3 as a 16-row operand
  uint8_t* sA = smem + ((wbytes + 1023u) & ~1023u);
  constexpr uint32_t tile_bytes = 128u * 64u * ES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sA + 2 * tile_bytes);  // [0] weights, [1] MMA
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2);

  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    tc::mbar_init(&bars[0], 1);
    tc::mbar_init(&bars[1], 1);
    tc::fence_mbar_init();
  }
  __syncthreads();
  if (warp == 0) tc::tmem_alloc(tslot, kTmemCols);
  if (tid == 0) {
    tc::mbar_arrive_expect_tx(&bars[0], wbytes);
    tc::bulk_g2s(smem, p.tc_w, wbytes, &bars[0]);
  }
  bool ok = tc::mbar_wait(&bars[0], 0, kWaitLimitNs);
  tc::fence_before();
  bool bad = __syncthreads_or(!ok);
  tc::fence_after();
  const uint32_t tmem = *tslot;

  const TcScales sc = TcScales::make(kFP8, p.fp8_act_scale, p.fp8_w_scale);
  const float inv_sx = sc.inv_sx;
  const uint32_t t = (uint32_t)tid >> 7, row = (uint32_t)tid & 127u;
  uint8_t* A = sA + t * tile_bytes;
  const int din = p.d_in;
  uint32_t phase = 0;
  const uint32_t total = *p.counter;

  for (uint32_t base = blockIdx.x * kTcThreads; !bad && base < total; base += gridDim.x * kTcThreads) {
    const uint32_t h = base + (uint32_t)tid;
    const bool valid = h < total;
    int64_t ray = 0;
    // ---- 1. gather + encode -> A1 row ----
    if (valid) {
      RowWriter<kFP8> rw(A, row, chunks1, inv_sx);
      ray = encode_hit<kFP8>(p, h, K1, rw);
    } else {
      for (uint32_t c = 0; c < chunks1; ++c)
        *reinterpret_cast<uint4*>(A + tc::core_off(row, c, chunks1)) = make_uint4(0, 0, 0, 0);
    }
    float4 rgba;
    if (!tc_mlp_run<kFP8>(sA, sB1, sB2, sB3, K1, tmem, &bars[1], phase, sc, rgba)) {
      bad = true;
      break;
    }
    if (valid) store_rgba(p, h, ray, rgba);
  }
  if (bad) {
    if (tid == 0) atomicOr(p.counter + 1, INOLF_FLAG_WAIT_TIMEOUT);
    // let MMAs still in flight finish: the failed wait already flipped `phase`,
    // so the phase in flight has parity phase ^ 1
    tc::mbar_wait(&bars[1], phase ^ 1u, kWaitLimitNs);
  }
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

// ---------------------------------------------------------------------------
// Split tensor-core shade, used when the render workspace holds operand tiles
// for a sub-range of the hit list.  k_encode_tc gathers and encodes the hits
// [tc_h_begin, tc_h_end) into tiles in global memory, in the layout of the
// MMA's A operand (128 rows per tile, K-major 8x16-byte core matrices, K1
// columns); k_mlp_tc copies two tiles at a time into shared memory by bulk
// copy and runs the three layers on the tensor cores.  The gather then runs
// at the occupancy its registers allow: no operand tiles, tensor memory or
// MLP barriers hold its warps.
static constexpr int kEncThreads = 256;

template <int kOp>
__global__ void __launch_bounds__(kEncThreads, 4) k_encode_tc(const __grid_constant__ Params p) {
  constexpr bool kFP8 = kOp == kOpFP8;
  constexpr uint32_t ES = op_bytes<kOp>();
  const uint32_t K1 = (uint32_t)p.tc_k1, chunks1 = K1 * ES / 16u, tile_gbytes = 128u * K1 * ES;
  const float inv_sx = kFP8 ? 1.0f / p.fp8_act_scale[0] : 1.0f;
  const uint32_t end = min(p.tc_h_end, *p.counter);  // launches past the last hit return at once
  const uint32_t stride = gridDim.x * kEncThreads;
  uint32_t h = p.tc_h_begin + blockIdx.x * kEncThreads + threadIdx.x;
  if constexpr (kFP8) {
    // the next hit's record is loaded while this one is encoded (measured
    // faster for FP8; the BF16 kernel spills with it and is not)
    uint2 rec = h < end ? p.hits[h] : make_uint2(0u, 0u);
    for (; h < end; h += stride) {
      const uint2 next = h + stride < end ? p.hits[h + stride] : make_uint2(0u, 0u);
      const uint32_t i = h - p.tc_h_begin;
      RowWriter<kOp> rw(p.tc_a + (size_t)(i >> 7) * tile_gbytes, i & 127u, chunks1, inv_sx);
      encode_rec<kOp>(p, rec, h, K1, rw);
      rec = next;
    }
  } else {
    for (; h < end; h += stride) {
      const uint32_t i = h - p.tc_h_begin;
      RowWriter<kOp> rw(p.tc_a + (size_t)(i >> 7) * tile_gbytes, i & 127u, chunks1, inv_sx);
      encode_hit<kOp>(p, h, K1, rw);
    }
  }
}

template <bool kFP8>
__global__ void __launch_bounds__(kTcThreads, 4) k_mlp_tc(const __grid_constant__ Params p) {
  extern __shared__ __align__(1024) uint8_t smem[];
  // a range past the last hit: nothing to stage (uniform over the grid)
  if (p.tc_h_begin >= *p.counter) return;
  constexpr uint32_t ES = kFP8 ? 1u : 2u;
  const uint32_t K1 = (uint32_t)p.tc_k1;
  const uint32_t wbytes = p.tc_wbytes;
  const uint32_t tile_gbytes = 128u * K1 * ES;  // one tile in global memory
  uint8_t* sB1 = smem;
  uint8_t* sB2 = smem + 64u * K1 * ES;
  const uint8_t* sB3 = sB2 + 64u * 64u * ES;
  uint8_t* sA = smem + ((wbytes + 1023u) & ~1023u);
  constexpr uint32_t tile_bytes = 128u * 64u * ES;  // one tile in shared memory (room for 64 columns)
  uint64_t* bars = reinterpret_cast<uint64_t*>(sA + 2 * tile_bytes);  // [0] weights, [1] MMA, [2] tiles
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 3);

  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    for (int b = 0; b < 3; ++b) tc::mbar_init(&bars[b], 1);
    tc::fence_mbar_init();
  }
  __syncthreads();
  if (warp == 0) tc::tmem_alloc(tslot, kTmemCols);
  if (tid == 0) {
    tc::mbar_arrive_expect_tx(&bars[0], wbytes);
    tc::bulk_g2s(smem, p.tc_w, wbytes, &bars[0]);
  }
  const bool ok = tc::mbar_wait(&bars[0], 0, kWaitLimitNs);
  tc::fence_before();
  bool bad = __syncthreads_or(!ok);
  tc::fence_after();
  const uint32_t tmem = *tslot;
  const TcScales sc = TcScales::make(kFP8, p.fp8_act_scale, p.fp8_w_scale);
  uint32_t phase = 0, tphase = 0;
  bool tiles_in_flight = false;
  const uint32_t end = min(p.tc_h_end, *p.counter);

  for (uint32_t base = p.tc_h_begin + blockIdx.x * kTcThreads; !bad && base < end;
       base += gridDim.x * kTcThreads) {
    const uint32_t t0 = (base - p.tc_h_begin) >> 7;  // first of the two tiles
    if (tid == 0) {
      tc::fence_async_smem();  // the previous pair's in-place writes precede the copy
      tc::mbar_arrive_expect_tx(&bars[2], 2u * tile_gbytes);
      tc::bulk_g2s(sA, p.tc_a + (size_t)t0 * tile_gbytes, tile_gbytes, &bars[2]);
      tc::bulk_g2s(sA + tile_bytes, p.tc_a + (size_t)(t0 + 1u) * tile_gbytes, tile_gbytes, &bars[2]);
    }
    tiles_in_flight = true;
    // the hit's ray index is loaded now, while the tiles and the MMAs are in flight
    const uint32_t h = base + (uint32_t)tid;
    const uint32_t ray = h < end ? p.hits[h].x : 0u;
    const bool landed = tc::mbar_wait(&bars[2], tphase, kWaitLimitNs);
    tphase ^= 1u;
    if (__syncthreads_or(!landed)) {
      bad = true;
      break;
    }
    tiles_in_flight = false;
    float4 rgba;
    if (!tc_mlp_run<kFP8>(sA, sB1, sB2, sB3, K1, tmem, &bars[1], phase, sc, rgba)) {
      bad = true;
      break;
    }
    if (h < end) store_rgba(p, h, (int64_t)ray, rgba);
  }
  if (bad) {
    if (tid == 0) atomicOr(p.counter + 1, INOLF_FLAG_WAIT_TIMEOUT);
    // copies and MMAs still in flight finish before the CTA leaves; a failed
    // wait already flipped its parity, so the one in flight has parity ^ 1
    if (tiles_in_flight) tc::mbar_wait(&bars[2], tphase ^ 1u, kWaitLimitNs);
    tc::mbar_wait(&bars[1], phase ^ 1u, kWaitLimitNs);
  }
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

// FP32 path of the split shade: the tiles hold raw FP32 layer-1 inputs
// (written by k_encode_tc<kOpF32>).  A CTA runs two independent pipelines of
// 128 threads, each over its own 128-row tiles with its own hi / lo buffers,
// mbarriers, 64 tensor-memory columns and named barrier, so that one
// pipeline's MMAs overlap the other's tile copy, split and epilogues.  Per
// tile: one bulk copy into the hi buffer, the split into TF32 hi / lo parts
// in place, and the three layers as split-TF32 products (tc_mlp_run_tf32).
// The weights, split on the host, arrive by one bulk copy.  One CTA per SM
// (about 200 KB of shared memory).
static constexpr uint32_t kTf32TileBytes = 128u * 64u * 4u;

__global__ void __launch_bounds__(kTcThreads, 1) k_mlp_tf32(const __grid_constant__ Params p) {
  extern __shared__ __align__(1024) uint8_t smem[];
  if (p.tc_h_begin >= *p.counter) return;  // a range past the last hit (uniform over the grid)
  const uint32_t K1 = (uint32_t)p.tc_k1;
  const uint32_t wbytes = p.tc_wbytes;
  const uint32_t tile_gbytes = 128u * K1 * 4u;
  uint8_t* sA = smem + ((wbytes + 1023u) & ~1023u);  // per pipeline: hi buffer, lo buffer
  // [0] weights; pipeline q: [1 + 2 q] its MMAs, [2 + 2 q] its tile copy
  uint64_t* bars = reinterpret_cast<uint64_t*>(sA + 4u * kTf32TileBytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 5);

  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t pipe = (uint32_t)tid >> 7, row = (uint32_t)tid & 127u;
  const bool lead = row == 0u;
  if (tid == 0) {
    for (int b = 0; b < 5; ++b) tc::mbar_init(&bars[b], 1);
    tc::fence_mbar_init();
  }
  __syncthreads();
  if (warp == 0) tc::tmem_alloc(tslot, kTmemCols);
  if (tid == 0) {
    tc::mbar_arrive_expect_tx(&bars[0], wbytes);
    tc::bulk_g2s(smem, p.tc_w, wbytes, &bars[0]);
  }
  const bool ok = tc::mbar_wait(&bars[0], 0, kWaitLimitNs);
  tc::fence_before();
  bool bad = __syncthreads_or(!ok);
  tc::fence_after();
  const uint32_t tmem = *tslot + pipe * 64u;
  uint8_t* Ah = sA + pipe * 2u * kTf32TileBytes;
  uint8_t* Al = Ah + kTf32TileBytes;
  uint64_t* mbar = &bars[1 + 2 * pipe];
  uint64_t* tbar = &bars[2 + 2 * pipe];
  const uint32_t bid = 1u + pipe;
  uint32_t phase = 0, tphase = 0;
  bool tile_in_flight = false;
  const uint32_t end = min(p.tc_h_end, *p.counter);
  const uint32_t step = gridDim.x * 256u;
  // lead thread: copy of the tile at hit `b` into Ah, and a prefetch of the
  // pipeline's tile after it into L2
  auto issue_copy = [&](uint32_t b) {
    tc::fence_async_smem();  // earlier in-place writes to Ah precede the copy
    tc::mbar_arrive_expect_tx(tbar, tile_gbytes);
    tc::bulk_g2s(Ah, p.tc_a + (size_t)((b - p.tc_h_begin) >> 7) * tile_gbytes, tile_gbytes, tbar);
    if (b + step < end) tc::bulk_prefetch_l2(p.tc_a + (size_t)((b + step - p.tc_h_begin) >> 7) * tile_gbytes, tile_gbytes);
  };
  uint32_t base = p.tc_h_begin + (blockIdx.x * 2u + pipe) * 128u;
  if (!bad && base < end) {
    if (lead) issue_copy(base);
    tile_in_flight = true;
  }
  for (; !bad && base < end; base += step) {
    const uint32_t h = base + row;
    const uint32_t ray = h < end ? p.hits[h].x : 0u;
    const bool landed = tc::mbar_wait(tbar, tphase, kWaitLimitNs);
    tphase ^= 1u;
    if (pipe_or(bid, !landed)) {
      bad = true;
      break;
    }
    tile_in_flight = false;
    const bool more = base + step < end;
    float4 rgba;
    // the next tile's copy starts as soon as the last layer's MMAs have
    // read this tile's operands, ahead of the output epilogue
    if (!tc_mlp_run_tf32(Ah, Al, smem, K1, tmem, lead, bid, mbar, phase, rgba, [&] {
          if (lead && more) issue_copy(base + step);
        })) {
      bad = true;
      break;
    }
    tile_in_flight = more;
    if (h < end) store_rgba(p, h, (int64_t)ray, rgba);
  }
  if (bad) {
    if (lead) atomicOr(p.counter + 1, INOLF_FLAG_WAIT_TIMEOUT);
    // the pipeline's copy and MMAs still in flight finish before the CTA
    // leaves; a failed wait already flipped its parity
    if (tile_in_flight) tc::mbar_wait(tbar, tphase ^ 1u, kWaitLimitNs);
    tc::mbar_wait(mbar, phase ^ 1u, kWaitLimitNs);
  }
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(*tslot, kTmemCols);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static uint32_t round_up(uint32_t v, uint32_t m) { return (v + m - 1) / m * m; }

// Split-TF32 weight blob: [W1 hi | W1 lo | W2 hi | W2 lo | W3 hi | W3 lo],
// W1 64 x K1 (columns from din on zero), W2 64 x 64, W3 16 x 64 (rows 4..15
// zero), each K-major in core matrices of 8 rows x 4 FP32 values; hi =
// tf32(w), lo = tf32(w - hi).  Returns the offset of element (n, k) of a
// matrix with `chunks` 16-byte chunks per row.
static inline uint32_t tf32_off(uint32_t n, uint32_t k, uint32_t chunks) {
  return tc::core_off(n, k / 4, chunks) + (k % 4) * 4;
}
static void tf32_split_host(float w, uint32_t& hi, uint32_t& lo) {
  uint32_t u;
  std::memcpy(&u, &w, 4);
  hi = tf32_rna_bits(u);
  float h, r;
  std::memcpy(&h, &hi, 4);
  r = w - h;
  std::memcpy(&u, &r, 4);
  lo = tf32_rna_bits(u);
}
static std::vector<uint8_t> tf32_blob_host(const float* w1, const float* w2, const float* w3, int din, uint32_t K1) {
  const int H = INOLF_HIDDEN, O = INOLF_OUT;
  const size_t m1 = (size_t)H * K1 * 4, m2 = (size_t)H * H * 4, m3 = (size_t)kW3Rows * H * 4;
  std::vector<uint8_t> blob(2 * (m1 + m2 + m3), 0);
  auto put = [&](uint8_t* hi_base, size_t lo_delta, uint32_t n, uint32_t k, uint32_t chunks, float w) {
    uint32_t hi, lo;
    tf32_split_host(w, hi, lo);
    std::memcpy(hi_base + tf32_off(n, k, chunks), &hi, 4);
    std::memcpy(hi_base + lo_delta + tf32_off(n, k, chunks), &lo, 4);
  };
  uint8_t* b1 = blob.data();
  uint8_t* b2 = b1 + 2 * m1;
  uint8_t* b3 = b2 + 2 * m2;
  for (int n = 0; n < H; ++n)
    for (int k = 0; k < din; ++k) put(b1, m1, n, k, K1 / 4, w1[(size_t)n * din + k]);
  for (int n = 0; n < H; ++n)
    for (int k = 0; k < H; ++k) put(b2, m2, n, k, 16, w2[(size_t)n * H + k]);
  for (int n = 0; n < O; ++n)
    for (int k = 0; k < H; ++k) put(b3, m3, n, k, 16, w3[(size_t)n * H + k]);
  return blob;
}

// Weight blob in the operand layout (K-major core matrices, rows = output
// neurons): [W1: 64 x K1][W2: 64 x 64][W3: 16 x 64, rows 4..15 zero]
inolf_status prepare_tc_weights(Object& obj, const float* w1, const float* w2, const float* w3, void* stream) {
  const int din = obj.d_in, H = INOLF_HIDDEN, O = INOLF_OUT;
  cudaStream_t st = (cudaStream_t)stream;
  auto amax = [](const float* w, size_t n) {
    float m = 0.f;
    for (size_t i = 0; i < n; ++i) m = std::max(m, std::fabs(w[i]));
    return m;
  };
  // ---- BF16 ----
  {
    const uint32_t K1 = round_up((uint32_t)din, 16), ch1 = K1 / 8, ch2 = 8;
    std::vector<uint8_t> blob((size_t)H * K1 * 2 + (size_t)H * H * 2 + (size_t)kW3Rows * H * 2, 0);
    for (int n = 0; n < H; ++n)
      for (int k = 0; k < din; ++k) {
        __nv_bfloat16 v = __float2bfloat16_rn(w1[(size_t)n * din + k]);
        std::memcpy(&blob[tc::core_off(n, k / 8, ch1) + (k % 8) * 2], &v, 2);
      }
    uint8_t* b2 = blob.data() + (size_t)H * K1 * 2;
    for (int n = 0; n < H; ++n)
      for (int k = 0; k < H; ++k) {
        __nv_bfloat16 v = __float2bfloat16_rn(w2[(size_t)n * H + k]);
        std::memcpy(&b2[tc::core_off(n, k / 8, ch2) + (k % 8) * 2], &v, 2);
      }
    uint8_t* b3 = b2 + (size_t)H * H * 2;  // W3: 16 rows (4 outputs, 12 zero rows) x 64
    for (int n = 0; n < O; ++n)
      for (int k = 0; k < H; ++k) {
        __nv_bfloat16 v = __float2bfloat16_rn(w3[(size_t)n * H + k]);
        std::memcpy(&b3[tc::core_off(n, k / 8, ch2) + (k % 8) * 2], &v, 2);
      }
    if (!obj.w_bf16) {
      if (cudaMalloc(&obj.w_bf16, blob.size()) != cudaSuccess) return fail(INOLF_E_OOM, "cudaMalloc bf16 weights");
      obj.bytes += blob.size();
    }
    if (cudaMemcpyAsync(obj.w_bf16, blob.data(), blob.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return fail(INOLF_E_CUDA, "upload bf16 weights");
    obj.tc_k1_bf16 = (int32_t)K1;
    obj.tc_bytes_bf16 = (uint32_t)blob.size();
  }
  // ---- FP32 as split TF32: per layer the hi parts, then the lo parts ----
  {
    const uint32_t K1 = round_up((uint32_t)din, 8);
    const std::vector<uint8_t> blob = tf32_blob_host(w1, w2, w3, din, K1);
    if (!obj.w_tf32) {
      if (cudaMalloc(&obj.w_tf32, blob.size()) != cudaSuccess) return fail(INOLF_E_OOM, "cudaMalloc tf32 weights");
      obj.bytes += blob.size();
    }
    if (cudaMemcpyAsync(obj.w_tf32, blob.data(), blob.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return fail(INOLF_E_CUDA, "upload tf32 weights");
    obj.tc_k1_tf32 = (int32_t)K1;
    obj.tc_bytes_tf32 = (uint32_t)blob.size();
  }
  // ---- FP8 e4m3, per-tensor scales amax / 448 ----
  {
    const uint32_t K1 = round_up((uint32_t)din, 32), ch1 = K1 / 16, ch2 = 4;
    const float s1 = amax(w1, (size_t)H * din), s2 = amax(w2, (size_t)H * H), s3 = amax(w3, (size_t)O * H);
    obj.fp8_w_scale[0] = s1 > 0 ? s1 / 448.0f : 1.0f;
    obj.fp8_w_scale[1] = s2 > 0 ? s2 / 448.0f : 1.0f;
    obj.fp8_w_scale[2] = s3 > 0 ? s3 / 448.0f : 1.0f;
    auto q = [](float v, float s) { return (uint8_t)__nv_cvt_float_to_fp8(v / s, __NV_SATFINITE, __NV_E4M3); };
    std::vector<uint8_t> blob((size_t)H * K1 + (size_t)H * H + (size_t)kW3Rows * H, 0);
    for (int n = 0; n < H; ++n)
      for (int k = 0; k < din; ++k)
        blob[tc::core_off(n, k / 16, ch1) + (k % 16)] = q(w1[(size_t)n * din + k], obj.fp8_w_scale[0]);
    uint8_t* b2 = blob.data() + (size_t)H * K1;
    for (int n = 0; n < H; ++n)
      for (int k = 0; k < H; ++k) b2[tc::core_off(n, k / 16, ch2) + (k % 16)] = q(w2[(size_t)n * H + k], obj.fp8_w_scale[1]);
    uint8_t* b3 = b2 + (size_t)H * H;  // W3: 16 rows (4 outputs, 12 zero rows) x 64
    for (int n = 0; n < O; ++n)
      for (int k = 0; k < H; ++k) b3[tc::core_off(n, k / 16, ch2) + (k % 16)] = q(w3[(size_t)n * H + k], obj.fp8_w_scale[2]);
    if (!obj.w_fp8) {
      if (cudaMalloc(&obj.w_fp8, blob.size()) != cudaSuccess) return fail(INOLF_E_OOM, "cudaMalloc fp8 weights");
      obj.bytes += blob.size();
    }
    if (cudaMemcpyAsync(obj.w_fp8, blob.data(), blob.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return fail(INOLF_E_CUDA, "upload fp8 weights");
    obj.tc_k1_fp8 = (int32_t)K1;
    obj.tc_bytes_fp8 = (uint32_t)blob.size();
  }
  if (!obj.w_scale_dev) {
    if (cudaMalloc(&obj.w_scale_dev, 4 * sizeof(float)) != cudaSuccess) return fail(INOLF_E_OOM, "cudaMalloc scales");
    obj.bytes += 4 * sizeof(float);
  }
  if (cudaMemcpyAsync(obj.w_scale_dev, obj.fp8_w_scale, 3 * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(INOLF_E_CUDA, "upload fp8 weight scales");
  return INOLF_OK;
}

// Device-side repacking of all weight formats from device FP32 weights (one
// CTA; the MLP has ~7 500 weights): the per-tensor FP8 weight scales amax /
// 448, the FP32 SIMT blob and the BF16 / FP8 operand blobs, each written
// exactly as prepare_tc_weights and upload_weights write them on the host
// (the zero rows of W3 included).
__device__ float block_amax(const float* w, int n, float* red) {
  float m = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmaxf(m, fabsf(w[i]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  m = 0.f;
  for (int k = 0; k < (int)(blockDim.x >> 5); ++k) m = fmaxf(m, red[k]);
  return m;
}

__device__ __forceinline__ void tf32_put(uint8_t* hi_base, size_t lo_delta, uint32_t n, uint32_t k, uint32_t chunks,
                                         float w) {
  const uint32_t hi = tf32_rna_bits(__float_as_uint(w));
  const uint32_t lo = tf32_rna_bits(__float_as_uint(w - __uint_as_float(hi)));
  const uint32_t off = tc::core_off(n, k / 4, chunks) + (k % 4) * 4;
  *reinterpret_cast<uint32_t*>(hi_base + off) = hi;
  *reinterpret_cast<uint32_t*>(hi_base + lo_delta + off) = lo;
}

__global__ void k_pack_weights(const float* __restrict__ w1, const float* __restrict__ w2,
                               const float* __restrict__ w3, int din, uint32_t K1b, uint32_t K1f, uint32_t K1t,
                               float* f32, uint8_t* bf16, uint8_t* fp8, uint8_t* tf32, float* scales) {
  constexpr int H = INOLF_HIDDEN, O = INOLF_OUT;
  __shared__ float red[32];
  const float a1 = block_amax(w1, H * din, red), a2 = block_amax(w2, H * H, red), a3 = block_amax(w3, O * H, red);
  const float s1 = a1 > 0 ? a1 / 448.0f : 1.0f, s2 = a2 > 0 ? a2 / 448.0f : 1.0f, s3 = a3 > 0 ? a3 / 448.0f : 1.0f;
  if (threadIdx.x == 0) {
    scales[0] = s1;
    scales[1] = s2;
    scales[2] = s3;
  }
  auto q = [](float v, float sc) { return (uint8_t)__nv_cvt_float_to_fp8(v / sc, __NV_SATFINITE, __NV_E4M3); };
  const int tid = threadIdx.x, nt = blockDim.x;
  // FP32: W1T [din][64] | W2 [64][64] | W3T [64][4]
  for (int i = tid; i < H * din; i += nt) {
    const int j = i / din, k = i - j * din;
    f32[k * H + j] = w1[i];
  }
  for (int i = tid; i < H * H; i += nt) f32[din * H + i] = w2[i];
  for (int i = tid; i < O * H; i += nt) {
    const int j = i / H, k = i - j * H;
    f32[din * H + H * H + k * O + j] = w3[i];
  }
  // BF16: W1 (64 x K1b, zero padded) | W2 (64 x 64) in core matrices | W3^T FP32 of the rounded values
  const uint32_t ch1 = K1b / 8;
  for (int i = tid; i < H * (int)K1b; i += nt) {
    const int n = i / (int)K1b, k = i - n * (int)K1b;
    const __nv_bfloat16 v = __float2bfloat16_rn(k < din ? w1[n * din + k] : 0.0f);
    *reinterpret_cast<__nv_bfloat16*>(bf16 + tc::core_off(n, k / 8, ch1) + (k % 8) * 2) = v;
  }
  uint8_t* b2 = bf16 + (size_t)H * K1b * 2;
  for (int i = tid; i < H * H; i += nt) {
    const int n = i / H, k = i - n * H;
    *reinterpret_cast<__nv_bfloat16*>(b2 + tc::core_off(n, k / 8, 8) + (k % 8) * 2) = __float2bfloat16_rn(w2[i]);
  }
  uint8_t* b3 = b2 + (size_t)H * H * 2;  // rows 4..15 stay zero
  for (int i = tid; i < kW3Rows * H; i += nt) {
    const int n = i / H, k = i - n * H;
    *reinterpret_cast<__nv_bfloat16*>(b3 + tc::core_off(n, k / 8, 8) + (k % 8) * 2) =
        __float2bfloat16_rn(n < O ? w3[i] : 0.0f);
  }
  // FP8 e4m3: W1 (64 x K1f, zero padded) | W2 | W3^T FP32 of the dequantised values
  const uint32_t cf1 = K1f / 16;
  for (int i = tid; i < H * (int)K1f; i += nt) {
    const int n = i / (int)K1f, k = i - n * (int)K1f;
    fp8[tc::core_off(n, k / 16, cf1) + (k % 16)] = k < din ? q(w1[n * din + k], s1) : (uint8_t)0;
  }
  uint8_t* f2 = fp8 + (size_t)H * K1f;
  for (int i = tid; i < H * H; i += nt) {
    const int n = i / H, k = i - n * H;
    f2[tc::core_off(n, k / 16, 4) + (k % 16)] = q(w2[i], s2);
  }
  uint8_t* f3 = f2 + (size_t)H * H;
  for (int i = tid; i < kW3Rows * H; i += nt) {
    const int n = i / H, k = i - n * H;
    f3[tc::core_off(n, k / 16, 4) + (k % 16)] = n < O ? q(w3[i], s3) : (uint8_t)0;
  }
  // split TF32: [W1 hi | W1 lo (64 x K1t, zero padded) | W2 hi | W2 lo | W3 hi | W3 lo (16 rows)]
  const size_t m1 = (size_t)H * K1t * 4, m2 = (size_t)H * H * 4, m3 = (size_t)kW3Rows * H * 4;
  for (int i = tid; i < H * (int)K1t; i += nt) {
    const int n = i / (int)K1t, k = i - n * (int)K1t;
    tf32_put(tf32, m1, n, k, K1t / 4, k < din ? w1[n * din + k] : 0.0f);
  }
  uint8_t* t2 = tf32 + 2 * m1;
  for (int i = tid; i < H * H; i += nt) tf32_put(t2, m2, i / H, i % H, 16, w2[i]);
  uint8_t* t3 = t2 + 2 * m2;
  for (int i = tid; i < kW3Rows * H; i += nt) {
    const int n = i / H, k = i - n * H;
    tf32_put(t3, m3, n, k, 16, n < O ? w3[i] : 0.0f);
  }
}

inolf_status pack_weights_device(Object& obj, const float* w1, const float* w2, const float* w3, void* stream) {
  if (!obj.w_f32 || !obj.w_bf16 || !obj.w_fp8 || !obj.w_tf32 || !obj.w_scale_dev)
    return fail(INOLF_E_INVALID, "pack_weights_device: object weights not allocated");
  k_pack_weights<<<1, 1024, 0, (cudaStream_t)stream>>>(
      w1, w2, w3, obj.d_in, (uint32_t)obj.tc_k1_bf16, (uint32_t)obj.tc_k1_fp8, (uint32_t)obj.tc_k1_tf32, obj.w_f32,
      (uint8_t*)obj.w_bf16, (uint8_t*)obj.w_fp8, (uint8_t*)obj.w_tf32, obj.w_scale_dev);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(INOLF_E_CUDA, std::string("k_pack_weights: ") + cudaGetErrorString(e));
  return INOLF_OK;
}

// Largest weight blob: K1 = 64 (BF16: 64 x 64 x 2 + 64 x 64 x 2 + 16 x 64 x 2 bytes).
static constexpr uint32_t kMaxTcWeightBytes = 18432;

static size_t tc_smem_bytes(uint32_t wbytes, bool fp8) {
  const size_t tile = 128u * 64u * (fp8 ? 1u : 2u);
  return ((wbytes + 1023u) & ~1023u) + 2 * tile + 64;
}

// Largest split-TF32 weight blob (K1 = 64) and the shared memory of
// k_mlp_tf32: the blob, hi and lo buffers of two tiles, three mbarriers and
// the tensor-memory slot.
static constexpr uint32_t kMaxTf32WeightBytes = 2u * (64u * 64u + 64u * 64u + 16u * 64u) * 4u;
static size_t tf32_smem_bytes(uint32_t wbytes) { return ((wbytes + 1023u) & ~1023u) + 4u * kTf32TileBytes + 64; }

inolf_status launch_shade_tc(const Params& p_in, inolf_precision prec, cudaStream_t st) {
  const bool fp8 = prec == INOLF_FP8, f32 = prec == INOLF_FP32;
  Params p = p_in;
  p.tc_w = f32 ? p.w_tf32 : (fp8 ? p.w_fp8 : p.w_bf16);
  p.tc_k1 = f32 ? p.tc_k1_tf32 : (fp8 ? p.tc_k1_fp8 : p.tc_k1_bf16);
  p.tc_wbytes = f32 ? p.tc_bytes_tf32 : (fp8 ? p.tc_bytes_fp8 : p.tc_bytes_bf16);
  if (!p.tc_w || p.tc_wbytes == 0 || (p.tc_wbytes & 15u)) return fail(INOLF_E_INVALID, "tensor-core weights missing");
  if (f32 && !p.tc_a) return fail(INOLF_E_INVALID, "FP32 tensor-core shade: no operand tiles in the workspace");
  const size_t smem = f32 ? tf32_smem_bytes(p.tc_wbytes) : tc_smem_bytes(p.tc_wbytes, fp8);
  const int dev = device_index();
  if (dev < 0) return fail(INOLF_E_UNSUPPORTED, "k_shade_tc: no current device, or an index beyond 63");
  static int grid_bf16_dev[kMaxDevices], grid_fp8_dev[kMaxDevices];
  static int grid_enc_dev[kMaxDevices][3], grid_mlp_dev[kMaxDevices][3];  // [operand kind: BF16, FP8, FP32]
  static std::once_flag once[kMaxDevices];
  std::call_once(once[dev], [&] {
    int sms = 1, regs_sm = 65536, smem_sm = 0;
    int& grid_bf16 = grid_bf16_dev[dev];
    int& grid_fp8 = grid_fp8_dev[dev];
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    auto ctas_per_sm = [&](const void* fn, size_t smem_b) {
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b);
      cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      cudaFuncAttributes fa{};
      cudaFuncGetAttributes(&fa, fn);
      // registers are allocated per warp in units of 256
      const int regs_warp = ((std::max(fa.numRegs, 1) * 32 + 255) / 256) * 256;
      const int by_regs = regs_sm / (regs_warp * (kTcThreads / 32));
      const int by_smem = (int)(smem_sm / (smem_b + fa.sharedSizeBytes + 1024));
      const int by_tmem = 512 / (int)kTmemCols;  // each CTA holds kTmemCols of 512 TMEM columns
      int n = std::min(std::min(by_regs, by_smem), by_tmem);
      // optional cap (tuning knob): fewer resident CTAs leave more of the
      // unified L1/shared storage to the L1 cache that the gather relies on
      if (const char* e = std::getenv("INOLF_TC_CTAS_PER_SM")) n = std::min(n, std::atoi(e));
      return std::max(1, n);
    };
    grid_bf16 = sms * ctas_per_sm((const void*)k_shade_tc<false>, tc_smem_bytes(kMaxTcWeightBytes, false));
    grid_fp8 = sms * ctas_per_sm((const void*)k_shade_tc<true>, tc_smem_bytes(kMaxTcWeightBytes, true));
    grid_mlp_dev[dev][0] = sms * ctas_per_sm((const void*)k_mlp_tc<false>, tc_smem_bytes(kMaxTcWeightBytes, false));
    grid_mlp_dev[dev][1] = sms * ctas_per_sm((const void*)k_mlp_tc<true>, tc_smem_bytes(kMaxTcWeightBytes, true));
    // the encode kernel holds neither shared nor tensor memory: registers decide
    auto enc_ctas = [&](const void* fn) {
      cudaFuncAttributes fa{};
      cudaFuncGetAttributes(&fa, fn);
      const int regs_warp = ((std::max(fa.numRegs, 1) * 32 + 255) / 256) * 256;
      return std::max(1, std::min(regs_sm / (regs_warp * (kEncThreads / 32)), 2048 / kEncThreads));
    };
    grid_mlp_dev[dev][2] = sms * ctas_per_sm((const void*)k_mlp_tf32, tf32_smem_bytes(kMaxTf32WeightBytes));
    grid_enc_dev[dev][0] = sms * enc_ctas((const void*)k_encode_tc<kOpBF16>);
    grid_enc_dev[dev][1] = sms * enc_ctas((const void*)k_encode_tc<kOpFP8>);
    grid_enc_dev[dev][2] = sms * enc_ctas((const void*)k_encode_tc<kOpF32>);
    cudaGetLastError();
  });
  if (smem > (f32 ? tf32_smem_bytes(kMaxTf32WeightBytes) : tc_smem_bytes(kMaxTcWeightBytes, fp8)))
    return fail(INOLF_E_INVALID, "tensor-core weights too large");
  const int grid = fp8 ? grid_fp8_dev[dev] : grid_bf16_dev[dev];
  if (p.tc_a) {
    // split path: sub-ranges of the hit list as large as the workspace's
    // operand tiles hold (a multiple of the MLP kernel's 256 rows); the hit
    // count is known on the device only, so the ranges span the chunk's ray
    // count and launches past the last hit return at once
    const uint64_t row_bytes = (uint64_t)p.tc_k1 * (f32 ? 4u : (fp8 ? 1u : 2u));
    const uint64_t rows = std::min<uint64_t>(p.tc_a_bytes / row_bytes / 256u * 256u, 0x80000000ull);
    if (rows < 256) return fail(INOLF_E_INVALID, "split shade: operand tile region smaller than 256 rows");
    for (int64_t h0 = 0; h0 < p.n_rays; h0 += (int64_t)rows) {
      Params q = p;
      q.tc_h_begin = (uint32_t)h0;
      q.tc_h_end = (uint32_t)std::min<int64_t>(h0 + (int64_t)rows, p.n_rays);
      {
        LaunchTimer lt(f32 ? "k_encode_tc_f32" : (fp8 ? "k_encode_tc_fp8" : "k_encode_tc_bf16"), st);
        if (f32) k_encode_tc<kOpF32><<<grid_enc_dev[dev][2], kEncThreads, 0, st>>>(q);
        else if (fp8) k_encode_tc<kOpFP8><<<grid_enc_dev[dev][1], kEncThreads, 0, st>>>(q);
        else k_encode_tc<kOpBF16><<<grid_enc_dev[dev][0], kEncThreads, 0, st>>>(q);
      }
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return fail(INOLF_E_CUDA, std::string("k_encode_tc: ") + cudaGetErrorString(e));
      {
        LaunchTimer lt(f32 ? "k_mlp_tc_f32" : (fp8 ? "k_mlp_tc_fp8" : "k_mlp_tc_bf16"), st);
        if (f32) k_mlp_tf32<<<grid_mlp_dev[dev][2], kTcThreads, smem, st>>>(q);
        else if (fp8) k_mlp_tc<true><<<grid_mlp_dev[dev][1], kTcThreads, smem, st>>>(q);
        else k_mlp_tc<false><<<grid_mlp_dev[dev][0], kTcThreads, smem, st>>>(q);
      }
      e = cudaGetLastError();
      if (e != cudaSuccess) return fail(INOLF_E_CUDA, std::string("k_mlp_tc: ") + cudaGetErrorString(e));
    }
    return INOLF_OK;
  }
  {
    LaunchTimer lt(fp8 ? "k_shade_tc_fp8" : "k_shade_tc_bf16", st);
    if (fp8) k_shade_tc<true><<<grid, kTcThreads, smem, st>>>(p);
    else k_shade_tc<false><<<grid, kTcThreads, smem, st>>>(p);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(INOLF_E_CUDA, std::string("k_shade_tc: ") + cudaGetErrorString(e));
  return INOLF_OK;
}

}  // namespace inolf
