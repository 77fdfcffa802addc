// Forward i-NOLF rendering on sm_103a: one network query per ray (Sec. 4.2).
//
// Two kernels per batch of rays:
//   k_trace  one thread per ray: pinhole ray generation, closest-hit BVH
//            traversal of the proxy mesh (FP32 Moller-Trumbore, closest =
//            lexicographic (t, triangle id) minimum), then warp-ballot
//            compaction of the hitting rays into a dense hit list
//            (one global atomic per CTA).  Misses write RGBA = 0.
//   shade    over the hit list: the Sec. 4.1 grid cell of the hit point on
//            every level, its 8 corner features (one Eq. 1 slot of the lowest
//            corner and one corner-bundle read per level in the render
//            kernels; Eq. 1 slots of all 8 corners in the per-ray kernel),
//            trilinear interpolation, SH view encoding and the MLP F_s of
//            Eq. 3.  With operand tiles in the workspace every precision runs
//            on the tensor cores as an encode kernel and an MLP kernel
//            (mlp_tc.cu; FP32 as split TF32).  Without them: the fused BF16 /
//            FP8 kernel (mlp_tc.cu), or FP32 on the CUDA cores in this file:
//            k_shade_f32_ws (gather and MLP on separate warps;
//            k_shade_f32_tiled where the register split cannot be used).
//            The per-ray k_shade_f32 serves stage outputs and FP8 calibration.
//
// The FP32 steps that decide integers (ray generation, triangle test, hit
// point, cell index) are written with explicit round-to-nearest intrinsics
// so that no multiply-add is contracted and every result is the IEEE result
// of the stated operation order.
#include <cuda_runtime.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "inolf_internal.h"
#include "kernels_common.cuh"
#include "tc_ptx.cuh"

namespace inolf {

// ---------------------------------------------------------------------------
// k_trace / k_march
// ---------------------------------------------------------------------------
// Ray of this thread: mode 0 = 16 x 16 pixel tile per CTA, each warp an 8 x 4
// block of pixels; mode 1 = explicit rays, 256 per CTA.
__device__ __forceinline__ bool thread_ray(const Params& p, int32_t tiles_x, int32_t tiles_y, int64_t& ray, float o[3],
                                           float d[3]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  bool valid;
  if (p.mode == 0) {
    const int64_t tiles = (int64_t)tiles_x * tiles_y;
    const int view = (int)(blockIdx.x / tiles);
    const int64_t tr = blockIdx.x - (int64_t)view * tiles;
    const int ty = (int)(tr / tiles_x), tx = (int)(tr - (int64_t)ty * tiles_x);
    const int i = tx * 16 + (warp & 1) * 8 + (lane & 7);
    const int j = ty * 16 + (warp >> 1) * 4 + (lane >> 3);
    valid = (i < p.W) && (j < p.H);
    ray = (int64_t)view * p.W * p.H + (int64_t)j * p.W + i;
    if (valid) make_ray(p.cams + 13 * view, p.W, p.H, i, j, o, d);
  } else {
    ray = (int64_t)blockIdx.x * 256 + threadIdx.x;
    valid = ray < p.n_rays;
    if (valid) {
      for (int k = 0; k < 3; ++k) { o[k] = p.ro[3 * ray + k]; d[k] = p.rd[3 * ray + k]; }
    }
  }
  return valid;
}

// Compaction: warp ballot + per-CTA prefix + one global atomic per CTA, so
// the hits of a 16 x 16 pixel tile stay contiguous in the hit list and a
// shade tile covers neighbouring pixels (cache locality of the gather).
// Returns this thread's hit-list position (meaningful when hit).
__device__ __forceinline__ uint32_t compact_hit(const Params& p, bool hit) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ uint32_t s_warp[8];
  __shared__ uint32_t s_base;
  const uint32_t mask = __ballot_sync(0xffffffffu, hit);
  if (lane == 0) s_warp[warp] = __popc(mask);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (int w = 0; w < 8; ++w) { uint32_t c = s_warp[w]; s_warp[w] = acc; acc += c; }
    s_base = acc ? atomicAdd(p.counter, acc) : 0u;
  }
  __syncthreads();
  return s_base + s_warp[warp] + __popc(mask & ((1u << lane) - 1u));
}

// Workspace words 8 .. 13 (three uint64): with kCount, k_trace adds each
// packet's inner-node visits, triangle tests and hit rays there.
static constexpr int kTraceCountWord = 8;

template <bool kCount>
__global__ void __launch_bounds__(256) k_trace(const __grid_constant__ Params p, int32_t tiles_x, int32_t tiles_y) {
  int64_t ray;
  float o[3], d[3];
  const bool valid = thread_ray(p, tiles_x, tiles_y, ray, o, d);
  int32_t tri = -1;
  float t = 0.0f;
  if (p.mode == 0) {
    // pinhole views: the 8 x 4 pixel block of a warp is coherent, traverse it as a packet
    if (!valid) {
#pragma unroll
      for (int k = 0; k < 3; ++k) { o[k] = 0.0f; d[k] = 1.0f; }
    }
    uint32_t visits = 0, tests = 0;
    closest_hit_packet<kCount>(p.nodes, p.tris, p.counter + 1, valid, o, d, tri, t, &visits, &tests);
    if (kCount) {
      const uint32_t hits = __popc(__ballot_sync(0xffffffffu, valid && tri >= 0));
      if ((threadIdx.x & 31) == 0) {
        unsigned long long* c = reinterpret_cast<unsigned long long*>(p.counter + kTraceCountWord);
        atomicAdd(c + 0, (unsigned long long)visits);
        atomicAdd(c + 1, (unsigned long long)tests);
        atomicAdd(c + 2, (unsigned long long)hits);
      }
    }
  } else if (valid) {
    closest_hit(p, o, d, tri, t);
  }
  const bool hit = valid && tri >= 0;
  const uint32_t pos = compact_hit(p, hit);
  if (valid) {
    const int64_t g = p.ray_base + ray;
    if (hit) {
      p.hits[pos] = make_uint2((uint32_t)ray, __float_as_uint(t));
    } else if (p.rgba) {
      p.rgba[g] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (p.tri_out) p.tri_out[g] = tri;
    if (p.t_out) p.t_out[g] = hit ? t : 0.0f;
  }
}

// Hit list of explicit rays from a forward pass's per-ray results (closest
// triangle, -1 = miss, and t), with the same compaction, for a backward pass
// that does not trace again.
__global__ void __launch_bounds__(256) k_hits_from_results(const __grid_constant__ Params p, const int32_t* tri,
                                                          const float* t) {
  const int64_t ray = (int64_t)blockIdx.x * 256 + threadIdx.x;
  const bool valid = ray < p.n_rays;
  const int32_t id = valid ? tri[ray] : -1;
  const bool hit = valid && id >= 0;
  const uint32_t pos = compact_hit(p, hit);
  if (hit) p.hits[pos] = make_uint2((uint32_t)ray, __float_as_uint(t[ray]));
}

// The decoupled variant's hit estimation (Sec. 4.2, Eq. 4) in place of the
// proxy trace: the density march of each ray, then the same compaction; the
// hit record carries the hit sample's t and alpha_c goes alongside.
// tri_out receives the hit sample k (-1 = miss), alpha_out alpha_c.
__global__ void __launch_bounds__(256, 5) k_march(const __grid_constant__ Params p, int32_t tiles_x, int32_t tiles_y) {
  int64_t ray;
  float o[3], d[3];
  const bool valid = thread_ray(p, tiles_x, tiles_y, ray, o, d);
  int32_t k = -1;
  float t = 0.0f, alpha = 0.0f;
  if (valid) march_ray(p.cub, p.lo, p.scale, o, d, k, t, alpha);
  const bool hit = valid && k >= 0;
  const uint32_t pos = compact_hit(p, hit);
  if (valid) {
    const int64_t g = p.ray_base + ray;
    if (hit) {
      p.hits[pos] = make_uint2((uint32_t)ray, __float_as_uint(t));
      p.hit_alpha[pos] = alpha;
    } else if (p.rgba) {
      p.rgba[g] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (p.tri_out) p.tri_out[g] = k;
    if (p.t_out) p.t_out[g] = hit ? t : 0.0f;
    if (p.alpha_out) p.alpha_out[g] = alpha;
  }
}

// ---------------------------------------------------------------------------
// k_shade (FP32 SIMT MLP), k_encode (stage outputs for parity checks) and
// the FP8 calibration pass (FP32 shade that records the largest |input| of
// each MLP layer instead of writing RGBA)
// ---------------------------------------------------------------------------
enum ShadeMode { kShade = 0, kEncode = 1, kAmax = 2 };

__device__ __forceinline__ void atomic_max_nonneg(uint32_t* addr, float v) {
  // non-negative floats order like their bit patterns
  atomicMax(addr, __float_as_uint(v));
}

template <int kMode>
__global__ void __launch_bounds__(128) k_shade_f32(const __grid_constant__ Params p) {
  constexpr bool kEncodeOnly = kMode == kEncode;
  extern __shared__ float4 smem4[];
  const int din = p.d_in;
  float amax_x = 0.f, amax_h1 = 0.f, amax_h2 = 0.f;
  const int nw = din * 64 + 64 * 64 + 64 * 4;
  if (!kEncodeOnly) {
    for (int k = threadIdx.x; k < nw / 4; k += blockDim.x)
      smem4[k] = reinterpret_cast<const float4*>(p.w_f32)[k];
    __syncthreads();
  }
  const float4* W1T = smem4;                       // [din][16] float4
  const float4* W2 = smem4 + din * 16;             // [64][16]
  const float4* W3T = smem4 + din * 16 + 64 * 16;  // [64] float4
  const uint32_t total = *p.counter;
  for (uint32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < total; h += gridDim.x * blockDim.x) {
    const uint2 rec = p.hits[h];
    const int64_t ray = rec.x;
    const float t = __uint_as_float(rec.y);
    float o[3], d[3];
    ray_of(p, ray, o, d);
    float x[3];
    hit_unit_coords(p, o, d, t, x);
    float h1[64];
    if (!kEncodeOnly) {
#pragma unroll
      for (int j = 0; j < 64; ++j) h1[j] = 0.0f;
    }
    encode_all_levels(p, x, [&](int l, float e0, float e1, const uint32_t* slots) {
      if (kEncodeOnly) {
        const int64_t g = p.ray_base + ray;
#pragma unroll
        for (int c = 0; c < 8; ++c) p.slots_out[(g * p.L + l) * 8 + c] = slots[c];
        p.feat_out[(g * p.L + l) * 2 + 0] = e0;
        p.feat_out[(g * p.L + l) * 2 + 1] = e1;
      } else {
        if (kMode == kAmax) amax_x = fmaxf(amax_x, fmaxf(fabsf(e0), fabsf(e1)));
        const float4* r0 = W1T + (2 * l) * 16;
        const float4* r1 = r0 + 16;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const float4 a = r0[q], b = r1[q];
          h1[4 * q + 0] += a.x * e0 + b.x * e1;
          h1[4 * q + 1] += a.y * e0 + b.y * e1;
          h1[4 * q + 2] += a.z * e0 + b.z * e1;
          h1[4 * q + 3] += a.w * e0 + b.w * e1;
        }
      }
    });
    if (kEncodeOnly) continue;
    float sh[16];
    sh16(p, d, sh);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float4* r = W1T + (2 * p.L + k) * 16;
      const float s = sh[k];
      if (kMode == kAmax) amax_x = fmaxf(amax_x, fabsf(s));
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const float4 a = r[q];
        h1[4 * q + 0] += a.x * s;
        h1[4 * q + 1] += a.y * s;
        h1[4 * q + 2] += a.z * s;
        h1[4 * q + 3] += a.w * s;
      }
    }
    if (p.variant) {  // alpha_c, the last input of F_s (Eq. 5)
      const float a_c = p.hit_alpha[h];
      if (kMode == kAmax) amax_x = fmaxf(amax_x, a_c);
      const float4* r = W1T + (2 * p.L + 16) * 16;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const float4 a = r[q];
        h1[4 * q + 0] += a.x * a_c;
        h1[4 * q + 1] += a.y * a_c;
        h1[4 * q + 2] += a.z * a_c;
        h1[4 * q + 3] += a.w * a_c;
      }
    }
#pragma unroll
    for (int j = 0; j < 64; ++j) {
      h1[j] = fmaxf(h1[j], 0.0f);
      if (kMode == kAmax) amax_h1 = fmaxf(amax_h1, h1[j]);
    }
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 2
    for (int j = 0; j < 64; ++j) {
      const float4* r = W2 + j * 16;
      float z = 0.0f;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const float4 a = r[q];
        z += a.x * h1[4 * q + 0];
        z += a.y * h1[4 * q + 1];
        z += a.z * h1[4 * q + 2];
        z += a.w * h1[4 * q + 3];
      }
      z = fmaxf(z, 0.0f);
      if (kMode == kAmax) amax_h2 = fmaxf(amax_h2, z);
      const float4 w3 = W3T[j];
      acc.x += w3.x * z;
      acc.y += w3.y * z;
      acc.z += w3.z * z;
      acc.w += w3.w * z;
    }
    if (kMode == kShade) {
      float4 out = make_float4(sigmoidf_(acc.x), sigmoidf_(acc.y), sigmoidf_(acc.z), sigmoidf_(acc.w));
      if (p.variant) {  // c = c_d + tint c_s (Eq. 7)
        const float4 dc = cube_diffuse(p.cub, x);
        out = make_float4(fmaf(dc.w, out.x, dc.x), fmaf(dc.w, out.y, dc.y), fmaf(dc.w, out.z, dc.z), out.w);
      }
      p.rgba[p.ray_base + ray] = out;
    }
  }
  if (kMode == kAmax) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      amax_x = fmaxf(amax_x, __shfl_xor_sync(0xffffffffu, amax_x, o));
      amax_h1 = fmaxf(amax_h1, __shfl_xor_sync(0xffffffffu, amax_h1, o));
      amax_h2 = fmaxf(amax_h2, __shfl_xor_sync(0xffffffffu, amax_h2, o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomic_max_nonneg(p.counter + 4, amax_x);
      atomic_max_nonneg(p.counter + 5, amax_h1);
      atomic_max_nonneg(p.counter + 6, amax_h2);
    }
  }
}

// ---------------------------------------------------------------------------
// k_shade_f32_tiled: FP32 SIMT shade over tiles of 128 hit rays per 256-thread
// CTA.  Gather: two threads per ray, each taking every other level (halving
// the chain of dependent Phi -> feature loads per thread); features and SH go
// to a shared [k][ray] FP32 tile.  MLP: each thread computes a 4-ray x
// 8-neuron block of a layer from shared memory (32 accumulators), the
// activations of the tile are exchanged through one 32 KB shared buffer, and
// layer 3 (64 -> 4) plus the sigmoid are computed per ray.
// ---------------------------------------------------------------------------
static constexpr int kF32Tile = 128;
static constexpr int kF32Threads = 256;

// (c0, c1) += a * (w.x, w.y) as one packed FP32 instruction: two IEEE fused
// multiply-adds rounded to nearest, the results of fmaf(a, w.x, c0), fmaf(a,
// w.y, c1).
__device__ __forceinline__ void fma2_rn(float& c0, float& c1, float a, float2 w) {
  uint64_t c = ((uint64_t)__float_as_uint(c1) << 32) | __float_as_uint(c0);
  const uint64_t av = ((uint64_t)__float_as_uint(a) << 32) | __float_as_uint(a);
  const uint64_t wv = ((uint64_t)__float_as_uint(w.y) << 32) | __float_as_uint(w.x);
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(c) : "l"(av), "l"(wv));
  c0 = __uint_as_float((uint32_t)c);
  c1 = __uint_as_float((uint32_t)(c >> 32));
}

// acc[i][j] = sum_k act[k][r0 + i] wT[k][n_j]: act [K][kF32Tile] (ray
// fastest), wT [K][64]; the 8 neurons n_j sit at columns w0 .. w0 + 3 and
// w1 .. w1 + 3 of wT (c0 and c0 + 4 in the natural layout).
__device__ __forceinline__ void block_gemm_4x8(const float* __restrict__ act, const float* __restrict__ wT, int K,
                                               int r0, int w0c, int w1c, float acc[4][8]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    const float4 a = *reinterpret_cast<const float4*>(act + k * kF32Tile + r0);
    const float4 w0 = *reinterpret_cast<const float4*>(wT + k * 64 + w0c);
    const float4 w1 = *reinterpret_cast<const float4*>(wT + k * 64 + w1c);
    const float av[4] = {a.x, a.y, a.z, a.w};
    const float2 wp[4] = {make_float2(w0.x, w0.y), make_float2(w0.z, w0.w), make_float2(w1.x, w1.y),
                          make_float2(w1.z, w1.w)};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) fma2_rn(acc[i][2 * j], acc[i][2 * j + 1], av[i], wp[j]);
  }
}

// Input tile of one hit ray, written by its two gather threads (half 0 and
// 1): features of levels half, half + 2, ... from the corner bundles (each
// with the next level's Phi entry in flight), the SH encoding and alpha_c (half 1), the diffuse colour
// and tint of the variant (half 0), all into the [k][kF32Tile] FP32 tile;
// invalid slots are zero.  Returns the ray index of the hit record.
// kStaged: the offset tables of levels 0 .. p.phis_levels - 1 are read from
// their shared-memory copies at sphi + p.phis_off[l].
template <bool kStaged>
__device__ __forceinline__ int64_t gather_tile_f32(const Params& p, uint32_t h, bool valid, int ray_slot, int half,
                                                   float* act, float* dif, const uint32_t* sphi = nullptr) {
  if (!valid) {
    for (int k = half; k < p.d_in; k += 2) act[k * kF32Tile + ray_slot] = 0.0f;
    return 0;
  }
  const uint2 rec = p.hits[h];
  const int64_t ray = rec.x;
  float o[3], d[3], x[3];
  ray_of(p, ray, o, d);
  hit_unit_coords(p, o, d, __uint_as_float(rec.y), x);
  auto fetch = [&](int l, LevelFetchB& f) {
    if (kStaged && l < p.phis_levels)
      fetch_bundle_phi_from(p.lv[l], sphi + p.phis_off[l], x, f);
    else
      fetch_bundle_phi(p.lv[l], x, f);
  };
  LevelFetchB fa, fb;
  if (half < p.L) fetch(half, fa);
  for (int l = half; l < p.L; l += 4) {  // levels half, half + 2, ... in pairs, no state copies
    float e0, e1;
    if (l + 2 < p.L) fetch(l + 2, fb);
    finish_bundle(p.lv[l], p.fp16, fa, e0, e1);
    act[(2 * l) * kF32Tile + ray_slot] = e0;
    act[(2 * l + 1) * kF32Tile + ray_slot] = e1;
    if (l + 2 >= p.L) break;
    if (l + 4 < p.L) fetch(l + 4, fa);
    finish_bundle(p.lv[l + 2], p.fp16, fb, e0, e1);
    act[(2 * (l + 2)) * kF32Tile + ray_slot] = e0;
    act[(2 * (l + 2) + 1) * kF32Tile + ray_slot] = e1;
  }
  if (half == 1) {
    float sh[16];
    sh16(p, d, sh);
#pragma unroll
    for (int k = 0; k < 16; ++k) act[(2 * p.L + k) * kF32Tile + ray_slot] = sh[k];
    if (p.variant) act[(2 * p.L + 16) * kF32Tile + ray_slot] = p.hit_alpha[h];  // alpha_c (Eq. 5)
  } else if (p.variant) {
    const float4 dc = cube_diffuse(p.cub, x);
    dif[0 * kF32Tile + ray_slot] = dc.x;
    dif[1 * kF32Tile + ray_slot] = dc.y;
    dif[2 * kF32Tile + ray_slot] = dc.z;
    dif[3 * kF32Tile + ray_slot] = dc.w;
  }
  return ray;
}

__global__ void __launch_bounds__(kF32Threads, 3) k_shade_f32_tiled(const __grid_constant__ Params p) {
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  const int din = p.d_in;
  float* W1T = sm;                 // [din][64]
  float* W2T = W1T + din * 64;     // [64][64]  (W2 transposed: [in][out])
  float* W3 = W2T + 64 * 64;       // [4][64]
  float* act = W3 + 4 * 64;        // [64][kF32Tile] activations of the tile
  float* dif = act + 64 * kF32Tile;  // variant: [4][kF32Tile] (c_d r, g, b, tint) of the tile's rays
  const int tid = threadIdx.x;
  // stage weights: W1T as packed on the host, W2 transposed here, W3 from W3T
  {
    const float* g = p.w_f32;
    for (int k = tid; k < din * 64; k += kF32Threads) W1T[k] = g[k];
    const float* g2 = g + din * 64;  // W2 [out][in]
    for (int k = tid; k < 64 * 64; k += kF32Threads) W2T[(k & 63) * 64 + (k >> 6)] = g2[k];
    const float* g3 = g2 + 64 * 64;  // W3T [in][4]
    for (int k = tid; k < 64 * 4; k += kF32Threads) W3[(k & 3) * 64 + (k >> 2)] = g3[k];
  }
  __syncthreads();
  const uint32_t total = *p.counter;
  const int ray_slot = tid & (kF32Tile - 1), half = tid >> 7;
  // MLP block of this thread: rays r0..r0+3, neurons c0..c0+7
  const int r0 = (tid & 31) * 4, c0 = (tid >> 5) * 8;
  for (uint32_t base = blockIdx.x * kF32Tile; base < total; base += gridDim.x * kF32Tile) {
    const uint32_t h = base + (uint32_t)ray_slot;
    const bool valid = h < total;
    const int64_t ray = gather_tile_f32<false>(p, h, valid, ray_slot, half, act, dif);
    __syncthreads();
    float acc[4][8];
    block_gemm_4x8(act, W1T, din, r0, c0, c0 + 4, acc);
    __syncthreads();  // every thread has read the inputs
#pragma unroll
    for (int j = 0; j < 8; ++j)
      *reinterpret_cast<float4*>(act + (c0 + j) * kF32Tile + r0) =
          make_float4(fmaxf(acc[0][j], 0.f), fmaxf(acc[1][j], 0.f), fmaxf(acc[2][j], 0.f), fmaxf(acc[3][j], 0.f));
    __syncthreads();
    block_gemm_4x8(act, W2T, 64, r0, c0, c0 + 4, acc);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 8; ++j)
      *reinterpret_cast<float4*>(act + (c0 + j) * kF32Tile + r0) =
          make_float4(fmaxf(acc[0][j], 0.f), fmaxf(acc[1][j], 0.f), fmaxf(acc[2][j], 0.f), fmaxf(acc[3][j], 0.f));
    __syncthreads();
    // layer 3: output channel pair (2 half, 2 half + 1) of ray ray_slot
    {
      float z0 = 0.f, z1 = 0.f;
      const float* w0 = W3 + (2 * half) * 64;
      const float* w1 = w0 + 64;
#pragma unroll 8
      for (int j = 0; j < 64; ++j) {
        const float a = act[j * kF32Tile + ray_slot];
        z0 = fmaf(w0[j], a, z0);
        z1 = fmaf(w1[j], a, z1);
      }
      if (valid) {
        float* out = reinterpret_cast<float*>(p.rgba + (p.ray_base + ray));
        float2 v = make_float2(sigmoidf_(z0), sigmoidf_(z1));
        if (p.variant) {  // c = c_d + tint c_s (Eq. 7); alpha stays F_s's
          const float tint = dif[3 * kF32Tile + ray_slot];
          v.x = fmaf(tint, v.x, dif[(2 * half) * kF32Tile + ray_slot]);
          if (half == 0) v.y = fmaf(tint, v.y, dif[1 * kF32Tile + ray_slot]);
        }
        *reinterpret_cast<float2*>(out + 2 * half) = v;
      }
    }
    __syncthreads();  // before the next tile overwrites the activations
  }
}

// ---------------------------------------------------------------------------
// k_shade_f32_ws: the FP32 shade of k_shade_f32_tiled with the gather and the
// MLP on separate warps, so that the latency-bound gather of some tiles runs
// beside the FMA-bound MLP of others.  One persistent CTA of 768 threads per
// SM:
//   * kWsTeams = 2 gather teams of 256 threads (two per ray, as in
//     gather_tile_f32) fill a ring of kWsSlots input tiles in shared memory;
//     local tile k goes to slot k % kWsSlots and is gathered by team
//     k % kWsTeams;
//   * 256 MLP threads take the tiles in order.  Warp w owns rays
//     16 w .. 16 w + 15 and all 64 neurons; lane l computes the 4-ray x
//     8-neuron block (rays 16 w + 4 (l & 3) .., neurons 8 (l >> 2) ..).
//     Layer 1 reads the slot (released right after it), layer 2 a private
//     hidden tile; layer 3 is folded into layer 2's epilogue: each lane
//     forms the partial sums of its 8 neurons for its 4 rays x 4 outputs,
//     and the 8 lanes of a ray group add them by a butterfly over lane bits
//     2..4 that leaves each lane one ray's channel pair.
// The staged W1^T and W2^T rows are permuted so that the first and second
// float4 of the 8 neuron octets are 128 contiguous bytes each: a warp's
// float4 weight load reads 8 distinct, bank-disjoint 16-byte chunks.
// Slot hand-over uses two mbarriers per slot (full: 256 gather arrivals,
// empty: 256 MLP arrivals), every wait bounded by the global timer (limit
// p.wait_ns); a warp whose wait runs out sets INOLF_FLAG_WAIT_TIMEOUT in the
// workspace error word and stops, and the others then run out in turn.  No other barrier joins warps: a gather
// warp writes its own rays of a tile, and an MLP warp's hidden activations
// are its own 16 columns of the hidden tile, so every warp runs at its own
// pace between the slot barriers.  Registers are split with
// setmaxnreg: the CTA is launched with kWsLaunchRegs per thread (the host
// checks the compiled count before launching), the gather warpgroups give
// registers back and the MLP warpgroups take them.
// ---------------------------------------------------------------------------
static constexpr int kWsTeams = 2, kWsSlots = 4, kWsMlp = 256;
static constexpr int kWsThreads = 256 * kWsTeams + kWsMlp;
static constexpr int kWsLaunchRegs = 80, kWsGatherRegs = 64, kWsMlpRegs = 112;
static_assert(kWsTeams * 256 * kWsGatherRegs + kWsMlp * kWsMlpRegs <= kWsThreads * kWsLaunchRegs,
              "register split exceeds the CTA's launch allocation");
static_assert(kWsThreads * kWsLaunchRegs <= 65536, "launch allocation exceeds the register file");
// Shared memory of one ws CTA with its staged offset tables.  The SM splits
// its 256 KB between shared memory and L1 in steps; below the 196 KB step
// (less the 1 KB the CTA reserves) about 60 KB of L1 stay for the fine
// levels' tables.  On the full scene this stages levels 0-2 (0.3% faster
// than none); staging level 3 as well crosses the step and measured 8%
// slower.
static constexpr size_t kWsPhiSmemLimit = 195 * 1024;
static constexpr uint64_t kRingWaitLimitNs = 2000000000ull;  // default hand-over limit: 2 s; a tile takes microseconds

// shared-memory floats of one ring slot: inputs [d_in][tile], diffuse
// [4][tile], ray ids [tile]
__host__ __device__ constexpr int ws_slot_floats(int din) { return (din + 5) * kF32Tile; }
// Bytes before the staged offset tables: weights, hidden tile, ring, the
// full/empty barriers and the staging barrier (padded to 16 bytes, so the
// tables that follow start 16-byte aligned).
__host__ __device__ constexpr size_t ws_smem_bytes(int din) {
  return (size_t)(din * 64 + 64 * 64 + 4 * 64 + 64 * kF32Tile + kWsSlots * ws_slot_floats(din)) * sizeof(float) +
         (2 * kWsSlots + 2) * sizeof(uint64_t);
}
static_assert(ws_smem_bytes(2 * INOLF_MAX_LEVELS + 17) <= 227 * 1024,
              "the largest input tile (16 levels, alpha_c) must fit one CTA's shared memory");
static_assert(ws_smem_bytes(0) % 16 == 0 && ws_smem_bytes(1) % 16 == 0, "staged tables must start 16-byte aligned");
// The raw FP32 weights land in the ring before it carries tiles: the ring
// holds them for every d_in >= 4 (d_in is at least 18: one level and the 16
// direction coefficients).
static_assert((size_t)kWsSlots * ws_slot_floats(4) >= (size_t)(4 * 64 + 64 * 64 + 4 * 64),
              "ring too small for the weight blob");
// column of neuron c in the permuted W^T rows: octet c / 8, float4 half (c / 4) & 1
__device__ __forceinline__ int ws_wcol(int c) { return ((c >> 2) & 1) * 32 + (c >> 3) * 4 + (c & 3); }

// Adds v over the lanes that differ in lane bit `bit`, keeping the half of
// the n values selected by that bit (reduce-scatter step): v[0 .. n/2) is
// the kept half afterwards.
template <int n>
__device__ __forceinline__ void butterfly_keep(float (&v)[16], int bit) {
  const bool hi = (threadIdx.x >> bit) & 1;
#pragma unroll
  for (int m = 0; m < n / 2; ++m) {
    const float mine = hi ? v[n / 2 + m] : v[m];
    const float give = hi ? v[m] : v[n / 2 + m];
    v[m] = mine + __shfl_xor_sync(0xffffffffu, give, 1 << bit);
  }
}

__global__ void __launch_bounds__(kWsThreads, 1) k_shade_f32_ws(const __grid_constant__ Params p) {
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  const int din = p.d_in;
  float* W1T = sm;              // [din][64], permuted columns
  float* W2T = W1T + din * 64;  // [64][64] (W2 transposed: [in][out]), permuted columns
  float* W3T = W2T + 64 * 64;   // [64][4]
  float* hid = W3T + 4 * 64;    // [64][kF32Tile] hidden activations (MLP threads)
  float* ring = hid + 64 * kF32Tile;
  const int slot_floats = ws_slot_floats(din);
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + kWsSlots * slot_floats);
  uint64_t* empty = full + kWsSlots;
  uint64_t* staged = empty + kWsSlots;                           // weights and tables landed
  const uint32_t* sphi = reinterpret_cast<uint32_t*>(staged + 2);  // 16-byte aligned
  const int tid = threadIdx.x;
  // Staging by the bulk-copy engine: the raw weight blob into the (still
  // unused) ring, and the offset tables of levels 0 .. phis_levels - 1 to
  // their place after the barriers, all completing on one barrier.
  const uint32_t wbytes = (uint32_t)(din * 64 + 64 * 64 + 64 * 4) * 4u;
  if (tid == 0) {
    for (int s = 0; s < kWsSlots; ++s) {
      tc::mbar_init(&full[s], 256);
      tc::mbar_init(&empty[s], kWsMlp);
    }
    tc::mbar_init(staged, 1);
    tc::fence_mbar_init();
    tc::mbar_arrive_expect_tx(staged, wbytes + p.phis_off[p.phis_levels] * 4u);
    tc::bulk_g2s(ring, p.w_f32, wbytes, staged);
    for (int l = 0; l < p.phis_levels; ++l)
      tc::bulk_g2s(const_cast<uint32_t*>(sphi) + p.phis_off[l], p.lv[l].phi,
                   (p.phis_off[l + 1] - p.phis_off[l]) * 4u, staged);
  }
  __syncthreads();  // barrier initialised before anyone polls it
  if (!tc::mbar_wait(staged, 0u, p.wait_ns)) {
    if (tid == 0) atomicOr(p.counter + 1, INOLF_FLAG_WAIT_TIMEOUT);
    tc::mbar_wait(staged, 0u, p.wait_ns);  // copies still in flight land before the CTA leaves
    return;
  }
  {
    const float* g = ring;  // W1^T [din][64]
    for (int k = tid; k < din * 64; k += kWsThreads) W1T[(k & ~63) + ws_wcol(k & 63)] = g[k];
    const float* g2 = g + din * 64;  // W2 [out][in]
    for (int k = tid; k < 64 * 64; k += kWsThreads) W2T[(k & 63) * 64 + ws_wcol(k >> 6)] = g2[k];
    const float* g3 = g2 + 64 * 64;  // W3^T [in][4]
    for (int k = tid; k < 64 * 4; k += kWsThreads) W3T[k] = g3[k];
  }
  __syncthreads();  // the ring's weight copy is read before the gathers overwrite it
  const uint32_t total = *p.counter;
  const uint32_t n_tiles = (total + kF32Tile - 1) / kF32Tile;
  const uint32_t n_k = blockIdx.x < n_tiles ? (n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0u;

  if (tid < 256 * kWsTeams) {  // ---- gather team tid / 256 ----
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(kWsGatherRegs));
    const int team = tid >> 8, gt = tid & 255;
    const int ray_slot = gt & (kF32Tile - 1), half = gt >> 7;
    for (uint32_t k = (uint32_t)team; k < n_k; k += kWsTeams) {
      const uint32_t s = k % kWsSlots;
      if (k >= (uint32_t)kWsSlots) {  // the MLP threads released the tile k - kWsSlots
        const bool ok = tc::mbar_wait(&empty[s], (k / kWsSlots - 1u) & 1u, p.wait_ns);
        if (__any_sync(0xffffffffu, !ok)) {
          if ((gt & 31) == 0) atomicOr(p.counter + 1, INOLF_FLAG_WAIT_TIMEOUT);
          break;
        }
      }
      float* in = ring + s * slot_floats;
      float* dif = in + din * kF32Tile;
      uint32_t* rid = reinterpret_cast<uint32_t*>(dif + 4 * kF32Tile);
      const uint32_t h = (blockIdx.x + k * gridDim.x) * kF32Tile + (uint32_t)ray_slot;
      const int64_t ray = gather_tile_f32<true>(p, h, h < total, ray_slot, half, in, dif, sphi);
      if (half == 0) rid[ray_slot] = (uint32_t)ray;
      if (!(p.inject & INOLF_INJECT_RING_STALL)) tc::mbar_arrive(&full[s]);  // injected stall: never handed over
    }
    return;
  }

  // ---- MLP threads ----
  asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(kWsMlpRegs));
  const int mt = tid - 256 * kWsTeams, lane = mt & 31, warp = mt >> 5;
  const int r0 = warp * 16 + (lane & 3) * 4, nb = lane >> 2, c0 = nb * 8;
  // after the butterfly: ray r0 + out_i, channels 2 out_cp, 2 out_cp + 1
  const int out_i = ((lane >> 4) & 1) * 2 + ((lane >> 3) & 1), out_cp = (lane >> 2) & 1;
  const int out_ray = r0 + out_i;
  for (uint32_t k = 0; k < n_k; ++k) {
    const uint32_t s = k % kWsSlots;
    const bool ok = tc::mbar_wait(&full[s], (k / kWsSlots) & 1u, p.wait_ns);
    if (__any_sync(0xffffffffu, !ok)) {
      if (lane == 0) atomicOr(p.counter + 1, INOLF_FLAG_WAIT_TIMEOUT);
      break;
    }
    const float* in = ring + s * slot_floats;
    const float* dif = in + din * kF32Tile;
    const uint32_t* rid = reinterpret_cast<const uint32_t*>(dif + 4 * kF32Tile);
    const uint32_t h = (blockIdx.x + k * gridDim.x) * kF32Tile + (uint32_t)out_ray;
    const bool valid = h < total;
    // what the output needs from the slot, read before the slot is released
    const uint32_t ray = valid ? rid[out_ray] : 0u;
    float dc0 = 0.f, dc1 = 0.f, tint = 0.f;
    if (p.variant && valid) {
      dc0 = dif[(2 * out_cp) * kF32Tile + out_ray];
      dc1 = dif[(2 * out_cp + 1) * kF32Tile + out_ray];  // unused for the alpha channel
      tint = dif[3 * kF32Tile + out_ray];
    }
    float acc[4][8];
    block_gemm_4x8(in, W1T, din, r0, nb * 4, 32 + nb * 4, acc);
    if (k + kWsSlots < n_k) tc::mbar_arrive(&empty[s]);
#pragma unroll
    for (int j = 0; j < 8; ++j)
      *reinterpret_cast<float4*>(hid + (c0 + j) * kF32Tile + r0) =
          make_float4(fmaxf(acc[0][j], 0.f), fmaxf(acc[1][j], 0.f), fmaxf(acc[2][j], 0.f), fmaxf(acc[3][j], 0.f));
    __syncwarp();  // the warp's own 16 hidden columns
    block_gemm_4x8(hid, W2T, 64, r0, nb * 4, 32 + nb * 4, acc);
    // layer 3 partial sums of this lane's 8 neurons: v[4 i + c], ray r0 + i, output c
    float v[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float4 w = *reinterpret_cast<const float4*>(W3T + (c0 + j) * 4);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float a = fmaxf(acc[i][j], 0.f);
        v[4 * i + 0] = fmaf(w.x, a, v[4 * i + 0]);
        v[4 * i + 1] = fmaf(w.y, a, v[4 * i + 1]);
        v[4 * i + 2] = fmaf(w.z, a, v[4 * i + 2]);
        v[4 * i + 3] = fmaf(w.w, a, v[4 * i + 3]);
      }
    }
    butterfly_keep<16>(v, 4);  // rays (0, 1) or (2, 3)
    butterfly_keep<8>(v, 3);   // one ray
    butterfly_keep<4>(v, 2);   // one channel pair: v[0], v[1]
    if (valid) {
      float2 o = make_float2(sigmoidf_(v[0]), sigmoidf_(v[1]));
      if (p.variant) {  // c = c_d + tint c_s (Eq. 7); alpha stays F_s's
        o.x = fmaf(tint, o.x, dc0);
        if (out_cp == 0) o.y = fmaf(tint, o.y, dc1);
      }
      *reinterpret_cast<float2*>(reinterpret_cast<float*>(p.rgba + (p.ray_base + (int64_t)ray)) + 2 * out_cp) = o;
    }
    __syncwarp();  // layer 2 has read the hidden columns before the next tile's layer 1 writes them
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static constexpr size_t kWsHeader = 256;

// Operand tiles of the split tensor-core shade: 128 bytes per hit row (the
// widest first-layer row, 64 BF16 inputs) for up to tc_chunk_rows() hits at
// a time, plus 256 bytes of alignment slack.  4 Mi rows (512 MiB): 64 4K
// views take about 95 encode/MLP launch pairs, as fast as 16 Mi rows and 5 %
// faster than 1 Mi.  INOLF_TC_CHUNK_ROWS overrides it (read at every call;
// below 256 the fused kernel runs).
static size_t tc_chunk_rows() {
  const char* e = std::getenv("INOLF_TC_CHUNK_ROWS");
  return e ? (size_t)std::max(0ll, std::atoll(e)) : ((size_t)1 << 22);
}
static size_t tc_region_bytes(int64_t n_rays) {
  const size_t n = ((size_t)std::max<int64_t>(n_rays, 1) + 255) / 256 * 256;
  return std::min(n, tc_chunk_rows()) * 128 + 256;
}
size_t workspace_bytes(int64_t n_rays) {
  return kWsHeader + (size_t)std::max<int64_t>(n_rays, 1) * 12 + tc_region_bytes(n_rays);
}
static size_t workspace_bytes_min() { return workspace_bytes(1); }

std::atomic<int64_t> g_wait_ns{0};     // inolf_set_wait_limit_ns (0 = default)
std::atomic<uint32_t> g_inject{0};     // inolf_set_fault_injection

int device_index() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  return dev >= 0 && dev < kMaxDevices ? dev : -1;
}

static int sm_count() {
  static int n[kMaxDevices] = {};
  static std::once_flag once[kMaxDevices];
  const int dev = std::max(device_index(), 0);
  std::call_once(once[dev], [dev] {
    cudaDeviceGetAttribute(&n[dev], cudaDevAttrMultiProcessorCount, dev);
    if (n[dev] <= 0) n[dev] = 1;
  });
  return n[dev];
}

static void fill_common(const Object& obj, Params& p) {
  p.nodes = (const float4*)obj.nodes;
  p.tris = (const float4*)obj.tris;
  p.L = obj.L;
  p.lo = obj.lo;
  p.scale = obj.scale;
  p.fp16 = obj.fp16;
  for (int l = 0; l < obj.L; ++l) p.lv[l] = obj.lv[l];
  p.d_in = obj.d_in;
  p.w_f32 = obj.w_f32;
  p.w_bf16 = obj.w_bf16;
  p.w_fp8 = obj.w_fp8;
  p.w_tf32 = obj.w_tf32;
  p.tc_k1_tf32 = obj.tc_k1_tf32;
  p.tc_bytes_tf32 = obj.tc_bytes_tf32;
  p.tc_k1_bf16 = obj.tc_k1_bf16;
  p.tc_k1_fp8 = obj.tc_k1_fp8;
  p.tc_bytes_bf16 = obj.tc_bytes_bf16;
  p.tc_bytes_fp8 = obj.tc_bytes_fp8;
  p.fp8_w_scale = obj.w_scale_dev;
  for (int k = 0; k < 3; ++k) p.fp8_act_scale[k] = obj.fp8_act_scale[k];
  sh_constants(p.shc);
  p.variant = obj.variant;
  p.cub = obj.cub;
  const int64_t w = g_wait_ns.load();
  p.wait_ns = w > 0 ? (uint64_t)w : kRingWaitLimitNs;
  p.inject = g_inject.load();
}

// Hit list (cap records) and, for the variant, the alpha_c array after it.
static int64_t place_hit_list(const Object& obj, void* workspace, size_t ws_bytes, Params& p) {
  const int64_t cap = (int64_t)((ws_bytes - kWsHeader) / hit_bytes_per_ray(obj));
  p.counter = (uint32_t*)workspace;
  p.hits = (uint2*)((char*)workspace + kWsHeader);
  p.hit_alpha = obj.variant ? reinterpret_cast<float*>(p.hits + cap) : nullptr;
  return cap;
}

static inolf_status check_launch(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(INOLF_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
  return INOLF_OK;
}

inolf_status flags_status(uint32_t flags, const char* what) {
  if (!flags) return INOLF_OK;
  char hex[16];
  std::snprintf(hex, sizeof(hex), "0x%x", flags);
  std::string m = std::string(what) + ": device-side failure flags " + hex + " (";
  if (flags & INOLF_FLAG_WAIT_TIMEOUT) m += " a bounded wait in a shade kernel ran out;";
  if (flags & INOLF_FLAG_STACK_OVERFLOW) m += " a BVH traversal stack overflowed;";
  if (flags & INOLF_FLAG_TRAVERSAL_LIMIT) m += " a BVH traversal exceeded its step limit;";
  m += " the results of the rays concerned are incomplete)";
  return fail((flags & INOLF_FLAG_WAIT_TIMEOUT) ? INOLF_E_TIMEOUT : INOLF_E_DEVICE, m);
}

inolf_status read_device_flags(const void* ws, void* stream, uint32_t* flags) {
  cudaStream_t st = (cudaStream_t)stream;
  const void* hdr = ws;
  if (!hdr) {
    void* sc = nullptr;
    inolf_status s = noalloc_scratch_address(&sc);
    if (s != INOLF_OK) return s;
    hdr = sc;
  }
  uint32_t f = 0;
  if (cudaMemcpyAsync(&f, static_cast<const uint32_t*>(hdr) + 1, sizeof(f), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(INOLF_E_CUDA, "reading the device failure flags failed");
  *flags = f;
  return INOLF_OK;
}

inolf_status launch_shade_tc(const Params& p, inolf_precision prec, cudaStream_t st);  // mlp_tc.cu

inolf_status launch_render(const Object& obj, const RayBatch& rays, inolf_precision prec, float* rgba,
                           int32_t* tri_out, float* t_out, uint32_t* slots_out, float* feat_out,
                           void* workspace, size_t ws_bytes, void* stream, bool amax, float* alpha_out,
                           bool hits_only, bool count_trace, bool clear_flags) {
  cudaStream_t st = (cudaStream_t)stream;
  if (!workspace || ws_bytes < workspace_bytes(1) || ((uintptr_t)workspace & 15))
    return fail(INOLF_E_INVALID, "render: workspace missing, too small or not 16-byte aligned");
  const int dev = device_index();
  if (dev < 0) return fail(INOLF_E_UNSUPPORTED, "render: no current device, or a device index beyond 63");
  const bool encode = slots_out != nullptr;
  if (!encode && prec != INOLF_FP32 && prec != INOLF_BF16 && prec != INOLF_FP8)
    return fail(INOLF_E_INVALID, "render: unknown precision");
  if (!encode && prec == INOLF_FP8 && !(obj.fp8_act_scale[0] > 0))
    return fail(INOLF_E_INVALID, "render: FP8 needs activation scales (inolf_object_set_fp8_scales)");
  Params p{};
  fill_common(obj, p);
  // The split tensor-core shade keeps its operand tiles at the end of the
  // workspace beside one view's (or all the rays') hit records: the full
  // tile region when the workspace holds it, else what the hit records
  // leave, as long as that is at least 256 rows of this precision;
  // otherwise the fused kernel (BF16 / FP8) or the FP32 SIMT kernel runs.
  size_t hit_ws = ws_bytes;
  if (!encode && !amax && !hits_only && tc_chunk_rows() >= 256) {
    const int64_t n_call = rays.mode == 0 ? (int64_t)rays.n_views * rays.W * rays.H : rays.n;
    const int64_t min_hits = rays.mode == 0 ? (int64_t)rays.W * rays.H : n_call;
    const size_t hits_min = kWsHeader + (size_t)min_hits * hit_bytes_per_ray(obj);
    size_t a_bytes = tc_region_bytes(n_call);
    if (ws_bytes < hits_min + a_bytes && ws_bytes > hits_min) a_bytes = (ws_bytes - hits_min) / 256 * 256;
    const size_t row_bytes = prec == INOLF_FP32 ? 4u * (size_t)obj.tc_k1_tf32
                             : prec == INOLF_FP8 ? (size_t)obj.tc_k1_fp8
                                                 : 2u * (size_t)obj.tc_k1_bf16;
    if (ws_bytes >= hits_min + a_bytes && row_bytes > 0 && a_bytes >= 256 + 256 * row_bytes) {
      hit_ws = (ws_bytes - a_bytes + 255) / 256 * 256;
      p.tc_a = (uint8_t*)workspace + hit_ws;
      p.tc_a_bytes = (uint64_t)(ws_bytes - hit_ws);
    }
  }
  const int64_t cap = place_hit_list(obj, workspace, hit_ws, p);
  uint32_t* counter = p.counter;
  p.mode = rays.mode;
  p.rgba = (float4*)rgba;
  p.tri_out = tri_out;
  p.t_out = t_out;
  p.slots_out = slots_out;
  p.feat_out = feat_out;
  p.alpha_out = alpha_out;

  const size_t smem_f32 = (size_t)(obj.d_in * 64 + 64 * 64 + 64 * 4) * sizeof(float);
  static std::once_flag attr_once[kMaxDevices];
  std::call_once(attr_once[dev], [&] {
    cudaFuncSetAttribute(k_shade_f32<kShade>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    cudaFuncSetAttribute(k_shade_f32<kShade>, cudaFuncAttributePreferredSharedMemoryCarveout, 50);
    cudaFuncSetAttribute(k_shade_f32<kAmax>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
  });
  const int shade_grid = sm_count() * 8;
  const size_t smem_f32_tiled =
      (size_t)(obj.d_in * 64 + 64 * 64 + 4 * 64 + 64 * kF32Tile + (obj.variant ? 4 * kF32Tile : 0)) * sizeof(float);
  static std::once_flag tiled_once[kMaxDevices];
  static int f32_ctas_dev[kMaxDevices];
  std::call_once(tiled_once[dev], [&] {
    int& f32_ctas = f32_ctas_dev[dev];
    // the largest configuration: 16 levels, alpha_c input and the diffuse tile
    const size_t mx =
        (size_t)((2 * INOLF_MAX_LEVELS + 17) * 64 + 64 * 64 + 4 * 64 + 64 * kF32Tile + 4 * kF32Tile) * sizeof(float);
    cudaFuncSetAttribute(k_shade_f32_tiled, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&f32_ctas, k_shade_f32_tiled, kF32Threads, mx);
    if (f32_ctas < 1) f32_ctas = 1;
    cudaGetLastError();
  });
  const int f32_grid = sm_count() * f32_ctas_dev[dev];
  static std::once_flag ws_once[kMaxDevices];
  static bool ws_ok_dev[kMaxDevices];  // compiled with the register count its split assumes
  static size_t ws_smem_max_dev[kMaxDevices];
  std::call_once(ws_once[dev], [&] {
    cudaFuncAttributes fa{};
    ws_ok_dev[dev] = cudaFuncGetAttributes(&fa, k_shade_f32_ws) == cudaSuccess && fa.numRegs == kWsLaunchRegs;
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t mx = std::max((size_t)optin, ws_smem_bytes(2 * INOLF_MAX_LEVELS + 17)) - fa.sharedSizeBytes;
    ws_smem_max_dev[dev] = cudaFuncSetAttribute(k_shade_f32_ws, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)mx) == cudaSuccess ? mx : ws_smem_bytes(2 * INOLF_MAX_LEVELS + 17);
    cudaGetLastError();
  });

  const bool ws_ok = ws_ok_dev[dev];
  // The offset tables of the coarsest levels go to shared memory
  // while they fit beside the tiles (each padded to 16 bytes, as allocated).
  size_t smem_ws = ws_smem_bytes(obj.d_in);
  p.phis_levels = 0;
  p.phis_off[0] = 0;
  for (int l = 0; l < obj.L && ws_ok; ++l) {
    const size_t r = (size_t)obj.lv[l].r, words = (r * r * r + 3) / 4 * 4;  // as allocated
    if (smem_ws + (p.phis_off[l] + words) * 4 > std::min(ws_smem_max_dev[dev], kWsPhiSmemLimit)) break;
    p.phis_off[l + 1] = p.phis_off[l] + (uint32_t)words;
    p.phis_levels = l + 1;
  }
  smem_ws += (size_t)p.phis_off[p.phis_levels] * 4;
  // the hit counter restarts with every chunk; the failure flags (word 1)
  // accumulate over the call
  bool first_chunk = clear_flags;
  auto run_chunk = [&](int64_t n_chunk, int32_t tiles_x, int32_t tiles_y, int64_t trace_blocks) -> inolf_status {
    if (cudaMemsetAsync(counter, 0, first_chunk ? 8 : 4, st) != cudaSuccess)
      return fail(INOLF_E_CUDA, "cudaMemsetAsync failed");
    first_chunk = false;
    (void)n_chunk;
    if (obj.variant) {
      {
        LaunchTimer lt("k_march", st);
        k_march<<<(unsigned)trace_blocks, 256, 0, st>>>(p, tiles_x, tiles_y);
      }
      inolf_status s = check_launch("k_march");
      if (s != INOLF_OK) return s;
    } else {
      {
        LaunchTimer lt("k_trace", st);
        if (count_trace) k_trace<true><<<(unsigned)trace_blocks, 256, 0, st>>>(p, tiles_x, tiles_y);
        else k_trace<false><<<(unsigned)trace_blocks, 256, 0, st>>>(p, tiles_x, tiles_y);
      }
      inolf_status s = check_launch("k_trace");
      if (s != INOLF_OK) return s;
    }
    if (hits_only) return INOLF_OK;
    if (encode) {
      LaunchTimer lt("k_encode", st);
      k_shade_f32<kEncode><<<shade_grid, 128, 0, st>>>(p);
      return check_launch("k_encode");
    }
    if (amax) {
      LaunchTimer lt("k_shade_amax", st);
      k_shade_f32<kAmax><<<shade_grid, 128, smem_f32, st>>>(p);
      return check_launch("k_shade_amax");
    }
    if (prec == INOLF_FP32 && !p.tc_a) {
      {
        LaunchTimer lt("k_shade_f32", st);
        if (ws_ok) k_shade_f32_ws<<<sm_count(), kWsThreads, smem_ws, st>>>(p);
        else k_shade_f32_tiled<<<f32_grid, kF32Threads, smem_f32_tiled, st>>>(p);
      }
      return check_launch("k_shade_f32");
    }
    return launch_shade_tc(p, prec, st);
  };

  if (rays.mode == 0) {
    const int64_t per_view = (int64_t)rays.W * rays.H;
    if (per_view > 0xFFFFFFFFll) return fail(INOLF_E_INVALID, "render: view too large");
    int64_t vpc = std::min<int64_t>(kMaxViewsPerLaunch, cap / per_view);
    vpc = std::min<int64_t>(vpc, (int64_t)0xFFFFFFFFll / per_view);
    if (vpc < 1) return fail(INOLF_E_INVALID, "render: workspace smaller than one view's hit list");
    p.W = rays.W;
    p.H = rays.H;
    const int32_t tx = (rays.W + 15) / 16, ty = (rays.H + 15) / 16;
    for (int32_t v0 = 0; v0 < rays.n_views; v0 += (int32_t)vpc) {
      const int32_t nv = (int32_t)std::min<int64_t>(vpc, rays.n_views - v0);
      for (int k = 0; k < 13 * nv; ++k) p.cams[k] = rays.cams[13 * v0 + k];
      p.ray_base = (int64_t)v0 * per_view;
      p.n_rays = (int64_t)nv * per_view;
      inolf_status s = run_chunk(p.n_rays, tx, ty, (int64_t)nv * tx * ty);
      if (s != INOLF_OK) return s;
    }
  } else {
    int64_t chunk = std::min<int64_t>(cap, 0xFFFFFFFFll);
    for (int64_t r0 = 0; r0 < rays.n; r0 += chunk) {
      const int64_t nr = std::min(chunk, rays.n - r0);
      p.ro = rays.o + 3 * r0;
      p.rd = rays.d + 3 * r0;
      p.ray_base = r0;
      p.n_rays = nr;
      // outputs are indexed by ray_base + local index; inputs by local index
      inolf_status s = run_chunk(nr, 0, 0, (nr + 255) / 256);
      if (s != INOLF_OK) return s;
    }
  }
  return INOLF_OK;
}

inolf_status launch_backward(const Params& p, const BwdParams& b, cudaStream_t st);  // backward.cu

inolf_status launch_backward_rays(const Object& obj, const float* o, const float* d, int64_t n, const float* d_rgba,
                                  float* const* grad_tables, float* gw1, float* gw2, float* gw3, void* workspace,
                                  size_t ws_bytes, void* stream, const int32_t* tri_in, const float* t_in) {
  cudaStream_t st = (cudaStream_t)stream;
  if (obj.variant)
    return fail(INOLF_E_UNSUPPORTED, "backward: objects with density cubes have no backward in this library");
  if (!workspace || ws_bytes < workspace_bytes(1) || ((uintptr_t)workspace & 15))
    return fail(INOLF_E_INVALID, "backward: workspace missing, too small or not 16-byte aligned");
  const int64_t cap = (int64_t)((ws_bytes - kWsHeader) / 8);
  Params p{};
  fill_common(obj, p);
  p.mode = 1;
  p.counter = (uint32_t*)workspace;
  p.hits = (uint2*)((char*)workspace + kWsHeader);
  BwdParams b{};
  for (int l = 0; l < obj.L; ++l) b.gtab[l] = grad_tables[l];
  b.gw1 = gw1;
  b.gw2 = gw2;
  b.gw3 = gw3;
  b.d_rgba = d_rgba;
  const int64_t chunk = std::min<int64_t>(cap, 0xFFFFFFFFll);
  for (int64_t r0 = 0; r0 < n; r0 += chunk) {
    const int64_t nr = std::min(chunk, n - r0);
    p.ro = o + 3 * r0;
    p.rd = d + 3 * r0;
    p.ray_base = r0;
    p.n_rays = nr;
    // hit counter per chunk, failure flags (word 1) once per call
    if (cudaMemsetAsync(p.counter, 0, r0 == 0 ? 8 : 4, st) != cudaSuccess)
      return fail(INOLF_E_CUDA, "cudaMemsetAsync failed");
    inolf_status s;
    if (tri_in) {  // the forward's hits: compact them instead of tracing again
      {
        LaunchTimer lt("k_hits_from_results", st);
        k_hits_from_results<<<(unsigned)((nr + 255) / 256), 256, 0, st>>>(p, tri_in + r0, t_in + r0);
      }
      s = check_launch("k_hits_from_results");
    } else {
      {
        LaunchTimer lt("k_trace", st);
        k_trace<false><<<(unsigned)((nr + 255) / 256), 256, 0, st>>>(p, 0, 0);
      }
      s = check_launch("k_trace");
    }
    if (s != INOLF_OK) return s;
    s = launch_backward(p, b, st);
    if (s != INOLF_OK) return s;
  }
  return INOLF_OK;
}

}  // namespace inolf

using namespace inolf;

extern "C" inolf_status inolf_backward(const inolf_object* obj, const float* o, const float* d, int64_t n,
                                       const float* d_rgba, float* const* grad_tables, float* grad_w1,
                                       float* grad_w2, float* grad_w3, void* workspace, size_t workspace_bytes,
                                       void* stream) {
  clear_error();
  if (!obj || n < 0 || (n > 0 && (!o || !d || !d_rgba || !grad_tables || !grad_w1 || !grad_w2 || !grad_w3)))
    return fail(INOLF_E_INVALID, "inolf_backward: bad argument");
  for (int l = 0; n > 0 && l < obj->o.L; ++l)
    if (!grad_tables[l]) return fail(INOLF_E_INVALID, "inolf_backward: missing gradient table");
  if (n == 0) return INOLF_OK;
  return launch_backward_rays(obj->o, o, d, n, d_rgba, grad_tables, grad_w1, grad_w2, grad_w3, workspace,
                              workspace_bytes, stream, nullptr, nullptr);
}

extern "C" inolf_status inolf_backward_hits(const inolf_object* obj, const float* o, const float* d, int64_t n,
                                            const int32_t* tri, const float* t, const float* d_rgba,
                                            float* const* grad_tables, float* grad_w1, float* grad_w2,
                                            float* grad_w3, void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  if (!obj || n < 0 ||
      (n > 0 && (!o || !d || !tri || !t || !d_rgba || !grad_tables || !grad_w1 || !grad_w2 || !grad_w3)))
    return fail(INOLF_E_INVALID, "inolf_backward_hits: bad argument");
  for (int l = 0; n > 0 && l < obj->o.L; ++l)
    if (!grad_tables[l]) return fail(INOLF_E_INVALID, "inolf_backward_hits: missing gradient table");
  if (n == 0) return INOLF_OK;
  return launch_backward_rays(obj->o, o, d, n, d_rgba, grad_tables, grad_w1, grad_w2, grad_w3, workspace,
                              workspace_bytes, stream, tri, t);
}

extern "C" size_t inolf_render_workspace_bytes(int64_t n_rays) { return inolf::workspace_bytes(n_rays); }

extern "C" inolf_status inolf_workspace_flags(const void* workspace, uint32_t* flags, void* stream) {
  clear_error();
  if (!flags) return fail(INOLF_E_INVALID, "inolf_workspace_flags: NULL flags");
  *flags = 0;
  inolf_status s = read_device_flags(workspace, stream, flags);
  if (s != INOLF_OK) return s;
  return flags_status(*flags, "inolf_workspace_flags");
}

extern "C" inolf_status inolf_set_wait_limit_ns(int64_t ns) {
  clear_error();
  if (ns < 0) return fail(INOLF_E_INVALID, "inolf_set_wait_limit_ns: negative limit");
  g_wait_ns.store(ns);
  return INOLF_OK;
}

extern "C" inolf_status inolf_set_fault_injection(uint32_t mask) {
  clear_error();
  g_inject.store(mask);
  return INOLF_OK;
}

extern "C" inolf_status inolf_render(const inolf_object* obj, const float* cams, int32_t n_views, int32_t W,
                                     int32_t H, inolf_precision prec, float* rgba_out, int32_t* tri_out,
                                     float* t_out, void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  if (!obj || !cams || !rgba_out || n_views < 0 || W <= 0 || H <= 0)
    return fail(INOLF_E_INVALID, "inolf_render: bad argument");
  if (n_views == 0) return INOLF_OK;
  RayBatch rb{};
  rb.mode = 0;
  rb.cams = cams;
  rb.n_views = n_views;
  rb.W = W;
  rb.H = H;
  rb.n = (int64_t)n_views * W * H;
  return launch_render(obj->o, rb, prec, rgba_out, tri_out, t_out, nullptr, nullptr, workspace, workspace_bytes,
                       stream);
}

extern "C" inolf_status inolf_trace_stats(const inolf_object* obj, const float* cams, int32_t n_views, int32_t W,
                                          int32_t H, int64_t* out, void* workspace, size_t workspace_bytes,
                                          void* stream) {
  clear_error();
  if (!obj || !cams || !out || n_views <= 0 || W <= 0 || H <= 0)
    return fail(INOLF_E_INVALID, "inolf_trace_stats: bad argument");
  if (obj->o.variant) return fail(INOLF_E_INVALID, "inolf_trace_stats: the object has no proxy mesh");
  if (!workspace || workspace_bytes < inolf::workspace_bytes(1) || ((uintptr_t)workspace & 15))
    return fail(INOLF_E_INVALID, "inolf_trace_stats: workspace missing, too small or not 16-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  uint64_t* dev = reinterpret_cast<uint64_t*>(static_cast<uint32_t*>(workspace) + kTraceCountWord);
  if (cudaMemsetAsync(dev, 0, 3 * sizeof(uint64_t), st) != cudaSuccess)
    return fail(INOLF_E_CUDA, "cudaMemsetAsync failed");
  RayBatch rb{};
  rb.mode = 0;
  rb.cams = cams;
  rb.n_views = n_views;
  rb.W = W;
  rb.H = H;
  rb.n = (int64_t)n_views * W * H;
  inolf_status s = launch_render(obj->o, rb, INOLF_FP32, nullptr, nullptr, nullptr, nullptr, nullptr, workspace,
                                 workspace_bytes, stream, false, nullptr, true, true);
  if (s != INOLF_OK) return s;
  uint64_t h[3] = {0, 0, 0};
  if (cudaMemcpyAsync(h, dev, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(INOLF_E_CUDA, "inolf_trace_stats: reading the counters failed");
  uint32_t flags = 0;
  s = read_device_flags(workspace, stream, &flags);
  if (s != INOLF_OK) return s;
  s = flags_status(flags, "inolf_trace_stats");
  if (s != INOLF_OK) return s;
  out[0] = rb.n;
  out[1] = (int64_t)h[2];
  out[2] = (int64_t)h[0];
  out[3] = (int64_t)h[1];
  out[4] = (int64_t)n_views * ((W + 15) / 16) * ((H + 15) / 16) * 8;  // 8 x 4-ray packets
  return INOLF_OK;
}

extern "C" inolf_status inolf_render_rays(const inolf_object* obj, const float* o, const float* d, int64_t n,
                                          inolf_precision prec, float* rgba_out, int32_t* tri_out, float* t_out,
                                          void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  if (!obj || n < 0 || (n > 0 && (!o || !d || !rgba_out))) return fail(INOLF_E_INVALID, "inolf_render_rays: bad argument");
  if (n == 0) return INOLF_OK;
  RayBatch rb{};
  rb.mode = 1;
  rb.o = o;
  rb.d = d;
  rb.n = n;
  return launch_render(obj->o, rb, prec, rgba_out, tri_out, t_out, nullptr, nullptr, workspace, workspace_bytes,
                       stream);
}

extern "C" inolf_status inolf_calibrate_fp8(inolf_object* obj, const float* cams, int32_t n_views, int32_t W,
                                            int32_t H, void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  if (!obj || !cams || n_views <= 0 || W <= 0 || H <= 0 || !workspace || workspace_bytes < workspace_bytes_min())
    return fail(INOLF_E_INVALID, "inolf_calibrate_fp8: bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t* hdr = (uint32_t*)workspace;
  if (cudaMemsetAsync(hdr, 0, 32, st) != cudaSuccess) return fail(INOLF_E_CUDA, "cudaMemsetAsync failed");
  RayBatch rb{};
  rb.mode = 0;
  rb.cams = cams;
  rb.n_views = n_views;
  rb.W = W;
  rb.H = H;
  rb.n = (int64_t)n_views * W * H;
  inolf_status s = launch_render(obj->o, rb, INOLF_FP32, nullptr, nullptr, nullptr, nullptr, nullptr, workspace,
                                 workspace_bytes, stream, true);
  if (s != INOLF_OK) return s;
  uint32_t bits[3], flags = 0;
  if (cudaMemcpyAsync(bits, hdr + 4, sizeof(bits), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemcpyAsync(&flags, hdr + 1, sizeof(flags), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(INOLF_E_CUDA, "inolf_calibrate_fp8: readback failed");
  s = flags_status(flags, "inolf_calibrate_fp8");
  if (s != INOLF_OK) return s;
  for (int k = 0; k < 3; ++k) {
    float a;
    std::memcpy(&a, &bits[k], 4);
    obj->o.fp8_act_scale[k] = a > 0 ? a / 448.0f : 1.0f;
  }
  return INOLF_OK;
}

extern "C" inolf_status inolf_object_get_fp8_scales(const inolf_object* obj, float act[3], float weight[3]) {
  if (!obj || !act || !weight) return fail(INOLF_E_INVALID, "inolf_object_get_fp8_scales: NULL argument");
  // the weight scales live on the device (repacked there by inolf_object_load_params)
  if (cudaMemcpy(weight, obj->o.w_scale_dev, 3 * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(INOLF_E_CUDA, "inolf_object_get_fp8_scales: readback failed");
  for (int k = 0; k < 3; ++k) act[k] = obj->o.fp8_act_scale[k];
  return INOLF_OK;
}

extern "C" inolf_status inolf_encode_rays(const inolf_object* obj, const float* o, const float* d, int64_t n,
                                          uint32_t* slots_out, float* feat_out, void* workspace,
                                          size_t workspace_bytes, void* stream) {
  clear_error();
  if (!obj || n < 0 || (n > 0 && (!o || !d || !slots_out || !feat_out)))
    return fail(INOLF_E_INVALID, "inolf_encode_rays: bad argument");
  if (n == 0) return INOLF_OK;
  RayBatch rb{};
  rb.mode = 1;
  rb.o = o;
  rb.d = d;
  rb.n = n;
  return launch_render(obj->o, rb, INOLF_FP32, nullptr, nullptr, nullptr, slots_out, feat_out, workspace,
                       workspace_bytes, stream);
}

extern "C" inolf_status inolf_march_rays(const inolf_object* obj, const float* o, const float* d, int64_t n,
                                         int32_t* k_out, float* t_out, float* alpha_out, void* workspace,
                                         size_t workspace_bytes, void* stream) {
  clear_error();
  if (!obj || n < 0 || (n > 0 && (!o || !d))) return fail(INOLF_E_INVALID, "inolf_march_rays: bad argument");
  if (!obj->o.variant) return fail(INOLF_E_INVALID, "inolf_march_rays: the object has no density cubes");
  if (n == 0) return INOLF_OK;
  RayBatch rb{};
  rb.mode = 1;
  rb.o = o;
  rb.d = d;
  rb.n = n;
  return launch_render(obj->o, rb, INOLF_FP32, nullptr, k_out, t_out, nullptr, nullptr, workspace, workspace_bytes,
                       stream, false, alpha_out, true);
}

// Device address of a host buffer the device can store to directly (pinned
// and mapped into the device's address space, 16-byte aligned), or NULL.
static float* mapped_host_target(float* host) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer || ((uintptr_t)a.devicePointer & 15)) return nullptr;
  return static_cast<float*>(a.devicePointer);
}

extern "C" inolf_status inolf_render_host(const inolf_object* obj, const float* cams, int32_t n_views, int32_t W,
                                          int32_t H, inolf_precision prec, float* rgba_host, void* staging,
                                          size_t staging_bytes, void* workspace, size_t workspace_bytes,
                                          void* stream) {
  clear_error();
  if (!obj || !cams || !rgba_host || n_views < 0 || W <= 0 || H <= 0 || !staging || ((uintptr_t)staging & 15))
    return fail(INOLF_E_INVALID, "inolf_render_host: bad argument");
  if (n_views == 0) return INOLF_OK;

  const size_t view_bytes = (size_t)W * H * 4 * sizeof(float);
  const int64_t slot_views = (int64_t)(staging_bytes / 2 / view_bytes);
  if (slot_views < 1) return fail(INOLF_E_INVALID, "inolf_render_host: staging holds less than two views");
  if (float* direct = mapped_host_target(rgba_host)) {
    // pinned, mapped host memory: the kernels store the frames straight into it
    // (over the GPU-host link), with no staging copy
    RayBatch rb{};
    rb.mode = 0;
    rb.cams = cams;
    rb.n_views = n_views;
    rb.W = W;
    rb.H = H;
    rb.n = (int64_t)n_views * W * H;
    inolf_status st = launch_render(obj->o, rb, prec, direct, nullptr, nullptr, nullptr, nullptr, workspace,
                                    workspace_bytes, stream);
    if (st != INOLF_OK) return st;
    uint32_t flags = 0;
    st = read_device_flags(workspace, stream, &flags);  // synchronises `stream`
    if (st != INOLF_OK) return st;
    return flags_status(flags, "inolf_render_host");
  }
  cudaStream_t cs = (cudaStream_t)stream;
  cudaStream_t xs = nullptr;
  cudaEvent_t rendered[2] = {nullptr, nullptr}, copied[2] = {nullptr, nullptr};
  inolf_status st = INOLF_OK;
  if (cudaStreamCreateWithFlags(&xs, cudaStreamNonBlocking) != cudaSuccess)
    return fail(INOLF_E_CUDA, "inolf_render_host: cudaStreamCreate failed");
  for (int k = 0; k < 2 && st == INOLF_OK; ++k)
    if (cudaEventCreateWithFlags(&rendered[k], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&copied[k], cudaEventDisableTiming) != cudaSuccess)
      st = fail(INOLF_E_CUDA, "inolf_render_host: cudaEventCreate failed");
  // chunk c renders into staging slot c & 1 on the caller's stream while the
  // copy stream moves chunk c - 1 to host memory; a slot is rendered into
  // again only after its previous copy finished
  for (int64_t v0 = 0, c = 0; st == INOLF_OK && v0 < n_views; v0 += slot_views, ++c) {
    const int32_t nv = (int32_t)std::min<int64_t>(slot_views, n_views - v0);
    const int slot = (int)(c & 1);
    float* dst = reinterpret_cast<float*>((char*)staging + (size_t)slot * slot_views * view_bytes);
    if (c >= 2 && cudaStreamWaitEvent(cs, copied[slot], 0) != cudaSuccess) {
      st = fail(INOLF_E_CUDA, "inolf_render_host: cudaStreamWaitEvent failed");
      break;
    }
    RayBatch rb{};
    rb.mode = 0;
    rb.cams = cams + 13 * v0;
    rb.n_views = nv;
    rb.W = W;
    rb.H = H;
    rb.n = (int64_t)nv * W * H;
    st = launch_render(obj->o, rb, prec, dst, nullptr, nullptr, nullptr, nullptr, workspace, workspace_bytes, stream,
                       false, nullptr, false, false, /*clear_flags=*/c == 0);
    if (st != INOLF_OK) break;
    if (cudaEventRecord(rendered[slot], cs) != cudaSuccess || cudaStreamWaitEvent(xs, rendered[slot], 0) != cudaSuccess ||
        cudaMemcpyAsync(rgba_host + (size_t)v0 * W * H * 4, dst, (size_t)nv * view_bytes, cudaMemcpyDeviceToHost, xs) !=
            cudaSuccess ||
        cudaEventRecord(copied[slot], xs) != cudaSuccess)
      st = fail(INOLF_E_CUDA, "inolf_render_host: copy scheduling failed");
  }
  const bool synced = cudaStreamSynchronize(xs) == cudaSuccess && cudaStreamSynchronize(cs) == cudaSuccess;
  if (st == INOLF_OK && !synced) st = fail(INOLF_E_CUDA, "inolf_render_host: synchronisation failed");
  if (st == INOLF_OK) {  // device-side failures of any chunk
    uint32_t flags = 0;
    st = read_device_flags(workspace, stream, &flags);
    if (st == INOLF_OK) st = flags_status(flags, "inolf_render_host");
  }
  for (int k = 0; k < 2; ++k) {
    if (rendered[k]) cudaEventDestroy(rendered[k]);
    if (copied[k]) cudaEventDestroy(copied[k]);
  }
  cudaStreamDestroy(xs);
  return st;
}
