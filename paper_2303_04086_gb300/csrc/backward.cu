// Backward pass of the i-NOLF per-ray path for training (Sec. 4.2,
// "Training", Eq. 8): given dLoss/dRGBA per ray, accumulate the gradients of
// the MLP weights W1, W2, W3 and of the perfect-hash feature tables.
//
// Forward activations are recomputed, not stored.  One CTA (256 threads) per
// SM works on tiles of 64 hit rays:
//   1. gather (4 threads per ray, every 4th level each) -> X [k][ray] in
//      shared memory, as in the forward kernels;
//   2. Z1 = W1 X, A1 = relu(Z1); Z2 = W2 A1, A2 = relu(Z2); y = sigmoid(W3 A2)
//      (FP32 on the CUDA cores, 4 x 4 register blocks per thread);
//   3. dZ3 = g * y (1 - y); dW3 += dZ3 A2^T; dZ2 = (W3^T dZ3) * [A2 > 0];
//      dZ1 = (W2^T dZ2) * [A1 > 0]; dX = W1^T dZ1 (feature rows only);
//   4. the weight gradients dW2 += dZ2 A1^T and dW1 += dZ1 X^T, contractions
//      over the rays of the tile, on the tensor cores (tcgen05, TF32 operands
//      in a hi/lo split, FP32 accumulation in tensor memory that persists over
//      all tiles of the CTA);
//   5. scatter: for every level and corner, table_grad[slot] += w_corner dX
//      (float2 atomics; slots and trilinear weights recomputed).
// Each CTA adds its accumulated weight gradients to global memory once, at
// the end.
//
// Step 4 as one MMA problem with M = 128 (one TMEM lane per row):
//   A = [dZ2; dZ1]   128 rows (layer-2 neurons, then layer-1 neurons) x K
//   B = [A1; X; 0]   64 + kNx rows (layer-1 activations, the MLP inputs, zero
//                    rows up to a multiple of 16) x K,   K = rays of the tile
//   D[128][64 + kNx] += A B^T,  so  D[j][i] = dW2[j][i] and
//   D[64 + j][64 + k] = dW1[j][k]; the two off-diagonal blocks are discarded.
// FP32 accuracy from TF32 tensor cores: each operand is split x = hi + lo with
// hi = tf32(x) and lo = tf32(x - hi) (round to nearest), and each K step of 8
// rays issues hi_a hi_b + hi_a lo_b + lo_a hi_b (the lo_a lo_b term, about
// 2^-22 of the product, is dropped) -- the split-TF32 method.  The operands
// are staged from the [row][ray] activation tiles into K-major core-matrix
// tiles (8 rows x 16 bytes); the MMAs of a tile run while the CTA computes
// dX, scatters and starts the next tile, and are waited for (bounded) only
// before the staging buffers are written again.
#include <cuda_runtime.h>

#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "inolf_internal.h"
#include "kernels_common.cuh"
#include "tc_ptx.cuh"

namespace inolf {

static constexpr int kBT = 64;         // rays per tile (= K of one weight-gradient contraction)
static constexpr int kBThreads = 256;
static constexpr int kBS = 68;         // row stride of [k][ray] tiles (bank-conflict padding)
static constexpr int kMaxDin = 2 * INOLF_MAX_LEVELS + INOLF_N_SH;  // 48
// tensor-core operands: K-major core matrices, kBT * 4 bytes per row
static constexpr uint32_t kOpChunks = kBT * 4 / 16;                // 16-byte chunks per row (16)
static constexpr uint32_t kOpRowBytes = kOpChunks * 16;            // 256
static constexpr uint32_t kOpABytes = 128u * kOpRowBytes;          // A: 128 rows (hi or lo half)
static constexpr uint32_t kOpBRowsMax = 64u + kMaxDin;             // B: 64 + 48 rows at most
static constexpr uint32_t kOpBBytes = kOpBRowsMax * kOpRowBytes;
static constexpr uint32_t kOpBytes = 2u * kOpABytes + 2u * kOpBBytes;  // hi/lo of A and B: 120 KB
static constexpr uint32_t kBTmemCols = 128;                        // >= 64 + 48 FP32 columns
static constexpr uint64_t kBWaitLimitNs = 2000000000ull;           // 2 s; the MMAs of a tile take microseconds

static_assert(kBT % 8 == 0, "a tile is a whole number of TF32 K steps (8 rays)");
static_assert(kOpBRowsMax % 16 == 0, "N of the weight-gradient MMA must be a multiple of 16 for M = 128");

__host__ __device__ constexpr size_t bwd_floats() {
  return (size_t)kMaxDin * 64 + 64 * 64 * 2 + 4 * 64 + (size_t)(kMaxDin + 64 + 64 + 4) * kBS;
}
__host__ __device__ constexpr size_t bwd_smem_bytes_c() { return kOpBytes + bwd_floats() * sizeof(float) + 16; }
static_assert(bwd_smem_bytes_c() <= 227 * 1024, "backward tiles must fit one CTA's shared memory");

// out[r][c] (+)= sum_k act[k][r] * w[k][c] for rays r0..r0+3, columns c0..c0+3
__device__ __forceinline__ void gemm_4x4(const float* act, const float* w, int K, int wstride, int r0, int c0,
                                         float acc[4][4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    const float4 a = *reinterpret_cast<const float4*>(act + k * kBS + r0);
    const float4 b = *reinterpret_cast<const float4*>(w + k * wstride + c0);
    const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
  }
}

// Copies rows [0, n_rows) of a [row][kBS] FP32 tile into rows dst_row0 ..
// of a K-major core-matrix operand (hi and lo halves, TF32 split).  Eight
// consecutive threads take the 8 rows of one core matrix and one 16-byte
// chunk (4 rays), so both the reads (row stride 272 bytes) and the writes
// (128 contiguous bytes) are free of bank conflicts.
__device__ __forceinline__ void stage_rows(const float* src, int n_rows, uint8_t* hi, uint8_t* lo, uint32_t dst_row0) {
  const int n = (n_rows + 7) / 8 * 8 * (int)kOpChunks;  // whole 8-row groups; rows >= n_rows are skipped
  for (int idx = threadIdx.x; idx < n; idx += kBThreads) {
    const int rr = idx & 7, c = (idx >> 3) & (int)(kOpChunks - 1), g = idx >> 7;
    const int row = 8 * g + rr;
    if (row >= n_rows) continue;
    const float4 v = *reinterpret_cast<const float4*>(src + row * kBS + 4 * c);
    const float4 h = make_float4(tc::round_tf32(v.x), tc::round_tf32(v.y), tc::round_tf32(v.z), tc::round_tf32(v.w));
    const float4 l = make_float4(tc::round_tf32(v.x - h.x), tc::round_tf32(v.y - h.y), tc::round_tf32(v.z - h.z),
                                 tc::round_tf32(v.w - h.w));
    const uint32_t off = tc::core_off(dst_row0 + (uint32_t)row, (uint32_t)c, kOpChunks);
    *reinterpret_cast<float4*>(hi + off) = h;
    *reinterpret_cast<float4*>(lo + off) = l;
  }
}

__global__ void __launch_bounds__(kBThreads, 1) k_backward(const __grid_constant__ Params p,
                                                          const __grid_constant__ BwdParams b) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* sAhi = smem;
  uint8_t* sAlo = sAhi + kOpABytes;
  uint8_t* sBhi = sAlo + kOpABytes;
  uint8_t* sBlo = sBhi + kOpBBytes;
  float* sm = reinterpret_cast<float*>(smem + kOpBytes);
  const int din = p.d_in, nf = 2 * p.L;
  const uint32_t nx = ((uint32_t)din + 15u) & ~15u;  // X rows of B, zero padded
  const uint32_t nB = 64u + nx;                       // N of the weight-gradient MMA
  float* W1T = sm;                  // [din][64]
  float* W2T = W1T + kMaxDin * 64;  // [64 in][64 out]
  float* W2 = W2T + 64 * 64;        // [64 out][64 in]
  float* W3 = W2 + 64 * 64;         // [4][64]
  float* X = W3 + 4 * 64;           // [din][kBS]   inputs, later dX
  float* A1 = X + kMaxDin * kBS;    // [64][kBS]    relu(Z1), later dZ1
  float* A2 = A1 + 64 * kBS;        // [64][kBS]    relu(Z2), later dZ2
  float* DZ3 = A2 + 64 * kBS;       // [4][kBS]
  uint64_t* bar = reinterpret_cast<uint64_t*>(DZ3 + 4 * kBS);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  {
    const float* g = p.w_f32;  // W1T [din][64], W2 [64][64], W3T [64][4]
    for (int k = tid; k < din * 64; k += kBThreads) W1T[k] = g[k];
    const float* g2 = g + din * 64;
    for (int k = tid; k < 64 * 64; k += kBThreads) {
      const float v = g2[k];
      W2[k] = v;
      W2T[(k & 63) * 64 + (k >> 6)] = v;
    }
    const float* g3 = g2 + 64 * 64;
    for (int k = tid; k < 64 * 4; k += kBThreads) W3[(k & 3) * 64 + (k >> 2)] = g3[k];
    // zero the operand tiles: the padding rows of B stay zero
    for (uint32_t k = tid; k < kOpBytes / 16u; k += kBThreads) reinterpret_cast<uint4*>(smem)[k] = make_uint4(0, 0, 0, 0);
  }
  if (tid == 0) {
    tc::mbar_init(bar, 1);
    tc::fence_mbar_init();
  }
  __syncthreads();
  if (warp == 0) tc::tmem_alloc(tslot, kBTmemCols);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t id = tc::idesc(128, nB, 2u);  // kind::tf32, D FP32, M = 128
  float gw3 = 0.0f;                            // dW3 partial: row tid / 64, column tid & 63
  uint32_t phase = 0;
  bool pending = false, issued = false, bad = false;

  const uint32_t total = *p.counter;
  const int ray_slot = tid & (kBT - 1), part = tid >> 6;
  const int r0 = (tid & 15) * 4, c0 = (tid >> 4) * 4;  // 4 x 4 GEMM block
  for (uint32_t base = blockIdx.x * kBT; base < total; base += gridDim.x * kBT) {
    const uint32_t h = base + (uint32_t)ray_slot;
    const bool valid = h < total;
    int64_t ray = 0;
    float x[3] = {0.f, 0.f, 0.f};
    // ---- 1. gather ----
    if (valid) {
      const uint2 rec = p.hits[h];
      ray = rec.x;
      float o[3], d[3];
      ray_of(p, ray, o, d);
      hit_unit_coords(p, o, d, __uint_as_float(rec.y), x);
      LevelFetch cur, nxt;
      if (part < p.L) fetch_phi(p.lv[part], x, cur);
      for (int l = part; l < p.L; l += 4) {
        if (l + 4 < p.L) fetch_phi(p.lv[l + 4], x, nxt);
        uint32_t slots[8];
        float e0, e1;
        finish_level(p.lv[l], p.fp16, cur, slots, e0, e1);
        X[(2 * l) * kBS + ray_slot] = e0;
        X[(2 * l + 1) * kBS + ray_slot] = e1;
        cur = nxt;
      }
      if (part == 3) {
        float sh[16];
        sh16(p, d, sh);
#pragma unroll
        for (int k = 0; k < 16; ++k) X[(nf + k) * kBS + ray_slot] = sh[k];
      }
    } else {
      for (int k = part; k < din; k += 4) X[k * kBS + ray_slot] = 0.0f;
    }
    __syncthreads();
    // ---- 2. forward MLP ----
    float acc[4][4];
    gemm_4x4(X, W1T, din, 64, r0, c0, acc);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      *reinterpret_cast<float4*>(A1 + (c0 + j) * kBS + r0) =
          make_float4(fmaxf(acc[0][j], 0.f), fmaxf(acc[1][j], 0.f), fmaxf(acc[2][j], 0.f), fmaxf(acc[3][j], 0.f));
    __syncthreads();
    gemm_4x4(A1, W2T, 64, 64, r0, c0, acc);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      *reinterpret_cast<float4*>(A2 + (c0 + j) * kBS + r0) =
          make_float4(fmaxf(acc[0][j], 0.f), fmaxf(acc[1][j], 0.f), fmaxf(acc[2][j], 0.f), fmaxf(acc[3][j], 0.f));
    __syncthreads();
    // ---- 3. output layer and dZ3 (thread = (ray, channel part)) ----
    {
      const int c = part;  // 4 output channels
      float z = 0.f;
#pragma unroll 8
      for (int j = 0; j < 64; ++j) z = fmaf(W3[c * 64 + j], A2[j * kBS + ray_slot], z);
      const float y = sigmoidf_(z);
      const float g = valid ? b.d_rgba[(p.ray_base + ray) * 4 + c] : 0.0f;
      DZ3[c * kBS + ray_slot] = g * y * (1.0f - y);
    }
    __syncthreads();
    // dW3[c][j] += sum_r dZ3[c][r] A2[j][r]
    {
      const int c = tid >> 6, j = tid & 63;
      float s = 0.f;
      for (int r = 0; r < kBT; r += 4) {
        const float4 dz = *reinterpret_cast<const float4*>(DZ3 + c * kBS + r);
        const float4 a = *reinterpret_cast<const float4*>(A2 + j * kBS + r);
        s = fmaf(dz.x, a.x, fmaf(dz.y, a.y, fmaf(dz.z, a.z, fmaf(dz.w, a.w, s))));
      }
      gw3 += s;
    }
    __syncthreads();
    // dZ2[j][r] = (sum_c W3[c][j] dZ3[c][r]) * [A2[j][r] > 0], in place of A2
    for (int e = tid; e < 64 * kBT; e += kBThreads) {
      const int j = e / kBT, r = e % kBT;
      const float da = W3[j] * DZ3[r] + W3[64 + j] * DZ3[kBS + r] + W3[128 + j] * DZ3[2 * kBS + r] +
                       W3[192 + j] * DZ3[3 * kBS + r];
      float* a2 = A2 + j * kBS + r;
      *a2 = *a2 > 0.f ? da : 0.f;
    }
    // the previous tile's weight-gradient MMAs must have read the operand
    // tiles before they are written again
    if (pending) {
      const bool ok = tc::mbar_wait(bar, phase, kBWaitLimitNs);
      if (__syncthreads_or(!ok)) {  // still pending: drained (bounded) before TMEM is freed
        bad = true;
        break;
      }
      phase ^= 1u;
      pending = false;
      tc::fence_after();
    } else {
      __syncthreads();
    }
    // operands of the weight gradients: dZ2 -> A rows 0..63, A1 -> B rows 0..63
    stage_rows(A2, 64, sAhi, sAlo, 0u);
    stage_rows(A1, 64, sBhi, sBlo, 0u);
    // dA1[r][i] = sum_j dZ2[j][r] W2[j][i]
    gemm_4x4(A2, W2, 64, 64, r0, c0, acc);
    float mask[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float4 a = *reinterpret_cast<const float4*>(A1 + (c0 + j) * kBS + r0);
      mask[0][j] = a.x; mask[1][j] = a.y; mask[2][j] = a.z; mask[3][j] = a.w;
    }
    __syncthreads();  // all reads of A1 (staging and masks) are done
#pragma unroll
    for (int j = 0; j < 4; ++j)
      *reinterpret_cast<float4*>(A1 + (c0 + j) * kBS + r0) =
          make_float4(mask[0][j] > 0.f ? acc[0][j] : 0.f, mask[1][j] > 0.f ? acc[1][j] : 0.f,
                      mask[2][j] > 0.f ? acc[2][j] : 0.f, mask[3][j] > 0.f ? acc[3][j] : 0.f);
    __syncthreads();
    // ---- 4. dZ1 -> A rows 64..127, X -> B rows 64 .. 64 + din; then the MMAs ----
    stage_rows(A1, 64, sAhi, sAlo, 64u);
    stage_rows(X, din, sBhi, sBlo, 64u);
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      const uint32_t sbo = kOpChunks * 128u;
      for (uint32_t s = 0; s < (uint32_t)kBT / 8u; ++s) {  // K steps of 8 rays (32 bytes)
        const uint64_t ah = tc::desc_kmajor(tc::smem_u32(sAhi) + s * 256u, 128u, sbo);
        const uint64_t al = tc::desc_kmajor(tc::smem_u32(sAlo) + s * 256u, 128u, sbo);
        const uint64_t bh = tc::desc_kmajor(tc::smem_u32(sBhi) + s * 256u, 128u, sbo);
        const uint64_t bl = tc::desc_kmajor(tc::smem_u32(sBlo) + s * 256u, 128u, sbo);
        tc::mma_tf32(tmem, ah, bh, id, (issued || s > 0) ? 1u : 0u);
        tc::mma_tf32(tmem, ah, bl, id, 1u);
        tc::mma_tf32(tmem, al, bh, id, 1u);
      }
      tc::mma_commit(bar);
    }
    pending = true;
    issued = true;
    // dX[k][ray] = sum_j dZ1[j][ray] W1[j][k], k < 2L (features only), in place of X
    // (X was staged above, before the barrier)
    {
      float dx[8];  // up to 8 feature rows per thread part (2 L <= 32)
      const int nk = (nf + 3) / 4;
#pragma unroll
      for (int q = 0; q < 8; ++q) dx[q] = 0.f;
      for (int j = 0; j < 64; ++j) {
        const float dz = A1[j * kBS + ray_slot];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int k = part * nk + q;
          if (q < nk && k < nf) dx[q] = fmaf(dz, W1T[k * 64 + j], dx[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int k = part * nk + q;
        if (q < nk && k < nf) X[k * kBS + ray_slot] = dx[q];
      }
    }
    __syncthreads();
    // ---- 5. scatter into the feature tables ----
    if (valid) {
      for (int l = part; l < p.L; l += 4) {
        LevelFetch s;
        fetch_phi(p.lv[l], x, s);
        uint32_t slots[8];
        const int32_t m = p.lv[l].m;
#pragma unroll
        for (int cc = 0; cc < 8; ++cc) {
          int32_t sx = ((cc & 1) ? s.h0n[0] : s.h0[0]) + (int32_t)(s.ph[cc] & 1023u);
          int32_t sy = ((cc & 2) ? s.h0n[1] : s.h0[1]) + (int32_t)((s.ph[cc] >> 10) & 1023u);
          int32_t sz = ((cc & 4) ? s.h0n[2] : s.h0[2]) + (int32_t)((s.ph[cc] >> 20) & 1023u);
          sx -= sx >= m ? m : 0;
          sy -= sy >= m ? m : 0;
          sz -= sz >= m ? m : 0;
          slots[cc] = (uint32_t)(sx + m * (sy + m * sz));
        }
        const float g0 = X[(2 * l) * kBS + ray_slot], g1 = X[(2 * l + 1) * kBS + ray_slot];
        const float gx = 1.0f - s.f[0], gy = 1.0f - s.f[1], gz = 1.0f - s.f[2];
        float2* tab = reinterpret_cast<float2*>(b.gtab[l]);
#pragma unroll
        for (int cc = 0; cc < 8; ++cc) {
          const float w = ((cc & 1) ? s.f[0] : gx) * ((cc & 2) ? s.f[1] : gy) * ((cc & 4) ? s.f[2] : gz);
          atomicAdd(tab + slots[cc], make_float2(w * g0, w * g1));
        }
      }
    }
    __syncthreads();  // before the next tile reuses the buffers
  }
  if (pending && !bad) {
    const bool ok = tc::mbar_wait(bar, phase, kBWaitLimitNs);
    bad = __syncthreads_or(!ok);
    if (!bad) {
      phase ^= 1u;
      pending = false;
    }
  }
  if (bad) {
    if (tid == 0) atomicOr(p.counter + 1, INOLF_FLAG_WAIT_TIMEOUT);
    if (pending) tc::mbar_wait(bar, phase, kBWaitLimitNs);  // let MMAs still in flight finish
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  // ---- per-CTA weight gradients -> global ----
  if (gw3 != 0.f) atomicAdd(b.gw3 + (tid >> 6) * 64 + (tid & 63), gw3);
  if (issued && !bad) {
    // warp w reads TMEM lanes 32 (w % 4) .. + 31, i.e. rows of D; warps w and
    // w + 4 split the columns.  Rows 0..63: dW2 (columns 0..63); rows
    // 64..127: dW1 (columns 64 .. 64 + din).
    const uint32_t q = (uint32_t)warp & 3u, half = (uint32_t)warp >> 2;
    const uint32_t row = 32u * q + (uint32_t)lane;
    const uint32_t taddr = tmem + ((32u * q) << 16);
    if (q < 2) {
      for (uint32_t c = 32u * half; c < 32u * half + 32u; c += 16u) {
        float v[16];
        tc::tmem_ld16(taddr + c, v);
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (v[i] != 0.f) atomicAdd(b.gw2 + row * 64 + c + i, v[i]);
      }
    } else {
      const uint32_t j = row - 64u;
      for (uint32_t c = 16u * half; c < nx; c += 32u) {
        float v[16];
        tc::tmem_ld16(taddr + 64u + c, v);
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if ((int)(c + i) < din && v[i] != 0.f) atomicAdd(b.gw1 + j * din + c + i, v[i]);
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, kBTmemCols);
  }
}

static size_t bwd_smem_bytes() { return bwd_smem_bytes_c(); }

inolf_status launch_backward(const Params& p, const BwdParams& b, cudaStream_t st) {
  const int dev = device_index();
  if (dev < 0) return fail(INOLF_E_UNSUPPORTED, "k_backward: no current device, or an index beyond 63");
  static int grid_dev[kMaxDevices];
  static std::once_flag once[kMaxDevices];
  std::call_once(once[dev], [dev] {
    int sms = 1, occ = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_smem_bytes());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_backward, kBThreads, bwd_smem_bytes());
    // each resident CTA holds kBTmemCols of the SM's 512 tensor-memory columns
    grid_dev[dev] = sms * std::min(std::max(1, occ), 512 / (int)kBTmemCols);
    cudaGetLastError();
  });
  const int grid = grid_dev[dev];
  {
    LaunchTimer lt("k_backward", st);
    k_backward<<<grid, kBThreads, bwd_smem_bytes(), st>>>(p, b);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(INOLF_E_CUDA, std::string("k_backward: ") + cudaGetErrorString(e));
  return INOLF_OK;
}

}  // namespace inolf

// ---------------------------------------------------------------------------
// parameter updates from device buffers (training)
// ---------------------------------------------------------------------------
using namespace inolf;

__global__ void k_tables_to_fp16(const float2* __restrict__ src, __half2* __restrict__ dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = __floats2half2_rn(src[i].x, src[i].y);
}

// Eq. 1 for a vertex p of the level (each coordinate in [0, N]): the slot
// ((p mod m) + Phi[p mod r]) mod m per axis, linearised x + m (y + m z).
__device__ __forceinline__ uint32_t psh_slot_of(const inolf::LevelDev& lv, uint32_t px, uint32_t py, uint32_t pz) {
  const uint32_t m = (uint32_t)lv.m, r = (uint32_t)lv.r;
  const uint32_t e = lv.phi[(px % r) + r * ((py % r) + r * (pz % r))];
  uint32_t sx = px % m + (e & 1023u), sy = py % m + ((e >> 10) & 1023u), sz = pz % m + (e >> 20);
  sx = sx >= m ? sx - m : sx;
  sy = sy >= m ? sy - m : sy;
  sz = sz >= m ? sz - m : sz;
  return sx + m * (sy + m * sz);
}

// Corner bundles of one level: for every hashed vertex c (packed x | y << 21
// | z << 42) whose coordinates are all below N, bundle row h(c) receives the
// rows T[h(c + d)] of the 8 corners d of the cell above c (x fastest).
template <class Row>
__global__ void k_build_bundles(const uint64_t* __restrict__ pts, int64_t n, const inolf::LevelDev lv,
                                Row* __restrict__ bundle) {
  const Row* table = reinterpret_cast<const Row*>(lv.table);
  const uint32_t N = (uint32_t)lv.N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t pk = pts[i];
    const uint32_t cx = (uint32_t)(pk & 0x1FFFFFu), cy = (uint32_t)((pk >> 21) & 0x1FFFFFu),
                   cz = (uint32_t)((pk >> 42) & 0x1FFFFFu);
    if (cx >= N || cy >= N || cz >= N) continue;  // no cell has c as its lowest corner
    Row* out = bundle + 8 * (size_t)psh_slot_of(lv, cx, cy, cz);
#pragma unroll
    for (int cc = 0; cc < 8; ++cc)
      out[cc] = table[psh_slot_of(lv, cx + (cc & 1), cy + ((cc >> 1) & 1), cz + (cc >> 2))];
  }
}

namespace inolf {
inolf_status build_level_bundles(Object& o, int l, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const LevelDev& lv = o.lv[l];
  const size_t rows = (size_t)lv.m * lv.m * lv.m * 8;
  if (cudaMemsetAsync(const_cast<void*>(lv.bundle), 0, rows * (o.fp16 ? 4 : 8), st) != cudaSuccess)
    return fail(INOLF_E_CUDA, "corner bundles: cudaMemsetAsync failed");
  if (o.n_pts[l] > 0) {
    if (o.fp16)
      k_build_bundles<__half2><<<1024, 256, 0, st>>>(o.pts[l], o.n_pts[l], lv, (__half2*)lv.bundle);
    else
      k_build_bundles<float2><<<1024, 256, 0, st>>>(o.pts[l], o.n_pts[l], lv, (float2*)lv.bundle);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(INOLF_E_CUDA, std::string("k_build_bundles: ") + cudaGetErrorString(e));
  return INOLF_OK;
}
}  // namespace inolf

extern "C" inolf_status inolf_object_load_params(inolf_object* obj, const float* const* tables_dev,
                                                 const float* w1_dev, const float* w2_dev, const float* w3_dev,
                                                 void* stream) {
  inolf::clear_error();
  if (!obj) return inolf::fail(INOLF_E_INVALID, "inolf_object_load_params: NULL object");
  if ((w1_dev || w2_dev || w3_dev) && !(w1_dev && w2_dev && w3_dev))
    return fail(INOLF_E_INVALID, "inolf_object_load_params: give all three weight matrices or none");
  inolf::Object& o = obj->o;
  cudaStream_t st = (cudaStream_t)stream;
  if (tables_dev) {
    for (int l = 0; l < o.L; ++l) {
      if (!tables_dev[l]) continue;
      if (o.fp16) {
        k_tables_to_fp16<<<256, 256, 0, st>>>((const float2*)tables_dev[l], (__half2*)o.lv[l].table, o.rows[l]);
        if (cudaGetLastError() != cudaSuccess) return fail(INOLF_E_CUDA, "load_params: conversion launch failed");
      } else if (cudaMemcpyAsync((void*)o.lv[l].table, tables_dev[l], 8 * o.rows[l], cudaMemcpyDeviceToDevice, st) !=
                 cudaSuccess) {
        return fail(INOLF_E_CUDA, "load_params: table copy failed");
      }
      inolf_status es = inolf::build_level_bundles(o, l, stream);
      if (es != INOLF_OK) return es;
    }
  }
  if (w1_dev) return inolf::pack_weights_device(o, w1_dev, w2_dev, w3_dev, stream);  // no host round trip
  return INOLF_OK;
}
