// Backward pass of the i-NOLF per-ray path for training (Sec. 4.2,
// "Training", Eq. 8): given dLoss/dRGBA per ray, accumulate the gradients of
// the MLP weights W1, W2, W3 and of the perfect-hash feature tables.
//
// Forward activations are recomputed, not stored.  One CTA (256 threads)
// works on tiles of 64 hit rays:
//   1. gather (4 threads per ray, every 4th level each) -> X [k][ray] in
//      shared memory, as in the forward kernels;
//   2. Z1 = W1 X, A1 = relu(Z1); Z2 = W2 A1, A2 = relu(Z2); y = sigmoid(W3 A2)
//      (FP32, 4 x 4 register blocks per thread);
//   3. dZ3 = g * y (1 - y); dW3 += dZ3 A2^T; dZ2 = (W3^T dZ3) * [A2 > 0];
//      dW2 += dZ2 A1^T; dZ1 = (W2^T dZ2) * [A1 > 0]; dW1 += dZ1 X^T;
//      dX = W1^T dZ1 (feature rows only);
//   4. scatter: for every level and corner, table_grad[slot] += w_corner dX
//      (float2 atomics; slots and trilinear weights recomputed).
// The weight gradients of all tiles a CTA processes stay in registers and
// are added to global memory once per CTA.
#include <cuda_runtime.h>

#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "inolf_internal.h"
#include "kernels_common.cuh"

namespace inolf {

static constexpr int kBT = 64;         // rays per tile
static constexpr int kBThreads = 256;
static constexpr int kBS = 68;         // row stride of [k][ray] tiles (bank-conflict padding)
static constexpr int kMaxDin = 2 * INOLF_MAX_LEVELS + INOLF_N_SH;  // 48

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

__global__ void __launch_bounds__(kBThreads, 2) k_backward(const __grid_constant__ Params p,
                                                          const __grid_constant__ BwdParams b) {
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  const int din = p.d_in, nf = 2 * p.L;
  float* W1T = sm;                  // [din][64]
  float* W1 = W1T + kMaxDin * 64;   // [64][din]
  float* W2T = W1 + kMaxDin * 64;   // [64 in][64 out]
  float* W2 = W2T + 64 * 64;        // [64 out][64 in]
  float* W3 = W2 + 64 * 64;         // [4][64]
  float* X = W3 + 4 * 64;           // [din][kBS]   inputs, later dX
  float* A1 = X + kMaxDin * kBS;    // [64][kBS]    relu(Z1), later dZ1
  float* A2 = A1 + 64 * kBS;        // [64][kBS]    relu(Z2), later dZ2
  float* DZ3 = A2 + 64 * kBS;       // [4][kBS]
  const int tid = threadIdx.x;
  {
    const float* g = p.w_f32;  // W1T [din][64], W2 [64][64], W3T [64][4]
    for (int k = tid; k < din * 64; k += kBThreads) {
      const float v = g[k];
      W1T[k] = v;
      W1[(k & 63) * din + (k >> 6)] = v;
    }
    const float* g2 = g + din * 64;
    for (int k = tid; k < 64 * 64; k += kBThreads) {
      const float v = g2[k];
      W2[k] = v;
      W2T[(k & 63) * 64 + (k >> 6)] = v;
    }
    const float* g3 = g2 + 64 * 64;
    for (int k = tid; k < 64 * 4; k += kBThreads) W3[(k & 3) * 64 + (k >> 2)] = g3[k];
  }
  // per-thread weight-gradient partials
  float gw1[kMaxDin / 4] = {};   // row j1 = tid / 4, columns (tid & 3) + 4 q
  float gw2[16] = {};            // row j1, columns (tid & 3) + 4 q
  float gw3 = 0.0f;              // row tid / 64, column tid & 63
  const int j1 = tid >> 2, cq = tid & 3;
  __syncthreads();

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
    __syncthreads();
    // dW2[j1][i] += sum_r dZ2[j1][r] A1[i][r]
#pragma unroll 1
    for (int r = 0; r < kBT; r += 4) {
      const float4 dz = *reinterpret_cast<const float4*>(A2 + j1 * kBS + r);
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const float4 a = *reinterpret_cast<const float4*>(A1 + (cq + 4 * q) * kBS + r);
        gw2[q] = fmaf(dz.x, a.x, fmaf(dz.y, a.y, fmaf(dz.z, a.z, fmaf(dz.w, a.w, gw2[q]))));
      }
    }
    // dA1[r][i] = sum_j dZ2[j][r] W2[j][i]
    gemm_4x4(A2, W2, 64, 64, r0, c0, acc);
    float mask[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float4 a = *reinterpret_cast<const float4*>(A1 + (c0 + j) * kBS + r0);
      mask[0][j] = a.x; mask[1][j] = a.y; mask[2][j] = a.z; mask[3][j] = a.w;
    }
    __syncthreads();  // all reads of A1 (dW2 and masks) are done
#pragma unroll
    for (int j = 0; j < 4; ++j)
      *reinterpret_cast<float4*>(A1 + (c0 + j) * kBS + r0) =
          make_float4(mask[0][j] > 0.f ? acc[0][j] : 0.f, mask[1][j] > 0.f ? acc[1][j] : 0.f,
                      mask[2][j] > 0.f ? acc[2][j] : 0.f, mask[3][j] > 0.f ? acc[3][j] : 0.f);
    __syncthreads();
    // dW1[j1][k] += sum_r dZ1[j1][r] X[k][r]
#pragma unroll 1
    for (int r = 0; r < kBT; r += 4) {
      const float4 dz = *reinterpret_cast<const float4*>(A1 + j1 * kBS + r);
#pragma unroll
      for (int q = 0; q < kMaxDin / 4; ++q) {
        const int k = cq + 4 * q;
        if (k < din) {
          const float4 a = *reinterpret_cast<const float4*>(X + k * kBS + r);
          gw1[q] = fmaf(dz.x, a.x, fmaf(dz.y, a.y, fmaf(dz.z, a.z, fmaf(dz.w, a.w, gw1[q]))));
        }
      }
    }
    // dX[k][ray] = sum_j dZ1[j][ray] W1[j][k], k < 2L (features only)
    float dx[kMaxDin / 4 * 2 / 2];  // up to 8 feature rows per thread
    const int nk = (nf + 3) / 4;    // rows per thread part
    for (int q = 0; q < nk; ++q) dx[q] = 0.f;
    for (int j = 0; j < 64; ++j) {
      const float dz = A1[j * kBS + ray_slot];
      for (int q = 0; q < nk; ++q) {
        const int k = part * nk + q;
        if (k < nf) dx[q] = fmaf(dz, W1[j * din + k], dx[q]);
      }
    }
    __syncthreads();  // all reads of X (dW1) are done
    for (int q = 0; q < nk; ++q) {
      const int k = part * nk + q;
      if (k < nf) X[k * kBS + ray_slot] = dx[q];
    }
    __syncthreads();
    // ---- 4. scatter into the feature tables ----
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
  // ---- per-CTA weight gradients -> global ----
  for (int q = 0; q < kMaxDin / 4; ++q) {
    const int k = cq + 4 * q;
    if (k < din && gw1[q] != 0.f) atomicAdd(b.gw1 + j1 * din + k, gw1[q]);
  }
#pragma unroll
  for (int q = 0; q < 16; ++q)
    if (gw2[q] != 0.f) atomicAdd(b.gw2 + j1 * 64 + cq + 4 * q, gw2[q]);
  if (gw3 != 0.f) atomicAdd(b.gw3 + (tid >> 6) * 64 + (tid & 63), gw3);
}

static size_t bwd_smem_bytes() {
  return (size_t)(kMaxDin * 64 * 2 + 64 * 64 * 2 + 4 * 64 + (kMaxDin + 64 + 64 + 4) * kBS) * sizeof(float);
}

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
    grid_dev[dev] = sms * std::max(1, occ);
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

// Unwrapped table: row X + S (Y + S Z) of the S = 2m sided copy holds the
// canonical row (X mod m) + m ((Y mod m) + m (Z mod m)).
template <class Row>
__global__ void k_expand_table(const Row* __restrict__ src, Row* __restrict__ dst, uint32_t m, uint32_t S,
                               uint64_t n) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t X = (uint32_t)(i % S), Y = (uint32_t)((i / S) % S), Z = (uint32_t)(i / ((uint64_t)S * S));
    const uint32_t x = X >= m ? X - m : X, y = Y >= m ? Y - m : Y, z = Z >= m ? Z - m : Z;
    dst[i] = src[x + (uint64_t)m * (y + (uint64_t)m * z)];
  }
}

namespace inolf {
inolf_status expand_level_table(Object& o, int l, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const LevelDev& lv = o.lv[l];
  const uint64_t n = (uint64_t)lv.S * lv.S * lv.S;
  if (o.fp16)
    k_expand_table<__half2><<<1024, 256, 0, st>>>((const __half2*)lv.table, (__half2*)lv.tablex, (uint32_t)lv.m,
                                                  (uint32_t)lv.S, n);
  else
    k_expand_table<float2><<<1024, 256, 0, st>>>((const float2*)lv.table, (float2*)lv.tablex, (uint32_t)lv.m,
                                                 (uint32_t)lv.S, n);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(INOLF_E_CUDA, std::string("k_expand_table: ") + cudaGetErrorString(e));
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
      inolf_status es = inolf::expand_level_table(o, l, stream);
      if (es != INOLF_OK) return es;
    }
  }
  if (w1_dev) return inolf::pack_weights_device(o, w1_dev, w2_dev, w3_dev, stream);  // no host round trip
  return INOLF_OK;
}
