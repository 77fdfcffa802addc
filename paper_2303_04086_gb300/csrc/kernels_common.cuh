// Device building blocks of the i-NOLF per-ray path, shared by the forward,
// tensor-core and backward kernels of libinolf.so.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cmath>
#include <cstdint>

#include "inolf_internal.h"

namespace inolf {

static constexpr int kMaxViewsPerLaunch = 64;
static constexpr int kStackDepth = 48;  // >= BVH depth (checked at object creation)

struct Params {
  // geometry proxy
  const float4* nodes;
  const float4* tris;
  // rays of this launch
  int32_t mode;             // 0 = pinhole views (cams), 1 = explicit rays (ro, rd)
  int32_t W, H;
  int64_t n_rays;
  int64_t ray_base;         // global index of this launch's first ray (outputs)
  const float* ro;
  const float* rd;
  float cams[13 * kMaxViewsPerLaunch];
  // encoder
  int32_t L;
  int32_t fp16;
  float lo, scale;
  LevelDev lv[INOLF_MAX_LEVELS];
  // MLP
  int32_t d_in;
  const float* w_f32;
  const void* w_bf16;
  const void* w_fp8;
  const void* w_tf32;                 // FP32 weights split into TF32 hi / lo operands
  int32_t tc_k1_bf16, tc_k1_fp8, tc_k1_tf32;  // padded input width of the tensor-core layer 1
  uint32_t tc_bytes_bf16, tc_bytes_fp8, tc_bytes_tf32;
  const void* tc_w;                   // blob used by this launch
  int32_t tc_k1;
  uint32_t tc_wbytes;
  // split tensor-core shade: operand tiles of the hits [tc_h_begin,
  // tc_h_end) in the workspace (NULL: the fused kernel runs instead)
  uint8_t* tc_a;
  uint64_t tc_a_bytes;
  uint32_t tc_h_begin, tc_h_end;
  const float* fp8_w_scale;           // device [3]
  float fp8_act_scale[3];
  float shc[10];
  // outputs
  float4* rgba;
  int32_t* tri_out;
  float* t_out;
  uint32_t* slots_out;
  float* feat_out;
  // decoupled variant (Sec. 4.2): density march, alpha_c input, diffuse cubes
  int32_t variant;
  CubesDev cub;
  float* alpha_out;    // march stage output (inolf_march_rays), or NULL
  // bounded waits and test fault injection (process-wide settings)
  uint64_t wait_ns;    // limit of the gather/MLP hand-over waits
  uint32_t inject;     // INOLF_INJECT_* bits
  // offset tables of levels 0 .. phis_levels - 1 staged in shared memory by
  // k_shade_f32_ws (word offsets of each level's copy, 16-byte aligned)
  int32_t phis_levels;
  uint32_t phis_off[INOLF_MAX_LEVELS + 1];
  // workspace
  uint32_t* counter;   // [0] hit count, [1] error flags (INOLF_FLAG_*), [4..6] activation amax bits
  uint2* hits;         // (ray index in launch, t bits)
  float* hit_alpha;    // variant: alpha_c of each hit-list entry
};

// Backward-pass arguments (passed by value: every pointer is device memory).
struct BwdParams {
  float* gtab[INOLF_MAX_LEVELS];  // per level: m^3 x 2 FP32 gradient table (slot order)
  float* gw1;                     // [64][d_in]
  float* gw2;                     // [64][64]
  float* gw3;                     // [4][64]
  const float* d_rgba;            // [n][4] upstream gradient
};

// Real SH constants of bands 0..3 (no Condon-Shortley phase), from
// Y_l^m = K_l^m P_l^|m|(cos th) {sqrt2 cos(m ph), 1, sqrt2 sin(|m| ph)} with
// K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) written as polynomials of the
// unit direction (x, y, z):
//   Y00 = c0;  Y1,-1 = c1 y, Y10 = c1 z, Y11 = c1 x
//   Y2,-2 = c2a x y, Y2,-1 = c2a y z, Y20 = c2b (3 z^2 - 1), Y21 = c2a x z, Y22 = c2c (x^2 - y^2)
//   Y3,-3 = c3a y (3 x^2 - y^2), Y3,-2 = c3b x y z, Y3,-1 = c3d y (5 z^2 - 1), Y30 = c3e z (5 z^2 - 3),
//   Y31 = c3d x (5 z^2 - 1), Y32 = c3c z (x^2 - y^2), Y33 = c3a x (x^2 - 3 y^2)
inline void sh_constants(float c[10]) {
  const double pi = 3.14159265358979323846;
  c[0] = (float)(0.5 / std::sqrt(pi));             // c0
  c[1] = (float)std::sqrt(3.0 / (4.0 * pi));       // c1
  c[2] = (float)std::sqrt(15.0 / (4.0 * pi));      // c2a
  c[3] = (float)std::sqrt(5.0 / (16.0 * pi));      // c2b
  c[4] = (float)std::sqrt(15.0 / (16.0 * pi));     // c2c
  c[5] = (float)std::sqrt(35.0 / (32.0 * pi));     // c3a
  c[6] = (float)std::sqrt(105.0 / (4.0 * pi));     // c3b
  c[7] = (float)std::sqrt(105.0 / (16.0 * pi));    // c3c
  c[8] = (float)std::sqrt(21.0 / (32.0 * pi));     // c3d
  c[9] = (float)std::sqrt(7.0 / (16.0 * pi));      // c3e
}

__device__ __forceinline__ void sh16c(const float* c, const float d[3], float y[16]) {
  const float x = d[0], yy = d[1], z = d[2];
  const float x2 = x * x, y2 = yy * yy, z2 = z * z;
  y[0] = c[0];
  y[1] = c[1] * yy;
  y[2] = c[1] * z;
  y[3] = c[1] * x;
  y[4] = c[2] * x * yy;
  y[5] = c[2] * yy * z;
  y[6] = c[3] * (3.0f * z2 - 1.0f);
  y[7] = c[2] * x * z;
  y[8] = c[4] * (x2 - y2);
  y[9] = c[5] * yy * (3.0f * x2 - y2);
  y[10] = c[6] * x * yy * z;
  y[11] = c[8] * yy * (5.0f * z2 - 1.0f);
  y[12] = c[9] * z * (5.0f * z2 - 3.0f);
  y[13] = c[8] * x * (5.0f * z2 - 1.0f);
  y[14] = c[7] * z * (x2 - y2);
  y[15] = c[5] * x * (x2 - 3.0f * y2);
}

__device__ __forceinline__ void sh16(const Params& p, const float d[3], float y[16]) { sh16c(p.shc, d, y); }

__device__ __forceinline__ float sigmoidf_(float z) { return 1.0f / (1.0f + expf(-z)); }

// Pinhole ray of pixel (i, j), row 0 at the top (exact FP32 operation order):
//   tx = (tan * W) / H, a = (2i+1)/W - 1, b = 1 - (2j+1)/H
//   v = ((a tx) right + (b tan) up) + fwd, d = v * (1 / sqrt((vx^2 + vy^2) + vz^2))
__device__ __forceinline__ void make_ray(const float* cam, int W, int H, int i, int j, float o[3], float d[3]) {
  const float th = cam[12];
  const float fW = __int2float_rn(W), fH = __int2float_rn(H);
  const float tx = __fdiv_rn(__fmul_rn(th, fW), fH);
  const float a = __fsub_rn(__fdiv_rn(__int2float_rn(2 * i + 1), fW), 1.0f);
  const float b = __fsub_rn(1.0f, __fdiv_rn(__int2float_rn(2 * j + 1), fH));
  const float px = __fmul_rn(a, tx), py = __fmul_rn(b, th);
  float v[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) v[k] = __fadd_rn(__fadd_rn(__fmul_rn(px, cam[3 + k]), __fmul_rn(py, cam[6 + k])), cam[9 + k]);
  const float len2 = __fadd_rn(__fadd_rn(__fmul_rn(v[0], v[0]), __fmul_rn(v[1], v[1])), __fmul_rn(v[2], v[2]));
  const float inv = __fdiv_rn(1.0f, __fsqrt_rn(len2));
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    o[k] = cam[k];
    d[k] = __fmul_rn(v[k], inv);
  }
}

__device__ __forceinline__ void ray_of(const Params& p, int64_t ray, float o[3], float d[3]) {
  if (p.mode == 0) {
    const int64_t per_view = (int64_t)p.W * p.H;
    const int view = (int)(ray / per_view);
    const int64_t pix = ray - (int64_t)view * per_view;
    const int j = (int)(pix / p.W), i = (int)(pix - (int64_t)j * p.W);
    make_ray(p.cams + 13 * view, p.W, p.H, i, j, o, d);
  } else {
#pragma unroll
    for (int k = 0; k < 3; ++k) { o[k] = p.ro[3 * ray + k]; d[k] = p.rd[3 * ray + k]; }
  }
}

// Moller-Trumbore, two-sided, exact FP32 operation order; accepts when
// det != 0, u >= 0, v >= 0, u + v <= 1, t > 1e-6 and, when best_id >= 0,
// (t, id) can still win over (best_t, best_id).
//
// The result equals evaluating every quantity with its IEEE operations in the
// stated order.  Before paying for the division, tests that are implied by
// the numerators alone reject early: with n/det of opposite signs and
// neither value near the underflow or overflow range, RN(n * RN(1/det)) is
// strictly negative; with |n| > |det| (1 + 2^-16) it is strictly above 1 (or
// above best_t for t), since the three roundings change the quotient by less
// than 2^-22 relative.  These early exits reject only triangles the exact
// test rejects.
__device__ __forceinline__ bool mt_hit(const float o[3], const float d[3], const float4 v0, const float4 e1,
                                       const float4 e2, float best_t, bool have_best, float& t_out) {
  const float p0 = __fsub_rn(__fmul_rn(d[1], e2.z), __fmul_rn(d[2], e2.y));
  const float p1 = __fsub_rn(__fmul_rn(d[2], e2.x), __fmul_rn(d[0], e2.z));
  const float p2 = __fsub_rn(__fmul_rn(d[0], e2.y), __fmul_rn(d[1], e2.x));
  const float det = __fadd_rn(__fadd_rn(__fmul_rn(e1.x, p0), __fmul_rn(e1.y, p1)), __fmul_rn(e1.z, p2));
  if (det == 0.0f) return false;
  const float s0 = __fsub_rn(o[0], v0.x), s1 = __fsub_rn(o[1], v0.y), s2 = __fsub_rn(o[2], v0.z);
  const float nu = __fadd_rn(__fadd_rn(__fmul_rn(s0, p0), __fmul_rn(s1, p1)), __fmul_rn(s2, p2));
  const float adet = fabsf(det);
  const bool safe = adet < 1e12f && adet > 1e-30f;
  const float lim1 = adet * 1.0000153f;  // |det| (1 + 2^-16)
  const bool neg_det = det < 0.0f;
  if (safe && fabsf(nu) > 1e-30f && ((nu < 0.0f) != neg_det)) return false;  // u < 0
  if (safe && fabsf(nu) > lim1) return false;                                // |u| > 1
  const float q0 = __fsub_rn(__fmul_rn(s1, e1.z), __fmul_rn(s2, e1.y));
  const float q1 = __fsub_rn(__fmul_rn(s2, e1.x), __fmul_rn(s0, e1.z));
  const float q2 = __fsub_rn(__fmul_rn(s0, e1.y), __fmul_rn(s1, e1.x));
  const float nv = __fadd_rn(__fadd_rn(__fmul_rn(d[0], q0), __fmul_rn(d[1], q1)), __fmul_rn(d[2], q2));
  if (safe && fabsf(nv) > 1e-30f && ((nv < 0.0f) != neg_det)) return false;  // v < 0
  if (safe && fabsf(nv) > lim1) return false;                                // v > 1 (so u + v > 1)
  const float nt = __fadd_rn(__fadd_rn(__fmul_rn(e2.x, q0), __fmul_rn(e2.y, q1)), __fmul_rn(e2.z, q2));
  if (safe && fabsf(nt) > 1e-30f && ((nt < 0.0f) != neg_det)) return false;  // t < 0
  if (safe && have_best && fabsf(nt) > adet * best_t * 1.0000153f) return false;  // t > best_t
  const float inv = __fdiv_rn(1.0f, det);
  const float u = __fmul_rn(nu, inv);
  if (!(u >= 0.0f) || !(u <= 1.0f)) return false;  // u > 1 implies u + v > 1 or v < 0
  const float v = __fmul_rn(nv, inv);
  if (!(v >= 0.0f) || !(__fadd_rn(u, v) <= 1.0f)) return false;
  const float t = __fmul_rn(nt, inv);
  if (!(t > 1e-6f)) return false;
  t_out = t;
  return true;
}

// Slab test of a padded box; returns entry distance or +inf.  oi = o * inv
// per axis, so each plane distance is one fused multiply-add (the boxes are
// padded and the comparison against the best hit has slack, so the rounding
// of this test never decides a result).
// Three-operand minimum and maximum (one instruction each on sm_100 and
// later; a NaN operand is ignored, as by fminf / fmaxf).
__device__ __forceinline__ float fmin3(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

__device__ __forceinline__ float box_enter(float lox, float hix, float loy, float hiy, float loz, float hiz,
                                           const float oi[3], const float inv[3], float tmax) {
  const float ax = fmaf(lox, inv[0], -oi[0]), bx = fmaf(hix, inv[0], -oi[0]);
  const float ay = fmaf(loy, inv[1], -oi[1]), by = fmaf(hiy, inv[1], -oi[1]);
  const float az = fmaf(loz, inv[2], -oi[2]), bz = fmaf(hiz, inv[2], -oi[2]);
  const float t0 = fmax3(fminf(ax, bx), fminf(ay, by), fmaxf(fminf(az, bz), 0.0f));
  const float t1 = fmin3(fmaxf(ax, bx), fmaxf(ay, by), fminf(fmaxf(az, bz), tmax));
  return t0 <= t1 ? t0 : INFINITY;
}

// The same test when the signs of the direction are known at compile time
// (bit k of kSign set: d[k] has its sign bit set, so inv[k] < 0).  Since
// lo <= hi and a rounded multiply-add is monotone in lo, the entry plane of
// axis k is lo for inv[k] > 0 and hi for inv[k] < 0: the same plane that
// fminf / fmaxf pick in box_enter, so both return the same value, with no
// per-axis minimum or maximum.
template <int kSign>
__device__ __forceinline__ float box_enter_signed(float lox, float hix, float loy, float hiy, float loz, float hiz,
                                                  const float oi[3], const float inv[3], float tmax) {
  const float nx = fmaf((kSign & 1) ? hix : lox, inv[0], -oi[0]), fx = fmaf((kSign & 1) ? lox : hix, inv[0], -oi[0]);
  const float ny = fmaf((kSign & 2) ? hiy : loy, inv[1], -oi[1]), fy = fmaf((kSign & 2) ? loy : hiy, inv[1], -oi[1]);
  const float nz = fmaf((kSign & 4) ? hiz : loz, inv[2], -oi[2]), fz = fmaf((kSign & 4) ? loz : hiz, inv[2], -oi[2]);
  const float t0 = fmax3(nx, ny, fmaxf(nz, 0.0f));
  const float t1 = fmin3(fx, fy, fminf(fz, tmax));
  return t0 <= t1 ? t0 : INFINITY;
}

// Closest hit over the proxy: lexicographic minimum of (t, triangle id).  A
// subtree is skipped only when its padded box is entered after the current
// best t plus a relative slack, which never drops an equal-or-better hit.
__device__ __forceinline__ void closest_hit_bvh(const float4* __restrict__ nodes, const float4* __restrict__ tris,
                                                uint32_t* err, const float o[3], const float d[3], int32_t& best_id,
                                                float& best_t) {
  float inv[3], oi[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float dk = fabsf(d[k]) < 1e-20f ? copysignf(1e-20f, d[k]) : d[k];
    inv[k] = 1.0f / dk;
    oi[k] = o[k] * inv[k];
  }
  best_id = -1;
  best_t = INFINITY;
  int32_t st_idx[kStackDepth];
  int32_t st_cnt[kStackDepth];
  float st_t[kStackDepth];
  int sp = 0;
  int32_t cur = 0, cur_cnt = 0;  // inner node 0
  // every step visits a new node of a finite tree; the bound only guards
  // against a malformed node array (flagged, traversal stops)
  for (int32_t guard = 0;; ++guard) {
    if (guard > (1 << 22)) {
      atomicOr(err, INOLF_FLAG_TRAVERSAL_LIMIT);
      break;
    }
    const float lim = best_id < 0 ? INFINITY : best_t * 1.00002f + 1e-5f;
    if ((cur_cnt & 15) == 0) {  // count words carry the parent's split axis above bit 4
      const float4 nx = __ldg(nodes + 4 * cur + 0);
      const float4 ny = __ldg(nodes + 4 * cur + 1);
      const float4 nz = __ldg(nodes + 4 * cur + 2);
      const int4 meta = __ldg(reinterpret_cast<const int4*>(nodes) + 4 * cur + 3);
      const float tl = box_enter(nx.x, nx.y, ny.x, ny.y, nz.x, nz.y, oi, inv, lim);
      const float tr = box_enter(nx.z, nx.w, ny.z, ny.w, nz.z, nz.w, oi, inv, lim);
      // a child with index < 0 and count 0 is empty
      const bool hl = tl != INFINITY && (meta.x >= 0), hr = tr != INFINITY && (meta.z >= 0);
      if (hl && hr) {
        const bool lfirst = tl <= tr;
        if (sp < kStackDepth) {
          st_idx[sp] = lfirst ? meta.z : meta.x;
          st_cnt[sp] = lfirst ? meta.w : meta.y;
          st_t[sp] = lfirst ? tr : tl;
          ++sp;
        } else {
          atomicOr(err, INOLF_FLAG_STACK_OVERFLOW);  // flagged, subtree skipped
        }
        cur = lfirst ? meta.x : meta.z;
        cur_cnt = lfirst ? meta.y : meta.w;
        continue;
      } else if (hl || hr) {
        cur = hl ? meta.x : meta.z;
        cur_cnt = hl ? meta.y : meta.w;
        continue;
      }
    } else {
      for (int32_t k = 0, n = cur_cnt & 15; k < n; ++k) {
        const float4 a = __ldg(tris + 3 * (cur + k) + 0);
        const float4 b = __ldg(tris + 3 * (cur + k) + 1);
        const float4 c = __ldg(tris + 3 * (cur + k) + 2);
        float t;
        if (mt_hit(o, d, a, b, c, best_t, best_id >= 0, t)) {
          const int32_t id = __float_as_int(a.w);
          if (t < best_t || (t == best_t && id < best_id)) { best_t = t; best_id = id; }
        }
      }
    }
    // pop the next subtree that can still hold a better hit
    bool found = false;
    while (sp > 0) {
      --sp;
      const float lim2 = best_id < 0 ? INFINITY : best_t * 1.00002f + 1e-5f;
      if (st_t[sp] <= lim2) {
        cur = st_idx[sp];
        cur_cnt = st_cnt[sp];
        found = true;
        break;
      }
    }
    if (!found) break;
  }
  if (best_id < 0) best_t = 0.0f;
}

__device__ __forceinline__ void closest_hit(const Params& p, const float o[3], const float d[3], int32_t& best_id,
                                            float& best_t) {
  closest_hit_bvh(p.nodes, p.tris, p.counter + 1, o, d, best_id, best_t);
}

// Closest hit for the 32 rays of a warp traversed together (packet
// traversal): the warp visits a node when any of its rays enters the node's
// box within its own current best distance, every ray tests every triangle
// of a visited leaf (warp-uniform loads), and a stacked subtree is skipped
// only when no ray still wants it.  Each ray's result is the lexicographic
// (t, id) minimum over the triangles it tested, which include every
// triangle it can hit (its boxes are never rejected), so the result equals
// the per-ray traversal's.  All control flow depends on warp votes only, so
// the warp stays converged; lanes without a ray pass active = false.  Must
// be called by all 32 lanes of the warp.
// kCount: also returns the warp's inner-node visits and triangle tests (the
// same in every lane: the packet moves as one).
// kSign < 8: every active lane's direction has the signs of kSign (bits as
// in box_enter_signed); 8: the signs differ across the packet.
template <bool kCount, int kSign>
__device__ __forceinline__ void closest_hit_packet_s(const float4* __restrict__ nodes, const float4* __restrict__ tris,
                                                     uint32_t* err, bool active, const float o[3], const float d[3],
                                                     int32_t& best_id, float& best_t, uint32_t* n_inner,
                                                     uint32_t* n_tests) {
  uint32_t visits = 0, tests = 0;
  float inv[3], oi[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float dk = fabsf(d[k]) < 1e-20f ? copysignf(1e-20f, d[k]) : d[k];
    inv[k] = 1.0f / dk;
    oi[k] = o[k] * inv[k];
  }
  best_id = -1;
  best_t = INFINITY;
  int32_t st_idx[kStackDepth];  // the same in every lane
  int32_t st_cnt[kStackDepth];
  float st_t[kStackDepth];      // this lane's entry distance (INFINITY: not wanted)
  int sp = 0;
  int32_t cur = 0, cur_cnt = 0;  // inner node 0
  // This lane's limit on entry distances: its best t plus a relative slack
  // (INFINITY before a hit); -1 for a lane without a ray, which every box
  // test then rejects.  Changes only after a leaf.
  float lim = active ? INFINITY : -1.0f;
  for (int32_t guard = 0;; ++guard) {
    if (guard > (1 << 22)) {  // warp-uniform
      atomicOr(err, INOLF_FLAG_TRAVERSAL_LIMIT);
      break;
    }
    if ((cur_cnt & 15) == 0) {  // count words carry the parent's split axis above bit 4
      if (kCount) ++visits;
      const float4 nx = __ldg(nodes + 4 * cur + 0);
      const float4 ny = __ldg(nodes + 4 * cur + 1);
      const float4 nz = __ldg(nodes + 4 * cur + 2);
      const int4 meta = __ldg(reinterpret_cast<const int4*>(nodes) + 4 * cur + 3);
      float tl, tr;
      if constexpr (kSign < 8) {
        // an empty child's box is stored inverted (lo = +inf, hi = -inf): its
        // entry plane is +inf, so the signed test rejects it
        tl = box_enter_signed<kSign>(nx.x, nx.y, ny.x, ny.y, nz.x, nz.y, oi, inv, lim);
        tr = box_enter_signed<kSign>(nx.z, nx.w, ny.z, ny.w, nz.z, nz.w, oi, inv, lim);
      } else {
        tl = box_enter(nx.x, nx.y, ny.x, ny.y, nz.x, nz.y, oi, inv, lim);
        tr = box_enter(nx.z, nx.w, ny.z, ny.w, nz.z, nz.w, oi, inv, lim);
        if (meta.x < 0) tl = INFINITY;
        if (meta.z < 0) tr = INFINITY;
      }
      const bool hl = tl != INFINITY, hr = tr != INFINITY;
      const bool wl = __any_sync(0xffffffffu, hl), wr = __any_sync(0xffffffffu, hr);
      if (wl && wr) {
        bool lfirst;
        if constexpr (kSign < 8) {
          // the left child holds the lower centroids along the node's split
          // axis: it goes first when the packet moves up that axis
          lfirst = !((kSign >> ((meta.y >> 4) & 3)) & 1);
        } else {
          // the child most rays enter first goes first
          const uint32_t first_l = __ballot_sync(0xffffffffu, hl && (!hr || tl <= tr));
          const uint32_t first_r = __ballot_sync(0xffffffffu, hr && (!hl || tr < tl));
          lfirst = __popc(first_l) >= __popc(first_r);
        }
        if (sp < kStackDepth) {
          st_idx[sp] = lfirst ? meta.z : meta.x;
          st_cnt[sp] = lfirst ? meta.w : meta.y;
          st_t[sp] = lfirst ? tr : tl;
          ++sp;
        } else {
          atomicOr(err, INOLF_FLAG_STACK_OVERFLOW);  // flagged, subtree skipped
        }
        cur = lfirst ? meta.x : meta.z;
        cur_cnt = lfirst ? meta.y : meta.w;
        continue;
      } else if (wl || wr) {
        cur = wl ? meta.x : meta.z;
        cur_cnt = wl ? meta.y : meta.w;
        continue;
      }
    } else {
      if (kCount) tests += (uint32_t)(cur_cnt & 15);
      for (int32_t k = 0, n = cur_cnt & 15; k < n; ++k) {
        const float4 a = __ldg(tris + 3 * (cur + k) + 0);
        const float4 b = __ldg(tris + 3 * (cur + k) + 1);
        const float4 c = __ldg(tris + 3 * (cur + k) + 2);
        float t;
        if (active && mt_hit(o, d, a, b, c, best_t, best_id >= 0, t)) {
          const int32_t id = __float_as_int(a.w);
          if (t < best_t || (t == best_t && id < best_id)) { best_t = t; best_id = id; }
        }
      }
      if (best_id >= 0) lim = best_t * 1.00002f + 1e-5f;
    }
    // pop the next subtree that some ray of the warp still wants
    bool found = false;
    while (sp > 0) {
      --sp;
      if (__any_sync(0xffffffffu, st_t[sp] <= lim)) {
        cur = st_idx[sp];
        cur_cnt = st_cnt[sp];
        found = true;
        break;
      }
    }
    if (!found) break;
  }
  if (best_id < 0) best_t = 0.0f;
  if (kCount) {
    *n_inner = visits;
    *n_tests = tests;
  }
}

// Dispatches the packet to the traversal specialised for its direction
// signs when all its active rays share them (the usual case for a camera
// tile: only tiles that a plane d[k] = 0 crosses take the general test).
template <bool kCount = false>
__device__ __forceinline__ void closest_hit_packet(const float4* __restrict__ nodes, const float4* __restrict__ tris,
                                                   uint32_t* err, bool active, const float o[3], const float d[3],
                                                   int32_t& best_id, float& best_t, uint32_t* n_inner = nullptr,
                                                   uint32_t* n_tests = nullptr) {
  const uint32_t sgn = (signbit(d[0]) ? 1u : 0u) | (signbit(d[1]) ? 2u : 0u) | (signbit(d[2]) ? 4u : 0u);
  const uint32_t act = __ballot_sync(0xffffffffu, active);
  uint32_t kind = 8u;
  if (act) {
    const uint32_t s0 = __shfl_sync(0xffffffffu, sgn, __ffs(act) - 1);
    if (__all_sync(0xffffffffu, !active || sgn == s0)) kind = s0;
  }
#define INOLF_PACKET_CASE(k)                                                                               \
  case k:                                                                                                  \
    closest_hit_packet_s<kCount, k>(nodes, tris, err, active, o, d, best_id, best_t, n_inner, n_tests); \
    break;
  switch (kind) {
    INOLF_PACKET_CASE(0)
    INOLF_PACKET_CASE(1)
    INOLF_PACKET_CASE(2)
    INOLF_PACKET_CASE(3)
    INOLF_PACKET_CASE(4)
    INOLF_PACKET_CASE(5)
    INOLF_PACKET_CASE(6)
    INOLF_PACKET_CASE(7)
    default:
      closest_hit_packet_s<kCount, 8>(nodes, tris, err, active, o, d, best_id, best_t, n_inner, n_tests);
  }
#undef INOLF_PACKET_CASE
}

// Scene-unit coordinates of the hit point: P = o + t d, x = (P - lo) * scale.
__device__ __forceinline__ void hit_unit_coords_ls(float lo, float scale, const float o[3], const float d[3], float t,
                                                   float x[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float P = __fadd_rn(o[k], __fmul_rn(t, d[k]));
    x[k] = __fmul_rn(__fsub_rn(P, lo), scale);
  }
}
__device__ __forceinline__ void hit_unit_coords(const Params& p, const float o[3], const float d[3], float t,
                                                float x[3]) {
  hit_unit_coords_ls(p.lo, p.scale, o, d, t, x);
}

// a mod m for 0 <= a < 2^21 and 1 <= m < 2048 by division by an invariant
// integer (Granlund and Montgomery 1994): with magic = ceil(2^32 / m), the
// high word of a * magic is floor(a/m + e), 0 <= e < a / 2^32 < 2^-11, and a/m
// is never within 2^-11 below an integer when m < 2048, so the quotient is
// exact; the one correction covers m = 1, whose magic is clamped to 2^32 - 1.
__device__ __forceinline__ int32_t mod_small(int32_t a, int32_t m, uint32_t magic) {
  const uint32_t q = __umulhi((uint32_t)a, magic);
  uint32_t r = (uint32_t)a - q * (uint32_t)m;
  r -= (r >= (uint32_t)m) ? (uint32_t)m : 0u;
  return (int32_t)r;
}

// Cell of level `lv` (Sec. 4.1, p = floor(N x)): c = clamp(floor(u), 0, N-1),
// f = u - c with u = N x, all in FP32.
__device__ __forceinline__ void cell_of(const LevelDev& lv, const float x[3], int32_t c[3], float f[3]) {
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float u = __fmul_rn(lv.N_f, x[k]);
    int32_t ci = (int32_t)floorf(u);
    ci = ci < 0 ? 0 : (ci > lv.N - 1 ? lv.N - 1 : ci);
    c[k] = ci;
    f[k] = __fsub_rn(u, __int2float_rn(ci));
  }
}

// Per-level state between the two dependent loads of the gather: the 8 Phi
// entries (in flight), the wrapped h0 coordinates and the cell fractions.
struct LevelFetch {
  uint32_t ph[8];
  int32_t h0[3], h0n[3];
  float f[3];
};

// Cell of the level, h0 / h1 coordinates of the 8 corners c + (dx, dy, dz)
// (x fastest), and the loads of their Phi entries (Eq. 1, first half).
__device__ __forceinline__ void fetch_phi(const LevelDev& lv, const float x[3], LevelFetch& s) {
  int32_t c[3];
  cell_of(lv, x, c, s.f);
  const int32_t m = lv.m, r = lv.r;
  int32_t qx[2], qy[2], qz[2];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    s.h0[k] = mod_small(c[k], m, lv.magic_m);
    s.h0n[k] = s.h0[k] + 1 == m ? 0 : s.h0[k] + 1;
  }
  {
    const int32_t a = mod_small(c[0], r, lv.magic_r);
    qx[0] = a;
    qx[1] = a + 1 == r ? 0 : a + 1;
    const int32_t b = mod_small(c[1], r, lv.magic_r);
    qy[0] = b * r;
    qy[1] = (b + 1 == r ? 0 : b + 1) * r;
    const int32_t z = mod_small(c[2], r, lv.magic_r);
    qz[0] = z * r * r;
    qz[1] = (z + 1 == r ? 0 : z + 1) * r * r;
  }
#pragma unroll
  for (int cc = 0; cc < 8; ++cc) s.ph[cc] = __ldg(lv.phi + (qx[cc & 1] + qy[(cc >> 1) & 1] + qz[cc >> 2]));
}

// Second half of Eq. 1: slots (h0 + phi) mod m of the 8 corners, the feature
// gather and the trilinear interpolation of the F = 2 features.
__device__ __forceinline__ void finish_level(const LevelDev& lv, int fp16, const LevelFetch& s, uint32_t slots[8],
                                             float& e0, float& e1) {
  const int32_t m = lv.m;
#pragma unroll
  for (int cc = 0; cc < 8; ++cc) {
    // (h0 + phi) mod m per axis as min(s, s - m) in unsigned arithmetic
    // (s < 2m: s - m wraps above s exactly when s < m)
    const uint32_t um = (uint32_t)m;
    uint32_t sx = (uint32_t)((cc & 1) ? s.h0n[0] : s.h0[0]) + (s.ph[cc] & 1023u);
    uint32_t sy = (uint32_t)((cc & 2) ? s.h0n[1] : s.h0[1]) + ((s.ph[cc] >> 10) & 1023u);
    uint32_t sz = (uint32_t)((cc & 4) ? s.h0n[2] : s.h0[2]) + (s.ph[cc] >> 20);
    sx = min(sx, sx - um);
    sy = min(sy, sy - um);
    sz = min(sz, sz - um);
    slots[cc] = sx + um * (sy + um * sz);
  }
  float2 v[8];
  if (fp16) {
    const __half2* tb = reinterpret_cast<const __half2*>(lv.table);
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) v[cc] = __half22float2(__ldg(tb + slots[cc]));
  } else {
    const float2* tb = reinterpret_cast<const float2*>(lv.table);
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) v[cc] = __ldg(tb + slots[cc]);
  }
  // trilinear interpolation as nested lerps along x, then y, then z
  const float* f = s.f;
  float ax[4], bx[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    ax[k] = fmaf(f[0], v[2 * k + 1].x - v[2 * k].x, v[2 * k].x);
    bx[k] = fmaf(f[0], v[2 * k + 1].y - v[2 * k].y, v[2 * k].y);
  }
  const float ay0 = fmaf(f[1], ax[1] - ax[0], ax[0]), ay1 = fmaf(f[1], ax[3] - ax[2], ax[2]);
  const float by0 = fmaf(f[1], bx[1] - bx[0], bx[0]), by1 = fmaf(f[1], bx[3] - bx[2], bx[2]);
  e0 = fmaf(f[2], ay1 - ay0, ay0);
  e1 = fmaf(f[2], by1 - by0, by0);
}

// The same level fetch on the corner bundles (see LevelDev): Eq. 1 gives
// the slot h(c) of the cell's lowest corner c, and bundle row h(c) holds the
// feature rows of all 8 corners, so a level costs one Phi load and one
// 64-byte (FP32) or 32-byte (FP16) read -- half a 128-byte cache line -- in
// place of 8 Phi loads and 8 scattered row loads.  The rows are those of the
// canonical slots h(c + d), so the result equals finish_level's.
struct LevelFetchB {
  uint32_t ph;     // packed Phi entry of h1(c) (in flight)
  uint32_t h0[3];  // h0(c) per axis
  float f[3];
};

// Cell, fractions, h0(c) and the load of Phi[h1(c)] (Eq. 1, first half);
// `phi` is lv.phi or a copy of it staged in shared memory.
__device__ __forceinline__ void fetch_bundle_phi_from(const LevelDev& lv, const uint32_t* phi, const float x[3],
                                                      LevelFetchB& s) {
  int32_t c[3];
  cell_of(lv, x, c, s.f);
  const uint32_t r = (uint32_t)lv.r;
#pragma unroll
  for (int k = 0; k < 3; ++k) s.h0[k] = (uint32_t)mod_small(c[k], lv.m, lv.magic_m);
  const uint32_t q = (uint32_t)mod_small(c[0], lv.r, lv.magic_r) +
                     r * ((uint32_t)mod_small(c[1], lv.r, lv.magic_r) + r * (uint32_t)mod_small(c[2], lv.r, lv.magic_r));
  s.ph = phi[q];
}

__device__ __forceinline__ void fetch_bundle_phi(const LevelDev& lv, const float x[3], LevelFetchB& s) {
  int32_t c[3];
  cell_of(lv, x, c, s.f);
  const uint32_t r = (uint32_t)lv.r;
#pragma unroll
  for (int k = 0; k < 3; ++k) s.h0[k] = (uint32_t)mod_small(c[k], lv.m, lv.magic_m);
  const uint32_t q = (uint32_t)mod_small(c[0], lv.r, lv.magic_r) +
                     r * ((uint32_t)mod_small(c[1], lv.r, lv.magic_r) + r * (uint32_t)mod_small(c[2], lv.r, lv.magic_r));
  s.ph = __ldg(lv.phi + q);
}

// Second half of Eq. 1 for the lowest corner, the bundle read and the
// trilinear interpolation (the same operations, in the same order, as
// finish_level).
__device__ __forceinline__ void finish_bundle(const LevelDev& lv, int fp16, const LevelFetchB& s, float& e0,
                                              float& e1) {
  const uint32_t um = (uint32_t)lv.m;
  uint32_t sx = s.h0[0] + (s.ph & 1023u), sy = s.h0[1] + ((s.ph >> 10) & 1023u), sz = s.h0[2] + (s.ph >> 20);
  sx = min(sx, sx - um);  // (h0 + phi) mod m, as in finish_level
  sy = min(sy, sy - um);
  sz = min(sz, sz - um);
  const size_t slot = (size_t)(sx + um * (sy + um * sz));
  float2 v[8];
  if (fp16) {
    const uint4* b = reinterpret_cast<const uint4*>(lv.bundle) + 2 * slot;
    const uint4 u0 = __ldg(b), u1 = __ldg(b + 1);
    const uint32_t w[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) v[cc] = __half22float2(*reinterpret_cast<const __half2*>(&w[cc]));
  } else {
    const float4* b = reinterpret_cast<const float4*>(lv.bundle) + 4 * slot;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float4 u = __ldg(b + k);
      v[2 * k] = make_float2(u.x, u.y);
      v[2 * k + 1] = make_float2(u.z, u.w);
    }
  }
  const float* f = s.f;
  float ax[4], bx[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    ax[k] = fmaf(f[0], v[2 * k + 1].x - v[2 * k].x, v[2 * k].x);
    bx[k] = fmaf(f[0], v[2 * k + 1].y - v[2 * k].y, v[2 * k].y);
  }
  const float ay0 = fmaf(f[1], ax[1] - ax[0], ax[0]), ay1 = fmaf(f[1], ax[3] - ax[2], ax[2]);
  const float by0 = fmaf(f[1], bx[1] - bx[0], bx[0]), by1 = fmaf(f[1], bx[3] - bx[2], bx[2]);
  e0 = fmaf(f[2], ay1 - ay0, ay0);
  e1 = fmaf(f[2], by1 - by0, by0);
}

// Eq. 1 slots of the 8 corners and the interpolated features of one level.
__device__ __forceinline__ void encode_level(const LevelDev& lv, int fp16, const float x[3], uint32_t slots[8],
                                             float& e0, float& e1) {
  LevelFetch s;
  fetch_phi(lv, x, s);
  finish_level(lv, fp16, s, slots, e0, e1);
}

// All levels of one hit point, with the Phi loads of level l + 1 issued
// before the feature loads of level l are consumed (two dependent load
// rounds per level overlap across levels).  emit(l, e0, e1, slots) receives
// each level's result in order.
template <class Emit>
__device__ __forceinline__ void encode_all_levels(const Params& p, const float x[3], Emit&& emit) {
  LevelFetch cur, nxt;
  fetch_phi(p.lv[0], x, cur);
  for (int l = 0; l < p.L; ++l) {
    if (l + 1 < p.L) fetch_phi(p.lv[l + 1], x, nxt);
    uint32_t slots[8];
    float e0, e1;
    finish_level(p.lv[l], p.fp16, cur, slots, e0, e1);
    emit(l, e0, e1, slots);
    cur = nxt;
  }
}

// ---------------------------------------------------------------------------
// Density texture cubes (Sec. 4.2): the hit-point march of Eq. 4 and the
// diffuse lookup of Eq. 7.
// ---------------------------------------------------------------------------
static constexpr int32_t kMaxMarchSteps = 1 << 20;  // > side sqrt(3) / step + 1, checked at creation
static constexpr float kSkipMargin = 0.05f;          // fine cells kept between a skipped sample and a block face

// Span [t0, t1] of the ray inside the scene cube [lo, hi]^3: per axis the
// plane distances (plane - o) / d in FP32, axes with d = 0 only test o.
__device__ __forceinline__ bool cube_span(float lo, float hi, const float o[3], const float d[3], float& t0,
                                          float& t1) {
  float a = 0.0f, z = INFINITY;
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    if (d[q] == 0.0f) {
      if (o[q] < lo || o[q] > hi) return false;
      continue;
    }
    const float ta = __fdiv_rn(__fsub_rn(lo, o[q]), d[q]);
    const float tb = __fdiv_rn(__fsub_rn(hi, o[q]), d[q]);
    a = fmaxf(a, fminf(ta, tb));
    z = fminf(z, fmaxf(ta, tb));
  }
  if (a > z) return false;
  t0 = a;
  t1 = z;
  return true;
}

// a + f (b - a) with each operation rounded on its own
__device__ __forceinline__ float lerp_rn(float a, float b, float f) { return __fadd_rn(a, __fmul_rn(f, __fsub_rn(b, a))); }

// Fine cell (clamped to the grid), in-cell fractions and unclamped fine
// coordinates of the point with scene-unit coordinates x.
__device__ __forceinline__ void fine_cell(const CubesDev& c, const float x[3], int32_t ci[3], float f[3],
                                          float u[3]) {
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    u[q] = __fmul_rn(c.K_f, x[q]);
    int32_t v = (int32_t)floorf(u[q]);
    v = v < 0 ? 0 : (v > c.K - 1 ? c.K - 1 : v);
    ci[q] = v;
    f[q] = __fsub_rn(u[q], __int2float_rn(v));
  }
}

// The march of one ray (Eq. 4): samples t_k = t0 + k step, sigma_k from the
// cubes, w_k = T_k (1 - e_k), T_{k+1} = T_k e_k, e_k = exp(-sigma_k step),
// stop once T < t_min; hit = first sample of largest w_k, alpha_c = 1 - T.
// Samples where sigma = 0 change nothing.  The octant distance fields mark,
// for the ray's octant, a block of such samples that starts at the current
// cell and extends the way the ray travels: unlisted base cells between the
// cubes, or fine cells that are not live inside a cube (clipped to the cube).
// The march skips the samples that provably stay inside that block (with a
// margin of kSkipMargin fine cells, far above the FP32 error of the sample
// coordinates), so the samples it evaluates, and therefore the result, are
// those of the plain loop.
__device__ __forceinline__ void march_ray(const CubesDev& c, float lo, float scale, const float o[3],
                                          const float d[3], int32_t& k_hit, float& t_hit, float& alpha) {
  k_hit = -1;
  t_hit = 0.0f;
  alpha = 0.0f;
  float t0, t1;
  if (!cube_span(lo, c.hi, o, d, t0, t1)) return;
  float inv_du[3];  // samples per fine cell along each axis (0: the ray does not move along it)
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const float du = fabsf(c.K_f * scale * d[q] * c.step);
    inv_du[q] = du > 0.0f ? 1.0f / du : 0.0f;
  }
  const bool neg[3] = {d[0] < 0.0f, d[1] < 0.0f, d[2] < 0.0f};
  const int32_t oct = (neg[0] ? 1 : 0) | (neg[1] ? 2 : 0) | (neg[2] ? 4 : 0);
  const int32_t R1 = c.r + 1, r3 = c.r * c.r * c.r;
  const uint8_t* bdist = c.bdist + (size_t)oct * c.b * c.b * c.b;
  const uint8_t* fdist = c.fdist + (size_t)oct * c.n_cubes * r3;
  float T = 1.0f, wmax = 0.0f, tbest = 0.0f;
  int32_t kbest = -1;
  int32_t k = 0;
  for (int32_t guard = 0; guard < kMaxMarchSteps; ++guard) {  // k grows by >= 1 per iteration
    const float t = __fadd_rn(t0, __fmul_rn(__int2float_rn(k), c.step));
    if (t > t1) break;
    float x[3], u[3], f[3];
    int32_t ci[3];
    hit_unit_coords_ls(lo, scale, o, d, t, x);
    fine_cell(c, x, ci, f, u);
    const int32_t bq[3] = {ci[0] >> c.rshift, ci[1] >> c.rshift, ci[2] >> c.rshift};
    const int32_t lin = bq[0] + c.b * (bq[1] + c.b * bq[2]);
    const int32_t e = __ldg(c.grid + lin);
    const int32_t Db = __ldg(bdist + lin);
    const int32_t lf[3] = {ci[0] - (bq[0] << c.rshift), ci[1] - (bq[1] << c.rshift), ci[2] - (bq[2] << c.rshift)};
    // the face of the empty block the ray leaves through, per axis (fine cells)
    int32_t D, face[3];
    if (e < 0) {
      D = Db;
#pragma unroll
      for (int q = 0; q < 3; ++q) face[q] = (neg[q] ? bq[q] - D + 1 : bq[q] + D) * c.r;
    } else {
      D = __ldg(fdist + (size_t)e * r3 + lf[0] + c.r * (lf[1] + c.r * lf[2]));
#pragma unroll
      for (int q = 0; q < 3; ++q)
        face[q] = neg[q] ? max(bq[q] * c.r, ci[q] - D + 1) : min((bq[q] + 1) * c.r, ci[q] + D);
    }
    if (D > 0) {
      float s = 1048576.0f;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        if (inv_du[q] > 0.0f) {
          const float rem = neg[q] ? u[q] - __int2float_rn(face[q]) : __int2float_rn(face[q]) - u[q];
          s = fminf(s, (rem - kSkipMargin) * inv_du[q]);
        }
      }
      k += 1 + (s >= 1.0f ? (int32_t)s : 0);
      continue;
    }
    const float* v0 = c.dens + (size_t)e * R1 * R1 * R1 + lf[0] + R1 * (lf[1] + R1 * lf[2]);
    const float s000 = __ldg(v0), s100 = __ldg(v0 + 1);
    const float s010 = __ldg(v0 + R1), s110 = __ldg(v0 + R1 + 1);
    const float s001 = __ldg(v0 + R1 * R1), s101 = __ldg(v0 + R1 * R1 + 1);
    const float s011 = __ldg(v0 + R1 * R1 + R1), s111 = __ldg(v0 + R1 * R1 + R1 + 1);
    const float a00 = lerp_rn(s000, s100, f[0]), a10 = lerp_rn(s010, s110, f[0]);
    const float a01 = lerp_rn(s001, s101, f[0]), a11 = lerp_rn(s011, s111, f[0]);
    const float sigma = lerp_rn(lerp_rn(a00, a10, f[1]), lerp_rn(a01, a11, f[1]), f[2]);
    if (sigma != 0.0f) {  // sigma = 0: w = 0 and T unchanged
      const float ek = expf(-__fmul_rn(sigma, c.step));
      const float w = __fmul_rn(T, __fsub_rn(1.0f, ek));
      T = __fmul_rn(T, ek);
      if (w > wmax) {
        wmax = w;
        kbest = k;
        tbest = t;
      }
      if (T < c.t_min) break;
    }
    ++k;
  }
  alpha = __fsub_rn(1.0f, T);
  if (alpha > c.alpha_miss && kbest >= 0) {
    k_hit = kbest;
    t_hit = tbest;
  }
}

// (c_d r, g, b, tint) at the point with scene-unit coordinates x: trilinear
// interpolation of its fine cell's 8 diffuse samples (zero if the cell's
// cube is not listed, which a hit point's never is).
__device__ __forceinline__ float4 cube_diffuse(const CubesDev& c, const float x[3]) {
  float u[3], f[3];
  int32_t ci[3];
  fine_cell(c, x, ci, f, u);
  const int32_t bx = ci[0] >> c.rshift, by = ci[1] >> c.rshift, bz = ci[2] >> c.rshift;
  const int32_t e = __ldg(c.grid + bx + c.b * (by + c.b * bz));
  if (e < 0) return make_float4(0.f, 0.f, 0.f, 0.f);
  const int32_t R1 = c.r + 1;
  const float4* v0 = c.diff + (size_t)e * R1 * R1 * R1 + (ci[0] - (bx << c.rshift)) +
                     R1 * ((ci[1] - (by << c.rshift)) + R1 * (ci[2] - (bz << c.rshift)));
  float4 v[8];
  v[0] = __ldg(v0);
  v[1] = __ldg(v0 + 1);
  v[2] = __ldg(v0 + R1);
  v[3] = __ldg(v0 + R1 + 1);
  v[4] = __ldg(v0 + R1 * R1);
  v[5] = __ldg(v0 + R1 * R1 + 1);
  v[6] = __ldg(v0 + R1 * R1 + R1);
  v[7] = __ldg(v0 + R1 * R1 + R1 + 1);
  auto lerp4 = [](float4 a, float4 b, float t) {
    return make_float4(fmaf(t, b.x - a.x, a.x), fmaf(t, b.y - a.y, a.y), fmaf(t, b.z - a.z, a.z),
                       fmaf(t, b.w - a.w, a.w));
  };
  const float4 y0 = lerp4(lerp4(v[0], v[1], f[0]), lerp4(v[2], v[3], f[0]), f[1]);
  const float4 y1 = lerp4(lerp4(v[4], v[5], f[0]), lerp4(v[6], v[7], f[0]), f[1]);
  return lerp4(y0, y1, f[2]);
}

}  // namespace inolf
