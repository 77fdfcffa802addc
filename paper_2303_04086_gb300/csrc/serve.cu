// Continuous-batching request loop for many viewers over several resident
// i-NOLF objects on one GPU (the paper's render farm and frame composer,
// Sec. 5-6, collapsed onto a single device).
//
// A persistent kernel (one or a few CTAs per SM) claims work units -- 16x16
// pixel tiles of any live request -- from a ring that the host publishes in
// mapped host memory.  Requests that arrive while others are being rendered
// are published into the same ring, so their tiles interleave with the
// earlier requests' tiles on the device: there is no per-request launch and
// no waiting for a batch to drain.  For every pixel of a tile the CTA
//   1. generates the viewer's pinhole ray (world frame);
//   2. intersects every resident object's proxy in that object's local frame
//      (translation-only placement) and keeps the K nearest hits, ordered by
//      (t, object id);
//   3. shades each hit with its object's encoding and MLP (one query per hit,
//      Sec. 4.2), the object's weights staged in shared memory;
//   4. composites the hits front to back with the straight-alpha "over"
//      operator (depth-ordered fusion, the frame composer of Sec. 5.1):
//      C += (1 - A) a c, A += (1 - A) a, and writes (C / A, A).
// The last tile of a request publishes its completion to mapped host memory.
// Admission is by slot count and by an arena of device memory for the
// frames (the HBM budget).  Every device-side wait is bounded by the global
// timer: an idle kernel exits after idle_limit_ns (the host relaunches it on
// the next submission), and a tile whose request descriptor does not appear
// within wait_limit_ns completes with INOLF_E_TIMEOUT.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <map>
#include <atomic>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "inolf_internal.h"
#include "kernels_common.cuh"
#include "tc_mlp.cuh"
#include "tc_ptx.cuh"

namespace inolf {

static constexpr int kServeMaxObjects = 16;
static constexpr int kServeMaxK = 4;
static constexpr int kServeTile = 16;
static constexpr int kServeThreads = kServeTile * kServeTile;
static constexpr int kServeMaxSlots = 256;
static constexpr int kServeMaxDin = 2 * INOLF_MAX_LEVELS + INOLF_N_SH + 1;  // + alpha_c (density-cube objects)
static constexpr unsigned long long kServeClaim = 16;  // tiles claimed per atomic

struct ServeObj {
  const float4* nodes;
  const float4* tris;
  const float* w_f32;
  const void* w_bf16;      // tensor-core operand blob (BF16)
  int32_t tc_k1_bf16;
  uint32_t tc_bytes_bf16;
  int32_t L, fp16, d_in, pad;
  float lo, scale;
  float T[3];  // object placement: local = world - T
  float bs_c[3], bs_r2;  // bounding sphere of the proxy (local frame), padded
  int32_t variant;       // 1: hit by the density march, alpha_c input, c = c_d + tint c_s
  CubesDev cub;
  LevelDev lv[INOLF_MAX_LEVELS];
};

struct ServeSlot {  // mapped host memory, written by the host at submission
  uint32_t gen;
  int32_t W, H, prec;
  float* out;
  float cam[13];
  uint32_t tiles_x, tiles_total;
  uint32_t cancelled;
};

struct __align__(16) ServeTile {  // ring entry, mapped host memory (two 16-byte loads)
  uint32_t slot, gen, tx, ty;
  uint32_t tiles_total, pad0, pad1, pad2;
};

struct ServeDone {  // completion record, mapped host memory, written by the device
  uint32_t gen;
  int32_t status;
};

struct ServeCtl {  // mapped host memory
  unsigned long long published;  // tiles published so far (host)
  uint32_t stop;                 // host asks the kernel to exit
  uint32_t pad;
};

// Profile of the request loop (inolf_serve_profile), summed over CTAs when
// each persistent CTA exits: SM cycles per phase, then event counts.
enum ServeProf {
  kProfClaim = 0,   // claiming tiles and reading request descriptors (includes waiting for work)
  kProfTrace,       // ray generation, every object's proxy traced, K nearest hits sorted and grouped
  kProfShade,       // per object: weights staged, encoding gathered, MLP
  kProfComposite,   // front-to-back compositing and the frame store
  kProfDone,        // completion counting and publication
  kProfTiles,       // tiles processed
  kProfHits,        // hits shaded (<= K per pixel)
  kProfBatches,     // MLP batches (one 256-row tensor-core pass, or one FP32 pass of an object)
  kProfWeightLoads, // weight stagings into shared memory
  kProfCount
};

struct ServeDevState {  // device memory
  unsigned long long head;           // tiles claimed so far
  unsigned long long last_activity;  // global timer of the last claim
  uint32_t tiles_done[kServeMaxSlots];
  int32_t status[kServeMaxSlots];
  uint32_t err;
  uint32_t pad;
  unsigned long long prof[kProfCount];
};

struct ServeKParams {
  const ServeObj* objs;
  int32_t n_objs;
  int32_t K;
  ServeCtl* ctl;
  ServeDone* done;
  const ServeSlot* slots;
  const ServeTile* ring;
  unsigned long long ring_cap;
  ServeDevState* st;
  unsigned long long wait_limit_ns;
  unsigned long long idle_limit_ns;
  float shc[10];
};

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned long long ld_acq_sys_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_acq_sys_u32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_vol_u32(const uint32_t* p) { return *(const volatile uint32_t*)p; }
__device__ __forceinline__ float ld_vol_f32(const float* p) { return *(const volatile float*)p; }
__device__ __forceinline__ uint4 ld_vol_v4(const void* p) {
  uint4 v;
  asm volatile("ld.volatile.global.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p)
               : "memory");
  return v;
}
__device__ __forceinline__ void st_rel_sys_u32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// FP32 MLP F_s of one hit from shared-memory weights (W1T [d_in][64],
// W2 [64][64], W3T [64][4]); x = features (2L) followed by 16 SH values.
__device__ __forceinline__ float4 mlp_f32(const float4* W1T, const float4* W2, const float4* W3T, const float* x,
                                          int din) {
  float h1[64];
#pragma unroll
  for (int j = 0; j < 64; ++j) h1[j] = 0.0f;
  for (int i = 0; i < din; ++i) {
    const float v = x[i];
    const float4* r = W1T + i * 16;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const float4 a = r[q];
      h1[4 * q + 0] += a.x * v;
      h1[4 * q + 1] += a.y * v;
      h1[4 * q + 2] += a.z * v;
      h1[4 * q + 3] += a.w * v;
    }
  }
#pragma unroll
  for (int j = 0; j < 64; ++j) h1[j] = fmaxf(h1[j], 0.0f);
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 2
  for (int j = 0; j < 64; ++j) {
    const float4* r = W2 + j * 16;
    float z = 0.0f;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const float4 a = r[q];
      z += a.x * h1[4 * q + 0] + a.y * h1[4 * q + 1] + a.z * h1[4 * q + 2] + a.w * h1[4 * q + 3];
    }
    z = fmaxf(z, 0.0f);
    const float4 w3 = W3T[j];
    acc.x += w3.x * z;
    acc.y += w3.y * z;
    acc.z += w3.z * z;
    acc.w += w3.w * z;
  }
  return make_float4(sigmoidf_(acc.x), sigmoidf_(acc.y), sigmoidf_(acc.z), sigmoidf_(acc.w));
}

// Pixel of thread t within a 16 x 16 tile: each warp covers an 8 x 4 block
// (the 8 warps tile 2 x 4 blocks), so that a warp's rays are coherent packets.
__device__ __forceinline__ int serve_px(int t) { return ((t >> 5) & 1) * 8 + (t & 7); }
__device__ __forceinline__ int serve_py(int t) { return (t >> 6) * 4 + ((t >> 3) & 3); }

// The density-cube path kept out of line, so that the march and the diffuse
// lookup do not raise the register pressure of the mesh-object path.
__device__ __noinline__ void serve_march(const CubesDev& c, float lo, float scale, const float* o, const float* d,
                                         int32_t* k, float* t, float* alpha) {
  march_ray(c, lo, scale, o, d, *k, *t, *alpha);
}
__device__ __noinline__ float4 serve_diffuse(const CubesDev& c, const float* x) { return cube_diffuse(c, x); }

// Shared-memory plan of k_serve (dynamic part):
//   [0, serve_wbytes)      FP32 weights of one object (FP32 requests) or its
//                           BF16 operand blob (BF16 requests)
//   A tiles                2 x 128 rows x 64 BF16 (tensor-core operand)
//   rgba of every hit      256 pixels x K float4
//   hit list by object     256 x K u16 (pixel * K + rank)
//   2 mbarriers + TMEM address slot
// The kernel is compiled twice: for scenes of mesh objects only, and for
// scenes that also hold density-cube objects (alpha_c input, d_in up to 49),
// so that the mesh-only loop keeps its lean register and memory plan.
// FP32 weights: (d_in 64 + 64 64 + 64 4) floats, rounded up to 1 KB so the
// A tiles stay 1 KB aligned.
__host__ __device__ constexpr uint32_t serve_wbytes(bool cubes) {
  return (((cubes ? kServeMaxDin : kServeMaxDin - 1) * 64 + 64 * 64 + 64 * 4) * 4 + 1023) / 1024 * 1024;
}
static constexpr uint32_t kServeABytes = 2u * 128u * 64u * 2u;  // 32 768
__host__ __device__ constexpr size_t serve_smem(bool cubes) {
  return serve_wbytes(cubes) + kServeABytes + kServeThreads * kServeMaxK * 16 + kServeThreads * kServeMaxK * 2 + 64;
}

template <bool kCubes>
__global__ void __launch_bounds__(kServeThreads, 2) k_serve(const __grid_constant__ ServeKParams kp) {
  extern __shared__ __align__(1024) uint8_t smem[];
  float4* sWf = reinterpret_cast<float4*>(smem);
  uint8_t* sA = smem + serve_wbytes(kCubes);
  float4* s_rgba = reinterpret_cast<float4*>(sA + kServeABytes);
  uint16_t* s_list = reinterpret_cast<uint16_t*>(s_rgba + kServeThreads * kServeMaxK);
  uint64_t* bars = reinterpret_cast<uint64_t*>(s_list + kServeThreads * kServeMaxK);  // [0] weights, [1] MMA
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2);
  __shared__ int s_cmd;
  __shared__ unsigned long long s_idx;
  __shared__ uint32_t s_slot, s_gen, s_tx, s_ty, s_tiles_total;
  __shared__ int s_W, s_H, s_status, s_skip, s_prec, s_have;
  __shared__ float* s_out;
  __shared__ float s_cam[13];
  __shared__ uint32_t s_cnt[kServeMaxObjects], s_off[kServeMaxObjects + 1];
  __shared__ float s_ht[kServeThreads * kServeMaxK];
  __shared__ float s_ah[kCubes ? kServeThreads * kServeMaxK : 1];  // alpha_c of each hit (density-cube objects)
  __shared__ uint4 s_ring[kServeClaim][2];                           // ring entries of the claimed batch
  __shared__ int s_wcache;  // object (+ 1000 for FP32 weights) whose weights are staged, -1: none
  const int tid = threadIdx.x;
  const unsigned long long t_start = gtimer();
  if (tid == 0) {
    s_have = 0;
    s_slot = 0xFFFFFFFFu;
    s_wcache = -1;
    tc::mbar_init(&bars[0], 1);
    tc::mbar_init(&bars[1], 1);
    tc::fence_mbar_init();
  }
  __syncthreads();
  if (tid < 32) tc::tmem_alloc(tslot, 128);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  uint32_t w_phase = 0, mma_phase = 0;
  bool broken = false;

  unsigned long long batch_next = 0, batch_end = 0;  // tiles claimed but not yet processed (thread 0)
  unsigned long long prof[kProfCount] = {};          // thread 0's phase cycles and counts
  long long clk = clock64();
  auto lap = [&](int phase) {
    if (tid == 0) {
      const long long now = clock64();
      prof[phase] += (unsigned long long)(now - clk);
      clk = now;
    }
  };
  // completion counts not yet published (thread 0): tiles of one request
  // generation finished by this CTA since its last flush
  uint32_t pend_slot = 0, pend_gen = 0, pend_n = 0, pend_total = 0;
  auto flush_done = [&]() {  // thread 0, after a CTA barrier that follows the frame stores
    if (!pend_n) return;
    // bar.sync orders the CTA's frame writes before thread 0's device-scope
    // fence and counter update; the CTA that completes the request observes
    // every other CTA's update and issues the one system-scope fence before
    // the completion record, which makes the whole frame visible to the host
    __threadfence();
    const uint32_t n = atomicAdd(&kp.st->tiles_done[pend_slot], pend_n) + pend_n;
    if (n == pend_total) {
      const int status = atomicExch(&kp.st->status[pend_slot], 0);
      kp.st->tiles_done[pend_slot] = 0;
      __threadfence_system();
      *(volatile int32_t*)&kp.done[pend_slot].status = status;
      st_rel_sys_u32(&kp.done[pend_slot].gen, pend_gen);
    }
    pend_n = 0;
  };
  unsigned long long batch_start = 0;
  while (!broken) {
    // ---- claim a batch of up to kServeClaim published tiles (thread 0), bounded idle wait ----
    if (tid < 32) {
      int fresh = 0;  // a new batch was claimed: warp 0 copies its ring entries
      if (tid == 0) {
        int cmd = 1;
        if (batch_next < batch_end) {
          s_idx = batch_next++;
          cmd = 0;
        }
        while (cmd) {
          if (ld_vol_u32(&kp.ctl->stop)) break;
          const unsigned long long pub = ld_acq_sys_u64(&kp.ctl->published);
          unsigned long long h = *(volatile unsigned long long*)&kp.st->head;
          bool claimed = false;
          while (h < pub) {  // one CAS claims min(kServeClaim, pub - h) consecutive tiles
            const unsigned long long n = min((unsigned long long)kServeClaim, pub - h);
            const unsigned long long prev = atomicCAS(&kp.st->head, h, h + n);
            if (prev == h) {
              s_idx = h;
              batch_start = h;
              batch_next = h + 1;
              batch_end = h + n;
              claimed = true;
              break;
            }
            h = prev;
          }
          if (claimed) {
            cmd = 0;
            fresh = 1;
            atomicMax(&kp.st->last_activity, gtimer());
            break;
          }
          const unsigned long long now = gtimer();
          const unsigned long long last =
              max(*(volatile unsigned long long*)&kp.st->last_activity, t_start);
          if (now > last + kp.idle_limit_ns) break;  // idle: exit, the host relaunches on new work
          __nanosleep(1000);
        }
        s_cmd = cmd;
      }
      // the ring lives in mapped host memory: one round trip for the whole batch
      fresh = __shfl_sync(0xffffffffu, fresh, 0);
      if (fresh) {
        const unsigned long long b0 = __shfl_sync(0xffffffffu, batch_start, 0);
        const unsigned long long nb = __shfl_sync(0xffffffffu, batch_end - batch_start, 0);
        if ((unsigned long long)tid < nb) {
          const ServeTile* e = kp.ring + ((b0 + (unsigned long long)tid) % kp.ring_cap);
          s_ring[tid][0] = ld_vol_v4(e);
          s_ring[tid][1] = ld_vol_v4(reinterpret_cast<const uint4*>(e) + 1);
        }
      }
      __syncwarp();
      if (tid == 0 && s_cmd == 0) {
        const uint4 e0 = s_ring[s_idx - batch_start][0], e1 = s_ring[s_idx - batch_start][1];
        const bool same = e0.x == s_slot && e0.y == s_gen && s_have;  // descriptor cached from the last tile
        s_slot = e0.x;
        s_gen = e0.y;
        s_tx = e0.z;
        s_ty = e0.w;
        s_tiles_total = e1.x;
        const ServeSlot* sl = kp.slots + s_slot;
        int status = 0;
        if (!same) {
          // bounded wait for the request descriptor of this generation
          const unsigned long long t0 = gtimer();
          while (ld_acq_sys_u32(&sl->gen) != s_gen) {
            if (gtimer() - t0 > kp.wait_limit_ns) {
              status = INOLF_E_TIMEOUT;
              break;
            }
            __nanosleep(500);
          }
          if (!status) {
            s_W = (int)ld_vol_u32((const uint32_t*)&sl->W);
            s_H = (int)ld_vol_u32((const uint32_t*)&sl->H);
            s_prec = (int)ld_vol_u32((const uint32_t*)&sl->prec);
            s_out = *(float* const volatile*)&sl->out;
            for (int k = 0; k < 13; ++k) s_cam[k] = ld_vol_f32(&sl->cam[k]);
          }
          s_have = status == 0;
        }
        s_status = status;
        s_skip = status != 0;
        // cancellation is checked every 16 tiles of a request
        if (!status && ((s_idx & 15ull) == 0 || !same) && ld_vol_u32(&sl->cancelled)) {
          s_status = INOLF_E_CANCELLED;
          s_skip = 1;
        }
      }
    }
    if (tid < kServeMaxObjects) s_cnt[tid] = 0;
    __syncthreads();
    lap(kProfClaim);
    if (s_cmd) break;

    // ---- trace every object, keep the K nearest hits of this pixel ----
    float ht[kServeMaxK], ha[kServeMaxK];
    int hk[kServeMaxK];
    int nh = 0;
    const int i = (int)s_tx * kServeTile + serve_px(tid), j = (int)s_ty * kServeTile + serve_py(tid);
    const bool valid = !s_skip && i < s_W && j < s_H;
    float o[3] = {0.f, 0.f, 0.f}, d[3] = {1.f, 1.f, 1.f};
    if (valid) make_ray(s_cam, s_W, s_H, i, j, o, d);
    // every lane runs the object loop: a warp (16 x 2 pixels of the tile)
    // traverses each mesh object's BVH as one packet; density-cube objects
    // are marched ray by ray
    for (int k = 0; k < kp.n_objs; ++k) {
      const ServeObj& ob = kp.objs[k];
      float ol[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) ol[a] = __fsub_rn(o[a], ob.T[a]);
      int32_t id = -1;
      float t = 0.0f, ac = 0.0f;
      if (kCubes && ob.variant) {  // uniform: the density march of this ray (Eq. 4), no warp votes
        if (valid) serve_march(ob.cub, ob.lo, ob.scale, ol, d, &id, &t, &ac);
        if (id < 0) continue;
      } else {
        bool act = valid;
        {  // skip objects whose padded bounding sphere the ray misses
          const float cx = ol[0] - ob.bs_c[0], cy = ol[1] - ob.bs_c[1], cz = ol[2] - ob.bs_c[2];
          const float b = cx * d[0] + cy * d[1] + cz * d[2];
          const float c2 = cx * cx + cy * cy + cz * cz - ob.bs_r2;
          if (c2 > 0.f && (b > 0.f || b * b < c2)) act = false;
        }
        if (!__any_sync(0xffffffffu, act)) continue;
        closest_hit_packet_s<false, 8>(ob.nodes, ob.tris, &kp.st->err, act, ol, d, id, t, nullptr, nullptr);
        if (!act || id < 0) continue;
      }
      {
        // insert (t, k) into the sorted list (ties by object id: k increases)
        int pos = nh < kp.K ? nh : kp.K;
        while (pos > 0 && ht[pos - 1] > t) {
          if (pos < kp.K) {
            ht[pos] = ht[pos - 1];
            hk[pos] = hk[pos - 1];
            if (kCubes) ha[pos] = ha[pos - 1];
          }
          --pos;
        }
        if (pos < kp.K) {
          ht[pos] = t;
          hk[pos] = k;
          if (kCubes) ha[pos] = ac;
          if (nh < kp.K) ++nh;
        }
      }
    }
    // group the tile's hits by object: rank within the object's list
    uint32_t rank[kServeMaxK];
    for (int q = 0; q < nh; ++q) {
      rank[q] = atomicAdd(&s_cnt[hk[q]], 1u);
      s_ht[tid * kServeMaxK + q] = ht[q];
      if (kCubes) s_ah[tid * kServeMaxK + q] = ha[q];
    }
    __syncthreads();
    if (tid == 0) {
      uint32_t acc = 0;
      for (int k = 0; k < kServeMaxObjects; ++k) { s_off[k] = acc; acc += s_cnt[k]; }
      s_off[kServeMaxObjects] = acc;
    }
    __syncthreads();
    for (int q = 0; q < nh; ++q) s_list[s_off[hk[q]] + rank[q]] = (uint16_t)(tid * kServeMaxK + q);
    __syncthreads();

    lap(kProfTrace);
    if (tid == 0) {
      prof[kProfTiles] += 1;
      prof[kProfHits] += s_off[kServeMaxObjects];
    }
    // ---- shade the hits object by object ----
    for (int k = 0; k < kp.n_objs && !broken; ++k) {
      const uint32_t cnt = s_cnt[k];
      if (!cnt) continue;  // uniform: no pixel of the tile hits object k
      const ServeObj& ob = kp.objs[k];
      const int din = ob.d_in;
      if (s_prec == INOLF_FP32) {
        // the object's FP32 weights, unless they are still staged from the last pass
        const bool need = s_wcache != 1000 + k;
        const int nw4 = (din * 64 + 64 * 64 + 64 * 4) / 4;
        if (tid == 0) {
          prof[kProfWeightLoads] += need ? 1 : 0;
          prof[kProfBatches] += 1;
        }
        if (need)
          for (int q = tid; q < nw4; q += kServeThreads) sWf[q] = reinterpret_cast<const float4*>(ob.w_f32)[q];
        __syncthreads();
        if (tid == 0 && need) s_wcache = 1000 + k;
        for (int q = 0; q < nh; ++q) {
          if (hk[q] != k) continue;
          float ol[3], x3[3];
#pragma unroll
          for (int a = 0; a < 3; ++a) ol[a] = __fsub_rn(o[a], ob.T[a]);
          hit_unit_coords_ls(ob.lo, ob.scale, ol, d, ht[q], x3);
          float x[kCubes ? kServeMaxDin : kServeMaxDin - 1];
          {
            LevelFetchB fa, fb;
            fetch_bundle_phi(ob.lv[0], x3, fa);
            for (int l = 0; l < ob.L; l += 2) {  // levels in pairs, the next level's Phi entry in flight
              if (l + 1 < ob.L) fetch_bundle_phi(ob.lv[l + 1], x3, fb);
              finish_bundle(ob.lv[l], ob.fp16, fa, x[2 * l], x[2 * l + 1]);
              if (l + 1 >= ob.L) break;
              if (l + 2 < ob.L) fetch_bundle_phi(ob.lv[l + 2], x3, fa);
              finish_bundle(ob.lv[l + 1], ob.fp16, fb, x[2 * l + 2], x[2 * l + 3]);
            }
          }
          sh16c(kp.shc, d, x + 2 * ob.L);
          if (kCubes && ob.variant) x[2 * ob.L + 16] = ha[q];  // alpha_c (Eq. 5)
          float4 c = mlp_f32(sWf, sWf + din * 16, sWf + din * 16 + 64 * 16, x, din);
          if (kCubes && ob.variant) {  // c = c_d + tint c_s (Eq. 7)
            const float4 dc = serve_diffuse(ob.cub, x3);
            c = make_float4(fmaf(dc.w, c.x, dc.x), fmaf(dc.w, c.y, dc.y), fmaf(dc.w, c.z, dc.z), c.w);
          }
          s_rgba[tid * kServeMaxK + q] = c;
        }
        __syncthreads();
      } else {
        // BF16 tensor-core MLP: stage the object's operand blob by one bulk copy,
        // unless it is still staged from the last pass
        const uint32_t K1 = (uint32_t)ob.tc_k1_bf16, chunks1 = K1 / 8u;
        const bool need = s_wcache != k;
        bool okw = true;
        if (need) {
          if (tid == 0) {
            tc::fence_async_smem();  // after generic writes (FP32 weights) to the same bytes
            tc::mbar_arrive_expect_tx(&bars[0], ob.tc_bytes_bf16);
            tc::bulk_g2s(smem, ob.w_bf16, ob.tc_bytes_bf16, &bars[0]);
            prof[kProfWeightLoads] += 1;
          }
          okw = tc::mbar_wait(&bars[0], w_phase, kWaitLimitNs);
          w_phase ^= 1u;
        }
        if (__syncthreads_or(!okw)) { broken = true; break; }
        if (tid == 0 && need) s_wcache = k;
        const uint8_t* sB1 = smem;
        const uint8_t* sB2 = smem + 64u * K1 * 2u;
        const uint8_t* sB3 = sB2 + 64u * 64u * 2u;  // W3 as a 16-row operand
        const uint32_t t = (uint32_t)tid >> 7, row = (uint32_t)tid & 127u;
        uint8_t* A = sA + t * (128u * 64u * 2u);
        for (uint32_t base = 0; base < cnt; base += kServeThreads) {
          const bool mine = base + (uint32_t)tid < cnt;
          uint32_t entry = 0;
          if (mine) {
            entry = s_list[s_off[k] + base + tid];
            const int p = (int)(entry / kServeMaxK);
            const float th = s_ht[entry];
            const int pi = (int)s_tx * kServeTile + serve_px(p), pj = (int)s_ty * kServeTile + serve_py(p);
            float po[3], pd[3], ol[3], x3[3];
            make_ray(s_cam, s_W, s_H, pi, pj, po, pd);
#pragma unroll
            for (int a = 0; a < 3; ++a) ol[a] = __fsub_rn(po[a], ob.T[a]);
            hit_unit_coords_ls(ob.lo, ob.scale, ol, pd, th, x3);
            {
              LevelFetchB fa, fb;
              fetch_bundle_phi(ob.lv[0], x3, fa);
              for (int l = 0; l < ob.L; l += 2) {  // levels in pairs, the next level's Phi entry in flight
                float e0, e1;
                if (l + 1 < ob.L) fetch_bundle_phi(ob.lv[l + 1], x3, fb);
                finish_bundle(ob.lv[l], ob.fp16, fa, e0, e1);
                store_pair<false>(A, row, 2u * l, chunks1, e0, e1, 1.f);
                if (l + 1 >= ob.L) break;
                if (l + 2 < ob.L) fetch_bundle_phi(ob.lv[l + 2], x3, fa);
                finish_bundle(ob.lv[l + 1], ob.fp16, fb, e0, e1);
                store_pair<false>(A, row, 2u * (l + 1), chunks1, e0, e1, 1.f);
              }
            }
            float sh[16];
            sh16c(kp.shc, pd, sh);
#pragma unroll
            for (int u = 0; u < 8; ++u) store_pair<false>(A, row, 2u * ob.L + 2u * u, chunks1, sh[2 * u], sh[2 * u + 1], 1.f);
            uint32_t k0 = 2u * ob.L + 16u;
            if (kCubes && ob.variant) {  // alpha_c (Eq. 5)
              store_pair<false>(A, row, k0, chunks1, s_ah[entry], 0.f, 1.f);
              k0 += 2u;
            }
            for (uint32_t kk = k0; kk < K1; kk += 2) store_pair<false>(A, row, kk, chunks1, 0.f, 0.f, 1.f);
          } else {
            for (uint32_t c = 0; c < chunks1; ++c)
              *reinterpret_cast<uint4*>(A + tc::core_off(row, c, chunks1)) = make_uint4(0, 0, 0, 0);
          }
          float4 rgba;
          const TcScales sc = TcScales::make(false, nullptr, nullptr);
          if (tid == 0) prof[kProfBatches] += 1;
          if (!tc_mlp_run<false>(sA, sB1, sB2, sB3, K1, tmem, &bars[1], mma_phase, sc, rgba)) {
            broken = true;
            break;
          }
          if (mine) {
            if (kCubes && ob.variant) {  // c = c_d + tint c_s (Eq. 7), diffuse read at the hit point
              const int p = (int)(entry / kServeMaxK);
              const int pi = (int)s_tx * kServeTile + serve_px(p), pj = (int)s_ty * kServeTile + serve_py(p);
              float po[3], pd[3], ol[3], x3[3];
              make_ray(s_cam, s_W, s_H, pi, pj, po, pd);
#pragma unroll
              for (int a = 0; a < 3; ++a) ol[a] = __fsub_rn(po[a], ob.T[a]);
              hit_unit_coords_ls(ob.lo, ob.scale, ol, pd, s_ht[entry], x3);
              const float4 dc = serve_diffuse(ob.cub, x3);
              rgba = make_float4(fmaf(dc.w, rgba.x, dc.x), fmaf(dc.w, rgba.y, dc.y), fmaf(dc.w, rgba.z, dc.z), rgba.w);
            }
            s_rgba[entry] = rgba;
          }
        }
      }
    }
    __syncthreads();

    lap(kProfShade);
    // ---- composite front to back, straight alpha out ----
    if (valid && !broken) {
      float C0 = 0.f, C1 = 0.f, C2 = 0.f, A = 0.f;
      for (int q = 0; q < nh; ++q) {
        const float4 c = s_rgba[tid * kServeMaxK + q];
        const float w = (1.0f - A) * c.w;
        C0 += w * c.x;
        C1 += w * c.y;
        C2 += w * c.z;
        A += w;
      }
      const float4 px = A > 0.f ? make_float4(C0 / A, C1 / A, C2 / A, A) : make_float4(0.f, 0.f, 0.f, 0.f);
      reinterpret_cast<float4*>(s_out)[(size_t)j * s_W + i] = px;
    }
    __syncthreads();
    lap(kProfComposite);
    // ---- tile done: its count joins this CTA's pending completions, which are
    // published (one fence) when the next tile belongs to another request or
    // the claimed batch is used up; the last tile of a request publishes it ----
    if (tid == 0) {
      const uint32_t slot = s_slot;
      const int st = broken ? INOLF_E_TIMEOUT : s_status;
      if (broken) atomicOr(&kp.st->err, 4u);
      if (st) atomicCAS(&kp.st->status[slot], 0, st);
      if (pend_n && (pend_slot != slot || pend_gen != s_gen)) flush_done();
      pend_slot = slot;
      pend_gen = s_gen;
      pend_total = s_tiles_total;
      ++pend_n;
      bool keep = !broken && batch_next < batch_end;
      if (keep) {
        const uint4 nx = s_ring[batch_next - batch_start][0];
        keep = nx.x == slot && nx.y == s_gen;
      }
      if (!keep) flush_done();
    }
    __syncthreads();
    lap(kProfDone);
  }
  if (tid == 0) {
    flush_done();  // normally nothing is pending here
    for (int k = 0; k < kProfCount; ++k)
      if (prof[k]) atomicAdd(&kp.st->prof[k], prof[k]);
  }
  if (broken) {  // let tensor-core work still in flight finish before freeing TMEM
    tc::mbar_wait(&bars[1], mma_phase ^ 1u, kWaitLimitNs);
  }
  __syncthreads();
  if (tid < 32) {
    tc::fence_after();
    tc::tmem_dealloc(tmem, 128);
  }
}

}  // namespace inolf

// ===========================================================================
// host side
// ===========================================================================
using namespace inolf;

namespace {

using Clock = std::chrono::steady_clock;

struct SlotMeta {
  bool busy = false;
  bool published = false;
  bool done_seen = false;
  uint64_t ticket = 0;
  uint32_t gen = 0;
  size_t off = 0, bytes = 0;
  int W = 0, H = 0;
  Clock::time_point submitted;
  int64_t latency_ns = 0;
  int32_t status = 0;
};

}  // namespace

struct inolf_server {
  std::mutex mu;
  int device = 0;
  inolf_serve_params prm{};
  cudaStream_t stream = nullptr;
  cudaEvent_t kernel_done = nullptr;
  bool launched = false;
  int occ_diag[4] = {0, 0, 0, 0};  // mesh-only kernel: registers, static / dynamic shared bytes, CTAs per SM
  int grid = 0;        // persistent CTAs of the mesh-only kernel
  int grid_cubes = 0;  // and of the kernel that also serves density-cube objects
  // objects
  std::vector<ServeObj> objs;
  ServeObj* d_objs = nullptr;
  bool objs_dirty = true;
  // mapped host memory
  ServeCtl* h_ctl = nullptr;
  ServeCtl* d_ctl = nullptr;
  ServeDone* h_done = nullptr;
  ServeDone* d_done = nullptr;
  ServeSlot* h_slots = nullptr;
  ServeSlot* d_slots = nullptr;
  ServeTile* h_ring = nullptr;
  ServeTile* d_ring = nullptr;
  unsigned long long ring_cap = 0;
  unsigned long long published = 0;
  // device state and frame arena
  ServeDevState* d_st = nullptr;
  uint8_t* arena = nullptr;
  std::map<size_t, size_t> free_blocks;  // offset -> size
  std::vector<SlotMeta> slots;
  std::vector<uint32_t> slot_gen;  // last generation issued per slot
  std::map<uint64_t, int> by_ticket;
  uint64_t next_ticket = 1;
  // scheduling (policy 1: Algorithm 1) and the host dispatcher thread
  inolf_sched* sched = nullptr;
  std::thread loop;
  std::atomic<bool> quit{false};
  int64_t n_admitted = 0, n_refused = 0, n_denied = 0, n_completed = 0;
};

static int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count();
}

static bool arena_alloc(inolf_server* s, size_t bytes, size_t* off) {
  for (auto it = s->free_blocks.begin(); it != s->free_blocks.end(); ++it) {
    if (it->second >= bytes) {
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t noff = it->first + bytes;
      s->free_blocks.erase(it);
      if (rest) s->free_blocks[noff] = rest;
      return true;
    }
  }
  return false;
}

static void arena_free(inolf_server* s, size_t off, size_t bytes) {
  auto it = s->free_blocks.emplace(off, bytes).first;
  auto nx = std::next(it);
  if (nx != s->free_blocks.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    s->free_blocks.erase(nx);
  }
  if (it != s->free_blocks.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      s->free_blocks.erase(it);
    }
  }
}

static void serve_free(inolf_server* s) {
  s->quit = true;
  if (s->loop.joinable()) s->loop.join();
  if (s->sched) inolf_sched_destroy(s->sched);
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->kernel_done) cudaEventDestroy(s->kernel_done);
  if (s->stream) cudaStreamDestroy(s->stream);
  if (s->h_ctl) cudaFreeHost(s->h_ctl);
  if (s->h_done) cudaFreeHost(s->h_done);
  if (s->h_slots) cudaFreeHost(s->h_slots);
  if (s->h_ring) cudaFreeHost(s->h_ring);
  if (s->d_st) cudaFree(s->d_st);
  if (s->d_objs) cudaFree(s->d_objs);
  if (s->arena) cudaFree(s->arena);
  delete s;
}

static bool scene_has_cubes(const inolf_server* s) {
  for (const ServeObj& o : s->objs)
    if (o.variant) return true;
  return false;
}

// Launches the persistent kernel if it is not running (must hold s->mu).
static inolf_status ensure_running(inolf_server* s) {
  if (s->launched) {
    const cudaError_t q = cudaEventQuery(s->kernel_done);
    if (q == cudaErrorNotReady) return INOLF_OK;
    if (q != cudaSuccess) return fail(INOLF_E_CUDA, std::string("serve kernel: ") + cudaGetErrorString(q));
    s->launched = false;
  }
  if (s->objs_dirty) {
    if (cudaMemcpyAsync(s->d_objs, s->objs.data(), sizeof(ServeObj) * s->objs.size(), cudaMemcpyHostToDevice,
                        s->stream) != cudaSuccess)
      return fail(INOLF_E_CUDA, "serve: object table upload failed");
    s->objs_dirty = false;
  }
  ServeKParams kp{};
  kp.objs = s->d_objs;
  kp.n_objs = (int32_t)s->objs.size();
  kp.K = s->prm.max_hits;
  kp.ctl = s->d_ctl;
  kp.done = s->d_done;
  kp.slots = s->d_slots;
  kp.ring = s->d_ring;
  kp.ring_cap = s->ring_cap;
  kp.st = s->d_st;
  kp.wait_limit_ns = (unsigned long long)s->prm.wait_limit_ns;
  kp.idle_limit_ns = (unsigned long long)s->prm.idle_limit_ns;
  sh_constants(kp.shc);
  {
    LaunchTimer lt("k_serve", s->stream);
    if (scene_has_cubes(s))
      k_serve<true><<<s->grid_cubes, kServeThreads, serve_smem(true), s->stream>>>(kp);
    else
      k_serve<false><<<s->grid, kServeThreads, serve_smem(false), s->stream>>>(kp);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(INOLF_E_CUDA, std::string("k_serve launch: ") + cudaGetErrorString(e));
  cudaEventRecord(s->kernel_done, s->stream);
  s->launched = true;
  return INOLF_OK;
}

// Publishes the tiles of an admitted request to the device ring (must hold s->mu).
static inolf_status publish_locked(inolf_server* s, int slot) {
  SlotMeta& m = s->slots[slot];
  const uint32_t tx = (uint32_t)((m.W + kServeTile - 1) / kServeTile);
  const uint32_t ty = (uint32_t)((m.H + kServeTile - 1) / kServeTile);
  for (uint32_t y = 0; y < ty; ++y)
    for (uint32_t x = 0; x < tx; ++x) {
      ServeTile& e = s->h_ring[(s->published + (unsigned long long)y * tx + x) % s->ring_cap];
      e.slot = (uint32_t)slot;
      e.gen = m.gen;
      e.tx = x;
      e.ty = y;
      e.tiles_total = tx * ty;
    }
  s->published += (unsigned long long)tx * ty;
  __atomic_store_n(&s->h_ctl->published, s->published, __ATOMIC_RELEASE);
  m.published = true;
  return ensure_running(s);
}

// Records the requests the device has completed (must hold s->mu).
static void completions_locked(inolf_server* s) {
  const int64_t t = now_ns();
  for (int k = 0; k < (int)s->slots.size(); ++k) {
    SlotMeta& m = s->slots[k];
    if (!m.busy || !m.published || m.done_seen) continue;
    if (__atomic_load_n(&s->h_done[k].gen, __ATOMIC_ACQUIRE) != m.gen) continue;
    m.done_seen = true;
    m.status = __atomic_load_n(&s->h_done[k].status, __ATOMIC_ACQUIRE);
    m.latency_ns = std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - m.submitted).count();
    ++s->n_completed;
    if (s->sched) inolf_sched_complete(s->sched, m.ticket, t);
  }
}

// Dispatches admitted requests in the policy's order (must hold s->mu).
static inolf_status dispatch_locked(inolf_server* s) {
  if (!s->sched) return INOLF_OK;
  uint64_t id = 0;
  while (inolf_sched_next(s->sched, now_ns(), &id) == INOLF_OK) {
    auto it = s->by_ticket.find(id);
    if (it == s->by_ticket.end()) continue;
    const inolf_status st = publish_locked(s, it->second);
    if (st != INOLF_OK) return st;
  }
  return INOLF_OK;
}

// The host side of the request loop: observes completions, dispatches
// queued requests and relaunches the persistent kernel when it went idle
// with work outstanding.
static void dispatcher(inolf_server* s) {
  while (!s->quit) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      completions_locked(s);
      dispatch_locked(s);
      bool outstanding = false;
      for (auto& m : s->slots) outstanding |= m.busy && m.published && !m.done_seen;
      if (outstanding) ensure_running(s);
    }
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

extern "C" inolf_status inolf_serve_create(const inolf_serve_params* prm, inolf_server** out) {
  clear_error();
  if (!out) return fail(INOLF_E_INVALID, "inolf_serve_create: out is NULL");
  *out = nullptr;
  inolf_serve_params p{};
  p.hbm_budget = (size_t)4 << 30;
  p.max_slots = 48;
  p.max_width = 3840;
  p.max_height = 2160;
  p.max_hits = 4;
  p.wait_limit_ns = 1000000000;
  p.idle_limit_ns = 20000000;
  p.ctas_per_sm = 0;
  p.policy = 0;
  p.max_rays_in_flight = 0;
  if (prm) p = *prm;
  if (p.hbm_budget < 4096 || p.max_slots < 1 || p.max_slots > kServeMaxSlots || p.max_width < 1 ||
      p.max_height < 1 || p.max_width > 16384 || p.max_height > 16384 || p.max_hits < 1 ||
      p.max_hits > kServeMaxK || p.wait_limit_ns <= 0 || p.idle_limit_ns <= 0 || p.ctas_per_sm < 0 ||
      p.policy < 0 || p.policy > 1 || p.max_rays_in_flight < 0)
    return fail(INOLF_E_INVALID, "inolf_serve_create: bad parameters");
  inolf_server* s = new (std::nothrow) inolf_server();
  if (!s) return fail(INOLF_E_OOM, "inolf_serve_create: oom");
  s->prm = p;
  cudaGetDevice(&s->device);
  const unsigned long long tiles_max = (unsigned long long)((p.max_width + kServeTile - 1) / kServeTile) *
                                       ((p.max_height + kServeTile - 1) / kServeTile);
  s->ring_cap = tiles_max * (unsigned long long)p.max_slots;
  auto bad = [&](const char* what) {
    serve_free(s);
    return fail(INOLF_E_OOM, std::string("inolf_serve_create: ") + what);
  };
  if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) return bad("stream");
  if (cudaEventCreateWithFlags(&s->kernel_done, cudaEventDisableTiming) != cudaSuccess) return bad("event");
  const unsigned fl = cudaHostAllocMapped | cudaHostAllocPortable;
  if (cudaHostAlloc((void**)&s->h_ctl, sizeof(ServeCtl), fl) != cudaSuccess) return bad("control block");
  if (cudaHostAlloc((void**)&s->h_done, sizeof(ServeDone) * p.max_slots, fl) != cudaSuccess) return bad("done");
  if (cudaHostAlloc((void**)&s->h_slots, sizeof(ServeSlot) * p.max_slots, fl) != cudaSuccess) return bad("slots");
  if (cudaHostAlloc((void**)&s->h_ring, sizeof(ServeTile) * s->ring_cap, fl) != cudaSuccess) return bad("ring");
  std::memset(s->h_ctl, 0, sizeof(ServeCtl));
  std::memset(s->h_done, 0, sizeof(ServeDone) * p.max_slots);
  std::memset(s->h_slots, 0, sizeof(ServeSlot) * p.max_slots);
  if (cudaHostGetDevicePointer((void**)&s->d_ctl, s->h_ctl, 0) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&s->d_done, s->h_done, 0) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&s->d_slots, s->h_slots, 0) != cudaSuccess ||
      cudaHostGetDevicePointer((void**)&s->d_ring, s->h_ring, 0) != cudaSuccess)
    return bad("mapped pointers");
  if (cudaMalloc(&s->d_st, sizeof(ServeDevState)) != cudaSuccess) return bad("device state");
  if (cudaMemset(s->d_st, 0, sizeof(ServeDevState)) != cudaSuccess) return bad("device state");
  if (cudaMalloc(&s->d_objs, sizeof(ServeObj) * kServeMaxObjects) != cudaSuccess) return bad("object table");
  if (cudaMalloc(&s->arena, p.hbm_budget) != cudaSuccess) return bad("frame arena (HBM budget)");
  s->free_blocks[0] = p.hbm_budget;
  s->slots.resize(p.max_slots);
  s->slot_gen.assign(p.max_slots, 0);
  int sms = 1, regs_sm = 65536, smem_sm = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, s->device);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, s->device);
  // resident CTAs per SM from the kernel's registers, shared memory and tensor
  // memory (the occupancy query reports one CTA for this tensor-memory kernel;
  // a CTA that does not fit only starts when another exits, and no CTA waits
  // on another, so an over-estimate is harmless)
  auto grid_of = [&](const void* fn, size_t smem) {
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, fn);
    const int regs_warp = ((std::max(fa.numRegs, 1) * 32 + 255) / 256) * 256;  // allocated per warp in units of 256
    const int by_regs = regs_sm / (regs_warp * (kServeThreads / 32));
    const int by_smem = (int)(smem_sm / (smem + fa.sharedSizeBytes + 1024));
    int occ = std::max(1, std::min(std::min(by_regs, by_smem), 4));  // each CTA holds 128 of 512 TMEM columns
    if (p.ctas_per_sm > 0) occ = std::min(occ, p.ctas_per_sm);
    return sms * occ;
  };
  s->grid = grid_of((const void*)k_serve<false>, serve_smem(false));
  {
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, (const void*)k_serve<false>);
    s->occ_diag[0] = fa.numRegs;
    s->occ_diag[1] = (int)fa.sharedSizeBytes;
    s->occ_diag[2] = (int)serve_smem(false);
    s->occ_diag[3] = s->grid / std::max(1, sms);
  }
  s->grid_cubes = grid_of((const void*)k_serve<true>, serve_smem(true));
  cudaGetLastError();
  if (p.policy == 1 && inolf_sched_create(p.max_rays_in_flight, &s->sched) != INOLF_OK) return bad("scheduler");
  s->loop = std::thread(dispatcher, s);
  *out = s;
  return INOLF_OK;
}

extern "C" inolf_status inolf_serve_set_viewer(inolf_server* s, uint32_t viewer_id, double target_fps) {
  clear_error();
  if (!s || !(target_fps > 0)) return fail(INOLF_E_INVALID, "inolf_serve_set_viewer: bad argument");
  std::lock_guard<std::mutex> lk(s->mu);
  if (!s->sched) return INOLF_OK;  // policy 0 ignores target rates
  return inolf_sched_set_viewer(s->sched, viewer_id, target_fps, now_ns());
}

extern "C" inolf_status inolf_serve_counters(inolf_server* s, int64_t* admitted, int64_t* refused, int64_t* denied,
                                             int64_t* completed) {
  clear_error();
  if (!s) return fail(INOLF_E_INVALID, "inolf_serve_counters: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  if (admitted) *admitted = s->n_admitted;
  if (refused) *refused = s->n_refused;
  if (denied) *denied = s->n_denied;
  if (completed) *completed = s->n_completed;
  return INOLF_OK;
}

extern "C" inolf_status inolf_serve_profile(inolf_server* s, int64_t* out, int32_t reset) {
  clear_error();
  if (!s || !out) return fail(INOLF_E_INVALID, "inolf_serve_profile: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  // the persistent CTAs add their counters when they exit: wait until the
  // kernel has gone idle and returned
  if (s->launched && cudaEventSynchronize(s->kernel_done) != cudaSuccess)
    return fail(INOLF_E_CUDA, "inolf_serve_profile: waiting for the kernel failed");
  unsigned long long v[kProfCount];
  if (cudaMemcpy(v, s->d_st->prof, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(INOLF_E_CUDA, "inolf_serve_profile: read failed");
  for (int k = 0; k < kProfCount; ++k) out[k] = (int64_t)v[k];
  out[kProfCount] = scene_has_cubes(s) ? s->grid_cubes : s->grid;  // persistent CTAs per launch
  for (int k = 0; k < 4; ++k) out[kProfCount + 1 + k] = s->occ_diag[k];
  if (reset && cudaMemset(s->d_st->prof, 0, sizeof(v)) != cudaSuccess)
    return fail(INOLF_E_CUDA, "inolf_serve_profile: reset failed");
  return INOLF_OK;
}

extern "C" inolf_status inolf_serve_add_object(inolf_server* s, const inolf_object* obj, const float translation[3]) {
  clear_error();
  if (!s || !obj || !translation) return fail(INOLF_E_INVALID, "inolf_serve_add_object: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  for (auto& m : s->slots)
    if (m.busy) return fail(INOLF_E_INVALID, "inolf_serve_add_object: requests are in flight");
  if ((int)s->objs.size() >= kServeMaxObjects) return fail(INOLF_E_INVALID, "inolf_serve_add_object: 16 objects max");
  const Object& o = obj->o;
  ServeObj so{};
  so.nodes = (const float4*)o.nodes;
  so.tris = (const float4*)o.tris;
  so.w_f32 = o.w_f32;
  so.w_bf16 = o.w_bf16;
  so.tc_k1_bf16 = o.tc_k1_bf16;
  so.tc_bytes_bf16 = o.tc_bytes_bf16;
  so.L = o.L;
  so.fp16 = o.fp16;
  so.d_in = o.d_in;
  so.lo = o.lo;
  so.scale = o.scale;
  for (int k = 0; k < 3; ++k) so.T[k] = translation[k];
  for (int k = 0; k < 3; ++k) so.bs_c[k] = o.bsphere[k];
  so.bs_r2 = o.bsphere[3] * o.bsphere[3];
  for (int l = 0; l < o.L; ++l) so.lv[l] = o.lv[l];
  so.variant = o.variant;
  so.cub = o.cub;
  s->objs.push_back(so);
  s->objs_dirty = true;
  return INOLF_OK;
}

extern "C" inolf_status inolf_serve_submit(inolf_server* s, const inolf_request* r, uint64_t* ticket) {
  clear_error();
  if (!s || !r || !ticket) return fail(INOLF_E_INVALID, "inolf_serve_submit: NULL argument");
  if (r->width < 1 || r->height < 1 || r->width > s->prm.max_width || r->height > s->prm.max_height)
    return fail(INOLF_E_INVALID, "inolf_serve_submit: resolution outside (0, max]");
  if (r->precision != INOLF_FP32 && r->precision != INOLF_BF16)
    return fail(INOLF_E_UNSUPPORTED, "inolf_serve_submit: FP32 and BF16 shading are served");
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->objs.empty()) return fail(INOLF_E_INVALID, "inolf_serve_submit: no objects");
  int slot = -1;
  for (int k = 0; k < (int)s->slots.size(); ++k)
    if (!s->slots[k].busy) { slot = k; break; }
  if (slot < 0) {
    ++s->n_refused;
    return fail(INOLF_E_BUDGET, "inolf_serve_submit: all request slots are in use");
  }
  const size_t bytes = ((size_t)r->width * r->height * 16 + 255) & ~(size_t)255;
  size_t off = 0;
  if (!arena_alloc(s, bytes, &off)) {
    ++s->n_refused;
    return fail(INOLF_E_BUDGET, "inolf_serve_submit: HBM budget exhausted");
  }
  const uint64_t tk = s->next_ticket++;
  if (s->sched) {
    const inolf_status a = inolf_sched_admit(s->sched, r->viewer_id, tk, (int64_t)r->width * r->height, now_ns());
    if (a != INOLF_OK) {
      arena_free(s, off, bytes);
      ++s->n_denied;
      return a;  // INOLF_E_BUDGET in the starvation state
    }
  }
  ++s->n_admitted;
  SlotMeta& m = s->slots[slot];
  m = SlotMeta();
  m.busy = true;
  m.ticket = tk;
  m.gen = ++s->slot_gen[slot];
  if (m.gen == 0) m.gen = s->slot_gen[slot] = 1;
  m.off = off;
  m.bytes = bytes;
  m.W = r->width;
  m.H = r->height;
  m.submitted = Clock::now();
  s->by_ticket[m.ticket] = slot;
  const uint32_t tx = (uint32_t)((r->width + kServeTile - 1) / kServeTile);
  const uint32_t ty = (uint32_t)((r->height + kServeTile - 1) / kServeTile);
  ServeSlot& hs = s->h_slots[slot];
  hs.W = r->width;
  hs.H = r->height;
  hs.prec = r->precision;
  hs.out = reinterpret_cast<float*>(s->arena + off);
  std::memcpy(hs.cam, r->camera, sizeof(hs.cam));
  hs.tiles_x = tx;
  hs.tiles_total = tx * ty;
  __atomic_store_n(&hs.cancelled, 0u, __ATOMIC_RELAXED);
  // the generation is written last: the device reads the descriptor once it
  // sees this generation (the test-only flag leaves it out)
  if (!(r->flags & INOLF_REQ_TEST_DROP_DESCRIPTOR)) __atomic_store_n(&hs.gen, m.gen, __ATOMIC_RELEASE);
  *ticket = m.ticket;
  if (!s->sched) return publish_locked(s, slot);  // policy 0: arrival order
  return dispatch_locked(s);
}

extern "C" inolf_status inolf_serve_poll(inolf_server* s, uint64_t ticket, inolf_result* res) {
  clear_error();
  if (!s) return fail(INOLF_E_INVALID, "inolf_serve_poll: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->by_ticket.find(ticket);
  if (it == s->by_ticket.end()) return fail(INOLF_E_UNKNOWN_TICKET, "inolf_serve_poll: unknown ticket");
  SlotMeta& m = s->slots[it->second];
  if (!m.done_seen) {
    completions_locked(s);
    if (!m.done_seen) {
      inolf_status e = dispatch_locked(s);
      if (e == INOLF_OK && m.published) e = ensure_running(s);  // relaunch if the kernel went idle
      return e != INOLF_OK ? e : INOLF_PENDING;
    }
  }
  if (res) {
    res->frame = reinterpret_cast<const float*>(s->arena + m.off);
    res->width = m.W;
    res->height = m.H;
    res->latency_ns = m.latency_ns;
    res->rays = (int64_t)m.W * m.H;
  }
  if (m.status == INOLF_E_TIMEOUT) return fail(INOLF_E_TIMEOUT, "request descriptor did not arrive in time");
  if (m.status == INOLF_E_CANCELLED) return fail(INOLF_E_CANCELLED, "request cancelled");
  return INOLF_OK;
}

extern "C" inolf_status inolf_serve_cancel(inolf_server* s, uint64_t ticket) {
  clear_error();
  if (!s) return fail(INOLF_E_INVALID, "inolf_serve_cancel: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->by_ticket.find(ticket);
  if (it == s->by_ticket.end()) return fail(INOLF_E_UNKNOWN_TICKET, "inolf_serve_cancel: unknown ticket");
  SlotMeta& m = s->slots[it->second];
  if (!m.published && s->sched && inolf_sched_cancel(s->sched, ticket) == INOLF_OK) {
    m.done_seen = true;  // never reached the device
    m.status = INOLF_E_CANCELLED;
    m.latency_ns = std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - m.submitted).count();
    return INOLF_OK;
  }
  __atomic_store_n(&s->h_slots[it->second].cancelled, 1u, __ATOMIC_RELEASE);
  return INOLF_OK;
}

extern "C" inolf_status inolf_serve_release(inolf_server* s, uint64_t ticket) {
  clear_error();
  if (!s) return fail(INOLF_E_INVALID, "inolf_serve_release: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->by_ticket.find(ticket);
  if (it == s->by_ticket.end()) return fail(INOLF_E_UNKNOWN_TICKET, "inolf_serve_release: unknown ticket");
  SlotMeta& m = s->slots[it->second];
  if (!m.done_seen) return fail(INOLF_E_INVALID, "inolf_serve_release: request not complete (poll first)");
  arena_free(s, m.off, m.bytes);
  m.busy = false;
  s->by_ticket.erase(it);
  return INOLF_OK;
}

extern "C" inolf_status inolf_serve_destroy(inolf_server* s) {
  clear_error();
  if (!s) return INOLF_OK;
  s->quit = true;
  if (s->loop.joinable()) s->loop.join();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    __atomic_store_n(&s->h_ctl->stop, 1u, __ATOMIC_RELEASE);
  }
  serve_free(s);
  return INOLF_OK;
}
