// Internal declarations shared by the translation units of libinolf.so.
#pragma once

#include <cstdint>
#include <cstddef>
#include <string>

#include <vector_types.h>

#include "../../include/inolf.h"

namespace inolf {

// Thread-local error message + status helper.
inolf_status fail(inolf_status st, const std::string& msg);
void clear_error();

// The library may run on several devices of one process; kernel attributes
// and grid sizes are set up once per device (index < kMaxDevices), with that
// device current.  device_index() returns the current device, or -1 when it
// cannot be read or lies beyond kMaxDevices.
static constexpr int kMaxDevices = 64;
int device_index();

// Failure flags of a call (word 1 of the workspace header, INOLF_FLAG_*):
// synchronises `stream`, reads the word and turns it into a status (message
// prefixed by `what`).  ws = NULL reads the allocation-free scratch.
inolf_status read_device_flags(const void* ws, void* stream, uint32_t* flags);
inolf_status flags_status(uint32_t flags, const char* what);
// Device address of the allocation-free scratch on the current device
// (render_noalloc.cu).
inolf_status noalloc_scratch_address(void** out);

// Per-level encoder description as the kernels see it.
struct LevelDev {
  int32_t N;              // cells per axis
  int32_t m;              // hash-table side
  int32_t r;              // offset-table side
  float N_f;              // (float)N
  uint32_t magic_m;       // ceil(2^32 / m) (2^32 - 1 for m = 1): a mod m by one high multiply
  uint32_t magic_r;       // the same for r
  const uint32_t* phi;    // r^3 packed offsets
  const void* table;      // m^3 rows of F=2 features: float2 (FP32) or __half2 (FP16)
  // Corner bundles read by the shade kernels (Sec. 4.1: one memory request
  // per sample point, half a cache line): row s = h(c) of the vertex c holds
  // the feature rows T[h(c + d)] of the 8 corners d in {0,1}^3 (x fastest) of
  // the cell whose lowest corner is c -- 64 bytes (FP32) or 32 bytes (FP16);
  // rows of empty slots, and of vertices with a coordinate equal to N (no
  // cell above them), are zero.  Derived from `table` (rebuilt whenever the
  // table changes).
  const void* bundle;     // m^3 rows of 8 x (float2 or __half2)
};

// Density and diffuse texture cubes as the kernels see them (Sec. 4.2).
// grid[x + b (y + b z)] of a base cell is its cube's index, or -1 when no
// cube is listed there.  Octant distances (octant bit q set: axis q
// decreasing): bdist[oct][cell] is the size D of the largest block of D^3
// unlisted base cells that starts at the cell and extends along the octant;
// fdist[oct][cube][fine cell] the same in fine cells within a cube for cells
// that are not live (no vertex of non-zero density), 0 for live cells.
struct CubesDev {
  const int32_t* grid;   // b^3
  const float* dens;     // n x (r+1)^3 sigma, x fastest
  const float4* diff;    // n x (r+1)^3 (c_d r, g, b, tint)
  const uint8_t* bdist;  // 8 x b^3
  const uint8_t* fdist;  // 8 x n x r^3
  int64_t n_cubes;
  int32_t b, r, rshift;  // r = 1 << rshift
  int32_t K;             // fine cells per axis, b r
  float K_f;             // (float)K
  float hi;              // lo + side (FP32): upper corner of the scene cube
  float step, t_min, alpha_miss;
};

// Device-resident object (all pointers are device memory unless noted).
struct Object {
  int device = 0;
  int L = 0, F = 2, d_in = 0;
  int fp16 = 0;
  float lo = -1.5f, scale = 1.0f / 3.0f;
  float bsphere[4] = {0, 0, 0, 0};  // proxy bounding sphere (centre, padded radius), object frame
  LevelDev lv[INOLF_MAX_LEVELS] = {};
  int64_t rows[INOLF_MAX_LEVELS] = {};
  // the hashed vertices of each level, packed x | y << 21 | z << 42 (device),
  // kept to rebuild the corner bundles when the tables change
  uint64_t* pts[INOLF_MAX_LEVELS] = {};
  int64_t n_pts[INOLF_MAX_LEVELS] = {};
  // BVH: nodes are 4 x float4 (child boxes x, y, z + child refs), triangles
  // 3 x float4 (v0 + id bits, e1, e2)
  void* nodes = nullptr;
  int32_t n_nodes = 0;
  void* tris = nullptr;
  int32_t n_tris = 0;
  // FP32 weights packed for the SIMT MLP: W1T [d_in][64], W2 [64][64], W3T [64][4]
  float* w_f32 = nullptr;
  // BF16 / FP8 operands for the tensor-core MLP (K-major rows, see mlp kernels)
  void* w_bf16 = nullptr;
  void* w_fp8 = nullptr;
  void* w_tf32 = nullptr;  // FP32 weights as split-TF32 operands (hi then lo per layer)
  int32_t tc_k1_bf16 = 0, tc_k1_fp8 = 0, tc_k1_tf32 = 0;
  uint32_t tc_bytes_bf16 = 0, tc_bytes_fp8 = 0, tc_bytes_tf32 = 0;
  float fp8_w_scale[3] = {0, 0, 0};  // host copy of the FP8 weight scales (refreshed on demand)
  float* w_scale_dev = nullptr;       // device copy, read by the kernels
  float fp8_act_scale[3] = {0, 0, 0};
  // decoupled variant (density march, alpha_c input, diffuse cubes)
  int variant = 0;
  CubesDev cub = {};
  size_t bytes = 0;
};

// Hit-list bytes per ray: (ray, t) records, plus alpha_c for the variant.
inline size_t hit_bytes_per_ray(const Object& o) { return o.variant ? 12 : 8; }

// Brackets one kernel launch with CUDA events when statistics are enabled
// (stats.cpp).
class LaunchTimer {
 public:
  LaunchTimer(const char* name, struct CUstream_st* st);
  ~LaunchTimer();

 private:
  const char* name_;
  struct CUstream_st* st_;
  void* a_ = nullptr;
  void* b_ = nullptr;
  bool active_ = false;
};

// Launch helpers (render.cu).
struct RayBatch {
  int mode;                // 0 = pinhole views, 1 = explicit rays
  const float* cams;       // device [n_views][13] (mode 0)
  int32_t n_views, W, H;
  const float* o;          // device [n][3] (mode 1)
  const float* d;
  int64_t n;               // total rays
};

// clear_flags: zero the header's failure flags first (false when a caller
// accumulates the flags of several launch_render calls, e.g. chunks of views).
inolf_status launch_render(const Object& obj, const RayBatch& rays, inolf_precision prec, float* rgba,
                           int32_t* tri_out, float* t_out, uint32_t* slots_out, float* feat_out,
                           void* workspace, size_t workspace_bytes, void* stream, bool amax = false,
                           float* alpha_out = nullptr, bool hits_only = false, bool count_trace = false,
                           bool clear_flags = true);

size_t workspace_bytes(int64_t n_rays);

// Weight repacking for the tensor-core paths (mlp_tc.cu) and the upload of
// all weight formats (host.cpp); both reuse existing device buffers.
inolf_status prepare_tc_weights(Object& obj, const float* w1, const float* w2, const float* w3, void* stream);
// The same packing (FP32, BF16 and FP8 blobs, FP8 weight scales) on the
// device from device weights, asynchronously on `stream` (mlp_tc.cu).
inolf_status pack_weights_device(Object& obj, const float* w1, const float* w2, const float* w3, void* stream);
inolf_status upload_weights(Object& obj, const float* w1, const float* w2, const float* w3, void* stream);

// Lays out level l's corner bundles from its table and hashed points
// (backward.cu).
inolf_status build_level_bundles(Object& o, int l, void* stream);

// Backward over explicit rays (render.cu + backward.cu).
inolf_status launch_backward_rays(const Object& obj, const float* o, const float* d, int64_t n, const float* d_rgba,
                                  float* const* grad_tables, float* gw1, float* gw2, float* gw3, void* workspace,
                                  size_t workspace_bytes, void* stream, const int32_t* tri_in = nullptr,
                                  const float* t_in = nullptr);

}  // namespace inolf

struct inolf_object {
  inolf::Object o;
};
