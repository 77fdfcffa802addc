/*
 * inolf.h -- C ABI of libinolf.so, the GB300 (sm_103a) implementation of the
 * i-NOLF per-ray hot path of "NEPHELE: A Neural Platform for Highly Realistic
 * Cloud Radiance Rendering" (arXiv 2303.04086):
 *
 *   one network query per ray (Sec. 4.2, Eqs. 2-3): the ray's first hit on a
 *   triangle-mesh geometry proxy, a multi-level perfect-spatial-hash feature
 *   fetch h(p) = h0(p) + Phi[h1(p)] (Sec. 4.1, Eq. 1) with trilinear
 *   interpolation, and a fused MLP F_s mapping the features plus a spherical
 *   harmonics encoding of the view direction to RGBA.
 *
 * Conventions for every call:
 *   - Every call returns an inolf_status; no C++ exception crosses the ABI.
 *     On error, inolf_last_error() returns a message (thread-local).
 *   - Dimension and pointer errors return INOLF_E_INVALID before any launch.
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory of the current device (e.g. a PyTorch CUDA tensor).
 *   - Callers own every buffer they pass in; the library owns the handles it
 *     returns (inolf_hash, inolf_object, inolf_server) and frees them in the
 *     matching *_free / *_destroy call.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device work is enqueued on it and the call returns without
 *     synchronising unless stated otherwise.
 *
 * Geometry conventions (shared with the synthetic scene records):
 *   - object frame: the scene cube [lo, lo + 1/scale]^3; grid level l has
 *     N_l cells per axis and vertices at integer coordinates 0..N_l;
 *   - a hit point P maps to x = (P - lo) * scale, u = N_l * x,
 *     c = clamp(floor(u), 0, N_l - 1), f = u - c (all FP32, Sec. 4.1);
 *   - camera record: 13 floats eye[3], right[3], up[3], fwd[3], tan(fovy/2);
 *     pixel (i, j), row 0 at the top, looks along
 *     normalize(((2i+1)/W - 1) tan W/H right + (1 - (2j+1)/H) tan up + fwd);
 *   - MLP input: level-major features (F per level) then 16 real SH values of
 *     the unit view direction, index l*l + l + m, no Condon-Shortley phase;
 *     hidden layers 64 wide with ReLU, output 4 with sigmoid, no biases;
 *     weights row-major [out][in].
 */
#ifndef INOLF_H
#define INOLF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int inolf_status;

#define INOLF_OK 0
#define INOLF_PENDING 1            /* serve_poll: the request is still in flight */
#define INOLF_E_INVALID (-1)       /* bad argument: nothing was launched */
#define INOLF_E_OOM (-2)           /* host or device allocation failed */
#define INOLF_E_CUDA (-3)          /* a CUDA runtime call failed */
#define INOLF_E_BUDGET (-4)        /* serving admission refused: HBM budget or slots exhausted */
#define INOLF_E_TIMEOUT (-5)       /* a bounded wait ran out */
#define INOLF_E_HASH_FAILED (-6)   /* perfect hash construction failed after max_retries */
#define INOLF_E_UNKNOWN_TICKET (-7) /* serve_poll: no such request */
#define INOLF_E_UNSUPPORTED (-8)   /* valid request this build cannot serve */
#define INOLF_E_CANCELLED (-9)     /* serve_poll: the request was cancelled */
#define INOLF_E_DEVICE (-10)       /* a kernel reported an internal failure (inolf_workspace_flags) */

#define INOLF_MAX_LEVELS 16
#define INOLF_HIDDEN 64
#define INOLF_OUT 4
#define INOLF_N_SH 16

typedef enum {
  INOLF_FP32 = 0, /* FP32 MLP: on the tensor cores as split TF32 (each FP32 operand as a TF32
                     hi and lo part, three products per step, FP32 accumulation: FP32-level
                     accuracy) when the workspace holds operand tiles, else on the CUDA cores */
  INOLF_BF16 = 1, /* BF16 weights/activations, FP32 accumulation (tensor cores) */
  INOLF_FP8 = 2   /* FP8 e4m3 weights/activations with per-tensor scales, FP32 accumulation */
} inolf_precision;

/* Message of the last error raised on the calling thread ("" if none). */
const char* inolf_last_error(void);

/* Library version string. */
const char* inolf_version(void);

/* ------------------------------------------------------------------------ */
/* Perfect spatial hash (Sec. 4.1, Eq. 1; construction after Lefebvre and    */
/* Hoppe 2006, which the paper cites for Phi).                               */
/* ------------------------------------------------------------------------ */
typedef struct {
  double sigma;        /* offset-table size r^3 ~ sigma * n (default 1/6) */
  double slot_slack;   /* hash-table size m^3 >= slot_slack * n (default 1.0) */
  int32_t max_retries; /* growth steps of r (then m) before INOLF_E_HASH_FAILED */
  uint64_t seed;       /* start of the offset search */
} inolf_hash_params;

typedef struct {
  int32_t m;          /* hash-table side: m^3 slots, m <= 1024 */
  int32_t r;          /* offset-table side: r^3 entries, gcd(m, r) = 1, m r > extent */
  int64_t n;          /* number of hashed points */
  uint32_t* phi;      /* host, r^3 entries, offset (x, y, z) packed x | y << 10 | z << 20 */
  uint32_t* slot_of;  /* host, n entries: h(p_i) linearised x + m (y + m z) */
  int32_t* coords;    /* host, n x 3: the hashed points in input order (a copy owned by the
                         handle); inolf_object_create reads them to lay out each level's
                         corner bundles */
} inolf_hash;

/* Host-only, pure.  Builds a collision-free hash of n distinct integer points
 * coords[n][3] (host, int32, each in [0, grid_extent]): h0(p) = p mod m,
 * h1(p) = p mod r per axis, h(p) = (h0(p) + Phi[h1(p)]) mod m per axis.
 * Offsets of 6-neighbouring Phi entries are tried first so that adjacent
 * points tend to land in adjacent slots (the coherence the paper's
 * Sec. 4.1 / Fig. 3 relies on).  Deterministic for given inputs and params
 * (params may be NULL for the defaults).  On success *out is a new handle that
 * the caller releases with inolf_hash_free.  Errors: INOLF_E_INVALID (bad
 * pointer, n < 0, coordinates out of range, duplicate points, m > 1024),
 * INOLF_E_OOM, INOLF_E_HASH_FAILED. */
inolf_status inolf_build_hash(const int32_t* coords, int64_t n, int32_t grid_extent,
                              const inolf_hash_params* params, inolf_hash** out);
void inolf_hash_free(inolf_hash* h);

/* ------------------------------------------------------------------------ */
/* Density and diffuse texture cubes (Sec. 4.2, "Density Texture Cubes",     */
/* "Diffuse Texture Cubes"): the paper's own hit-point estimation and the   */
/* decoupled diffuse/specular variant of the renderer.                       */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t b;              /* base grid: b^3 cells over the scene cube; power of two */
  int32_t r;              /* cube resolution: r^3 fine cells, (r+1)^3 vertex samples; power of
                             two; the fine grid K = b r is at most 4096 */
  int64_t n_cubes;        /* listed cubes (cells with any non-zero density) */
  const int32_t* cells;   /* host [n_cubes][3]: base cell of cube i, distinct, each in [0, b) */
  const float* density;   /* host [n_cubes][(r+1)^3]: sigma >= 0 at fine vertices cells[i] r +
                             (0..r)^3, x fastest; vertices shared by two cubes must agree */
  const float* diffuse;   /* host [n_cubes][(r+1)^3][4]: (c_d r, g, b, tint) at the same vertices */
  float side;             /* edge of the scene cube [domain_lo, domain_lo + side]^3 */
  float step;             /* march step delta (object units); side sqrt(3) / step < 2^20 */
  float t_min;            /* the march stops once the transmittance falls below t_min (0..1) */
  float alpha_miss;       /* a ray whose coarse opacity alpha_c <= alpha_miss misses (0..1) */
} inolf_cubes_desc;

/* ------------------------------------------------------------------------ */
/* Object: proxy mesh + per-level hashes and feature tables + MLP weights.   */
/* ------------------------------------------------------------------------ */
typedef struct {
  /* geometry proxy (host): n_vertices x 3 FP32, n_triangles x 3 int32 */
  int32_t n_vertices, n_triangles;
  const float* vertices;
  const int32_t* triangles;
  /* encoder levels (Sec. 4.1 grid + Eq. 1 hash per level) */
  int32_t n_levels;                 /* 1..INOLF_MAX_LEVELS */
  int32_t n_features;               /* F, must be 2 */
  const int32_t* resolution;        /* host [n_levels]: N_l */
  const inolf_hash* const* hashes;  /* host [n_levels]: hash of level l's vertex set */
  const float* const* features;     /* host [n_levels]: n_l x F FP32, row i belongs to the
                                       point i given to inolf_build_hash */
  int32_t features_fp16;            /* 1: tables stored as FP16 on the device */
  /* MLP F_s: d_in = n_levels * F + 16, hidden 64, out 4 (host, row-major) */
  const float* w1;                  /* [64][d_in] */
  const float* w2;                  /* [64][64] */
  const float* w3;                  /* [4][64] */
  /* FP8 activation scales (amax / 448) of the MLP inputs of layers 1, 2, 3;
     0 = calibrate later with inolf_object_set_fp8_scales */
  float fp8_act_scale[3];
  /* object frame */
  float domain_lo;                  /* lo (same on all axes), e.g. -1.5 */
  float domain_scale;               /* scale = 1 / side, e.g. (float)(1/3) */
  /* NULL: hit points come from the proxy mesh (one query per ray, Eqs. 2-3).
     Set: the decoupled variant of Sec. 4.2 -- the mesh may be empty
     (n_vertices = n_triangles = 0), hit points come from the density march
     (Eq. 4), the MLP takes alpha_c as one more input (Eq. 5: d_in = n_levels *
     F + 17, w1 is [64][d_in]) and the colour is c = c_d + tint c_s (Eq. 7)
     with (c_d, tint) from the diffuse cubes; the alpha channel is F_s's. */
  const inolf_cubes_desc* cubes;
} inolf_object_desc;

typedef struct inolf_object inolf_object;

/* Copies the description into library-owned device memory on the current
 * device (BVH built on the host, feature rows scattered into slot order).
 * Per level it also lays out the corner bundles the shade kernels read: for
 * every hashed vertex c (from the hash's `coords`), bundle row h(c) holds the
 * feature rows of the 8 corners of the cell whose lowest corner is c, so one
 * hit point costs one Phi entry and one 64-byte read (32 bytes for FP16
 * tables) per level, half a cache line (Sec. 4.1).  The bundles are rebuilt
 * by inolf_object_load_params.
 * Synchronous with respect to `stream` (returns after the uploads finish).
 * Errors: INOLF_E_INVALID (also: a hash with points but no coords),
 * INOLF_E_OOM, INOLF_E_CUDA. */
inolf_status inolf_object_create(const inolf_object_desc* desc, void* stream, inolf_object** out);
void inolf_object_destroy(inolf_object* obj);

/* Device bytes held by the object (tables, Phi, BVH, weights). */
inolf_status inolf_object_bytes(const inolf_object* obj, size_t* bytes);

/* Sets the FP8 activation scales (amax / 448 of the inputs of layers 1-3). */
inolf_status inolf_object_set_fp8_scales(inolf_object* obj, const float scales[3]);

/* Reads back the object's device feature tables (slot order) and weights into
 * host buffers: table_l has m_l^3 x F floats (FP16 tables are widened). */
inolf_status inolf_object_read_params(const inolf_object* obj, float* const* tables, float* w1, float* w2,
                                      float* w3);

/* Number of slots m_l^3 of level l (size of its feature table in rows). */
inolf_status inolf_object_table_rows(const inolf_object* obj, int32_t level, int64_t* rows);

/* ------------------------------------------------------------------------ */
/* Forward rendering (Sec. 4.2, one query per ray).                          */
/* ------------------------------------------------------------------------ */

/* Workspace bytes inolf_render / inolf_render_rays / inolf_march_rays need
 * for n_rays rays: a 256-byte header, 12 bytes per ray (the hit list and,
 * for density-cube objects, each hit's alpha_c), and the operand tiles of
 * the tensor-core shade, 128 bytes per ray for at most 4 Mi rays (512 MiB;
 * the environment variable INOLF_TC_CHUNK_ROWS, read at every call, sets
 * that row count) plus 256 bytes.  With these tiles the shade runs as two
 * kernels over sub-ranges of the hit list: one gathers and encodes the hits
 * into the tiles (rows of 2 d_in bytes BF16, d_in rounded up to 32 bytes
 * FP8, 4 d_in rounded up to 8 columns FP32), the other runs the MLP on the
 * tensor cores.  A smaller workspace (down to the header and the hit list of
 * one view, or of all rays for ray batches) is accepted: the tiles then take
 * what one view's hit records leave, if that is at least 256 rows; with less
 * room the BF16 / FP8 shade runs as one fused kernel with the same results
 * and the FP32 shade on the CUDA cores (within 2e-5 of the tensor-core
 * result, both within the FP32 bar of 1e-4 against the FP64 reference). */
size_t inolf_render_workspace_bytes(int64_t n_rays);

/* Renders n_views pinhole views of W x H pixels.
 *   cams       host, n_views x 13 floats (camera records)
 *   rgba_out   device, [n_views][H][W][4] FP32, straight alpha; rays that miss
 *              the proxy get (0, 0, 0, 0)
 *   tri_out    device [n_views][H][W] int32 closest triangle (-1 = miss), or NULL;
 *              for objects with density cubes: the hit sample k of the march
 *   t_out      device [n_views][H][W] FP32 hit distance (0 on miss), or NULL
 *   workspace  device, >= inolf_render_workspace_bytes(n_views * W * H) bytes,
 *              16-byte aligned, owned by the caller; contents undefined after
 * Calls on one workspace must not overlap in time. */
inolf_status inolf_render(const inolf_object* obj, const float* cams, int32_t n_views, int32_t W, int32_t H,
                          inolf_precision prec, float* rgba_out, int32_t* tri_out, float* t_out,
                          void* workspace, size_t workspace_bytes, void* stream);

/* Device-side failure flags.  The kernels of a call OR these bits into word 1
 * of the workspace header (the call zeroes the word when it starts); the
 * results of the rays concerned are incomplete:
 *   INOLF_FLAG_STACK_OVERFLOW   a BVH traversal stack overflowed (a subtree
 *                               was skipped; the BVH is deeper than 48)
 *   INOLF_FLAG_TRAVERSAL_LIMIT  a traversal exceeded 2^22 steps (malformed BVH)
 *   INOLF_FLAG_WAIT_TIMEOUT     a bounded wait in a shade kernel ran out (a
 *                               pipeline hand-over or a tensor-core completion);
 *                               some hit rays were not shaded */
#define INOLF_FLAG_STACK_OVERFLOW 1u
#define INOLF_FLAG_TRAVERSAL_LIMIT 2u
#define INOLF_FLAG_WAIT_TIMEOUT 4u

/* Reads the failure flags of the last call that used `workspace` (device
 * memory, as passed to that call; NULL = the fixed scratch of
 * inolf_render_rays_noalloc on the current device).  Synchronises `stream`
 * (the stream of that call) first.  *flags receives the bits above.  Returns
 * INOLF_OK when no bit is set, INOLF_E_TIMEOUT when INOLF_FLAG_WAIT_TIMEOUT is
 * set, INOLF_E_DEVICE for the traversal bits (the message names them),
 * INOLF_E_INVALID for a NULL flags pointer, INOLF_E_CUDA when the read fails.
 * A call without work (no rays) launches nothing and leaves the word as it
 * was.  The asynchronous calls (inolf_render, inolf_render_rays, inolf_backward, ...)
 * leave the check to the caller; the synchronising ones (inolf_render_host,
 * inolf_calibrate_fp8, inolf_trace_stats, inolf_render_rays_noalloc) make it
 * themselves and return its status. */
inolf_status inolf_workspace_flags(const void* workspace, uint32_t* flags, void* stream);

/* Limit of the bounded hand-over waits between the gather and MLP warps of
 * the warp-specialised shade kernels, for all later launches of the process
 * (ns; 0 restores the default of 2 s).  A wait that runs out sets
 * INOLF_FLAG_WAIT_TIMEOUT and the kernel returns.  Errors: INOLF_E_INVALID for
 * ns < 0. */
inolf_status inolf_set_wait_limit_ns(int64_t ns);

/* Fault injection for tests of the failure path (process-wide, 0 = off):
 * with INOLF_INJECT_RING_STALL the gather warps of the warp-specialised shade
 * kernels never hand their tiles over, so every hand-over wait runs out (after
 * the limit of inolf_set_wait_limit_ns) and the call's flags report
 * INOLF_FLAG_WAIT_TIMEOUT.  No GPU fault is involved: every wait is bounded. */
#define INOLF_INJECT_RING_STALL 1u
inolf_status inolf_set_fault_injection(uint32_t mask);

/* Renders n_views pinhole views into HOST memory (the frames a render farm
 * hands to its encoder, Sec. 5.1).  When rgba_host is pinned memory mapped
 * into the device's address space (cudaHostAlloc / cudaHostRegister with a
 * device pointer, 16-byte aligned), the kernels store the frames straight
 * into it over the GPU-host link and the staging buffer is not used.
 * Otherwise views go in chunks into two halves of a caller-owned device
 * staging buffer on `stream` while a library-owned stream copies the previous
 * chunk out, so the copies hide behind the rendering.
 *   rgba_host  host [n_views][H][W][4] FP32 (pinned memory; pageable memory
 *              works but copies synchronously)
 *   staging    device, 16-byte aligned; each half holds
 *              floor(staging_bytes / 2 / (W H 16)) >= 1 views
 *   workspace  as for inolf_render, for one chunk of views
 * Returns after the last frame is in host memory.  Errors: INOLF_E_INVALID
 * (including staging smaller than two views), INOLF_E_CUDA. */
inolf_status inolf_render_host(const inolf_object* obj, const float* cams, int32_t n_views, int32_t W, int32_t H,
                               inolf_precision prec, float* rgba_host, void* staging, size_t staging_bytes,
                               void* workspace, size_t workspace_bytes, void* stream);

/* Renders n explicit rays: o, d device [n][3] FP32 (d unit length, object
 * frame).  rgba_out device [n][4]; tri_out / t_out optional [n]. */
inolf_status inolf_render_rays(const inolf_object* obj, const float* o, const float* d, int64_t n,
                               inolf_precision prec, float* rgba_out, int32_t* tri_out, float* t_out,
                               void* workspace, size_t workspace_bytes, void* stream);

/* Hit-point estimation alone, for objects with density cubes (Sec. 4.2,
 * "Hit Point Estimation and Opacity Refinement", Eq. 4).  For n explicit rays
 * (o, d device [n][3] FP32, object frame, d unit length): samples t_k = t0 +
 * k step (FP32) from the ray's entry t0 >= 0 into the scene cube while t_k <=
 * its exit, density sigma_k = trilinear interpolation (successive FP32 lerps
 * along x, y, z) of the fine cell's 8 vertex samples (0 outside listed cubes),
 * w_k = T_k (1 - e_k), T_{k+1} = T_k e_k with e_k = exp(-sigma_k step); the
 * march stops after the sample that brings T below t_min.  The hit is the
 * first sample of largest w_k, alpha_c = 1 - T; alpha_c <= alpha_miss is a
 * miss.  Outputs (device, [n], each may be NULL): k_out hit sample (-1 =
 * miss), t_out its t (0 on miss), alpha_out alpha_c.  Errors: INOLF_E_INVALID
 * (also for objects without cubes), INOLF_E_CUDA. */
inolf_status inolf_march_rays(const inolf_object* obj, const float* o, const float* d, int64_t n, int32_t* k_out,
                              float* t_out, float* alpha_out, void* workspace, size_t workspace_bytes, void* stream);

/* ------------------------------------------------------------------------ */
/* Training (Sec. 4.2 "Training", Eq. 8).                                     */
/* ------------------------------------------------------------------------ */

/* Backward of the FP32 per-ray path for n explicit rays (o, d device [n][3]):
 * given d_rgba (device [n][4], dLoss/dRGBA), ACCUMULATES (+=) the gradients
 * of the feature tables into grad_tables (host array of n_levels device
 * pointers, each m_l^3 x 2 FP32 in slot order, see inolf_object_table_rows)
 * and of the weights into grad_w1 [64][d_in], grad_w2 [64][64], grad_w3
 * [4][64] (device FP32, row-major).  Activations are recomputed from the
 * object's current parameters; rays that miss contribute nothing.  Feature
 * gradients are scattered with atomics, weight gradients are reduced per
 * CTA first.  workspace as for inolf_render_rays.  Objects with density
 * cubes: INOLF_E_UNSUPPORTED (their training path, the hash-grid diffuse
 * branch of Eq. 6, is not part of this library). */
inolf_status inolf_backward(const inolf_object* obj, const float* o, const float* d, int64_t n,
                            const float* d_rgba, float* const* grad_tables, float* grad_w1, float* grad_w2,
                            float* grad_w3, void* workspace, size_t workspace_bytes, void* stream);

/* inolf_backward for rays whose forward pass already ran: tri and t (device
 * [n]) are that pass's tri_out / t_out (inolf_render_rays on the same rays,
 * the object's proxy unchanged since), and the hit list is compacted from them
 * instead of tracing the rays again.  Same outputs as inolf_backward. */
inolf_status inolf_backward_hits(const inolf_object* obj, const float* o, const float* d, int64_t n,
                                 const int32_t* tri, const float* t, const float* d_rgba, float* const* grad_tables,
                                 float* grad_w1, float* grad_w2, float* grad_w3, void* workspace,
                                 size_t workspace_bytes, void* stream);

/* Replaces the object's parameters from DEVICE buffers (e.g. after an
 * optimiser step): tables_dev (host array of n_levels device pointers, each
 * m_l^3 x 2 FP32 in slot order; NULL array or NULL entries keep a level) and
 * the three weight matrices (all or none; row-major FP32).  Tables are copied
 * on `stream`; new weights are repacked for every precision on the device
 * (FP8 weight scales recomputed there), also on `stream`: the call does not
 * synchronise, so it can sit inside a training loop. */
inolf_status inolf_object_load_params(inolf_object* obj, const float* const* tables_dev, const float* w1_dev,
                                      const float* w2_dev, const float* w3_dev, void* stream);

/* FP8 calibration (per-tensor activation scales): renders the given views
 * with the FP32 path, records the largest |input| of each MLP layer and sets
 * the object's activation scales to amax / 448 (the e4m3 maximum).  Weight
 * scales are set from the weights at inolf_object_create.  Synchronises
 * `stream`.  workspace as for inolf_render. */
inolf_status inolf_calibrate_fp8(inolf_object* obj, const float* cams, int32_t n_views, int32_t W, int32_t H,
                                 void* workspace, size_t workspace_bytes, void* stream);

/* Current FP8 scales: act[3] of the inputs of layers 1-3, weight[3] of W1-W3. */
inolf_status inolf_object_get_fp8_scales(const inolf_object* obj, float act[3], float weight[3]);

/* Stage outputs for parity checks of the encoder: for each ray that hits,
 * slots_out[n][L][8] uint32 (corner (dx,dy,dz), x fastest) and
 * feat_out[n][L*F] FP32 interpolated features; rows of missing rays are left
 * untouched.  Device buffers; workspace as for inolf_render_rays. */
inolf_status inolf_encode_rays(const inolf_object* obj, const float* o, const float* d, int64_t n,
                               uint32_t* slots_out, float* feat_out, void* workspace, size_t workspace_bytes,
                               void* stream);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of many viewers over resident objects (the   */
/* render farm + frame composer of Sec. 5-6 on one GPU).                     */
/* ------------------------------------------------------------------------ */
typedef struct inolf_server inolf_server;

typedef struct {
  size_t hbm_budget;       /* device bytes for served frames (admission budget), default 4 GiB */
  int32_t max_slots;       /* requests admitted at once (1..256), default 48 */
  int32_t max_width, max_height; /* largest admitted frame, default 3840 x 2160 */
  int32_t max_hits;        /* K: hits composited per ray (1..4), default 4 */
  int64_t wait_limit_ns;   /* bound of the device wait for a request descriptor, default 1 s */
  int64_t idle_limit_ns;   /* the persistent kernel exits after this long without work, default 20 ms */
  int32_t ctas_per_sm;     /* persistent CTAs per SM, 0 = as many as fit */
  int32_t policy;          /* 0: dispatch in arrival order; 1: Algorithm 1 (inolf_sched_*) */
  int64_t max_rays_in_flight; /* policy 1: ray budget of the device (0 = none) */
} inolf_serve_params;

#define INOLF_REQ_TEST_DROP_DESCRIPTOR 1u /* fault injection: the request descriptor is never published */

typedef struct {
  float camera[13];        /* camera record (world frame) */
  int32_t width, height;
  inolf_precision precision; /* INOLF_FP32 */
  uint32_t viewer_id;
  uint32_t flags;          /* 0, or INOLF_REQ_TEST_DROP_DESCRIPTOR in fault tests */
} inolf_request;

typedef struct {
  const float* frame;      /* device [height][width][4] straight RGBA, valid until inolf_serve_release */
  int32_t width, height;
  int64_t latency_ns;      /* submission to the first poll that saw the request complete */
  int64_t rays;
} inolf_result;

/* Creates a server on the current device: a frame arena of hbm_budget bytes,
 * mapped host memory for the request ring, and its own stream on which the
 * persistent kernel runs.  params may be NULL (defaults). */
inolf_status inolf_serve_create(const inolf_serve_params* params, inolf_server** out);

/* Makes an object resident in the scene at a translation (object frame =
 * world - translation).  Up to 16 objects; only while no request is in
 * flight.  The object must outlive the server.  Mesh-proxy objects and
 * density-cube objects (hit by the march, alpha_c input, c = c_d + t c_s) can
 * be mixed; every object's hits are composited by distance. */
inolf_status inolf_serve_add_object(inolf_server* srv, const inolf_object* obj, const float translation[3]);

/* Target frame rate of a viewer for policy 1 (default 50 Hz: one camera
 * update every 20 ms, as the paper's clients send). */
inolf_status inolf_serve_set_viewer(inolf_server* srv, uint32_t viewer_id, double target_fps);

/* Admits a request (INOLF_E_BUDGET when every slot is busy or the frame
 * does not fit the HBM budget: nothing is queued, retry later) and publishes
 * its 16x16 tiles to the running kernel (launching it if idle).  Each pixel
 * composites, front to back by (t, object id), up to max_hits hits over all
 * resident objects with the straight-alpha over operator and stores
 * (C / A, A).  *ticket identifies the request. */
inolf_status inolf_serve_submit(inolf_server* srv, const inolf_request* req, uint64_t* ticket);

/* INOLF_PENDING while in flight (and relaunches the kernel if it went idle);
 * INOLF_OK with *result filled when complete; INOLF_E_TIMEOUT or
 * INOLF_E_CANCELLED for requests that ended so; INOLF_E_UNKNOWN_TICKET. */
inolf_status inolf_serve_poll(inolf_server* srv, uint64_t ticket, inolf_result* result);

/* Asks the device to skip the remaining tiles of a request; poll then
 * returns INOLF_E_CANCELLED once its tiles have drained. */
inolf_status inolf_serve_cancel(inolf_server* srv, uint64_t ticket);

/* Returns the frame memory and the slot of a completed request. */
inolf_status inolf_serve_release(inolf_server* srv, uint64_t ticket);

/* Stops the persistent kernel (it finishes the tiles it holds) and frees
 * everything. */
inolf_status inolf_serve_destroy(inolf_server* srv);

/* Counters of the request loop: admitted, refused at admission (slots/HBM
 * budget), denied by the starvation state (policy 1), completed. */
inolf_status inolf_serve_counters(inolf_server* srv, int64_t* admitted, int64_t* refused, int64_t* denied,
                                  int64_t* completed);

/* Profile of the request loop (measurement support, no paper counterpart),
 * summed over the persistent CTAs, which add their figures when they exit:
 * the call first waits for the kernel to go idle and return.  out (host):
 * SM clock cycles spent in [0] claiming tiles and reading request
 * descriptors (including waiting for work), [1] tracing every object and
 * ordering the hits, [2] shading (weights staged, encoding, MLP), [3]
 * compositing and storing, [4] completion; then [5] tiles, [6] hits shaded,
 * [7] MLP batches (256-row tensor-core passes or FP32 passes of one object),
 * [8] weight stagings, [9] persistent CTAs per launch, and the launch plan of
 * the mesh-only kernel: [10] registers per thread, [11] static and [12]
 * dynamic shared-memory bytes per CTA, [13] CTAs per SM (out holds 14
 * entries).  reset != 0 zeroes the counters after reading. */
inolf_status inolf_serve_profile(inolf_server* srv, int64_t* out, int32_t reset);

/* ------------------------------------------------------------------------ */
/* Multi-user scheduling policy (Sec. 6.2, Algorithm 1, Eq. 13), host-only.  */
/* Every call takes the current time in ns from the caller (deterministic).  */
/* ------------------------------------------------------------------------ */
typedef struct inolf_sched inolf_sched;

/* max_rays_in_flight: the device's ray budget (0 = unlimited). */
inolf_status inolf_sched_create(int64_t max_rays_in_flight, inolf_sched** out);
void inolf_sched_destroy(inolf_sched* s);
/* Registers a viewer (a client) with its target frame rate FPS_i. */
inolf_status inolf_sched_set_viewer(inolf_sched* s, uint32_t viewer, double target_fps, int64_t now_ns);
/* Queues frame `id` of `viewer` with `rays` rays.  INOLF_E_BUDGET when the
 * scheduler is in the starvation state and the viewer is a new client. */
inolf_status inolf_sched_admit(inolf_sched* s, uint32_t viewer, uint64_t id, int64_t rays, int64_t now_ns);
/* Next frame to dispatch: starved frames first (a frame is starved when its
 * viewer's target time last_frame + w, w = 1/FPS - t, t the moving average
 * of completion times, has passed), else by the viewers' (frames in flight,
 * target time) while the rays in flight fit the budget.  INOLF_PENDING when
 * nothing may be dispatched now. */
inolf_status inolf_sched_next(inolf_sched* s, int64_t now_ns, uint64_t* id);
/* Frame `id` finished: updates its viewer's moving average and last frame. */
inolf_status inolf_sched_complete(inolf_sched* s, uint64_t id, int64_t now_ns);
/* Drops a frame that is still pending. */
inolf_status inolf_sched_cancel(inolf_sched* s, uint64_t id);
/* State: starvation flag, rays in flight, frames pending, admissions denied. */
inolf_status inolf_sched_state(inolf_sched* s, int64_t now_ns, int32_t* starving, int64_t* rays_in_flight,
                               int64_t* pending, int64_t* denied);
/* Current wait time w_i (Eq. 13) and target time of a viewer. */
inolf_status inolf_sched_wait_ns(inolf_sched* s, uint32_t viewer, int64_t* w_ns, int64_t* target_ns);

/* ------------------------------------------------------------------------ */
/* Allocation-free rendering (the paper has no counterpart: this exists for   */
/* callers of the library, not for the method).                              */
/* ------------------------------------------------------------------------ */
#define INOLF_NOALLOC_MAX_RAYS 1048576

/* Renders n explicit rays exactly like inolf_render_rays, but without a
 * workspace and without allocating anything.  It is meant for callers that
 * cannot allocate device memory where they render: a frame loop whose memory
 * budget is fixed at start-up, a plug-in whose host application owns every
 * device allocation, or a latency-critical thread that cannot afford the
 * device-wide synchronisation of cudaMalloc/cudaFree.  The hit list lives in
 * a fixed 8 MiB + 256 B array inside the library's device image, which every
 * GPU that loads the library keeps until the process exits.
 *   - n must be <= INOLF_NOALLOC_MAX_RAYS; larger n returns INOLF_E_INVALID
 *     and launches nothing.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current) and caches it; make
 *     that first call before any stream capture.
 *   - All calls on a device share the one array; the call clears its counters
 *     itself.  Calls whose GPU work overlaps in time (other streams or host
 *     threads) race on the array and produce wrong results: order them, e.g.
 *     on one stream.
 *   - The call synchronises `stream` before it returns, so that it can read
 *     the device-side failure flags of its kernels from the array (where the
 *     caller cannot reach them) and report them: INOLF_E_TIMEOUT or
 *     INOLF_E_DEVICE as inolf_workspace_flags describes.
 * o, d, rgba_out, tri_out, t_out, prec and stream are as for
 * inolf_render_rays. */
inolf_status inolf_render_rays_noalloc(const inolf_object* obj, const float* o, const float* d, int64_t n,
                                       inolf_precision prec, float* rgba_out, int32_t* tri_out, float* t_out,
                                       void* stream);

/* ------------------------------------------------------------------------ */
/* Launch statistics (measurement support, no paper counterpart).           */
/* ------------------------------------------------------------------------ */
typedef struct {
  char name[32];     /* kernel name */
  int64_t launches;  /* launches since the last reset */
  double ms;         /* summed device time between the events around each launch */
} inolf_kernel_stat;

/* When on != 0, every kernel launch of the library is bracketed by two CUDA
 * events recorded on its stream (process-wide switch). */
inolf_status inolf_stats_enable(int32_t on);
/* Drops all recorded launches. */
inolf_status inolf_stats_reset(void);
/* Waits for the recorded events and returns per-kernel totals: up to `max`
 * entries in out (host), the number of kernels in *n. */
inolf_status inolf_stats_read(inolf_kernel_stat* out, int32_t max, int32_t* n);

/* Traversal statistics of the closest-hit BVH step (Sec. 4.2's hit point on
 * the proxy mesh) for n_views pinhole views of W x H pixels, as rendered by
 * inolf_render: the trace kernel alone runs, each warp's 8 x 4-pixel packet
 * counting its own steps.  out (host, 5 entries): [0] rays, [1] hit rays,
 * [2] inner-node visits summed over packets, [3] triangle tests summed over
 * packets, [4] packets.  Every ray of a packet takes all of its packet's
 * steps, so [2] / [4] is the node visits per ray.  cams is host memory as for
 * inolf_render; workspace as for inolf_render (>= the size for the rays of
 * one view).  Synchronises `stream`.  E_INVALID for objects without a proxy
 * mesh (density cubes). */
inolf_status inolf_trace_stats(const inolf_object* obj, const float* cams, int32_t n_views, int32_t W, int32_t H,
                               int64_t* out, void* workspace, size_t workspace_bytes, void* stream);

/* Device peaks measured by microbenchmarks, the denominators of the rooflines
 * that the HBM copy and BF16 GEMM figures do not cover:
 *   l2_read_gbs     streaming 16-byte reads of an L2-resident 32 MB buffer,
 *                   bypassing L1 (GB/s);
 *   l2_gather_gsps  independent random 8-byte reads of the same buffer,
 *                   bypassing L1: one 32-byte sector each (G reads/s);
 *   fp32_tflops     packed FP32 fused multiply-adds (fma.rn.f32x2) on
 *                   registers (TFLOP/s, 2 flop per multiply-add).
 * Allocates and frees a 32 MB device buffer; synchronises `stream`. */
typedef struct {
  double l2_read_gbs;
  double l2_gather_gsps;
  double fp32_tflops;
} inolf_peaks;
inolf_status inolf_probe_peaks(inolf_peaks* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* INOLF_H */
