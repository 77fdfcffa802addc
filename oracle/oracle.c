/*
 * FP64 CPU oracle for the i-NOLF per-ray path (one network query per ray,
 * Sec. 4.2 "Opacity Light Field", Eqs. 2-3).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code with the CUDA path: it reads the seeded inputs (mesh, sorted vertex
 * keys with their features, MLP weights, camera records) and computes the
 * plain definition of what a ray renders to:
 *
 *   1. the pinhole ray of a pixel (FP32, fixed operation order);
 *   2. the closest triangle hit, the lexicographic minimum of (t, triangle id)
 *      over ALL triangles of the proxy mesh with an FP32 Moller-Trumbore test
 *      (the geometry proxy of Sec. 4.2 / the Lumigraph-style proxy of Sec. 1);
 *      an independent median-split BVH only skips boxes that cannot hold a
 *      better hit, and is checked against brute force by the tests;
 *   3. the hit point P = o + t d and, per level, the grid vertex p = floor(N x)
 *      of Sec. 4.1 (FP32, fixed operation order);
 *   4. the F features of the 8 voxel corners looked up in a sorted map keyed by
 *      integer vertex coordinate (what a collision-free spatial hash stores,
 *      Sec. 4.1 and Fig. 3), trilinearly interpolated in FP64;
 *   5. real spherical harmonics of degree 0..3 of the view direction (16
 *      values) from the associated-Legendre definition, FP64;
 *   6. the MLP F_s of Eq. 3: 64 ReLU, 64 ReLU, 4 sigmoid, no bias, FP64;
 *   7. misses render (0, 0, 0, 0);
 *   8. the analytic FP64 gradient of the per-ray outputs with respect to the
 *      weights and the corner features, for the L2 objective of Eq. 8;
 *   9. the paper's decoupled variant (Sec. 4.2, Eqs. 4-7): the hit point is
 *      the march sample of largest blending weight w_i = T_i (1 - exp(-sigma_i
 *      delta)) (Eq. 4) through a density field given as texture cubes, the
 *      coarse opacity alpha_c = sum_i w_i is an extra input of F_s (Eq. 5),
 *      and the colour is c = c_d + t c_s (Eq. 7) with (c_d, t) read from
 *      diffuse texture cubes at the hit point;
 *  10. the depth fusion of several objects' renders of one frame (the frame
 *      composer of Sec. 5.1): per ray, the K nearest hits over all objects by
 *      (t, object index), composited front to back with the straight-alpha
 *      over operator.
 *
 * Every FP32 step is written as separate IEEE operations; this file must be
 * compiled with -ffp-contract=off (no fused multiply-add), so that the same
 * FP32 operations give the same bits on any IEEE host.
 *
 * Where the paper is silent the following readings are used: domain cube
 * [-1.5, 1.5]^3 with x = (P - lo) * (float)(1/3); cell index clamped to
 * [0, N-1]; camera record eye, right, up, fwd, tan(fovy/2) with the pixel
 * centre convention below; corner order (dx, dy, dz) with x fastest; feature
 * order level-major; SH without the Condon-Shortley phase, index l*l + l + m.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include <float.h>
#if !defined(FLT_EVAL_METHOD) || FLT_EVAL_METHOD != 0
#error "the oracle needs FP32 expressions evaluated in FP32 (FLT_EVAL_METHOD == 0)"
#endif

#define ORC_MAX_LEVELS 32
#define ORC_T_MIN 1e-6f

/* ------------------------------------------------------------------------ */
/* 1. pinhole ray for pixel (i = column, j = row, row 0 at the top)          */
/*    px = ((2i+1)/W - 1) * tan(fovy/2) * W/H,  py = (1 - (2j+1)/H) tan(fovy/2) */
/*    d = normalize(px right + py up + fwd), o = eye                         */
/* ------------------------------------------------------------------------ */
void orc_ray(const float cam[13], int32_t W, int32_t H, int32_t i, int32_t j, float o[3], float d[3]) {
  const float th = cam[12];
  const float tx = (th * (float)W) / (float)H;
  const float a = ((float)(2 * i + 1) / (float)W) - 1.0f;
  const float b = 1.0f - ((float)(2 * j + 1) / (float)H);
  const float px = a * tx;
  const float py = b * th;
  float v[3];
  for (int k = 0; k < 3; ++k) {
    float r = px * cam[3 + k];
    float u = py * cam[6 + k];
    v[k] = (r + u) + cam[9 + k];
  }
  const float xx = v[0] * v[0];
  const float yy = v[1] * v[1];
  const float zz = v[2] * v[2];
  const float len2 = (xx + yy) + zz;
  const float inv = 1.0f / sqrtf(len2);
  for (int k = 0; k < 3; ++k) {
    o[k] = cam[k];
    d[k] = v[k] * inv;
  }
}

void orc_raygen(const float* cam, int32_t W, int32_t H, const int64_t* pix, int64_t n, float* o, float* d) {
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < n; ++r) {
    int64_t p = pix ? pix[r] : r;
    orc_ray(cam, W, H, (int32_t)(p % W), (int32_t)(p / W), o + 3 * r, d + 3 * r);
  }
}

/* ------------------------------------------------------------------------ */
/* 2. Moller-Trumbore (1997), two-sided, FP32, edges e1 = v1-v0, e2 = v2-v0.  */
/* Returns 1 and (t, u, v) when det != 0, u >= 0, v >= 0, u+v <= 1, t > 1e-6. */
/* ------------------------------------------------------------------------ */
static int mt_fp32(const float o[3], const float d[3], const float v0[3], const float e1[3], const float e2[3],
                   float* tt, float* uu, float* vv) {
  float p0 = d[1] * e2[2] - d[2] * e2[1];
  float p1 = d[2] * e2[0] - d[0] * e2[2];
  float p2 = d[0] * e2[1] - d[1] * e2[0];
  float det = (e1[0] * p0 + e1[1] * p1) + e1[2] * p2;
  if (det == 0.0f) return 0;
  float inv = 1.0f / det;
  float s0 = o[0] - v0[0], s1 = o[1] - v0[1], s2 = o[2] - v0[2];
  float u = ((s0 * p0 + s1 * p1) + s2 * p2) * inv;
  float q0 = s1 * e1[2] - s2 * e1[1];
  float q1 = s2 * e1[0] - s0 * e1[2];
  float q2 = s0 * e1[1] - s1 * e1[0];
  float v = ((d[0] * q0 + d[1] * q1) + d[2] * q2) * inv;
  float t = ((e2[0] * q0 + e2[1] * q1) + e2[2] * q2) * inv;
  if (!(u >= 0.0f) || !(v >= 0.0f) || !((u + v) <= 1.0f) || !(t > ORC_T_MIN)) return 0;
  *tt = t; *uu = u; *vv = v;
  return 1;
}

/* Same test in FP64 for information (rays whose FP64 winner differs). */
static int mt_fp64(const float o[3], const float d[3], const double v0[3], const double e1[3],
                   const double e2[3], double* tt) {
  double p0 = d[1] * e2[2] - d[2] * e2[1], p1 = d[2] * e2[0] - d[0] * e2[2], p2 = d[0] * e2[1] - d[1] * e2[0];
  double det = e1[0] * p0 + e1[1] * p1 + e1[2] * p2;
  if (det == 0.0) return 0;
  double inv = 1.0 / det;
  double s0 = o[0] - v0[0], s1 = o[1] - v0[1], s2 = o[2] - v0[2];
  double u = (s0 * p0 + s1 * p1 + s2 * p2) * inv;
  double q0 = s1 * e1[2] - s2 * e1[1], q1 = s2 * e1[0] - s0 * e1[2], q2 = s0 * e1[1] - s1 * e1[0];
  double v = (d[0] * q0 + d[1] * q1 + d[2] * q2) * inv;
  double t = (e2[0] * q0 + e2[1] * q1 + e2[2] * q2) * inv;
  if (u < 0 || v < 0 || u + v > 1 || !(t > 1e-6)) return 0;
  *tt = t;
  return 1;
}

typedef struct {
  int32_t nF;
  float* tri; /* per triangle: v0[3], e1[3], e2[3] in FP32 */
} orc_mesh;

static orc_mesh* mesh_create(const float* V, const int32_t* F, int32_t nF) {
  orc_mesh* m = (orc_mesh*)calloc(1, sizeof(orc_mesh));
  m->nF = nF;
  m->tri = (float*)malloc(sizeof(float) * 9 * (size_t)(nF > 0 ? nF : 1));
  for (int32_t k = 0; k < nF; ++k) {
    const float* a = V + 3 * F[3 * k + 0];
    const float* b = V + 3 * F[3 * k + 1];
    const float* c = V + 3 * F[3 * k + 2];
    float* r = m->tri + 9 * (size_t)k;
    for (int q = 0; q < 3; ++q) {
      r[q] = a[q];
      r[3 + q] = b[q] - a[q];
      r[6 + q] = c[q] - a[q];
    }
  }
  return m;
}

/* closest hit = lexicographic min of (t, triangle id) */
static inline void consider(const orc_mesh* m, int32_t k, const float o[3], const float d[3],
                            float* bt, int32_t* bid, float* bu, float* bv) {
  float t, u, v;
  const float* r = m->tri + 9 * (size_t)k;
  if (mt_fp32(o, d, r, r + 3, r + 6, &t, &u, &v)) {
    if (*bid < 0 || t < *bt || (t == *bt && k < *bid)) {
      *bt = t; *bid = k; *bu = u; *bv = v;
    }
  }
}

/* near-edge: the winning hit lies within 1e-6 (barycentric) of an edge */
static inline int32_t near_edge(float u, float v) {
  float w = 1.0f - u - v;
  float m = u < v ? u : v;
  m = m < w ? m : w;
  return m < 1e-6f;
}

/* Brute force over all triangles.  fp64_tri (optional) receives the FP64
 * winner for information. */
void orc_hit_brute(const float* V, const int32_t* F, int32_t nF, const float* o, const float* d, int64_t n,
                   int32_t* tri, float* t, int32_t* edge, int32_t* fp64_tri) {
  orc_mesh* m = mesh_create(V, F, nF);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t r = 0; r < n; ++r) {
    float bt = 0.0f, bu = 0.0f, bv = 0.0f;
    int32_t bid = -1;
    for (int32_t k = 0; k < nF; ++k) consider(m, k, o + 3 * r, d + 3 * r, &bt, &bid, &bu, &bv);
    tri[r] = bid;
    t[r] = bid >= 0 ? bt : 0.0f;
    if (edge) edge[r] = bid >= 0 ? near_edge(bu, bv) : 0;
    if (fp64_tri) {
      double best = 0.0;
      int32_t id = -1;
      for (int32_t k = 0; k < nF; ++k) {
        const int32_t* f = F + 3 * k;
        double a[3], e1[3], e2[3], tt;
        for (int q = 0; q < 3; ++q) {
          a[q] = V[3 * f[0] + q];
          e1[q] = (double)V[3 * f[1] + q] - a[q];
          e2[q] = (double)V[3 * f[2] + q] - a[q];
        }
        if (mt_fp64(o + 3 * r, d + 3 * r, a, e1, e2, &tt) && (id < 0 || tt < best)) {
          best = tt;
          id = k;
        }
      }
      fp64_tri[r] = id;
    }
  }
  free(m->tri);
  free(m);
}

/* ------------------------------------------------------------------------ */
/* Median-split BVH (acceleration only).  A node is skipped only when its    */
/* padded box is entered strictly after the current best t (plus slack), so  */
/* the result is the same lexicographic minimum as brute force.              */
/* ------------------------------------------------------------------------ */
typedef struct {
  double lo[3], hi[3];
  int32_t left, right; /* children, or -1 */
  int32_t first, count; /* leaf range in order[] */
} orc_node;

typedef struct {
  orc_mesh* mesh;
  orc_node* nodes;
  int32_t n_nodes;
  int32_t* order;
} orc_bvh;

typedef struct { orc_bvh* b; const float* V; const int32_t* F; double* cen; } bvh_ctx;

static const double* g_sort_cen; /* build is single-threaded */
static int g_sort_axis;
static int cmp_centroid(const void* pa, const void* pb) {
  int32_t a = *(const int32_t*)pa, b = *(const int32_t*)pb;
  double ca = g_sort_cen[3 * a + g_sort_axis], cb = g_sort_cen[3 * b + g_sort_axis];
  if (ca < cb) return -1;
  if (ca > cb) return 1;
  return (a > b) - (a < b);
}

static int32_t bvh_rec(bvh_ctx* c, int32_t first, int32_t count) {
  orc_bvh* b = c->b;
  int32_t id = b->n_nodes++;
  orc_node* nd = &b->nodes[id];
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  double clo[3] = {1e300, 1e300, 1e300}, chi[3] = {-1e300, -1e300, -1e300};
  for (int32_t i = first; i < first + count; ++i) {
    int32_t k = b->order[i];
    for (int v = 0; v < 3; ++v)
      for (int q = 0; q < 3; ++q) {
        double x = c->V[3 * c->F[3 * k + v] + q];
        if (x < lo[q]) lo[q] = x;
        if (x > hi[q]) hi[q] = x;
      }
    for (int q = 0; q < 3; ++q) {
      double x = c->cen[3 * k + q];
      if (x < clo[q]) clo[q] = x;
      if (x > chi[q]) chi[q] = x;
    }
  }
  for (int q = 0; q < 3; ++q) {
    double pad = 1e-5 * (1.0 + fabs(lo[q]) + fabs(hi[q]));
    nd->lo[q] = lo[q] - pad;
    nd->hi[q] = hi[q] + pad;
  }
  nd->left = nd->right = -1;
  nd->first = first;
  nd->count = count;
  if (count <= 4) return id;
  int axis = 0;
  for (int q = 1; q < 3; ++q)
    if (chi[q] - clo[q] > chi[axis] - clo[axis]) axis = q;
  if (chi[axis] - clo[axis] <= 0.0) return id;
  /* median split: order the range by (centroid[axis], triangle id) */
  int32_t half = count / 2;
  g_sort_cen = c->cen;
  g_sort_axis = axis;
  qsort(b->order + first, (size_t)count, sizeof(int32_t), cmp_centroid);
  int32_t l = bvh_rec(c, first, half);
  int32_t r = bvh_rec(c, first + half, count - half);
  b->nodes[id].left = l;
  b->nodes[id].right = r;
  return id;
}

void* orc_bvh_build(const float* V, const int32_t* F, int32_t nF) {
  orc_bvh* b = (orc_bvh*)calloc(1, sizeof(orc_bvh));
  b->mesh = mesh_create(V, F, nF);
  b->nodes = (orc_node*)calloc((size_t)2 * (nF > 0 ? nF : 1), sizeof(orc_node));
  b->order = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nF > 0 ? nF : 1));
  double* cen = (double*)malloc(sizeof(double) * 3 * (size_t)(nF > 0 ? nF : 1));
  for (int32_t k = 0; k < nF; ++k) {
    b->order[k] = k;
    for (int q = 0; q < 3; ++q)
      cen[3 * k + q] = ((double)V[3 * F[3 * k] + q] + V[3 * F[3 * k + 1] + q] + V[3 * F[3 * k + 2] + q]) / 3.0;
  }
  bvh_ctx c = {b, V, F, cen};
  if (nF > 0) bvh_rec(&c, 0, nF);
  free(cen);
  return b;
}

void orc_bvh_free(void* h) {
  orc_bvh* b = (orc_bvh*)h;
  if (!b) return;
  free(b->mesh->tri);
  free(b->mesh);
  free(b->nodes);
  free(b->order);
  free(b);
}

static int box_enter(const orc_node* nd, const float o[3], const double inv[3], double tmax, double* tin) {
  double t0 = 0.0, t1 = tmax;
  for (int q = 0; q < 3; ++q) {
    double a = (nd->lo[q] - o[q]) * inv[q];
    double b = (nd->hi[q] - o[q]) * inv[q];
    if (isnan(a) || isnan(b)) { /* ray parallel to the slab and starting on its plane */
      if (o[q] < nd->lo[q] || o[q] > nd->hi[q]) return 0;
      continue;
    }
    double lo = a < b ? a : b, hi = a < b ? b : a;
    if (lo > t0) t0 = lo;
    if (hi < t1) t1 = hi;
    if (t0 > t1) return 0;
  }
  *tin = t0;
  return 1;
}

static void bvh_closest(const orc_bvh* b, const float o[3], const float d[3], int32_t* tri, float* t,
                        int32_t* edge) {
  double inv[3];
  for (int q = 0; q < 3; ++q) inv[q] = 1.0 / (double)d[q];
  float bt = 0.0f, bu = 0.0f, bv = 0.0f;
  int32_t bid = -1;
  int32_t stack[128];
  int sp = 0;
  if (b->n_nodes > 0) stack[sp++] = 0;
  while (sp > 0) {
    const orc_node* nd = &b->nodes[stack[--sp]];
    double tin;
    double lim = bid < 0 ? 1e300 : (double)bt * (1.0 + 1e-5) + 1e-5;
    if (!box_enter(nd, o, inv, lim, &tin)) continue;
    if (nd->left < 0) {
      for (int32_t i = nd->first; i < nd->first + nd->count; ++i)
        consider(b->mesh, b->order[i], o, d, &bt, &bid, &bu, &bv);
    } else {
      stack[sp++] = nd->left;
      stack[sp++] = nd->right;
    }
  }
  *tri = bid;
  *t = bid >= 0 ? bt : 0.0f;
  if (edge) *edge = bid >= 0 ? near_edge(bu, bv) : 0;
}

void orc_bvh_hit(const void* h, const float* o, const float* d, int64_t n, int32_t* tri, float* t, int32_t* edge) {
  const orc_bvh* b = (const orc_bvh*)h;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t r = 0; r < n; ++r) bvh_closest(b, o + 3 * r, d + 3 * r, tri + r, t + r, edge ? edge + r : 0);
}

/* ------------------------------------------------------------------------ */
/* 3. Hit point and grid vertex of Sec. 4.1 (p = floor(N x)), FP32.          */
/* ------------------------------------------------------------------------ */
typedef struct { float lo, scale; } orc_domain;

static void cell_of(orc_domain dom, int32_t N, const float o[3], const float d[3], float t,
                    int32_t c[3], float f[3]) {
  for (int q = 0; q < 3; ++q) {
    float P = o[q] + t * d[q];
    float x = (P - dom.lo) * dom.scale;
    float u = (float)N * x;
    float fl = floorf(u);
    int32_t ci = (int32_t)fl;
    if (ci < 0) ci = 0;
    if (ci > N - 1) ci = N - 1;
    c[q] = ci;
    f[q] = u - (float)ci;
  }
}

void orc_cells(float lo, float scale, int32_t N, const float* o, const float* d, const float* t, int64_t n,
               int32_t* cells, float* fracs) {
  orc_domain dom = {lo, scale};
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < n; ++r) cell_of(dom, N, o + 3 * r, d + 3 * r, t[r], cells + 3 * r, fracs + 3 * r);
}

/* ------------------------------------------------------------------------ */
/* Scene: mesh BVH, per-level sorted key maps with FP64 features, FP64 MLP.  */
/* ------------------------------------------------------------------------ */
typedef struct {
  orc_bvh* bvh;
  orc_domain dom;
  int32_t L, nfeat, d_in, hidden, d_out;
  int32_t alpha_in; /* 1: the last MLP input is alpha_c (Eq. 5) */
  int32_t N[ORC_MAX_LEVELS];
  int64_t nkeys[ORC_MAX_LEVELS];
  uint64_t* keys[ORC_MAX_LEVELS];
  double* feats[ORC_MAX_LEVELS];
  double *w1, *w2, *w3;
} orc_scene;

static uint64_t pack_key(int64_t x, int64_t y, int64_t z) {
  return (uint64_t)x | ((uint64_t)y << 21) | ((uint64_t)z << 42);
}

/* index of key in the sorted list, -1 when absent */
static int64_t find_key(const uint64_t* keys, int64_t n, uint64_t key) {
  int64_t lo = 0, hi = n - 1;
  while (lo <= hi) {
    int64_t mid = lo + ((hi - lo) >> 1);
    if (keys[mid] == key) return mid;
    if (keys[mid] < key) lo = mid + 1;
    else hi = mid - 1;
  }
  return -1;
}

void* orc_scene_create(const float* V, const int32_t* F, int32_t nF, int32_t L, const int32_t* N,
                       const uint64_t* const* keys, const int64_t* nkeys, const float* const* feats, int32_t nfeat,
                       const float* w1, const float* w2, const float* w3, int32_t d_in, int32_t hidden,
                       int32_t d_out, float lo, float scale) {
  if (L < 1 || L > ORC_MAX_LEVELS || (d_in != L * nfeat + 16 && d_in != L * nfeat + 17)) return 0;
  orc_scene* s = (orc_scene*)calloc(1, sizeof(orc_scene));
  s->bvh = (orc_bvh*)orc_bvh_build(V, F, nF);
  s->dom.lo = lo;
  s->dom.scale = scale;
  s->L = L; s->nfeat = nfeat; s->d_in = d_in; s->hidden = hidden; s->d_out = d_out;
  s->alpha_in = d_in == L * nfeat + 17;
  for (int32_t l = 0; l < L; ++l) {
    s->N[l] = N[l];
    s->nkeys[l] = nkeys[l];
    s->keys[l] = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(nkeys[l] > 0 ? nkeys[l] : 1));
    memcpy(s->keys[l], keys[l], sizeof(uint64_t) * (size_t)nkeys[l]);
    s->feats[l] = (double*)malloc(sizeof(double) * (size_t)(nkeys[l] * nfeat > 0 ? nkeys[l] * nfeat : 1));
    for (int64_t i = 0; i < nkeys[l] * nfeat; ++i) s->feats[l][i] = feats[l][i];
  }
  s->w1 = (double*)malloc(sizeof(double) * (size_t)hidden * d_in);
  s->w2 = (double*)malloc(sizeof(double) * (size_t)hidden * hidden);
  s->w3 = (double*)malloc(sizeof(double) * (size_t)d_out * hidden);
  for (int64_t i = 0; i < (int64_t)hidden * d_in; ++i) s->w1[i] = w1[i];
  for (int64_t i = 0; i < (int64_t)hidden * hidden; ++i) s->w2[i] = w2[i];
  for (int64_t i = 0; i < (int64_t)d_out * hidden; ++i) s->w3[i] = w3[i];
  return s;
}

void orc_scene_free(void* h) {
  orc_scene* s = (orc_scene*)h;
  if (!s) return;
  orc_bvh_free(s->bvh);
  for (int32_t l = 0; l < s->L; ++l) { free(s->keys[l]); free(s->feats[l]); }
  free(s->w1); free(s->w2); free(s->w3);
  free(s);
}

/* FP64 parameter arrays, exposed so that the tests can perturb them for
 * finite differences: which = 0/1/2 -> W1/W2/W3, 3 -> features of `level`. */
double* orc_scene_param(void* h, int32_t which, int32_t level, int64_t* count) {
  orc_scene* s = (orc_scene*)h;
  switch (which) {
    case 0: *count = (int64_t)s->hidden * s->d_in; return s->w1;
    case 1: *count = (int64_t)s->hidden * s->hidden; return s->w2;
    case 2: *count = (int64_t)s->d_out * s->hidden; return s->w3;
    case 3: *count = s->nkeys[level] * s->nfeat; return s->feats[level];
  }
  *count = 0;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* 4. Encoding E(x) of Sec. 4.1: features of the 8 corners of the cell,      */
/*    trilinear weights prod_axis (corner bit ? f : 1 - f), FP64.            */
/*    corner k = (dx, dy, dz) = (k & 1, k >> 1 & 1, k >> 2 & 1).             */
/*    idx (optional) receives the key index of every corner (-1 if absent).  */
/* ------------------------------------------------------------------------ */
static int64_t encode_ray(const orc_scene* s, const float o[3], const float d[3], float t, double* E,
                          int64_t* idx, double* wts) {
  int64_t missing = 0;
  for (int32_t l = 0; l < s->L; ++l) {
    int32_t c[3];
    float f[3];
    cell_of(s->dom, s->N[l], o, d, t, c, f);
    for (int32_t k = 0; k < s->nfeat; ++k) E[l * s->nfeat + k] = 0.0;
    for (int corner = 0; corner < 8; ++corner) {
      int dx = corner & 1, dy = (corner >> 1) & 1, dz = (corner >> 2) & 1;
      double w = (dx ? (double)f[0] : 1.0 - (double)f[0]) * (dy ? (double)f[1] : 1.0 - (double)f[1]) *
                 (dz ? (double)f[2] : 1.0 - (double)f[2]);
      int64_t i = find_key(s->keys[l], s->nkeys[l], pack_key(c[0] + dx, c[1] + dy, c[2] + dz));
      if (idx) idx[l * 8 + corner] = i;
      if (wts) wts[l * 8 + corner] = w;
      if (i < 0) { ++missing; continue; }
      for (int32_t k = 0; k < s->nfeat; ++k) E[l * s->nfeat + k] += w * s->feats[l][i * s->nfeat + k];
    }
  }
  return missing;
}

/* ------------------------------------------------------------------------ */
/* 5. Real spherical harmonics, bands 0..3, of a unit direction (Sec. 4.2:    */
/*    the view direction v that enters F_s).  Y_l^m = K_l^m P_l^|m|(cos th)   */
/*    times sqrt2 cos(m ph) (m > 0), 1 (m = 0), sqrt2 sin(|m| ph) (m < 0),    */
/*    K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), P_l^m without the            */
/*    Condon-Shortley phase, from the three-term recurrence in l.            */
/* ------------------------------------------------------------------------ */
static double factorial(int n) { double r = 1; for (int i = 2; i <= n; ++i) r *= i; return r; }

static double assoc_legendre(int l, int m, double x) {
  double pmm = 1.0, s = sqrt((1.0 - x) * (1.0 + x));
  for (int i = 1; i <= m; ++i) pmm *= (2.0 * i - 1.0) * s;
  if (l == m) return pmm;
  double pm1 = x * (2.0 * m + 1.0) * pmm;
  if (l == m + 1) return pm1;
  double pll = 0.0;
  for (int ll = m + 2; ll <= l; ++ll) {
    pll = ((2.0 * ll - 1.0) * x * pm1 - (ll + m - 1.0) * pmm) / (ll - m);
    pmm = pm1;
    pm1 = pll;
  }
  return pll;
}

void orc_sh16(const double dir[3], double out[16]) {
  double n = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
  double z = dir[2] / n;
  if (z > 1.0) z = 1.0;
  if (z < -1.0) z = -1.0;
  double ph = atan2(dir[1], dir[0]);
  for (int l = 0; l <= 3; ++l)
    for (int m = -l; m <= l; ++m) {
      int am = m < 0 ? -m : m;
      double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - am) / factorial(l + am));
      double P = assoc_legendre(l, am, z);
      double v;
      if (m > 0) v = sqrt(2.0) * K * P * cos(m * ph);
      else if (m < 0) v = sqrt(2.0) * K * P * sin(am * ph);
      else v = K * P;
      out[l * l + l + m] = v;
    }
}

/* ------------------------------------------------------------------------ */
/* 6. F_s (Eq. 3): x -> relu(W1 x) -> relu(W2 .) -> sigmoid(W3 .), FP64.     */
/* ------------------------------------------------------------------------ */
static double sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }

static void mlp_forward(const orc_scene* s, const double* x, double* z1, double* a1, double* z2, double* a2,
                        double* out) {
  const int32_t H = s->hidden, D = s->d_in, O = s->d_out;
  for (int32_t j = 0; j < H; ++j) {
    double acc = 0.0;
    for (int32_t i = 0; i < D; ++i) acc += s->w1[(size_t)j * D + i] * x[i];
    z1[j] = acc;
    a1[j] = acc > 0.0 ? acc : 0.0;
  }
  for (int32_t j = 0; j < H; ++j) {
    double acc = 0.0;
    for (int32_t i = 0; i < H; ++i) acc += s->w2[(size_t)j * H + i] * a1[i];
    z2[j] = acc;
    a2[j] = acc > 0.0 ? acc : 0.0;
  }
  for (int32_t j = 0; j < O; ++j) {
    double acc = 0.0;
    for (int32_t i = 0; i < H; ++i) acc += s->w3[(size_t)j * H + i] * a2[i];
    out[j] = sigmoid(acc);
  }
}

/* Plain MLP on caller-given arrays (for hand-evaluated checks). */
void orc_mlp(const double* w1, const double* w2, const double* w3, int32_t d_in, int32_t hidden, int32_t d_out,
             const double* x, int64_t n, double* out) {
  for (int64_t r = 0; r < n; ++r) {
    double a1[256], a2[256];
    for (int32_t j = 0; j < hidden; ++j) {
      double acc = 0.0;
      for (int32_t i = 0; i < d_in; ++i) acc += w1[(size_t)j * d_in + i] * x[r * d_in + i];
      a1[j] = acc > 0.0 ? acc : 0.0;
    }
    for (int32_t j = 0; j < hidden; ++j) {
      double acc = 0.0;
      for (int32_t i = 0; i < hidden; ++i) acc += w2[(size_t)j * hidden + i] * a1[i];
      a2[j] = acc > 0.0 ? acc : 0.0;
    }
    for (int32_t j = 0; j < d_out; ++j) {
      double acc = 0.0;
      for (int32_t i = 0; i < hidden; ++i) acc += w3[(size_t)j * hidden + i] * a2[i];
      out[r * d_out + j] = sigmoid(acc);
    }
  }
}

/* ------------------------------------------------------------------------ */
/* One ray end to end (steps 3-7) given its closest hit.                      */
/* ------------------------------------------------------------------------ */
#define ORC_MAXD 256

static int64_t shade_ray(const orc_scene* s, const float o[3], const float d[3], float t, double* rgba,
                         double* E_out) {
  double x[ORC_MAXD], z1[ORC_MAXD], a1[ORC_MAXD], z2[ORC_MAXD], a2[ORC_MAXD];
  int64_t miss = encode_ray(s, o, d, t, x, 0, 0);
  double dir[3] = {d[0], d[1], d[2]};
  orc_sh16(dir, x + s->L * s->nfeat);
  if (E_out) memcpy(E_out, x, sizeof(double) * (size_t)s->d_in);
  mlp_forward(s, x, z1, a1, z2, a2, rgba);
  return miss;
}

/* Full path for explicit rays.  tri/t/edge/E may be NULL.  Returns the number
 * of corner lookups that found no vertex (0 for a valid scene). */
int64_t orc_render_rays(const void* h, const float* o, const float* d, int64_t n, double* rgba, int32_t* tri,
                        float* t, int32_t* edge, double* E) {
  const orc_scene* s = (const orc_scene*)h;
  int64_t missing = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : missing)
  for (int64_t r = 0; r < n; ++r) {
    int32_t id;
    float tt;
    int32_t e;
    bvh_closest(s->bvh, o + 3 * r, d + 3 * r, &id, &tt, &e);
    if (tri) tri[r] = id;
    if (t) t[r] = tt;
    if (edge) edge[r] = e;
    if (id < 0) {
      for (int32_t k = 0; k < s->d_out; ++k) rgba[r * s->d_out + k] = 0.0;
      if (E) for (int32_t k = 0; k < s->d_in; ++k) E[r * s->d_in + k] = 0.0;
      continue;
    }
    missing += shade_ray(s, o + 3 * r, d + 3 * r, tt, rgba + r * s->d_out, E ? E + r * s->d_in : 0);
  }
  return missing;
}

/* Full path for pixels of one pinhole view (pix = j * W + i; NULL = all). */
int64_t orc_render_pixels(const void* h, const float* cam, int32_t W, int32_t H, const int64_t* pix, int64_t n,
                          double* rgba, int32_t* tri, float* t, int32_t* edge) {
  const orc_scene* s = (const orc_scene*)h;
  int64_t missing = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : missing)
  for (int64_t r = 0; r < n; ++r) {
    int64_t p = pix ? pix[r] : r;
    float o[3], d[3];
    orc_ray(cam, W, H, (int32_t)(p % W), (int32_t)(p / W), o, d);
    int32_t id;
    float tt;
    int32_t e;
    bvh_closest(s->bvh, o, d, &id, &tt, &e);
    if (tri) tri[r] = id;
    if (t) t[r] = tt;
    if (edge) edge[r] = e;
    if (id < 0) {
      for (int32_t k = 0; k < s->d_out; ++k) rgba[r * s->d_out + k] = 0.0;
      continue;
    }
    missing += shade_ray(s, o, d, tt, rgba + r * s->d_out, 0);
  }
  return missing;
}

/* Corner key indices and weights of every level for given hits (for
 * slot-level parity): idx[r][l][8], w[r][l][8]. */
void orc_corners(const void* h, const float* o, const float* d, const float* t, int64_t n, int64_t* idx,
                 double* w) {
  const orc_scene* s = (const orc_scene*)h;
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < n; ++r) {
    double E[ORC_MAXD];
    encode_ray(s, o + 3 * r, d + 3 * r, t[r], E, idx + r * s->L * 8, w + r * s->L * 8);
  }
}

/* ------------------------------------------------------------------------ */
/* 8. Analytic FP64 backward of the per-ray outputs (Eq. 8's gradient path). */
/*    d_out[r][4] = dLoss/dRGBA.  Gradients are ACCUMULATED into gw1, gw2,   */
/*    gw3 and gfeat[l] (indexed like the sorted keys).  Single-threaded so   */
/*    the summation order is fixed.                                          */
/* ------------------------------------------------------------------------ */
void orc_backward(const void* h, const float* o, const float* d, int64_t n, const double* d_out, double* gw1,
                  double* gw2, double* gw3, double* const* gfeat) {
  const orc_scene* s = (const orc_scene*)h;
  const int32_t H = s->hidden, D = s->d_in, O = s->d_out, L = s->L, NF = s->nfeat;
  for (int64_t r = 0; r < n; ++r) {
    int32_t id;
    float tt;
    bvh_closest(s->bvh, o + 3 * r, d + 3 * r, &id, &tt, 0);
    if (id < 0) continue;
    double x[ORC_MAXD], z1[ORC_MAXD], a1[ORC_MAXD], z2[ORC_MAXD], a2[ORC_MAXD], y[16];
    int64_t idx[ORC_MAX_LEVELS * 8];
    double wts[ORC_MAX_LEVELS * 8];
    encode_ray(s, o + 3 * r, d + 3 * r, tt, x, idx, wts);
    double dir[3] = {d[3 * r], d[3 * r + 1], d[3 * r + 2]};
    orc_sh16(dir, x + L * NF);
    mlp_forward(s, x, z1, a1, z2, a2, y);
    double dz3[16], da2[ORC_MAXD], dz2[ORC_MAXD], da1[ORC_MAXD], dz1[ORC_MAXD], dx[ORC_MAXD];
    for (int32_t j = 0; j < O; ++j) dz3[j] = d_out[r * O + j] * y[j] * (1.0 - y[j]);
    for (int32_t j = 0; j < O; ++j)
      for (int32_t i = 0; i < H; ++i) gw3[(size_t)j * H + i] += dz3[j] * a2[i];
    for (int32_t i = 0; i < H; ++i) {
      double acc = 0.0;
      for (int32_t j = 0; j < O; ++j) acc += s->w3[(size_t)j * H + i] * dz3[j];
      da2[i] = acc;
      dz2[i] = z2[i] > 0.0 ? acc : 0.0;
    }
    for (int32_t j = 0; j < H; ++j)
      for (int32_t i = 0; i < H; ++i) gw2[(size_t)j * H + i] += dz2[j] * a1[i];
    for (int32_t i = 0; i < H; ++i) {
      double acc = 0.0;
      for (int32_t j = 0; j < H; ++j) acc += s->w2[(size_t)j * H + i] * dz2[j];
      da1[i] = acc;
      dz1[i] = z1[i] > 0.0 ? acc : 0.0;
    }
    for (int32_t j = 0; j < H; ++j)
      for (int32_t i = 0; i < D; ++i) gw1[(size_t)j * D + i] += dz1[j] * x[i];
    for (int32_t i = 0; i < L * NF; ++i) {
      double acc = 0.0;
      for (int32_t j = 0; j < H; ++j) acc += s->w1[(size_t)j * D + i] * dz1[j];
      dx[i] = acc;
    }
    for (int32_t l = 0; l < L; ++l)
      for (int c = 0; c < 8; ++c) {
        int64_t i = idx[l * 8 + c];
        if (i < 0) continue;
        for (int32_t k = 0; k < NF; ++k) gfeat[l][i * NF + k] += wts[l * 8 + c] * dx[l * NF + k];
      }
    (void)da2; (void)da1;
  }
}

/* Pre-activation values z1, z2 (hidden each) of the given rays: used by the
 * gradient check to find parameters whose perturbation crosses a ReLU kink. */
void orc_preacts(const void* h, const float* o, const float* d, int64_t n, double* z1_out, double* z2_out) {
  const orc_scene* s = (const orc_scene*)h;
  for (int64_t r = 0; r < n; ++r) {
    int32_t id;
    float tt;
    bvh_closest(s->bvh, o + 3 * r, d + 3 * r, &id, &tt, 0);
    double x[ORC_MAXD], z1[ORC_MAXD], a1[ORC_MAXD], z2[ORC_MAXD], a2[ORC_MAXD], y[16];
    if (id < 0) {
      for (int32_t j = 0; j < s->hidden; ++j) z1_out[r * s->hidden + j] = z2_out[r * s->hidden + j] = 0.0;
      continue;
    }
    shade_ray(s, o + 3 * r, d + 3 * r, tt, y, x);
    mlp_forward(s, x, z1, a1, z2, a2, y);
    memcpy(z1_out + r * s->hidden, z1, sizeof(double) * (size_t)s->hidden);
    memcpy(z2_out + r * s->hidden, z2, sizeof(double) * (size_t)s->hidden);
  }
}

/* ------------------------------------------------------------------------ */
/* PSH check (Eq. 1): h(p) = h0(p) + Phi[h1(p)] with h0 = p mod m,           */
/* h1 = p mod r per axis, Phi entries packed 10 bits per axis, slot          */
/* linearised x + m (y + m z) after the per-axis sum mod m.  Used to verify  */
/* a hash built by the library: injective over the set, in range, equal to  */
/* the dense map.                                                            */
/* ------------------------------------------------------------------------ */
void orc_psh_slots(const uint32_t* phi, int32_t m, int32_t r, const int32_t* coords, int64_t n, int64_t* slots) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t h0[3], h1[3], ph[3];
    for (int q = 0; q < 3; ++q) {
      h0[q] = coords[3 * i + q] % m;
      h1[q] = coords[3 * i + q] % r;
    }
    uint32_t e = phi[h1[0] + (int64_t)r * (h1[1] + (int64_t)r * h1[2])];
    ph[0] = e & 1023u;
    ph[1] = (e >> 10) & 1023u;
    ph[2] = (e >> 20) & 1023u;
    int64_t s[3];
    for (int q = 0; q < 3; ++q) s[q] = (h0[q] + ph[q]) % m;
    slots[i] = s[0] + (int64_t)m * (s[1] + (int64_t)m * s[2]);
  }
}

/* ------------------------------------------------------------------------ */
/* 9. The decoupled variant (Sec. 4.2 "Hit Point Estimation and Opacity      */
/*    Refinement", "Diffuse and Specular Component", "Density Texture        */
/*    Cubes", "Diffuse Texture Cubes").                                      */
/*                                                                            */
/* Density: a field on the fine vertex lattice K = b r of the scene cube,    */
/* given as cubes: cube i covers base cell cells[i] and lists the values of  */
/* its (r+1)^3 vertices cells[i] r + (0..r)^3 (x fastest).  The value at a   */
/* vertex is the one listed by any cube that contains it, 0 when no cube     */
/* does.  The density at a point is the trilinear interpolation of its fine  */
/* cell's 8 vertices written as successive linear interpolations along x,   */
/* then y, then z, lerp(a, b, f) = a + f (b - a), in FP32 (the filtering a  */
/* texture unit performs; FP32 because it decides the argmax below).        */
/*                                                                            */
/* March: samples t_k = t0 + k delta (FP32), k = 0, 1, ... while t_k <= t1,  */
/* where [t0, t1] is the ray's span inside the scene cube (t0 >= 0).  With   */
/* T_0 = 1 and e_k = exp(-sigma_k delta):  w_k = T_k (1 - e_k),              */
/* T_{k+1} = T_k e_k (Eq. 4 evaluated sample by sample, FP32).  The march    */
/* stops after the sample that brings T below t_min.  The hit sample is the  */
/* first k of largest w_k; alpha_c = 1 - T at the stop (= sum_k w_k, the     */
/* accumulated weights of Eq. 5); the ray misses when alpha_c <= alpha_miss. */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t b, r;
  int64_t K, n;
  uint64_t* ckeys;  /* sorted base-cell keys of the listed cubes */
  int64_t* cidx;    /* cube index of ckeys[i] */
  const float* dens;
  const float* diff;
  float lo, scale, side, step, t_min, alpha_miss;
} orc_cubes;

static int cmp_u64pair(const void* a, const void* b) {
  const uint64_t x = ((const uint64_t*)a)[0], y = ((const uint64_t*)b)[0];
  return (x > y) - (x < y);
}

/* The density / diffuse arrays are referenced, not copied: the caller keeps
 * them alive while the handle exists. */
void* orc_cubes_create(int32_t b, int32_t r, int64_t n, const int32_t* cells, const float* dens, const float* diff,
                       float lo, float scale, float side, float step, float t_min, float alpha_miss) {
  if (b < 1 || r < 1 || n < 0 || !(step > 0.0f)) return 0;
  orc_cubes* c = (orc_cubes*)calloc(1, sizeof(orc_cubes));
  c->b = b; c->r = r; c->K = (int64_t)b * r; c->n = n;
  c->dens = dens; c->diff = diff;
  c->lo = lo; c->scale = scale; c->side = side; c->step = step; c->t_min = t_min; c->alpha_miss = alpha_miss;
  uint64_t* pairs = (uint64_t*)malloc(sizeof(uint64_t) * 2 * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) {
    pairs[2 * i] = pack_key(cells[3 * i], cells[3 * i + 1], cells[3 * i + 2]);
    pairs[2 * i + 1] = (uint64_t)i;
  }
  qsort(pairs, (size_t)n, 2 * sizeof(uint64_t), cmp_u64pair);
  c->ckeys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
  c->cidx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) { c->ckeys[i] = pairs[2 * i]; c->cidx[i] = (int64_t)pairs[2 * i + 1]; }
  free(pairs);
  return c;
}

void orc_cubes_free(void* h) {
  orc_cubes* c = (orc_cubes*)h;
  if (!c) return;
  free(c->ckeys);
  free(c->cidx);
  free(c);
}

/* Cube index and in-cube vertex offset of fine vertex v, or -1 when no cube
 * lists it.  Candidate cubes along an axis: v / r, and v / r - 1 when v is on
 * a cube face. */
static int64_t vertex_entry(const orc_cubes* c, const int64_t v[3], int64_t* at) {
  int64_t cand[3][2];
  int nc[3];
  for (int q = 0; q < 3; ++q) {
    nc[q] = 0;
    int64_t a = v[q] / c->r;
    if (a < c->b) cand[q][nc[q]++] = a;
    if (v[q] % c->r == 0 && a - 1 >= 0) cand[q][nc[q]++] = a - 1;
  }
  for (int iz = 0; iz < nc[2]; ++iz)
    for (int iy = 0; iy < nc[1]; ++iy)
      for (int ix = 0; ix < nc[0]; ++ix) {
        int64_t k = find_key(c->ckeys, c->n, pack_key(cand[0][ix], cand[1][iy], cand[2][iz]));
        if (k < 0) continue;
        int64_t lx = v[0] - cand[0][ix] * c->r, ly = v[1] - cand[1][iy] * c->r, lz = v[2] - cand[2][iz] * c->r;
        *at = lx + (int64_t)(c->r + 1) * (ly + (int64_t)(c->r + 1) * lz);
        return c->cidx[k];
      }
  return -1;
}

static float vertex_density(const orc_cubes* c, const int64_t v[3]) {
  int64_t at;
  int64_t i = vertex_entry(c, v, &at);
  return i < 0 ? 0.0f : c->dens[i * (int64_t)(c->r + 1) * (c->r + 1) * (c->r + 1) + at];
}

static float lerp32(float a, float b, float f) {
  float diff = b - a;
  float step = f * diff;
  return a + step;
}

/* fine cell and fractions of the point o + t d (the FP32 steps of cell_of at N = K) */
static void fine_cell(const orc_cubes* c, const float o[3], const float d[3], float t, int64_t cell[3],
                      float f[3]) {
  orc_domain dom = {c->lo, c->scale};
  int32_t ci[3];
  cell_of(dom, (int32_t)c->K, o, d, t, ci, f);
  for (int q = 0; q < 3; ++q) cell[q] = ci[q];
}

static float density_at(const orc_cubes* c, const float o[3], const float d[3], float t) {
  int64_t cell[3];
  float f[3];
  fine_cell(c, o, d, t, cell, f);
  float s[8];
  for (int k = 0; k < 8; ++k) {
    int64_t v[3] = {cell[0] + (k & 1), cell[1] + ((k >> 1) & 1), cell[2] + ((k >> 2) & 1)};
    s[k] = vertex_density(c, v);
  }
  float a00 = lerp32(s[0], s[1], f[0]);  /* y0 z0 */
  float a10 = lerp32(s[2], s[3], f[0]);  /* y1 z0 */
  float a01 = lerp32(s[4], s[5], f[0]);  /* y0 z1 */
  float a11 = lerp32(s[6], s[7], f[0]);  /* y1 z1 */
  float b0 = lerp32(a00, a10, f[1]);
  float b1 = lerp32(a01, a11, f[1]);
  return lerp32(b0, b1, f[2]);
}

void orc_density(const void* h, const float* o, const float* d, const float* t, int64_t n, float* sigma) {
  const orc_cubes* c = (const orc_cubes*)h;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) sigma[i] = density_at(c, o + 3 * i, d + 3 * i, t[i]);
}

/* Span [t0, t1] of the ray inside the scene cube [lo, lo + side]^3 (slab
 * test in FP32: per axis (plane - o) / d, axes with d = 0 only test o).
 * Returns 0 when the ray does not enter it. */
static int cube_span(const orc_cubes* c, const float o[3], const float d[3], float* t0, float* t1) {
  const float lo = c->lo, hi = c->lo + c->side;
  float a = 0.0f, z = INFINITY;
  for (int q = 0; q < 3; ++q) {
    if (d[q] == 0.0f) {
      if (o[q] < lo || o[q] > hi) return 0;
      continue;
    }
    float ta = (lo - o[q]) / d[q];
    float tb = (hi - o[q]) / d[q];
    float tn = ta < tb ? ta : tb, tf = ta < tb ? tb : ta;
    if (tn > a) a = tn;
    if (tf < z) z = tf;
  }
  if (a > z) return 0;
  *t0 = a;
  *t1 = z;
  return 1;
}

typedef struct {
  int32_t k;      /* hit sample, -1 = miss */
  float t;        /* its t (0 on miss) */
  float alpha;    /* alpha_c = 1 - T at the stop */
  float wmax;     /* largest weight */
  int32_t k2;     /* sample of the second largest weight (-1 if none) */
  float w2;
  int32_t n;      /* samples taken */
  float T_prev;   /* transmittance before the last sample (stop-decision margin) */
} orc_march_res;

static void march_ray(const orc_cubes* c, const float o[3], const float d[3], orc_march_res* m) {
  m->k = -1; m->t = 0.0f; m->alpha = 0.0f; m->wmax = 0.0f; m->k2 = -1; m->w2 = 0.0f; m->n = 0; m->T_prev = 1.0f;
  float t0, t1;
  if (!cube_span(c, o, d, &t0, &t1)) return;
  float T = 1.0f;
  int32_t kbest = -1;
  float tbest = 0.0f;
  for (int32_t k = 0;; ++k) {
    float t = t0 + (float)k * c->step;
    if (t > t1) break;
    m->n = k + 1;
    float sigma = density_at(c, o, d, t);
    float e = expf(-(sigma * c->step));
    float w = T * (1.0f - e);
    m->T_prev = T;
    T = T * e;
    if (w > m->wmax) {
      m->w2 = m->wmax; m->k2 = kbest;
      m->wmax = w; kbest = k; tbest = t;
    } else if (w > m->w2) {
      m->w2 = w; m->k2 = k;
    }
    if (T < c->t_min) break;
  }
  m->alpha = 1.0f - T;
  if (m->alpha > c->alpha_miss && kbest >= 0) {
    m->k = kbest;
    m->t = tbest;
  }
}

/* Stage output of the march for n explicit rays (any output may be NULL). */
void orc_march(const void* h, const float* o, const float* d, int64_t n, int32_t* k, float* t, float* alpha,
               float* wmax, int32_t* k2, float* w2, int32_t* nsamp, float* T_prev) {
  const orc_cubes* c = (const orc_cubes*)h;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) {
    orc_march_res m;
    march_ray(c, o + 3 * i, d + 3 * i, &m);
    if (k) k[i] = m.k;
    if (t) t[i] = m.t;
    if (alpha) alpha[i] = m.alpha;
    if (wmax) wmax[i] = m.wmax;
    if (k2) k2[i] = m.k2;
    if (w2) w2[i] = m.w2;
    if (nsamp) nsamp[i] = m.n;
    if (T_prev) T_prev[i] = m.T_prev;
  }
}

/* Diffuse (c_d r, g, b, tint) at the point o + t d: FP64 trilinear of the 4
 * channels of its fine cell's vertices, weights prod_axis (bit ? f : 1 - f).
 * Returns the number of corners no cube lists (their channels count as 0). */
static int diffuse_at(const orc_cubes* c, const float o[3], const float d[3], float t, double out[4]) {
  int64_t cell[3];
  float f[3];
  fine_cell(c, o, d, t, cell, f);
  int missing = 0;
  for (int ch = 0; ch < 4; ++ch) out[ch] = 0.0;
  const int64_t nv = (int64_t)(c->r + 1) * (c->r + 1) * (c->r + 1);
  for (int k = 0; k < 8; ++k) {
    int64_t v[3] = {cell[0] + (k & 1), cell[1] + ((k >> 1) & 1), cell[2] + ((k >> 2) & 1)};
    double w = 1.0;
    for (int q = 0; q < 3; ++q) w *= ((k >> q) & 1) ? (double)f[q] : 1.0 - (double)f[q];
    int64_t at;
    int64_t i = vertex_entry(c, v, &at);
    if (i < 0 || !c->diff) { ++missing; continue; }
    const float* p = c->diff + (size_t)(i * nv + at) * 4;
    for (int ch = 0; ch < 4; ++ch) out[ch] += w * (double)p[ch];
  }
  return missing;
}

/* Shading of the variant at a given hit: x = [E(P), SH(d), alpha_c] (Eq. 5),
 * (c_s, alpha) = F_s(x), (c_d, tint) from the diffuse cubes, c = c_d + tint
 * c_s (Eq. 7); rgba = (c, alpha).  Returns missing corner lookups. */
static int64_t shade_variant(const orc_scene* s, const orc_cubes* c, const float o[3], const float d[3], float t,
                             float alpha_c, double* rgba) {
  double x[ORC_MAXD], z1[ORC_MAXD], a1[ORC_MAXD], z2[ORC_MAXD], a2[ORC_MAXD], out[8];
  int64_t miss = encode_ray(s, o, d, t, x, 0, 0);
  double dir[3] = {d[0], d[1], d[2]};
  orc_sh16(dir, x + s->L * s->nfeat);
  x[s->L * s->nfeat + 16] = (double)alpha_c;
  mlp_forward(s, x, z1, a1, z2, a2, out);
  double df[4];
  miss += diffuse_at(c, o, d, t, df);
  for (int ch = 0; ch < 3; ++ch) rgba[ch] = df[ch] + df[3] * out[ch];
  rgba[3] = out[3];
  return miss;
}

void orc_shade_variant_at(const void* hs, const void* hc, const float* o, const float* d, const float* t,
                          const float* alpha_c, int64_t n, double* rgba) {
  const orc_scene* s = (const orc_scene*)hs;
  const orc_cubes* c = (const orc_cubes*)hc;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) shade_variant(s, c, o + 3 * i, d + 3 * i, t[i], alpha_c[i], rgba + 4 * i);
}

/* The variant end to end for explicit rays or for pixels of one view
 * (cam != NULL: pix = j * W + i, NULL = all).  k / t / alpha may be NULL.
 * Misses render (0, 0, 0, 0).  Returns missing corner lookups. */
static int64_t render_variant_one(const orc_scene* s, const orc_cubes* c, const float o[3], const float d[3],
                                  double* rgba, int32_t* k, float* t, float* alpha) {
  orc_march_res m;
  march_ray(c, o, d, &m);
  if (k) *k = m.k;
  if (t) *t = m.t;
  if (alpha) *alpha = m.alpha;
  if (m.k < 0) {
    for (int ch = 0; ch < 4; ++ch) rgba[ch] = 0.0;
    return 0;
  }
  return shade_variant(s, c, o, d, m.t, m.alpha, rgba);
}

int64_t orc_render_variant_rays(const void* hs, const void* hc, const float* o, const float* d, int64_t n,
                                double* rgba, int32_t* k, float* t, float* alpha) {
  const orc_scene* s = (const orc_scene*)hs;
  const orc_cubes* c = (const orc_cubes*)hc;
  int64_t missing = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : missing)
  for (int64_t i = 0; i < n; ++i)
    missing += render_variant_one(s, c, o + 3 * i, d + 3 * i, rgba + 4 * i, k ? k + i : 0, t ? t + i : 0,
                                  alpha ? alpha + i : 0);
  return missing;
}

int64_t orc_render_variant_pixels(const void* hs, const void* hc, const float* cam, int32_t W, int32_t H,
                                  const int64_t* pix, int64_t n, double* rgba, int32_t* k, float* t, float* alpha) {
  const orc_scene* s = (const orc_scene*)hs;
  const orc_cubes* c = (const orc_cubes*)hc;
  int64_t missing = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : missing)
  for (int64_t i = 0; i < n; ++i) {
    int64_t p = pix ? pix[i] : i;
    float o[3], d[3];
    orc_ray(cam, W, H, (int32_t)(p % W), (int32_t)(p / W), o, d);
    missing += render_variant_one(s, c, o, d, rgba + 4 * i, k ? k + i : 0, t ? t + i : 0, alpha ? alpha + i : 0);
  }
  return missing;
}

/* ------------------------------------------------------------------------ */
/* 10. Depth fusion of several objects (the frame composer of Sec. 5.1,     */
/*     which merges the per-object renders of a frame "according to the     */
/*     depth").  Reading: objects are placed by translation, so a ray's t is */
/*     the same in the world and in each object's frame; the ray's hits on   */
/*     all objects are ordered by (t, object index), the first K are kept,   */
/*     and they are composited front to back with the straight-alpha "over"  */
/*     operator,                                                             */
/*         C <- C + (1 - A) a c,   A <- A + (1 - A) a,                       */
/*     starting from C = 0, A = 0.  The pixel stores the straight colour     */
/*     C / A and the coverage A, or (0, 0, 0, 0) when A = 0.                 */
/*     Inputs, per object k and ray r (object-major): hit[k][r] (non-zero =  */
/*     hit), t[k][r], rgba[k][r][4] straight RGBA of that object's render.   */
/*     Output out[r][4]; used[r] (optional) = hits composited (<= K).        */
/* ------------------------------------------------------------------------ */
#define ORC_MAX_OBJECTS 64

void orc_composite(int32_t n_obj, int64_t n, const int32_t* hit, const float* t, const double* rgba, int32_t K,
                   double* out, int32_t* used) {
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < n; ++r) {
    int32_t order[ORC_MAX_OBJECTS];
    int32_t m = 0;
    /* insertion into a list sorted by (t, object index) */
    for (int32_t k = 0; k < n_obj && k < ORC_MAX_OBJECTS; ++k) {
      if (!hit[(int64_t)k * n + r]) continue;
      const float tk = t[(int64_t)k * n + r];
      int32_t pos = m;
      while (pos > 0) {
        const int32_t q = order[pos - 1];
        const float tq = t[(int64_t)q * n + r];
        if (tq < tk || (tq == tk && q < k)) break;
        order[pos] = q;
        --pos;
      }
      order[pos] = k;
      ++m;
    }
    if (m > K) m = K;
    double C[3] = {0.0, 0.0, 0.0}, A = 0.0;
    for (int32_t i = 0; i < m; ++i) {
      const double* c = rgba + ((int64_t)order[i] * n + r) * 4;
      const double w = (1.0 - A) * c[3];
      C[0] += w * c[0];
      C[1] += w * c[1];
      C[2] += w * c[2];
      A += w;
    }
    double* o = out + r * 4;
    if (A > 0.0) {
      o[0] = C[0] / A;
      o[1] = C[1] / A;
      o[2] = C[2] / A;
      o[3] = A;
    } else {
      o[0] = o[1] = o[2] = o[3] = 0.0;
    }
    if (used) used[r] = m;
  }
}

int32_t orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int32_t n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
