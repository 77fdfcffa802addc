// Host side of libinolf.so: error reporting, the perfect spatial hash
// builder (Sec. 4.1, Eq. 1), the BVH builder for the geometry proxy and the
// upload of an object into device memory.
#include <cuda_runtime.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <thread>
#include <vector>

#include "inolf_internal.h"

namespace inolf {

static thread_local std::string g_err;

inolf_status fail(inolf_status st, const std::string& msg) {
  g_err = msg;
  return st;
}
void clear_error() { g_err.clear(); }
const char* last_error_cstr() { return g_err.c_str(); }

}  // namespace inolf

using namespace inolf;

extern "C" const char* inolf_last_error(void) { return inolf::last_error_cstr(); }
extern "C" const char* inolf_version(void) { return "inolf-gb300 0.1 (sm_103a)"; }

// ===========================================================================
// Perfect spatial hash (Sec. 4.1, Eq. 1).
//
// h0(p) = p mod m and h1(p) = p mod r per axis.  With gcd(m, r) = 1 and
// m r > extent, p -> (h0(p), h1(p)) is injective on [0, extent]^3 (Chinese
// remainder theorem), so a collision-free offset table Phi exists in
// principle.  Phi is filled greedily, in the manner of Lefebvre and Hoppe
// (2006): points are grouped by q = h1(p); groups are placed largest first
// (by size class, and in q order within a class); for each group, offsets
// already chosen by its 6 neighbours in the offset
// table are tried first (so that neighbouring points land in neighbouring
// slots), then every offset that puts the group's first point on a free
// slot, scanning free slots from a seeded start.  A group that fits nowhere
// makes the attempt fail; r (then m) is grown and the construction restarts.
// ===========================================================================
namespace {

uint64_t mix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

int64_t gcd64(int64_t a, int64_t b) {
  while (b) { int64_t t = a % b; a = b; b = t; }
  return a;
}

struct PshResult {
  std::vector<uint32_t> phi;
  std::vector<uint32_t> slot_of;
};

enum TryStatus { TRY_OK, TRY_FULL, TRY_DUPLICATE };

TryStatus psh_try(const int32_t* coords, int64_t n, int32_t m, int32_t r, uint64_t seed, PshResult& res) {
  const int64_t R3 = (int64_t)r * r * r;
  const int64_t M3 = (int64_t)m * m * m;
  const int64_t Mm = (int64_t)m * m;
  // group points by q = h1(p) (counting sort)
  std::vector<uint32_t> start(R3 + 1, 0);
  std::vector<uint32_t> qof(n);
  for (int64_t i = 0; i < n; ++i) {
    const int32_t* p = coords + 3 * i;
    uint32_t q = (uint32_t)((p[0] % r) + (int64_t)r * ((p[1] % r) + (int64_t)r * (p[2] % r)));
    qof[i] = q;
    start[q + 1]++;
  }
  uint32_t max_size = 0;
  for (int64_t q = 0; q < R3; ++q) max_size = std::max(max_size, start[q + 1]);
  for (int64_t q = 0; q < R3; ++q) start[q + 1] += start[q];
  std::vector<uint32_t> members(n);
  {
    std::vector<uint32_t> fill(start.begin(), start.end() - 1);
    for (int64_t i = 0; i < n; ++i) members[fill[qof[i]]++] = (uint32_t)i;
  }
  std::vector<uint32_t>().swap(qof);
  // group order: size class descending (class = bit length of the size, so
  // groups of similar size are placed together), then q ascending, which
  // visits neighbouring groups of a class one after the other
  auto size_class = [](uint32_t k) { return k ? 32 - __builtin_clz(k) : 0; };
  const uint32_t max_class = (uint32_t)size_class(max_size);
  std::vector<uint32_t> size_start(max_class + 2, 0);
  for (int64_t q = 0; q < R3; ++q) size_start[max_class - size_class(start[q + 1] - start[q]) + 1]++;
  for (uint32_t s = 0; s <= max_class; ++s) size_start[s + 1] += size_start[s];
  std::vector<uint32_t> order(R3);
  for (int64_t q = 0; q < R3; ++q) order[size_start[max_class - size_class(start[q + 1] - start[q])]++] = (uint32_t)q;

  std::vector<uint64_t> used((M3 + 63) / 64, 0);
  res.phi.assign(R3, 0);
  res.slot_of.assign(n, 0);
  std::vector<uint8_t> assigned(R3, 0);
  std::vector<int32_t> hx, hy, hz;
  std::vector<uint32_t> slots;

  auto try_offset = [&](uint32_t k, int32_t px, int32_t py, int32_t pz) -> bool {
    for (uint32_t a = 0; a < k; ++a) {
      int32_t sx = hx[a] + px; if (sx >= m) sx -= m;
      int32_t sy = hy[a] + py; if (sy >= m) sy -= m;
      int32_t sz = hz[a] + pz; if (sz >= m) sz -= m;
      uint64_t s = (uint64_t)sx + (uint64_t)m * ((uint64_t)sy + (uint64_t)m * (uint64_t)sz);
      if ((used[s >> 6] >> (s & 63)) & 1ull) return false;
      slots[a] = (uint32_t)s;
    }
    return true;
  };

  for (int64_t oi = 0; oi < R3; ++oi) {
    const uint32_t q = order[oi];
    const uint32_t k = start[q + 1] - start[q];
    if (k == 0) break;  // size classes are descending
    hx.resize(k); hy.resize(k); hz.resize(k); slots.resize(k);
    for (uint32_t a = 0; a < k; ++a) {
      const int32_t* p = coords + 3 * (int64_t)members[start[q] + a];
      hx[a] = p[0] % m; hy[a] = p[1] % m; hz[a] = p[2] % m;
    }
    if (k > 1) {  // two points with the same (h0, h1) are the same point
      std::vector<uint64_t> lin(k);
      for (uint32_t a = 0; a < k; ++a) lin[a] = (uint64_t)hx[a] + (uint64_t)m * (hy[a] + (uint64_t)m * hz[a]);
      std::sort(lin.begin(), lin.end());
      for (uint32_t a = 1; a < k; ++a)
        if (lin[a] == lin[a - 1]) return TRY_DUPLICATE;
    }
    bool ok = false;
    int32_t fx = 0, fy = 0, fz = 0;
    // 1) offsets of the 6 neighbours in the offset table (coherence)
    const int32_t qx = (int32_t)(q % r), qy = (int32_t)((q / r) % r), qz = (int32_t)(q / ((uint32_t)r * r));
    const int32_t nb[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
    for (int e = 0; e < 6 && !ok; ++e) {
      int32_t ax = (qx + nb[e][0] + r) % r, ay = (qy + nb[e][1] + r) % r, az = (qz + nb[e][2] + r) % r;
      uint32_t nq = (uint32_t)(ax + (int64_t)r * (ay + (int64_t)r * az));
      if (!assigned[nq]) continue;
      uint32_t e32 = res.phi[nq];
      fx = (int32_t)(e32 & 1023u); fy = (int32_t)((e32 >> 10) & 1023u); fz = (int32_t)((e32 >> 20) & 1023u);
      ok = try_offset(k, fx, fy, fz);
    }
    // 2) every offset that puts the first point on a free slot
    if (!ok) {
      const uint64_t s0 = mix64(seed ^ ((uint64_t)q * 0x9E37ull)) % (uint64_t)M3;
      const int64_t nwords = (int64_t)used.size();
      int64_t w = (int64_t)(s0 >> 6);
      uint64_t first_mask = ~0ull << (s0 & 63);
      for (int64_t step = 0; step <= nwords && !ok; ++step) {
        uint64_t freebits = ~used[w];
        if (step == 0) freebits &= first_mask;
        if (step == nwords) freebits &= ~first_mask;  // wrapped back to the first word
        while (freebits && !ok) {
          int b = __builtin_ctzll(freebits);
          freebits &= freebits - 1;
          int64_t s = w * 64 + b;
          if (s >= M3) break;
          int32_t sx = (int32_t)(s % m), sy = (int32_t)((s / m) % m), sz = (int32_t)(s / Mm);
          fx = sx - hx[0]; if (fx < 0) fx += m;
          fy = sy - hy[0]; if (fy < 0) fy += m;
          fz = sz - hz[0]; if (fz < 0) fz += m;
          ok = try_offset(k, fx, fy, fz);
        }
        if (++w == nwords) w = 0;
      }
    }
    if (!ok) return TRY_FULL;
    res.phi[q] = (uint32_t)fx | ((uint32_t)fy << 10) | ((uint32_t)fz << 20);
    assigned[q] = 1;
    for (uint32_t a = 0; a < k; ++a) {
      used[slots[a] >> 6] |= 1ull << (slots[a] & 63);
      res.slot_of[members[start[q] + a]] = slots[a];
    }
  }
  return TRY_OK;
}

}  // namespace

extern "C" inolf_status inolf_build_hash(const int32_t* coords, int64_t n, int32_t grid_extent,
                                         const inolf_hash_params* params, inolf_hash** out) {
  clear_error();
  if (!out) return fail(INOLF_E_INVALID, "inolf_build_hash: out is NULL");
  *out = nullptr;
  if (n < 0 || (n > 0 && !coords)) return fail(INOLF_E_INVALID, "inolf_build_hash: bad coords / n");
  if (grid_extent < 0 || grid_extent > (1 << 21) - 1) return fail(INOLF_E_INVALID, "inolf_build_hash: bad grid_extent");
  if (n > 0xFFFFFFFFll) return fail(INOLF_E_INVALID, "inolf_build_hash: n too large");
  inolf_hash_params p = {1.0 / 6.0, 1.0, 8, 0};
  if (params) p = *params;
  if (!(p.sigma > 0) || !(p.slot_slack >= 1.0) || p.max_retries < 0)
    return fail(INOLF_E_INVALID, "inolf_build_hash: bad params");
  for (int64_t i = 0; i < 3 * n; ++i)
    if (coords[i] < 0 || coords[i] > grid_extent)
      return fail(INOLF_E_INVALID, "inolf_build_hash: coordinate outside [0, grid_extent]");
  const int64_t extent1 = (int64_t)grid_extent + 1;
  auto cube_root_ceil = [](double v) {
    int64_t c = (int64_t)std::ceil(std::cbrt(std::max(v, 1.0)));
    while (c > 1 && (double)(c - 1) * (c - 1) * (c - 1) >= v) --c;
    while ((double)c * c * c < v) ++c;
    return c;
  };
  int64_t m = cube_root_ceil((double)n * p.slot_slack);
  int64_t r = cube_root_ceil(p.sigma * (double)n);
  for (int attempt = 0; attempt <= p.max_retries; ++attempt) {
    while (gcd64(m, r) != 1 || m * r < extent1) ++r;
    if (m > 1024) return fail(INOLF_E_INVALID, "inolf_build_hash: table side m > 1024 (too many points)");
    if (r * r * r > (int64_t)1 << 31) return fail(INOLF_E_HASH_FAILED, "inolf_build_hash: offset table too large");
    PshResult res;
    TryStatus st;
    try {
      st = psh_try(coords, n, (int32_t)m, (int32_t)r, p.seed, res);
    } catch (const std::bad_alloc&) {
      return fail(INOLF_E_OOM, "inolf_build_hash: out of host memory");
    }
    if (st == TRY_DUPLICATE) return fail(INOLF_E_INVALID, "inolf_build_hash: duplicate points");
    if (st == TRY_OK) {
      inolf_hash* h = (inolf_hash*)std::calloc(1, sizeof(inolf_hash));
      if (!h) return fail(INOLF_E_OOM, "inolf_build_hash: out of host memory");
      h->m = (int32_t)m; h->r = (int32_t)r; h->n = n;
      h->phi = (uint32_t*)std::malloc(sizeof(uint32_t) * res.phi.size());
      h->slot_of = (uint32_t*)std::malloc(sizeof(uint32_t) * (n > 0 ? n : 1));
      h->coords = (int32_t*)std::malloc(sizeof(int32_t) * 3 * (n > 0 ? n : 1));
      if (!h->phi || !h->slot_of || !h->coords) { inolf_hash_free(h); return fail(INOLF_E_OOM, "inolf_build_hash: oom"); }
      std::memcpy(h->phi, res.phi.data(), sizeof(uint32_t) * res.phi.size());
      if (n) std::memcpy(h->slot_of, res.slot_of.data(), sizeof(uint32_t) * n);
      if (n) std::memcpy(h->coords, coords, sizeof(int32_t) * 3 * n);
      *out = h;
      return INOLF_OK;
    }
    // grow the offset table first, then the hash table
    r += std::max<int64_t>(1, r / 8);
    if (attempt % 2 == 1) m += std::max<int64_t>(1, m / 64);
  }
  return fail(INOLF_E_HASH_FAILED, "inolf_build_hash: no collision-free offset table after max_retries");
}

extern "C" void inolf_hash_free(inolf_hash* h) {
  if (!h) return;
  std::free(h->phi);
  std::free(h->slot_of);
  std::free(h->coords);
  std::free(h);
}

// ===========================================================================
// BVH over the proxy triangles: binary, binned SAH (16 bins per axis), leaves
// of at most 8 triangles.  Each node stores the boxes of both children so the
// traversal tests two boxes per node fetch.  Boxes are padded outwards by
// 1e-5 (1 + |coordinate|) so that FP32 slab tests never reject a box that
// holds an accepted triangle hit.
// ===========================================================================
namespace {

struct Box {
  float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  void grow(const float* p) {
    for (int k = 0; k < 3; ++k) { lo[k] = std::min(lo[k], p[k]); hi[k] = std::max(hi[k], p[k]); }
  }
  void grow(const Box& b) {
    for (int k = 0; k < 3; ++k) { lo[k] = std::min(lo[k], b.lo[k]); hi[k] = std::max(hi[k], b.hi[k]); }
  }
  float area() const {
    float d[3];
    for (int k = 0; k < 3; ++k) d[k] = std::max(0.0f, hi[k] - lo[k]);
    return 2.0f * (d[0] * d[1] + d[1] * d[2] + d[2] * d[0]);
  }
  bool empty() const { return lo[0] > hi[0]; }
};

struct ChildRef {
  Box box;
  int32_t index = -1;  // inner: node index; leaf: first triangle slot
  int32_t count = 0;   // > 0: leaf with this many triangles
};

struct Builder {
  const float* V;
  const int32_t* F;
  std::vector<Box> tb;
  std::vector<float> cen;
  std::vector<int32_t> idx;
  std::vector<float> nodes;  // 16 floats per node
  int max_depth = 0;
  static constexpr int kBins = 16;
  static constexpr int kMaxLeaf = 8;

  ChildRef make(int32_t first, int32_t count, int depth = 0) {
    ChildRef ref;
    max_depth = std::max(max_depth, depth);
    Box cb;
    for (int32_t i = first; i < first + count; ++i) {
      ref.box.grow(tb[idx[i]]);
      cb.grow(&cen[3 * idx[i]]);
    }
    auto leaf = [&]() { ref.index = first; ref.count = count; return ref; };
    if (count <= 2) return leaf();
    // binned SAH over centroid bounds
    float best_cost = INFINITY;
    int best_axis = -1, best_split = -1;
    for (int a = 0; a < 3; ++a) {
      float ext = cb.hi[a] - cb.lo[a];
      if (!(ext > 0)) continue;
      Box bb[kBins];
      int bc[kBins] = {0};
      for (int32_t i = first; i < first + count; ++i) {
        int b = std::min(kBins - 1, (int)((cen[3 * idx[i] + a] - cb.lo[a]) * (kBins / ext)));
        bc[b]++;
        bb[b].grow(tb[idx[i]]);
      }
      float left_area[kBins];
      int left_count[kBins];
      Box acc;
      int cnt = 0;
      for (int b = 0; b < kBins - 1; ++b) {
        acc.grow(bb[b]); cnt += bc[b];
        left_area[b] = acc.area(); left_count[b] = cnt;
      }
      Box racc;
      int rcnt = 0;
      for (int b = kBins - 1; b > 0; --b) {
        racc.grow(bb[b]); rcnt += bc[b];
        int lc = left_count[b - 1];
        if (lc == 0 || rcnt == 0) continue;
        float cost = left_area[b - 1] * lc + racc.area() * rcnt;
        if (cost < best_cost) { best_cost = cost; best_axis = a; best_split = b; }
      }
    }
    const float leaf_cost = ref.box.area() * count;
    if (best_axis < 0 || (count <= kMaxLeaf && best_cost + ref.box.area() >= leaf_cost)) {
      if (count <= kMaxLeaf) return leaf();
    }
    int32_t mid;
    int split_axis = 0;  // the left child holds the lower centroids along this axis
    if (best_axis >= 0) {
      split_axis = best_axis;
      const int a = best_axis;
      const float ext = cb.hi[a] - cb.lo[a];
      auto it = std::partition(idx.begin() + first, idx.begin() + first + count, [&](int32_t t) {
        int b = std::min(kBins - 1, (int)((cen[3 * t + a] - cb.lo[a]) * (kBins / ext)));
        return b < best_split;
      });
      mid = (int32_t)(it - idx.begin());
    } else {
      mid = first;
    }
    if (mid == first || mid == first + count) {  // degenerate: median by (centroid x, id)
      mid = first + count / 2;
      split_axis = 0;
      std::nth_element(idx.begin() + first, idx.begin() + mid, idx.begin() + first + count,
                       [&](int32_t x, int32_t y) { return cen[3 * x] < cen[3 * y] || (cen[3 * x] == cen[3 * y] && x < y); });
    }
    int32_t node = (int32_t)(nodes.size() / 16);
    nodes.resize(nodes.size() + 16);
    ChildRef l = make(first, mid - first, depth + 1);
    ChildRef r = make(mid, first + count - mid, depth + 1);
    write_node(node, l, r, split_axis);
    ref.index = node;
    ref.count = 0;
    return ref;
  }

  static float pad_lo(float v) { return (float)((double)v - 1e-5 * (1.0 + std::fabs((double)v))); }
  static float pad_hi(float v) { return (float)((double)v + 1e-5 * (1.0 + std::fabs((double)v))); }

  void write_node(int32_t node, const ChildRef& l, const ChildRef& r, int split_axis) {
    float* nd = &nodes[16 * (size_t)node];
    const ChildRef* c[2] = {&l, &r};
    // layout: [lx0 lx1 rx0 rx1] [ly0 ly1 ry0 ry1] [lz0 lz1 rz0 rz1] [l.index l.count r.index r.count]
    // where each count word is (triangles of a leaf, 0 for an inner node) | split axis << 4
    for (int k = 0; k < 3; ++k)
      for (int s = 0; s < 2; ++s) {
        const Box& b = c[s]->box;
        if (b.empty() || c[s]->index < 0) {
          nd[4 * k + 2 * s + 0] = INFINITY;   // lo > hi: never entered (the traversal's signed slab test relies on it)
          nd[4 * k + 2 * s + 1] = -INFINITY;
        } else {
          nd[4 * k + 2 * s + 0] = pad_lo(b.lo[k]);
          nd[4 * k + 2 * s + 1] = pad_hi(b.hi[k]);
        }
      }
    static_assert(kMaxLeaf < 16, "leaf counts take the low 4 bits of a count word");
    int32_t meta[4] = {l.index, l.count | (split_axis << 4), r.index, r.count | (split_axis << 4)};
    std::memcpy(nd + 12, meta, sizeof(meta));
  }
};

}  // namespace

// ===========================================================================
// Objects
// ===========================================================================
#define CUDA_TRY(call)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      destroy_object(o);                                                                   \
      return fail(INOLF_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));      \
    }                                                                                      \
  } while (0)

// FP32 weights packed for the SIMT kernels (W1T [d_in][64], W2 [64][64],
// W3T [64][4]) and the tensor-core blobs, into existing buffers when present.
namespace inolf {
inolf_status upload_weights(Object& o, const float* w1, const float* w2, const float* w3, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const int din = o.d_in, H = INOLF_HIDDEN, O = INOLF_OUT;
  std::vector<float> w((size_t)din * H + H * H + H * O);
  for (int j = 0; j < H; ++j)
    for (int i = 0; i < din; ++i) w[(size_t)i * H + j] = w1[(size_t)j * din + i];
  std::memcpy(&w[(size_t)din * H], w2, sizeof(float) * H * H);
  for (int j = 0; j < O; ++j)
    for (int i = 0; i < H; ++i) w[(size_t)din * H + H * H + (size_t)i * O + j] = w3[(size_t)j * H + i];
  if (!o.w_f32) {
    if (cudaMalloc(&o.w_f32, w.size() * sizeof(float)) != cudaSuccess) return fail(INOLF_E_OOM, "cudaMalloc weights");
    o.bytes += w.size() * sizeof(float);
  }
  if (cudaMemcpyAsync(o.w_f32, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(INOLF_E_CUDA, "upload weights");
  return prepare_tc_weights(o, w1, w2, w3, stream);
}
}  // namespace inolf

static void destroy_object(Object& o) {
  auto f = [](void* p) { if (p) cudaFree(p); };
  f(o.nodes); f(o.tris); f(o.w_f32); f(o.w_bf16); f(o.w_fp8); f(o.w_tf32); f(o.w_scale_dev);
  f((void*)o.cub.grid); f((void*)o.cub.dens); f((void*)o.cub.diff); f((void*)o.cub.fdist); f((void*)o.cub.bdist);
  for (int l = 0; l < o.L; ++l) {
    f((void*)o.lv[l].phi); f((void*)o.lv[l].table); f((void*)o.lv[l].bundle); f((void*)o.pts[l]);
  }
  o = Object();
}

// Octant distances of an n^3 grid of cells with obstacles: for every cell
// and every octant s (bit q set: axis q decreasing, else increasing), the
// largest D <= cap such that the block of D^3 cells that starts at the cell
// and extends along s holds no obstacle (0 for an obstacle).  The block of
// size D is empty exactly when the cell is empty and the blocks of size D - 1
// of its 7 forward neighbours are, so one sweep against s per octant gives
// D = 1 + min over those neighbours (cells beyond the grid do not constrain).
// out: [8][n^3], cell x + n (y + n z).
static void octant_distance(const uint8_t* obstacle, int32_t n, int32_t cap, uint8_t* out) {
  const int64_t n3 = (int64_t)n * n * n;
  for (int oct = 0; oct < 8; ++oct) {
    const int32_t s[3] = {(oct & 1) ? -1 : 1, (oct & 2) ? -1 : 1, (oct & 4) ? -1 : 1};
    uint8_t* D = out + (size_t)oct * n3;
    for (int32_t iz = 0; iz < n; ++iz) {
      const int32_t z = s[2] > 0 ? n - 1 - iz : iz;
      for (int32_t iy = 0; iy < n; ++iy) {
        const int32_t y = s[1] > 0 ? n - 1 - iy : iy;
        for (int32_t ix = 0; ix < n; ++ix) {
          const int32_t x = s[0] > 0 ? n - 1 - ix : ix;
          const int64_t c = x + (int64_t)n * (y + (int64_t)n * z);
          if (obstacle[c]) {
            D[c] = 0;
            continue;
          }
          int32_t m = cap;
          for (int e = 1; e < 8; ++e) {
            const int32_t nx = x + ((e & 1) ? s[0] : 0), ny = y + ((e & 2) ? s[1] : 0), nz = z + ((e & 4) ? s[2] : 0);
            if (nx < 0 || ny < 0 || nz < 0 || nx >= n || ny >= n || nz >= n) continue;
            m = std::min<int32_t>(m, D[nx + (int64_t)n * (ny + (int64_t)n * nz)]);
          }
          D[c] = (uint8_t)std::min<int32_t>(cap, m + 1);
        }
      }
    }
  }
}

// Uploads the density / diffuse cubes and builds the base grid of cube
// indices and empty-space distances.
static inolf_status create_cubes(Object& o, const inolf_cubes_desc& C, cudaStream_t st) {
  const int32_t b = C.b, r = C.r;
  const int64_t nb = (int64_t)b * b * b, nv = (int64_t)(r + 1) * (r + 1) * (r + 1);
  std::vector<int32_t> grid(nb, -1);  // cube index, -1 for unlisted cells
  std::vector<uint8_t> listed(nb, 0);
  for (int64_t i = 0; i < C.n_cubes; ++i) {
    const int32_t x = C.cells[3 * i], y = C.cells[3 * i + 1], z = C.cells[3 * i + 2];
    const int64_t lin = x + (int64_t)b * (y + (int64_t)b * z);
    if (listed[lin]) return fail(INOLF_E_INVALID, "inolf_object_create: cube listed twice");
    listed[lin] = 1;
    grid[lin] = (int32_t)i;
  }
  // empty space between the cubes: octant distances of the unlisted base cells
  std::vector<uint8_t> bdist((size_t)8 * nb);
  octant_distance(listed.data(), b, std::min<int32_t>(b, 255), bdist.data());
  // inside each cube: octant distances (in fine cells, within the cube) of the
  // cells that are not live -- a live cell has a vertex of non-zero density;
  // a cell that is not live has sigma = 0 at every point, so the march skips
  // blocks of such cells as it skips unlisted base cells.
  const int64_t cpc = (int64_t)r * r * r;
  const int64_t nfd = std::max<int64_t>(C.n_cubes * cpc, 1);
  std::vector<uint8_t> fdist((size_t)8 * nfd, 0);
  {
    const int32_t fcap = std::min<int32_t>(r, 255);
    const int nt = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
    auto work = [&](int tid) {
      std::vector<uint8_t> dead((size_t)cpc), od((size_t)8 * cpc);
      for (int64_t q = tid; q < C.n_cubes; q += nt) {
        const float* blk = C.density + (size_t)(q * nv);
        auto at = [&](int32_t i, int32_t j, int32_t k) { return blk[i + (r + 1) * (j + (r + 1) * k)]; };
        for (int32_t k = 0; k < r; ++k)
          for (int32_t j = 0; j < r; ++j)
            for (int32_t i = 0; i < r; ++i) {
              bool any = false;
              for (int c = 0; c < 8 && !any; ++c) any = at(i + (c & 1), j + ((c >> 1) & 1), k + ((c >> 2) & 1)) > 0.0f;
              dead[i + (size_t)r * (j + (size_t)r * k)] = any;  // live cells are the obstacles
            }
        octant_distance(dead.data(), r, fcap, od.data());
        for (int oct = 0; oct < 8; ++oct)
          std::memcpy(&fdist[(size_t)oct * nfd + (size_t)(q * cpc)], &od[(size_t)oct * cpc], (size_t)cpc);
      }
    };
    std::vector<std::thread> th;
    for (int t = 1; t < nt; ++t) th.emplace_back(work, t);
    work(0);
    for (auto& t : th) t.join();
  }
  void* dg = nullptr;
  void* dd = nullptr;
  void* df = nullptr;
  void* dz = nullptr;
  void* db = nullptr;
  if (cudaMalloc(&dg, sizeof(int32_t) * nb) != cudaSuccess) return fail(INOLF_E_OOM, "cudaMalloc cube grid");
  o.cub.grid = (const int32_t*)dg;
  if (cudaMalloc(&db, bdist.size()) != cudaSuccess) return fail(INOLF_E_OOM, "cudaMalloc base distances");
  o.cub.bdist = (const uint8_t*)db;
  const size_t dbytes = sizeof(float) * (size_t)std::max<int64_t>(C.n_cubes * nv, 1);
  const size_t fbytes = sizeof(float4) * (size_t)std::max<int64_t>(C.n_cubes * nv, 1);
  if (cudaMalloc(&dd, dbytes) != cudaSuccess) return fail(INOLF_E_OOM, "cudaMalloc density cubes");
  o.cub.dens = (const float*)dd;
  if (cudaMalloc(&df, fbytes) != cudaSuccess) return fail(INOLF_E_OOM, "cudaMalloc diffuse cubes");
  o.cub.diff = (const float4*)df;
  if (cudaMalloc(&dz, fdist.size()) != cudaSuccess) return fail(INOLF_E_OOM, "cudaMalloc cube distances");
  o.cub.fdist = (const uint8_t*)dz;
  o.bytes += sizeof(int32_t) * nb + bdist.size() + dbytes + fbytes + fdist.size();
  if (cudaMemcpyAsync(dg, grid.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(db, bdist.data(), bdist.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(dz, fdist.data(), fdist.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      (C.n_cubes > 0 &&
       (cudaMemcpyAsync(dd, C.density, sizeof(float) * C.n_cubes * nv, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(df, C.diffuse, sizeof(float4) * C.n_cubes * nv, cudaMemcpyHostToDevice, st) !=
            cudaSuccess)) ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return fail(INOLF_E_CUDA, "inolf_object_create: cube upload failed");
  CubesDev& c = o.cub;
  c.b = b;
  c.r = r;
  c.rshift = 0;
  while ((1 << c.rshift) < r) ++c.rshift;
  c.K = b * r;
  c.K_f = (float)c.K;
  c.n_cubes = C.n_cubes;
  c.hi = o.lo + C.side;
  c.step = C.step;
  c.t_min = C.t_min;
  c.alpha_miss = C.alpha_miss;
  return INOLF_OK;
}

static bool pow2(int32_t v) { return v >= 1 && (v & (v - 1)) == 0; }

// Argument checks of a cube description (before anything is allocated).
static inolf_status check_cubes(const inolf_cubes_desc& C) {
  if (!pow2(C.b) || !pow2(C.r) || (int64_t)C.b * C.r > 4096)
    return fail(INOLF_E_INVALID, "inolf_object_create: cubes need b, r powers of two with b r <= 4096");
  if (C.n_cubes < 0 || C.n_cubes > (int64_t)C.b * C.b * C.b ||
      (C.n_cubes > 0 && (!C.cells || !C.density || !C.diffuse)))
    return fail(INOLF_E_INVALID, "inolf_object_create: bad cube list");
  if (!(C.side > 0) || !std::isfinite(C.side) || !(C.step > 0) || !std::isfinite(C.step) ||
      !((double)C.side * std::sqrt(3.0) / C.step < (double)(1 << 20) - 2))
    return fail(INOLF_E_INVALID, "inolf_object_create: bad march side / step");
  if (!(C.t_min > 0 && C.t_min <= 1) || !(C.alpha_miss >= 0 && C.alpha_miss < 1))
    return fail(INOLF_E_INVALID, "inolf_object_create: bad t_min / alpha_miss");
  for (int64_t i = 0; i < 3 * C.n_cubes; ++i)
    if (C.cells[i] < 0 || C.cells[i] >= C.b) return fail(INOLF_E_INVALID, "inolf_object_create: cube cell out of range");
  {
    std::vector<int64_t> lin((size_t)C.n_cubes);
    for (int64_t i = 0; i < C.n_cubes; ++i)
      lin[(size_t)i] = C.cells[3 * i] + (int64_t)C.b * (C.cells[3 * i + 1] + (int64_t)C.b * C.cells[3 * i + 2]);
    std::sort(lin.begin(), lin.end());
    if (std::adjacent_find(lin.begin(), lin.end()) != lin.end())
      return fail(INOLF_E_INVALID, "inolf_object_create: cube listed twice");
  }
  const int64_t nv = (int64_t)(C.r + 1) * (C.r + 1) * (C.r + 1);
  for (int64_t i = 0; i < C.n_cubes * nv; ++i)
    if (!(C.density[i] >= 0) || !std::isfinite(C.density[i]))
      return fail(INOLF_E_INVALID, "inolf_object_create: densities must be finite and >= 0");
  return INOLF_OK;
}

extern "C" inolf_status inolf_object_create(const inolf_object_desc* desc, void* stream, inolf_object** out) {
  clear_error();
  if (!desc || !out) return fail(INOLF_E_INVALID, "inolf_object_create: NULL argument");
  *out = nullptr;
  const inolf_object_desc& D = *desc;
  const bool variant = D.cubes != nullptr;
  if (variant) {
    inolf_status cs = check_cubes(*D.cubes);
    if (cs != INOLF_OK) return cs;
  }
  const bool have_mesh = D.n_vertices > 0 && D.n_triangles > 0;
  if (!variant && (!have_mesh || !D.vertices || !D.triangles))
    return fail(INOLF_E_INVALID, "inolf_object_create: empty or missing proxy mesh");
  if (variant && (D.n_vertices != 0 || D.n_triangles != 0))
    return fail(INOLF_E_INVALID, "inolf_object_create: objects with density cubes take no proxy mesh");
  if (D.n_levels < 1 || D.n_levels > INOLF_MAX_LEVELS || D.n_features != 2 || !D.resolution || !D.hashes ||
      !D.features)
    return fail(INOLF_E_INVALID, "inolf_object_create: bad level description (1..16 levels, F = 2)");
  if (!D.w1 || !D.w2 || !D.w3) return fail(INOLF_E_INVALID, "inolf_object_create: missing weights");
  if (!(D.domain_scale > 0)) return fail(INOLF_E_INVALID, "inolf_object_create: bad domain");
  for (int32_t t = 0; t < 3 * D.n_triangles; ++t)
    if (D.triangles[t] < 0 || D.triangles[t] >= D.n_vertices)
      return fail(INOLF_E_INVALID, "inolf_object_create: triangle index out of range");
  for (int l = 0; l < D.n_levels; ++l) {
    const inolf_hash* h = D.hashes[l];
    if (!h || !h->phi || (h->n > 0 && (!h->slot_of || !D.features[l])) || h->m < 1 || h->m > 1024 || h->r < 1 ||
        D.resolution[l] < 1 || D.resolution[l] > (1 << 20))
      return fail(INOLF_E_INVALID, "inolf_object_create: bad hash / features of level " + std::to_string(l));
    if (h->r >= 2048)
      return fail(INOLF_E_UNSUPPORTED, "inolf_object_create: offset-table side r = " + std::to_string(h->r) +
                                           " of level " + std::to_string(l) + " exceeds 2047");
    if (h->n > 0 && !h->coords)
      return fail(INOLF_E_INVALID, "inolf_object_create: the hash of level " + std::to_string(l) +
                                       " carries no coords (the corner bundles need the hashed points)");
    for (int64_t i = 0; i < 3 * h->n; ++i)
      if (h->coords[i] < 0 || h->coords[i] > D.resolution[l])
        return fail(INOLF_E_INVALID, "inolf_object_create: a hashed point of level " + std::to_string(l) +
                                         " lies outside [0, N]");
  }
  inolf_object* obj = new (std::nothrow) inolf_object();
  if (!obj) return fail(INOLF_E_OOM, "inolf_object_create: oom");
  Object& o = obj->o;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaGetDevice(&o.device) != cudaSuccess) { delete obj; return fail(INOLF_E_CUDA, "cudaGetDevice failed"); }
  o.L = D.n_levels;
  o.F = D.n_features;
  o.d_in = D.n_levels * D.n_features + INOLF_N_SH + (variant ? 1 : 0);
  o.variant = variant ? 1 : 0;
  o.fp16 = D.features_fp16 ? 1 : 0;
  o.lo = D.domain_lo;
  o.scale = D.domain_scale;
  for (int k = 0; k < 3; ++k) o.fp8_act_scale[k] = D.fp8_act_scale[k];

  if (variant) {
    inolf_status cs = create_cubes(o, *D.cubes, st);
    if (cs != INOLF_OK) { destroy_object(o); delete obj; return cs; }
  }

  // --- bounding sphere of the proxy (box centre, farthest vertex), padded
  //     so that FP32 rounding of the ray-sphere test never culls a hit ---
  if (!variant) {
    double lo3[3] = {1e300, 1e300, 1e300}, hi3[3] = {-1e300, -1e300, -1e300};
    for (int32_t v = 0; v < D.n_vertices; ++v)
      for (int k = 0; k < 3; ++k) {
        lo3[k] = std::min(lo3[k], (double)D.vertices[3 * v + k]);
        hi3[k] = std::max(hi3[k], (double)D.vertices[3 * v + k]);
      }
    double c[3], r2 = 0.0;
    for (int k = 0; k < 3; ++k) c[k] = 0.5 * (lo3[k] + hi3[k]);
    for (int32_t v = 0; v < D.n_vertices; ++v) {
      double q = 0.0;
      for (int k = 0; k < 3; ++k) q += (D.vertices[3 * v + k] - c[k]) * (D.vertices[3 * v + k] - c[k]);
      r2 = std::max(r2, q);
    }
    const double r = std::sqrt(r2);
    for (int k = 0; k < 3; ++k) o.bsphere[k] = (float)c[k];
    o.bsphere[3] = (float)(r * 1.001 + 1e-3 * (1.0 + std::fabs(c[0]) + std::fabs(c[1]) + std::fabs(c[2]) + r));
  }

  // --- BVH ---
  if (!variant) {
  Builder b;
  b.V = D.vertices;
  b.F = D.triangles;
  const int32_t nF = D.n_triangles;
  b.tb.resize(nF);
  b.cen.resize(3 * (size_t)nF);
  b.idx.resize(nF);
  for (int32_t t = 0; t < nF; ++t) {
    for (int v = 0; v < 3; ++v) b.tb[t].grow(D.vertices + 3 * D.triangles[3 * t + v]);
    for (int k = 0; k < 3; ++k)
      b.cen[3 * t + k] = (float)(((double)D.vertices[3 * D.triangles[3 * t] + k] +
                                  D.vertices[3 * D.triangles[3 * t + 1] + k] +
                                  D.vertices[3 * D.triangles[3 * t + 2] + k]) / 3.0);
    b.idx[t] = t;
  }
  b.nodes.resize(16);  // root
  {
    ChildRef root = b.make(0, nF);
    if (root.count > 0) {  // whole mesh is one leaf: root = (leaf, empty)
      ChildRef none;
      b.write_node(0, root, none, 0);
    } else {
      // make() appended the real root at index 1.. copy it into slot 0
      std::copy(b.nodes.begin() + 16 * (size_t)root.index, b.nodes.begin() + 16 * (size_t)root.index + 16,
                b.nodes.begin());
    }
  }
  o.n_nodes = (int32_t)(b.nodes.size() / 16);
  // the traversal keeps at most one deferred child per level on its stack
  if (b.max_depth >= 48) {
    destroy_object(o);
    delete obj;
    return fail(INOLF_E_UNSUPPORTED, "inolf_object_create: BVH deeper than the traversal stack (48)");
  }
  std::vector<float> tri(12 * (size_t)nF);
  for (int32_t s = 0; s < nF; ++s) {
    const int32_t t = b.idx[s];
    const float* a = D.vertices + 3 * D.triangles[3 * t + 0];
    const float* bb = D.vertices + 3 * D.triangles[3 * t + 1];
    const float* c = D.vertices + 3 * D.triangles[3 * t + 2];
    float* r = &tri[12 * (size_t)s];
    for (int k = 0; k < 3; ++k) {
      r[k] = a[k];
      r[4 + k] = bb[k] - a[k];  // e1 = v1 - v0 (one FP32 subtraction)
      r[8 + k] = c[k] - a[k];   // e2 = v2 - v0
    }
    std::memcpy(&r[3], &t, 4);
    r[7] = 0.0f;
    r[11] = 0.0f;
  }
  o.n_tris = nF;
  CUDA_TRY(cudaMalloc(&o.nodes, b.nodes.size() * sizeof(float)));
  CUDA_TRY(cudaMemcpyAsync(o.nodes, b.nodes.data(), b.nodes.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMalloc(&o.tris, tri.size() * sizeof(float)));
  CUDA_TRY(cudaMemcpyAsync(o.tris, tri.data(), tri.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  o.bytes += b.nodes.size() * sizeof(float) + tri.size() * sizeof(float);
  CUDA_TRY(cudaStreamSynchronize(st));
  }  // !variant

  // --- levels: Phi and feature tables in slot order ---
  for (int l = 0; l < o.L; ++l) {
    const inolf_hash* h = D.hashes[l];
    LevelDev& lv = o.lv[l];
    lv.N = D.resolution[l];
    lv.m = h->m;
    lv.r = h->r;
    lv.N_f = (float)lv.N;
    auto magic = [](int64_t d) { return (uint32_t)std::min<uint64_t>(0xFFFFFFFFull, ((1ull << 32) + d - 1) / d); };
    lv.magic_m = magic(lv.m);
    lv.magic_r = magic(lv.r);
    const int64_t R3 = (int64_t)h->r * h->r * h->r;
    const int64_t M3 = (int64_t)h->m * h->m * h->m;
    o.rows[l] = M3;
    // Phi padded with zeros to a multiple of 16 bytes, so that one bulk copy
    // of the whole table (a multiple of 16 bytes) stays inside the allocation
    const int64_t R3p = (R3 + 3) / 4 * 4;
    void* dphi = nullptr;
    CUDA_TRY(cudaMalloc(&dphi, sizeof(uint32_t) * R3p));
    lv.phi = (const uint32_t*)dphi;
    CUDA_TRY(cudaMemsetAsync(dphi, 0, sizeof(uint32_t) * R3p, st));
    CUDA_TRY(cudaMemcpyAsync(dphi, h->phi, sizeof(uint32_t) * R3, cudaMemcpyHostToDevice, st));
    const size_t row_bytes = o.fp16 ? 4 : 8;
    std::vector<uint8_t> table((size_t)M3 * row_bytes, 0);
    for (int64_t i = 0; i < h->n; ++i) {
      const uint32_t s = h->slot_of[i];
      if ((int64_t)s >= M3) { destroy_object(o); delete obj; return fail(INOLF_E_INVALID, "slot out of range"); }
      const float* fr = D.features[l] + 2 * i;
      if (o.fp16) {
        __half2 v = __floats2half2_rn(fr[0], fr[1]);
        std::memcpy(&table[(size_t)s * 4], &v, 4);
      } else {
        std::memcpy(&table[(size_t)s * 8], fr, 8);
      }
    }
    void* dt = nullptr;
    CUDA_TRY(cudaMalloc(&dt, table.size()));
    lv.table = dt;
    CUDA_TRY(cudaMemcpyAsync(dt, table.data(), table.size(), cudaMemcpyHostToDevice, st));
    o.bytes += sizeof(uint32_t) * R3p + table.size();
    // the hashed points (packed x | y << 21 | z << 42) and the corner bundles
    // built from them on the device
    {
      std::vector<uint64_t> pk((size_t)std::max<int64_t>(h->n, 1), 0);
      for (int64_t i = 0; i < h->n; ++i)
        pk[(size_t)i] = (uint64_t)(uint32_t)h->coords[3 * i] | ((uint64_t)(uint32_t)h->coords[3 * i + 1] << 21) |
                        ((uint64_t)(uint32_t)h->coords[3 * i + 2] << 42);
      CUDA_TRY(cudaMalloc(&o.pts[l], pk.size() * sizeof(uint64_t)));
      o.n_pts[l] = h->n;
      CUDA_TRY(cudaMemcpyAsync(o.pts[l], pk.data(), pk.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
      const size_t bbytes = (size_t)M3 * 8 * row_bytes;
      void* db = nullptr;
      CUDA_TRY(cudaMalloc(&db, bbytes));
      lv.bundle = db;
      o.bytes += pk.size() * sizeof(uint64_t) + bbytes;
      inolf_status es = build_level_bundles(o, l, stream);
      if (es != INOLF_OK) { destroy_object(o); delete obj; return es; }
      CUDA_TRY(cudaStreamSynchronize(st));
    }
  }

  inolf_status ws = upload_weights(o, D.w1, D.w2, D.w3, stream);
  if (ws != INOLF_OK) { destroy_object(o); delete obj; return ws; }
  *out = obj;
  return INOLF_OK;
}

extern "C" void inolf_object_destroy(inolf_object* obj) {
  if (!obj) return;
  destroy_object(obj->o);
  delete obj;
}

extern "C" inolf_status inolf_object_bytes(const inolf_object* obj, size_t* bytes) {
  if (!obj || !bytes) return fail(INOLF_E_INVALID, "inolf_object_bytes: NULL argument");
  *bytes = obj->o.bytes;
  return INOLF_OK;
}

extern "C" inolf_status inolf_object_set_fp8_scales(inolf_object* obj, const float scales[3]) {
  if (!obj || !scales) return fail(INOLF_E_INVALID, "inolf_object_set_fp8_scales: NULL argument");
  for (int k = 0; k < 3; ++k)
    if (!(scales[k] > 0) || !std::isfinite(scales[k]))
      return fail(INOLF_E_INVALID, "inolf_object_set_fp8_scales: scales must be positive");
  for (int k = 0; k < 3; ++k) obj->o.fp8_act_scale[k] = scales[k];
  return INOLF_OK;
}

extern "C" inolf_status inolf_object_table_rows(const inolf_object* obj, int32_t level, int64_t* rows) {
  if (!obj || !rows || level < 0 || level >= obj->o.L) return fail(INOLF_E_INVALID, "inolf_object_table_rows");
  *rows = obj->o.rows[level];
  return INOLF_OK;
}

extern "C" inolf_status inolf_object_read_params(const inolf_object* obj, float* const* tables, float* w1,
                                                 float* w2, float* w3) {
  clear_error();
  if (!obj) return fail(INOLF_E_INVALID, "inolf_object_read_params: NULL object");
  const Object& o = obj->o;
  const int din = o.d_in, H = INOLF_HIDDEN, O = INOLF_OUT;
  if (tables) {
    for (int l = 0; l < o.L; ++l) {
      if (!tables[l]) continue;
      const int64_t M3 = o.rows[l];
      if (o.fp16) {
        std::vector<__half2> tmp(M3);
        if (cudaMemcpy(tmp.data(), o.lv[l].table, 4 * M3, cudaMemcpyDeviceToHost) != cudaSuccess)
          return fail(INOLF_E_CUDA, "read_params: cudaMemcpy failed");
        for (int64_t i = 0; i < M3; ++i) {
          float2 v = __half22float2(tmp[i]);
          tables[l][2 * i] = v.x;
          tables[l][2 * i + 1] = v.y;
        }
      } else if (cudaMemcpy(tables[l], o.lv[l].table, 8 * M3, cudaMemcpyDeviceToHost) != cudaSuccess) {
        return fail(INOLF_E_CUDA, "read_params: cudaMemcpy failed");
      }
    }
  }
  if (w1 || w2 || w3) {
    std::vector<float> w((size_t)din * H + H * H + H * O);
    if (cudaMemcpy(w.data(), o.w_f32, w.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(INOLF_E_CUDA, "read_params: cudaMemcpy failed");
    if (w1)
      for (int j = 0; j < H; ++j)
        for (int i = 0; i < din; ++i) w1[(size_t)j * din + i] = w[(size_t)i * H + j];
    if (w2) std::memcpy(w2, &w[(size_t)din * H], sizeof(float) * H * H);
    if (w3)
      for (int j = 0; j < O; ++j)
        for (int i = 0; i < H; ++i) w3[(size_t)j * H + i] = w[(size_t)din * H + H * H + (size_t)i * O + j];
  }
  return INOLF_OK;
}

