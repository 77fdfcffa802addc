// Seeded synthetic scene generator for i-NOLF workloads.
//
// This module produces INPUTS only: proxy meshes, the occupied-vertex sets of
// each encoder level (the "voxels surrounding the hit points" of Sec. 4.2,
// "Implementation with PSH encoding"), per-vertex feature values keyed by
// integer coordinate, Xavier-initialised MLP weights and pinhole cameras.
// It contains none of the renderer's arithmetic (ray generation, ray-triangle
// tests, hashing, interpolation, view encoding, MLP): the CUDA path and the
// FP64 oracle each implement those on their own and consume what this file
// writes.  Everything is deterministic for a given seed and thread count.
//
// Conventions shared by both consumers (they are properties of the inputs):
//   * vertex key  pack(x, y, z) = x | y << 21 | z << 42, all coords in [0, N];
//     the key lists returned per level are sorted ascending and unique;
//   * camera record (13 floats): eye[3], right[3], up[3], fwd[3], tan(fovy/2);
//   * weights row-major [out][in], layer order W1, W2, W3.

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>
#include <algorithm>
#include <array>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

inline uint64_t splitmix64(uint64_t x) {
  // SplitMix64 finaliser (Steele, Lea, Flood 2014).
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

inline double u01(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

struct V3 { double x, y, z; };
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline V3 normalize(V3 a) { double s = 1.0 / std::sqrt(dot(a, a)); return s * a; }

// The 12 icosahedron vertices (0, ±1, ±g), (±1, ±g, 0), (±g, 0, ±1) and its
// 20 faces, found as the vertex triples that are pairwise at edge length 2;
// each face is oriented counter-clockwise seen from outside.
void icosahedron(std::vector<V3>& v, std::vector<std::array<int, 3>>& f) {
  const double g = (1.0 + std::sqrt(5.0)) / 2.0;
  v.clear();
  for (int s1 = -1; s1 <= 1; s1 += 2)
    for (int s2 = -1; s2 <= 1; s2 += 2) {
      v.push_back({0.0, (double)s1, s2 * g});
      v.push_back({(double)s1, s2 * g, 0.0});
      v.push_back({s2 * g, 0.0, (double)s1});
    }
  f.clear();
  auto is_edge = [&](int a, int b) {
    V3 d = v[a] - v[b];
    return std::fabs(dot(d, d) - 4.0) < 1e-9;
  };
  const int n = (int)v.size();
  for (int a = 0; a < n; ++a)
    for (int b = a + 1; b < n; ++b)
      for (int c = b + 1; c < n; ++c)
        if (is_edge(a, b) && is_edge(b, c) && is_edge(a, c)) {
          V3 nrm = cross(v[b] - v[a], v[c] - v[a]);
          V3 cen = (1.0 / 3.0) * (v[a] + v[b] + v[c]);
          if (dot(nrm, cen) > 0) f.push_back({a, b, c});
          else f.push_back({a, c, b});
        }
}

template <class T>
T* dup(const std::vector<T>& src) {
  T* p = (T*)std::malloc(sizeof(T) * (src.empty() ? 1 : src.size()));
  if (p && !src.empty()) std::memcpy(p, src.data(), sizeof(T) * src.size());
  return p;
}

// Lattice value noise in [-1, 1]: SplitMix64 values at integer lattice points,
// smoothstep-weighted trilinear blend inside each lattice cell.
double lattice_value(uint64_t seed, int64_t i, int64_t j, int64_t k) {
  const uint64_t off = 1ull << 20;
  uint64_t key = (uint64_t)(i + off) | ((uint64_t)(j + off) << 21) | ((uint64_t)(k + off) << 42);
  return 2.0 * u01(splitmix64(splitmix64(seed ^ 0x6E6F697365ull) ^ key)) - 1.0;
}

double value_noise(uint64_t seed, V3 q) {
  double fx = std::floor(q.x), fy = std::floor(q.y), fz = std::floor(q.z);
  int64_t i = (int64_t)fx, j = (int64_t)fy, k = (int64_t)fz;
  double tx = q.x - fx, ty = q.y - fy, tz = q.z - fz;
  double sx = tx * tx * (3 - 2 * tx), sy = ty * ty * (3 - 2 * ty), sz = tz * tz * (3 - 2 * tz);
  double acc = 0.0;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        double w = (dx ? sx : 1 - sx) * (dy ? sy : 1 - sy) * (dz ? sz : 1 - sz);
        acc += w * lattice_value(seed, i + dx, j + dy, k + dz);
      }
  return acc;
}

// Three octaves, amplitude halving and frequency doubling, base frequency 2,
// normalised by the sum of the amplitudes so the result stays in [-1, 1].
double fractal_noise(uint64_t seed, V3 p) {
  double acc = 0.0, norm = 0.0;
  for (int o = 0; o < 3; ++o) {
    double a = std::ldexp(1.0, -o);
    double fr = 2.0 * std::ldexp(1.0, o);
    acc += a * value_noise(seed + (uint64_t)o, fr * p);
    norm += a;
  }
  return acc / norm;
}

// Exact squared distance from point p to triangle (a, b, c), by classifying p
// against the Voronoi regions of the triangle's vertices, edges and face.
double point_triangle_dist2(V3 p, V3 a, V3 b, V3 c) {
  V3 ab = b - a, ac = c - a, ap = p - a;
  double d1 = dot(ab, ap), d2 = dot(ac, ap);
  if (d1 <= 0 && d2 <= 0) return dot(ap, ap);
  V3 bp = p - b;
  double d3 = dot(ab, bp), d4 = dot(ac, bp);
  if (d3 >= 0 && d4 <= d3) return dot(bp, bp);
  double vc = d1 * d4 - d3 * d2;
  if (vc <= 0 && d1 >= 0 && d3 <= 0) {
    double t = d1 / (d1 - d3);
    V3 q = p - (a + t * ab);
    return dot(q, q);
  }
  V3 cp = p - c;
  double d5 = dot(ab, cp), d6 = dot(ac, cp);
  if (d6 >= 0 && d5 <= d6) return dot(cp, cp);
  double vb = d5 * d2 - d1 * d6;
  if (vb <= 0 && d2 >= 0 && d6 <= 0) {
    double t = d2 / (d2 - d6);
    V3 q = p - (a + t * ac);
    return dot(q, q);
  }
  double va = d3 * d6 - d5 * d4;
  if (va <= 0 && (d4 - d3) >= 0 && (d5 - d6) >= 0) {
    double t = (d4 - d3) / ((d4 - d3) + (d5 - d6));
    V3 q = p - (b + t * (c - b));
    return dot(q, q);
  }
  double den = 1.0 / (va + vb + vc);
  double v = vb * den, w = vc * den;
  V3 q = p - (a + v * ab + w * ac);
  return dot(q, q);
}

inline void bit_set(uint64_t* bits, uint64_t i) {
  __atomic_fetch_or(&bits[i >> 6], 1ull << (i & 63), __ATOMIC_RELAXED);
}
inline bool bit_get(const uint64_t* bits, uint64_t i) {
  return (__atomic_load_n(&bits[i >> 6], __ATOMIC_RELAXED) >> (i & 63)) & 1ull;
}

// All 8 corners of the cells set in `occ` (N^3 cells, bit x + N (y + N z)),
// packed and sorted ascending.  Returns 0, or -2 when memory runs out.
int cells_to_keys(const uint64_t* occ, int32_t N, uint64_t** keys_out, int64_t* n_out) {
  const uint64_t n1 = (uint64_t)N, ncell = n1 * n1 * n1;
  const uint64_t nv1 = n1 + 1, nvert = nv1 * nv1 * nv1;
  uint64_t* vbits = (uint64_t*)std::calloc((nvert + 63) / 64, 8);
  if (!vbits) return -2;
  const int64_t nwords = (int64_t)((ncell + 63) / 64);
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t w = 0; w < nwords; ++w) {
    uint64_t word = occ[w];
    while (word) {
      int b = __builtin_ctzll(word);
      word &= word - 1;
      uint64_t lin = (uint64_t)w * 64 + (uint64_t)b;
      uint64_t x = lin % n1, y = (lin / n1) % n1, z = lin / (n1 * n1);
      for (int d = 0; d < 8; ++d) {
        uint64_t vx = x + (d & 1), vy = y + ((d >> 1) & 1), vz = z + ((d >> 2) & 1);
        bit_set(vbits, vx + nv1 * (vy + nv1 * vz));
      }
    }
  }
  const int64_t vwords = (int64_t)((nvert + 63) / 64);
  int64_t count = 0;
#pragma omp parallel for reduction(+ : count) schedule(static)
  for (int64_t w = 0; w < vwords; ++w) count += __builtin_popcountll(vbits[w]);
  uint64_t* keys = (uint64_t*)std::malloc(sizeof(uint64_t) * (count ? count : 1));
  if (!keys) { std::free(vbits); return -2; }
  // Ordered extraction: linear index x + (N+1)(y + (N+1) z) increases with
  // (z, y, x), which is also the order of the packed keys.
  int64_t pos = 0;
  for (int64_t w = 0; w < vwords; ++w) {
    uint64_t word = vbits[w];
    while (word) {
      int b = __builtin_ctzll(word);
      word &= word - 1;
      uint64_t lin = (uint64_t)w * 64 + (uint64_t)b;
      uint64_t x = lin % nv1, y = (lin / nv1) % nv1, z = lin / (nv1 * nv1);
      keys[pos++] = x | (y << 21) | (z << 42);
    }
  }
  std::free(vbits);
  *keys_out = keys;
  *n_out = count;
  return 0;
}

// Radial signed distance of point p to the surface r = radius (1 + amp n(q)),
// q = p / |p|, n = fractal_noise (the displaced sphere of syn_geodesic when
// radius = 1; a plain sphere when amp = 0).
double shell_distance(uint64_t seed, double radius, double amp, V3 p) {
  const double len = std::sqrt(dot(p, p));
  if (len < 1e-12) return -radius;
  const V3 q = (1.0 / len) * p;
  const double R = radius * (1.0 + (amp != 0.0 ? amp * fractal_noise(seed, q) : 0.0));
  return len - R;
}

}  // namespace

extern "C" {

void syn_free(void* p) { std::free(p); }

uint64_t syn_splitmix64(uint64_t x) { return splitmix64(x); }

// Level-`level` icosphere of the given radius: the icosahedron, each triangle
// split into 4 through its edge midpoints `level` times, every new vertex
// projected to the sphere in FP64.  20 * 4^level triangles.
int syn_icosphere(int32_t level, double radius, float** V, int32_t* nV, int32_t** F, int32_t* nF) {
  if (level < 0 || level > 9 || !V || !nV || !F || !nF) return -1;
  std::vector<V3> v;
  std::vector<std::array<int, 3>> f;
  icosahedron(v, f);
  for (auto& p : v) p = normalize(p);
  for (int it = 0; it < level; ++it) {
    std::map<std::pair<int, int>, int> mid;
    auto midpoint = [&](int a, int b) {
      auto key = std::make_pair(std::min(a, b), std::max(a, b));
      auto itm = mid.find(key);
      if (itm != mid.end()) return itm->second;
      int id = (int)v.size();
      v.push_back(normalize(0.5 * (v[key.first] + v[key.second])));
      mid[key] = id;
      return id;
    };
    std::vector<std::array<int, 3>> g;
    g.reserve(f.size() * 4);
    for (auto& t : f) {
      int a = t[0], b = t[1], c = t[2];
      int ab = midpoint(a, b), bc = midpoint(b, c), ca = midpoint(c, a);
      g.push_back({a, ab, ca});
      g.push_back({b, bc, ab});
      g.push_back({c, ca, bc});
      g.push_back({ab, bc, ca});
    }
    f.swap(g);
  }
  std::vector<float> vf(v.size() * 3);
  for (size_t i = 0; i < v.size(); ++i) {
    vf[3 * i + 0] = (float)(radius * v[i].x);
    vf[3 * i + 1] = (float)(radius * v[i].y);
    vf[3 * i + 2] = (float)(radius * v[i].z);
  }
  std::vector<int32_t> fi(f.size() * 3);
  for (size_t i = 0; i < f.size(); ++i)
    for (int k = 0; k < 3; ++k) fi[3 * i + k] = f[i][k];
  *V = dup(vf); *F = dup(fi);
  *nV = (int32_t)v.size(); *nF = (int32_t)f.size();
  return (*V && *F) ? 0 : -2;
}

// Class-I geodesic sphere of frequency `freq` (20 * freq^2 triangles): every
// icosahedron face carries the barycentric lattice (f-i-j, i, j)/f, points
// are projected to the unit sphere and displaced radially to
// r = 1 + amp * fractal_noise(seed, p).  Lattice points on shared edges and
// corners are built once from a canonical (sorted-vertex) key, so the mesh is
// closed.
int syn_geodesic(int32_t freq, double amp, uint64_t seed, float** V, int32_t* nV, int32_t** F, int32_t* nF) {
  if (freq < 1 || freq > 2000 || !V || !nV || !F || !nF) return -1;
  std::vector<V3> ico;
  std::vector<std::array<int, 3>> faces;
  icosahedron(ico, faces);
  typedef std::array<int, 6> Key;  // (vertex, weight) x 3, sorted by vertex, unused = (-1, 0)
  std::map<Key, int> index;
  std::vector<Key> keys;
  auto vid = [&](const int ids[3], const int w[3]) {
    std::array<std::pair<int, int>, 3> e;
    int m = 0;
    for (int k = 0; k < 3; ++k)
      if (w[k] != 0) e[m++] = {ids[k], w[k]};
    for (int k = m; k < 3; ++k) e[k] = {INT32_MAX, 0};
    std::sort(e.begin(), e.end());
    Key key;
    for (int k = 0; k < 3; ++k) {
      key[2 * k] = e[k].first == INT32_MAX ? -1 : e[k].first;
      key[2 * k + 1] = e[k].second;
    }
    auto it = index.find(key);
    if (it != index.end()) return it->second;
    int id = (int)keys.size();
    keys.push_back(key);
    index[key] = id;
    return id;
  };
  std::vector<int32_t> fi;
  fi.reserve((size_t)20 * freq * freq * 3);
  std::vector<int> lat((size_t)(freq + 1) * (freq + 1));
  for (auto& t : faces) {
    const int ids[3] = {t[0], t[1], t[2]};
    for (int i = 0; i <= freq; ++i)
      for (int j = 0; i + j <= freq; ++j) {
        int w[3] = {freq - i - j, i, j};
        lat[(size_t)i * (freq + 1) + j] = vid(ids, w);
      }
    auto P = [&](int i, int j) { return lat[(size_t)i * (freq + 1) + j]; };
    for (int i = 0; i < freq; ++i)
      for (int j = 0; i + j < freq; ++j) {
        fi.push_back(P(i, j)); fi.push_back(P(i + 1, j)); fi.push_back(P(i, j + 1));
        if (i + j + 2 <= freq) {
          fi.push_back(P(i + 1, j)); fi.push_back(P(i + 1, j + 1)); fi.push_back(P(i, j + 1));
        }
      }
  }
  std::vector<float> vf(keys.size() * 3);
#pragma omp parallel for schedule(static)
  for (long long q = 0; q < (long long)keys.size(); ++q) {
    const Key& k = keys[q];
    V3 p = {0, 0, 0};
    for (int e = 0; e < 3; ++e)
      if (k[2 * e] >= 0) p = p + ((double)k[2 * e + 1] / (double)freq) * ico[k[2 * e]];
    V3 u = normalize(p);
    double r = 1.0 + amp * fractal_noise(seed, u);
    vf[3 * q + 0] = (float)(r * u.x);
    vf[3 * q + 1] = (float)(r * u.y);
    vf[3 * q + 2] = (float)(r * u.z);
  }
  *V = dup(vf); *F = dup(fi);
  *nV = (int32_t)keys.size(); *nF = (int32_t)(fi.size() / 3);
  return (*V && *F) ? 0 : -2;
}

// Occupied vertex set of one encoder level.  The domain is the cube
// [lo, lo + side]^3 split into N^3 cells of size h = side / N.  A cell is
// occupied when the FP64 distance from its centre to the mesh is at most
// `band + sqrt(3)/2 * h`, which guarantees that every cell the surface passes
// through is occupied.  The returned keys are all 8 corners of all occupied
// cells, packed and sorted ascending.
int syn_band_vertices(const float* V, int32_t nV, const int32_t* F, int32_t nF, int32_t N,
                      double lo, double side, double band, uint64_t** keys_out, int64_t* n_out) {
  if (!V || !F || nV <= 0 || nF <= 0 || N < 1 || N > (1 << 20) - 2 || !keys_out || !n_out) return -1;
  const double h = side / N;
  const double R = band + 0.5 * std::sqrt(3.0) * h;
  const uint64_t n1 = (uint64_t)N, ncell = n1 * n1 * n1;
  uint64_t* occ = (uint64_t*)std::calloc((ncell + 63) / 64, 8);
  if (!occ) return -2;
#pragma omp parallel for schedule(dynamic, 64)
  for (int32_t tri = 0; tri < nF; ++tri) {
    V3 a, b, c;
    const float* pa = V + 3 * F[3 * tri + 0];
    const float* pb = V + 3 * F[3 * tri + 1];
    const float* pc = V + 3 * F[3 * tri + 2];
    a = {pa[0], pa[1], pa[2]}; b = {pb[0], pb[1], pb[2]}; c = {pc[0], pc[1], pc[2]};
    double mn[3] = {std::min({a.x, b.x, c.x}) - R, std::min({a.y, b.y, c.y}) - R, std::min({a.z, b.z, c.z}) - R};
    double mx[3] = {std::max({a.x, b.x, c.x}) + R, std::max({a.y, b.y, c.y}) + R, std::max({a.z, b.z, c.z}) + R};
    int64_t c0[3], c1[3];
    for (int k = 0; k < 3; ++k) {
      // cells whose centre lo + (i + 0.5) h lies inside [mn, mx]
      c0[k] = (int64_t)std::ceil((mn[k] - lo) / h - 0.5);
      c1[k] = (int64_t)std::floor((mx[k] - lo) / h - 0.5);
      if (c0[k] < 0) c0[k] = 0;
      if (c1[k] > N - 1) c1[k] = N - 1;
    }
    for (int64_t z = c0[2]; z <= c1[2]; ++z)
      for (int64_t y = c0[1]; y <= c1[1]; ++y)
        for (int64_t x = c0[0]; x <= c1[0]; ++x) {
          uint64_t lin = (uint64_t)x + n1 * ((uint64_t)y + n1 * (uint64_t)z);
          if (bit_get(occ, lin)) continue;
          V3 p = {lo + (x + 0.5) * h, lo + (y + 0.5) * h, lo + (z + 0.5) * h};
          if (point_triangle_dist2(p, a, b, c) <= R * R) bit_set(occ, lin);
        }
  }
  const int rc = cells_to_keys(occ, N, keys_out, n_out);
  std::free(occ);
  return rc;
}

void syn_unpack_keys(const uint64_t* keys, int64_t n, int32_t* coords) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    coords[3 * i + 0] = (int32_t)(keys[i] & 0x1FFFFF);
    coords[3 * i + 1] = (int32_t)((keys[i] >> 21) & 0x1FFFFF);
    coords[3 * i + 2] = (int32_t)((keys[i] >> 42) & 0x1FFFFF);
  }
}

// Feature k of the vertex with packed key `key` on level `level`:
// 0.1 * a standard normal deviate (Box-Muller on two SplitMix64 draws),
// keyed by (seed, level, key, k) and therefore independent of where the
// vertex ends up in any table.  Rounded to FP32, or to FP16 when fp16 != 0
// (the FP16 value is returned widened to FP32).
void syn_features(uint64_t seed, int32_t level, const uint64_t* keys, int64_t n, int32_t nf,
                  int32_t fp16, float* out) {
  const uint64_t base = splitmix64(seed ^ 0x66656174ull) ^ ((uint64_t)level << 58);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    for (int32_t k = 0; k < nf; ++k) {
      uint64_t key = splitmix64(base ^ (keys[i] * 8 + (uint64_t)k));
      double u1 = ((double)(splitmix64(key) >> 11) + 1.0) * (1.0 / 9007199254740992.0);
      double u2 = u01(splitmix64(key ^ 0x5bd1e995ull));
      double g = std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
      float v = (float)(0.1 * g);
      if (fp16) v = (float)(_Float16)v;
      out[(size_t)i * nf + k] = v;
    }
}

// Xavier-uniform weights: U(-a, a), a = sqrt(6 / (fan_in + fan_out)), drawn
// from one SplitMix64 stream in the order W1, W2, W3 (each row-major
// [out][in]) and rounded to FP32.
void syn_xavier(uint64_t seed, int32_t d_in, int32_t hidden, int32_t d_out,
                float* w1, float* w2, float* w3) {
  uint64_t ctr = splitmix64(seed ^ 0x78617669ull);
  auto fill = [&](float* w, int fo, int fi) {
    double a = std::sqrt(6.0 / (double)(fi + fo));
    for (int i = 0; i < fo * fi; ++i) w[i] = (float)((2.0 * u01(splitmix64(ctr++)) - 1.0) * a);
  };
  fill(w1, hidden, d_in);
  fill(w2, hidden, hidden);
  fill(w3, d_out, hidden);
}

// Pinhole camera looking from `eye` at `target`: fwd = normalize(target -
// eye), right = normalize(fwd x up), up' = right x fwd, tan(fovy/2); all in
// FP64, rounded to FP32 into the 13-float record.
void syn_camera(const double eye[3], const double target[3], const double up[3], double fovy_deg,
                float out[13]) {
  V3 e = {eye[0], eye[1], eye[2]}, t = {target[0], target[1], target[2]}, u = {up[0], up[1], up[2]};
  V3 f = normalize(t - e);
  V3 r = normalize(cross(f, u));
  V3 uu = cross(r, f);
  const V3 rows[4] = {e, r, uu, f};
  for (int i = 0; i < 4; ++i) {
    out[3 * i + 0] = (float)rows[i].x;
    out[3 * i + 1] = (float)rows[i].y;
    out[3 * i + 2] = (float)rows[i].z;
  }
  out[12] = (float)std::tan(0.5 * fovy_deg * M_PI / 180.0);
}

// Density and diffuse texture cubes of a shell around the surface
// r = radius (1 + amp n(q)) (the inputs of Sec. 4.2 "Density Texture Cubes"
// and "Diffuse Texture Cubes", standing in for a trained density field and a
// cached diffuse network).  The domain cube [lo, lo + side]^3 has a base grid
// of b^3 cells; cube c (base cell, 0..b-1 per axis) holds the (r+1)^3 fine
// vertices v = c r + (0..r)^3 (x fastest) of the fine grid K = b r, vertex v
// at position lo + v side / K.  Per fine vertex, in FP64 rounded to FP32:
//   density  sigma(v) = sigma_max max(0, 1 - |s(v)| / w), s = shell_distance;
//   diffuse  (c_d r, g, b, tint) = 0.05 + 0.9 u01(SplitMix64 draw keyed by
//            (seed, vertex key, channel)) when `diffuse` != 0.
// A cube is listed when at least one of its vertices has sigma > 0; listed
// cubes are sorted by x + b (y + b z).  Vertices are skipped (left 0) only
// when a Lipschitz bound on s proves |s| >= w, so every vertex's value is the
// formula's, whichever cube holds it.  Returns 0, -1 (bad argument), -2 (oom).
int syn_density_cubes(uint64_t seed, double radius, double amp, int32_t b, int32_t r, double lo, double side,
                      double w, double sigma_max, int32_t diffuse, int32_t** cells_out, float** density_out,
                      float** diffuse_out, int64_t* n_out) {
  if (b < 1 || r < 1 || b > 1024 || r > 64 || !(w > 0) || !(side > 0) || !cells_out || !density_out ||
      !n_out || (diffuse && !diffuse_out))
    return -1;
  const int64_t K = (int64_t)b * r;
  const double hb = side / b, hf = side / (double)K;
  // |grad s| <= sqrt(1 + (|grad n| amp radius / |p|)^2) for |p| >= radius / 2,
  // |grad n| <= 3 sqrt(3) (2 + 0.5 * 4 + 0.25 * 8) / 1.75 < 18 (smoothstep slope
  // 1.5 times the lattice value range 2, per octave times its frequency)
  const double lip = std::sqrt(1.0 + std::pow(18.0 * amp * 2.0, 2.0)) + 1e-3;
  const int64_t nb = (int64_t)b * b * b;
  std::vector<uint8_t> cand((size_t)nb, 0);
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t lin = 0; lin < nb; ++lin) {
    const int64_t x = lin % b, y = (lin / b) % b, z = lin / ((int64_t)b * b);
    const V3 c = {lo + (x + 0.5) * hb, lo + (y + 0.5) * hb, lo + (z + 0.5) * hb};
    const double s = shell_distance(seed, radius, amp, c);
    cand[(size_t)lin] = std::fabs(s) < w + lip * 0.5 * std::sqrt(3.0) * hb + 1e-9;
  }
  std::vector<int64_t> cl;
  for (int64_t lin = 0; lin < nb; ++lin)
    if (cand[(size_t)lin]) cl.push_back(lin);
  const int64_t nc = (int64_t)cl.size();
  const int64_t nv = (int64_t)(r + 1) * (r + 1) * (r + 1);
  std::vector<float> dens((size_t)(nc * nv), 0.0f);
  std::vector<uint8_t> keep((size_t)nc, 0);
  // sub-blocks of up to 4^3 fine cells, each tested at its centre first
  const int sb = std::min(4, r);
  const int nsb = (r + sb - 1) / sb;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t q = 0; q < nc; ++q) {
    const int64_t lin = cl[(size_t)q];
    const int64_t cx = lin % b, cy = (lin / b) % b, cz = lin / ((int64_t)b * b);
    float* blk = dens.data() + (size_t)(q * nv);
    bool any = false;
    for (int bz = 0; bz < nsb; ++bz)
      for (int by = 0; by < nsb; ++by)
        for (int bx = 0; bx < nsb; ++bx) {
          const int x0 = bx * sb, y0 = by * sb, z0 = bz * sb;
          const int x1 = std::min(r, x0 + sb), y1 = std::min(r, y0 + sb), z1 = std::min(r, z0 + sb);
          const V3 m = {lo + (cx * r + 0.5 * (x0 + x1)) * hf, lo + (cy * r + 0.5 * (y0 + y1)) * hf,
                        lo + (cz * r + 0.5 * (z0 + z1)) * hf};
          const double half_diag = 0.5 * hf * std::sqrt((double)((x1 - x0) * (x1 - x0) + (y1 - y0) * (y1 - y0) +
                                                                 (z1 - z0) * (z1 - z0)));
          if (std::fabs(shell_distance(seed, radius, amp, m)) >= w + lip * half_diag + 1e-9) continue;
          for (int k = z0; k <= z1; ++k)
            for (int j = y0; j <= y1; ++j)
              for (int i = x0; i <= x1; ++i) {
                const V3 p = {lo + (double)(cx * r + i) * hf, lo + (double)(cy * r + j) * hf,
                              lo + (double)(cz * r + k) * hf};
                const double s = shell_distance(seed, radius, amp, p);
                const double v = sigma_max * std::max(0.0, 1.0 - std::fabs(s) / w);
                const float fv = (float)v;
                blk[(size_t)i + (size_t)(r + 1) * ((size_t)j + (size_t)(r + 1) * (size_t)k)] = fv;
                if (fv > 0.0f) any = true;
              }
        }
    keep[(size_t)q] = any;
  }
  int64_t n = 0;
  for (int64_t q = 0; q < nc; ++q) n += keep[(size_t)q];
  int32_t* cells = (int32_t*)std::malloc(sizeof(int32_t) * 3 * (size_t)std::max<int64_t>(n, 1));
  float* dout = (float*)std::malloc(sizeof(float) * (size_t)std::max<int64_t>(n * nv, 1));
  float* fout = diffuse ? (float*)std::malloc(sizeof(float) * 4 * (size_t)std::max<int64_t>(n * nv, 1)) : nullptr;
  if (!cells || !dout || (diffuse && !fout)) {
    std::free(cells); std::free(dout); std::free(fout);
    return -2;
  }
  std::vector<int64_t> dst((size_t)nc, -1);
  for (int64_t q = 0, o = 0; q < nc; ++q)
    if (keep[(size_t)q]) dst[(size_t)q] = o++;
  const uint64_t dseed = splitmix64(seed ^ 0x64696666ull);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t q = 0; q < nc; ++q) {
    const int64_t o = dst[(size_t)q];
    if (o < 0) continue;
    const int64_t lin = cl[(size_t)q];
    const int64_t cx = lin % b, cy = (lin / b) % b, cz = lin / ((int64_t)b * b);
    cells[3 * o + 0] = (int32_t)cx;
    cells[3 * o + 1] = (int32_t)cy;
    cells[3 * o + 2] = (int32_t)cz;
    std::memcpy(dout + (size_t)(o * nv), dens.data() + (size_t)(q * nv), sizeof(float) * (size_t)nv);
    if (fout) {
      float* f = fout + (size_t)(o * nv) * 4;
      for (int k = 0; k <= r; ++k)
        for (int j = 0; j <= r; ++j)
          for (int i = 0; i <= r; ++i) {
            const uint64_t key = (uint64_t)(cx * r + i) | ((uint64_t)(cy * r + j) << 21) | ((uint64_t)(cz * r + k) << 42);
            const size_t at = (size_t)i + (size_t)(r + 1) * ((size_t)j + (size_t)(r + 1) * (size_t)k);
            for (int ch = 0; ch < 4; ++ch)
              f[at * 4 + ch] = (float)(0.05 + 0.9 * u01(splitmix64(dseed ^ (key * 4 + (uint64_t)ch))));
          }
    }
  }
  *cells_out = cells;
  *density_out = dout;
  if (diffuse_out) *diffuse_out = fout;
  *n_out = n;
  return 0;
}

// Occupied vertex sets of the encoder levels for a density-cube object: the
// voxels surrounding every possible hit point (Sec. 4.2, "Implementation with
// PSH encoding").  A hit point is a march sample with sigma > 0, so it lies in
// a live fine cell (a fine cell with a vertex of non-zero density, found from
// the cube blocks of syn_density_cubes).  With K = b r a power of two, K x is
// exact in FP32, so a point of fine cell c satisfies c / K <= x < (c+1) / K
// and the FP32 product N x lands in level cells (N c) div K .. (N (c+1)) div K
// (monotone rounding), clamped to N - 1.  Every such level cell is occupied;
// keys_out[l] receives the sorted packed keys of all 8 corners of level l's
// occupied cells.  Returns 0, -1 or -2.
int syn_live_level_vertices(const int32_t* cells, const float* density, int64_t n_cubes, int32_t b, int32_t r,
                            int32_t n_levels, const int32_t* N, uint64_t** keys_out, int64_t* n_out) {
  if (!cells || !density || n_cubes < 0 || b < 1 || r < 1 || n_levels < 1 || !N || !keys_out || !n_out) return -1;
  const int64_t K = (int64_t)b * r;
  const int64_t nv = (int64_t)(r + 1) * (r + 1) * (r + 1);
  // live fine cells as (cube, local cell) bitmask rows of r^3 bits
  const int64_t cpc = (int64_t)r * r * r, words = (cpc + 63) / 64;
  std::vector<uint64_t> live((size_t)(n_cubes * words), 0);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t q = 0; q < n_cubes; ++q) {
    const float* blk = density + (size_t)(q * nv);
    auto at = [&](int i, int j, int k) { return blk[i + (r + 1) * (j + (r + 1) * k)]; };
    for (int k = 0; k < r; ++k)
      for (int j = 0; j < r; ++j)
        for (int i = 0; i < r; ++i) {
          bool any = false;
          for (int d = 0; d < 8 && !any; ++d) any = at(i + (d & 1), j + ((d >> 1) & 1), k + ((d >> 2) & 1)) > 0.0f;
          if (any) {
            const int64_t c = i + (int64_t)r * (j + (int64_t)r * k);
            live[(size_t)(q * words + (c >> 6))] |= 1ull << (c & 63);
          }
        }
  }
  for (int32_t l = 0; l < n_levels; ++l) {
    const int64_t n1 = N[l];
    if (n1 < 1 || n1 > (1 << 20) - 2) return -1;
    const uint64_t ncell = (uint64_t)n1 * n1 * n1;
    uint64_t* occ = (uint64_t*)std::calloc((ncell + 63) / 64, 8);
    if (!occ) return -2;
    std::vector<int64_t> lo_of((size_t)K), hi_of((size_t)K);
    for (int64_t c = 0; c < K; ++c) {
      lo_of[(size_t)c] = std::min(n1 - 1, (n1 * c) / K);
      hi_of[(size_t)c] = std::min(n1 - 1, (n1 * (c + 1)) / K);
    }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t q = 0; q < n_cubes; ++q) {
      const int64_t bx = cells[3 * q], by = cells[3 * q + 1], bz = cells[3 * q + 2];
      for (int64_t c = 0; c < cpc; ++c) {
        if (!((live[(size_t)(q * words + (c >> 6))] >> (c & 63)) & 1ull)) continue;
        const int64_t fx = bx * r + c % r, fy = by * r + (c / r) % r, fz = bz * r + c / ((int64_t)r * r);
        for (int64_t z = lo_of[(size_t)fz]; z <= hi_of[(size_t)fz]; ++z)
          for (int64_t y = lo_of[(size_t)fy]; y <= hi_of[(size_t)fy]; ++y)
            for (int64_t x = lo_of[(size_t)fx]; x <= hi_of[(size_t)fx]; ++x) {
              const uint64_t lin = (uint64_t)x + (uint64_t)n1 * ((uint64_t)y + (uint64_t)n1 * (uint64_t)z);
              if (!bit_get(occ, lin)) bit_set(occ, lin);
            }
      }
    }
    const int rc = cells_to_keys(occ, (int32_t)n1, &keys_out[l], &n_out[l]);
    std::free(occ);
    if (rc != 0) {
      for (int32_t m = 0; m < l; ++m) { std::free(keys_out[m]); keys_out[m] = nullptr; }
      return rc;
    }
  }
  return 0;
}

}  // extern "C"
