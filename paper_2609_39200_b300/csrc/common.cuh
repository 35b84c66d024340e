// common.cuh - shared device helpers of the HAMLS library (sm_103a).
//
// Neighbour structure. Points on S^2 are bucketed into B latitude bands and P
// longitude cells per band. The band coordinate is
//   zeta(z) = sign(z) (1 - sqrt(1 - |z|)),
// which is close to linear in the colatitude (bands are 2.8/B to 4/B rad
// wide), and the longitude coordinate is the "diamond" parameter
//   psi = quadrant + |.| / (|x| + |y|)  in [0, 4),
// a monotone function of the longitude that needs one IEEE division and no
// transcendental function. Keys key = band * P + cell are therefore computed
// bit-identically by any IEEE-754 implementation that uses the same formula.
// Sorting the points by key makes every (band, cell range) a contiguous run
// of the sorted arrays, so a spherical cap is enumerated as at most two
// contiguous runs per band, found through a CSR array start[B*P + 1].
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

namespace hamls {

constexpr unsigned FULL = 0xffffffffu;
constexpr int KMAX = 4;          // MLS degree limit (m <= 15)
constexpr int KNN_MAX = 128;     // largest n for the k-nearest-neighbour search

// device status bits (reported by hamls_sync)
enum : unsigned {
  ST_UNDERDET = 1u,     // fewer than m nodes in a support after the guard
  ST_SUPPORT = 2u,      // delta >= pi/2
  ST_NONFINITE = 4u,    // non-finite value
  ST_BADNODE = 8u,      // node not a unit vector / not finite
  ST_KNN = 16u,         // k-nearest-neighbour search did not converge (M < n)
  ST_VORONOI = 32u,     // a Voronoi cell could not be formed (reaches 1.5 rad, > 32 edges)
};

// device counters
enum { C_SUM_N = 0, C_MIN_N, C_MAX_N, C_REG, C_GUARD, C_REDO, C_DROP, C_GUARD_LIST, C_REDO_LIST,
       C_BATCH, C_TILE, C_KNN_CAND, C_KNN_SCAN, C_KNN_EXACT_FB, C_LIST_BATCH, C_OP_TOTAL, C_REG_LIST, C_NCOUNT };

struct DevStatus {
  unsigned flags;
  unsigned tc_err;          // tensor-core tiles that gave up waiting (batched step 3)
  unsigned long long cnt[C_NCOUNT];
};

// A point set with its band/cell structure (sorted order).
struct Cells {
  int B, P;                 // bands, cells per band (P multiple of 4)
  int n;                    // number of points
  const uint32_t* start;    // CSR over cells, B*P + 1 entries
  const float4* pf;         // sorted points, FP32 (x, y, z, value slot)
  const double* px;         // sorted points, FP64 SoA
  const double* py;
  const double* pz;
  const uint32_t* perm;     // sorted position -> original index
  // per band edge e = 0..B (zeta = -1 + 2e/B): sin and cos of half its
  // colatitude and its z (edge_half_angles, tabulated once per plan)
  const float4* edge;
};

// ---------------------------------------------------------------- warp utils
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

__device__ __forceinline__ void set_flag(DevStatus* st, unsigned f) { atomicOr(&st->flags, f); }

// ------------------------------------------------------------ exact cell key
// Bit-exact: only IEEE add/sub/mul/div/sqrt with round-to-nearest, no FMA.
__device__ __forceinline__ uint32_t cell_key64(double x, double y, double z, int B, int P) {
  double az = fabs(z);
  double s = __dsqrt_rn(__dsub_rn(1.0, az));
  double om = __dsub_rn(1.0, s);
  double zeta = (z < 0) ? -om : om;
  int band = (int)floor(__dmul_rn(__dadd_rn(zeta, 1.0), (double)(B / 2)));
  band = min(max(band, 0), B - 1);
  double ax = fabs(x), ay = fabs(y);
  double den = __dadd_rn(ax, ay);
  int q;
  double num;
  if (x > 0 && y >= 0) { q = 0; num = ay; }
  else if (x <= 0 && y > 0) { q = 1; num = ax; }
  else if (x < 0 && y <= 0) { q = 2; num = ay; }
  else if (x >= 0 && y < 0) { q = 3; num = ax; }
  else { q = 0; num = 0.0; }
  double frac = den > 0 ? __ddiv_rn(num, den) : 0.0;
  int qc = P / 4;
  int w = (int)floor(__dmul_rn(frac, (double)qc));
  w = min(max(w, 0), qc - 1);
  return (uint32_t)(band * P + q * qc + w);
}

// The same key from FP32 arithmetic where that is provably the same: false
// when a band or cell coordinate lies within 2e-3 of an integer (the FP32
// error there is below 7e-4 for B/2, P/4 <= 2048) or when x or y rounds to
// zero in FP32, and the caller then takes cell_key64. t = 1 - |z| comes
// from FP64, so that the polar cancellation is exact; xf, yf, zf are x, y, z
// rounded to FP32.
__device__ __forceinline__ bool cell_key_fast(float xf, float yf, float zf, float t, int B, int P, uint32_t& key) {
  if (xf == 0.f || yf == 0.f) return false;
  const float om = 1.f - sqrtf(t);
  const float zeta = zf < 0.f ? -om : om;
  const float bf = (zeta + 1.f) * (float)(B / 2);
  const float fb = floorf(bf);
  if (!(bf - fb > 2e-3f && bf - fb < 1.f - 2e-3f)) return false;
  const float ax = fabsf(xf), ay = fabsf(yf);
  int q;
  float num;
  if (xf > 0.f && yf > 0.f) { q = 0; num = ay; }
  else if (xf < 0.f && yf > 0.f) { q = 1; num = ax; }
  else if (xf < 0.f) { q = 2; num = ay; }
  else { q = 3; num = ax; }
  const int qc = P / 4;
  const float cf = (num / (ax + ay)) * (float)qc;
  const float fc = floorf(cf);
  if (!(cf - fc > 2e-3f && cf - fc < 1.f - 2e-3f)) return false;
  const int band = min(max((int)fb, 0), B - 1);
  const int w = min(max((int)fc, 0), qc - 1);
  key = (uint32_t)(band * P + q * qc + w);
  return true;
}

// FP32 versions used only to enumerate candidates (with margins).
__device__ __forceinline__ int band_of_f(float z, int B) {
  float s = sqrtf(fmaxf(0.f, 1.f - fabsf(z)));
  float zeta = (z < 0.f) ? -(1.f - s) : (1.f - s);
  int b = (int)floorf((zeta + 1.f) * (0.5f * (float)B));
  return min(max(b, 0), B - 1);
}


// Continuous cell coordinate q P/4 + frac P/4 in [0, P] of a longitude: the
// FP64 cell index of a point is its floor (clamped within the quadrant). It
// is monotone and continuous in longitude, across quadrants too, so a run of
// cells for an arc of longitudes is floor(lo - eps) .. floor(hi + eps).
__device__ __forceinline__ float cell_coord_f(float x, float y, int P) {
  const float ax = fabsf(x), ay = fabsf(y), den = ax + ay;
  int q;
  float num;
  if (x > 0.f && y >= 0.f) { q = 0; num = ay; }
  else if (x <= 0.f && y > 0.f) { q = 1; num = ax; }
  else if (x < 0.f && y <= 0.f) { q = 2; num = ay; }
  else if (x >= 0.f && y < 0.f) { q = 3; num = ax; }
  else { q = 0; num = 0.f; }
  const float frac = den > 0.f ? __fdividef(num, den) : 0.f;
  return ((float)q + frac) * (float)(P / 4);
}

// ------------------------------------------------------------- cap queries
// Geodesic cap of radius r around a unit vector q, prepared for candidate
// enumeration in FP32. Every margin enlarges the enumerated set; the caller
// decides membership with its own exact test.
//
// The longitude half-width dphi of the cap at colatitude theta follows from
// the spherical law of cosines; written as
//   1 - cos(dphi) = 2 sin((r + dt)/2) sin((r - dt)/2) / (sin(theta) sin(theta_q)),
// dt = theta - theta_q, it has no cancellation near the poles or near the
// cap's rim. Everything is carried as sines and cosines of half angles, so a
// band costs products and square roots only: a band edge zeta has
// sin(theta/2) = (1 - zeta)/sqrt 2 (zeta >= 0) or cos(theta/2) = (1 + zeta)/sqrt 2
// (zeta < 0), the exact inverse of zeta(z); the half angles of (r + dt)/2 and
// (r - dt)/2 follow by the addition theorems.
struct Cap {
  float zq, sq;             // cos and sin of the colatitude of q
  float hs, hc;             // sin and cos of half the colatitude of q
  float rs, rc;             // sin and cos of half the (widened) radius
  float cph, sph;           // cos/sin longitude of q
  float zlo, zhi;           // z extent of the cap, widened (band index range)
  float zstar, cstar;       // z of the widest longitude extent (3 if none), cos of that half-width
  int polar;                // enumerate whole bands (q at a pole, or a cap beyond ~86 degrees)
};

// FP32 is enough here: rounding q moves it by < 1e-7 rad, far inside the widening of r
__device__ __forceinline__ Cap make_cap_f(float fx, float fy, float fz, float rf) {
  const float PI_F = 3.14159265f;
  Cap c;
  const float sq = sqrtf(fx * fx + fy * fy);
  c.zq = fz;
  c.sq = sq;
  // approximate divisions below: their 2-ulp errors are far inside the
  // margins added to the half-widths and to the runs
  if (sq > 1e-12f) {
    const float isq = __fdividef(1.f, sq);
    c.cph = fx * isq;
    c.sph = fy * isq;
  } else {
    c.cph = 1.f;
    c.sph = 0.f;
  }
  const float r = fminf(rf * (1.f + 2e-5f) + 2e-6f, PI_F);
  sincosf(0.5f * r, &c.rs, &c.rc);
  if (fz >= 0.f) {
    c.hc = sqrtf(0.5f * (1.f + fz));
    c.hs = __fdividef(sq, 2.f * c.hc);
  } else {
    c.hs = sqrtf(0.5f * (1.f - fz));
    c.hc = __fdividef(sq, 2.f * c.hs);
  }
  const float sr = 2.f * c.rs * c.rc, cr = (c.rc - c.rs) * (c.rc + c.rs);
  const bool north = c.hs * c.rc <= c.hc * c.rs;   // theta_q <= r
  const bool south = c.hc * c.rc <= c.hs * c.rs;   // theta_q + r >= pi
  c.polar = (sq < 1e-6f) || (r >= 1.5f);
  c.zhi = north ? 1.f : fminf(1.f, fz * cr + sq * sr + 4e-6f);
  c.zlo = south ? -1.f : fmaxf(-1.f, fz * cr - sq * sr - 4e-6f);
  const float ratio = __fdividef(sr, fmaxf(sq, 1e-30f));
  if (ratio < 1.f && !c.polar) {
    c.cstar = sqrtf(1.f - ratio * ratio);
    c.zstar = __fdividef(fz, cr);                     // cos of the colatitude of the widest extent
  } else {
    c.cstar = -1.f;
    c.zstar = 3.f;
  }
  return c;
}

__device__ __forceinline__ Cap make_cap(double qx, double qy, double qz, double r) {
  return make_cap_f((float)qx, (float)qy, (float)qz, (float)r);
}

// Half angles (a = sin(theta/2), b = cos(theta/2)) of the band edge zeta.
__device__ __forceinline__ void edge_half_angles(float zeta, float& a, float& b) {
  if (zeta >= 0.f) {
    a = (1.f - zeta) * 0.70710678f;
    b = sqrtf(fmaxf(0.f, 1.f - a * a));
  } else {
    b = (1.f + zeta) * 0.70710678f;
    a = sqrtf(fmaxf(0.f, 1.f - b * b));
  }
}

// cos of the cap's longitude half-width at the colatitude with half angles
// (a, b): 1 where that colatitude is outside the cap's range (the band's part
// of the cap then ends at the cap's rim, width 0), -1 where the whole circle
// of latitude is inside or the geometry degenerates (whole band).
__device__ __forceinline__ float cap_cos_halfwidth(const Cap& c, float a, float b) {
  const float sdt = a * c.hc - b * c.hs, cdt = b * c.hc + a * c.hs;   // sin, cos of dt/2
  const float sp = c.rs * cdt + c.rc * sdt, sm = c.rs * cdt - c.rc * sdt;
  if (!(sp > 0.f) || !(sm > 0.f)) return 1.f;
  const float den = 2.f * a * b * c.sq;
  if (!(den > 1e-12f)) return -1.f;
  return 1.f - __fdividef(2.f * sp * sm, den);
}

// The (at most two) contiguous runs of sorted points of band b that can lie
// in the cap: [s0, s0+n0) and [s1, s1+n1).
__device__ __forceinline__ void band_runs(const Cells& g, const Cap& c, int b, uint32_t& s0,
                                          uint32_t& n0, uint32_t& s1, uint32_t& n1) {
  n0 = n1 = 0;
  s0 = s1 = 0;
  const int P = g.P;
  // band b spans zeta in [-1 + 2b/B, -1 + 2(b+1)/B)
  const float4 eb = g.edge[b], et = g.edge[b + 1];
  const float ab = eb.x, bb = eb.y, z_bot = eb.z, at = et.x, bt = et.y, z_top = et.z;
  if (z_top < c.zlo || z_bot > c.zhi) return;               // band outside the cap's colatitudes
  const uint32_t base = (uint32_t)b * (uint32_t)P;
  bool full = c.polar;
  if (!full) {
    float cmin = fminf(cap_cos_halfwidth(c, at, bt), cap_cos_halfwidth(c, ab, bb));
    if (c.zstar > z_bot - 1e-4f && c.zstar < z_top + 1e-4f) cmin = fminf(cmin, c.cstar);
    cmin = cmin - 2e-5f * (1.f - cmin) - 1e-6f;
    full = !(cmin > 0.f);
    if (!full) {
      cmin = fminf(cmin, 1.f);
      const float sd = sqrtf(fmaxf(0.f, 1.f - cmin * cmin));
      const float xa = c.cph * cmin + c.sph * sd, ya = c.sph * cmin - c.cph * sd;   // phi_q - dphi
      const float xb = c.cph * cmin - c.sph * sd, yb = c.sph * cmin + c.cph * sd;   // phi_q + dphi
      // the FP32 coordinates are within 5e-4 cells of the exact ones (P <= 8192)
      const float ga = cell_coord_f(xa, ya, P), gb = cell_coord_f(xb, yb, P);
      int lo_c = (int)floorf(ga - 2e-3f), hi_c = (int)floorf(gb + 2e-3f);
      if (ga > gb) hi_c += P;
      if (hi_c - lo_c + 1 >= P) {
        full = true;
      } else if (lo_c < 0) {
        s0 = g.start[base + lo_c + P];
        n0 = g.start[base + P] - s0;
        s1 = g.start[base];
        n1 = g.start[base + hi_c + 1] - s1;
      } else if (hi_c >= P) {
        s0 = g.start[base + lo_c];
        n0 = g.start[base + P] - s0;
        s1 = g.start[base];
        n1 = g.start[base + hi_c - P + 1] - s1;
      } else {
        s0 = g.start[base + lo_c];
        n0 = g.start[base + hi_c + 1] - s0;
      }
    }
  }
  if (full) {
    s0 = g.start[base];
    n0 = g.start[base + P] - s0;
    n1 = 0;
  }
}

__device__ __forceinline__ void cap_band_range(const Cells& g, const Cap& c, int& b_lo, int& b_hi) {
  b_lo = max(band_of_f(c.zlo, g.B) - 1, 0);
  b_hi = min(band_of_f(c.zhi, g.B) + 1, g.B - 1);
}

// ---------------------------------------------------------- lane groups
// A query can be served by a group of G consecutive lanes (G = 8, 16 or 32):
// every shuffle below has width G, so the groups of a warp run the same
// instructions side by side on their own queries. Loops run while any group
// still has work (warp-wide votes keep the warp converged); a group without
// work takes part with neutral values.
//
// Group-cooperative enumeration of every sorted point index that can lie in
// the cap. The runs of G consecutive bands are concatenated and dealt to the
// group's lanes G at a time, so consecutive lanes read consecutive points.
// f(valid, idx) is called by all 32 lanes together; an inactive group (or a
// lane past the end) gets valid = false.
//
// With MIDOUT the bands are visited from the cap centre's band outwards
// (offsets 0, +1, -1, +2, -2, ...), so candidates arrive roughly nearest
// first; searches that keep the n nearest then rarely update after a while.
// stop() (warp-uniform) ends the enumeration early; the default never does.
struct NoStop {
  __device__ __forceinline__ constexpr bool operator()() const { return false; }
};

template <int G, bool MIDOUT = false, class F, class S = NoStop>
__device__ __forceinline__ void for_cap_candidates_g(const Cells& g, const Cap& c, bool active, F&& f,
                                                     S stop = S()) {
  const int gl = threadIdx.x & (G - 1);
  int b_lo, b_hi;
  cap_band_range(g, c, b_lo, b_hi);
  const int bc = MIDOUT ? min(max(band_of_f(c.zq, g.B), b_lo), b_hi) : b_lo;
  int span = MIDOUT ? 2 * max(bc - b_lo, b_hi - bc) + 1 : b_hi - b_lo + 1;
  if (!active) span = 0;
  for (int k0 = 0; __any_sync(FULL, k0 < span) && !stop(); k0 += G) {
    const int k = k0 + gl;
    const int b = MIDOUT ? bc + ((k & 1) ? (k + 1) / 2 : -(k / 2)) : b_lo + k;
    uint32_t s0 = 0, n0 = 0, s1 = 0, n1 = 0;
    if (k < span && b >= b_lo && b <= b_hi) band_runs(g, c, b, s0, n0, s1, n1);
    const uint32_t len = n0 + n1;
    uint32_t incl = len;
#pragma unroll
    for (int o = 1; o < G; o <<= 1) {
      const uint32_t t = __shfl_up_sync(FULL, incl, o, G);
      if (gl >= o) incl += t;
    }
    const uint32_t excl = incl - len;
    const uint32_t total = __shfl_sync(FULL, incl, G - 1, G);
    for (uint32_t base = 0; __any_sync(FULL, base < total) && !stop(); base += G) {
      const uint32_t v = base + gl;
      int owner = 0;
#pragma unroll
      for (int step = G / 2; step > 0; step >>= 1) {
        const int cand = owner + step;
        const uint32_t e = __shfl_sync(FULL, excl, cand & (G - 1), G);
        if (cand < G && e <= v) owner = cand;
      }
      const uint32_t oe = __shfl_sync(FULL, excl, owner, G);
      const uint32_t os0 = __shfl_sync(FULL, s0, owner, G);
      const uint32_t on0 = __shfl_sync(FULL, n0, owner, G);
      const uint32_t os1 = __shfl_sync(FULL, s1, owner, G);
      const bool valid = v < total;
      const uint32_t off = v - oe;
      const uint32_t idx = valid ? ((off < on0) ? os0 + off : os1 + (off - on0)) : 0u;
      f(valid, idx);
    }
  }
}

// The warp-per-query enumeration (one group of 32 lanes).
template <bool MIDOUT = false, class F, class S = NoStop>
__device__ __forceinline__ void for_cap_candidates(const Cells& g, const Cap& c, F&& f, S stop = S()) {
  for_cap_candidates_g<32, MIDOUT>(g, c, true, f, stop);
}

// Number of candidates the enumeration would visit (no point is read).
__device__ __forceinline__ uint32_t cap_box_count(const Cells& g, const Cap& c) {
  const int lane = threadIdx.x & 31;
  int b_lo, b_hi;
  cap_band_range(g, c, b_lo, b_hi);
  uint32_t tot = 0;
  for (int b0 = b_lo; b0 <= b_hi; b0 += 32) {
    const int b = b0 + lane;
    uint32_t s0 = 0, n0 = 0, s1 = 0, n1 = 0;
    if (b <= b_hi) band_runs(g, c, b, s0, n0, s1, n1);
    tot += n0 + n1;
  }
  return warp_sum(tot);
}

// ----------------------------------------------------------- exact distance
// |x - q|^2 in FP64 with a fixed order and no contraction.
__device__ __forceinline__ double chord2_exact(double x, double y, double z, double qx, double qy, double qz) {
  double dx = __dsub_rn(x, qx), dy = __dsub_rn(y, qy), dz = __dsub_rn(z, qz);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Wendland phi_{3,2}(r) = (1-r)^6 (35 r^2 + 18 r + 3) on [0,1).
template <typename T>
__device__ __forceinline__ T wendland(T r) {
  T om = r < T(1) ? T(1) - r : T(0);
  T om2 = om * om;
  T om6 = om2 * om2 * om2;
  return om6 * ((T(35) * r + T(18)) * r + T(3));
}

// Wendland phi_{3,1}(r) = (1-r)^4 (4 r + 1) on [0,1).
template <typename T>
__device__ __forceinline__ T wendland31(T r) {
  T om = r < T(1) ? T(1) - r : T(0);
  T om2 = om * om;
  return om2 * om2 * (T(4) * r + T(1));
}

// phi of eq. weight_function_radial: fn 0 -> phi_{3,2} (default), 1 -> phi_{3,1}
template <typename T>
__device__ __forceinline__ T weight_phi(int fn, T r) {
  return fn == 1 ? wendland31(r) : wendland(r);
}

__device__ __forceinline__ double geodesic_from_chord2(double c2) { return 2.0 * asin(0.5 * sqrt(c2)); }
__device__ __forceinline__ float geodesic_from_chord2(float c2) { return 2.f * asinf(0.5f * sqrtf(c2)); }

// The same in FP32 by the Maclaurin series of arcsin,
//   asin(s) = sum_k (2k)! / (4^k (k!)^2 (2k + 1)) s^(2k+1),
// through s^11 where s = sqrt(c2)/2 <= 1/4 (the first omitted term is below
// 1.1e-9 of the sum there, far below FP32 rounding), asinf beyond: the MLS
// weights of supports up to about 29 degrees without the general routine.
__device__ __forceinline__ float geodesic_series_f(float c2) {
  const float s = 0.5f * sqrtf(c2);
  if (s > 0.25f) return 2.f * asinf(s);
  const float t = s * s;
  float p = 63.f / 2816.f;
  p = __fmaf_rn(p, t, 35.f / 1152.f);
  p = __fmaf_rn(p, t, 5.f / 112.f);
  p = __fmaf_rn(p, t, 3.f / 40.f);
  p = __fmaf_rn(p, t, 1.f / 6.f);
  p = __fmaf_rn(p, t, 1.f);
  return 2.f * s * p;
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

}  // namespace hamls
