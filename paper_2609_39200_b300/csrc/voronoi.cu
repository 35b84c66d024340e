// voronoi.cu - spherical Voronoi cell areas of the nodes: the weights v_i
// that rescale the local MLS weights (Sec. 2.2, the remark after Theorem 2.1;
// every experiment of Sec. 3 uses them).
//
// The cell of node x_i is V_i = { p in S^2 : p . x_i >= p . x_j for all j }.
// In the gnomonic chart at x_i, p = x_i + u e1 + v e2 with (e1, e2) a
// tangent frame, great circles are straight lines and node x_j
// (d = x_j - x_i) keeps the half-plane
//     u a_j + v b_j <= h_j,   a_j = e1.d,  b_j = e2.d,  h_j = -x_i.d
// (h_j = |d|^2 / 2 for unit vectors), so V_i is a convex polygon around the
// origin as long as it lies in the open hemisphere around x_i. One warp per
// node keeps that polygon with one edge and its first vertex per lane (at
// most 32 edges) and clips it by one node at a time, starting from the
// square |u|, |v| <= tan 1.5.
//
// Which nodes can cut? Node x_j cuts off a vertex c only if it is closer to c
// than x_i (it lies in the "flower" cap of c, radius |c - x_i|). So:
//  1. every node within angle r of x_i, nearest first, with r = r0 (two mean
//     node spacings) and doubled, for the new annulus only, until no side of
//     the square is left (a cell at the rim of a hole is closed by the rim
//     nodes near it: their bisectors all pass near the hole's centre) and,
//     up to 4 r0, until every vertex is settled. A vertex c with
//     |c - x_i| <= r / 2 (chords) is a vertex of V_i: a node of its flower
//     cap lies within 2 |c - x_i| <= r of x_i;
//  2. for every vertex still unsettled, the nodes of its own flower cap: the
//     first round that holds one cuts the vertex off by the node closest to
//     it, and the search ends; the new vertices get searches of their own.
//     A search that finds none settles the vertex. For a cell at a hole's
//     rim the flower cap is about the hole, whose cells hold no node.
// In step 1 a candidate whose line lies farther from the origin than every
// vertex (h^2 >= R^2 (a^2 + b^2)) cannot cut; the others are tested against
// every vertex at once, and only those that cut are clipped, one at a time.
//
// Precision. The clipping runs in FP32 on differences d taken from a hi/lo
// split of the nodes (hi = the FP32 copy of the cell structure, lo = the FP32
// rounding of the remainder), accurate to about 1e-7 relative, with no FP64
// arithmetic per candidate (sm_103a runs FP64 at 1/64 of the FP32 rate). Mixed plans take the
// area from the FP32 polygon. FP64 plans keep its edges (the nodes that bound
// the cell) and recompute lines, vertices and area in FP64: a decision that
// FP32 gets wrong near a degenerate vertex adds or drops an edge of relative
// length about 1e-7, which changes the area by about 1e-14 relative.
//
// Area: the fan of solid angles (x_i, c_k, c_k+1), by the formula of van
// Oosterom and Strackee (1983); with c = (u, v, 1) in the frame (e1, e2, x_i)
//   E_k = 2 atan2(u_k v_k+1 - u_k+1 v_k,
//                 1 + n_k + n_k+1 + n_k n_k+1 + u_k u_k+1 + v_k v_k+1),
//   n = sqrt(1 + u^2 + v^2).
//
// Exact duplicates of x_i share the cell equally (nodes closer than about
// 1e-15, which the hi/lo split cannot tell apart, count as duplicates). A cell
// that reaches 1.5 rad from its node, needs more than 32 edges or more than
// VOR_FLOWER_LIMIT flower searches sets ST_VORONOI and gets a NaN area.
#include "common.cuh"
#include "kernels.h"

namespace hamls {

constexpr int VOR_WARPS = 4;
constexpr int VOR_FLOWER_LIMIT = 512;   // flower-cap searches per cell
constexpr int VOR_GROW_LIMIT = 16;      // doublings of the cap around the node
constexpr float VOR_THETA_MAX = 1.5f;   // the square's inscribed circle (angle, rad)
constexpr float VOR_EPS = 6e-8f;

// The warp's polygon: lane k < n holds edge k (u a + v b <= h) and vertex k,
// where edge k-1 meets edge k; counter-clockwise around the origin.
struct VPoly {
  int n;          // number of edges (the same in every lane)
  float a, b, h;
  float u, v;
  int id;         // sorted position of the node of the edge; -1: a side of the square
  bool fin;       // the vertex is known to be a vertex of the cell
  bool tag;       // the vertex whose flower cap is being searched
};

struct VorNode {
  float3 hi, lo;            // the node: hi + lo
  float3 e1, e2;            // tangent frame
  int s;                    // its sorted position
};

__device__ __forceinline__ void vor_meet(float a1, float b1, float h1, float a2, float b2, float h2, float& u,
                                         float& v) {
  const float det = a1 * b2 - a2 * b1;
  u = (h1 * b2 - h2 * b1) / det;
  v = (a1 * h2 - a2 * h1) / det;
}

// the square |u|, |v| <= L: edges u <= L, v <= L, -u <= L, -v <= L; vertex k
// (edge k-1 meets edge k) at (L, -L), (L, L), (-L, L), (-L, -L)
__device__ __forceinline__ void vor_square(VPoly& P, float L) {
  const int k = threadIdx.x & 3;
  P.n = 4;
  P.a = (k == 0) ? 1.f : (k == 2) ? -1.f : 0.f;
  P.b = (k == 1) ? 1.f : (k == 3) ? -1.f : 0.f;
  P.h = L;
  P.u = (k <= 1) ? L : -L;
  P.v = (k == 1 || k == 2) ? L : -L;
  P.id = -1;
  P.fin = false;
  P.tag = false;
}

// largest squared distance of a vertex from the origin
__device__ __forceinline__ float vor_r2(const VPoly& P) {
  const int lane = threadIdx.x & 31;
  const float r2 = lane < P.n ? P.u * P.u + P.v * P.v : 0.f;
  return __uint_as_float(__reduce_max_sync(FULL, __float_as_uint(r2)));
}

// Clip the polygon by u A + v B <= H (the line of node cid). The vertices
// outside form one cyclic run; rounding can mark a vertex that lies on the
// line as outside on its own, so the run is the one around the vertex
// farthest outside. Returns false if the polygon would need more than 32
// edges, every vertex is outside or a new vertex is not finite.
__device__ __forceinline__ bool vor_clip(VPoly& P, float A, float B, float H, int cid) {
  const int lane = threadIdx.x & 31;
  const int n = P.n;
  const float s = A * P.u + B * P.v - H;
  const float tol = 8.f * VOR_EPS * (fabsf(A * P.u) + fabsf(B * P.v) + H);
  const bool out = lane < n && s > tol;
  const unsigned m = __ballot_sync(FULL, out);
  if (m == 0u) return true;
  const unsigned key = out ? __float_as_uint(s) : 0u;
  const unsigned kmax = __reduce_max_sync(FULL, key);
  const int km = __ffs(__ballot_sync(FULL, out && key == kmax)) - 1;
  const unsigned long long nmask = (n == 32) ? 0xffffffffull : ((1ull << n) - 1ull);
  const unsigned long long mm = (unsigned long long)m;
  const unsigned long long r = ((mm >> km) | (mm << (n - km))) & nmask;   // rotated: km at bit 0
  const int fwd = __ffsll((long long)~r) - 1;                              // km and the run after it
  if (fwd >= n) return false;
  const int back = __clzll((long long)~(r << (64 - n)));                   // the run before km
  const int rl = fwd + back;
  const int np = n - rl + 2;
  if (np > 32) return false;
  int s0 = km - back;
  if (s0 < 0) s0 += n;
  // new position p <= n - rl takes old edge and vertex s0 + rl - 1 + p; the
  // new edge goes last; the vertices at both ends of the new edge are new
  int src = s0 + rl - 1 + lane;
  if (src >= n) src -= n;
  if (src >= n) src = 0;
  const float ga = __shfl_sync(FULL, P.a, src), gb = __shfl_sync(FULL, P.b, src), gh = __shfl_sync(FULL, P.h, src);
  const float gu = __shfl_sync(FULL, P.u, src), gv = __shfl_sync(FULL, P.v, src);
  const int gid = __shfl_sync(FULL, P.id, src);
  const int gfl = __shfl_sync(FULL, (P.fin ? 1 : 0) | (P.tag ? 2 : 0), src);
  const float pa = __shfl_up_sync(FULL, ga, 1), pb = __shfl_up_sync(FULL, gb, 1), ph = __shfl_up_sync(FULL, gh, 1);
  if (lane <= n - rl) {
    P.a = ga;
    P.b = gb;
    P.h = gh;
    P.u = gu;
    P.v = gv;
    P.id = gid;
    P.fin = (gfl & 1) != 0;
    P.tag = (gfl & 2) != 0;
  }
  if (lane == 0) {
    vor_meet(A, B, H, ga, gb, gh, P.u, P.v);
    P.fin = false;
    P.tag = false;
  }
  if (lane == np - 1) {
    P.a = A;
    P.b = B;
    P.h = H;
    P.id = cid;
    vor_meet(pa, pb, ph, A, B, H, P.u, P.v);
    P.fin = false;
    P.tag = false;
  }
  P.n = np;
  return __all_sync(FULL, lane >= np || (isfinite(P.u) && isfinite(P.v)));
}

// The half-plane of the node at sorted position idx (FP32, from the hi/lo
// split). Returns false for an exact duplicate of the node.
__device__ __forceinline__ bool vor_line(const Cells& g, const float4* __restrict__ lo, const VorNode& q,
                                         uint32_t idx, float& a, float& b, float& h) {
  const float4 ph = g.pf[idx], pl = lo[idx];
  const float dx = (ph.x - q.hi.x) + (pl.x - q.lo.x);
  const float dy = (ph.y - q.hi.y) + (pl.y - q.lo.y);
  const float dz = (ph.z - q.hi.z) + (pl.z - q.lo.z);
  a = q.e1.x * dx + q.e1.y * dy + q.e1.z * dz;
  b = q.e2.x * dx + q.e2.y * dy + q.e2.z * dz;
  h = 0.5f * (dx * dx + dy * dy + dz * dz);
  return !(dx == 0.f && dy == 0.f && dz == 0.f);
}

// does the line u a + v b = h leave the point (u, v) outside (beyond rounding)
__device__ __forceinline__ bool vor_outside(float a, float b, float h, float u, float v) {
  return a * u + b * v - h > 8.f * VOR_EPS * (fabsf(a * u) + fabsf(b * v) + h);
}

// One round of candidates around the node (one per lane): skip those whose
// line lies farther from the origin than every vertex, test the rest against
// every vertex at once, and clip by the ones that cut, the nearest first.
// Nodes with h below hskip were handled by a smaller cap. Returns false on a
// polygon failure.
__device__ __forceinline__ bool vor_round(const Cells& g, const float4* __restrict__ lo, const VorNode& q, VPoly& P,
                                          float& R2, bool valid, uint32_t idx, int& dups, bool count_dups,
                                          float hskip) {
  const int lane = threadIdx.x & 31;
  float ca = 0.f, cb = 0.f, ch = 0.f;
  bool pend = valid && (int)idx != q.s;
  if (pend) {
    if (!vor_line(g, lo, q, idx, ca, cb, ch)) {
      if (count_dups) ++dups;
      pend = false;
    } else if (!(ch > 0.f) || ch < hskip) {
      pend = false;
    }
  }
  for (;;) {
    // the line lies h / |(a, b)| from the origin: it cuts only if that is
    // below the polygon's radius
    if (pend && !(ch * ch < R2 * 1.0001f * (ca * ca + cb * cb))) pend = false;
    if (__ballot_sync(FULL, pend) == 0u) return true;
    bool cut = false;
    for (int k = 0; k < P.n; ++k) {
      const float uk = __shfl_sync(FULL, P.u, k), vk = __shfl_sync(FULL, P.v, k);
      cut = cut || vor_outside(ca, cb, ch, uk, vk);
    }
    pend = pend && cut;
    if (__ballot_sync(FULL, pend) == 0u) return true;
    const unsigned key = pend ? __float_as_uint(ch) : 0xffffffffu;
    const unsigned kmin = __reduce_min_sync(FULL, key);
    const int j = __ffs(__ballot_sync(FULL, pend && key == kmin)) - 1;
    const float A = __shfl_sync(FULL, ca, j), B = __shfl_sync(FULL, cb, j), H = __shfl_sync(FULL, ch, j);
    const int cid = __shfl_sync(FULL, (int)idx, j);
    if (lane == j) pend = false;
    if (__any_sync(FULL, lane < P.n && P.id == cid)) continue;   // already an edge
    if (!vor_clip(P, A, B, H, cid)) return false;
    R2 = vor_r2(P);
  }
}

// One round of the flower cap of the vertex (fu, fv): the nodes closer to it
// than x_i are exactly those whose line leaves it outside. Clip by the one
// closest to the vertex (largest a fu + b fv - h, which is proportional to
// p.x_j - p.x_i at the vertex p) and report the vertex as cut. Returns false
// on a polygon failure.
__device__ __forceinline__ bool vor_flower_round(const Cells& g, const float4* __restrict__ lo, const VorNode& q,
                                                 VPoly& P, float& R2, bool valid, uint32_t idx, float fu, float fv,
                                                 bool& cut_vertex) {
  float ca = 0.f, cb = 0.f, ch = 0.f;
  bool pend = valid && (int)idx != q.s;
  if (pend) pend = vor_line(g, lo, q, idx, ca, cb, ch) && ch > 0.f && vor_outside(ca, cb, ch, fu, fv);
  const int lane = threadIdx.x & 31;
  const float depth = ca * fu + cb * fv - ch;
  for (;;) {
    if (__ballot_sync(FULL, pend) == 0u) return true;
    const unsigned key = pend ? __float_as_uint(depth) : 0u;          // depth > 0 where pending
    const unsigned kmax = __reduce_max_sync(FULL, key);
    const int j = __ffs(__ballot_sync(FULL, pend && key == kmax)) - 1;
    const float A = __shfl_sync(FULL, ca, j), B = __shfl_sync(FULL, cb, j), H = __shfl_sync(FULL, ch, j);
    const int cid = __shfl_sync(FULL, (int)idx, j);
    if (lane == j) pend = false;
    if (__any_sync(FULL, lane < P.n && P.id == cid)) continue;   // already an edge
    cut_vertex = true;
    if (!vor_clip(P, A, B, H, cid)) return false;
    R2 = vor_r2(P);
    return true;
  }
}

// R^2 of the vertices settled by a cap of angle r: chord at most half its chord
__device__ __forceinline__ float vor_settled_r2(float r) {
  if (r >= 3.14159265f) return 1e30f;
  const float t = tanf(2.f * asinf(0.5f * sinf(0.5f * r)));
  return t * t * (1.f - 1e-4f);
}

// FP64 area of the cell bounded by the nodes of the polygon's edges
__device__ __forceinline__ double vor_area64(const Cells& g, int s, const VPoly& P) {
  const int lane = threadIdx.x & 31;
  const double qx = g.px[s], qy = g.py[s], qz = g.pz[s];
  const double tx = fabs(qz) < 0.9 ? 0.0 : 1.0, tz = 1.0 - tx;
  double e1x = -tz * qy, e1y = tz * qx - tx * qz, e1z = tx * qy;
  const double inv = 1.0 / sqrt(e1x * e1x + e1y * e1y + e1z * e1z);
  e1x *= inv;
  e1y *= inv;
  e1z *= inv;
  const double e2x = qy * e1z - qz * e1y, e2y = qz * e1x - qx * e1z, e2z = qx * e1y - qy * e1x;
  double a = 0.0, b = 0.0, h = 1.0;
  if (lane < P.n) {
    const int j = P.id;
    const double dx = g.px[j] - qx, dy = g.py[j] - qy, dz = g.pz[j] - qz;
    a = e1x * dx + e1y * dy + e1z * dz;
    b = e2x * dx + e2y * dy + e2z * dz;
    h = -(qx * dx + qy * dy + qz * dz);
  }
  // vertex k: edge k-1 meets edge k
  const int pv = lane == 0 ? P.n - 1 : lane - 1;
  const double pa = __shfl_sync(FULL, a, pv), pb = __shfl_sync(FULL, b, pv), ph = __shfl_sync(FULL, h, pv);
  const double det = pa * b - a * pb;
  const double u = (ph * b - h * pb) / det, v = (pa * h - a * ph) / det;
  const double n1 = sqrt(1.0 + u * u + v * v);
  const int nx = (lane + 1 == P.n) ? 0 : lane + 1;
  const double u2 = __shfl_sync(FULL, u, nx), v2 = __shfl_sync(FULL, v, nx), n2 = __shfl_sync(FULL, n1, nx);
  double E = 0.0;
  if (lane < P.n) E = 2.0 * atan2(u * v2 - u2 * v, 1.0 + n1 + n2 + n1 * n2 + u * u2 + v * v2);
  return warp_sum(E);
}

template <bool F64>
__global__ void __launch_bounds__(VOR_WARPS * 32) voronoi_kernel(Cells g, const float4* __restrict__ lo, float r0,
                                                                 double* __restrict__ out, double* __restrict__ sw,
                                                                 float* __restrict__ swf, DevStatus* st) {
  const float PI_F = 3.14159265f;
  const int lane = threadIdx.x & 31;
  const int s = blockIdx.x * VOR_WARPS + (threadIdx.x >> 5);
  if (s >= g.n) return;
  VorNode q;
  q.s = s;
  {
    const float4 h4 = g.pf[s], l4 = lo[s];
    q.hi = make_float3(h4.x, h4.y, h4.z);
    q.lo = make_float3(l4.x, l4.y, l4.z);
    // tangent frame e1 = t x q / |t x q| (t = z, or x near the poles), e2 = q x e1
    const float tx = fabsf(h4.z) < 0.9f ? 0.f : 1.f, tz = 1.f - tx;
    float e1x = -tz * h4.y, e1y = tz * h4.x - tx * h4.z, e1z = tx * h4.y;
    const float inv = rsqrtf(e1x * e1x + e1y * e1y + e1z * e1z);
    e1x *= inv;
    e1y *= inv;
    e1z *= inv;
    q.e1 = make_float3(e1x, e1y, e1z);
    q.e2 = make_float3(h4.y * e1z - h4.z * e1y, h4.z * e1x - h4.x * e1z, h4.x * e1y - h4.y * e1x);
  }
  VPoly P;
  vor_square(P, tanf(VOR_THETA_MAX));
  float R2 = vor_r2(P);
  int dups = 0;
  bool good = true, closed = false;
  // 1. caps around x_i of angle r0, 2 r0, ...
  float r = r0, rdone = 0.f, hskip = -1.f;
  for (int grow = 0; grow < VOR_GROW_LIMIT; ++grow) {
    const Cap c = make_cap_f(q.hi.x, q.hi.y, q.hi.z, r);
    for_cap_candidates<true>(g, c, [&](bool valid, uint32_t idx) {
      if (good) good = vor_round(g, lo, q, P, R2, valid, idx, dups, grow == 0, hskip);
    });
    rdone = r;
    if (!good) break;
    closed = !__any_sync(FULL, lane < P.n && P.id < 0);
    if (r >= PI_F) break;          // every node seen
    if (closed) {
      const float R2a = vor_settled_r2(r);
      if (r >= 4.f * r0 || !__any_sync(FULL, lane < P.n && P.u * P.u + P.v * P.v > R2a)) break;
    }
    const float cp = 2.f * sinf(0.5f * r);
    hskip = 0.5f * cp * cp * (1.f - 1e-5f);
    r = fminf(2.f * r, PI_F);
  }
  bool ok = false;
  if (good && closed) {
    const float R2a = vor_settled_r2(rdone);
    // 2. the flower caps of the other vertices
    int it = 0;
    while (good) {
      P.fin = P.fin || (lane < P.n && P.u * P.u + P.v * P.v <= R2a);
      const unsigned need = __ballot_sync(FULL, lane < P.n && !P.fin);
      if (need == 0u) break;
      if (++it > VOR_FLOWER_LIMIT) {
        good = false;
        break;
      }
      const int k = __ffs(need) - 1;
      P.tag = (lane == k);
      const float fu = __shfl_sync(FULL, P.u, k), fv = __shfl_sync(FULL, P.v, k);
      // the vertex on the sphere, at angle atan |(u, v)| from x_i
      const float cx = q.hi.x + fu * q.e1.x + fv * q.e2.x;
      const float cy = q.hi.y + fu * q.e1.y + fv * q.e2.y;
      const float cz = q.hi.z + fu * q.e1.z + fv * q.e2.z;
      const float ic = rsqrtf(cx * cx + cy * cy + cz * cz);
      const float rg = atanf(sqrtf(fu * fu + fv * fv)) * 1.0001f + 1e-6f;
      if (!(rg < 1.6f)) {
        good = false;
        break;
      }
      const Cap cf = make_cap_f(cx * ic, cy * ic, cz * ic, rg);
      bool cut_vertex = false;
      for_cap_candidates<true>(
          g, cf,
          [&](bool valid, uint32_t idx) {
            if (good && !cut_vertex) good = vor_flower_round(g, lo, q, P, R2, valid, idx, fu, fv, cut_vertex);
          },
          [&]() { return cut_vertex || !good; });
      // not cut: no node is closer to the vertex than x_i
      P.fin = P.fin || P.tag;
      P.tag = false;
    }
    ok = good;
  }
  double E = 0.0;
  if (ok) {
    if (F64) {
      E = vor_area64(g, s, P);
      ok = isfinite(E);
    } else {
      const int nx = (lane + 1 == P.n) ? 0 : lane + 1;
      const float u2 = __shfl_sync(FULL, P.u, nx), v2 = __shfl_sync(FULL, P.v, nx);
      float e = 0.f;
      if (lane < P.n) {
        const float n1 = sqrtf(1.f + P.u * P.u + P.v * P.v), n2 = sqrtf(1.f + u2 * u2 + v2 * v2);
        e = 2.f * atan2f(P.u * v2 - u2 * P.v, 1.f + n1 + n2 + n1 * n2 + P.u * u2 + P.v * v2);
      }
      E = (double)warp_sum(e);
    }
  }
  dups = warp_sum(dups);
  if (lane == 0) {
    double area = E / (double)(1 + dups);
    if (!ok) {
      area = __longlong_as_double(0x7ff8000000000000ll);
      set_flag(st, ST_VORONOI);
    }
    if (out) out[g.perm[s]] = area;
    if (sw) sw[s] = area;
    if (swf) swf[s] = (float)area;
  }
}

// lo = the FP32 rounding of (node - its FP32 copy)
__global__ void vor_split_kernel(Cells g, float4* __restrict__ lo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  const float4 h = g.pf[i];
  lo[i] = make_float4((float)(g.px[i] - (double)h.x), (float)(g.py[i] - (double)h.y),
                      (float)(g.pz[i] - (double)h.z), 0.f);
}

void run_voronoi(const Cells& g, bool mixed, float4* lo_scratch, double* out, double* sw, float* swf,
                 DevStatus* st, cudaStream_t s, int64_t* launches) {
  if (g.n <= 0) return;
  vor_split_kernel<<<(g.n + 255) / 256, 256, 0, s>>>(g, lo_scratch);
  // the first cap reaches two mean node spacings
  const float r0 = (float)fmin(2.0 * sqrt(4.0 * M_PI / (double)g.n), 3.14159265);
  const int blocks = (g.n + VOR_WARPS - 1) / VOR_WARPS;
  if (mixed)
    voronoi_kernel<false><<<blocks, VOR_WARPS * 32, 0, s>>>(g, lo_scratch, r0, out, sw, swf, st);
  else
    voronoi_kernel<true><<<blocks, VOR_WARPS * 32, 0, s>>>(g, lo_scratch, r0, out, sw, swf, st);
  *launches += 2;
}

}  // namespace hamls
