// k_links.cu — wall links of the finest level's adjacent cells.
//
// Paper (Sec. "Identification of Cells Near the Boundary"): interpolated
// boundary conditions need, for each boundary cell, the distance to the wall
// along the lattice directions (the quadrature abscissae of the velocity set).
// A link of cell x along c_i is the segment x + t c_i h, t in [0, 1]; its
// fraction q is the smallest t at which it meets a face of the cell's
// adjacency list (with d_L >= h_L/2 the segment lies inside the inflated cell
// box, so no other face can be met).  Coplanar segments miss; ties keep the
// smallest face id.
//
// One thread per adjacent cell.  Per face the thread forms the vertex offsets
// from the cell centre as exact double-float pairs, the three edge cross
// products (shared by all directions) and the plane offset num = n.(v0 - x)
// in double-float from the face's double-float normal.  Per direction the
// inside test is the sign of three sums of cross-product components, each
// with a forward error bound; t = num / (h c_i.n) is accurate to a few ulps.
// Undecided signs go to an FP64 evaluation.  Links leave in (cell, direction)
// order through a single-pass ticketed look-back over thread blocks.
#include "internal.cuh"

namespace amr {

namespace {

constexpr int kLThreads = 128;

__constant__ int c_d3q19[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},
                                   {0, 0, 1},  {0, 0, -1},  {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},
                                   {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                   {0, 1, 1},  {0, -1, -1}, {0, 1, -1},  {0, -1, 1}};
__constant__ int c_d2q9[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1}, {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};

// D3Q19 direction i (1..18), component a, as a compile-time constant when i and
// a are: 1..6 = +x,-x,+y,-y,+z,-z; 7..18 = xy, xz, yz plane diagonals, each
// (+,+),(-,-),(+,-),(-,+).
__host__ __device__ constexpr int d3q19_c(int i, int a) {
  return i <= 6 ? (((i - 1) >> 1) == a ? ((i & 1) ? 1 : -1) : 0)
                : ((((i - 7) >> 2) == 0 ? (a == 0 ? 1 : (a == 1 ? 2 : 0))
                                        : (((i - 7) >> 2) == 1 ? (a == 0 ? 1 : (a == 2 ? 2 : 0))
                                                               : (a == 1 ? 1 : (a == 2 ? 2 : 0)))) == 1
                       ? ((((i - 7) & 3) == 0 || ((i - 7) & 3) == 2) ? 1 : -1)
                       : ((((i - 7) >> 2) == 0 ? (a == 0 ? 1 : (a == 1 ? 2 : 0))
                                               : (((i - 7) >> 2) == 1 ? (a == 0 ? 1 : (a == 2 ? 2 : 0))
                                                                      : (a == 1 ? 1 : (a == 2 ? 2 : 0)))) == 2
                              ? ((((i - 7) & 3) == 0 || ((i - 7) & 3) == 3) ? 1 : -1)
                              : 0));
}
static_assert(d3q19_c(1, 0) == 1 && d3q19_c(2, 0) == -1 && d3q19_c(5, 2) == 1 && d3q19_c(6, 2) == -1, "axes");
static_assert(d3q19_c(7, 0) == 1 && d3q19_c(7, 1) == 1 && d3q19_c(8, 0) == -1 && d3q19_c(8, 1) == -1, "xy");
static_assert(d3q19_c(9, 0) == 1 && d3q19_c(9, 1) == -1 && d3q19_c(10, 0) == -1 && d3q19_c(10, 1) == 1, "xy");
static_assert(d3q19_c(13, 0) == 1 && d3q19_c(13, 2) == -1 && d3q19_c(13, 1) == 0, "xz");
static_assert(d3q19_c(18, 1) == -1 && d3q19_c(18, 2) == 1 && d3q19_c(18, 0) == 0, "yz");

__device__ __forceinline__ void d3q19_dir(int i, int& cx, int& cy, int& cz) {
  cx = cy = cz = 0;
  if (i <= 6) {
    const int s = (i & 1) ? 1 : -1;
    const int ax = (i - 1) >> 1;
    if (ax == 0) cx = s;
    else if (ax == 1) cy = s;
    else cz = s;
    return;
  }
  const int p = (i - 7) >> 2, j = (i - 7) & 3;
  const int s1 = (j == 0 || j == 2) ? 1 : -1;
  const int s2 = (j == 0 || j == 3) ? 1 : -1;
  if (p == 0) {
    cx = s1;
    cy = s2;
  } else if (p == 1) {
    cx = s1;
    cz = s2;
  } else {
    cy = s1;
    cz = s2;
  }
}

// Directions whose link segment box [0, c h] can meet the face's box (the hit
// point lies in both): per axis the face must straddle 0 (c_a = 0), reach
// [0, h] (c_a = +1) or [-h, 0] (c_a = -1), with a tolerance for the rounding
// of the local coordinates.  Bit i-1 set = direction i may hit.
__device__ __forceinline__ uint32_t d3q19_candidates(const float (*p)[3], float h) {
  bool z[3], pos[3], neg[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float mn = fminf(fminf(p[0][a], p[1][a]), p[2][a]);
    const float mx = fmaxf(fmaxf(p[0][a], p[1][a]), p[2][a]);
    const float tol = 8.0f * kU32 * (fmaxf(fabsf(mn), fabsf(mx)) + h);
    z[a] = mn <= tol && mx >= -tol;
    pos[a] = mx >= -tol && mn <= h + tol;
    neg[a] = mn <= tol && mx >= -h - tol;
  }
  uint32_t m = 0;
#pragma unroll
  for (int i = 1; i <= 18; ++i) {
    int c[3];
    d3q19_dir(i, c[0], c[1], c[2]);
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) ok = ok && (c[a] == 0 ? z[a] : (c[a] > 0 ? pos[a] : neg[a]));
    m |= ok ? (1u << (i - 1)) : 0u;
  }
  return m;
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf(a, b, -p);
}

struct LinkHit {
  bool hit;
  bool band;
  double t;
};

__device__ __noinline__ LinkHit link_fp64_3(const float* V, const double* xc, const int* ci, double h);

// FP64 evaluation of direction di for the cell (block coordinates blk3, cell bit),
// with the cell centre formed in FP64 (the slow path of undecided signs).
__device__ __noinline__ LinkHit link_fallback_3(const float* V, const int* blk3, uint32_t bit, const double* origin,
                                                double h, int di) {
  int ci[3];
  d3q19_dir(di, ci[0], ci[1], ci[2]);
  double xc[3];
  for (int c = 0; c < 3; ++c) {
    const int gc = 4 * blk3[c] + (int)((bit >> (2 * c)) & 3u);
    xc[c] = __dadd_rn(origin[c], __dmul_rn((double)gc + 0.5, h));
  }
  return link_fp64_3(V, xc, ci, h);
}

// FP64 evaluation of one (link, face) pair, same definition as the FP32 path.
__device__ __noinline__ LinkHit link_fp64_3(const float* V, const double* xc, const int* ci, double h) {
  LinkHit r{false, false, 0.0};
  double p[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) p[k][c] = (double)V[3 * k + c] - xc[c];
  const double d[3] = {ci[0] * h, ci[1] * h, ci[2] * h};
  const double u[3] = {p[1][0] - p[0][0], p[1][1] - p[0][1], p[1][2] - p[0][2]};
  const double w[3] = {p[2][0] - p[0][0], p[2][1] - p[0][1], p[2][2] - p[0][2]};
  const double n[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
  const double ln = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  if (ln == 0.0) return r;
  const double den = d[0] * n[0] + d[1] * n[1] + d[2] * n[2];
  if (den == 0.0) return r;
  const double ld = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  if (fabs(den) <= kBandRel * ld * ln) r.band = true;
  auto vol = [&](const double* a, const double* b) {
    const double c0 = a[1] * b[2] - a[2] * b[1], c1 = a[2] * b[0] - a[0] * b[2], c2 = a[0] * b[1] - a[1] * b[0];
    return d[0] * c0 + d[1] * c1 + d[2] * c2;
  };
  const double l0 = vol(p[1], p[2]) / den, l1 = vol(p[2], p[0]) / den, l2 = vol(p[0], p[1]) / den;
  const double t = (p[0][0] * n[0] + p[0][1] * n[1] + p[0][2] * n[2]) / den;
  const double mu = fmin(fmin(fmin(l0, l1), l2), fmin(t, 1.0 - t));
  if (fabs(mu) <= kBandRel) r.band = true;
  r.hit = mu >= 0.0;
  r.t = t;
  return r;
}

__device__ __noinline__ LinkHit link_fp64_2(const float* V, const double* xc, const int* ci, double h) {
  LinkHit r{false, false, 0.0};
  const double p0[2] = {(double)V[0] - xc[0], (double)V[1] - xc[1]};
  const double p1[2] = {(double)V[2] - xc[0], (double)V[3] - xc[1]};
  const double e[2] = {p1[0] - p0[0], p1[1] - p0[1]};
  const double le = sqrt(e[0] * e[0] + e[1] * e[1]);
  if (le == 0.0) return r;
  const double d[2] = {ci[0] * h, ci[1] * h};
  const double den = d[0] * e[1] - d[1] * e[0];
  if (den == 0.0) return r;
  const double ld = sqrt(d[0] * d[0] + d[1] * d[1]);
  if (fabs(den) <= kBandRel * ld * le) r.band = true;
  const double t = (p0[0] * e[1] - p0[1] * e[0]) / den;
  const double s = (p0[0] * d[1] - p0[1] * d[0]) / den;
  const double mu = fmin(fmin(t, 1.0 - t), fmin(s, 1.0 - s));
  if (fabs(mu) <= kBandRel) r.band = true;
  r.hit = mu >= 0.0;
  r.t = t;
  return r;
}

template <int D>
__global__ void __launch_bounds__(kLThreads) k_links(LinkArgs a, uint64_t* state, unsigned* ticket) {
  constexpr int Q1 = D == 3 ? 18 : 8;
  constexpr int NC = D == 3 ? 64 : 16;
  __shared__ unsigned s_tile;
  __shared__ float s_q[Q1][kLThreads];
  __shared__ uint32_t s_f[Q1][kLThreads];
  __shared__ uint32_t s_warp[kLThreads / 32];
  __shared__ uint64_t s_prefix;
  const int tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  const uint64_t row0 = a.run ? a.run[0] : 0ull;
  const uint64_t link0 = a.run ? a.run[2] : 0ull;
  int64_t nrows = a.level_tot ? (int64_t)(*a.level_tot >> 32) : a.cap_rows;
  if ((int64_t)row0 + nrows > a.cap_rows) {
    if (blockIdx.x == 0 && tid == 0) atomicOr(a.err, ERR_OVERFLOW);
    nrows = a.cap_rows - (int64_t)row0 > 0 ? a.cap_rows - (int64_t)row0 : 0;
  }
  const int64_t ntiles = (nrows + kLThreads - 1) / kLThreads;
  if (ntiles == 0) {
    if (blockIdx.x == 0 && tid == 0) *a.n_links = 0;
    return;
  }
  unsigned long long n_fb = 0, n_band = 0;
  for (;;) {
  if (tid == 0) s_tile = atomicAdd(ticket, 1u);
  __syncthreads();
  const long long tile = s_tile;
  if (tile >= ntiles) break;
  const int64_t local = tile * (int64_t)kLThreads + tid;
  const int64_t row = (int64_t)row0 + local;
#pragma unroll
  for (int i = 0; i < Q1; ++i) {
    s_q[i][tid] = INFINITY;
    s_f[i][tid] = 0xffffffffu;
  }
  if (local < nrows) {
    const uint32_t id = a.adj_cell[row];
    const uint32_t blk = id / NC, bit = id % NC;
    const GeomParams& P = a.table ? a.table[a.gid ? a.gid[blk] : 0u] : a.g0;
    const FastGeom g = fast_geom(P, a.level);
    // cell centre origin + (2 c + 1) (h/2) as hi + lo; the FP64 centre only for fallbacks
    double xc[3] = {0, 0, 0};
    float ohi[3] = {0, 0, 0}, olo[3] = {0, 0, 0};
    const double hL = scalbn(P.h0, -a.level);
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const int gc = 4 * a.blocks[(int64_t)blk * D + c] + (int)((bit >> (2 * c)) & 3u);
      df_position(P.org_hi[c], P.org_lo[c], (float)(2 * gc + 1), 0.5f * g.h_hi, 0.5f * g.h_lo, ohi[c], olo[c]);
      xc[c] = D == 3 ? 0.0 : __dadd_rn(P.origin[c], __dmul_rn((double)gc + 0.5, hL));
    }
    const float h32 = g.h_hi;
    struct GeomView {
      double h;
    } G{hL};
    const uint32_t e0 = a.adj_off[row], e1 = a.adj_off[row + 1];
    for (uint32_t e = e0; e < e1; ++e) {
      const uint32_t f = a.adj_ids[e];
      float V[D * D];
#pragma unroll
      for (int j = 0; j < D * D; ++j) V[j] = a.X[(int64_t)j * a.nf + f];
      if constexpr (D == 2) {
        // 2D workloads are small: evaluate every link in FP64
#pragma unroll
        for (int di = 1; di <= Q1; ++di) {
          const int ci[2] = {c_d2q9[di][0], c_d2q9[di][1]};
          const LinkHit r = link_fp64_2(V, xc, ci, G.h);
          if (r.band) ++n_band;
          if (r.hit) {
            const float t = (float)r.t;
            if (t < s_q[di - 1][tid]) {
              s_q[di - 1][tid] = t;
              s_f[di - 1][tid] = f;
            }
          }
        }
      } else {
        // vertex offsets from the cell centre: p = (V - ohi) - olo as hi + lo
        float ph[3][3], pl[3][3], p[3][3];
        float pmax = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            float s, err;
            two_sum(V[3 * k + c], -ohi[c], s, err);
            ph[k][c] = s;
            pl[k][c] = err - olo[c];
            p[k][c] = s + pl[k][c];
            pmax = fmaxf(pmax, fabsf(p[k][c]));
          }
        uint32_t cand = d3q19_candidates(p, h32);
        if (!cand) continue;
        const float nh[3] = {a.nrm[f], a.nrm[a.nf + f], a.nrm[2 * a.nf + f]};
        const float nl[3] = {a.nrm[3 * a.nf + f], a.nrm[4 * a.nf + f], a.nrm[5 * a.nf + f]};
        // num = n . (v0 - x) in double-float
        float ns, ne;
        two_prod(nh[0], ph[0][0], ns, ne);
#pragma unroll
        for (int c = 1; c < 3; ++c) {
          float pp, pe, s, t;
          two_prod(nh[c], ph[0][c], pp, pe);
          two_sum(ns, pp, s, t);
          ns = s;
          ne += t + pe;
        }
        float n1 = fabsf(nh[0]) + fabsf(nh[1]) + fabsf(nh[2]);
#pragma unroll
        for (int c = 0; c < 3; ++c) ne = fmaf(nh[c], pl[0][c], fmaf(nl[c], ph[0][c], ne));
        const float num = ns + ne;
        const float xmax = fmaxf(fmaxf(fabsf(ohi[0]), fabsf(ohi[1])), fabsf(ohi[2]));
        const float eps_num = 16.0f * kU32 * kU32 * n1 * (xmax + pmax) + 4.0f * kU32 * fabsf(ne);
        // edge cross products C_k = p_a x p_b, (a,b) = (1,2),(2,0),(0,1), and their magnitudes
        // and the largest component magnitude bound Mk = max_c (|A_a B_b| + |A_b B_a|)
        float C[3][3], M[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float* A = p[(k + 1) % 3];
          const float* B = p[(k + 2) % 3];
          C[k][0] = fmaf(A[1], B[2], -A[2] * B[1]);
          C[k][1] = fmaf(A[2], B[0], -A[0] * B[2]);
          C[k][2] = fmaf(A[0], B[1], -A[1] * B[0]);
          M[k] = fmaxf(fmaxf(fabsf(A[1] * B[2]) + fabsf(A[2] * B[1]), fabsf(A[2] * B[0]) + fabsf(A[0] * B[2])),
                       fabsf(A[0] * B[1]) + fabsf(A[1] * B[0]));
        }
        const float nn2 = sqrtf(nh[0] * nh[0] + nh[1] * nh[1] + nh[2] * nh[2]);
#pragma unroll
        for (int di = 1; di <= 18; ++di) {
          const int cx = d3q19_c(di, 0), cy = d3q19_c(di, 1), cz = d3q19_c(di, 2);
          if (!((cand >> (di - 1)) & 1u)) continue;
          // den_n = c . n in double-float: exact for an axis direction, one TwoSum for a diagonal
          const float t0 = cx * nh[0], t1 = cy * nh[1], t2 = cz * nh[2];
          const int cl_i = (cx != 0) + (cy != 0) + (cz != 0);
          float dh, dl;
          if (cl_i == 1) {
            dh = t0 + t1 + t2;
            dl = cx * nl[0] + cy * nl[1] + cz * nl[2];
          } else {
            float e2;
            two_sum(cx != 0 ? t0 : t1, cz != 0 ? t2 : t1, dh, e2);
            dl = e2 + (cx * nl[0] + cy * nl[1] + cz * nl[2]);
          }
          const float den = dh + dl;
          if (den == 0.0f && dh == 0.0f) continue;  // c_i parallel to the face plane: no hit
          const float sg = den > 0.f ? 1.f : -1.f;
          // inside test: sg * (c . C_k) >= 0 for k = 0..2
          bool out = false, unc = fabsf(den) <= (cl_i == 1 ? 1e-5f : 1.41421356e-5f) * nn2;
          bool all_in = true;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const float u = sg * (cx * C[k][0] + cy * C[k][1] + cz * C[k][2]);
            const float eu = 8.0f * kU32 * (float)cl_i * M[k];
            if (u < -eu) out = true;
            if (!(u > eu)) all_in = false;
          }
          if (out && !unc) continue;
          float t = 0.f;
          bool hit = false;
          if (!unc && all_in) {
            // t = num / (h den): range [0,1] with certified ends
            const float sn = sg * num;
            t = num / (h32 * den);
            if (sn < -eps_num || t > 1.0f + 8.0f * kU32) continue;
            if (sn > eps_num && t < 1.0f - 8.0f * kU32) {
              hit = true;
            } else {
              unc = true;
            }
          } else {
            unc = true;
          }
          if (unc) {
            const LinkHit r = link_fallback_3(V, a.blocks + (int64_t)blk * 3, bit, P.origin, G.h, di);
            ++n_fb;
            if (r.band) ++n_band;
            if (!r.hit) continue;
            hit = true;
            t = (float)r.t;
          }
          if (hit && t < s_q[di - 1][tid]) {
            s_q[di - 1][tid] = t;
            s_f[di - 1][tid] = f;
          }
        }
      }
    }
  }
  uint32_t hits = 0;
#pragma unroll
  for (int i = 0; i < Q1; ++i) hits += s_f[i][tid] != 0xffffffffu ? 1u : 0u;
  // block scan of per-cell link counts, then look-back for the global offset
  const uint32_t incl = warp_inclusive_scan<uint32_t>(hits);
  if (lane == 31) s_warp[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    uint32_t w = lane < kLThreads / 32 ? s_warp[lane] : 0u;
    w = warp_inclusive_scan<uint32_t>(w);
    if (lane < kLThreads / 32) s_warp[lane] = w;
  }
  __syncthreads();
  const uint32_t wex = wid > 0 ? s_warp[wid - 1] : 0u;
  if (tid == 0) {
    const uint64_t agg = s_warp[kLThreads / 32 - 1];
    const uint64_t pre = lookback_exclusive(state, tile, agg, a.err);
    s_prefix = pre;
    if (tile == ntiles - 1) {
      *a.n_links = pre + agg;
      if ((int64_t)(link0 + pre + agg) > a.link_cap) atomicOr(a.err, ERR_OVERFLOW);
    }
  }
  __syncthreads();
  uint64_t pos = link0 + s_prefix + wex + incl - hits;
#pragma unroll
  for (int i = 0; i < Q1; ++i) {
    const uint32_t f = s_f[i][tid];
    if (f != 0xffffffffu) {
      if ((int64_t)pos < a.link_cap) {
        a.link_cell[pos] = (uint32_t)row;
        a.link_dir[pos] = (uint8_t)(i + 1);
        a.link_q[pos] = s_q[i][tid];
        a.link_face[pos] = f;
      }
      ++pos;
    }
  }
  __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n_fb += __shfl_xor_sync(0xffffffffu, n_fb, o);
    n_band += __shfl_xor_sync(0xffffffffu, n_band, o);
  }
  if (lane == 0) {
    if (n_fb) atomicAdd(&a.counters[CNT_LINK_FALLBACK], n_fb);
    if (n_band) atomicAdd(&a.counters[CNT_LINK_BAND], n_band);
  }
}

// close = true: write the CSR end marker of this level's adjacency rows,
// adj_off[run[0] + cells] = run[1] + pairs (needed by the link kernel);
// close = false: advance the running totals past this level.
__global__ void k_advance(const uint64_t* level_tot, const uint64_t* n_links, uint64_t* run, uint32_t* adj_off,
                          int64_t cap_cells, unsigned* err, bool close) {
  const uint64_t t = *level_tot;
  if (close) {
    const uint64_t end = run[0] + (t >> 32);
    if ((int64_t)end <= cap_cells)
      adj_off[end] = (uint32_t)(run[1] + (t & 0xffffffffull));
    else
      atomicOr(err, ERR_OVERFLOW);
    return;
  }
  run[0] += t >> 32;
  run[1] += t & 0xffffffffull;
  run[2] += n_links ? *n_links : 0ull;
}

}  // namespace

size_t links_scratch_bytes(int64_t n_adj) {
  const int64_t tiles = (n_adj + kLThreads - 1) / kLThreads;
  return 16 + (size_t)(tiles > 0 ? tiles : 1) * 8;
}

int launch_links(const LinkArgs& a, void* scratch, int num_sms, cudaStream_t st) {
  cudaMemsetAsync(scratch, 0, links_scratch_bytes(a.cap_rows), st);
  int64_t tiles = (a.cap_rows + kLThreads - 1) / kLThreads;
  if (tiles < 1) tiles = 1;
  if (tiles > (int64_t)num_sms * 12) tiles = (int64_t)num_sms * 12;
  unsigned* ticket = reinterpret_cast<unsigned*>(scratch);
  uint64_t* state = reinterpret_cast<uint64_t*>(static_cast<char*>(scratch) + 16);
  if (a.dim == 3)
    k_links<3><<<(unsigned)tiles, kLThreads, 0, st>>>(a, state, ticket);
  else
    k_links<2><<<(unsigned)tiles, kLThreads, 0, st>>>(a, state, ticket);
  return 1;
}

int launch_advance(const uint64_t* level_tot, const uint64_t* n_links, uint64_t* run, uint32_t* adj_off,
                   int64_t cap_cells, unsigned* err, bool close, cudaStream_t st) {
  k_advance<<<1, 1, 0, st>>>(level_tot, n_links, run, adj_off, cap_cells, err, close);
  return 1;
}

}  // namespace amr
