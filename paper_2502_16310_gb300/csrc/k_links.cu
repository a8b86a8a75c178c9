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
// Blocks take tiles of adjacent cells, and a lane one (cell, face) pair of a
// tile at a time.  Per pair the lane forms the vertex offsets from the cell
// centre as exact double-float pairs, the three edge cross products (shared by
// all directions) and the plane offset num = n.(v0 - x) in double-float from
// the face's double-float normal.  Per direction the inside test is the sign
// of three sums of cross-product components, each with a forward error bound;
// t = num / (h c_i.n) is accurate to a few ulps.  Undecided signs go to an
// FP64 evaluation.  Each tile of cells appends its
// links, in (cell, direction) order, to a staging area at a position taken
// from one counter; a scan of the per-tile counts in tile order then gives
// every tile its place in the output, and a second kernel moves the links
// there.  No tile waits for the tiles before it.
#include <atomic>

#include "internal.cuh"

namespace amr {

namespace {

#ifndef AMR_LINK_TILE
#define AMR_LINK_TILE 128
#endif
constexpr int kLThreads = AMR_LINK_TILE;  // threads per block
constexpr int kLRows = AMR_LINK_TILE;     // adjacent cells per tile (one per thread in phases 0 and 2)
static_assert(kLThreads == kLRows, "phase 0 and 2 map thread i to row i");

__constant__ int c_d2q9[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1}, {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};

// D3Q19 direction i (1..18), component a: 1..6 = +x,-x,+y,-y,+z,-z; 7..18 =
// the xy, xz and yz plane diagonals, each as (+,+), (-,-), (+,-), (-,+).
__host__ __device__ constexpr int d3q19_c(int i, int a) {
  if (i <= 6) return ((i - 1) >> 1) == a ? ((i & 1) ? 1 : -1) : 0;
  const int p = (i - 7) >> 2, j = (i - 7) & 3;
  const int a1 = p == 2 ? 1 : 0;  // first axis of the plane
  const int a2 = p == 0 ? 1 : 2;  // second axis
  if (a == a1) return (j == 0 || j == 2) ? 1 : -1;
  if (a == a2) return (j == 0 || j == 3) ? 1 : -1;
  return 0;
}
static_assert(d3q19_c(1, 0) == 1 && d3q19_c(2, 0) == -1 && d3q19_c(5, 2) == 1 && d3q19_c(6, 2) == -1, "axes");
static_assert(d3q19_c(7, 0) == 1 && d3q19_c(7, 1) == 1 && d3q19_c(8, 0) == -1 && d3q19_c(8, 1) == -1, "xy");
static_assert(d3q19_c(9, 0) == 1 && d3q19_c(9, 1) == -1 && d3q19_c(10, 0) == -1 && d3q19_c(10, 1) == 1, "xy");
static_assert(d3q19_c(13, 0) == 1 && d3q19_c(13, 2) == -1 && d3q19_c(13, 1) == 0, "xz");
static_assert(d3q19_c(18, 1) == -1 && d3q19_c(18, 2) == 1 && d3q19_c(18, 0) == 0, "yz");

__device__ __forceinline__ void d3q19_dir(int i, int& cx, int& cy, int& cz) {
  cx = d3q19_c(i, 0);
  cy = d3q19_c(i, 1);
  cz = d3q19_c(i, 2);
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

// Sort key of a hit: the FP32 bits of t >= 0 order like t, the face id breaks ties.
__device__ __forceinline__ unsigned long long hit_key(float t, uint32_t f) {
  if (!(t > 0.0f)) t = 0.0f;  // also maps -0 to +0
  return ((unsigned long long)__float_as_uint(t) << 32) | f;
}

// A staged link in 64 bits: the FP32 bits of q (q <= 1, so below 2^30), the
// direction (5 bits) and the face id (29 bits; face counts stay below 2^29).
constexpr uint32_t kOneBits = 0x3f800000u;
static_assert(kOneBits < (1u << 30), "q in [0, 1] fits 30 bits");
static_assert(kMaxFaces <= (1 << 29), "face ids fit 29 bits");
__device__ __forceinline__ unsigned long long stage_key(unsigned long long k, int dir) {
  const uint32_t tb = (uint32_t)(k >> 32);
  return ((unsigned long long)(tb < kOneBits ? tb : kOneBits) << 34) | ((unsigned long long)dir << 29) |
         (k & ((1ull << 29) - 1));
}

// Per-launch bookkeeping of the tiles (all in the scratch buffer but the staging area).
struct LinkTiles {
  unsigned* ticket;              // next tile to take
  unsigned long long* bump;      // staging entries claimed so far
  uint64_t* n_tiles;             // tiles of this launch (written by block 0)
  uint64_t* count;               // per tile: its links
  uint64_t* start;               // per tile: its first staging entry
  uint64_t* place;               // per tile: its first output entry past the level's start (scan of count)
  unsigned long long* stage_key; // staged links (stage_key)
  uint8_t* stage_row;            // their row within the tile
  int64_t stage_cap;
};

// D3Q19 components packed two bits per direction (value + 1), for lanes that
// each hold a different direction.
__host__ __device__ constexpr uint64_t pack_dir_axis(int a) {
  uint64_t k = 0;
  for (int i = 1; i <= 18; ++i) k |= (uint64_t)(d3q19_c(i, a) + 1) << (2 * i);
  return k;
}
constexpr uint64_t kDirX = pack_dir_axis(0), kDirY = pack_dir_axis(1), kDirZ = pack_dir_axis(2);
__device__ __forceinline__ float dir_comp(uint64_t k, int i) { return (float)((int)((k >> (2 * i)) & 3ull) - 1); }

// Per-pair quantities the direction tests share (one record per lane, 7 x 16 B
// so that lanes reading different records hit different banks).
struct PairRec {
  float4 q[7];
};

// The lattice splits into 9 lines (an axis or a plane diagonal, both senses):
// direction 2l+1 = +d_l and 2l+2 = -d_l, with d_l = x, y, z, x+y, x-y, x+z,
// x-z, y+z, y-z.  A direction can hit the face plane within the link only if
// t = num / (h c.n) lies in [0, 1]: this keeps every direction for which that
// is possible under the error bounds of num (eps_num) and of D = d_l.n in FP32
// (eD), a superset of the hits that the exact per-direction test then decides.
__device__ __forceinline__ uint32_t line_candidates(const float (&nh)[3], float num, float eps_num, float h32) {
  const float lim = fabsf(num) - eps_num;  // lower bound of |num|
  const bool pos = num >= -eps_num, neg = num <= eps_num;
  const float a0 = fabsf(nh[0]), a1 = fabsf(nh[1]), a2 = fabsf(nh[2]);
  const float Dl[9] = {nh[0], nh[1], nh[2], nh[0] + nh[1], nh[0] - nh[1], nh[0] + nh[2], nh[0] - nh[2],
                       nh[1] + nh[2], nh[1] - nh[2]};
  const float El[9] = {a0, a1, a2, a0 + a1, a0 + a1, a0 + a2, a0 + a2, a1 + a2, a1 + a2};
  uint32_t cand = 0;
#pragma unroll
  for (int l = 0; l < 9; ++l) {
    const float eD = 4.0f * kU32 * El[l];
    const float reach = h32 * (fabsf(Dl[l]) + eD) * (1.0f + 16.0f * kU32);
    if (lim > reach) continue;
    const bool dp = Dl[l] >= -eD, dn = Dl[l] <= eD;
    if ((pos && dp) || (neg && dn)) cand |= 1u << (2 * l);
    if ((pos && dn) || (neg && dp)) cand |= 2u << (2 * l);
  }
  return cand;
}

// Links of one tile of kLRows adjacent cells.  Phase 0: per row, the cell
// centre (double-float) and the row's slice of the pair list.  Phase 1: warps
// take chunks of 32 (cell, face) pairs.  Stage 1 (lane = pair): vertex offsets,
// plane offset num, edge cross products and the candidate directions of the
// 9 lattice lines.  Stage 2 (lane = candidate): the candidates of the chunk,
// queued in shared memory, are tested densely, each by the certified
// per-direction test (FP64 when a sign is not certified); hits keep the
// per-(cell, direction) minimum of (t, face) in shared memory.  Phase 2: one
// thread per row counts its links; a block scan gives each row its place in
// the tile's run of the staging area, claimed with one atomic per tile.
template <int D>
__global__ void __launch_bounds__(kLThreads) k_links(LinkArgs a, LinkTiles lt) {
  constexpr int Q1 = D == 3 ? 18 : 8;
  constexpr int NC = D == 3 ? 64 : 16;
  constexpr int NW = kLThreads / 32;
  constexpr int NPR = D == 3 ? 32 : 1;
  // per (direction, row) the least hit key, and per row the directions hit; both are back to
  // empty (~0, 0) at the end of every tile, since phase 2 resets what it reads
  __shared__ unsigned long long s_key[Q1][kLRows];
  __shared__ uint32_t s_mask[kLRows];
  __shared__ uint32_t s_off[kLRows + 1];
  constexpr uint32_t kRowCap = 1024;    // pairs of a tile whose row is tabulated (more: binary search)
  __shared__ uint8_t s_row[kRowCap];    // row of the tile's pair p0 + k
  __shared__ float s_o[2 * D][kLRows];
  __shared__ float s_h[kLRows];
  __shared__ PairRec s_pr[NW][NPR];
  __shared__ uint16_t s_q[NW][D == 3 ? 32 * 18 : 1];
  __shared__ uint32_t s_warp[NW];
  __shared__ uint64_t s_prefix;
  // a tile's links gathered for the store: keys in the pair records, rows in the queue
  constexpr uint32_t kCompact = D == 3 ? (uint32_t)(sizeof(s_pr) / 8) : 0u;
  static_assert(D == 2 || sizeof(s_q) >= sizeof(s_pr) / 8, "a row byte per gathered key");
  __shared__ unsigned s_tile, s_chunk;
  const int tid = threadIdx.x;
  const int lane = tid & 31, wid = tid >> 5;
  const uint64_t row0 = a.run ? a.run[0] : 0ull;
  int64_t nrows = a.level_tot ? (int64_t)(*a.level_tot >> 32) : a.cap_rows;
  if ((int64_t)row0 + nrows > a.cap_rows) {
    if (blockIdx.x == 0 && tid == 0) atomicOr(a.err, ERR_OVERFLOW);
    nrows = a.cap_rows - (int64_t)row0 > 0 ? a.cap_rows - (int64_t)row0 : 0;
  }
  const int64_t ntiles = (nrows + kLRows - 1) / kLRows;
  if (blockIdx.x == 0 && tid == 0) *lt.n_tiles = (uint64_t)ntiles;  // for the scan of the tile counts
  if (ntiles == 0) return;
  unsigned long long n_fb = 0, n_band = 0, n_cand = 0;  // n_cand: warp-uniform
#pragma unroll
  for (int q = 0; q < Q1; ++q) s_key[q][tid] = ~0ull;
  s_mask[tid] = 0u;
  // tiles by ticket; phase 2 of each tile takes the next ticket, so its latency is hidden
  if (tid == 0) s_tile = atomicAdd(lt.ticket, 1u);
  __syncthreads();
  for (;;) {
    const long long tile = s_tile;
    if (tile >= ntiles) break;
    if (tid == 0) s_chunk = 0u;
    const int64_t first = (int64_t)row0 + tile * (int64_t)kLRows;
    const int nr = (int)(nrows - tile * (int64_t)kLRows < kLRows ? nrows - tile * (int64_t)kLRows : kLRows);
    // phase 0 (kLThreads == kLRows: thread i owns row i)
    {
      const int i = tid;
      s_off[i] = a.adj_off[first + (i < nr ? i : nr)];
      if (i == 0) s_off[kLRows] = a.adj_off[first + nr];
      if (i < nr) {
        // the row of each of this row's pairs (the first kRowCap pairs of the tile)
        const uint32_t t0 = a.adj_off[first], e0 = a.adj_off[first + i], e1 = a.adj_off[first + i + 1];
        for (uint32_t e = e0; e < e1 && e - t0 < kRowCap; ++e) s_row[e - t0] = (uint8_t)i;
      }
      if (i < nr) {
        const uint32_t id = a.adj_cell[first + i];
        const uint32_t blk = id / NC, bit = id % NC;
        const GeomParams& P = a.table ? a.table[a.gid ? a.gid[blk] : 0u] : a.g0;
        const FastGeom g = fast_geom(P, a.level);
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const int gc = 4 * a.blocks[(int64_t)blk * D + c] + (int)((bit >> (2 * c)) & 3u);
          df_position(P.org_hi[c], P.org_lo[c], (float)(2 * gc + 1), 0.5f * g.h_hi, 0.5f * g.h_lo, s_o[c][i],
                      s_o[D + c][i]);
        }
        s_h[i] = g.h_hi;
      }
    }
    __syncthreads();
    // phase 1 (the clamp only matters after an overflow, which the host reports)
    const uint32_t p0 = s_off[0];
    const uint32_t p1 = (int64_t)s_off[nr] <= a.cap_pairs ? s_off[nr] : (uint32_t)a.cap_pairs;
    const uint32_t nchunks = p1 > p0 ? (p1 - p0 + 31u) / 32u : 0u;
    for (;;) {
      uint32_t ch = 0;
      if (lane == 0) ch = atomicAdd(&s_chunk, 1u);
      ch = __shfl_sync(0xffffffffu, ch, 0);
      if (ch >= nchunks) break;
      const uint32_t e = p0 + ch * 32u + (uint32_t)lane;
      uint32_t cand = 0;
      int r = 0;
      uint32_t f = 0xffffffffu;
      if (e < p1) {
        if (e - p0 < kRowCap) {
          r = s_row[e - p0];
        } else {
          int lo = 0, hi = nr;  // s_off[lo] <= e < s_off[hi]
          while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s_off[mid] <= e)
              lo = mid;
            else
              hi = mid;
          }
          r = lo;
        }
        f = a.adj_ids[e];
        if ((int64_t)f >= a.nf) f = 0xffffffffu;
      }
      if (f != 0xffffffffu) {
        if constexpr (D == 2) {
          // 2D workloads are small: every link in FP64
          const uint32_t id = a.adj_cell[first + r];
          const uint32_t blk = id / NC, bit = id % NC;
          const GeomParams& P = a.table ? a.table[a.gid ? a.gid[blk] : 0u] : a.g0;
          const double hL = scalbn(P.h0, -a.level);
          double xc[2];
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const int gc = 4 * a.blocks[(int64_t)blk * 2 + c] + (int)((bit >> (2 * c)) & 3u);
            xc[c] = __dadd_rn(P.origin[c], __dmul_rn((double)gc + 0.5, hL));
          }
          float V[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) V[j] = a.X[(int64_t)j * a.nf + f];
#pragma unroll
          for (int di = 1; di <= Q1; ++di) {
            const int ci[2] = {c_d2q9[di][0], c_d2q9[di][1]};
            const LinkHit h = link_fp64_2(V, xc, ci, hL);
            if (h.band) ++n_band;
            if (h.hit) {
              atomicMin(&s_key[di - 1][r], hit_key((float)h.t, f));
              atomicOr(&s_mask[r], 1u << (di - 1));
            }
          }
        } else {
          // stage 1
          const float4* R = reinterpret_cast<const float4*>(a.rec + f);
          const float4 r0 = __ldg(R), r1 = __ldg(R + 1), r2 = __ldg(R + 2), r3 = __ldg(R + 3);
          const float V[9] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z, r1.w, r2.x};
          const float nh[3] = {r2.y, r2.z, r2.w};
          const float nl[3] = {r3.x, r3.y, r3.z};
          const float ohi[3] = {s_o[0][r], s_o[1][r], s_o[2][r]};
          const float olo[3] = {s_o[3][r], s_o[4][r], s_o[5][r]};
          const float h32 = s_h[r];
          // vertex offsets from the cell centre: p = (V - ohi) - olo as hi + lo
          float ph0[3], pl0[3], p[3][3];
          float pmax = 0.f;
#pragma unroll
          for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              float sm, err;
              two_sum(V[3 * k + c], -ohi[c], sm, err);
              const float l = err - olo[c];
              if (k == 0) {
                ph0[c] = sm;
                pl0[c] = l;
              }
              p[k][c] = sm + l;
              pmax = fmaxf(pmax, fabsf(p[k][c]));
            }
          // num = n . (v0 - x) in double-float
          float ns, ne;
          two_prod(nh[0], ph0[0], ns, ne);
#pragma unroll
          for (int c = 1; c < 3; ++c) {
            float pp, pe, sm, t;
            two_prod(nh[c], ph0[c], pp, pe);
            two_sum(ns, pp, sm, t);
            ns = sm;
            ne += t + pe;
          }
          const float n1 = fabsf(nh[0]) + fabsf(nh[1]) + fabsf(nh[2]);
#pragma unroll
          for (int c = 0; c < 3; ++c) ne = fmaf(nh[c], pl0[c], fmaf(nl[c], ph0[c], ne));
          const float num = ns + ne;
          const float xmax = fmaxf(fmaxf(fabsf(ohi[0]), fabsf(ohi[1])), fabsf(ohi[2]));
          const float eps_num = 16.0f * kU32 * kU32 * n1 * (xmax + pmax) + 4.0f * kU32 * fabsf(ne);
          cand = line_candidates(nh, num, eps_num, h32);
          if (cand) {
            // edge cross products C_k = p_a x p_b, (a,b) = (1,2),(2,0),(0,1), and the
            // largest component magnitude bound M_k = max_c (|A_a B_b| + |A_b B_a|)
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
            // The two senses of a lattice line cross the face plane at one point, and the
            // stage-2 edge functions of either sense are the same numbers (c enters with its
            // sign twice).  Where they certify that point outside the face and the plane side
            // is far from stage 2's uncertain band, stage 2 rejects both senses: drop the line.
            // Line l's edge function k is c_l . C_k, a sum of at most two components of C_k,
            // equal (up to the sign of a zero) to stage 2's value; all 9 lines at once.
            {
              const float Dl[9] = {nh[0], nh[1], nh[2], nh[0] + nh[1], nh[0] - nh[1], nh[0] + nh[2], nh[0] - nh[2],
                                   nh[1] + nh[2], nh[1] - nh[2]};
              // s U < -e  <=>  fma(U, s, e) < 0 exactly (s = +-1, one rounding keeps the sign),
              // so the least of the three edges' values decides the line
              float lo[9];
#pragma unroll
              for (int k = 0; k < 3; ++k) {
                const float e1 = 8.0f * kU32 * 1.0f * M[k], e2 = 8.0f * kU32 * 2.0f * M[k];
                const float U[9] = {C[k][0], C[k][1], C[k][2], C[k][0] + C[k][1], C[k][0] - C[k][1],
                                    C[k][0] + C[k][2], C[k][0] - C[k][2], C[k][1] + C[k][2], C[k][1] - C[k][2]};
#pragma unroll
                for (int l = 0; l < 9; ++l) {
                  const float v = fmaf(U[l], Dl[l] > 0.f ? 1.0f : -1.0f, l < 3 ? e1 : e2);
                  lo[l] = k == 0 ? v : fminf(lo[l], v);
                }
              }
#pragma unroll
              for (int l = 0; l < 9; ++l)
                if (lo[l] < 0.0f && fabsf(Dl[l]) > 4.0e-5f * nn2) cand &= ~(3u << (2 * l));
            }
            if (cand) {
              float4* W = s_pr[wid][lane].q;
              W[0] = make_float4(C[0][0], C[0][1], C[0][2], C[1][0]);
              W[1] = make_float4(C[1][1], C[1][2], C[2][0], C[2][1]);
              W[2] = make_float4(C[2][2], M[0], M[1], M[2]);
              W[3] = make_float4(num, eps_num, h32, nn2);
              W[4] = make_float4(nh[0], nh[1], nh[2], __uint_as_float(f));
              W[5] = make_float4(nl[0], nl[1], nl[2], __int_as_float(r));
            }
          }
        }
      }
      if constexpr (D == 3) {
        // queue the chunk's candidates (lane-major), then test them 32 at a time
        const uint32_t nc = __popc(cand);
        const uint32_t incl = warp_inclusive_scan<uint32_t>(nc);
        const uint32_t T = __shfl_sync(0xffffffffu, incl, 31);
        n_cand += T;
        uint32_t pos = incl - nc;
        for (uint32_t m = cand; m; m &= m - 1) s_q[wid][pos++] = (uint16_t)(lane | (__ffs(m) << 5));
        __syncwarp();
        for (uint32_t base = 0; base < T; base += 32) {
          const uint32_t q = base + (uint32_t)lane;
          if (q < T) {
            const uint32_t qe = s_q[wid][q];
            const int src = (int)(qe & 31u), di = (int)(qe >> 5);
            const float4* Q = s_pr[wid][src].q;
            const float4 w0 = Q[0], w1 = Q[1], w2 = Q[2], w3 = Q[3], w4 = Q[4], w5 = Q[5];
            const float Cx[3][3] = {{w0.x, w0.y, w0.z}, {w0.w, w1.x, w1.y}, {w1.z, w1.w, w2.x}};
            const float Mk[3] = {w2.y, w2.z, w2.w};
            const float num = w3.x, eps_num = w3.y, h32 = w3.z, nn2 = w3.w;
            const float nh[3] = {w4.x, w4.y, w4.z};
            const float nl[3] = {w5.x, w5.y, w5.z};
            const uint32_t fq = __float_as_uint(w4.w);
            const int rq = __float_as_int(w5.w);
            const float cx = dir_comp(kDirX, di), cy = dir_comp(kDirY, di), cz = dir_comp(kDirZ, di);
            const float cl = fabsf(cx) + fabsf(cy) + fabsf(cz);
            // den = c . n in double-float (c has at most two non-zero unit entries)
            float s1, e1, dh, e2;
            two_sum(cx * nh[0], cy * nh[1], s1, e1);
            two_sum(s1, cz * nh[2], dh, e2);
            const float dl = (e1 + e2) + (cx * nl[0] + cy * nl[1] + cz * nl[2]);
            const float den = dh + dl;
            bool test = !(den == 0.0f && dh == 0.0f);  // else c_i parallel to the face plane: no hit
            const float ad = fabsf(den);
            const float sg = den > 0.f ? 1.f : -1.f;
            const bool unc = ad <= (cl == 1.0f ? 1e-5f : 1.41421356e-5f) * nn2;
            const float sn = sg * num, hd = h32 * ad;
            // certified t < 0 or t > 1 (h32 |den| is within 8u of h |den| when den is not tiny)
            if (!unc && (sn < -eps_num || sn - eps_num > hd * (1.0f + 8.0f * kU32))) test = false;
            if (test) {
              bool out = false, all_in = true;
#pragma unroll
              for (int k = 0; k < 3; ++k) {
                const float u = sg * (cx * Cx[k][0] + cy * Cx[k][1] + cz * Cx[k][2]);
                const float eu = 8.0f * kU32 * cl * Mk[k];
                if (u < -eu) out = true;
                if (!(u > eu)) all_in = false;
              }
              if (!(out && !unc)) {
                if (!unc && all_in && sn > eps_num && sn + eps_num < hd * (1.0f - 8.0f * kU32)) {
                  atomicMin(&s_key[di - 1][rq], hit_key(num / (h32 * den), fq));
                  atomicOr(&s_mask[rq], 1u << (di - 1));
                } else {
                  // undecided signs: FP64 evaluation from the FP64 cell centre
                  const uint32_t id = a.adj_cell[first + rq];
                  const uint32_t blk = id / NC, bit = id % NC;
                  const GeomParams& P = a.table ? a.table[a.gid ? a.gid[blk] : 0u] : a.g0;
                  const double o3[3] = {P.origin[0], P.origin[1], P.origin[2]};
                  const double hL = scalbn(P.h0, -a.level);
                  const float4* R = reinterpret_cast<const float4*>(a.rec + fq);
                  const float4 v0 = __ldg(R), v1 = __ldg(R + 1), v2 = __ldg(R + 2);
                  const float V[9] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w, v2.x};
                  const LinkHit h = link_fallback_3(V, a.blocks + (int64_t)blk * 3, bit, o3, hL, di);
                  ++n_fb;
                  if (h.band) ++n_band;
                  if (h.hit) {
                    atomicMin(&s_key[di - 1][rq], hit_key((float)h.t, fq));
                    atomicOr(&s_mask[rq], 1u << (di - 1));
                  }
                }
              }
            }
          }
        }
        __syncwarp();  // the next chunk reuses the records and the queue
      }
    }
    __syncthreads();
    // phase 2: the tile's links in (cell, direction) order
    unsigned next = 0u;
    if (tid == 0) next = atomicAdd(lt.ticket, 1u);  // stored at the end of the phase
    const uint32_t mask = s_mask[tid];  // rows past the tile's end have none
    s_mask[tid] = 0u;
    const uint32_t hits = __popc(mask);
    const uint32_t incl = warp_inclusive_scan<uint32_t>(hits);
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    uint32_t n = 0, loc = incl - hits;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      const uint32_t x = s_warp[w];
      loc += w < wid ? x : 0u;
      n += x;
    }
    if (tid == 0) {  // claim the tile's run of the staging area (read after the next barrier)
      const unsigned long long off = n ? atomicAdd(lt.bump, (unsigned long long)n) : 0ull;
      lt.count[tile] = n;
      lt.start[tile] = off;
      s_prefix = off;
    }
    if (n <= kCompact) {
      // gather the run in shared memory (the pair records are free now), then store it
      // with consecutive threads on consecutive entries
      unsigned long long* ck = reinterpret_cast<unsigned long long*>(&s_pr[0][0]);
      uint8_t* cr = reinterpret_cast<uint8_t*>(&s_q[0][0]);
      for (uint32_t m = mask; m; m &= m - 1, ++loc) {
        const int q = __ffs(m) - 1;
        ck[loc] = stage_key(s_key[q][tid], q + 1);
        cr[loc] = (uint8_t)tid;
        s_key[q][tid] = ~0ull;
      }
      __syncthreads();
      const uint64_t off = s_prefix;
      for (uint32_t i = tid; i < n; i += kLThreads) {
        if ((int64_t)(off + i) < lt.stage_cap) {
          lt.stage_key[off + i] = ck[i];
          lt.stage_row[off + i] = cr[i];
        }
      }
    } else {
      __syncthreads();
      const uint64_t off = s_prefix;
      for (uint32_t m = mask; m; m &= m - 1, ++loc) {
        const int q = __ffs(m) - 1;
        if ((int64_t)(off + loc) < lt.stage_cap) {
          lt.stage_key[off + loc] = stage_key(s_key[q][tid], q + 1);
          lt.stage_row[off + loc] = (uint8_t)tid;
        }
        s_key[q][tid] = ~0ull;
      }
    }
    if (tid == 0) s_tile = next;
    __syncthreads();  // the gathered run, s_warp and s_prefix are reused by the next tile
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n_fb += __shfl_xor_sync(0xffffffffu, n_fb, o);
    n_band += __shfl_xor_sync(0xffffffffu, n_band, o);
  }
  if (lane == 0) {
    if (n_fb) atomicAdd(&a.counters[CNT_LINK_FALLBACK], n_fb);
    if (n_band) atomicAdd(&a.counters[CNT_LINK_BAND], n_band);
    if (n_cand) atomicAdd(&a.counters[CNT_LINK_CAND], n_cand);
  }
}

// Move each tile's staged links to its place in the output: a warp per tile,
// lanes over its links, so reads and writes are both contiguous runs.
__global__ void __launch_bounds__(256, 4) k_links_place(LinkArgs a, LinkTiles lt) {
  const uint64_t row0 = a.run ? a.run[0] : 0ull;
  const uint64_t link0 = a.run ? a.run[2] : 0ull;
  if (blockIdx.x == 0 && threadIdx.x == 0 && (int64_t)(link0 + *a.n_links) > a.link_cap) atomicOr(a.err, ERR_OVERFLOW);
  const int64_t nt = (int64_t)*lt.n_tiles;
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  uint64_t nn = 0, ns = 0, np = 0;  // the next tile's count, start and place, loaded a tile ahead
  if (t < nt) {
    nn = lt.count[t];
    ns = lt.start[t];
    np = lt.place[t];
  }
  for (; t < nt; t += nw) {
    const uint64_t n = nn, src = ns, dst = link0 + np;
    if (t + nw < nt) {
      nn = lt.count[t + nw];
      ns = lt.start[t + nw];
      np = lt.place[t + nw];
    }
    const uint32_t first = (uint32_t)(row0 + (uint64_t)t * kLRows);
    for (uint64_t j0 = 0; j0 < n; j0 += 8 * 32) {  // eight loads in flight per lane
      unsigned long long k[8];
      uint32_t rw[8];
      bool ok[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const uint64_t j = j0 + 32u * u + (uint64_t)lane;
        ok[u] = j < n && (int64_t)(src + j) < lt.stage_cap && (int64_t)(dst + j) < a.link_cap;
        k[u] = ok[u] ? lt.stage_key[src + j] : 0ull;
        rw[u] = ok[u] ? lt.stage_row[src + j] : 0u;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const uint64_t d = dst + j0 + 32u * u + (uint64_t)lane;
        if (ok[u]) {
          a.link_cell[d] = first + rw[u];
          a.link_dir[d] = (uint8_t)((k[u] >> 29) & 31u);
          a.link_q[d] = __uint_as_float((uint32_t)(k[u] >> 34));
          a.link_face[d] = (uint32_t)(k[u] & ((1ull << 29) - 1));
        }
      }
    }
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

namespace {
constexpr size_t kLinkHead = 32;  // ticket, bump, tile count
int64_t link_tiles(int64_t n_adj) {
  const int64_t tiles = (n_adj + kLRows - 1) / kLRows;
  return tiles > 0 ? tiles : 1;
}
size_t align16(size_t n) { return (n + 15) & ~(size_t)15; }
}  // namespace

size_t links_scratch_bytes(int64_t n_adj) {
  const int64_t tiles = link_tiles(n_adj);
  return kLinkHead + align16(3 * sizeof(uint64_t) * (size_t)tiles) + scan_u64_scratch_bytes(tiles);
}

size_t links_stage_bytes(int64_t cap_links) {
  const int64_t n = cap_links > 0 ? cap_links : 1;
  return align16(sizeof(unsigned long long) * (size_t)n) + (size_t)n;
}

int launch_links(const LinkArgs& a, void* scratch, int num_sms, cudaStream_t st) {
  const int64_t cap_tiles = link_tiles(a.cap_rows);
  char* base = static_cast<char*>(scratch);
  LinkTiles lt{};
  lt.ticket = reinterpret_cast<unsigned*>(base);
  lt.bump = reinterpret_cast<unsigned long long*>(base + 8);
  lt.n_tiles = reinterpret_cast<uint64_t*>(base + 16);
  lt.count = reinterpret_cast<uint64_t*>(base + kLinkHead);
  lt.start = lt.count + cap_tiles;
  lt.place = lt.start + cap_tiles;
  void* scan_scratch = base + kLinkHead + align16(3 * sizeof(uint64_t) * (size_t)cap_tiles);
  const int64_t stage_cap = a.link_cap > 0 ? a.link_cap : 1;
  lt.stage_key = static_cast<unsigned long long*>(a.stage);
  lt.stage_row = static_cast<uint8_t*>(a.stage) + align16(sizeof(unsigned long long) * (size_t)stage_cap);
  lt.stage_cap = a.link_cap;
  cudaMemsetAsync(scratch, 0, kLinkHead, st);
  // persistent: as many blocks as fit on the GPU at once, tiles handed out by ticket
  // blocks per SM, asked once per dimension (contexts on several host threads may ask together)
  static std::atomic<int> occ[2] = {0, 0};
  int o = occ[a.dim == 3 ? 1 : 0].load(std::memory_order_relaxed);
  if (o == 0) {
    if (a.dim == 3)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_links<3>, kLThreads, 0);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_links<2>, kLThreads, 0);
    if (o < 1) o = 1;
    occ[a.dim == 3 ? 1 : 0].store(o, std::memory_order_relaxed);
  }
  int64_t grid = cap_tiles;
  if (grid > (int64_t)num_sms * o) grid = (int64_t)num_sms * o;
  if (a.dim == 3)
    k_links<3><<<(unsigned)grid, kLThreads, 0, st>>>(a, lt);
  else
    k_links<2><<<(unsigned)grid, kLThreads, 0, st>>>(a, lt);
  // the tiles' places (exclusive scan in tile order) and the level's link count
  const int n_scan = launch_scan_u64(lt.count, lt.place, cap_tiles, lt.n_tiles, a.n_links, scan_scratch, a.err,
                                     num_sms, st);
  int64_t pg = (cap_tiles + 7) / 8;  // 8 warps per block, a warp per tile
  if (pg > (int64_t)num_sms * 4) pg = (int64_t)num_sms * 4;  // resident at once
  k_links_place<<<(unsigned)pg, 256, 0, st>>>(a, lt);
  return 2 + n_scan;
}

int launch_advance(const uint64_t* level_tot, const uint64_t* n_links, uint64_t* run, uint32_t* adj_off,
                   int64_t cap_cells, unsigned* err, bool close, cudaStream_t st) {
  k_advance<<<1, 1, 0, st>>>(level_tot, n_links, run, adj_off, cap_cells, err, close);
  return 1;
}

}  // namespace amr
