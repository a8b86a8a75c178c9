// k_refine.cu — near-wall refinement of one grid level, child compaction and
// the finest level's adjacent-face lists.
//
// Paper (Sec. "Identification of Cells Near the Boundary", "Face Detection",
// "Spatial Binning Algorithm"): every cell of every block of the level checks
// the faces stored in the bins around it; a block with an adjacent cell is
// marked and M_RefineAndCoarsenBlocks subdivides it.  The paper maps one
// thread to one cell (thread block = cell block) and tests the cell centre
// against the face with Alg. 1.
//
// Here one warp owns one block of 4^D cells (two cells per lane in 3D).  The
// warp walks the bins overlapped by the block's query box (block inflated by
// d_L); each lane takes one bin entry, visits it only in its canonical bin
// (so a face seen in several bins is tested once), and runs the separating-axis
// test of the face against the whole inflated block.  Survivors leave their
// per-axis projection intervals in shared memory and every lane tests its
// cells against them.  The adjacency bits are combined with warp ballots.
//
// Decisions are exact: each FP32 axis test carries a forward error bound; a
// (cell, face) pair whose sign is not certified on every axis is re-evaluated
// in FP64 (and counted).  Block-level culls only use certified separations.
#include "internal.cuh"

namespace amr {

namespace {

constexpr float kEpsK = 16.0f;  // safety factor over the forward error bound (see axis_bound)

template <int D>
struct Surv;

// Per-survivor data in the block frame (origin = the block's lower corner).
// Axis order (3D): 0..2 box axes, 3 face normal, 4 + 3k + i = e_i x edge_k.
// Per axis the cell-centre projection x is tested against four thresholds
// t = (lo - eps, hi + eps, lo + eps, hi - eps), [lo, hi] being the face's
// projection widened by the cell's: x < t.x or x > t.y certifies separation,
// t.z < x < t.w certifies overlap, anything else is not certified.
template <>
struct Surv<3> {
  float4 en[3];  // e0.xyz e1.x | e1.yz e2.xy | e2.z n.xyz
  float4 t[13];
  uint32_t face;
  uint32_t pad[3];
};
// 2D: 0..1 box axes, 2 segment normal (-e_y, e_x).
template <>
struct Surv<2> {
  float4 t[3];
  float e[2];
  uint32_t face;
  uint32_t pad[1];
};

// FP64 decision of the separating-axis test of the box [x_c - r, x_c + r]^3
// and the closed triangle (vertices absolute FP32).  The margin of the
// definition is max over the 13 axes of gap_a / |a| (gap_a = the FP64 gap
// between the projected intervals); its sign is that of the largest gap_a, so
// the pair is adjacent exactly when no axis has gap_a > 0, and no square root
// or division is needed (a quotient of normal magnitudes does not underflow).
// *band: the margin lies within tol of 0, tested as gap_a^2 <= tol^2 |a|^2 on
// the deciding axes (a diagnostic count).  An axis with gap_a > tol |a| settles
// the pair at once: separated, outside the band.
__device__ __noinline__ bool sat_adjacent_fp64_3(const float* V, const double* xc, double r, double tol,
                                                 bool* band) {
  double p[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) p[k][c] = __dsub_rn((double)V[3 * k + c], xc[c]);
  const double tol2 = tol * tol;
  bool sep = false;        // some axis with a positive gap
  bool pos_small = true;   // every positive gap within tol |a|
  bool near0 = false;      // some axis with gap >= -tol |a|
  // false: the pair is settled (separated beyond the band)
  auto axis = [&](double a0, double a1, double a2) -> bool {
    const double l2sq = __dadd_rn(__dadd_rn(__dmul_rn(a0, a0), __dmul_rn(a1, a1)), __dmul_rn(a2, a2));
    if (l2sq == 0.0) return true;
    double lo = 1e300, hi = -1e300;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double s = __dadd_rn(__dadd_rn(__dmul_rn(p[k][0], a0), __dmul_rn(p[k][1], a1)), __dmul_rn(p[k][2], a2));
      lo = fmin(lo, s);
      hi = fmax(hi, s);
    }
    const double R = __dmul_rn(r, __dadd_rn(__dadd_rn(fabs(a0), fabs(a1)), fabs(a2)));
    const double g = fmax(__dsub_rn(lo, R), __dsub_rn(-R, hi));
    const bool small = __dmul_rn(g, g) <= __dmul_rn(tol2, l2sq);
    if (g > 0.0) {
      sep = true;
      if (!small) {
        pos_small = false;
        return false;
      }
    } else if (small) {
      near0 = true;
    }
    return true;
  };
  *band = false;
  if (!axis(1.0, 0.0, 0.0) || !axis(0.0, 1.0, 0.0) || !axis(0.0, 0.0, 1.0)) return false;
  const double u0 = __dsub_rn(p[1][0], p[0][0]), u1 = __dsub_rn(p[1][1], p[0][1]), u2 = __dsub_rn(p[1][2], p[0][2]);
  const double w0 = __dsub_rn(p[2][0], p[0][0]), w1 = __dsub_rn(p[2][1], p[0][1]), w2 = __dsub_rn(p[2][2], p[0][2]);
  if (!axis(__dsub_rn(__dmul_rn(u1, w2), __dmul_rn(u2, w1)), __dsub_rn(__dmul_rn(u2, w0), __dmul_rn(u0, w2)),
            __dsub_rn(__dmul_rn(u0, w1), __dmul_rn(u1, w0))))
    return false;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int k1 = (k + 1) % 3;
    const double ex = __dsub_rn(p[k1][0], p[k][0]), ey = __dsub_rn(p[k1][1], p[k][1]),
                 ez = __dsub_rn(p[k1][2], p[k][2]);
    if (!axis(0.0, -ez, ey) || !axis(ez, 0.0, -ex) || !axis(-ey, ex, 0.0)) return false;
  }
  *band = sep ? pos_small : near0;
  return !sep;
}

__device__ __noinline__ double margin_fp64_2(const float* V, const double* xc, double r) {
  double p[2][2];
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int c = 0; c < 2; ++c) p[k][c] = __dsub_rn((double)V[2 * k + c], xc[c]);
  double m = -1e300;
  auto axis = [&](double a0, double a1) {
    const double l2 = sqrt(__dadd_rn(__dmul_rn(a0, a0), __dmul_rn(a1, a1)));
    if (l2 == 0.0) return;
    const double s0 = __dadd_rn(__dmul_rn(p[0][0], a0), __dmul_rn(p[0][1], a1));
    const double s1 = __dadd_rn(__dmul_rn(p[1][0], a0), __dmul_rn(p[1][1], a1));
    const double lo = fmin(s0, s1), hi = fmax(s0, s1);
    const double R = __dmul_rn(r, __dadd_rn(fabs(a0), fabs(a1)));
    m = fmax(m, fmax(__dsub_rn(lo, R), __dsub_rn(-R, hi)) / l2);
  };
  axis(1.0, 0.0);
  axis(0.0, 1.0);
  const double e0 = __dsub_rn(p[1][0], p[0][0]), e1 = __dsub_rn(p[1][1], p[0][1]);
  axis(-e1, e0);
  return m;
}

// FP64 distance from the point xc to the closed face (vertices absolute FP32):
// the plane distance when the projection lies in the closed triangle, else the
// smallest distance to the three edges (the point predicate of Alg. 1).
__device__ __forceinline__ double seg_dist2_fp64(const double* a, const double* b, int dim) {
  double e[3] = {0, 0, 0}, ae = 0.0, ee = 0.0;
  for (int c = 0; c < dim; ++c) {
    e[c] = __dsub_rn(b[c], a[c]);
    ae = __fma_rn(-a[c], e[c], ae);
    ee = __fma_rn(e[c], e[c], ee);
  }
  const double t = ee > 0.0 ? fmin(1.0, fmax(0.0, ae / ee)) : 0.0;
  double d2 = 0.0;
  for (int c = 0; c < dim; ++c) {
    const double q = __fma_rn(t, e[c], a[c]);
    d2 = __fma_rn(q, q, d2);
  }
  return d2;
}

__device__ __noinline__ double point_dist_fp64(const float* V, const double* xc, int dim) {
  double p[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int k = 0; k < dim; ++k)
    for (int c = 0; c < dim; ++c) p[k][c] = __dsub_rn((double)V[dim * k + c], xc[c]);
  if (dim == 2) return sqrt(seg_dist2_fp64(p[0], p[1], 2));
  const double u[3] = {p[1][0] - p[0][0], p[1][1] - p[0][1], p[1][2] - p[0][2]};
  const double w[3] = {p[2][0] - p[0][0], p[2][1] - p[0][1], p[2][2] - p[0][2]};
  const double n[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
  const double nn = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
  if (nn > 0.0) {
    bool neg = true, pos = true;
    for (int k = 0; k < 3; ++k) {
      const double* a = p[k];
      const double* b = p[(k + 1) % 3];
      const double e[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
      const double m[3] = {e[1] * n[2] - e[2] * n[1], e[2] * n[0] - e[0] * n[2], e[0] * n[1] - e[1] * n[0]};
      const double sk = -(a[0] * m[0] + a[1] * m[1] + a[2] * m[2]);
      if (sk > 0.0) neg = false;
      if (sk < 0.0) pos = false;
    }
    if (neg || pos) return fabs(p[0][0] * n[0] + p[0][1] * n[1] + p[0][2] * n[2]) / sqrt(nn);
  }
  return sqrt(fmin(seg_dist2_fp64(p[0], p[1], 3), fmin(seg_dist2_fp64(p[1], p[2], 3), seg_dist2_fp64(p[2], p[0], 3))));
}

// Block-frame quantities shared by all lanes of the warp for one block.
template <int D>
struct BlockFrame {
  float Xb[3];     // block corner rounded to FP32 (the frame origin)
  float cB[3];     // block centre in the frame
  float h, r, rb;  // cell size, cell and block half-widths (inflated) in FP32
  float O;         // bound on |cell centre offsets| and |block centre| in the frame
};

// Per-face setup (one lane): edges, projections of the face on every axis in
// the block frame, the cell-level intervals [tmin - r|a|_1, tmax + r|a|_1] and
// their error bounds.  Returns false when some axis certifiably separates the
// face from the whole inflated block.
//
// Error bound per axis a: every computed projection, interval end and cell
// coordinate differs from its exact value by at most a few unit roundoffs of
// (P + O + r) |a|_1, where P bounds the vertex offsets in the frame (this also
// covers the rounding of the frame origin, of the edges when they are not
// exact and of the FP32 normal relative to the FP64 one).  eps = 16 u (P+O+r)|a|_1.
template <int D>
__device__ __forceinline__ bool setup_face(const float* V, const float* nh, const BlockFrame<D>& F, Surv<D>& S) {
  float p[3][3];
  float P = 0.f;
#pragma unroll
  for (int k = 0; k < D; ++k)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      p[k][c] = V[D * k + c] - F.Xb[c];
      P = fmaxf(P, fabsf(p[k][c]));
    }
  const float scale = kEpsK * kU32 * (P + F.O + F.r);
  // one axis: false when it certifiably separates the face from the whole inflated block
  auto axis = [&](int ai, float ax, float ay, float az) -> bool {
    const float A1 = fabsf(ax) + fabsf(ay) + fabsf(az);
    if (A1 == 0.0f) {
      S.t[ai] = make_float4(-INFINITY, INFINITY, -INFINITY, INFINITY);
      return true;
    }
    float tmin = INFINITY, tmax = -INFINITY;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float s = D == 3 ? fmaf(p[k][2], az, fmaf(p[k][1], ay, p[k][0] * ax)) : fmaf(p[k][1], ay, p[k][0] * ax);
      tmin = fminf(tmin, s);
      tmax = fmaxf(tmax, s);
    }
    const float eps = scale * A1;
    const float xb = D == 3 ? fmaf(F.cB[2], az, fmaf(F.cB[1], ay, F.cB[0] * ax)) : fmaf(F.cB[1], ay, F.cB[0] * ax);
    const float RB = F.rb * A1;
    // block interval [xb - RB, xb + RB] vs face interval [tmin, tmax]
    if (xb - RB - tmax > eps || tmin - (xb + RB) > eps) return false;
    const float R = F.r * A1;
    const float lo = tmin - R, hi = tmax + R;
    S.t[ai] = make_float4(lo - eps, hi + eps, lo + eps, hi - eps);
    return true;
  };
  if constexpr (D == 3) {
    float e[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int k1 = (k + 1) % 3;
#pragma unroll
      for (int c = 0; c < 3; ++c) e[k][c] = V[3 * k1 + c] - V[3 * k + c];
    }
    // box axes first: the cheap AABB cull
    if (!axis(0, 1.f, 0.f, 0.f) || !axis(1, 0.f, 1.f, 0.f) || !axis(2, 0.f, 0.f, 1.f)) return false;
    if (!axis(3, nh[0], nh[1], nh[2])) return false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float ex = e[k][0], ey = e[k][1], ez = e[k][2];
      if (!axis(4 + 3 * k, 0.f, -ez, ey)) return false;
      if (!axis(5 + 3 * k, ez, 0.f, -ex)) return false;
      if (!axis(6 + 3 * k, -ey, ex, 0.f)) return false;
    }
    S.en[0] = make_float4(e[0][0], e[0][1], e[0][2], e[1][0]);
    S.en[1] = make_float4(e[1][1], e[1][2], e[2][0], e[2][1]);
    S.en[2] = make_float4(e[2][2], nh[0], nh[1], nh[2]);
  } else {
    const float e0 = V[2] - V[0], e1 = V[3] - V[1];
    if (!axis(0, 1.f, 0.f, 0.f) || !axis(1, 0.f, 1.f, 0.f)) return false;
    if (!axis(2, -e1, e0, 0.f)) return false;
    S.e[0] = e0;
    S.e[1] = e1;
  }
  return true;
}

// Cell tests of the lane's two cells against one survivor: 0 = separated,
// 1 = intersecting, 2 = not certified (needs FP64).  o0 / o1 are the cell
// centres in the block frame.  All axes are evaluated (the warp runs the
// longest lane anyway); the thresholds come as one 16-byte load per axis.
template <int D>
__device__ __forceinline__ void cell_test2(const Surv<D>& S, const float* o0, const float* o1, int& r0, int& r1) {
  bool sep0 = false, in0 = true, sep1 = false, in1 = true;
  auto upd = [](float x, const float4& t, bool& sep, bool& in) {
    sep |= (x < t.x) | (x > t.y);
    in &= (x > t.z) & (x < t.w);
  };
  if constexpr (D == 3) {
#pragma unroll
    for (int ai = 0; ai < 3; ++ai) {
      const float4 t = S.t[ai];
      upd(o0[ai], t, sep0, in0);
      upd(o1[ai], t, sep1, in1);
    }
    const float4 q0 = S.en[0], q1 = S.en[1], q2 = S.en[2];
    const float e[3][3] = {{q0.x, q0.y, q0.z}, {q0.w, q1.x, q1.y}, {q1.z, q1.w, q2.x}};
    {
      const float4 t = S.t[3];
      upd(fmaf(o0[2], q2.w, fmaf(o0[1], q2.z, o0[0] * q2.y)), t, sep0, in0);
      upd(fmaf(o1[2], q2.w, fmaf(o1[1], q2.z, o1[0] * q2.y)), t, sep1, in1);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float ex = e[k][0], ey = e[k][1], ez = e[k][2];
      const float4 ta = S.t[4 + 3 * k], tb = S.t[5 + 3 * k], tc = S.t[6 + 3 * k];
      upd(fmaf(o0[2], ey, -o0[1] * ez), ta, sep0, in0);
      upd(fmaf(o1[2], ey, -o1[1] * ez), ta, sep1, in1);
      upd(fmaf(o0[0], ez, -o0[2] * ex), tb, sep0, in0);
      upd(fmaf(o1[0], ez, -o1[2] * ex), tb, sep1, in1);
      upd(fmaf(o0[1], ex, -o0[0] * ey), tc, sep0, in0);
      upd(fmaf(o1[1], ex, -o1[0] * ey), tc, sep1, in1);
    }
  } else {
#pragma unroll
    for (int ai = 0; ai < 2; ++ai) upd(o0[ai], S.t[ai], sep0, in0);
    upd(fmaf(o0[1], S.e[0], -o0[0] * S.e[1]), S.t[2], sep0, in0);
    sep1 = true;
  }
  r0 = sep0 ? 0 : (in0 ? 1 : 2);
  r1 = sep1 ? 0 : (in1 ? 1 : 2);
}

// Point predicate: survivor data in the block frame, stored over the
// thresholds of the box predicate.  3D layout: t[0..2] = vertex k (xyz) with
// 1/|n|^2 (0: zero-area face) and the error scale in .w of t[0] / t[1];
// t[3..5] = edge e_k = p_{k+1} - p_k with 1/|e_k|^2; t[6..8] = m_k = e_k x n
// with the edge-function error scale in t[6].w; t[9] = n.
// Error analysis (u = 2^-24, L = bound on |coordinates| in the frame, vertex
// offsets plus cell-centre offsets): every difference w = x - p_k carries one
// rounding (<= 2uL per component), the squared edge and plane distances are
// sums of a few products of such terms and are within 64 u (2 sqrt(3) L)^2 of
// their exact values; an edge function m_k . w_k is within 96 u L |e_k|_1 |n|_1.
template <int D>
__device__ __forceinline__ void setup_point(const float* V, const float* nh, const BlockFrame<D>& F, Surv<D>& S) {
  float p[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  float P = 0.f;
#pragma unroll
  for (int k = 0; k < D; ++k)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      p[k][c] = V[D * k + c] - F.Xb[c];
      P = fmaxf(P, fabsf(p[k][c]));
    }
  const float L = P + F.O;
  const float E = 64.0f * kU32 * 12.0f * L * L;
  if constexpr (D == 3) {
    float e[3][3], m[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) e[k][c] = p[(k + 1) % 3][c] - p[k][c];
    const float nn = nh[0] * nh[0] + nh[1] * nh[1] + nh[2] * nh[2];
    const float n1 = fabsf(nh[0]) + fabsf(nh[1]) + fabsf(nh[2]);
    float m1 = 0.f;  // bound on |m_k|_1 and on its rounding, max_k |e_k|_1 |n|_1
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      m[k][0] = e[k][1] * nh[2] - e[k][2] * nh[1];
      m[k][1] = e[k][2] * nh[0] - e[k][0] * nh[2];
      m[k][2] = e[k][0] * nh[1] - e[k][1] * nh[0];
      m1 = fmaxf(m1, (fabsf(e[k][0]) + fabsf(e[k][1]) + fabsf(e[k][2])) * n1);
    }
    S.t[0] = make_float4(p[0][0], p[0][1], p[0][2], nn > 0.f ? 1.0f / nn : 0.f);
    S.t[1] = make_float4(p[1][0], p[1][1], p[1][2], E);
    S.t[2] = make_float4(p[2][0], p[2][1], p[2][2], 0.f);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float ee = e[k][0] * e[k][0] + e[k][1] * e[k][1] + e[k][2] * e[k][2];
      S.t[3 + k] = make_float4(e[k][0], e[k][1], e[k][2], ee > 0.f ? 1.0f / ee : 0.f);
      S.t[6 + k] = make_float4(m[k][0], m[k][1], m[k][2], k == 0 ? 96.0f * kU32 * m1 * L : 0.f);
    }
    S.t[9] = make_float4(nh[0], nh[1], nh[2], 0.f);
  } else {
    const float e0 = p[1][0] - p[0][0], e1 = p[1][1] - p[0][1];
    const float ee = e0 * e0 + e1 * e1;
    S.t[0] = make_float4(p[0][0], p[0][1], e0, e1);
    S.t[1] = make_float4(ee > 0.f ? 1.0f / ee : 0.f, E, 0.f, 0.f);
  }
}

// Squared distance from w (= x - p) to the segment p + s e, s in [0, 1].
__device__ __forceinline__ float seg_dist2(float wx, float wy, float wz, const float4& e) {
  const float s = fminf(1.0f, fmaxf(0.0f, (wx * e.x + wy * e.y + wz * e.z) * e.w));
  const float qx = fmaf(-s, e.x, wx), qy = fmaf(-s, e.y, wy), qz = fmaf(-s, e.z, wz);
  return qx * qx + qy * qy + qz * qz;
}

// Point-predicate test of one cell centre o: 0 = farther than d, 1 = within
// d, 2 = not certified (FP64).  The plane distance A is a lower bound of the
// distance and the nearest edge distance Bv an upper bound; A applies when the
// projection is certainly inside the triangle, Bv when it is certainly outside.
template <int D>
__device__ __forceinline__ int point_test(const Surv<D>& S, const float* o, float R2) {
  if constexpr (D == 3) {
    const float4 t0 = S.t[0], t1 = S.t[1], t2 = S.t[2];
    const float E = t1.w;
    const float w[3][3] = {{o[0] - t0.x, o[1] - t0.y, o[2] - t0.z},
                           {o[0] - t1.x, o[1] - t1.y, o[2] - t1.z},
                           {o[0] - t2.x, o[1] - t2.y, o[2] - t2.z}};
    float Bv = INFINITY;
#pragma unroll
    for (int k = 0; k < 3; ++k) Bv = fminf(Bv, seg_dist2(w[k][0], w[k][1], w[k][2], S.t[3 + k]));
    if (Bv <= R2 - E) return 1;
    const float4 n = S.t[9];
    const float pn = w[0][0] * n.x + w[0][1] * n.y + w[0][2] * n.z;
    const float A = t0.w > 0.f ? pn * pn * t0.w : 0.f;
    if (A > R2 + E) return 0;
    const float es = S.t[6].w;
    bool neg = true, pos = true, lo = false, hi = false;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float4 m = S.t[6 + k];
      const float sk = w[k][0] * m.x + w[k][1] * m.y + w[k][2] * m.z;
      if (!(sk < -es)) neg = false;
      if (!(sk > es)) pos = false;
      if (sk < -es) lo = true;
      if (sk > es) hi = true;
    }
    const bool inside = t0.w > 0.f && (neg || pos);
    const bool outside = t0.w == 0.f || (lo && hi);
    if (inside) return A < R2 - E ? 1 : 2;
    if (outside) return Bv > R2 + E ? 0 : 2;
    return 2;
  } else {
    const float4 t0 = S.t[0], t1 = S.t[1];
    const float d2 = seg_dist2(o[0] - t0.x, o[1] - t0.y, 0.f, make_float4(t0.z, t0.w, 0.f, t1.x));
    if (d2 <= R2 - t1.y) return 1;
    if (d2 > R2 + t1.y) return 0;
    return 2;
  }
}

struct WarpCounters {
  unsigned long long fb = 0, band = 0, cand = 0, surv = 0, big = 0;
};

template <int D>
__device__ __noinline__ bool resolve_fp64(const RefineLevel& a, uint32_t gid, uint32_t face, const int* b,
                                          int cell_local, unsigned long long* fb, unsigned long long* band) {
  const LevelGeom G = level_geom(a.table ? a.table[gid] : a.g0, a.level);
  float V[D * D];
#pragma unroll
  for (int j = 0; j < D * D; ++j) V[j] = a.X[(int64_t)j * a.nf + face];
  double xc[3];
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const int li = (cell_local >> (2 * c)) & 3;
    xc[c] = __dadd_rn(G.origin[c], __dmul_rn((double)(4 * b[c] + li) + 0.5, G.h));
  }
  const double r = __dadd_rn(0.5 * G.h, G.d);
  ++*fb;
  if (D == 3 && a.pred != 1) {
    bool in_band = false;
    const bool adj = sat_adjacent_fp64_3(V, xc, r, kBandRel * G.h, &in_band);
    if (in_band) ++*band;
    return adj;
  }
  const double m = a.pred == 1 ? point_dist_fp64(V, xc, D) - G.d : margin_fp64_2(V, xc, r);
  if (fabs(m) <= kBandRel * G.h) ++*band;
  return m <= 0.0;
}

// Shared walk of one block: bins of the query box, canonical-bin dedup,
// block-level cull, cell tests.  For every surviving face the whole warp calls
// `on_surv(face, r0, r1)`, r0 / r1 = whether the face meets the lane's cell
// `lane` / `lane + 32`; h0 / h1 accumulate them.  kMarkOnly: only the mask is
// wanted, so marked cells skip further tests and the walk ends as soon as every
// cell of the block is marked.
//
// The block frame is built in FP32 from the geometry row's double-float h0 and
// origin: the block corner origin + 4 b h is formed as hi + lo (hi = the frame
// origin, lo = its rounding error, carried into the cell and block centres),
// so no FP64 instruction runs per block.  The bin query range is widened by
// a margin that covers the FP32 error of the bin coordinate (a superset of
// bins only adds candidates the block test rejects).
// Per-warp shared memory of the walk: survivor data, a double buffer of bin
// entries filled by TMA bulk copies with one mbarrier per buffer, and the
// block's survivor records.
template <int D>
struct WarpSmem {
  Surv<D> surv[32];
  typename EntryT<D>::type buf[2][32];
  uint64_t bar[2];
  uint64_t rm[kRecCap];  // survivor records of the block: cell-hit masks ...
  uint32_t rf[kRecCap];  // ... and face ids
};

template <int D>
__device__ __forceinline__ void warp_smem_init(WarpSmem<D>& sm, int lane) {
  if (lane == 0) {
    mbar_init(&sm.bar[0], 1);
    mbar_init(&sm.bar[1], 1);
    mbar_fence_init();
  }
  __syncwarp();
}

// The entries of the query box's x-rows (y, z fixed, x in [qlo_x, qhi_x]) are
// contiguous in the bin payload.  Lane i holds row i of the current group of
// (up to) 32 rows: its first entry `s`, its length `n` and the row's start
// `v` in the group's concatenated entry list.  Chunk c = entries [32c, 32c+32)
// of that list; every lane copies its row's part of the chunk into the buffer
// (lane 0 first announces the chunk's bytes on the buffer's mbarrier).
template <typename E>
__device__ __forceinline__ void issue_chunk(const E* payload, uint32_t s, uint32_t n, uint32_t v, uint32_t c,
                                            uint32_t T, E* buf, uint64_t* bar, int lane) {
  const uint32_t c0 = 32u * c, c1 = c0 + 32u < T ? c0 + 32u : T;
  if (lane == 0) mbar_arrive_expect_tx(bar, (c1 - c0) * (uint32_t)sizeof(E));
  __syncwarp();
  const uint32_t a0 = v > c0 ? v : c0, a1 = v + n < c1 ? v + n : c1;
  if (a0 < a1) {
    fence_proxy_async_smem();  // this warp's earlier reads of the buffer come first
    bulk_copy_g2s(buf + (a0 - c0), payload + s + (a0 - v), (a1 - a0) * (uint32_t)sizeof(E), bar);
  }
}

// Shared walk of one block: bins of the query box, canonical-bin dedup,
// block-level cull, cell tests.  For every surviving face the whole warp calls
// `on_surv(face, r0, r1)`, r0 / r1 = whether the face meets the lane's cell
// `lane` / `lane + 32`; h0 / h1 accumulate them.  kMarkOnly: only the mask is
// wanted, so marked cells skip further tests and the walk ends as soon as every
// cell of the block is marked.
//
// The block frame is built in FP32 from the geometry row's double-float h0 and
// origin: the block corner origin + 4 b h is formed as hi + lo (hi = the frame
// origin, lo = its rounding error, carried into the cell and block centres),
// so no FP64 instruction runs per block.  The bin query range is widened by
// a margin that covers the FP32 error of the bin coordinate (a superset of
// bins only adds candidates the block test rejects).
//
// The bin ranges of all x-rows of the box are read in parallel (one lane per
// row); entries then arrive in shared memory by TMA bulk copies in chunks of
// 32, double-buffered: the next chunk is requested before the warp tests the
// current one.
template <int D, int PRED, bool kMarkOnly, typename OnSurv>
__device__ __forceinline__ void walk_block(const RefineLevel& a, const GeomParams& P, uint32_t gid, const int* b,
                                           WarpSmem<D>& sm, uint32_t& phase, int lane, WarpCounters& wc, bool& h0,
                                           bool& h1, OnSurv on_surv) {
  using E = typename EntryT<D>::type;
  const FastGeom g = fast_geom(P, a.level);
  const float hf = g.h_hi;
  BlockFrame<D> F;
  int qlo[3] = {0, 0, 0}, qhi[3] = {0, 0, 0};
  float O = 4.0f * hf;
  float shift[3] = {0.f, 0.f, 0.f};
  const int Bn = P.B;
  const float margin = 1e-6f * (float)Bn + 1e-3f;
#pragma unroll
  for (int c = 0; c < D; ++c) {
    float lo;
    df_position(P.org_hi[c], P.org_lo[c], (float)(4 * b[c]), g.h_hi, g.h_lo, F.Xb[c], lo);
    shift[c] = lo;
    F.cB[c] = fmaf(2.0f, g.h_hi, lo);
    O = fmaxf(O, 4.0f * hf + 2.0f * fabsf(lo));
    // bin coordinates of the inflated block's ends relative to the domain origin
    const float k0 = (float)(4 * b[c]);
    const float xlo = fmaf(k0, g.h_hi, fmaf(k0, g.h_lo, -g.d));
    const float xhi = fmaf(k0 + 4.0f, g.h_hi, fmaf(k0 + 4.0f, g.h_lo, g.d));
    const float tlo = floorf(xlo * P.scale32[c] - margin);
    const float thi = floorf(xhi * P.scale32[c] + margin);
    qlo[c] = tlo < 0.f ? 0 : (tlo > (float)(Bn - 1) ? Bn - 1 : (int)tlo);
    qhi[c] = thi < 0.f ? 0 : (thi > (float)(Bn - 1) ? Bn - 1 : (int)thi);
  }
  F.h = hf;
  F.r = fmaf(0.5f, hf, g.d);
  // block-level cull: the box around the block centre that holds every cell's
  // test region (point predicate: the cell centres' box, 1.5 h, inflated by d)
  constexpr bool kPoint = PRED >= 1;   // point predicate (Alg. 1)
  constexpr bool kOwnBin = PRED == 2;  // the paper's binned search: each cell only sees its own bin
  F.rb = kPoint ? fmaf(1.5f, hf, g.d) : fmaf(2.0f, hf, g.d);
  const float R2 = g.d * g.d;
  F.O = O;
  // the paper's binned search: the query box is the bins of the block's cell
  // centres, and each cell only takes the entries of its own bin (bins of the
  // FP64 cell centres, as the definition computes them)
  uint32_t own0 = 0, own1 = 0, oz0 = 0, oz1 = 0;
  if constexpr (kOwnBin) {
    const double hL = scalbn(P.h0, -a.level);
    auto centre_bin = [&](int c, int l) {
      const double x = __dadd_rn(P.origin[c], __dmul_rn((double)(4 * b[c] + l) + 0.5, hL));
      return bin_coord(x, P.origin[c], P.bin_scale[c], P.B);
    };
    uint32_t cb0[3] = {0, 0, 0}, cb1[3] = {0, 0, 0};
#pragma unroll
    for (int c = 0; c < D; ++c) {
      qlo[c] = centre_bin(c, 0);
      qhi[c] = centre_bin(c, 3);
      cb0[c] = (uint32_t)centre_bin(c, (lane >> (2 * c)) & 3);
      if (D == 3) cb1[c] = (uint32_t)centre_bin(c, ((lane + 32) >> (2 * c)) & 3);
    }
    own0 = cb0[0] | (cb0[1] << 16);
    oz0 = cb0[2];
    own1 = cb1[0] | (cb1[1] << 16);
    oz1 = cb1[2];
  }
  // cell centres of this lane in the frame: lo + (l + 1/2) h
  float o0[3] = {0, 0, 0}, o1[3] = {0, 0, 0};
  const bool lane_cell = D == 3 || lane < 16;
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const float l0 = (float)((lane >> (2 * c)) & 3) + 0.5f;
    o0[c] = fmaf(l0, g.h_hi, fmaf(l0, g.h_lo, shift[c]));
    if (D == 3) {
      const float l1 = (float)(((lane + 32) >> (2 * c)) & 3) + 0.5f;
      o1[c] = fmaf(l1, g.h_hi, fmaf(l1, g.h_lo, shift[c]));
    }
  }
  const int64_t B = Bn;
  const E* payload = static_cast<const E*>(a.payload);
  const int nx = qhi[0] - qlo[0] + 1, ny = qhi[1] - qlo[1] + 1;
  const int nrows = ny * (D == 3 ? qhi[2] - qlo[2] + 1 : 1);
  for (int rg = 0; rg < nrows; rg += 32) {
    // this group's rows: one lane each
    uint32_t rs = 0, rn = 0;
    const int ri = rg + lane;
    if (ri < nrows) {
      const int y = qlo[1] + ri % ny, z = D == 3 ? qlo[2] + ri / ny : 0;
      const int64_t b0 = P.bin_base + qlo[0] + B * (y + B * (int64_t)z);
      rs = a.offsets[b0];
      rn = a.offsets[b0 + nx] - rs;
    }
    const uint32_t incl = warp_inclusive_scan<uint32_t>(rn);
    const uint32_t T = __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t rv = incl - rn;
    const uint32_t nch = (T + 31u) / 32u;
    if (nch == 0) continue;
    int cb = 0;
    issue_chunk<E>(payload, rs, rn, rv, 0u, T, sm.buf[0], &sm.bar[0], lane);
    for (uint32_t c = 0; c < nch; ++c) {
      const int nb = cb ^ 1;
      const bool more = c + 1 < nch;
      if (more) issue_chunk<E>(payload, rs, rn, rv, c + 1, T, sm.buf[nb], &sm.bar[nb], lane);
      mbar_wait_bounded(&sm.bar[cb], (phase >> cb) & 1u, a.err);
      phase ^= 1u << cb;
      const uint32_t n = T - 32u * c < 32u ? T - 32u * c : 32u;
      bool surv = false;
      if ((uint32_t)lane < n) {
        const E& ent = sm.buf[cb][lane];
        const uint32_t id = ent.id;
        // visit a face only in the first bin of its range inside the query box
        bool canon = kOwnBin || ((id >> 29) & 1u) || (int)ent.bin[0] == qlo[0];
        canon = canon && (kOwnBin || ((id >> 30) & 1u) || (int)ent.bin[1] == qlo[1]);
        if (D == 3) canon = canon && (kOwnBin || ((id >> 31) & 1u) || (int)ent.bin[2] == qlo[2]);
        if (canon) {
          wc.cand++;
          const uint32_t f = id & kIdMask;
          float nh[3] = {0.f, 0.f, 0.f};
          if constexpr (D == 3) {
            nh[0] = ent.n[0];
            nh[1] = ent.n[1];
            nh[2] = ent.n[2];
          }
          float V[D * D];
#pragma unroll
          for (int j = 0; j < D * D; ++j) V[j] = ent.v[j];
          surv = setup_face<D>(V, nh, F, sm.surv[lane]);
          if constexpr (kPoint) {
            if (surv) setup_point<D>(V, nh, F, sm.surv[lane]);
          }
          if constexpr (kOwnBin) {
            sm.surv[lane].pad[0] = ent.bin[0] | (ent.bin[1] << 16);
            if constexpr (D == 3) sm.surv[lane].pad[1] = ent.bin[2];
          }
          sm.surv[lane].face = f;
        }
      }
      unsigned m = __ballot_sync(0xffffffffu, surv);
      __syncwarp();
      wc.surv += __popc(m);
      while (m) {
        const int s = __ffs(m) - 1;
        m &= m - 1;
        const Surv<D>& S = sm.surv[s];
        int t0 = 0, t1 = 0;
        if (!(kMarkOnly && h0 && h1)) {
          if constexpr (kOwnBin) {
            const uint32_t sz = D == 3 ? S.pad[1] : 0u;
            t0 = (own0 == S.pad[0] && oz0 == sz) ? point_test<D>(S, o0, R2) : 0;
            t1 = D == 3 && own1 == S.pad[0] && oz1 == sz ? point_test<D>(S, o1, R2) : 0;
          } else if constexpr (kPoint) {
            t0 = point_test<D>(S, o0, R2);
            t1 = D == 3 ? point_test<D>(S, o1, R2) : 0;
          } else {
            cell_test2<D>(S, o0, o1, t0, t1);
          }
        }
        bool r0 = false, r1 = false;
        if (lane_cell && !(kMarkOnly && h0)) {
          if (t0 == 2) t0 = resolve_fp64<D>(a, gid, S.face, b, lane, &wc.fb, &wc.band) ? 1 : 0;
          r0 = t0 != 0;
        }
        if (D == 3 && !(kMarkOnly && h1)) {
          if (t1 == 2) t1 = resolve_fp64<D>(a, gid, S.face, b, lane + 32, &wc.fb, &wc.band) ? 1 : 0;
          r1 = t1 != 0;
        }
        h0 |= r0;
        h1 |= r1;
        on_surv(S.face, r0, r1);
      }
      __syncwarp();
      // marking only: once every cell of the block is marked, the rest of the walk cannot change the mask
      if (kMarkOnly && __all_sync(0xffffffffu, (h0 || !lane_cell) && (D == 2 || h1))) {
        if (more) {
          mbar_wait_bounded(&sm.bar[nb], (phase >> nb) & 1u, a.err);  // the copy already in flight
          phase ^= 1u << nb;
          __syncwarp();
        }
        return;
      }
      cb = nb;
    }
  }
}

// One survivor record past the shared-memory stage, into the warp's spill area
// (out of line: it is rare, and the walk's registers stay with the common case).
// The area of the calling warp: kSpillCap records per warp of the launch.
__device__ __forceinline__ SurvRec* warp_spill(SurvRec* spill) {
  return spill + ((uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * kSpillCap;
}

__device__ __noinline__ void spill_record(SurvRec* spill, uint32_t i, uint32_t face, uint64_t cells) {
  SurvRec r;
  r.face = face;
  r.pad = 0u;
  r.cells = cells;
  warp_spill(spill)[i] = r;
}

// The block's K survivor records (staged in shared memory, past kRecCap in the
// warp's spill area) into a contiguous range of the level's record array, and
// its descriptor: offset << 16 | K, 0 for none, ~0 when they are incomplete (the
// adjacency pass then walks the block again).  Whole warp.
template <int D>
__device__ __forceinline__ void store_records(const RefineLevel& a, WarpSmem<D>& sm, uint32_t K, unsigned blk,
                                              int lane);

// Block count of a launch: from device memory when given (bounded by the
// capacity; an overflow is reported), else the host count.
__device__ __forceinline__ int64_t launch_count(int64_t n, const uint64_t* n_dev, unsigned* err) {
  if (!n_dev) return n;
  const uint64_t nd = *n_dev;
  if ((int64_t)nd > n) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, ERR_OVERFLOW);
    return n;
  }
  return (int64_t)nd;
}

template <int D>
__device__ __forceinline__ void store_records(const RefineLevel& a, WarpSmem<D>& sm, uint32_t K, unsigned blk,
                                              int lane) {
  __syncwarp();  // the staged and spilled records are visible to the whole warp
  const uint32_t kmax = (uint32_t)kRecCap + (a.spill ? (uint32_t)kSpillCap : 0u);
  uint64_t base = ~0ull;
  if (K > 0 && K <= kmax) {
    if (lane == 0) base = atomicAdd(reinterpret_cast<unsigned long long*>(a.rec_count), (unsigned long long)K);
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((int64_t)(base + K) > a.cap_recs) base = ~0ull;
  }
  if (base != ~0ull) {
    for (uint32_t i = lane; i < K; i += 32) {
      SurvRec r;
      if (i < (uint32_t)kRecCap) {
        r.face = sm.rf[i];
        r.pad = 0u;
        r.cells = sm.rm[i];
      } else {
        r = warp_spill(a.spill)[i - kRecCap];
      }
      a.recs[base + i] = r;
    }
  }
  if (lane == 0) a.rec_desc[blk] = K == 0 ? 0ull : (base == ~0ull ? ~0ull : (base << 16) | K);
  __syncwarp();
}

template <int D, int PRED>
__global__ void __launch_bounds__(256) k_refine(RefineLevel a) {
  extern __shared__ __align__(16) unsigned char s_raw[];
  WarpSmem<D>& sm = reinterpret_cast<WarpSmem<D>*>(s_raw)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  warp_smem_init<D>(sm, lane);
  uint32_t phase = 0;
  const int64_t n = launch_count(a.n_blocks, a.n_dev, a.err);
  constexpr int NC = D == 3 ? 64 : 16;
  WarpCounters wc;
  // work in batches of a.batch consecutive blocks: one atomic and one coalesced
  // load of the batch's coordinates and geometry ids per batch
  const int batch = a.batch > 0 ? (a.batch < kMaxBatch ? a.batch : kMaxBatch) : 1;
  for (;;) {
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(a.work, (unsigned)batch);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= n) break;
    int cv = 0;
    uint32_t gv = 0;
    if (lane < batch * D && (int64_t)base + lane / D < n) cv = a.blocks[(int64_t)base * D + lane];
    if (a.gid && lane < batch && (int64_t)base + lane < n) gv = a.gid[base + lane];
  for (int q = 0; q < batch; ++q) {
    const unsigned blk = base + (unsigned)q;
    if (blk >= n) break;
    int b[3] = {0, 0, 0};
#pragma unroll
    for (int c = 0; c < D; ++c) b[c] = __shfl_sync(0xffffffffu, cv, q * D + c);
    const uint32_t gid = __shfl_sync(0xffffffffu, gv, q);
    const GeomParams& P = a.table ? a.table[gid] : a.g0;
    // per-cell face counts and survivor records only where the block's geometry ends here
    const bool fin = a.blockcnt && a.level == P.n_levels - 1;
    if (a.skip_mark_only && ((P.face_levels >> a.level) & 1u)) continue;  // marked face by face
    uint32_t cnt0 = 0, cnt1 = 0;
    bool h0 = false, h1 = false;
    if (fin) {
      uint32_t K = 0;  // records of this block (warp-uniform); past kRecCap into the warp's spill area
      walk_block<D, PRED, false>(a, P, gid, b, sm, phase, lane, wc, h0, h1, [&](uint32_t f, bool r0, bool r1) {
        cnt0 += r0 ? 1u : 0u;
        cnt1 += r1 ? 1u : 0u;
        if (a.recs) {
          const uint64_t cm = (uint64_t)__ballot_sync(0xffffffffu, r0) |
                              ((uint64_t)__ballot_sync(0xffffffffu, r1) << 32);
          if (cm) {
            if (lane == 0) {
              if (K < (uint32_t)kRecCap) {
                sm.rf[K] = f;
                sm.rm[K] = cm;
              } else if (a.spill && K < (uint32_t)(kRecCap + kSpillCap)) {
                spill_record(a.spill, K - kRecCap, f, cm);
              }
            }
            ++K;
          }
        }
      });
      if (a.recs) {
        if (K > (uint32_t)kRecCap) wc.big += 1;
        store_records<D>(a, sm, K, blk, lane);
      }
    } else {
      walk_block<D, PRED, true>(a, P, gid, b, sm, phase, lane, wc, h0, h1, [](uint32_t, bool, bool) {});
      cnt0 = h0 ? 1u : 0u;
      cnt1 = h1 ? 1u : 0u;
    }
    const uint64_t mask = (uint64_t)__ballot_sync(0xffffffffu, cnt0 > 0) |
                          ((uint64_t)__ballot_sync(0xffffffffu, cnt1 > 0) << 32);
    const uint64_t m = D == 3 ? mask : (mask & 0xffffull);
    if (lane == 0) {
      a.mask[blk] = m;
      a.flag[blk] = m != 0 ? 1 : 0;
    }
    if (a.blockcnt) {
      if (fin && a.cellcnt) {
        if (cnt0 > 0xffffu || cnt1 > 0xffffu) atomicOr(a.err, ERR_OVERFLOW);
        if (lane < NC) a.cellcnt[(int64_t)blk * NC + lane] = (uint16_t)min(cnt0, 0xffffu);
        if (D == 3) a.cellcnt[(int64_t)blk * NC + 32 + lane] = (uint16_t)min(cnt1, 0xffffu);
      }
      uint32_t pairs = fin ? cnt0 + cnt1 : 0u;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
      if (lane == 0) a.blockcnt[blk] = fin ? ((uint64_t)pairs | ((uint64_t)__popcll(m) << 32)) : 0ull;
    }
  }
  }
  // flush warp counters
  unsigned long long v[5] = {wc.fb, wc.band, wc.cand, wc.surv, wc.big};
#pragma unroll
  for (int i = 0; i < 5; ++i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  }
  if (lane == 0) {
    if (v[0]) atomicAdd(&a.counters[CNT_FALLBACK], v[0]);
    if (v[1]) atomicAdd(&a.counters[CNT_BAND], v[1]);
    atomicAdd(&a.counters[CNT_CANDIDATES], v[2]);       // per-lane counts
    atomicAdd(&a.counters[CNT_SURVIVORS], v[3] / 32);   // every lane counted the same survivors
    if (v[4]) atomicAdd(&a.counters[CNT_BIG_BLOCKS], v[4] / 32);
  }
}

// ---------------------------------------------------------------------------
// Refinement by parent groups (3D box predicate, levels below the roots).
//
// Every block of such a level is one of the 8 children of a marked parent,
// and the children of a parent are consecutive (slot order).  One warp takes a
// parent's 8 children together: it walks the bins of the parent box inflated
// by d_L once (the union of the children's query boxes), deduplicates, and
// culls each candidate against the whole inflated parent box; every survivor
// is then culled against each child's box (lane-parallel, certified, all 13
// axes), and only the remaining (face, child) pairs run the cell tests.  The
// bins are walked once per 8 children instead of once per child.
//
// The frame is the parent's corner (= child 0's corner); the cell thresholds
// of a survivor hold for all 512 cells of the group (its error bound takes
// the group's extent, 8 cells, as the bound on the cell-centre offsets).  The
// decisions are the per-block walk's (certified FP32 or the same FP64
// resolution), so the masks, counts and records are identical.
// ---------------------------------------------------------------------------
constexpr int kGroupPool = 24;  // survivor records of a group staged in shared memory (more: spill area)

struct GroupSmem {
  Surv<3> surv[32];
  Entry3 buf[2][32];
  uint64_t bar[2];
  SurvRec pool[kGroupPool];  // face, child (pad), cell mask
  uint16_t cnt[8][64];       // per child and cell: faces that meet the cell (finest level)
  uint8_t sidx[32];          // lanes of the chunk's survivors, in lane order
};

// Child j of the group may meet the face: no axis certifiably separates the
// projections of its cell centres (a box of half-width 1.5 h around the child
// centre cj) from the face's cell-level interval.  The widening by
// (t.z - t.x) = 2 eps absorbs the rounding of the child-centre projection and
// of the additions, so a culled child has no cell that meets the face.
__device__ __forceinline__ bool child_may_meet(const Surv<3>& S, const float* cj, float h15) {
  const float4 q0 = S.en[0], q1 = S.en[1], q2 = S.en[2];
  auto sep = [&](float x, float A1, const float4& t) {
    const float w = fmaf(h15, A1, t.z - t.x);
    return (x + w < t.x) | (x - w > t.y);
  };
  bool out = sep(cj[0], 1.f, S.t[0]) | sep(cj[1], 1.f, S.t[1]) | sep(cj[2], 1.f, S.t[2]);
  out |= sep(fmaf(cj[2], q2.w, fmaf(cj[1], q2.z, cj[0] * q2.y)), fabsf(q2.y) + fabsf(q2.z) + fabsf(q2.w), S.t[3]);
  const float e[3][3] = {{q0.x, q0.y, q0.z}, {q0.w, q1.x, q1.y}, {q1.z, q1.w, q2.x}};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float ex = e[k][0], ey = e[k][1], ez = e[k][2];
    out |= sep(fmaf(cj[2], ey, -cj[1] * ez), fabsf(ey) + fabsf(ez), S.t[4 + 3 * k]);
    out |= sep(fmaf(cj[0], ez, -cj[2] * ex), fabsf(ex) + fabsf(ez), S.t[5 + 3 * k]);
    out |= sep(fmaf(cj[1], ex, -cj[0] * ey), fabsf(ex) + fabsf(ey), S.t[6 + 3 * k]);
  }
  return !out;
}

// Per-warp counters of the group kernel (32-bit: a warp's counts stay far below 2^32).
struct GroupCounters {
  uint32_t fb = 0, band = 0, cand = 0, surv = 0, big = 0;
};

// FP64 decision of one (cell, face) pair of a group (the per-block walk's resolution).
__device__ __noinline__ bool resolve_group(const RefineLevel& a, uint32_t gid, uint32_t face, const int* b,
                                           int cell_local, GroupCounters& wc) {
  unsigned long long fb = 0, band = 0;
  const bool r = resolve_fp64<3>(a, gid, face, b, cell_local, &fb, &band);
  wc.fb += (uint32_t)fb;
  wc.band += (uint32_t)band;
  return r;
}

// One parent group: walk, culls and cell tests.  kMark: only the masks are
// wanted (the walk ends once every cell of the 8 children is marked); else the
// per-cell counts and the survivor records of the finest level are kept.
// hb0 / hb1: bit j = the lane's cell `lane` / `lane + 32` of child j is adjacent.
template <bool kMark>
__device__ __forceinline__ void walk_group(const RefineLevel& a, const GeomParams& P, uint32_t gid, const int* c0,
                                           GroupSmem& sm, uint32_t& phase, int lane, GroupCounters& wc,
                                           uint32_t& hb0, uint32_t& hb1, uint32_t& K, SurvRec* spill) {
  const FastGeom g = fast_geom(P, a.level);
  const float hf = g.h_hi;
  BlockFrame<3> F;
  int qlo[3], qhi[3];
  float O = 8.0f * hf;
  float shift[3];
  const int Bn = P.B;
  const float margin = 1e-6f * (float)Bn + 1e-3f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float lo;
    df_position(P.org_hi[c], P.org_lo[c], (float)(4 * c0[c]), g.h_hi, g.h_lo, F.Xb[c], lo);
    shift[c] = lo;
    F.cB[c] = fmaf(4.0f, g.h_hi, lo);
    O = fmaxf(O, 8.0f * hf + 2.0f * fabsf(lo));
    const float k0 = (float)(4 * c0[c]);
    const float xlo = fmaf(k0, g.h_hi, fmaf(k0, g.h_lo, -g.d));
    const float xhi = fmaf(k0 + 8.0f, g.h_hi, fmaf(k0 + 8.0f, g.h_lo, g.d));
    const float tlo = floorf(xlo * P.scale32[c] - margin);
    const float thi = floorf(xhi * P.scale32[c] + margin);
    qlo[c] = tlo < 0.f ? 0 : (tlo > (float)(Bn - 1) ? Bn - 1 : (int)tlo);
    qhi[c] = thi < 0.f ? 0 : (thi > (float)(Bn - 1) ? Bn - 1 : (int)thi);
  }
  F.h = hf;
  F.r = fmaf(0.5f, hf, g.d);
  F.rb = fmaf(4.0f, hf, g.d);  // the union of the 512 inflated cells: the parent box inflated by d
  F.O = O;
  const float h15 = 1.5f * hf;
  uint32_t full = 0;  // children whose 64 cells are all marked (kMark)
  const int64_t B = Bn;
  const Entry3* payload = static_cast<const Entry3*>(a.payload);
  const int nx = qhi[0] - qlo[0] + 1, ny = qhi[1] - qlo[1] + 1;
  const int nrows = ny * (qhi[2] - qlo[2] + 1);
  for (int rg = 0; rg < nrows; rg += 32) {
    uint32_t rs = 0, rn = 0;
    const int ri = rg + lane;
    if (ri < nrows) {
      const int y = qlo[1] + ri % ny, z = qlo[2] + ri / ny;
      const int64_t b0 = P.bin_base + qlo[0] + B * (y + B * (int64_t)z);
      rs = a.offsets[b0];
      rn = a.offsets[b0 + nx] - rs;
    }
    const uint32_t incl = warp_inclusive_scan<uint32_t>(rn);
    const uint32_t T = __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t rv = incl - rn;
    const uint32_t nch = (T + 31u) / 32u;
    if (nch == 0) continue;
    int cb = 0;
    issue_chunk<Entry3>(payload, rs, rn, rv, 0u, T, sm.buf[0], &sm.bar[0], lane);
    for (uint32_t c = 0; c < nch; ++c) {
      const int nb = cb ^ 1;
      const bool more = c + 1 < nch;
      if (more) issue_chunk<Entry3>(payload, rs, rn, rv, c + 1, T, sm.buf[nb], &sm.bar[nb], lane);
      mbar_wait_bounded(&sm.bar[cb], (phase >> cb) & 1u, a.err);
      phase ^= 1u << cb;
      const uint32_t n = T - 32u * c < 32u ? T - 32u * c : 32u;
      bool surv = false;
      if ((uint32_t)lane < n) {
        const Entry3& ent = sm.buf[cb][lane];
        const uint32_t id = ent.id;
        // visit a face only in the first bin of its range inside the query box
        const bool canon = (((id >> 29) & 1u) || (int)ent.bin[0] == qlo[0]) &&
                           (((id >> 30) & 1u) || (int)ent.bin[1] == qlo[1]) &&
                           (((id >> 31) & 1u) || (int)ent.bin[2] == qlo[2]);
        if (canon) {
          wc.cand++;
          const float nh[3] = {ent.n[0], ent.n[1], ent.n[2]};
          float V[9];
#pragma unroll
          for (int j = 0; j < 9; ++j) V[j] = ent.v[j];
          surv = setup_face<3>(V, nh, F, sm.surv[lane]);
          sm.surv[lane].face = id & kIdMask;
        }
      }
      unsigned m = __ballot_sync(0xffffffffu, surv);
      if (surv) sm.sidx[__popc(m & ((1u << lane) - 1u))] = (uint8_t)lane;
      __syncwarp();
      // child culls: lane = (survivor, child) pair
      const int ns = __popc(m);
      for (int base = 0; base < 8 * ns; base += 32) {
        const int p = base + lane;
        bool keep = false;
        int s = 0;
        if (p < 8 * ns) {
          s = sm.sidx[p >> 3];
          const int j = p & 7;
          float cj[3];
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const float l = (float)(4 * ((j >> q) & 1) + 2);
            cj[q] = fmaf(l, g.h_hi, fmaf(l, g.h_lo, shift[q]));
          }
          keep = child_may_meet(sm.surv[s], cj, h15);
        }
        const unsigned kb = __ballot_sync(0xffffffffu, keep);
        if ((lane & 7) == 0 && p < 8 * ns) sm.surv[s].pad[0] = (kb >> (lane & 24)) & 0xffu;
      }
      __syncwarp();
      while (m) {
        const int s = __ffs(m) - 1;
        m &= m - 1;
        const Surv<3>& S = sm.surv[s];
        uint32_t cm = S.pad[0];
        if (kMark) cm &= ~full;
        wc.surv += __popc(cm);
        while (cm) {
          const int j = __ffs(cm) - 1;
          cm &= cm - 1;
          // read the survivor's thresholds from shared memory per child (not held in registers
          // across the children, which spills)
          asm volatile("" ::: "memory");
          const int cx = j & 1, cy = (j >> 1) & 1, cz = (j >> 2) & 1;
          // the lane's cells `lane` and `lane + 32` of child j, centres in the frame
          float o0[3], o1[3];
          {
            const int d0[3] = {4 * cx, 4 * cy, 4 * cz};
#pragma unroll
            for (int q = 0; q < 3; ++q) {
              const float a0 = (float)(d0[q] + ((lane >> (2 * q)) & 3)) + 0.5f;
              const float a1 = (float)(d0[q] + (((lane + 32) >> (2 * q)) & 3)) + 0.5f;
              o0[q] = fmaf(a0, g.h_hi, fmaf(a0, g.h_lo, shift[q]));
              o1[q] = fmaf(a1, g.h_hi, fmaf(a1, g.h_lo, shift[q]));
            }
          }
          const bool m0 = kMark && ((hb0 >> j) & 1u), m1 = kMark && ((hb1 >> j) & 1u);
          int t0 = 0, t1 = 0;
          cell_test2<3>(S, o0, o1, t0, t1);
          const int bj[3] = {c0[0] + cx, c0[1] + cy, c0[2] + cz};  // child j's block coordinates
          bool r0 = false, r1 = false;
          if (!m0) {
            if (t0 == 2) t0 = resolve_group(a, gid, S.face, bj, lane, wc) ? 1 : 0;
            r0 = t0 != 0;
          }
          if (!m1) {
            if (t1 == 2) t1 = resolve_group(a, gid, S.face, bj, lane + 32, wc) ? 1 : 0;
            r1 = t1 != 0;
          }
          hb0 |= (uint32_t)r0 << j;
          hb1 |= (uint32_t)r1 << j;
          if constexpr (kMark) {
            if (__all_sync(0xffffffffu, ((hb0 & hb1) >> j) & 1u)) full |= 1u << j;
          } else {
            const uint32_t n0 = sm.cnt[j][lane], n1 = sm.cnt[j][lane + 32];
            if ((r0 && n0 == 0xffffu) || (r1 && n1 == 0xffffu)) atomicOr(a.err, ERR_OVERFLOW);
            sm.cnt[j][lane] = (uint16_t)min(n0 + (uint32_t)r0, 0xffffu);
            sm.cnt[j][lane + 32] = (uint16_t)min(n1 + (uint32_t)r1, 0xffffu);
            if (a.recs) {
              const uint64_t cells = (uint64_t)__ballot_sync(0xffffffffu, r0) |
                                     ((uint64_t)__ballot_sync(0xffffffffu, r1) << 32);
              if (cells) {
                if (lane == 0) {
                  SurvRec r;
                  r.face = S.face;
                  r.pad = (uint32_t)j;
                  r.cells = cells;
                  if (K < (uint32_t)kGroupPool)
                    sm.pool[K] = r;
                  else if (spill && K < (uint32_t)(kGroupPool + kSpillCap))
                    spill[K - kGroupPool] = r;
                }
                ++K;
              }
            }
          }
        }
      }
      __syncwarp();
      if (kMark && full == 0xffu) {
        if (more) {
          mbar_wait_bounded(&sm.bar[nb], (phase >> nb) & 1u, a.err);  // the copy already in flight
          phase ^= 1u << nb;
          __syncwarp();
        }
        return;
      }
      cb = nb;
    }
  }
}

// The group's K records into a contiguous range of the level's record array,
// grouped by child (each child's records in the order they were found), and
// every child's descriptor: offset << 16 | count, 0 for none, ~0 when the
// records are incomplete (the adjacency pass then walks the block again).
__device__ __noinline__ void store_group_records(const RefineLevel& a, GroupSmem& sm, const SurvRec* spill,
                                                  uint32_t K, unsigned blk0, int lane) {
  __syncwarp();  // the staged and spilled records are visible to the whole warp
  const uint32_t kmax = (uint32_t)kGroupPool + (spill ? (uint32_t)kSpillCap : 0u);
  uint64_t base = ~0ull;
  if (K > 0 && K <= kmax) {
    if (lane == 0) base = atomicAdd(reinterpret_cast<unsigned long long*>(a.rec_count), (unsigned long long)K);
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((int64_t)(base + K) > a.cap_recs) base = ~0ull;
  }
  if (K == 0 || base == ~0ull) {
    if (lane < 8) a.rec_desc[blk0 + lane] = K == 0 ? 0ull : ~0ull;
    __syncwarp();
    return;
  }
  auto rec = [&](uint32_t i) { return i < (uint32_t)kGroupPool ? sm.pool[i] : spill[i - kGroupPool]; };
  // records per child, then the child's first position
  uint32_t cntj = 0;  // lane j < 8: records of child j
  for (uint32_t i0 = 0; i0 < K; i0 += 32) {
    const uint32_t i = i0 + (uint32_t)lane;
    const uint32_t j = i < K ? rec(i).pad : 8u;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint32_t n = __popc(__ballot_sync(0xffffffffu, j == (uint32_t)q));
      if (lane == q) cntj += n;
    }
  }
  const uint32_t incl = warp_inclusive_scan<uint32_t>(lane < 8 ? cntj : 0u);
  const uint32_t first = incl - (lane < 8 ? cntj : 0u);
  if (lane < 8) a.rec_desc[blk0 + lane] = cntj == 0 ? 0ull : ((base + first) << 16) | cntj;
  uint32_t run = first;  // lane j < 8: next position of child j
  for (uint32_t i0 = 0; i0 < K; i0 += 32) {
    const uint32_t i = i0 + (uint32_t)lane;
    SurvRec r;
    r.pad = 8u;
    if (i < K) r = rec(i);
    uint32_t pos = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const unsigned bq = __ballot_sync(0xffffffffu, r.pad == (uint32_t)q);
      const uint32_t rq = __shfl_sync(0xffffffffu, run, q);
      if (r.pad == (uint32_t)q) pos = rq + __popc(bq & ((1u << lane) - 1u));
      if (lane == q) run += __popc(bq);
    }
    if (i < K) {
      SurvRec o;
      o.face = r.face;
      o.pad = 0u;
      o.cells = r.cells;
      a.recs[base + pos] = o;
    }
  }
  __syncwarp();
}

constexpr int kGroupWarps = 4;  // warps per CTA of k_refine_groups (4 CTAs per SM by registers and shared memory)

__global__ void __launch_bounds__(kGroupWarps * 32, 4) k_refine_groups(RefineLevel a) {
  extern __shared__ __align__(16) unsigned char s_raw[];
  GroupSmem& sm = reinterpret_cast<GroupSmem*>(s_raw)[threadIdx.x >> 5];
  const int lane = threadIdx.x & 31;
  if (lane == 0) {
    mbar_init(&sm.bar[0], 1);
    mbar_init(&sm.bar[1], 1);
    mbar_fence_init();
  }
  __syncwarp();
  uint32_t phase = 0;
  const int64_t n = launch_count(a.n_blocks, a.n_dev, a.err);
  if ((n & 7) != 0 && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(a.err, ERR_BADINDEX);  // children in eights
  const int64_t ng = n >> 3;
  SurvRec* spill = a.spill ? warp_spill(a.spill) : nullptr;
  GroupCounters wc;
  for (;;) {
    unsigned gi = 0;
    if (lane == 0) gi = atomicAdd(a.work, 1u);
    gi = __shfl_sync(0xffffffffu, gi, 0);
    if ((int64_t)gi >= ng) break;
    const unsigned blk0 = gi * 8u;
    int cv = lane < 3 ? a.blocks[(int64_t)blk0 * 3 + lane] : 0;
    int c0[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) c0[c] = __shfl_sync(0xffffffffu, cv, c);
    const uint32_t gid = a.gid ? a.gid[blk0] : 0u;
    const GeomParams& P = a.table ? a.table[gid] : a.g0;
    if (a.skip_mark_only && ((P.face_levels >> a.level) & 1u)) continue;  // marked face by face
    const bool fin = a.blockcnt && a.level == P.n_levels - 1;
    uint32_t hb0 = 0, hb1 = 0, K = 0;
    if (fin) {
      reinterpret_cast<uint4*>(sm.cnt)[lane] = make_uint4(0u, 0u, 0u, 0u);
      reinterpret_cast<uint4*>(sm.cnt)[lane + 32] = make_uint4(0u, 0u, 0u, 0u);
      __syncwarp();
      walk_group<false>(a, P, gid, c0, sm, phase, lane, wc, hb0, hb1, K, spill);
      if (a.recs) {
        if (K > (uint32_t)kGroupPool) wc.big += 1;
        store_group_records(a, sm, spill, K, blk0, lane);
      }
    } else {
      walk_group<true>(a, P, gid, c0, sm, phase, lane, wc, hb0, hb1, K, spill);
    }
    __syncwarp();
#pragma unroll 1
    for (int j = 0; j < 8; ++j) {
      const unsigned blk = blk0 + (unsigned)j;
      const uint64_t m = (uint64_t)__ballot_sync(0xffffffffu, (hb0 >> j) & 1u) |
                         ((uint64_t)__ballot_sync(0xffffffffu, (hb1 >> j) & 1u) << 32);
      if (lane == 0) {
        a.mask[blk] = m;
        a.flag[blk] = m != 0 ? 1 : 0;
      }
      if (a.blockcnt) {
        uint32_t pairs = 0;
        if (fin) {
          const uint32_t n0 = sm.cnt[j][lane], n1 = sm.cnt[j][lane + 32];
          if (a.cellcnt) {
            a.cellcnt[(int64_t)blk * 64 + lane] = (uint16_t)n0;
            a.cellcnt[(int64_t)blk * 64 + 32 + lane] = (uint16_t)n1;
          }
          pairs = n0 + n1;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
        }
        if (lane == 0) a.blockcnt[blk] = fin ? ((uint64_t)pairs | ((uint64_t)__popcll(m) << 32)) : 0ull;
      }
    }
  }
  // fb, band and cand are per-lane counts; surv and big, warp-uniform ones
  unsigned long long v[5] = {wc.fb, wc.band, wc.cand, wc.surv, wc.big};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  }
  if (lane == 0) {
    if (v[0]) atomicAdd(&a.counters[CNT_FALLBACK], v[0]);
    if (v[1]) atomicAdd(&a.counters[CNT_BAND], v[1]);
    atomicAdd(&a.counters[CNT_CANDIDATES], v[2]);
    atomicAdd(&a.counters[CNT_SURVIVORS], v[3]);  // (face, child) pairs that ran the cell tests
    if (v[4]) atomicAdd(&a.counters[CNT_BIG_BLOCKS], v[4]);
  }
}

// Ascending sort of P keys in shared memory (P a power of two; pad the tail
// with ~0), with a 64-bit payload per key when pay is given, by the whole warp:
// the bitonic network, one compare-exchange per lane and pair of each stage.
__device__ __noinline__ void warp_bitonic(uint32_t* k, uint64_t* pay, uint32_t P, int lane) {
  for (uint32_t s = 2; s <= P; s <<= 1)
    for (uint32_t j = s >> 1; j > 0; j >>= 1) {
      for (uint32_t i = (uint32_t)lane; i < P; i += 32) {
        const uint32_t l = i ^ j;
        if (l > i) {
          const bool up = (i & s) == 0;
          const uint32_t x = k[i], y = k[l];
          if (up ? x > y : x < y) {
            k[i] = y;
            k[l] = x;
            if (pay) {
              const uint64_t t = pay[i];
              pay[i] = pay[l];
              pay[l] = t;
            }
          }
        }
      }
      __syncwarp();
    }
}

// Ascending face ids in each of a block's cell lists (cell c's count and offset
// held by lane c, or lane c - 32 in n1 / off1): the warp sorts one list at a time
// in the shared memory at sf (room for cap keys); a longer list is sorted in
// place by one lane.  Out of line: only blocks walked again need it.
__device__ __noinline__ void sort_cell_lists(uint32_t* adj_ids, int NC, uint32_t n0, uint32_t n1, uint64_t off0,
                                             uint64_t off1, uint32_t* sf, uint32_t cap, int lane) {
  for (int c = 0; c < NC; ++c) {
    const uint32_t cnt = c < 32 ? __shfl_sync(0xffffffffu, n0, c) : __shfl_sync(0xffffffffu, n1, c - 32);
    const uint64_t off = c < 32 ? __shfl_sync(0xffffffffu, off0, c) : __shfl_sync(0xffffffffu, off1, c - 32);
    if (cnt <= 1) continue;
    uint32_t* L = adj_ids + off;
    if (cnt <= cap) {
      uint32_t P = 32;
      while (P < cnt) P <<= 1;
      for (uint32_t i = lane; i < P; i += 32) sf[i] = i < cnt ? L[i] : 0xffffffffu;
      __syncwarp();
      warp_bitonic(sf, nullptr, P, lane);
      for (uint32_t i = lane; i < cnt; i += 32) L[i] = sf[i];
      __syncwarp();
    } else if (lane == 0) {
      for (uint32_t i = 1; i < cnt; ++i) {
        const uint32_t v = L[i];
        uint32_t k = i;
        while (k > 0 && L[k - 1] > v) {
          L[k] = L[k - 1];
          --k;
        }
        L[k] = v;
      }
    }
    __syncwarp();
  }
}

// A block's K survivor records sorted by face id into shared memory at sf (the
// face ids; the cell masks follow them, returned), by the whole warp.
__device__ __noinline__ const uint64_t* sort_records(const SurvRec* recs, uint32_t K, uint32_t* sf, int lane) {
  uint32_t P = 64;
  while (P < K) P <<= 1;
  uint64_t* sk = reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(sf) + 4 * P);
  for (uint32_t i = lane; i < P; i += 32) {
    if (i < K) {
      const SurvRec r = recs[i];
      sf[i] = r.face;
      sk[i] = r.cells;
    } else {
      sf[i] = 0xffffffffu;
      sk[i] = 0ull;
    }
  }
  __syncwarp();
  warp_bitonic(sf, sk, P, lane);
  return sk;
}

// Shared memory of a warp that a sort may use: the survivor data and the entry
// buffers (not the mbarriers that follow them).
template <int D>
__host__ __device__ constexpr uint32_t sort_region_bytes() {
  return (uint32_t)(sizeof(Surv<D>) * 32 + sizeof(typename EntryT<D>::type) * 64);
}
// Largest power of two P with P keys (and P payloads of 8 bytes) in the region.
__host__ __device__ constexpr uint32_t pow2_floor(uint32_t x) {
  uint32_t p = 1;
  while (p * 2 <= x) p *= 2;
  return p;
}

// Emit the adjacent-face lists of the blocks whose geometry ends at this
// level, in two passes.  MODE 0 takes every block: it writes the block's rows
// (adjacent cells and their list offsets, from the block-level scan and the
// per-cell counts) and, when the refine pass kept at most kRecCap survivor
// records, ranks them by face id and lists each cell's faces in that order; it
// needs only a little shared memory, so many warps stay resident.  Other blocks
// go to a list that MODE 1 takes, with the walk's shared memory: more records
// are sorted there, and blocks without records are walked again (the same
// decisions as k_refine) and their lists sorted.  Rows and pairs continue after
// the running totals of earlier levels.
template <int D, int PRED, int MODE>
__device__ __forceinline__ void emit_block(const EmitArgs& a, unsigned blk, uint32_t gid, WarpSmem<D>& sm,
                                           uint32_t& phase, WarpCounters& wc, uint64_t* rm, uint32_t* rf,
                                           int lane, uint64_t run_cells, uint64_t run_pairs,
                                           const uint64_t* pre = nullptr) {
  // pre (MODE 0): the block's base and record descriptor, loaded with its batch
  constexpr int NC = D == 3 ? 64 : 16;
    const GeomParams& P = a.lv.table ? a.lv.table[gid] : a.lv.g0;
    if (a.lv.level != P.n_levels - 1) return;
    int b[3] = {0, 0, 0};
#pragma unroll
    for (int c = 0; c < D; ++c) b[c] = a.lv.blocks[(int64_t)blk * D + c];
    const uint64_t base = pre ? pre[0] : a.block_base[blk];
    const uint64_t pair_base = run_pairs + (base & 0xffffffffull);
    const uint64_t cell_base = run_cells + (base >> 32);
    const uint32_t n0 = lane < NC ? a.lv.cellcnt[(int64_t)blk * NC + lane] : 0u;
    const uint32_t n1 = D == 3 ? (uint32_t)a.lv.cellcnt[(int64_t)blk * NC + 32 + lane] : 0u;
    // exclusive prefixes over cells in bit order (cells 0..31 then 32..63)
    const uint32_t i0 = warp_inclusive_scan<uint32_t>(n0);
    const uint32_t tot0 = __shfl_sync(0xffffffffu, i0, 31);
    const uint32_t i1 = warp_inclusive_scan<uint32_t>(n1);
    const uint64_t off0 = pair_base + i0 - n0;
    const uint64_t off1 = pair_base + tot0 + i1 - n1;
    const uint32_t a0 = n0 > 0, a1 = n1 > 0;
    const uint32_t j0 = warp_inclusive_scan<uint32_t>(a0);
    const uint32_t atot0 = __shfl_sync(0xffffffffu, j0, 31);
    const uint32_t j1 = warp_inclusive_scan<uint32_t>(a1);
    bool bad = (int64_t)(off1 + n1) > a.cap_pairs || (int64_t)(off0 + n0) > a.cap_pairs;
    if (MODE == 0 && a0) {
      const uint64_t row = cell_base + j0 - 1;
      if ((int64_t)row < a.cap_cells) {
        a.adj_cell[row] = blk * (uint32_t)NC + lane;
        a.adj_off[row] = (uint32_t)off0;
      } else {
        bad = true;
      }
    }
    if (MODE == 0 && a1) {
      const uint64_t row = cell_base + atot0 + j1 - 1;
      if ((int64_t)row < a.cap_cells) {
        a.adj_cell[row] = blk * (uint32_t)NC + 32 + lane;
        a.adj_off[row] = (uint32_t)off1;
      } else {
        bad = true;
      }
    }
    uint32_t c0 = 0, c1 = 0;
    const bool can0 = (int64_t)(off0 + n0) <= a.cap_pairs, can1 = (int64_t)(off1 + n1) <= a.cap_pairs;
    auto put = [&](bool r0, bool r1, uint32_t f) {
      if (r0) {
        if (c0 < n0 && can0)
          a.adj_ids[off0 + c0] = f;
        else
          bad = true;
        ++c0;
      }
      if constexpr (D == 3) {
        if (r1) {
          if (c1 < n1 && can1)
            a.adj_ids[off1 + c1] = f;
          else
            bad = true;
          ++c1;
        }
      }
    };
    const uint64_t desc = pre ? pre[1] : (a.lv.recs ? a.lv.rec_desc[blk] : ~0ull);
    constexpr uint32_t kSortRecs = pow2_floor(sort_region_bytes<D>() / 12);  // key + payload per record
    constexpr uint32_t kSortKeys = pow2_floor(sort_region_bytes<D>() / 4);
    if constexpr (MODE == 0) {
    if (desc != ~0ull && (uint32_t)(desc & 0xffffu) <= (uint32_t)kRecCap) {
      // the refine pass left this block's surviving faces with their cell masks:
      // rank them by face id, then every lane lists its cells' faces in that order
      const uint32_t K = (uint32_t)(desc & 0xffffu);
      const uint64_t r0 = desc >> 16;
      uint32_t f[2] = {0xffffffffu, 0xffffffffu};
      uint64_t cm[2] = {0ull, 0ull};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t i = (uint32_t)lane + 32u * h;
        if (i < K) {
          const SurvRec r = a.lv.recs[r0 + i];
          f[h] = r.face;
          cm[h] = r.cells;
        }
      }
      uint32_t rank[2] = {0u, 0u};
      for (uint32_t j = 0; j < K; ++j) {
        const uint32_t fj = __shfl_sync(0xffffffffu, j < 32 ? f[0] : f[1], (int)(j & 31u));
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint32_t i = (uint32_t)lane + 32u * h;
          rank[h] += (fj < f[h] || (fj == f[h] && j < i)) ? 1u : 0u;
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint32_t i = (uint32_t)lane + 32u * h;
        if (i < K) {
          rf[rank[h]] = f[h];
          rm[rank[h]] = cm[h];
        }
      }
      __syncwarp();
      for (uint32_t j = 0; j < K; ++j) {
        const uint64_t mj = rm[j];
        put(lane < NC && ((mj >> lane) & 1ull), D == 3 && ((mj >> (lane + 32)) & 1ull), rf[j]);
      }
      __syncwarp();
      if (bad || c0 != n0 || c1 != n1) atomicOr(a.lv.err, ERR_OVERFLOW);
      return;
    }
      // more records than staged in shared memory, or none kept: the second pass takes the block
      if (lane == 0) {
        const unsigned pos = atomicAdd(a.defer_n, 1u);
        if ((int64_t)pos < a.defer_cap)
          a.defer[pos] = blk;
        else
          atomicOr(a.lv.err, ERR_OVERFLOW);
      }
      return;
    } else {
    if (desc != ~0ull && (uint32_t)(desc & 0xffffu) > (uint32_t)kRecCap &&
        (uint32_t)(desc & 0xffffu) <= kSortRecs) {
      // many records: sort them by face id in shared memory, then list the cells' faces in that order
      const uint32_t K = (uint32_t)(desc & 0xffffu);
      const uint64_t r0 = desc >> 16;
      uint32_t* sf = reinterpret_cast<uint32_t*>(&sm);
      const uint64_t* sk = sort_records(a.lv.recs + r0, K, sf, lane);
      for (uint32_t j = 0; j < K; ++j) {
        const uint64_t mj = sk[j];
        put(lane < NC && ((mj >> lane) & 1ull), D == 3 && ((mj >> (lane + 32)) & 1ull), sf[j]);
      }
      __syncwarp();
      if (bad || c0 != n0 || c1 != n1) atomicOr(a.lv.err, ERR_OVERFLOW);
      return;
    }
    bool h0 = false, h1 = false;
    walk_block<D, PRED, false>(a.lv, P, gid, b, sm, phase, lane, wc, h0, h1,
                         [&](uint32_t fc, bool r0, bool r1) { put(r0, r1, fc); });
    if (bad || c0 != n0 || c1 != n1) atomicOr(a.lv.err, ERR_OVERFLOW);
    if (!__all_sync(0xffffffffu, can0 && can1)) return;  // lists beyond the capacity (reported)
    // ascending face ids per cell
    sort_cell_lists(a.adj_ids, NC, n0, n1, off0, off1, reinterpret_cast<uint32_t*>(&sm), kSortKeys, lane);
    }
}

template <int D, int PRED, int MODE>
__global__ void __launch_bounds__(256) k_adjacency(EmitArgs a) {
  constexpr int kW = 8;  // warps per CTA at most
  __shared__ uint64_t s_rm[MODE == 0 ? kW : 1][kRecCap];
  __shared__ uint32_t s_rf[MODE == 0 ? kW : 1][kRecCap];
  extern __shared__ __align__(16) unsigned char s_raw[];  // MODE 1: the walk's per-warp memory
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  WarpSmem<D>& sm = reinterpret_cast<WarpSmem<D>*>(s_raw)[MODE == 0 ? 0 : wid];
  uint32_t phase = 0;
  if constexpr (MODE == 1) warp_smem_init<D>(sm, lane);
  uint64_t* rm = s_rm[MODE == 0 ? wid : 0];
  uint32_t* rf = s_rf[MODE == 0 ? wid : 0];
  const uint64_t run_cells = a.run ? a.run[0] : 0ull, run_pairs = a.run ? a.run[1] : 0ull;
  WarpCounters wc;
  if constexpr (MODE == 0) {
    const int64_t n = launch_count(a.lv.n_blocks, a.lv.n_dev, a.lv.err);
    // 32 blocks per atomic: each lane reads one block's mask, the warp then takes
    // the marked blocks of the group one after another
    for (;;) {
      unsigned base = 0;
      if (lane == 0) base = atomicAdd(a.lv.work, 32u);
      base = __shfl_sync(0xffffffffu, base, 0);
      if (base >= n) break;
      const bool in_range = (int64_t)base + lane < n;
      const uint64_t my_mask = in_range ? a.lv.mask[base + lane] : 0ull;
      const uint32_t my_gid = in_range && a.lv.gid ? a.lv.gid[base + lane] : 0u;
      // the marked blocks' row bases and record descriptors, one coalesced load for the batch
      const bool marked = my_mask != 0;
      const uint64_t my_base = marked ? a.block_base[base + lane] : 0ull;
      const uint64_t my_desc = marked && a.lv.recs ? a.lv.rec_desc[base + lane] : ~0ull;
      unsigned todo = __ballot_sync(0xffffffffu, marked);
      while (todo) {
        const int q = __ffs(todo) - 1;
        todo &= todo - 1;
        const uint32_t gid = __shfl_sync(0xffffffffu, my_gid, q);
        const uint64_t pre[2] = {__shfl_sync(0xffffffffu, my_base, q), __shfl_sync(0xffffffffu, my_desc, q)};
        emit_block<D, PRED, MODE>(a, base + (unsigned)q, gid, sm, phase, wc, rm, rf, lane, run_cells, run_pairs,
                                  pre);
      }
    }
  } else {
    const int64_t nd = (int64_t)*a.defer_n;
    const int64_t n = nd < a.defer_cap ? nd : a.defer_cap;
    for (;;) {
      unsigned i = 0;
      if (lane == 0) i = atomicAdd(a.lv.work, 1u);
      i = __shfl_sync(0xffffffffu, i, 0);
      if ((int64_t)i >= n) break;
      const unsigned blk = a.defer[i];
      const uint32_t gid = a.lv.gid ? a.lv.gid[blk] : 0u;
      emit_block<D, PRED, MODE>(a, blk, gid, sm, phase, wc, rm, rf, lane, run_cells, run_pairs);
    }
  }
}

// Children of the marked blocks whose geometry continues below this level,
// canonical order, single pass with look-back over ticketed tiles.
constexpr int kChThreads = 256;
constexpr int kChItems = 4;

template <int D>
__global__ void __launch_bounds__(kChThreads) k_children(ChildrenArgs a, uint64_t* state, unsigned* ticket) {
  __shared__ unsigned s_tile;
  __shared__ uint32_t s_warp[kChThreads / 32];
  __shared__ uint64_t s_prefix;
  const int64_t n = launch_count(a.n, a.n_dev, a.err);
  const int64_t ntiles = (n + (int64_t)kChThreads * kChItems - 1) / ((int64_t)kChThreads * kChItems);
  constexpr int NCH = D == 3 ? 8 : 4;
  if (ntiles == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.total = 0;
    return;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const long long tile = s_tile;
    if (tile >= ntiles) break;
    const int64_t base = tile * (int64_t)kChThreads * kChItems + (int64_t)threadIdx.x * kChItems;
    uint32_t fl[kChItems];
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < kChItems; ++i) {
      const int64_t j = base + i;
      bool emit = false;
      if (j < n && (a.flag ? a.flag[j] != 0 : a.mask[j] != 0)) {
        const GeomParams P = geom_row(a.g0, a.table, a.gid, j);
        emit = a.level < P.n_levels - 1;
      }
      fl[i] = emit ? 1u : 0u;
      sum += fl[i];
    }
    const uint32_t incl = warp_inclusive_scan<uint32_t>(sum);
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      uint32_t w = lane < kChThreads / 32 ? s_warp[lane] : 0u;
      w = warp_inclusive_scan<uint32_t>(w);
      if (lane < kChThreads / 32) s_warp[lane] = w;
    }
    __syncthreads();
    const uint32_t wex = wid > 0 ? s_warp[wid - 1] : 0u;
    if (wid == 0) {
      const uint64_t agg = s_warp[kChThreads / 32 - 1];
      const uint64_t pre = lookback_warp(state, tile, agg, a.err);
      if (lane == 0) {
        s_prefix = pre;
        if (tile == ntiles - 1) {
          const uint64_t tot = (pre + agg) * NCH;
          *a.total = tot;
          if ((int64_t)tot > a.cap_out) atomicOr(a.err, ERR_OVERFLOW);
        }
      }
    }
    __syncthreads();
    uint64_t k = s_prefix + wex + incl - sum;
    if (a.first_child) {
      uint64_t kk = k;
#pragma unroll
      for (int i = 0; i < kChItems; ++i) {
        const int64_t j = base + i;
        if (j < n) {
          const uint64_t o = kk * NCH;
          if (fl[i] && o >= 0x7fffffffull) atomicOr(a.err, ERR_OVERFLOW);
          a.first_child[j] = fl[i] ? (int32_t)o : -1;
        }
        kk += fl[i];
      }
    }
#pragma unroll
    for (int i = 0; i < kChItems; ++i) {
      if (fl[i]) {
        const int64_t p = base + i;
        int bc[3] = {0, 0, 0};
#pragma unroll
        for (int c = 0; c < D; ++c) bc[c] = a.blocks[p * D + c];
        const uint32_t g = a.gid ? a.gid[p] : 0u;
#pragma unroll
        for (int s = 0; s < NCH; ++s) {
          const int64_t o = (int64_t)k * NCH + s;
          if (o >= a.cap_out) break;
          a.child_blocks[o * D + 0] = 2 * bc[0] + (s & 1);
          a.child_blocks[o * D + 1] = 2 * bc[1] + ((s >> 1) & 1);
          if (D == 3) a.child_blocks[o * D + 2] = 2 * bc[2] + ((s >> 2) & 1);
          a.child_parent[o] = (int32_t)p;
          if (a.child_gid) a.child_gid[o] = g;
        }
        ++k;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Face-centric marking of a level whose masks are the only output (no
// adjacency lists): one warp per face tests the cells of the level whose test
// region can meet the face (the face's AABB widened by d, in cells) and ORs
// the hits into their blocks' masks.  Coarse levels are where this pays: a
// block there sees hundreds of faces, each of which the block walk tests
// against all of the block's cells, while a face covers only a few cells.
// The decisions are the block walk's: the same certified FP32 tests, in a
// frame at the lower corner of the face's cell range (the error bounds need
// only the frame's offset bounds P and O), and the same FP64 resolution.
// ---------------------------------------------------------------------------

// One cell's SAT test against a survivor: the projections of cell_test2.
template <int D>
__device__ __forceinline__ int cell_test1(const Surv<D>& S, const float* o) {
  bool sep = false, in = true;
  auto upd = [&](float x, const float4& t) {
    sep |= (x < t.x) | (x > t.y);
    in &= (x > t.z) & (x < t.w);
  };
  if constexpr (D == 3) {
#pragma unroll
    for (int ai = 0; ai < 3; ++ai) upd(o[ai], S.t[ai]);
    const float4 q0 = S.en[0], q1 = S.en[1], q2 = S.en[2];
    const float e[3][3] = {{q0.x, q0.y, q0.z}, {q0.w, q1.x, q1.y}, {q1.z, q1.w, q2.x}};
    upd(fmaf(o[2], q2.w, fmaf(o[1], q2.z, o[0] * q2.y)), S.t[3]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float ex = e[k][0], ey = e[k][1], ez = e[k][2];
      upd(fmaf(o[2], ey, -o[1] * ez), S.t[4 + 3 * k]);
      upd(fmaf(o[0], ez, -o[2] * ex), S.t[5 + 3 * k]);
      upd(fmaf(o[1], ex, -o[0] * ey), S.t[6 + 3 * k]);
    }
  } else {
    upd(o[0], S.t[0]);
    upd(o[1], S.t[1]);
    upd(fmaf(o[1], S.e[0], -o[0] * S.e[1]), S.t[2]);
  }
  return sep ? 0 : (in ? 1 : 2);
}

// setup_face without the block cull, lane-parallel: lane ai < 13 (2D: 3)
// computes axis ai with setup_face's arithmetic; lane 0 stores the edges.
template <int D>
__device__ __forceinline__ void setup_face_lanes(const float* V, const float* nh, const BlockFrame<D>& F, Surv<D>& S,
                                                 int lane) {
  constexpr int NA = D == 3 ? 13 : 3;
  float p[3][3];
  float P = 0.f;
#pragma unroll
  for (int k = 0; k < D; ++k)
#pragma unroll
    for (int c = 0; c < D; ++c) {
      p[k][c] = V[D * k + c] - F.Xb[c];
      P = fmaxf(P, fabsf(p[k][c]));
    }
  const float scale = kEpsK * kU32 * (P + F.O + F.r);
  if (lane < NA) {
    float ax = 0.f, ay = 0.f, az = 0.f;
    if constexpr (D == 3) {
      if (lane < 3) {
        ax = lane == 0 ? 1.f : 0.f;
        ay = lane == 1 ? 1.f : 0.f;
        az = lane == 2 ? 1.f : 0.f;
      } else if (lane == 3) {
        ax = nh[0];
        ay = nh[1];
        az = nh[2];
      } else {
        const int k = (lane - 4) / 3, i = (lane - 4) % 3;
        float ex = 0.f, ey = 0.f, ez = 0.f;
#pragma unroll
        for (int kk = 0; kk < 3; ++kk)
          if (kk == k) {
            const int kn = (kk + 1) % 3;
            ex = V[3 * kn + 0] - V[3 * kk + 0];
            ey = V[3 * kn + 1] - V[3 * kk + 1];
            ez = V[3 * kn + 2] - V[3 * kk + 2];
          }
        if (i == 0) {
          ax = 0.f;
          ay = -ez;
          az = ey;
        } else if (i == 1) {
          ax = ez;
          ay = 0.f;
          az = -ex;
        } else {
          ax = -ey;
          ay = ex;
          az = 0.f;
        }
      }
    } else {
      if (lane < 2) {
        ax = lane == 0 ? 1.f : 0.f;
        ay = lane == 1 ? 1.f : 0.f;
      } else {
        ax = -(V[3] - V[1]);
        ay = V[2] - V[0];
      }
    }
    const float A1 = fabsf(ax) + fabsf(ay) + fabsf(az);
    float4 t = make_float4(-INFINITY, INFINITY, -INFINITY, INFINITY);
    if (A1 != 0.0f) {
      float tmin = INFINITY, tmax = -INFINITY;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float s = D == 3 ? fmaf(p[k][2], az, fmaf(p[k][1], ay, p[k][0] * ax)) : fmaf(p[k][1], ay, p[k][0] * ax);
        tmin = fminf(tmin, s);
        tmax = fmaxf(tmax, s);
      }
      const float eps = scale * A1;
      const float R = F.r * A1;
      const float lo = tmin - R, hi = tmax + R;
      t = make_float4(lo - eps, hi + eps, lo + eps, hi - eps);
    }
    S.t[lane] = t;
  }
  if (lane == 0) {
    if constexpr (D == 3) {
      float e[3][3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int k1 = (k + 1) % 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) e[k][c] = V[3 * k1 + c] - V[3 * k + c];
      }
      S.en[0] = make_float4(e[0][0], e[0][1], e[0][2], e[1][0]);
      S.en[1] = make_float4(e[1][1], e[1][2], e[2][0], e[2][1]);
      S.en[2] = make_float4(e[2][2], nh[0], nh[1], nh[2]);
    } else {
      S.e[0] = V[2] - V[0];
      S.e[1] = V[3] - V[1];
    }
  }
}

constexpr int kMarkWarps = 4;  // warps per CTA of k_mark_faces
constexpr int kMarkSlots = 64;  // blocks of a face's range looked up once per face (more: per cell)

template <int D, int PRED>
__global__ void __launch_bounds__(kMarkWarps * 32, 6) k_mark_faces(MarkArgs m) {
  const RefineLevel& a = m.lv;
  __shared__ Surv<D> s_surv[kMarkWarps];
  __shared__ int32_t s_bi[kMarkWarps][kMarkSlots];    // block index of each slot of the range (-1: absent)
  __shared__ uint64_t s_mk[kMarkWarps][kMarkSlots];   // its mask when the face started (skips marked cells)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  Surv<D>& S = s_surv[wid];
  const int64_t nblk = launch_count(a.n_blocks, a.n_dev, a.err);
  // cell i meets the face's AABB [vmin, vmax] only if its test region does: box,
  // origin + [i h - d, (i + 1) h + d]; point, its centre origin + (i + 1/2) h
  // within [vmin - d, vmax + d]
  constexpr bool kPoint = PRED == 1;
  const int batch = m.batch > 0 ? (m.batch < kFaceBatch ? m.batch : kFaceBatch) : 1;
  WarpCounters wc;
  unsigned long long n_tests = 0;
  for (;;) {
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(a.work, (unsigned)batch);
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((int64_t)base >= a.nf) break;
    for (int q = 0; q < batch; ++q) {
      const int64_t f = (int64_t)base + q;
      if (f >= a.nf) break;
      // the face's geometry: only geometries marked face by face on this level (their blocks of the
      // level have the mask as the only output; the walk does the others)
      const uint32_t gid = a.table ? __ldg(m.face_gid + f) : 0u;
      const GeomParams& P = a.table ? a.table[gid] : a.g0;
      if (!((P.face_levels >> a.level) & 1u)) continue;
      const FastGeom g = fast_geom(P, a.level);
      const float hf = g.h_hi;
      const float inv_h = 1.0f / hf;
      const float R2 = g.d * g.d;
      int ncell[3] = {1, 1, 1};
#pragma unroll
      for (int c = 0; c < D; ++c) ncell[c] = (4 * P.root[c]) << a.level;
      float V[D * D], nh[3] = {0.f, 0.f, 0.f};
      if constexpr (D == 3) {
        const float4* R = reinterpret_cast<const float4*>(m.rec + f);
        const float4 r0 = __ldg(R), r1 = __ldg(R + 1), r2 = __ldg(R + 2);
        V[0] = r0.x; V[1] = r0.y; V[2] = r0.z; V[3] = r0.w; V[4] = r1.x;
        V[5] = r1.y; V[6] = r1.z; V[7] = r1.w; V[8] = r2.x;
        nh[0] = r2.y; nh[1] = r2.z; nh[2] = r2.w;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) V[j] = __ldg(a.X + (int64_t)j * a.nf + f);
      }
      // cell range per axis: cells whose test region can meet the face's AABB
      // (a superset: the margin covers the FP32 error of the cell coordinate)
      int lo[3] = {0, 0, 0}, n[3] = {1, 1, 1};
      BlockFrame<D> F;
      float shift[3] = {0.f, 0.f, 0.f};
      float O = 0.f;
      bool empty = false;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        float vmin = V[c], vmax = V[c];
#pragma unroll
        for (int k = 1; k < D; ++k) {
          vmin = fminf(vmin, V[D * k + c]);
          vmax = fmaxf(vmax, V[D * k + c]);
        }
        const float margin = 1e-3f + 16.0f * kU32 * (fmaxf(fabsf(vmin), fabsf(vmax)) + fabsf(P.org_hi[c])) * inv_h;
        const float xl = (vmin - P.org_hi[c] - g.d) * inv_h - (kPoint ? 0.5f : 1.0f);
        const float xh = (vmax - P.org_hi[c] + g.d) * inv_h - (kPoint ? 0.5f : 0.0f);
        if (!(xl <= xh)) empty = true;  // also a non-finite coordinate
        const float tl = floorf(xl - margin), th = floorf(xh + margin);
        const int il = tl < 0.f ? 0 : (tl > (float)(ncell[c] - 1) ? ncell[c] : (int)tl);
        const int ih = th < 0.f ? -1 : (th > (float)(ncell[c] - 1) ? ncell[c] - 1 : (int)th);
        if (ih < il) empty = true;
        lo[c] = il;
        n[c] = ih - il + 1;
        float flo;
        df_position(P.org_hi[c], P.org_lo[c], (float)il, g.h_hi, g.h_lo, F.Xb[c], flo);
        shift[c] = flo;
        F.cB[c] = 0.f;
        O = fmaxf(O, (float)(n[c] + 1) * hf + 2.0f * fabsf(flo));
      }
      if (empty) continue;
      F.h = hf;
      F.r = fmaf(0.5f, hf, g.d);
      F.rb = 0.f;
      F.O = O;
      wc.cand++;
      __syncwarp();  // the previous face's tests are done with S
      if constexpr (kPoint) {
        if (lane == 0) setup_point<D>(V, nh, F, S);
      } else {
        setup_face_lanes<D>(V, nh, F, S, lane);
      }
      __syncwarp();
      // the host keeps every range below 2^15 cells (largest face of the binning); a
      // larger one here means inconsistent inputs: reported, not tested
      const int64_t total = (int64_t)n[0] * n[1] * (D == 3 ? n[2] : 1);
      if (total > (1 << 20)) {
        if (lane == 0) atomicOr(a.err, ERR_OVERFLOW);
        continue;
      }
      // index of the level's block with coordinates b, or -1 when the level does not have it: its
      // root by the root order, then per level the ancestor's first child plus the slot (the
      // coordinates' bit of that level per axis); the upper levels' arrays stay in cache
      auto find = [&](const int* b) -> int64_t {
        const int L = a.level;
        int64_t i = P.root_base + (b[0] >> L) + (int64_t)P.root[0] * ((b[1] >> L) + (int64_t)P.root[1] * (b[2] >> L));
        for (int l = 1; l <= L && i >= 0; ++l) {
          const int sh = L - l;
          const int slot = ((b[0] >> sh) & 1) | (((b[1] >> sh) & 1) << 1) | (D == 3 ? ((b[2] >> sh) & 1) << 2 : 0);
          const int32_t c = __ldg(m.first_child[l - 1] + i);
          i = c >= 0 ? (int64_t)c + slot : -1;
        }
        return i < nblk ? i : -1;
      };
      // the range's blocks: looked up once, one lane per block, when they fit the slots
      int blo[3] = {0, 0, 0}, nbk[3] = {1, 1, 1};
#pragma unroll
      for (int c = 0; c < D; ++c) {
        blo[c] = lo[c] >> 2;
        nbk[c] = ((lo[c] + n[c] - 1) >> 2) - blo[c] + 1;
      }
      const int nslot = nbk[0] * nbk[1] * nbk[2];
      const bool slots = nslot <= kMarkSlots;
      // k = a + n b (0 <= a < n, k < 2^20): b = floor((k + 1/2) / n), exactly, from an FP32
      // reciprocal (the quotient is at least 1/(2n) from an integer; the error is below 2^-21 k / n)
      auto divn = [](int k, float inv) { return (int)(((float)k + 0.5f) * inv); };
      const float inv_b0 = 1.0f / (float)nbk[0], inv_b1 = 1.0f / (float)nbk[1];
      if (slots) {
        for (int k = lane; k < nslot; k += 32) {
          const int k1 = divn(k, inv_b0), k2 = divn(k1, inv_b1);
          const int b[3] = {blo[0] + k - k1 * nbk[0], blo[1] + k1 - k2 * nbk[1], blo[2] + k2};
          const int64_t bi = find(b);
          s_bi[wid][k] = (int32_t)bi;
          s_mk[wid][k] = bi >= 0 ? a.mask[bi] : ~0ull;  // absent: every cell skipped
        }
        __syncwarp();
      }
      const float inv_n0 = 1.0f / (float)n[0], inv_n1 = 1.0f / (float)n[1];
      for (int j = lane; j < (int)total; j += 32) {
        const int j1 = divn(j, inv_n0), j2 = D == 3 ? divn(j1, inv_n1) : 0;
        const int i0 = j - j1 * n[0];
        const int i1 = D == 3 ? j1 - j2 * n[1] : j1, i2 = j2;
        const int cell[3] = {lo[0] + i0, lo[1] + i1, D == 3 ? lo[2] + i2 : 0};
        int b[3] = {cell[0] >> 2, cell[1] >> 2, D == 3 ? cell[2] >> 2 : 0};
        const int local = (cell[0] & 3) | ((cell[1] & 3) << 2) | (D == 3 ? (cell[2] & 3) << 4 : 0);
        const uint64_t bit = 1ull << local;
        int64_t bi;
        uint64_t mk;
        if (slots) {
          const int k = (b[0] - blo[0]) + nbk[0] * ((b[1] - blo[1]) + nbk[1] * (b[2] - blo[2]));
          bi = s_bi[wid][k];
          mk = s_mk[wid][k];
        } else {
          bi = find(b);
          mk = bi >= 0 ? a.mask[bi] : ~0ull;
        }
        if (mk & bit) continue;  // absent block or already marked (a stale mask only costs a test)
        ++n_tests;
        const float l[3] = {(float)i0 + 0.5f, (float)i1 + 0.5f, (float)i2 + 0.5f};
        float o[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int c = 0; c < D; ++c) o[c] = fmaf(l[c], g.h_hi, fmaf(l[c], g.h_lo, shift[c]));
        int t = kPoint ? point_test<D>(S, o, R2) : cell_test1<D>(S, o);
        if (t == 2) {
          // not certified in FP32: FP64, unless another face has marked the cell meanwhile
          if (__ldcg(reinterpret_cast<const unsigned long long*>(a.mask + bi)) & bit) continue;
          t = resolve_fp64<D>(a, gid, (uint32_t)f, b, local, &wc.fb, &wc.band) ? 1 : 0;
        }
        if (t) {
          atomicOr(reinterpret_cast<unsigned long long*>(a.mask + bi), (unsigned long long)bit);
          a.flag[bi] = 1;
        }
      }
    }
  }
  unsigned long long v[4] = {wc.fb, wc.band, wc.cand, n_tests};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  }
  if (lane == 0) {
    if (v[0]) atomicAdd(&a.counters[CNT_FALLBACK], v[0]);
    if (v[1]) atomicAdd(&a.counters[CNT_BAND], v[1]);
    if (v[2]) atomicAdd(&a.counters[CNT_FACE_SETUPS], v[2] / 32);  // every lane counted the same faces
    if (v[3]) atomicAdd(&a.counters[CNT_FACE_TESTS], v[3]);
  }
}

// Warps per SM kept resident: 32 (CTAs of `warps` warps).
int grid_warps(int num_sms, int64_t n, int warps, bool persistent) {
  const int64_t cap = (int64_t)num_sms * (32 / warps > 0 ? 32 / warps : 1);
  if (persistent) return (int)cap;
  int64_t need = (n + warps - 1) / warps;
  if (need < 1) need = 1;
  return (int)(need < cap ? need : cap);
}

template <typename K>
void allow_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

int launch_refine(const RefineLevel& a, int num_sms, cudaStream_t st) {
  if (!a.n_dev && a.n_blocks <= 0) return 0;
  const int warps = a.warps > 0 ? a.warps : 4;
  const int g = grid_warps(num_sms, a.n_blocks, warps, a.n_dev != nullptr);
  const size_t smem = (size_t)warps * (a.dim == 3 ? sizeof(WarpSmem<3>) : sizeof(WarpSmem<2>));
  auto go = [&](auto kernel) {
    allow_smem(kernel, smem);
    kernel<<<g, warps * 32, smem, st>>>(a);
  };
  const int mode = a.search == 1 ? 2 : (a.pred == 1 ? 1 : 0);
  if (refine_by_groups(a.dim, a.level, a.pred, a.search)) {
    // one warp per parent group of 8 children
    const int gg = grid_warps(num_sms, a.n_blocks / 8, kGroupWarps, a.n_dev != nullptr);
    const size_t gsm = (size_t)kGroupWarps * sizeof(GroupSmem);
    allow_smem(k_refine_groups, gsm);
    k_refine_groups<<<gg, kGroupWarps * 32, gsm, st>>>(a);
    return 1;
  }
  if (a.dim == 3)
    mode == 2 ? go(k_refine<3, 2>) : (mode == 1 ? go(k_refine<3, 1>) : go(k_refine<3, 0>));
  else
    mode == 2 ? go(k_refine<2, 2>) : (mode == 1 ? go(k_refine<2, 1>) : go(k_refine<2, 0>));
  return 1;
}

int launch_adjacency(const EmitArgs& a, int num_sms, cudaStream_t st) {
  if (!a.lv.n_dev && a.lv.n_blocks <= 0) return 0;
  const int warps = a.lv.warps > 0 ? a.lv.warps : 4;
  const int mode = a.lv.search == 1 ? 2 : (a.lv.pred == 1 ? 1 : 0);
  // first pass: little shared memory, so up to 64 warps per SM
  {
    const int64_t cap = (int64_t)num_sms * (64 / warps > 0 ? 64 / warps : 1);
    int64_t g = a.lv.n_dev ? cap : (a.lv.n_blocks / 32 + warps) / warps;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    auto go = [&](auto kernel) { kernel<<<(unsigned)g, warps * 32, 0, st>>>(a); };
    if (a.lv.dim == 3)
      mode == 2 ? go(k_adjacency<3, 2, 0>) : (mode == 1 ? go(k_adjacency<3, 1, 0>) : go(k_adjacency<3, 0, 0>));
    else
      mode == 2 ? go(k_adjacency<2, 2, 0>) : (mode == 1 ? go(k_adjacency<2, 1, 0>) : go(k_adjacency<2, 0, 0>));
  }
  // second pass over the listed blocks (its count on the device): the walk's shared memory
  cudaMemsetAsync(a.lv.work, 0, sizeof(unsigned), st);
  {
    const int g = grid_warps(num_sms, 0, warps, true);
    const size_t smem = (size_t)warps * (a.lv.dim == 3 ? sizeof(WarpSmem<3>) : sizeof(WarpSmem<2>));
    auto go = [&](auto kernel) {
      allow_smem(kernel, smem);
      kernel<<<g, warps * 32, smem, st>>>(a);
    };
    if (a.lv.dim == 3)
      mode == 2 ? go(k_adjacency<3, 2, 1>) : (mode == 1 ? go(k_adjacency<3, 1, 1>) : go(k_adjacency<3, 0, 1>));
    else
      mode == 2 ? go(k_adjacency<2, 2, 1>) : (mode == 1 ? go(k_adjacency<2, 1, 1>) : go(k_adjacency<2, 0, 1>));
  }
  return 2;
}

int launch_mark_faces(const MarkArgs& m, int num_sms, cudaStream_t st) {
  if (m.lv.nf <= 0) return 0;
  constexpr int kWarps = kMarkWarps;
  const int batch = m.batch > 0 ? m.batch : kFaceBatch;
  int64_t need = (m.lv.nf + batch - 1) / batch;  // warps with work
  int64_t g = (need + kWarps - 1) / kWarps;
  const int64_t cap = (int64_t)num_sms * (32 / kWarps);
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  const int mode = m.lv.pred == 1 ? 1 : 0;
  if (m.lv.dim == 3)
    mode == 1 ? k_mark_faces<3, 1><<<(unsigned)g, kWarps * 32, 0, st>>>(m)
              : k_mark_faces<3, 0><<<(unsigned)g, kWarps * 32, 0, st>>>(m);
  else
    mode == 1 ? k_mark_faces<2, 1><<<(unsigned)g, kWarps * 32, 0, st>>>(m)
              : k_mark_faces<2, 0><<<(unsigned)g, kWarps * 32, 0, st>>>(m);
  return 1;
}

size_t children_scratch_bytes(int64_t n) {
  const int64_t tiles = (n + (int64_t)kChThreads * kChItems - 1) / ((int64_t)kChThreads * kChItems);
  return 16 + (size_t)(tiles > 0 ? tiles : 1) * 8;
}

int launch_children(const ChildrenArgs& a, void* scratch, int num_sms, cudaStream_t st) {
  cudaMemsetAsync(scratch, 0, children_scratch_bytes(a.n), st);
  int64_t tiles = (a.n + (int64_t)kChThreads * kChItems - 1) / ((int64_t)kChThreads * kChItems);
  if (tiles < 1) tiles = 1;
  if (a.n_dev && tiles > (int64_t)num_sms * 4) tiles = (int64_t)num_sms * 4;
  unsigned* ticket = reinterpret_cast<unsigned*>(scratch);
  uint64_t* state = reinterpret_cast<uint64_t*>(static_cast<char*>(scratch) + 16);
  if (a.dim == 3)
    k_children<3><<<(unsigned)tiles, kChThreads, 0, st>>>(a, state, ticket);
  else
    k_children<2><<<(unsigned)tiles, kChThreads, 0, st>>>(a, state, ticket);
  return 1;
}

}  // namespace amr
