// amr_oracle.cpp — plain serial FP64 oracle of the geometry-to-AMR hot path.
//
// TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the
// bench's CPU baseline; never by the product path.  Shares no code with the
// CUDA library.  Written for readability against the paper, not for speed:
// every cell gathers its candidate faces from the bins and tests each one.
//
// Paper: Jaber, Essel, Sullivan, "Towards a GPU-native adaptive mesh refinement
// scheme for the Lattice Boltzmann Method in complex geometries" (2025).
#include "amr_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <unordered_map>
#include <vector>

struct orc_geom {
  int dim = 0;
  int64_t nf = 0;
  std::vector<double> X;  // face-vertex list [nf][dim][dim] (FP32 inputs promoted exactly)
  // Binning state (Sec. "Spatial Binning Algorithm")
  int B = 0;
  orc_domain dom{};
  std::vector<int32_t> blo, bhi;  // per face bin range [nf][3]
  std::vector<uint32_t> offsets;  // start index of every bin ("binned_face_ids_N"), B^D + 1 entries
  std::vector<uint32_t> ids;      // face ids grouped by bin ("binned_face_ids"), ascending per bin
};

namespace {

constexpr double kInf = std::numeric_limits<double>::infinity();
constexpr double kBand = 1e-6;  // margin band: 1e-6 * h_L for the adjacency, 1e-6 (dimensionless) for links

void set_err(char* err, int len, const char* msg) {
  if (err && len > 0) std::snprintf(err, (size_t)len, "%s", msg);
}

double level_h(const orc_domain& d, int level) { return std::ldexp(d.h0, -level); }

// Bin coordinate of x along axis a: bins of length (domain size)/B, the first
// and last bin extended to infinity (faces outside the domain clamp inward).
int32_t bin_coord(const orc_domain& d, int B, int a, double x) {
  const double extent = (4.0 * (double)d.root[a]) * d.h0;
  const double s = (double)B / extent;
  const double t = std::floor((x - d.origin[a]) * s);
  if (!(t >= 0.0)) return 0;
  if (t > (double)(B - 1)) return B - 1;
  return (int32_t)t;
}

int64_t bin_linear(int dim, int B, const int32_t* c) {
  int64_t b = c[0] + (int64_t)B * c[1];
  if (dim == 3) b += (int64_t)B * B * c[2];
  return b;
}

// Faces stored in every bin whose box overlaps [lo, hi] per axis, ascending and
// without duplicates.  `widen` adds one bin on each side so that rounding in the
// query box bounds can never drop a bin; extra candidates cannot change a
// predicate that is evaluated exactly on each candidate.
void gather_candidates(const orc_geom& g, const double* lo, const double* hi, bool widen,
                       std::vector<uint32_t>& out) {
  out.clear();
  int32_t a0[3] = {0, 0, 0}, a1[3] = {0, 0, 0};
  for (int a = 0; a < g.dim; ++a) {
    a0[a] = bin_coord(g.dom, g.B, a, lo[a]);
    a1[a] = bin_coord(g.dom, g.B, a, hi[a]);
    if (widen) {
      a0[a] = std::max(0, a0[a] - 1);
      a1[a] = std::min(g.B - 1, a1[a] + 1);
    }
  }
  int32_t c[3];
  for (c[2] = a0[2]; c[2] <= a1[2]; ++c[2])
    for (c[1] = a0[1]; c[1] <= a1[1]; ++c[1])
      for (c[0] = a0[0]; c[0] <= a1[0]; ++c[0]) {
        const int64_t b = bin_linear(g.dim, g.B, c);
        for (uint32_t e = g.offsets[b]; e < g.offsets[b + 1]; ++e) out.push_back(g.ids[e]);
      }
  std::sort(out.begin(), out.end());
  out.erase(std::unique(out.begin(), out.end()), out.end());
}

// ---------------------------------------------------------------------------
// Adjacency predicate.  The paper marks a cell when it lies within the near-wall
// distance of a face (Sec. "Face Detection", Alg. 1).  The hot path here uses
// the box form of that criterion: the cell box inflated by d_L against the
// closed face, decided by the separating-axis theorem.  Margin = the largest
// normalised gap over the candidate axes; > 0 separated, <= 0 intersecting.
// ---------------------------------------------------------------------------

// One axis a: gap between the triangle's projection and the box projection
// [-r*|a|_1, r*|a|_1], divided by |a|_2.  Zero axes are skipped (return -inf).
double axis_gap(const double* a, const double (*p)[3], int nv, double r) {
  const double l2 = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  if (l2 == 0.0) return -kInf;
  double lo = kInf, hi = -kInf;
  for (int k = 0; k < nv; ++k) {
    const double s = p[k][0] * a[0] + p[k][1] * a[1] + p[k][2] * a[2];
    lo = std::min(lo, s);
    hi = std::max(hi, s);
  }
  const double R = r * (std::fabs(a[0]) + std::fabs(a[1]) + std::fabs(a[2]));
  const double gap = std::max(lo - R, -R - hi);
  return gap / l2;
}

double sat_margin(int dim, const double* v, double r) {
  double p[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  const int nv = dim;
  for (int k = 0; k < nv; ++k)
    for (int c = 0; c < dim; ++c) p[k][c] = v[k * dim + c];
  double m = -kInf;
  // the box face normals e_x, e_y (, e_z)
  for (int a = 0; a < dim; ++a) {
    double ax[3] = {0, 0, 0};
    ax[a] = 1.0;
    m = std::max(m, axis_gap(ax, p, nv, r));
  }
  if (dim == 2) {
    // the segment normal
    const double e0 = p[1][0] - p[0][0], e1 = p[1][1] - p[0][1];
    const double n[3] = {-e1, e0, 0.0};
    m = std::max(m, axis_gap(n, p, nv, r));
    return m;
  }
  double e[3][3];
  for (int k = 0; k < 3; ++k)
    for (int c = 0; c < 3; ++c) e[k][c] = p[(k + 1) % 3][c] - p[k][c];
  // the face normal n = (p1 - p0) x (p2 - p0)
  const double u[3] = {p[1][0] - p[0][0], p[1][1] - p[0][1], p[1][2] - p[0][2]};
  const double w[3] = {p[2][0] - p[0][0], p[2][1] - p[0][1], p[2][2] - p[0][2]};
  const double n[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
  m = std::max(m, axis_gap(n, p, nv, r));
  // the nine cross products e_i x edge_k
  for (int k = 0; k < 3; ++k) {
    const double* ek = e[k];
    const double ax[3] = {0.0, -ek[2], ek[1]};  // e_x x e_k
    const double ay[3] = {ek[2], 0.0, -ek[0]};  // e_y x e_k
    const double az[3] = {-ek[1], ek[0], 0.0};  // e_z x e_k
    m = std::max(m, axis_gap(ax, p, nv, r));
    m = std::max(m, axis_gap(ay, p, nv, r));
    m = std::max(m, axis_gap(az, p, nv, r));
  }
  return m;
}

// ---------------------------------------------------------------------------
// Point predicate (Alg. 1, Sec. "Face Detection"): a cell centre is adjacent
// to a face when its Euclidean distance to the closed face is at most the
// near-wall distance.  The paper checks spheres around the vertices, cylinders
// around the edges and the prism over the face; together they are exactly the
// points within that distance of the face, so the oracle evaluates the
// distance itself: the distance to the plane when the point's projection lies
// in the closed triangle, else the smallest distance to the three edges.
// ---------------------------------------------------------------------------

// Distance from the origin to the closed segment a-b.
double point_segment_dist(const double* a, const double* b, int dim) {
  double e[3] = {0, 0, 0}, ae = 0.0, ee = 0.0;
  for (int c = 0; c < dim; ++c) {
    e[c] = b[c] - a[c];
    ae += -a[c] * e[c];
    ee += e[c] * e[c];
  }
  const double t = ee > 0.0 ? std::min(1.0, std::max(0.0, ae / ee)) : 0.0;
  double d2 = 0.0;
  for (int c = 0; c < dim; ++c) {
    const double q = a[c] + t * e[c];
    d2 += q * q;
  }
  return std::sqrt(d2);
}

// Distance from the origin to the closed face with vertices v[dim][dim]
// (given relative to the point).
double point_face_dist(int dim, const double* v) {
  double p[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int k = 0; k < dim; ++k)
    for (int c = 0; c < dim; ++c) p[k][c] = v[k * dim + c];
  if (dim == 2) return point_segment_dist(p[0], p[1], 2);
  const double u[3] = {p[1][0] - p[0][0], p[1][1] - p[0][1], p[1][2] - p[0][2]};
  const double w[3] = {p[2][0] - p[0][0], p[2][1] - p[0][1], p[2][2] - p[0][2]};
  const double n[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
  const double nn = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
  if (nn > 0.0) {
    // the projection is in the closed triangle iff it is on the same side of
    // (or on) all three edge lines within the plane
    bool neg = true, pos = true;
    for (int k = 0; k < 3; ++k) {
      const double* a = p[k];
      const double* b = p[(k + 1) % 3];
      const double e[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
      const double m[3] = {e[1] * n[2] - e[2] * n[1], e[2] * n[0] - e[0] * n[2], e[0] * n[1] - e[1] * n[0]};
      const double s = -(a[0] * m[0] + a[1] * m[1] + a[2] * m[2]);  // (origin - a) . (e x n)
      if (s > 0.0) neg = false;
      if (s < 0.0) pos = false;
    }
    if (neg || pos) return std::fabs(p[0][0] * n[0] + p[0][1] * n[1] + p[0][2] * n[2]) / std::sqrt(nn);
  }
  return std::min(point_segment_dist(p[0], p[1], 3),
                  std::min(point_segment_dist(p[1], p[2], 3), point_segment_dist(p[2], p[0], 3)));
}

void cell_centre(const orc_domain& d, int level, const int32_t* cell, double* x) {
  const double h = level_h(d, level);
  for (int a = 0; a < d.dim; ++a) x[a] = d.origin[a] + ((double)cell[a] + 0.5) * h;
}

// Signed adjacency margin of cell centre x and face f (<= 0: adjacent).
// pred 0 (box): SAT margin of the box x +- r; pred 1 (point): distance - d.
double face_margin(const orc_geom& g, int64_t f, const double* x, double r, int pred, double d) {
  double loc[9];
  const int D = g.dim;
  for (int k = 0; k < D; ++k)
    for (int c = 0; c < D; ++c) loc[k * D + c] = g.X[(size_t)f * D * D + k * D + c] - x[c];
  if (pred == 1) return point_face_dist(D, loc) - d;
  return sat_margin(D, loc, r);
}

// ---------------------------------------------------------------------------
// Wall links: the segment from an adjacent cell's centre along lattice
// direction c_i (length |c_i| h) against the closed faces; q = smallest hit
// parameter t in [0, 1] (Sec. "Identification of Cells Near the Boundary":
// distances along the quadrature abscissae for interpolated boundaries).
// Coplanar / parallel segments miss.  Ties keep the smallest face id.
// ---------------------------------------------------------------------------
const int kD2Q9[9][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
                         {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};
const int kD3Q19[19][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},
                           {0, 0, 1},  {0, 0, -1}, {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},
                           {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                           {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

struct Hit {
  bool hit = false;
  bool band = false;
  double t = 0.0;
};

// p: face vertices relative to the link origin; d: link vector.
Hit link_face(int dim, const double (*p)[3], const double* d) {
  Hit h;
  if (dim == 2) {
    const double e[2] = {p[1][0] - p[0][0], p[1][1] - p[0][1]};
    const double le = std::hypot(e[0], e[1]);
    if (le == 0.0) return h;
    const double den = d[0] * e[1] - d[1] * e[0];
    if (den == 0.0) return h;
    const double ld = std::hypot(d[0], d[1]);
    if (std::fabs(den) <= kBand * ld * le) h.band = true;
    const double t = (p[0][0] * e[1] - p[0][1] * e[0]) / den;
    const double s = (p[0][0] * d[1] - p[0][1] * d[0]) / den;
    const double mu = std::min(std::min(t, 1.0 - t), std::min(s, 1.0 - s));
    if (std::fabs(mu) <= kBand) h.band = true;
    h.hit = mu >= 0.0;
    h.t = t;
    return h;
  }
  const double u[3] = {p[1][0] - p[0][0], p[1][1] - p[0][1], p[1][2] - p[0][2]};
  const double w[3] = {p[2][0] - p[0][0], p[2][1] - p[0][1], p[2][2] - p[0][2]};
  const double n[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
  const double ln = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  if (ln == 0.0) return h;
  const double den = d[0] * n[0] + d[1] * n[1] + d[2] * n[2];
  if (den == 0.0) return h;
  const double ld = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  if (std::fabs(den) <= kBand * ld * ln) h.band = true;
  // signed volumes d . (p_a x p_b): barycentric weights of the plane hit point
  auto vol = [&](const double* a, const double* b) {
    const double c[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
    return d[0] * c[0] + d[1] * c[1] + d[2] * c[2];
  };
  const double l0 = vol(p[1], p[2]) / den;
  const double l1 = vol(p[2], p[0]) / den;
  const double l2 = vol(p[0], p[1]) / den;
  const double t = (p[0][0] * n[0] + p[0][1] * n[1] + p[0][2] * n[2]) / den;
  const double mu = std::min(std::min(std::min(l0, l1), l2), std::min(t, 1.0 - t));
  if (std::fabs(mu) <= kBand) h.band = true;
  h.hit = mu >= 0.0;
  h.t = t;
  return h;
}

int lattice_q(int lattice) { return lattice == 9 ? 9 : (lattice == 19 ? 19 : 0); }

const int* lattice_c(int lattice, int i) { return lattice == 9 ? kD2Q9[i] : kD3Q19[i]; }

void face_local(const orc_geom& g, int64_t f, const double* o, double (*p)[3], const double* ov) {
  const int D = g.dim;
  for (int k = 0; k < 3; ++k) p[k][0] = p[k][1] = p[k][2] = 0.0;
  for (int k = 0; k < D; ++k)
    for (int c = 0; c < D; ++c) {
      const double v = ov ? ov[k * D + c] : g.X[(size_t)f * D * D + k * D + c];
      p[k][c] = v - o[c];
    }
}

// ---------------------------------------------------------------------------
// The paper's own binning (Sec. "Spatial Binning Algorithm", Fig. "Discretization
// of edges and triangles"): a face is discretised into points and belongs to
// every bin that holds at least one of them.  A segment v0-v1 gives the n + 1
// points v0 + (i/n)(v1 - v0), n = max(1, ceil(|v1 - v0| / s)); a triangle
// discretises its first edge v0-v1 so, then every segment from such a point to
// the opposite vertex v2 likewise.  s = half a bin length (the paper only says
// the number of nodes scales with the size of the face).  All arithmetic is FP64
// with one rounding per operation, in this order, so that another
// implementation can reproduce the points exactly.
// ---------------------------------------------------------------------------

int seg_points(const double* a, const double* b, int dim, double s) {
  double l2 = 0.0;
  for (int c = 0; c < dim; ++c) {
    const double e = b[c] - a[c];
    l2 = l2 + e * e;
  }
  const double n = std::ceil(std::sqrt(l2) / s);
  return n < 1.0 ? 1 : (n > 4096.0 ? 4096 : (int)n);
}

template <typename F>
void for_each_sample(const double* v, int dim, double s, F&& visit) {
  const double* v0 = v;
  const double* v1 = v + dim;
  const int n = seg_points(v0, v1, dim, s);
  for (int i = 0; i <= n; ++i) {
    const double t = (double)i / (double)n;
    double p[3] = {0, 0, 0};
    for (int c = 0; c < dim; ++c) p[c] = v0[c] + t * (v1[c] - v0[c]);
    if (dim == 2) {
      visit(p);
      continue;
    }
    const double* v2 = v + 2 * dim;
    const int m = seg_points(p, v2, 3, s);
    for (int j = 0; j <= m; ++j) {
      const double u = (double)j / (double)m;
      double q[3];
      for (int c = 0; c < 3; ++c) q[c] = p[c] + u * (v2[c] - p[c]);
      visit(q);
    }
  }
}

double sample_spacing(const orc_domain& d, int B) {
  double ext = kInf;
  for (int a = 0; a < d.dim; ++a) ext = std::min(ext, (4.0 * (double)d.root[a]) * d.h0);
  return 0.5 * (ext / (double)B);
}

// ---------------------------------------------------------------------------
// Refinement-mark propagation (Sec. "Spatial Binning Algorithm", Fig.
// "propagation"): each round, every marked block marks its 3^D - 1 neighbours of
// the same level that exist, through an intermediate value so that a block
// marked in this round does not spread further in the same round.
// ---------------------------------------------------------------------------

uint64_t block_key(const int32_t* c, int dim) {
  uint64_t k = 0;
  for (int a = 0; a < dim; ++a) k = (k << 21) | (uint64_t)(uint32_t)c[a];
  return k;
}

}  // namespace

extern "C" {

orc_geom* orc_geom_new(int dim, const float* coords, int64_t n_verts, const int32_t* idx, int64_t n_faces,
                       char* err, int errlen) {
  if (dim != 2 && dim != 3) {
    set_err(err, errlen, "dim must be 2 or 3");
    return nullptr;
  }
  if (n_faces < 0 || (n_faces > 0 && !coords)) {
    set_err(err, errlen, "bad face count or null coordinates");
    return nullptr;
  }
  if (idx && n_verts < 0) {
    set_err(err, errlen, "bad vertex count");
    return nullptr;
  }
  orc_geom* g = new orc_geom();
  g->dim = dim;
  g->nf = n_faces;
  g->X.resize((size_t)n_faces * dim * dim);
  // G_ConvertIndexListsToCoordsList: index list -> per-face vertex coordinates
  for (int64_t f = 0; f < n_faces; ++f)
    for (int k = 0; k < dim; ++k) {
      int64_t vi = 0;
      if (idx) {
        vi = idx[f * dim + k];
        if (vi < 0 || vi >= n_verts) {
          set_err(err, errlen, "vertex index out of range");
          delete g;
          return nullptr;
        }
      }
      for (int c = 0; c < dim; ++c) {
        const float x = idx ? coords[vi * dim + c] : coords[(f * dim + k) * dim + c];
        if (!std::isfinite(x)) {
          set_err(err, errlen, "non-finite coordinate");
          delete g;
          return nullptr;
        }
        g->X[(size_t)f * dim * dim + k * dim + c] = (double)x;
      }
    }
  return g;
}

void orc_geom_free(orc_geom* g) { delete g; }

int64_t orc_geom_nfaces(const orc_geom* g) { return g->nf; }

// Sec. "Spatial Binning Algorithm": faces are assigned to every bin they
// overlap; here overlap means the face's axis-aligned bounding box overlaps
// the bin (half-open bins [i/B, (i+1)/B), last bin closed, ends clamped).
int orc_bins_build(orc_geom* g, const orc_domain* dom, int B) {
  if (!g || !dom || B < 1 || dom->dim != g->dim) return 1;
  g->B = B;
  g->dom = *dom;
  const int D = g->dim;
  int64_t nb = (int64_t)B * B * (D == 3 ? B : 1);
  g->blo.assign((size_t)g->nf * 3, 0);
  g->bhi.assign((size_t)g->nf * 3, 0);
  std::vector<std::vector<uint32_t>> lists((size_t)nb);
  for (int64_t f = 0; f < g->nf; ++f) {
    int32_t* lo = &g->blo[(size_t)f * 3];
    int32_t* hi = &g->bhi[(size_t)f * 3];
    for (int a = 0; a < D; ++a) {
      double mn = kInf, mx = -kInf;
      for (int k = 0; k < D; ++k) {
        const double x = g->X[(size_t)f * D * D + k * D + a];
        mn = std::min(mn, x);
        mx = std::max(mx, x);
      }
      lo[a] = bin_coord(*dom, B, a, mn);
      hi[a] = bin_coord(*dom, B, a, mx);
    }
    int32_t c[3] = {0, 0, 0};
    for (c[2] = lo[2]; c[2] <= hi[2]; ++c[2])
      for (c[1] = lo[1]; c[1] <= hi[1]; ++c[1])
        for (c[0] = lo[0]; c[0] <= hi[0]; ++c[0]) lists[(size_t)bin_linear(D, B, c)].push_back((uint32_t)f);
  }
  g->offsets.assign((size_t)nb + 1, 0);
  g->ids.clear();
  for (int64_t b = 0; b < nb; ++b) {
    g->offsets[(size_t)b] = (uint32_t)g->ids.size();
    g->ids.insert(g->ids.end(), lists[(size_t)b].begin(), lists[(size_t)b].end());
  }
  g->offsets[(size_t)nb] = (uint32_t)g->ids.size();
  return 0;
}

// The paper's sampled binning: bins holding at least one sample point of the face.
int orc_bins_build_sampled(orc_geom* g, const orc_domain* dom, int B) {
  if (!g || !dom || B < 1 || dom->dim != g->dim) return 1;
  if (orc_bins_build(g, dom, B)) return 1;  // the AABB ranges (blo / bhi) and the domain
  const int D = g->dim;
  const double s = sample_spacing(*dom, B);
  int64_t nb = (int64_t)B * B * (D == 3 ? B : 1);
  std::vector<std::vector<uint32_t>> lists((size_t)nb);
  std::vector<int64_t> bins;
  for (int64_t f = 0; f < g->nf; ++f) {
    bins.clear();
    for_each_sample(&g->X[(size_t)f * D * D], D, s, [&](const double* q) {
      int32_t c[3] = {0, 0, 0};
      for (int a = 0; a < D; ++a) c[a] = bin_coord(*dom, B, a, q[a]);
      bins.push_back(bin_linear(D, B, c));
    });
    std::sort(bins.begin(), bins.end());
    bins.erase(std::unique(bins.begin(), bins.end()), bins.end());
    for (int64_t b : bins) lists[(size_t)b].push_back((uint32_t)f);
  }
  g->offsets.assign((size_t)nb + 1, 0);
  g->ids.clear();
  for (int64_t b = 0; b < nb; ++b) {
    g->offsets[(size_t)b] = (uint32_t)g->ids.size();
    g->ids.insert(g->ids.end(), lists[(size_t)b].begin(), lists[(size_t)b].end());
  }
  g->offsets[(size_t)nb] = (uint32_t)g->ids.size();
  return 0;
}

int64_t orc_face_samples(const orc_geom* g, int64_t f, double spacing, double* pts, int64_t cap) {
  if (!g || f < 0 || f >= g->nf) return -1;
  const int D = g->dim;
  int64_t k = 0;
  for_each_sample(&g->X[(size_t)f * D * D], D, spacing, [&](const double* q) {
    if (pts && k < cap)
      for (int c = 0; c < D; ++c) pts[k * D + c] = q[c];
    ++k;
  });
  return k;
}

int orc_propagate(int dim, const int32_t* blocks, int64_t n, uint8_t* flags, int rounds) {
  std::unordered_map<uint64_t, int64_t> where;
  where.reserve((size_t)n * 2);
  for (int64_t b = 0; b < n; ++b) where[block_key(blocks + b * dim, dim)] = b;
  for (int r = 0; r < rounds; ++r) {
    for (int64_t b = 0; b < n; ++b) {
      if (flags[b] != 1) continue;
      const int32_t* c = blocks + b * dim;
      const int nz = dim == 3 ? 1 : 0;
      for (int dz = -nz; dz <= nz; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            const int32_t q[3] = {c[0] + dx, c[1] + dy, dim == 3 ? c[2] + dz : 0};
            if (q[0] < 0 || q[1] < 0 || q[2] < 0) continue;
            const auto it = where.find(block_key(q, dim));
            if (it != where.end() && flags[it->second] == 0) flags[it->second] = 2;
          }
    }
    for (int64_t b = 0; b < n; ++b)
      if (flags[b] == 2) flags[b] = 1;
  }
  return 0;
}

// Node classification (the next step the paper names towards boundary
// conditions: which nodes are fluid and which are solid).  A node is solid when
// it lies inside the closed boundary mesh.  Inside is decided by the generalized
// winding number w: the sum of the signed solid angles the faces subtend at the
// node divided by 4 pi (2D: the signed angles of the segments divided by 2 pi),
// which is +-1 inside a closed, consistently oriented mesh and 0 outside, so
// solid iff |w| > 1/2 whatever the orientation.  Nodes within 1e-6 h of the
// mesh are band cases (either class is accepted).
double orc_winding_number(const orc_geom* g, const double* x) {
  const int D = g->dim;
  double w = 0.0;
  for (int64_t f = 0; f < g->nf; ++f) {
    const double* v = &g->X[(size_t)f * D * D];
    if (D == 2) {
      const double a[2] = {v[0] - x[0], v[1] - x[1]};
      const double b[2] = {v[2] - x[0], v[3] - x[1]};
      w += std::atan2(a[0] * b[1] - a[1] * b[0], a[0] * b[0] + a[1] * b[1]);
      continue;
    }
    double a[3], b[3], c[3];
    for (int k = 0; k < 3; ++k) {
      a[k] = v[k] - x[k];
      b[k] = v[3 + k] - x[k];
      c[k] = v[6 + k] - x[k];
    }
    const double la = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    const double lb = std::sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
    const double lc = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    const double det = a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
                       a[2] * (b[0] * c[1] - b[1] * c[0]);
    const double ab = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
    const double ac = a[0] * c[0] + a[1] * c[1] + a[2] * c[2];
    const double bc = b[0] * c[0] + b[1] * c[1] + b[2] * c[2];
    w += 2.0 * std::atan2(det, la * lb * lc + ab * lc + ac * lb + bc * la);
  }
  const double pi = 3.14159265358979323846;
  return D == 2 ? w / (2.0 * pi) : w / (4.0 * pi);
}

int orc_classify(const orc_geom* g, const orc_domain* dom, int level, const int32_t* cells, int64_t n,
                 uint8_t* solid, uint8_t* band) {
  if (!g || !dom || dom->dim != g->dim) return 1;
  const int D = g->dim;
  const double h = level_h(*dom, level);
  for (int64_t i = 0; i < n; ++i) {
    double x[3] = {0, 0, 0};
    cell_centre(*dom, level, cells + i * D, x);
    const double w = orc_winding_number(g, x);
    if (solid) solid[i] = std::fabs(w) > 0.5 ? 1 : 0;
    if (band) {
      double dmin = kInf;
      for (int64_t f = 0; f < g->nf; ++f) {
        double loc[9];
        for (int k = 0; k < D; ++k)
          for (int c = 0; c < D; ++c) loc[k * D + c] = g->X[(size_t)f * D * D + k * D + c] - x[c];
        dmin = std::min(dmin, point_face_dist(D, loc));
      }
      band[i] = dmin <= kBand * h ? 1 : 0;
    }
  }
  return 0;
}

int64_t orc_bins_nnz(const orc_geom* g) { return (int64_t)g->ids.size(); }

void orc_bins_copy(const orc_geom* g, uint32_t* offsets, uint32_t* ids) {
  if (offsets) std::memcpy(offsets, g->offsets.data(), g->offsets.size() * sizeof(uint32_t));
  if (ids && !g->ids.empty()) std::memcpy(ids, g->ids.data(), g->ids.size() * sizeof(uint32_t));
}

void orc_face_bin_range(const orc_geom* g, int64_t f, int32_t* lo, int32_t* hi) {
  for (int a = 0; a < 3; ++a) {
    lo[a] = g->blo[(size_t)f * 3 + a];
    hi[a] = g->bhi[(size_t)f * 3 + a];
  }
}

double orc_sat_margin(int dim, const double* verts_local, double r) { return sat_margin(dim, verts_local, r); }
double orc_point_face_dist(int dim, const double* verts_local) { return point_face_dist(dim, verts_local); }

// Sec. "Identification of Cells Near the Boundary": every cell of every block
// of the level checks the faces of the bins around it; a block is marked when
// any of its cells is adjacent.  The mask keeps the per-cell result.
int orc_refine_blocks(const orc_geom* g, const orc_domain* dom, int level, double d_abs, double d_rel, int pred,
                      int search, const int32_t* blocks, int64_t n, uint64_t* mask, uint64_t* band,
                      int64_t* n_band_pairs, int64_t* n_candidates) {
  if (!g || g->B < 1 || !dom || dom->dim != g->dim) return 1;
  const int D = g->dim;
  const double h = level_h(*dom, level);
  const double dL = d_abs + d_rel * h;
  const double r = 0.5 * h + dL;
  const double tol = kBand * h;
  const int ncell = D == 3 ? 64 : 16;
  std::vector<uint32_t> cand, cand_exact;
  int64_t nbp = 0, ncand = 0;
  for (int64_t b = 0; b < n; ++b) {
    uint64_t mk = 0, bd = 0;
    for (int c = 0; c < ncell; ++c) {
      const int32_t cell[3] = {4 * blocks[b * D + 0] + (c & 3), 4 * blocks[b * D + 1] + ((c >> 2) & 3),
                               D == 3 ? 4 * blocks[b * D + 2] + ((c >> 4) & 3) : 0};
      double x[3] = {0, 0, 0}, lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
      cell_centre(*dom, level, cell, x);
      for (int a = 0; a < D; ++a) {
        lo[a] = x[a] - r;
        hi[a] = x[a] + r;
      }
      if (search == 1)
        gather_candidates(*g, x, x, false, cand);  // the paper's binned search: the faces of the cell's own bin
      else
        gather_candidates(*g, lo, hi, true, cand);
      if (n_candidates) {
        gather_candidates(*g, lo, hi, false, cand_exact);
        ncand += (int64_t)cand_exact.size();
      }
      bool adj = false, robust = false, near = false;
      for (uint32_t f : cand) {
        const double m = face_margin(*g, f, x, r, pred, dL);
        if (m <= 0.0) adj = true;
        if (m < -tol) robust = true;
        if (std::fabs(m) <= tol) {
          near = true;
          ++nbp;
        }
      }
      if (adj) mk |= (uint64_t)1 << c;
      if (!robust && near) bd |= (uint64_t)1 << c;
    }
    mask[b] = mk;
    if (band) band[b] = bd;
  }
  if (n_band_pairs) *n_band_pairs = nbp;
  if (n_candidates) *n_candidates = ncand;
  return 0;
}

// M_RefineAndCoarsenBlocks (refine half): every marked block is replaced on
// the next level by its 2^D children.
int64_t orc_children(int dim, const int32_t* blocks, int64_t n, const uint64_t* mask, int32_t* child_blocks,
                     int32_t* child_parent) {
  int64_t k = 0;
  const int nch = dim == 3 ? 8 : 4;
  for (int64_t b = 0; b < n; ++b) {
    if (!mask[b]) continue;
    for (int s = 0; s < nch; ++s) {
      if (child_blocks) {
        child_blocks[k * dim + 0] = 2 * blocks[b * dim + 0] + (s & 1);
        child_blocks[k * dim + 1] = 2 * blocks[b * dim + 1] + ((s >> 1) & 1);
        if (dim == 3) child_blocks[k * dim + 2] = 2 * blocks[b * dim + 2] + ((s >> 2) & 1);
      }
      if (child_parent) child_parent[k] = (int32_t)b;
      ++k;
    }
  }
  return k;
}

// The faces a cell identifies (Sec. "Identification of Cells Near the Boundary":
// the cell may store the faces it detects for the solver routines).
int64_t orc_cell_faces(const orc_geom* g, const orc_domain* dom, int level, double d_abs, double d_rel, int pred,
                       int search, const int32_t* cells, int64_t n, int64_t* counts, uint32_t* ids, uint8_t* band,
                       int64_t cap) {
  if (!g || g->B < 1 || !dom) return -1;
  const int D = g->dim;
  const double h = level_h(*dom, level);
  const double dL = d_abs + d_rel * h;
  const double r = 0.5 * h + dL;
  const double tol = kBand * h;
  std::vector<uint32_t> cand;
  int64_t tot = 0;
  for (int64_t i = 0; i < n; ++i) {
    double x[3] = {0, 0, 0}, lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    cell_centre(*dom, level, cells + i * D, x);
    for (int a = 0; a < D; ++a) {
      lo[a] = x[a] - r;
      hi[a] = x[a] + r;
    }
    if (search == 1)
      gather_candidates(*g, x, x, false, cand);
    else
      gather_candidates(*g, lo, hi, true, cand);
    int64_t cnt = 0;
    for (uint32_t f : cand) {
      const double m = face_margin(*g, f, x, r, pred, dL);
      if (m <= 0.0 || std::fabs(m) <= tol) {
        // pairs inside the band are listed too, flagged, so a comparison can accept either answer
        if (tot < cap) {
          if (ids) ids[tot] = f;
          if (band) band[tot] = (uint8_t)(std::fabs(m) <= tol ? 1 : 0);
        }
        ++tot;
        ++cnt;
      }
    }
    if (counts) counts[i] = cnt;
  }
  return tot;
}

int orc_lattice_dir(int lattice, int i, int* c) {
  const int Q = lattice_q(lattice);
  if (!Q || i < 0 || i >= Q) return 1;
  const int* v = lattice_c(lattice, i);
  c[0] = v[0];
  c[1] = v[1];
  c[2] = v[2];
  return 0;
}

int orc_cell_links(const orc_geom* g, const orc_domain* dom, int level, int lattice, const int32_t* cells,
                   int64_t n, double* q, int64_t* face, uint8_t* band) {
  const int Q = lattice_q(lattice);
  if (!g || g->B < 1 || !dom || !Q || (Q == 9) != (g->dim == 2)) return 1;
  const int D = g->dim;
  const double h = level_h(*dom, level);
  std::vector<uint32_t> cand;
  for (int64_t i = 0; i < n; ++i) {
    double o[3] = {0, 0, 0};
    cell_centre(*dom, level, cells + i * D, o);
    for (int di = 1; di < Q; ++di) {
      const int* ci = lattice_c(lattice, di);
      double d[3] = {ci[0] * h, ci[1] * h, ci[2] * h};
      double lo[3], hi[3];
      for (int a = 0; a < D; ++a) {
        lo[a] = std::min(o[a], o[a] + d[a]);
        hi[a] = std::max(o[a], o[a] + d[a]);
      }
      gather_candidates(*g, lo, hi, true, cand);
      double best = kInf;
      int64_t bf = -1;
      bool bd = false;
      for (uint32_t f : cand) {
        double p[3][3];
        face_local(*g, f, o, p, nullptr);
        const Hit hh = link_face(D, p, d);
        if (hh.band) bd = true;
        if (hh.hit && hh.t < best) {
          best = hh.t;
          bf = f;
        }
      }
      const int64_t k = i * (Q - 1) + (di - 1);
      q[k] = bf >= 0 ? best : std::numeric_limits<double>::quiet_NaN();
      face[k] = bf;
      if (band) band[k] = (uint8_t)bd;
    }
  }
  return 0;
}

double orc_link_q(const orc_geom* g, const orc_domain* dom, int level, int lattice, const int32_t* cell, int dir,
                  int64_t f, const double* verts_override) {
  const int Q = lattice_q(lattice);
  if (!g || !dom || !Q || dir < 1 || dir >= Q) return std::numeric_limits<double>::quiet_NaN();
  const double h = level_h(*dom, level);
  double o[3] = {0, 0, 0};
  cell_centre(*dom, level, cell, o);
  const int* ci = lattice_c(lattice, dir);
  const double d[3] = {ci[0] * h, ci[1] * h, ci[2] * h};
  double p[3][3];
  face_local(*g, f, o, p, verts_override);
  const Hit hh = link_face(g->dim, p, d);
  return hh.hit ? hh.t : std::numeric_limits<double>::quiet_NaN();
}

// Analytic derivative of the hit parameter t of the plane (3D) / line (2D)
// through the face, with respect to the face vertices:
//   3D: t = (p0 . n)/(d . n), n = (p1-p0) x (p2-p0), w = (p0 - t d)/(d . n):
//       dt/dp1 = (p2-p0) x w, dt/dp2 = w x (p1-p0), dt/dp0 = n/(d.n) - dt/dp1 - dt/dp2.
//   2D: t = (p0 x e)/(d x e), e = p1 - p0, w = (p0 - t d)/(d x e):
//       dt/dp1 = (-w_y, w_x), dt/dp0 = (e_y, -e_x)/(d x e) - dt/dp1.
int orc_q_grad(const orc_geom* g, const orc_domain* dom, int level, int lattice, const int32_t* cells,
               const int32_t* dirs, const int64_t* faces, const double* grad_q, int64_t n_links, double* grad) {
  const int Q = lattice_q(lattice);
  if (!g || !dom || !Q) return 1;
  const int D = g->dim;
  const double h = level_h(*dom, level);
  for (int64_t k = 0; k < n_links; ++k) {
    const int64_t f = faces[k];
    if (f < 0 || f >= g->nf) return 2;
    double o[3] = {0, 0, 0};
    cell_centre(*dom, level, cells + k * D, o);
    const int* ci = lattice_c(lattice, dirs[k]);
    const double d[3] = {ci[0] * h, ci[1] * h, ci[2] * h};
    double p[3][3];
    face_local(*g, f, o, p, nullptr);
    const double gq = grad_q[k];
    double* G = grad + (size_t)f * D * D;
    if (D == 2) {
      const double e[2] = {p[1][0] - p[0][0], p[1][1] - p[0][1]};
      const double den = d[0] * e[1] - d[1] * e[0];
      if (den == 0.0) continue;
      const double t = (p[0][0] * e[1] - p[0][1] * e[0]) / den;
      const double w[2] = {(p[0][0] - t * d[0]) / den, (p[0][1] - t * d[1]) / den};
      const double g1[2] = {-w[1], w[0]};
      const double g0[2] = {e[1] / den - g1[0], -e[0] / den - g1[1]};
      G[0] += gq * g0[0];
      G[1] += gq * g0[1];
      G[2] += gq * g1[0];
      G[3] += gq * g1[1];
      continue;
    }
    const double e1[3] = {p[1][0] - p[0][0], p[1][1] - p[0][1], p[1][2] - p[0][2]};
    const double e2[3] = {p[2][0] - p[0][0], p[2][1] - p[0][1], p[2][2] - p[0][2]};
    const double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const double den = d[0] * n[0] + d[1] * n[1] + d[2] * n[2];
    if (den == 0.0) continue;
    const double t = (p[0][0] * n[0] + p[0][1] * n[1] + p[0][2] * n[2]) / den;
    const double w[3] = {(p[0][0] - t * d[0]) / den, (p[0][1] - t * d[1]) / den, (p[0][2] - t * d[2]) / den};
    const double g1[3] = {e2[1] * w[2] - e2[2] * w[1], e2[2] * w[0] - e2[0] * w[2], e2[0] * w[1] - e2[1] * w[0]};
    const double g2[3] = {w[1] * e1[2] - w[2] * e1[1], w[2] * e1[0] - w[0] * e1[2], w[0] * e1[1] - w[1] * e1[0]};
    for (int c = 0; c < 3; ++c) {
      const double g0 = n[c] / den - g1[c] - g2[c];
      G[0 * 3 + c] += gq * g0;
      G[1 * 3 + c] += gq * g1[c];
      G[2 * 3 + c] += gq * g2[c];
    }
  }
  return 0;
}

}  // extern "C"
