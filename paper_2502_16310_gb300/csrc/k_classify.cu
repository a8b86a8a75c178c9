// k_classify.cu — node classification of the finest adjacent cells and the
// restriction of the wall links to fluid nodes.
//
// Paper (Sec. "Conclusions": node classification is the next step towards the
// boundary conditions of the LBM): a node is solid when it lies inside the closed
// boundary mesh.  Each adjacent cell casts a ray from its centre along +x
// through its own row of bins and counts the faces the ray crosses: odd = solid
// (a closed mesh, any orientation).  A face is counted once, in the first of its
// bins along the walked row.  A face whose yz bounding box certainly misses the
// ray is skipped in FP32; the others are tested in FP64 (point in the projected
// triangle, crossing beyond the centre).  A ray that passes exactly through an
// edge or a vertex, or a crossing at the centre itself, is not decided by the
// crossing count: such a cell is classified by the generalized winding number
// of the whole mesh (sum of the signed solid angles / 4 pi; 2D: angles / 2 pi),
// |w| > 1/2 = solid, and counted.
#include "internal.cuh"

namespace amr {

namespace {

constexpr int kCThreads = 128;

// 0 = no crossing, 1 = crossing beyond the centre, 2 = undecided
template <int D>
__device__ int ray_cross(const float* v, const double* p) {
  if constexpr (D == 2) {
    // segment a-b against the ray y = p.y, x > p.x; the half-open rule (lower end in,
    // upper end out) counts a ray through a shared vertex exactly once
    const double ay = v[1], by = v[3];
    if (!((ay <= p[1] && p[1] < by) || (by <= p[1] && p[1] < ay))) return 0;
    const double ax = v[0], bx = v[2];
    const double t = __ddiv_rn(__dsub_rn(p[1], ay), __dsub_rn(by, ay));
    const double xh = __fma_rn(t, __dsub_rn(bx, ax), ax);
    if (fabs(xh - p[0]) <= 1e-12 * (fabs(xh) + fabs(p[0]))) return 2;  // the centre on the segment
    return xh > p[0] ? 1 : 0;
  } else {
    // projection onto the yz plane: edge functions of (p.y, p.z), each with a bound on
    // its rounding error; a sign within that bound is not decided
    constexpr double u64 = 1.1102230246251565e-16;
    double e[3];
    bool tie = false;
    for (int k = 0; k < 3; ++k) {
      const int k1 = (k + 1) % 3;
      const double ay = v[3 * k + 1], az = v[3 * k + 2], by = v[3 * k1 + 1], bz = v[3 * k1 + 2];
      const double t1 = __dmul_rn(__dsub_rn(by, ay), __dsub_rn(p[2], az));
      const double t2 = __dmul_rn(__dsub_rn(bz, az), __dsub_rn(p[1], ay));
      e[k] = __dsub_rn(t1, t2);
      if (fabs(e[k]) <= 8.0 * u64 * (fabs(t1) + fabs(t2))) tie = true;
    }
    if (tie) {
      // decided only when another edge function certainly puts the point outside
      const bool out = (e[0] > 0.0 || e[1] > 0.0 || e[2] > 0.0) && (e[0] < 0.0 || e[1] < 0.0 || e[2] < 0.0);
      return out ? 0 : 2;
    }
    const bool pos = e[0] > 0.0 && e[1] > 0.0 && e[2] > 0.0;
    const bool neg = e[0] < 0.0 && e[1] < 0.0 && e[2] < 0.0;
    if (!pos && !neg) {
      // outside unless an edge function is zero while the others agree in sign
      const bool maybe = (e[0] >= 0.0 && e[1] >= 0.0 && e[2] >= 0.0) || (e[0] <= 0.0 && e[1] <= 0.0 && e[2] <= 0.0);
      return maybe ? 2 : 0;
    }
    // crossing point: x on the face plane at (p.y, p.z), by barycentric weights e_k / sum
    const double s = __dadd_rn(__dadd_rn(e[0], e[1]), e[2]);
    const double xh = (e[1] * (double)v[0] + e[2] * (double)v[3] + e[0] * (double)v[6]) / s;
    if (fabs(xh - p[0]) <= 1e-12 * (fabs(xh) + fabs(p[0]))) return 2;  // the centre on the face
    return xh > p[0] ? 1 : 0;
  }
}

template <int D>
__device__ __noinline__ bool winding_solid(const float* X, int64_t nf, const double* p) {
  double w = 0.0;
  for (int64_t f = 0; f < nf; ++f) {
    if constexpr (D == 2) {
      const double a0 = (double)X[f] - p[0], a1 = (double)X[nf + f] - p[1];
      const double b0 = (double)X[2 * nf + f] - p[0], b1 = (double)X[3 * nf + f] - p[1];
      w += atan2(a0 * b1 - a1 * b0, a0 * b0 + a1 * b1);
    } else {
      double a[3], b[3], c[3];
      for (int k = 0; k < 3; ++k) {
        a[k] = (double)X[(int64_t)k * nf + f] - p[k];
        b[k] = (double)X[(int64_t)(3 + k) * nf + f] - p[k];
        c[k] = (double)X[(int64_t)(6 + k) * nf + f] - p[k];
      }
      const double la = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
      const double lb = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
      const double lc = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
      const double det = a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
                         a[2] * (b[0] * c[1] - b[1] * c[0]);
      const double ab = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
      const double ac = a[0] * c[0] + a[1] * c[1] + a[2] * c[2];
      const double bc = b[0] * c[0] + b[1] * c[1] + b[2] * c[2];
      w += 2.0 * atan2(det, la * lb * lc + ab * lc + ac * lb + bc * la);
    }
  }
  const double pi = 3.14159265358979323846;
  return fabs(D == 2 ? w / (2.0 * pi) : w / (4.0 * pi)) > 0.5;
}

template <int D>
__global__ void __launch_bounds__(kCThreads) k_classify(ClassifyArgs a) {
  using E = typename EntryT<D>::type;
  constexpr int NC = D == 3 ? 64 : 16;
  const E* payload = static_cast<const E*>(a.payload);
  unsigned long long n_fb = 0;
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < a.n_rows;
       row += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t id = a.adj_cell[a.row0 + row];
    const uint32_t blk = id / NC, bit = id % NC;
    const GeomParams& P = a.g0;
    const double hL = scalbn(P.h0, -a.level);
    double p[3] = {0, 0, 0};
    int cb[3] = {0, 0, 0};
#pragma unroll
    for (int c = 0; c < D; ++c) {
      const int gc = 4 * a.blocks[(int64_t)blk * D + c] + (int)((bit >> (2 * c)) & 3u);
      p[c] = __dadd_rn(P.origin[c], __dmul_rn((double)gc + 0.5, hL));
      cb[c] = bin_coord(p[c], P.origin[c], P.bin_scale[c], P.B);
    }
    const float py = (float)p[1], pz = D == 3 ? (float)p[2] : 0.f;
    const float tol = 1e-6f * (fabsf(py) + fabsf(pz) + 1.0f);
    const int64_t B = P.B;
    uint32_t cross = 0;
    bool undecided = false;
    for (int xb = cb[0]; xb < P.B && !undecided; ++xb) {
      const int64_t bin = P.bin_base + xb + B * (cb[1] + (D == 3 ? B * (int64_t)cb[2] : 0));
      const uint32_t j1 = a.offsets[bin + 1];
      for (uint32_t j = a.offsets[bin]; j < j1; ++j) {
        const E& ent = payload[j];
        // count each face once: in its first bin of the walked row
        if (!(((ent.id >> 29) & 1u) || (int)ent.bin[0] == cb[0])) continue;
        float v[9];
#pragma unroll
        for (int q = 0; q < D * D; ++q) v[q] = ent.v[q];
        // yz bounding box certainly misses the ray
        float lo1 = v[1], hi1 = v[1], lo2 = D == 3 ? v[2] : 0.f, hi2 = lo2;
#pragma unroll
        for (int k = 1; k < D; ++k) {
          lo1 = fminf(lo1, v[D * k + 1]);
          hi1 = fmaxf(hi1, v[D * k + 1]);
          if (D == 3) {
            lo2 = fminf(lo2, v[D * k + 2]);
            hi2 = fmaxf(hi2, v[D * k + 2]);
          }
        }
        if (py < lo1 - tol || py > hi1 + tol) continue;
        if (D == 3 && (pz < lo2 - tol || pz > hi2 + tol)) continue;
        const int r = ray_cross<D>(v, p);
        if (r == 2) {
          undecided = true;
          break;
        }
        cross += (uint32_t)r;
      }
    }
    bool solid = (cross & 1u) != 0;
    if (undecided) {
      solid = winding_solid<D>(a.X, a.nf, p);
      ++n_fb;
    }
    a.cls[a.row0 + row] = solid ? 1 : 0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) n_fb += __shfl_xor_sync(0xffffffffu, n_fb, o);
  if ((threadIdx.x & 31) == 0 && n_fb) atomicAdd(&a.counters[CNT_CLASS_FALLBACK], n_fb);
}

// Stable compaction of the links to those whose cell is fluid: keep flags and
// the per-block counts, then a scan gives the positions.
constexpr int kFThreads = 256;

__global__ void k_fluid_count(const uint32_t* link_cell, const uint8_t* cls, int64_t n, uint32_t* cnt) {
  __shared__ uint32_t s;
  if (threadIdx.x == 0) s = 0;
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)kFThreads + threadIdx.x;
  const bool keep = i < n && cls[link_cell[i]] == 0;
  const unsigned m = __ballot_sync(0xffffffffu, keep);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(&s, (uint32_t)__popc(m));
  __syncthreads();
  if (threadIdx.x == 0) cnt[blockIdx.x] = s;
}

__global__ void k_fluid_move(const uint32_t* link_cell, const uint8_t* link_dir, const float* link_q,
                             const uint32_t* link_face, const uint8_t* cls, int64_t n, const uint32_t* base,
                             uint32_t* o_cell, uint8_t* o_dir, float* o_q, uint32_t* o_face) {
  __shared__ uint32_t s_warp[kFThreads / 32];
  const int64_t i = blockIdx.x * (int64_t)kFThreads + threadIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const bool keep = i < n && cls[link_cell[i]] == 0;
  const unsigned m = __ballot_sync(0xffffffffu, keep);
  if (lane == 0) s_warp[wid] = (uint32_t)__popc(m);
  __syncthreads();
  uint32_t off = base[blockIdx.x];
  for (int w = 0; w < wid; ++w) off += s_warp[w];
  if (keep) {
    const uint32_t pos = off + (uint32_t)__popc(m & ((1u << lane) - 1u));
    o_cell[pos] = link_cell[i];
    o_dir[pos] = link_dir[i];
    o_q[pos] = link_q[i];
    o_face[pos] = link_face[i];
  }
}

}  // namespace

int launch_classify(const ClassifyArgs& a, cudaStream_t st) {
  if (a.n_rows <= 0) return 0;
  int64_t g = (a.n_rows + kCThreads - 1) / kCThreads;
  const int64_t cap = (int64_t)current_sm_count() * 16;
  if (g > cap) g = cap;
  if (a.dim == 3)
    k_classify<3><<<(unsigned)g, kCThreads, 0, st>>>(a);
  else
    k_classify<2><<<(unsigned)g, kCThreads, 0, st>>>(a);
  return 1;
}

int64_t fluid_blocks(int64_t n) { return (n + kFThreads - 1) / kFThreads; }

int launch_fluid_count(const uint32_t* link_cell, const uint8_t* cls, int64_t n, uint32_t* cnt, cudaStream_t st) {
  if (n <= 0) return 0;
  k_fluid_count<<<(unsigned)fluid_blocks(n), kFThreads, 0, st>>>(link_cell, cls, n, cnt);
  return 1;
}

int launch_fluid_move(const uint32_t* link_cell, const uint8_t* link_dir, const float* link_q,
                      const uint32_t* link_face, const uint8_t* cls, int64_t n, const uint32_t* base,
                      uint32_t* o_cell, uint8_t* o_dir, float* o_q, uint32_t* o_face, cudaStream_t st) {
  if (n <= 0) return 0;
  k_fluid_move<<<(unsigned)fluid_blocks(n), kFThreads, 0, st>>>(link_cell, link_dir, link_q, link_face, cls, n, base,
                                                                o_cell, o_dir, o_q, o_face);
  return 1;
}

}  // namespace amr
