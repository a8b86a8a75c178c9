// k_bin.cu — import and spatial binning kernels.
//
// Import (Sec. "Representation of the Complex Boundary Geometry"): the index
// list or the face-vertex list is gathered into one resident structure-of-arrays
// copy X[k][c][f] (vertex k, coordinate c, face f), the paper's geom_f_face_X.
//
// Binning (Sec. "Spatial Binning Algorithm"): the paper fills a per-face bin
// indicator array chunk by chunk (Cu_FillBins) and compacts it with Thrust.
// Here the bins are exact and sized in one pass: a face-AABB kernel counts the
// (face, bin) incidences with atomics, a single-pass decoupled look-back scan
// turns counts into the CSR start indices (binned_face_ids_N), and a scatter
// writes face ids plus a contiguous per-bin copy of the face coordinates.
#include <atomic>

#include "internal.cuh"

namespace amr {

int current_sm_count() {
  constexpr int kMaxDev = 64;
  static std::atomic<int> cache[kMaxDev];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    cudaGetLastError();
    return 1;
  }
  int n = cache[dev].load(std::memory_order_relaxed);
  if (n <= 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
      cudaGetLastError();
      return 1;
    }
    cache[dev].store(n, std::memory_order_relaxed);
  }
  return n;
}

namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t n, int threads, int cap = 0) {
  if (cap <= 0) cap = current_sm_count() * 16;
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

template <int D>
__global__ void k_load_indexed(const float* __restrict__ verts, int64_t nv, const int32_t* __restrict__ idx,
                               int64_t nf, float* __restrict__ X, int64_t ld, int64_t f0, unsigned* err) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
      int64_t vi = idx[f * D + k];
      const bool ok = vi >= 0 && vi < nv;
      if (!ok) {
        atomicOr(err, ERR_BADINDEX);
        vi = 0;
      }
#pragma unroll
      for (int c = 0; c < D; ++c) {
        float x = ok ? verts[vi * D + c] : 0.0f;
        if (!isfinite(x)) {
          atomicOr(err, ERR_NONFINITE);
          x = 0.0f;
        }
        X[(int64_t)(k * D + c) * ld + f0 + f] = x;
      }
    }
  }
}

template <int D>
__global__ void k_load_facelist(const float* __restrict__ coords, int64_t nf, float* __restrict__ X, int64_t ld,
                                int64_t f0, unsigned* err) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int j = 0; j < D * D; ++j) {
      float x = coords[f * D * D + j];
      if (!isfinite(x)) {
        atomicOr(err, ERR_NONFINITE);
        x = 0.0f;
      }
      X[(int64_t)j * ld + f0 + f] = x;
    }
  }
}

// Face normal n = (v1 - v0) x (v2 - v0) evaluated in FP64 (the edge differences
// and the products of FP32 inputs are exact there) and stored as an unevaluated
// FP32 sum hi + lo, so that later FP32 kernels can form plane offsets with
// double-float accuracy.  Layout nrm[6][nf] = hi.xyz, lo.xyz; rec (when given)
// gets the packed record (vertices, hi, lo) the link kernel reads.
__global__ void k_face_normals(const float* __restrict__ X, int64_t nf, float* __restrict__ nrm,
                               FaceRec3* __restrict__ rec) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
    double v[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int c = 0; c < 3; ++c) v[k][c] = (double)X[(int64_t)(k * 3 + c) * nf + f];
    const double u0 = __dsub_rn(v[1][0], v[0][0]), u1 = __dsub_rn(v[1][1], v[0][1]), u2 = __dsub_rn(v[1][2], v[0][2]);
    const double w0 = __dsub_rn(v[2][0], v[0][0]), w1 = __dsub_rn(v[2][1], v[0][1]), w2 = __dsub_rn(v[2][2], v[0][2]);
    const double n[3] = {__dsub_rn(__dmul_rn(u1, w2), __dmul_rn(u2, w1)),
                         __dsub_rn(__dmul_rn(u2, w0), __dmul_rn(u0, w2)),
                         __dsub_rn(__dmul_rn(u0, w1), __dmul_rn(u1, w0))};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float hi = (float)n[c];
      const float lo = (float)(n[c] - (double)hi);
      nrm[(int64_t)c * nf + f] = hi;
      nrm[(int64_t)(3 + c) * nf + f] = lo;
    }
    if (rec) {
      float4* R = reinterpret_cast<float4*>(rec + f);
      float h[3], l[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        h[c] = (float)n[c];
        l[c] = (float)(n[c] - (double)h[c]);
      }
      R[0] = make_float4((float)v[0][0], (float)v[0][1], (float)v[0][2], (float)v[1][0]);
      R[1] = make_float4((float)v[1][1], (float)v[1][2], (float)v[2][0], (float)v[2][1]);
      R[2] = make_float4((float)v[2][2], h[0], h[1], h[2]);
      R[3] = make_float4(l[0], l[1], l[2], 0.0f);
    }
  }
}

// ---------------------------------------------------------------------------
// The paper's sampled-point bin membership (Sec. "Spatial Binning Algorithm",
// Fig. "Discretization of edges and triangles"): the face is discretised into
// points, its first edge v0-v1 into n + 1 points v0 + (i/n)(v1 - v0) with
// n = max(1, ceil(|v1 - v0| / s)), then (3D) every segment from such a point to
// the opposite vertex likewise; the face belongs to every bin holding a point.
// FP64, one rounding per operation in this order (the definition's order), so
// that the points and their bins are reproducible exactly.
// ---------------------------------------------------------------------------
template <int Dm>
__device__ __forceinline__ int seg_points(const double* a, const double* b, double s) {
  double l2 = 0.0;
#pragma unroll
  for (int c = 0; c < Dm; ++c) {
    const double e = __dsub_rn(b[c], a[c]);
    l2 = __dadd_rn(l2, __dmul_rn(e, e));
  }
  const double n = ceil(__ddiv_rn(__dsqrt_rn(l2), s));
  return n < 1.0 ? 1 : (n > 4096.0 ? 4096 : (int)n);
}

template <int D, typename F>
__device__ __forceinline__ void for_each_sample(const double* v, double s, F&& visit) {
  const double* v0 = v;
  const double* v1 = v + D;
  const int n = seg_points<D>(v0, v1, s);
  for (int i = 0; i <= n; ++i) {
    const double t = __ddiv_rn((double)i, (double)n);
    double p[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int c = 0; c < D; ++c) p[c] = __dadd_rn(v0[c], __dmul_rn(t, __dsub_rn(v1[c], v0[c])));
    if constexpr (D == 2) {
      visit(p);
    } else {
      const double* v2 = v + 6;
      const int m = seg_points<3>(p, v2, s);
      for (int j = 0; j <= m; ++j) {
        const double u = __ddiv_rn((double)j, (double)m);
        double q[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) q[c] = __dadd_rn(p[c], __dmul_rn(u, __dsub_rn(v2[c], p[c])));
        visit(q);
      }
    }
  }
}

// Every bin (x, y, z) of face f's sampled membership, once.  Samples can only
// leave the AABB bin range [lo, hi] by rounding (one bin at most), so a bitmask
// over the range widened by one bin collects them; faces whose widened range
// has more than 64 bins test every bin of that range against all samples.
template <int D, typename F>
__device__ void sampled_bins(const float* X, int64_t nf, int64_t f, const GeomParams& P, double s, const int* lo,
                             const int* hi, F&& visit) {
  double v[9];
#pragma unroll
  for (int j = 0; j < D * D; ++j) v[j] = (double)X[(int64_t)j * nf + f];
  int wl[3] = {0, 0, 0}, wn[3] = {1, 1, 1};
#pragma unroll
  for (int c = 0; c < D; ++c) {
    wl[c] = lo[c] > 0 ? lo[c] - 1 : 0;
    const int wh = hi[c] < P.B - 1 ? hi[c] + 1 : P.B - 1;
    wn[c] = wh - wl[c] + 1;
  }
  auto cell = [&](const double* q, int* c) {
#pragma unroll
    for (int a = 0; a < D; ++a) c[a] = bin_coord(q[a], P.origin[a], P.bin_scale[a], P.B);
  };
  if (wn[0] * wn[1] * wn[2] <= 64) {
    uint64_t m = 0;
    for_each_sample<D>(v, s, [&](const double* q) {
      int c[3] = {0, 0, 0};
      cell(q, c);
      const int k = (c[0] - wl[0]) + wn[0] * ((c[1] - wl[1]) + wn[1] * (c[2] - wl[2]));
      if (k >= 0 && k < 64) m |= 1ull << k;  // (always: rounding moves a sample by < 1 bin)
    });
    for (; m; m &= m - 1) {
      const int k = __ffsll((long long)m) - 1;
      visit(wl[0] + k % wn[0], wl[1] + (k / wn[0]) % wn[1], wl[2] + k / (wn[0] * wn[1]));
    }
    return;
  }
  for (int z = wl[2]; z < wl[2] + wn[2]; ++z)
    for (int y = wl[1]; y < wl[1] + wn[1]; ++y)
      for (int x = wl[0]; x < wl[0] + wn[0]; ++x) {
        bool hit = false;
        for_each_sample<D>(v, s, [&](const double* q) {
          int c[3] = {0, 0, 0};
          cell(q, c);
          hit = hit || (c[0] == x && c[1] == y && c[2] == z);
        });
        if (hit) visit(x, y, z);
      }
}

// Per face: bin range of its AABB along each axis (packed lo | hi << 16, bins of
// its own geometry) and one count per (face, bin) incidence.
template <int D, bool SAMPLED>
__global__ void __launch_bounds__(kThreads) k_face_bins(FaceBinArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // The face-size statistics of the geometry of the block's first face collect in shared memory
  // and reach global memory once per block: one global address per geometry would otherwise take
  // an atomic from every warp of the launch.
  __shared__ unsigned long long s_stat[2];
  __shared__ uint32_t s_gid;
  if (threadIdx.x == 0) {
    const int64_t f1 = blockIdx.x * (int64_t)blockDim.x;
    s_gid = f1 < a.nf ? (a.face_gid ? a.face_gid[f1] : 0u) : 0xffffffffu;
    s_stat[0] = 0ull;
    s_stat[1] = 0ull;
  }
  __syncthreads();
  // warp-uniform trip count: lane i takes face f0 + i (the face-size statistics are reduced per warp)
  for (int64_t f0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); f0 < a.nf; f0 += stride) {
    const int64_t f = f0 + lane;
    uint32_t gid = 0xffffffffu;  // no face: a group of its own
    float rel = 0.f;
    if (f < a.nf) {
      gid = a.face_gid ? a.face_gid[f] : 0u;
      const GeomParams& P = a.table ? a.table[a.face_gid ? a.face_gid[f] : 0u] : a.g0;
      int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
      float ext = 0.f;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        float mn = a.X[(int64_t)c * a.nf + f], mx = mn;
#pragma unroll
        for (int k = 1; k < D; ++k) {
          const float x = a.X[(int64_t)(k * D + c) * a.nf + f];
          mn = fminf(mn, x);
          mx = fmaxf(mx, x);
        }
        ext = fmaxf(ext, mx - mn);
        lo[c] = bin_coord_fast(mn, P, c);
        hi[c] = bin_coord_fast(mx, P, c);
        a.frange[(int64_t)c * a.nf + f] = (uint32_t)lo[c] | ((uint32_t)hi[c] << 16);
      }
      if (!(ext <= 3.0e38f)) ext = INFINITY;  // a non-finite coordinate
      rel = ext / P.h0_hi;                     // in root cells of the face's own geometry
      const int64_t B = P.B;
      if constexpr (SAMPLED) {
        sampled_bins<D>(a.X, a.nf, f, P, a.sample_s, lo, hi, [&](int x, int y, int z) {
          atomicAdd(&a.count[P.bin_base + x + B * (y + B * (int64_t)z)], 1u);
        });
      } else {
        for (int z = lo[2]; z <= hi[2]; ++z)
          for (int y = lo[1]; y <= hi[1]; ++y)
            for (int x = lo[0]; x <= hi[0]; ++x) atomicAdd(&a.count[P.bin_base + x + B * (y + B * (int64_t)z)], 1u);
      }
    }
    if (a.fstat) {
      // per geometry: the largest ratio (non-negative FP32 bits order like the values) and the sum of
      // the ratios in fixed point 2^-16 (each clamped to 2^10 root cells, so 32 of them fit 32 bits)
      const unsigned grp = __match_any_sync(0xffffffffu, gid);
      const uint32_t mx = __reduce_max_sync(grp, __float_as_uint(rel));
      const uint32_t sm = __reduce_add_sync(grp, rel < 1024.0f ? (uint32_t)(rel * 65536.0f) : (1u << 26));
      if (gid != 0xffffffffu && lane == __ffs(grp) - 1) {
        unsigned long long* dst = gid == s_gid ? s_stat : a.fstat + 2 * (int64_t)gid;
        if (mx) atomicMax(dst, (unsigned long long)mx);
        if (sm) atomicAdd(dst + 1, (unsigned long long)sm);
      }
    }
  }
  if (a.fstat) {
    __syncthreads();
    if (threadIdx.x == 0 && s_gid != 0xffffffffu) {
      if (s_stat[0]) atomicMax(a.fstat + 2 * (int64_t)s_gid, s_stat[0]);
      if (s_stat[1]) atomicAdd(a.fstat + 2 * (int64_t)s_gid + 1, s_stat[1]);
    }
  }
}

// Scatter: every (face, bin) incidence claims a slot of the bin by decrementing
// the bin's count (which leaves the counts zeroed for the next call) and writes
// the face id and its payload entry (coordinates, normal, id | first-bin
// flags, bin coordinates) there.
template <int D, bool SAMPLED>
__global__ void __launch_bounds__(kThreads, SAMPLED ? 1 : 4) k_scatter(ScatterArgs a) {
  using E = typename EntryT<D>::type;
  constexpr int QE = (int)(sizeof(E) / 16);  // 16-byte quarters of an entry
  E* payload = static_cast<E*>(a.payload);
  const int64_t nf = a.f.nf;
  if constexpr (SAMPLED) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
      const GeomParams& P = a.f.table ? a.f.table[a.f.face_gid ? a.f.face_gid[f] : 0u] : a.f.g0;
      const int64_t B = P.B, bin_base = P.bin_base;
      int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const uint32_t r = a.f.frange[(int64_t)c * nf + f];
        lo[c] = (int)(r & 0xffffu);
        hi[c] = (int)(r >> 16);
      }
      E e{};
      if constexpr (D == 3) {
        // the face record's first 48 bytes are the entry's vertices and normal
        const float4* R = reinterpret_cast<const float4*>(a.rec + f);
        float4* q = reinterpret_cast<float4*>(&e);
        q[0] = __ldg(R);
        q[1] = __ldg(R + 1);
        q[2] = __ldg(R + 2);
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) e.v[j] = a.f.X[(int64_t)j * nf + f];
      }
      sampled_bins<D>(a.f.X, nf, f, P, a.f.sample_s, lo, hi, [&](int x, int y, int z) {
        const int64_t b = bin_base + x + B * (y + B * (int64_t)z);
        const uint32_t old = atomicSub(&a.f.count[b], 1u);
        const int64_t pos = (int64_t)a.offsets[b] + old - 1;
        a.ids[pos] = (uint32_t)f;
        uint32_t flags = (x == lo[0] ? (1u << 29) : 0u) | (y == lo[1] ? (1u << 30) : 0u);
        if (D == 3) flags |= (z == lo[2] ? (1u << 31) : 0u);
        e.id = (uint32_t)f | flags;
        e.bin[0] = (uint32_t)x;
        e.bin[1] = (uint32_t)y;
        e.bin[2] = (uint32_t)z;
        const float4* src = reinterpret_cast<const float4*>(&e);
        float4* dst = reinterpret_cast<float4*>(payload + pos);
#pragma unroll
        for (int q = 0; q < QE; ++q) dst[q] = src[q];
      });
    }
  } else {
    // Lane = face; the warp steps through the incidences of its 32 faces together.  Each
    // incidence's entry is staged in shared memory and the warp writes 32 / QE whole entries
    // per store instruction (QE lanes per entry), so every entry leaves as full 32-byte
    // sectors instead of QE scattered 16-byte pieces.
    __shared__ float4 s_ent[kThreads / 32][32 * QE];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t f0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); f0 < nf; f0 += stride) {
      const int64_t f = f0 + lane;
      int n = 0, nx = 1, ny = 1;
      int lo[3] = {0, 0, 0};
      int64_t B = 0, bin_base = 0;
      float4 head[QE - 1];  // the entry's coordinates (and normal), the same for all its bins
      if (f < nf) {
        const GeomParams& P = a.f.table ? a.f.table[a.f.face_gid ? a.f.face_gid[f] : 0u] : a.f.g0;
        B = P.B;
        bin_base = P.bin_base;
        int ext[3] = {1, 1, 1};
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const uint32_t r = a.f.frange[(int64_t)c * nf + f];
          lo[c] = (int)(r & 0xffffu);
          ext[c] = (int)(r >> 16) - lo[c] + 1;
        }
        nx = ext[0];
        ny = ext[1];
        n = ext[0] * ext[1] * ext[2];
        if constexpr (D == 3) {
          // the face record's first 48 bytes are the entry's vertices and normal
          const float4* R = reinterpret_cast<const float4*>(a.rec + f);
          head[0] = __ldg(R);
          head[1] = __ldg(R + 1);
          head[2] = __ldg(R + 2);
        } else {
          head[0] = make_float4(a.f.X[f], a.f.X[nf + f], a.f.X[2 * nf + f], a.f.X[3 * nf + f]);
        }
      }
      const int m = __reduce_max_sync(0xffffffffu, n);
      for (int k = 0; k < m; ++k) {
        int64_t pos = -1;
        if (k < n) {
          const int x = lo[0] + k % nx, y = lo[1] + (k / nx) % ny, z = lo[2] + k / (nx * ny);
          const int64_t b = bin_base + x + B * (y + B * (int64_t)z);
          const uint32_t old = atomicSub(&a.f.count[b], 1u);
          pos = (int64_t)a.offsets[b] + old - 1;
          a.ids[pos] = (uint32_t)f;
          uint32_t flags = (x == lo[0] ? (1u << 29) : 0u) | (y == lo[1] ? (1u << 30) : 0u);
          if (D == 3) flags |= (z == lo[2] ? (1u << 31) : 0u);
#pragma unroll
          for (int q = 0; q < QE - 1; ++q) s_ent[wid][lane * QE + q] = head[q];
          s_ent[wid][lane * QE + QE - 1] =
              make_float4(__uint_as_float((uint32_t)f | flags), __uint_as_float((uint32_t)x),
                          __uint_as_float((uint32_t)y), __uint_as_float((uint32_t)z));
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < QE; ++r) {
          const int j = r * (32 / QE) + lane / QE;  // entry written by this lane in round r
          const int64_t pj = __shfl_sync(0xffffffffu, pos, j);
          if (pj >= 0) reinterpret_cast<float4*>(payload + pj)[lane % QE] = s_ent[wid][j * QE + lane % QE];
        }
        __syncwarp();  // the next incidence reuses the staging area
      }
    }
  }
}

// Single-pass exclusive scan (decoupled look-back over ticket-ordered tiles).
// CTAs take tiles in ticket order until none is left, so the grid may be
// smaller than the tile count and the element count may come from device
// memory (n_dev, bounded by the capacity n_cap).
template <typename T, int ITEMS>
__global__ void __launch_bounds__(kThreads, 5) k_scan(const T* __restrict__ in, T* __restrict__ out, int64_t n_cap,
                                                    const uint64_t* n_dev, uint64_t* total, uint64_t* state,
                                                    unsigned* ticket, unsigned* err) {
  __shared__ unsigned s_tile;
  __shared__ uint64_t s_warp[kThreads / 32];
  __shared__ uint64_t s_prefix;
  int64_t n = n_cap;
  if (n_dev) {
    const uint64_t nd = *n_dev;
    if ((int64_t)nd > n_cap) {
      if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, ERR_OVERFLOW);
    } else {
      n = (int64_t)nd;
    }
  }
  const int64_t ntiles = (n + (int64_t)kThreads * ITEMS - 1) / ((int64_t)kThreads * ITEMS);
  if (ntiles == 0) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *total = 0;
    return;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  static_assert(ITEMS * sizeof(T) % 16 == 0, "a thread's items are whole 16-byte vectors");
  const bool vec = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15u) == 0;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
    __syncthreads();
    const long long tile = s_tile;
    if (tile >= ntiles) break;
    const int64_t base = tile * (int64_t)kThreads * ITEMS + (int64_t)threadIdx.x * ITEMS;
    T v[ITEMS];  // the items stay in their own width; sums and prefixes are 64-bit
    uint64_t sum = 0;
    const bool full = vec && base + ITEMS <= n;
    if (full) {
      // ITEMS * sizeof(T) bytes as 16-byte loads
      const uint4* src = reinterpret_cast<const uint4*>(in + base);
#pragma unroll
      for (int q = 0; q < (int)(ITEMS * sizeof(T) / 16); ++q) reinterpret_cast<uint4*>(v)[q] = src[q];
    } else {
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        const int64_t j = base + i;
        v[i] = j < n ? in[j] : (T)0;
      }
    }
#pragma unroll
    for (int i = 0; i < ITEMS; ++i) sum += (uint64_t)v[i];
    const uint64_t incl = warp_inclusive_scan<unsigned long long>(sum);
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      uint64_t w = lane < kThreads / 32 ? s_warp[lane] : 0ull;
      w = warp_inclusive_scan<unsigned long long>(w);
      if (lane < kThreads / 32) s_warp[lane] = w;
    }
    __syncthreads();
    const uint64_t warp_excl = wid > 0 ? s_warp[wid - 1] : 0ull;
    const uint64_t agg = s_warp[kThreads / 32 - 1];
    if (wid == 0) {
      const uint64_t p = lookback_warp(state, tile, agg, err);
      if (lane == 0) s_prefix = p;
    }
    __syncthreads();
    const uint64_t pre = s_prefix;
    if (threadIdx.x == 0 && tile == ntiles - 1) *total = pre + agg;
    uint64_t run = pre + warp_excl + incl - sum;
    if (full) {
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {  // exclusive prefixes in place
        const T x = v[i];
        v[i] = (T)run;
        run += x;
      }
      uint4* dst = reinterpret_cast<uint4*>(out + base);
#pragma unroll
      for (int q = 0; q < (int)(ITEMS * sizeof(T) / 16); ++q) dst[q] = reinterpret_cast<const uint4*>(v)[q];
    } else {
#pragma unroll
      for (int i = 0; i < ITEMS; ++i) {
        const int64_t j = base + i;
        if (j < n) out[j] = (T)run;
        run += v[i];
      }
    }
    __syncthreads();
  }
}

__global__ void k_write_total_u32(const uint64_t* total, uint32_t* dst, unsigned* err) {
  const uint64_t t = *total;
  if (t > 0xffffffffull) atomicOr(err, ERR_OVERFLOW);
  *dst = (uint32_t)t;
}

template <int D>
__global__ void k_root_blocks(int r0, int r1, int r2, int32_t* __restrict__ blocks, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = i % r0;
    const int64_t y = (i / r0) % r1;
    blocks[i * D + 0] = (int32_t)x;
    blocks[i * D + 1] = (int32_t)y;
    if (D == 3) blocks[i * D + 2] = (int32_t)(i / ((int64_t)r0 * r1));
  }
}

// Level-0 blocks of many geometries: geometry g owns entries
// [root_base_g, root_base_g + prod(root_g)), x fastest within it.
template <int D>
__global__ void k_root_blocks_multi(const GeomParams* __restrict__ table, int n_geom, int32_t* __restrict__ blocks,
                                    uint32_t* __restrict__ gid, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = n_geom - 1;
    while (lo < hi) {  // last geometry with root_base <= i
      const int mid = (lo + hi + 1) >> 1;
      if (table[mid].root_base <= i)
        lo = mid;
      else
        hi = mid - 1;
    }
    const GeomParams& P = table[lo];
    const int64_t j = i - P.root_base;
    blocks[i * D + 0] = (int32_t)(j % P.root[0]);
    blocks[i * D + 1] = (int32_t)((j / P.root[0]) % P.root[1]);
    if (D == 3) blocks[i * D + 2] = (int32_t)(j / ((int64_t)P.root[0] * P.root[1]));
    gid[i] = (uint32_t)lo;
  }
}

__global__ void k_face_gid(const GeomParams* __restrict__ table, int n_geom, int64_t nf, uint32_t* __restrict__ out) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = n_geom - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (table[mid].face_base <= f)
        lo = mid;
      else
        hi = mid - 1;
    }
    out[f] = (uint32_t)lo;
  }
}

constexpr int kScanItemsU32 = 16;
constexpr int kScanItemsU64 = 4;

size_t scan_scratch(int64_t n, int items) {
  const int64_t tiles = (n + (int64_t)kThreads * items - 1) / ((int64_t)kThreads * items);
  return 16 + (size_t)(tiles > 0 ? tiles : 1) * 8;
}

}  // namespace

int launch_load_indexed(int dim, const float* verts, int64_t nv, const int32_t* idx, int64_t nf, float* X,
                        unsigned* err, cudaStream_t st, int64_t ld, int64_t f0) {
  if (nf <= 0) return 0;
  if (ld < 0) ld = nf;
  const int g = grid_for(nf, kThreads);
  if (dim == 3)
    k_load_indexed<3><<<g, kThreads, 0, st>>>(verts, nv, idx, nf, X, ld, f0, err);
  else
    k_load_indexed<2><<<g, kThreads, 0, st>>>(verts, nv, idx, nf, X, ld, f0, err);
  return 1;
}

int launch_load_facelist(int dim, const float* coords, int64_t nf, float* X, unsigned* err, cudaStream_t st,
                         int64_t ld, int64_t f0) {
  if (nf <= 0) return 0;
  if (ld < 0) ld = nf;
  const int g = grid_for(nf, kThreads);
  if (dim == 3)
    k_load_facelist<3><<<g, kThreads, 0, st>>>(coords, nf, X, ld, f0, err);
  else
    k_load_facelist<2><<<g, kThreads, 0, st>>>(coords, nf, X, ld, f0, err);
  return 1;
}

int launch_face_normals(const float* X, int64_t nf, float* nrm, FaceRec3* rec, cudaStream_t st) {
  if (nf <= 0) return 0;
  k_face_normals<<<grid_for(nf, kThreads), kThreads, 0, st>>>(X, nf, nrm, rec);
  return 1;
}

int launch_face_bins(const FaceBinArgs& a, cudaStream_t st) {
  if (a.nf <= 0) return 0;
  const int gr = grid_for(a.nf, kThreads);
  if (a.dim == 3) {
    if (a.sampled)
      k_face_bins<3, true><<<gr, kThreads, 0, st>>>(a);
    else
      k_face_bins<3, false><<<gr, kThreads, 0, st>>>(a);
  } else {
    if (a.sampled)
      k_face_bins<2, true><<<gr, kThreads, 0, st>>>(a);
    else
      k_face_bins<2, false><<<gr, kThreads, 0, st>>>(a);
  }
  return 1;
}

int launch_face_bins(int dim, const float* X, int64_t nf, const BinGrid& g, uint32_t* frange, uint32_t* count,
                     cudaStream_t st) {
  FaceBinArgs a{};
  a.dim = dim;
  a.X = X;
  a.nf = nf;
  a.g0.B = g.B;
  for (int c = 0; c < 3; ++c) {
    a.g0.origin[c] = g.origin[c];
    a.g0.bin_scale[c] = g.scale[c];
    a.g0.org_hi[c] = (float)g.origin[c];
    a.g0.org_lo[c] = (float)(g.origin[c] - (double)a.g0.org_hi[c]);
    a.g0.scale32[c] = (float)g.scale[c];
  }
  a.frange = frange;
  a.count = count;
  return launch_face_bins(a, st);
}

size_t scan_u32_scratch_bytes(int64_t n) { return scan_scratch(n, kScanItemsU32); }
size_t scan_u64_scratch_bytes(int64_t n) { return scan_scratch(n, kScanItemsU64); }

int launch_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint64_t* total64, void* scratch, unsigned* err,
                    cudaStream_t st) {
  const size_t sb = scan_u32_scratch_bytes(n);
  cudaMemsetAsync(scratch, 0, sb, st);
  const int64_t tiles = (n + (int64_t)kThreads * kScanItemsU32 - 1) / ((int64_t)kThreads * kScanItemsU32);
  unsigned* ticket = reinterpret_cast<unsigned*>(scratch);
  uint64_t* state = reinterpret_cast<uint64_t*>(static_cast<char*>(scratch) + 16);
  k_scan<uint32_t, kScanItemsU32><<<(unsigned)(tiles > 0 ? tiles : 1), kThreads, 0, st>>>(in, out, n, nullptr,
                                                                                        total64, state, ticket, err);
  k_write_total_u32<<<1, 1, 0, st>>>(total64, out + n, err);
  return 2;
}

int launch_scan_u64(const uint64_t* in, uint64_t* out, int64_t n, const uint64_t* n_dev, uint64_t* total,
                    void* scratch, unsigned* err, int num_sms, cudaStream_t st) {
  const size_t sb = scan_u64_scratch_bytes(n);
  cudaMemsetAsync(scratch, 0, sb, st);
  int64_t tiles = (n + (int64_t)kThreads * kScanItemsU64 - 1) / ((int64_t)kThreads * kScanItemsU64);
  if (tiles < 1) tiles = 1;
  if (n_dev && tiles > (int64_t)num_sms * 4) tiles = (int64_t)num_sms * 4;
  unsigned* ticket = reinterpret_cast<unsigned*>(scratch);
  uint64_t* state = reinterpret_cast<uint64_t*>(static_cast<char*>(scratch) + 16);
  k_scan<uint64_t, kScanItemsU64><<<(unsigned)tiles, kThreads, 0, st>>>(in, out, n, n_dev, total, state, ticket, err);
  return 1;
}

int launch_scatter(const ScatterArgs& a, cudaStream_t st) {
  if (a.f.nf <= 0) return 0;
  const int g = grid_for(a.f.nf, kThreads);
  if (a.f.dim == 3) {
    if (a.f.sampled)
      k_scatter<3, true><<<g, kThreads, 0, st>>>(a);
    else
      k_scatter<3, false><<<g, kThreads, 0, st>>>(a);
  } else {
    if (a.f.sampled)
      k_scatter<2, true><<<g, kThreads, 0, st>>>(a);
    else
      k_scatter<2, false><<<g, kThreads, 0, st>>>(a);
  }
  return 1;
}

int launch_root_blocks_multi(int dim, const GeomParams* table, int n_geom, int32_t* blocks, uint32_t* gid, int64_t n,
                             cudaStream_t st) {
  if (n <= 0) return 0;
  const int g = grid_for(n, kThreads);
  if (dim == 3)
    k_root_blocks_multi<3><<<g, kThreads, 0, st>>>(table, n_geom, blocks, gid, n);
  else
    k_root_blocks_multi<2><<<g, kThreads, 0, st>>>(table, n_geom, blocks, gid, n);
  return 1;
}

int launch_face_gid(const GeomParams* table, int n_geom, int64_t nf, uint32_t* face_gid, cudaStream_t st) {
  if (nf <= 0) return 0;
  k_face_gid<<<grid_for(nf, kThreads), kThreads, 0, st>>>(table, n_geom, nf, face_gid);
  return 1;
}

int launch_root_blocks(int dim, const int* root, int32_t* blocks, int64_t n, cudaStream_t st) {
  if (n <= 0) return 0;
  const int g = grid_for(n, kThreads);
  if (dim == 3)
    k_root_blocks<3><<<g, kThreads, 0, st>>>(root[0], root[1], root[2], blocks, n);
  else
    k_root_blocks<2><<<g, kThreads, 0, st>>>(root[0], root[1], 1, blocks, n);
  return 1;
}

}  // namespace amr

// ---------------------------------------------------------------------------
// Binning without allocation (amr_bin_faces_static).
//
// Some callers cannot allocate device memory at all: a solver that reserved
// the device's memory up front for its own arena, a plugin whose host owns
// every device allocation, or a time-critical loop that must not pay the
// implicit synchronisation a cudaMalloc / cudaFree can cause.  For them this
// entry point bins faces with no allocation: its scratch (bin counts, face bin
// ranges, scan tile states) is one fixed array in device global memory, below.
// Every GPU that loads this library holds the array until the process exits.
// ---------------------------------------------------------------------------
#include <mutex>

#include "amrgeom.h"

namespace amr {
namespace {

constexpr int64_t kStaticMaxBins = AMR_STATIC_MAX_BINS;
constexpr int64_t kStaticMaxFaces = AMR_STATIC_MAX_FACES;
constexpr size_t kStCount = 0;                                                     // u32 [max bins]
constexpr size_t kStRange = kStCount + 4 * (size_t)kStaticMaxBins;                 // u32 [3][max faces]
constexpr size_t kStScan = kStRange + 12 * (size_t)kStaticMaxFaces;                // scan ticket + tile states
constexpr size_t kStScanBytes = 16 + 8 * (size_t)((kStaticMaxBins + kThreads * kScanItemsU32 - 1) /
                                                   (kThreads * kScanItemsU32));
constexpr size_t kStTotal = (kStScan + kStScanBytes + 255) / 256 * 256;            // u64 total
constexpr size_t kStErr = kStTotal + 8;                                            // u32 error word
constexpr size_t kStBytes = kStErr + 8;

static __device__ __align__(256) unsigned char g_bin_static_scratch[kStBytes];

// Device address of the array, looked up once per device (host code may not use
// the symbol itself as a device pointer).
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

cudaError_t static_scratch(int dev, unsigned char** out) {
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_bin_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return cudaSuccess;
}

// Face ids only (no coordinate payload): same slot claiming as k_scatter.
template <int D>
__global__ void k_scatter_ids(int64_t nf, const uint32_t* __restrict__ frange, const uint32_t* __restrict__ offsets,
                              uint32_t* __restrict__ count, uint32_t* __restrict__ ids, int Bi) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const uint32_t r = frange[(int64_t)a * nf + f];
      lo[a] = (int)(r & 0xffffu);
      hi[a] = (int)(r >> 16);
    }
    const int64_t B = Bi;
    for (int z = lo[2]; z <= hi[2]; ++z)
      for (int y = lo[1]; y <= hi[1]; ++y)
        for (int x = lo[0]; x <= hi[0]; ++x) {
          const int64_t b = x + B * (y + B * (int64_t)z);
          const uint32_t old = atomicSub(&count[b], 1u);
          ids[(int64_t)offsets[b] + old - 1] = (uint32_t)f;
        }
  }
}

// Every coordinate finite, else ERR_NONFINITE in the error word (the regular
// path rejects such faces at load; here the caller's array is binned as given).
__global__ void k_check_finite(const float* __restrict__ X, int64_t n, unsigned* err) {
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(X[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, ERR_NONFINITE);
}

// Device memory of device dev (or managed memory, which every device can reach).
bool on_device(const void* p, int dev) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeManaged || (at.type == cudaMemoryTypeDevice && at.device == dev);
}

}  // namespace
}  // namespace amr

extern "C" AMR_API amr_status amr_bin_faces_static(const amr_domain* dom, const float* faces, int64_t n_faces,
                                                   int bin_density, uint32_t* offsets, uint32_t* ids,
                                                   int64_t ids_capacity, int64_t* nnz) {
  using namespace amr;
  if (!dom || !offsets || !nnz || (dom->dim != 2 && dom->dim != 3) || !(dom->h0 > 0.0)) return AMR_EINVAL;
  const int D = dom->dim;
  const int B = bin_density;
  if (B < 1 || B > 65535 || n_faces < 0 || n_faces > kStaticMaxFaces || ids_capacity < 0) return AMR_EINVAL;
  int64_t nb = 1;
  for (int a = 0; a < D; ++a) {
    if (dom->root_blocks[a] < 1) return AMR_EINVAL;
    nb *= B;
    if (nb > kStaticMaxBins) return AMR_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return AMR_ECUDA;
  if (n_faces > 0 && (!faces || !on_device(faces, dev))) return AMR_EINVAL;
  if (!on_device(offsets, dev) || (ids_capacity > 0 && (!ids || !on_device(ids, dev)))) return AMR_EINVAL;
  unsigned char* s = nullptr;
  if (static_scratch(dev, &s) != cudaSuccess) return AMR_ECUDA;
  cudaStream_t st = dom->stream ? static_cast<cudaStream_t>(dom->stream) : cudaStreamLegacy;
  uint32_t* count = reinterpret_cast<uint32_t*>(s + kStCount);
  uint32_t* frange = reinterpret_cast<uint32_t*>(s + kStRange);
  uint64_t* total = reinterpret_cast<uint64_t*>(s + kStTotal);
  unsigned* err = reinterpret_cast<unsigned*>(s + kStErr);
  BinGrid g{};
  g.B = B;
  for (int a = 0; a < 3; ++a) {
    g.origin[a] = dom->origin[a];
    const double extent = (4.0 * (double)(a < D ? dom->root_blocks[a] : 1)) * dom->h0;
    g.scale[a] = (double)B / extent;
  }
  // the array keeps the previous call's contents: zero the counts, the total and the error word
  if (cudaMemsetAsync(count, 0, 4 * (size_t)nb, st) != cudaSuccess) return AMR_ECUDA;
  if (cudaMemsetAsync(s + kStTotal, 0, 16, st) != cudaSuccess) return AMR_ECUDA;
  if (n_faces > 0) {
    const int64_t nx = (int64_t)D * D * n_faces;
    k_check_finite<<<grid_for(nx, kThreads), kThreads, 0, st>>>(faces, nx, err);
  }
  launch_face_bins(D, faces, n_faces, g, frange, count, st);
  launch_scan_u32(count, offsets, nb, total, s + kStScan, err, st);
  uint64_t h_total = 0;
  unsigned h_err = 0;
  if (cudaMemcpyAsync(&h_total, total, 8, cudaMemcpyDeviceToHost, st) != cudaSuccess) return AMR_ECUDA;
  if (cudaMemcpyAsync(&h_err, err, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess) return AMR_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return AMR_ECUDA;
  if (h_err & ERR_NONFINITE) return AMR_EINVAL;
  if (h_err & ERR_TIMEOUT) return AMR_ETIMEOUT;
  if (h_err || h_total > 0xffffffffull) return AMR_EOVERFLOW;
  *nnz = (int64_t)h_total;
  if ((int64_t)h_total > ids_capacity) return AMR_EOVERFLOW;
  if (n_faces > 0) {
    const int gr = grid_for(n_faces, kThreads);
    if (D == 3)
      k_scatter_ids<3><<<gr, kThreads, 0, st>>>(n_faces, frange, offsets, count, ids, B);
    else
      k_scatter_ids<2><<<gr, kThreads, 0, st>>>(n_faces, frange, offsets, count, ids, B);
  }
  return cudaGetLastError() == cudaSuccess ? AMR_OK : AMR_ECUDA;
}
