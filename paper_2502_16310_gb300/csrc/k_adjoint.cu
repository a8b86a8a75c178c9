// k_adjoint.cu — vertex adjoint of the wall-link fractions q, deterministic.
//
// q of a link is the hit parameter t of the plane through its face (links are
// only formed on hits, Sec. "Identification of Cells Near the Boundary"):
//   t = ((v0 - x) . n) / (d . n),  n = (v1 - v0) x (v2 - v0),  d = c_i h.
// With w = (v0 - x - t d) / (d . n):
//   dt/dv1 = (v2 - v0) x w,  dt/dv2 = w x (v1 - v0),  dt/dv0 = n / (d . n) - dt/dv1 - dt/dv2
// (2D: t = ((v0 - x) x e) / (d x e), e = v1 - v0, dt/dv1 = (-w_y, w_x),
//  dt/dv0 = (e_y, -e_x) / (d x e) - dt/dv1).  The flags and the adjacency are
// not differentiated: gradients flow only through q of the hit face.
//
// Determinism without float atomics: links are grouped by face with a stable
// LSD radix sort (keys = face ids, values = link indices, so each face's links
// stay in ascending link order); one warp per face accumulates its links'
// contributions, lane j the links j, j + 32, ... of that order (double-float
// sums), then a fixed shuffle tree adds the lanes.  For indexed input the face
// corners are grouped by vertex the same way (once per load) and one thread
// per vertex sums its corners in ascending (face, corner) order.
#include "internal.cuh"

namespace amr {

namespace {

constexpr int kRThreads = 256;
constexpr int kRWarps = kRThreads / 32;
constexpr int kRItems = 16;                       // keys per thread
constexpr int kRTile = kRThreads * kRItems;       // 4096 keys per tile
constexpr int kRBits = 8;
constexpr int kRDigits = 1 << kRBits;

// Per tile: digit histogram, written digit-major so that one exclusive scan
// over [digit][tile] gives every (digit, tile) its output base.
__global__ void __launch_bounds__(kRThreads) k_radix_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                                          uint32_t* __restrict__ hist, int64_t n_tiles) {
  __shared__ uint32_t h[kRDigits];
  for (int i = threadIdx.x; i < kRDigits; i += kRThreads) h[i] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kRTile;
  for (int i = threadIdx.x; i < kRTile; i += kRThreads) {
    const int64_t j = base + i;
    if (j < n) atomicAdd(&h[(keys[j] >> shift) & (kRDigits - 1)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kRDigits; i += kRThreads) hist[(int64_t)i * n_tiles + blockIdx.x] = h[i];
}

// Stable scatter of one tile: warp w owns keys [w*512, (w+1)*512) of the tile;
// per-warp digit counts are prefixed across warps, then each warp walks its
// keys 32 at a time in order, ranking equal digits with __match_any_sync.
// vals_in null: the values are the keys' indices; keys_out null: keys not kept.
__global__ void __launch_bounds__(kRThreads) k_radix_scatter(const uint32_t* __restrict__ keys_in,
                                                             const uint32_t* __restrict__ vals_in, int64_t n, int shift,
                                                             const uint32_t* __restrict__ offs, int64_t n_tiles,
                                                             uint32_t* __restrict__ keys_out,
                                                             uint32_t* __restrict__ vals_out) {
  __shared__ uint32_t cnt[kRWarps][kRDigits];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kRWarps * kRDigits; i += kRThreads) (&cnt[0][0])[i] = 0;
  __syncthreads();
  const int64_t wbase = (int64_t)blockIdx.x * kRTile + (int64_t)wid * (kRTile / kRWarps);
  constexpr int kChunks = kRTile / kRWarps / 32;
  for (int c = 0; c < kChunks; ++c) {
    const int64_t j = wbase + c * 32 + lane;
    if (j < n) atomicAdd(&cnt[wid][(keys_in[j] >> shift) & (kRDigits - 1)], 1u);
  }
  __syncthreads();
  // exclusive prefix over warps per digit, plus the global base of (digit, tile)
  for (int d = threadIdx.x; d < kRDigits; d += kRThreads) {
    uint32_t run = offs[(int64_t)d * n_tiles + blockIdx.x];
    for (int w = 0; w < kRWarps; ++w) {
      const uint32_t c = cnt[w][d];
      cnt[w][d] = run;
      run += c;
    }
  }
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  for (int c = 0; c < kChunks; ++c) {
    const int64_t j = wbase + c * 32 + lane;
    const bool ok = j < n;
    const unsigned active = __ballot_sync(0xffffffffu, ok);
    uint32_t k = 0, v = 0, d = 0;
    if (ok) {
      k = keys_in[j];
      v = vals_in ? vals_in[j] : (uint32_t)j;  // no input values: the key's own index
      d = (k >> shift) & (kRDigits - 1);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, ok ? d : 0xffffffffu) & active;
    if (ok) {
      const uint32_t pos = cnt[wid][d] + __popc(peers & lt);
      if (keys_out) keys_out[pos] = k;
      vals_out[pos] = v;
    }
    __syncwarp();
    if (ok && (peers & lt) == 0) cnt[wid][d] += __popc(peers);
    __syncwarp();
  }
}

__global__ void k_iota(uint32_t* __restrict__ v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = (uint32_t)i;
}

__global__ void k_count_keys(const uint32_t* __restrict__ keys, int64_t n, uint32_t* __restrict__ cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[keys[i]], 1u);
}

__device__ __forceinline__ void acc2(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bb = s - hi;
  lo += (hi - (s - bb)) + (x - bb);
  hi = s;
}

__constant__ int c_dirs19[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},
                                    {0, 0, 1},  {0, 0, -1},  {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},
                                    {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                    {0, 1, 1},  {0, -1, -1}, {0, 1, -1},  {0, -1, 1}};
__constant__ int c_dirs9[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1}, {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};

// One warp per face: lane j sums grad_q * dt/dv_k over the face's links j,
// j + 32, ... of its ascending link list (double-float), then a fixed shuffle
// tree adds the lanes' sums into lane 0, which writes grad_face[f][k][c].  The
// order of every addition is fixed by the face's link list, so the result is
// the same bit for bit on every run.
template <int D>
__global__ void __launch_bounds__(256) k_face_grad(AdjointArgs a) {
  constexpr int NC = D == 3 ? 64 : 16;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t f = w0; f < a.nf; f += nw) {
    float hi[D * D], lo[D * D];
#pragma unroll
    for (int j = 0; j < D * D; ++j) hi[j] = lo[j] = 0.f;
    float V[D * D];
#pragma unroll
    for (int j = 0; j < D * D; ++j) V[j] = a.X[(int64_t)j * a.nf + f];
    const uint32_t b0 = a.face_off[f], b1 = a.face_off[f + 1];
    if (b1 == b0) {
      if (lane < D * D) a.grad_face[(int64_t)f * D * D + lane] = 0.f;
      continue;
    }
    // links of this face live on the finest level of its geometry
    const GeomParams& P = a.table ? a.table[a.face_gid ? a.face_gid[f] : 0u] : a.g0;
    const int Lf = P.n_levels - 1;
    const FastGeom fg = fast_geom(P, Lf);
    const int32_t* blocks = a.level_blocks[Lf];
    for (uint32_t s = b0 + (uint32_t)lane; s < b1; s += 32u) {
      const uint32_t l = a.face_links[s];
      const float gq = a.grad_q[l];
      const uint32_t cellrow = a.link_cell[l];
      const int dir = a.link_dir[l];
      const float t = a.link_q[l];
      const uint32_t id = a.adj_cell[cellrow];
      const uint32_t blk = id / NC, bit = id % NC;
      // vertex offsets from the cell centre (double-float, rounded once)
      float p[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
#pragma unroll
      for (int c = 0; c < D; ++c) {
        const int g = 4 * blocks[(int64_t)blk * D + c] + (int)((bit >> (2 * c)) & 3u);
        float ohi, olo;
        df_position(P.org_hi[c], P.org_lo[c], (float)(2 * g + 1), 0.5f * fg.h_hi, 0.5f * fg.h_lo, ohi, olo);
#pragma unroll
        for (int k = 0; k < D; ++k) p[k][c] = (V[D * k + c] - ohi) - olo;
      }
      const float h32 = fg.h_hi;
      if constexpr (D == 3) {
        const float dv[3] = {c_dirs19[dir][0] * h32, c_dirs19[dir][1] * h32, c_dirs19[dir][2] * h32};
        const float nh[3] = {a.nrm[f], a.nrm[a.nf + f], a.nrm[2 * a.nf + f]};
        const float nl[3] = {a.nrm[3 * a.nf + f], a.nrm[4 * a.nf + f], a.nrm[5 * a.nf + f]};
        const float den = h32 * ((c_dirs19[dir][0] * nh[0] + c_dirs19[dir][1] * nh[1] + c_dirs19[dir][2] * nh[2]) +
                                 (c_dirs19[dir][0] * nl[0] + c_dirs19[dir][1] * nl[1] + c_dirs19[dir][2] * nl[2]));
        if (den == 0.f) continue;
        const float inv = 1.0f / den;
        const float e1[3] = {V[3] - V[0], V[4] - V[1], V[5] - V[2]};
        const float e2[3] = {V[6] - V[0], V[7] - V[1], V[8] - V[2]};
        const float w[3] = {(p[0][0] - t * dv[0]) * inv, (p[0][1] - t * dv[1]) * inv, (p[0][2] - t * dv[2]) * inv};
        const float g1[3] = {e2[1] * w[2] - e2[2] * w[1], e2[2] * w[0] - e2[0] * w[2], e2[0] * w[1] - e2[1] * w[0]};
        const float g2[3] = {w[1] * e1[2] - w[2] * e1[1], w[2] * e1[0] - w[0] * e1[2], w[0] * e1[1] - w[1] * e1[0]};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float g0 = (nh[c] + nl[c]) * inv - g1[c] - g2[c];
          acc2(hi[c], lo[c], gq * g0);
          acc2(hi[3 + c], lo[3 + c], gq * g1[c]);
          acc2(hi[6 + c], lo[6 + c], gq * g2[c]);
        }
      } else {
        const float dv[2] = {c_dirs9[dir][0] * h32, c_dirs9[dir][1] * h32};
        const float e[2] = {V[2] - V[0], V[3] - V[1]};
        const float den = dv[0] * e[1] - dv[1] * e[0];
        if (den == 0.f) continue;
        const float inv = 1.0f / den;
        const float w[2] = {(p[0][0] - t * dv[0]) * inv, (p[0][1] - t * dv[1]) * inv};
        const float g1[2] = {-w[1], w[0]};
        const float g0[2] = {e[1] * inv - g1[0], -e[0] * inv - g1[1]};
        acc2(hi[0], lo[0], gq * g0[0]);
        acc2(hi[1], lo[1], gq * g0[1]);
        acc2(hi[2], lo[2], gq * g1[0]);
        acc2(hi[3], lo[3], gq * g1[1]);
      }
    }
    // lanes' double-float sums into lane 0 (fixed tree)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
      for (int j = 0; j < D * D; ++j) {
        const float ph = __shfl_down_sync(0xffffffffu, hi[j], o);
        const float pl = __shfl_down_sync(0xffffffffu, lo[j], o);
        acc2(hi[j], lo[j], ph);
        lo[j] += pl;
      }
    }
    float out = 0.f;
#pragma unroll
    for (int j = 0; j < D * D; ++j) {
      const float v = __shfl_sync(0xffffffffu, hi[j] + lo[j], 0);
      if (lane == j) out = v;
    }
    if (lane < D * D) a.grad_face[(int64_t)f * D * D + lane] = out;
  }
}

// One thread per vertex: sum of its face corners' gradients in ascending (face, corner) order.
template <int D>
__global__ void k_vertex_grad(const float* __restrict__ grad_face, const uint32_t* __restrict__ vert_off,
                              const uint32_t* __restrict__ vert_corners, int64_t nv, float* __restrict__ out) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < nv; v += (int64_t)gridDim.x * blockDim.x) {
    float hi[D], lo[D];
#pragma unroll
    for (int c = 0; c < D; ++c) hi[c] = lo[c] = 0.f;
    for (uint32_t s = vert_off[v]; s < vert_off[v + 1]; ++s) {
      const uint32_t corner = vert_corners[s];  // f * D + k
#pragma unroll
      for (int c = 0; c < D; ++c) acc2(hi[c], lo[c], grad_face[(int64_t)corner * D + c]);
    }
#pragma unroll
    for (int c = 0; c < D; ++c) out[v * D + c] = hi[c] + lo[c];
  }
}

inline int grid_1d(int64_t n, int threads = 256) {
  int64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  const int64_t cap = (int64_t)current_sm_count() * 32;
  if (g > cap) g = cap;
  return (int)g;
}

}  // namespace

size_t radix_sort_scratch_bytes(int64_t n) {
  const int64_t tiles = (n + kRTile - 1) / kRTile;
  const int64_t nh = (tiles > 0 ? tiles : 1) * kRDigits;
  // hist + offsets (nh + 1 each) + ping-pong keys/values (2n each) + scan scratch
  return (size_t)(2 * (nh + 1)) * 4 + (size_t)(4 * (n > 0 ? n : 1)) * 4 + scan_u32_scratch_bytes(nh) + 256;
}

int launch_stable_sort(const uint32_t* keys, int64_t n, int key_bits, uint32_t* sorted_keys, uint32_t* sorted_vals,
                       const uint32_t* vals_in, void* scratch, uint64_t* total, unsigned* err, cudaStream_t st) {
  // vals_in == nullptr: values are 0..n-1
  if (n <= 0) return 0;
  const int64_t tiles = (n + kRTile - 1) / kRTile;
  const int64_t nh = tiles * kRDigits;
  char* s = static_cast<char*>(scratch);
  uint32_t* hist = reinterpret_cast<uint32_t*>(s);
  uint32_t* offs = hist + (nh + 1);
  uint32_t* ka = offs + (nh + 1);
  uint32_t* va = ka + n;
  uint32_t* kb = va + n;
  uint32_t* vb = kb + n;
  void* scan_scr = reinterpret_cast<void*>(((uintptr_t)(vb + n) + 255) & ~(uintptr_t)255);
  int launches = 0;
  int passes = (key_bits + kRBits - 1) / kRBits;
  if (passes < 1) passes = 1;
  // the first pass reads the caller's keys (and values, or the indices), the last writes the
  // caller's outputs; the passes between ping-pong through the scratch
  const uint32_t* kin = keys;
  const uint32_t* vin = vals_in;
  for (int p = 0; p < passes; ++p) {
    const int shift = p * kRBits;
    const bool last = p == passes - 1;
    uint32_t* kout = last ? sorted_keys : (p % 2 == 0 ? kb : ka);
    uint32_t* vout = last ? sorted_vals : (p % 2 == 0 ? vb : va);
    k_radix_hist<<<(unsigned)tiles, kRThreads, 0, st>>>(kin, n, shift, hist, tiles);
    launches += 1 + launch_scan_u32(hist, offs, nh, total, scan_scr, err, st);
    k_radix_scatter<<<(unsigned)tiles, kRThreads, 0, st>>>(kin, vin, n, shift, offs, tiles, kout, vout);
    ++launches;
    kin = kout;
    vin = vout;
  }
  return launches;
}

int launch_count_keys(const uint32_t* keys, int64_t n, uint32_t* cnt, cudaStream_t st) {
  if (n <= 0) return 0;
  k_count_keys<<<grid_1d(n), 256, 0, st>>>(keys, n, cnt);
  return 1;
}

int launch_face_grad(const AdjointArgs& a, cudaStream_t st) {
  if (a.nf <= 0) return 0;
  // one warp per face, 8 warps per block
  if (a.dim == 3)
    k_face_grad<3><<<grid_1d(a.nf, 8), 256, 0, st>>>(a);
  else
    k_face_grad<2><<<grid_1d(a.nf, 8), 256, 0, st>>>(a);
  return 1;
}

int launch_vertex_grad(int dim, const float* grad_face, const uint32_t* vert_off, const uint32_t* vert_corners,
                       int64_t nv, float* out, cudaStream_t st) {
  if (nv <= 0) return 0;
  if (dim == 3)
    k_vertex_grad<3><<<grid_1d(nv), 256, 0, st>>>(grad_face, vert_off, vert_corners, nv, out);
  else
    k_vertex_grad<2><<<grid_1d(nv), 256, 0, st>>>(grad_face, vert_off, vert_corners, nv, out);
  return 1;
}

}  // namespace amr
