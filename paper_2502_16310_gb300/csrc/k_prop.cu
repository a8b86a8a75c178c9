// k_prop.cu — refinement-mark propagation over one level's block list.
//
// Paper (Sec. "Spatial Binning Algorithm", Fig. "propagation"): with binned
// face detection a cell can miss faces within the near-wall distance that lie
// in other bins, so blocks marked for refinement also mark their neighbouring
// blocks, N_prop = 1 + floor(d_spec / block length) times; each round goes
// through an intermediate value so that marks set in a round do not spread in
// the same round.  Neighbours are the 3^D - 1 blocks of the same level around a
// block that exist in the level's list, found through an open-addressing hash
// of the block coordinates built once per level.
#include "internal.cuh"

namespace amr {

namespace {

constexpr int kPThreads = 256;
constexpr unsigned long long kEmpty = 0ull;

__device__ __forceinline__ int64_t count_of(int64_t cap, const uint64_t* n_dev) {
  if (!n_dev) return cap;
  const int64_t n = (int64_t)*n_dev;
  return n < cap ? n : cap;
}

__global__ void k_hash_insert(int dim, const int32_t* __restrict__ blocks, const uint32_t* __restrict__ gid, int cb,
                              int64_t cap, const uint64_t* n_dev, unsigned long long* keys, uint32_t* vals,
                              uint32_t hmask, unsigned* err) {
  const int64_t n = count_of(cap, n_dev);
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = block_key_g(gid ? gid[b] : 0u, blocks + b * dim, dim, cb);
    uint32_t s = hash_slot(k, hmask);
    for (uint32_t probe = 0;; ++probe) {
      if (probe > hmask) {  // table full: cannot happen with twice the capacity
        atomicOr(err, ERR_OVERFLOW);
        break;
      }
      const unsigned long long prev = atomicCAS(keys + s, kEmpty, k);
      if (prev == kEmpty || prev == k) {
        vals[s] = (uint32_t)b;
        break;
      }
      s = (s + 1) & hmask;
    }
  }
}

// Round, first half: every marked block (flag 1) gives its unmarked existing
// neighbours the intermediate value 2.
__global__ void k_prop_mark(int dim, const int32_t* __restrict__ blocks, int64_t cap, const uint64_t* n_dev,
                            uint8_t* flags, const unsigned long long* keys, const uint32_t* vals, uint32_t hmask) {
  const int64_t n = count_of(cap, n_dev);
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < n; b += (int64_t)gridDim.x * blockDim.x) {
    if (flags[b] != 1) continue;
    const int32_t* c = blocks + b * dim;
    const int nz = dim == 3 ? 1 : 0;
    for (int dz = -nz; dz <= nz; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          if (dx == 0 && dy == 0 && dz == 0) continue;
          const int32_t q[3] = {c[0] + dx, c[1] + dy, dim == 3 ? c[2] + dz : 0};
          if (q[0] < 0 || q[1] < 0 || q[2] < 0) continue;
          const int64_t i = hash_find(keys, vals, hmask, block_key(q, dim));
          if (i >= 0 && flags[i] == 0) flags[i] = 2;
        }
  }
}

// Round, second half: intermediate values become marks.
__global__ void k_prop_commit(int64_t cap, const uint64_t* n_dev, uint8_t* flags) {
  const int64_t n = count_of(cap, n_dev);
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < n; b += (int64_t)gridDim.x * blockDim.x)
    if (flags[b] == 2) flags[b] = 1;
}

int grid_of(int64_t n) {
  int64_t g = (n + kPThreads - 1) / kPThreads;
  if (g < 1) g = 1;
  const int64_t cap = (int64_t)current_sm_count() * 8;
  if (g > cap) g = cap;
  return (int)g;
}

}  // namespace

uint32_t propagate_hash_slots(int64_t cap) {
  uint32_t s = 1024;
  while ((int64_t)s < 2 * cap && s < (1u << 31)) s <<= 1;
  return s;
}

int launch_hash_build(int dim, const int32_t* blocks, const uint32_t* gid, int cb, int64_t cap,
                      const uint64_t* n_dev, unsigned long long* keys, uint32_t* vals, uint32_t slots,
                      unsigned* err, cudaStream_t st) {
  if (cap <= 0) return 0;
  cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * slots, st);
  k_hash_insert<<<grid_of(cap), kPThreads, 0, st>>>(dim, blocks, gid, cb, cap, n_dev, keys, vals, slots - 1, err);
  return 1;
}

int launch_propagate(int dim, const int32_t* blocks, int64_t cap, const uint64_t* n_dev, uint8_t* flags,
                     int rounds, unsigned long long* keys, uint32_t* vals, uint32_t slots, unsigned* err,
                     cudaStream_t st) {
  if (rounds <= 0 || cap <= 0) return 0;
  cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * slots, st);
  const int g = grid_of(cap);
  k_hash_insert<<<g, kPThreads, 0, st>>>(dim, blocks, nullptr, 21, cap, n_dev, keys, vals, slots - 1, err);
  for (int r = 0; r < rounds; ++r) {
    k_prop_mark<<<g, kPThreads, 0, st>>>(dim, blocks, cap, n_dev, flags, keys, vals, slots - 1);
    k_prop_commit<<<g, kPThreads, 0, st>>>(cap, n_dev, flags);
  }
  return 1 + 2 * rounds;
}

}  // namespace amr

// ---------------------------------------------------------------------------
// Re-adaptation bookkeeping (moving geometry): between two successive
// hierarchies, per level, the index of every block of one list in the other
// list (-1: none).  new -> old = -1 marks a block created by refinement; old ->
// new = -1 a block removed by coarsening.  The same coordinate hash as above.
// ---------------------------------------------------------------------------
namespace amr {

namespace {

__global__ void k_map_lookup(int dim, const int32_t* __restrict__ query, int64_t n, const unsigned long long* keys,
                             const uint32_t* vals, uint32_t hmask, int32_t* out, unsigned long long* n_missing) {
  unsigned long long miss = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = hash_find(keys, vals, hmask, block_key(query + i * dim, dim));
    out[i] = (int32_t)j;
    miss += j < 0 ? 1ull : 0ull;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) miss += __shfl_xor_sync(0xffffffffu, miss, o);
  if ((threadIdx.x & 31) == 0 && miss) atomicAdd(n_missing, miss);
}

}  // namespace

int launch_block_map(int dim, const int32_t* ref, int64_t n_ref, const int32_t* query, int64_t n_query,
                     int32_t* out, unsigned long long* n_missing, unsigned long long* keys, uint32_t* vals,
                     uint32_t slots, unsigned* err, cudaStream_t st) {
  if (n_query <= 0) return 0;
  cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * slots, st);
  int k = 0;
  if (n_ref > 0) {
    k_hash_insert<<<grid_of(n_ref), kPThreads, 0, st>>>(dim, ref, nullptr, 21, n_ref, nullptr, keys, vals, slots - 1,
                                                        err);
    ++k;
  }
  k_map_lookup<<<grid_of(n_query), kPThreads, 0, st>>>(dim, query, n_query, keys, vals, slots - 1, out, n_missing);
  return k + 1;
}

}  // namespace amr
