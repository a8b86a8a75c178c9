// internal.cuh — device helpers and kernel launchers shared by the CUDA sources
// of the near-wall refinement library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace amr {

constexpr float kU32 = 5.9604644775390625e-8f;  // FP32 unit roundoff 2^-24
constexpr double kBandRel = 1e-6;               // margin band of the adjacency (x h) and link tests
constexpr int kMaxFaces = 1 << 29;              // face ids keep 3 flag bits in the bin payload
constexpr uint32_t kIdMask = (1u << 29) - 1u;
constexpr long long kSpinLimit = 1ll << 24;     // bounded waits: iterations before giving up
constexpr int kMaxLevels = 16;                  // grid levels at most (the C ABI's AMR_MAX_LEVELS)

// device error word bits
enum : unsigned {
  ERR_TIMEOUT = 1u,
  ERR_OVERFLOW = 2u,
  ERR_BADINDEX = 4u,
  ERR_NONFINITE = 8u,
};

// diagnostic counters (device, u64 each)
enum : int {
  CNT_FALLBACK = 0,
  CNT_BAND = 1,
  CNT_CANDIDATES = 2,
  CNT_SURVIVORS = 3,
  CNT_LINK_FALLBACK = 4,
  CNT_LINK_BAND = 5,
  CNT_LINK_CAND = 6,
  CNT_CLASS_FALLBACK = 7,
  CNT_FACE_SETUPS = 8,  // faces set up by the face-centric marking
  CNT_FACE_TESTS = 9,   // (face, cell) tests run by it
  CNT_BIG_BLOCKS = 10,  // finest blocks with more survivor records than shared memory stages
  CNT_N = 11,
};

// Per-geometry parameters.  A launch may cover the blocks (faces) of many
// geometries; each block (face) then carries its geometry id and reads its
// row of this table.  Single-geometry launches pass one row by value.
//   domain box   origin[a] + [0, 4 root[a] h0], level-L cell size h0 2^-L
//   bins         bin of x along a = clamp(floor((x - origin[a]) * bin_scale[a]), 0, B - 1)
//                (FP64), global bin index = bin_base + bx + B (by + B bz)
//   distance     d_L = d_abs + d_rel h_L
struct GeomParams {
  double origin[3];
  double h0;
  double d_abs, d_rel;
  double bin_scale[3];
  int B;
  int n_levels;
  int root[3];
  uint32_t face_levels;  // bit L: this geometry's mask-only blocks of level L are marked face by face
  int64_t bin_base;
  int64_t root_base;   // first level-0 block of this geometry in the concatenated list
  int64_t face_base;   // first face of this geometry in the concatenated face arrays
  // FP32 forms for the hot loops: h0 and origin as unevaluated pairs hi + lo,
  // the bin scale and the distance coefficients rounded once
  float h0_hi, h0_lo;
  float org_hi[3], org_lo[3];
  float scale32[3];
  float d_abs32, d_rel32;
};

__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void df_two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf(a, b, -p);
}

// origin + k * h as an unevaluated FP32 pair hi + lo (k an integer below 2^24,
// h = h_hi + h_lo): relative error about 2^-46, so the hi part is the
// position rounded to FP32 and lo its rounding error.
__device__ __forceinline__ void df_position(float org_hi, float org_lo, float k, float h_hi, float h_lo, float& hi,
                                            float& lo) {
  float p, e, s, t;
  df_two_prod(k, h_hi, p, e);
  df_two_sum(org_hi, p, s, t);
  const float rest = t + e + fmaf(k, h_lo, org_lo);
  df_two_sum(s, rest, hi, lo);
}

// Level-L quantities of a geometry in FP32: h_L = 2^-L h0 (exact scaling of
// both parts) and d_L = d_abs + d_rel h_L (a few ulps).
struct FastGeom {
  float h_hi, h_lo, d;
};

__device__ __forceinline__ FastGeom fast_geom(const GeomParams& P, int level) {
  FastGeom g;
  g.h_hi = ldexpf(P.h0_hi, -level);
  g.h_lo = ldexpf(P.h0_lo, -level);
  g.d = fmaf(P.d_rel32, g.h_hi, P.d_abs32);
  return g;
}

// Geometry of one block on one level, derived from its table row.
struct LevelGeom {
  double origin[3];
  double h, d;
  double scale[3];
  int B;
  int64_t bin_base;
  bool finest;
};

__device__ __forceinline__ LevelGeom level_geom(const GeomParams& P, int level) {
  LevelGeom g;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    g.origin[a] = P.origin[a];
    g.scale[a] = P.bin_scale[a];
  }
  g.h = scalbn(P.h0, -level);
  g.d = __dadd_rn(P.d_abs, __dmul_rn(P.d_rel, g.h));
  g.B = P.B;
  g.bin_base = P.bin_base;
  g.finest = level == P.n_levels - 1;
  return g;
}

// Table row of item i: the by-value row for single-geometry launches.
__device__ __forceinline__ GeomParams geom_row(const GeomParams& g0, const GeomParams* table, const uint32_t* gid,
                                               int64_t i) {
  if (!table) return g0;
  return table[gid ? gid[i] : 0u];
}

// Bin-grid parameters of one geometry (kept for the allocation-free binning entry).
struct BinGrid {
  int B;
  double origin[3];
  double scale[3];
};

// One bin entry with its face's coordinates (and, in 3D, the FP32 face
// normal), so that a bin's faces are one contiguous run of memory that TMA
// bulk copies stage in shared memory.  `id` holds the face id in the low 29
// bits and, in bits 29..31, whether this bin is the first of the face's bin
// range along x / y / z; with the entry's own bin coordinates that lets a
// query box visit each face once (in the first of its bins inside the box).
struct __align__(16) Entry3 {
  float v[9];
  float n[3];
  uint32_t id;
  uint32_t bin[3];  // this entry's bin coordinates (within its geometry's grid)
};
struct __align__(16) Entry2 {
  float v[4];
  uint32_t id;
  uint32_t bin[3];  // bin x, y; bin[2] = 0
};

template <int D>
struct EntryT;
template <>
struct EntryT<3> {
  using type = Entry3;
};
template <>
struct EntryT<2> {
  using type = Entry2;
};

__device__ __forceinline__ int bin_coord(double x, double o, double s, int B) {
  const double t = floor(__dmul_rn(__dsub_rn(x, o), s));
  if (!(t >= 0.0)) return 0;
  if (t > (double)(B - 1)) return B - 1;
  return (int)t;
}

// The same bin coordinate, decided in FP32 where that is certain.  The FP32
// estimate t = ((x - o_hi) - o_lo) * s32 differs from (x - o) s by less than
// 5u (|x| + |o|) |s|, and the FP64 value above by no more than that plus a few
// FP64 ulps; when t lies farther than 8u (|x| + |o|) |s| from every integer,
// both floors agree.  Otherwise (and for non-finite input) the FP64 formula
// decides, so the result is always that of bin_coord.
__device__ __forceinline__ int bin_coord_fast(float x, const GeomParams& P, int c) {
  const float d = (x - P.org_hi[c]) - P.org_lo[c];
  const float t = d * P.scale32[c];
  const float err = 8.0f * kU32 * (fabsf(x) + fabsf(P.org_hi[c])) * fabsf(P.scale32[c]);
  const float k = floorf(t);
  if (t - k > err && (k + 1.0f) - t > err) {
    if (!(k >= 0.0f)) return 0;
    if (k > (float)(P.B - 1)) return P.B - 1;
    return (int)k;
  }
  return bin_coord((double)x, P.origin[c], P.bin_scale[c], P.B);
}

__device__ __forceinline__ uint64_t ld_volatile_u64(const uint64_t* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}

// Decoupled look-back over ticket-ordered tiles (single-pass prefix sums).
// state[t] = flag(2 bits: 1 aggregate, 2 inclusive prefix) << 62 | value.
// Called by one whole warp of the CTA with the tile's aggregate (all lanes the
// same value); every lane returns the tile's exclusive prefix.  The warp reads
// the 32 preceding tiles' states at once: when all tiles after the nearest
// inclusive one have published, their aggregates and that prefix are summed
// (one round trip for the common case); without an inclusive one in the
// window, the window moves 32 tiles back.  A wait that exceeds kSpinLimit polls
// sets ERR_TIMEOUT and returns what it has (the caller's output is then
// invalid, and the host reports AMR_ETIMEOUT).
__device__ __forceinline__ uint64_t lookback_warp(uint64_t* state, long long tile, uint64_t aggregate,
                                                  unsigned* err) {
  constexpr uint64_t kAgg = 1ull << 62, kInc = 2ull << 62, kVal = (1ull << 62) - 1;
  const int lane = threadIdx.x & 31;
  if (tile == 0) {
    if (lane == 0)
      atomicExch(reinterpret_cast<unsigned long long*>(state), (unsigned long long)(kInc | (aggregate & kVal)));
    return 0;
  }
  if (lane == 0)
    atomicExch(reinterpret_cast<unsigned long long*>(state + tile), (unsigned long long)(kAgg | (aggregate & kVal)));
  uint64_t prefix = 0;
  long long base = tile - 1;  // lane l looks at tile base - l
  long long spins = 0;
  for (;;) {
    const long long t = base - lane;
    const uint64_t s = t >= 0 ? ld_volatile_u64(state + t) : kInc;  // before tile 0: prefix 0
    const uint32_t f = (uint32_t)(s >> 62);
    const unsigned inc = __ballot_sync(0xffffffffu, f == 2u);
    const int first = inc ? __ffs(inc) - 1 : 32;  // nearest tile with an inclusive prefix
    if (__ballot_sync(0xffffffffu, f == 0u && lane <= first)) {
      if (++spins > kSpinLimit) {
        if (lane == 0) atomicOr(err, ERR_TIMEOUT);
        break;
      }
      __nanosleep(20);
      continue;
    }
    uint64_t v = lane <= first ? (s & kVal) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    prefix += v;
    if (first < 32) break;
    base -= 32;
  }
  if (lane == 0)
    atomicExch(reinterpret_cast<unsigned long long*>(state + tile),
               (unsigned long long)(kInc | ((prefix + aggregate) & kVal)));
  return prefix;
}

// --- block-coordinate hash (open addressing, linear probing) --------------
// Key: the geometry id above the block's coordinates, cb bits per axis, plus
// one (0 marks an empty slot); value: the block's index in its level's list.
__device__ __forceinline__ unsigned long long block_key_g(uint32_t gid, const int32_t* c, int dim, int cb) {
  unsigned long long k = gid;
  const uint32_t m = (1u << cb) - 1u;
  for (int a = 0; a < dim; ++a) k = (k << cb) | (unsigned long long)((uint32_t)c[a] & m);
  return k + 1ull;
}
__device__ __forceinline__ unsigned long long block_key(const int32_t* c, int dim) {
  return block_key_g(0u, c, dim, 21);
}

__device__ __forceinline__ uint32_t hash_slot(unsigned long long k, uint32_t mask) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  return (uint32_t)k & mask;
}

// Index stored for key k, or -1.
__device__ __forceinline__ int64_t hash_find(const unsigned long long* keys, const uint32_t* vals, uint32_t hmask,
                                             unsigned long long k) {
  uint32_t s = hash_slot(k, hmask);
  for (uint32_t probe = 0; probe <= hmask; ++probe) {
    const unsigned long long v = keys[s];
    if (v == k) return (int64_t)vals[s];
    if (v == 0ull) return -1;
    s = (s + 1) & hmask;
  }
  return -1;
}

// --- shared-memory barriers and TMA bulk copies (inline PTX, sm_90+) -------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16)
// completing on `bar` with its byte count.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for a barrier phase.  On timeout: flag ERR_TIMEOUT, then wait
// once more (bounded) so that a copy still in flight lands before the caller
// moves on; returns false after a timeout (the caller's results are invalid
// and the host reports AMR_ETIMEOUT).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned* err) {
  for (long long i = 0; i < kSpinLimit; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (i > 32) __nanosleep(32);
  }
  atomicOr(err, ERR_TIMEOUT);
  for (long long i = 0; i < kSpinLimit; ++i) {
    if (mbar_try_wait(bar, parity)) break;
    __nanosleep(64);
  }
  return false;
}

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T n = __shfl_up_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) >= o) v += n;
  }
  return v;
}

// ---------------------------------------------------------------------------
// Launchers (host side).  All are asynchronous on `st` and return the number
// of kernels they launched.  Sizes marked "device" are read by the kernels
// from device memory (so that launches can be captured in a CUDA graph before
// the sizes are known); the host passes a capacity instead.
// ---------------------------------------------------------------------------
// Streaming multiprocessors of the current device (queried once per device);
// grids of the grid-stride kernels are capped at a multiple of it.
int current_sm_count();
// Gather nf faces into the SoA array X (row stride ld, default nf) starting at face f0.
int launch_load_indexed(int dim, const float* verts, int64_t nv, const int32_t* idx, int64_t nf, float* X,
                        unsigned* err, cudaStream_t st, int64_t ld = -1, int64_t f0 = 0);
int launch_load_facelist(int dim, const float* coords, int64_t nf, float* X, unsigned* err, cudaStream_t st,
                         int64_t ld = -1, int64_t f0 = 0);
// Packed 3D face record for the link kernel: vertices, then the double-float
// normal (hi, lo); 64 bytes, read as four 16-byte loads.
struct __align__(16) FaceRec3 {
  float v[9];
  float nh[3];
  float nl[3];
  float pad;
};
static_assert(sizeof(FaceRec3) == 64, "face record is 64 bytes");

// nrm[6][nf] (hi.xyz, lo.xyz) and the packed records rec[nf] (nullable).
int launch_face_normals(const float* X, int64_t nf, float* nrm, FaceRec3* rec, cudaStream_t st);

// Faces of one or many geometries: face_gid (nullable) selects the table row.
struct FaceBinArgs {
  int dim;
  const float* X;
  int64_t nf;
  GeomParams g0;
  const GeomParams* table;
  const uint32_t* face_gid;
  uint32_t* frange;
  uint32_t* count;
  int sampled;                 // 1: the paper's sampled-point membership (single geometry)
  double sample_s;             // sample spacing (half a bin length)
  unsigned long long* fstat;   // nullable, per geometry g: [2g] max over its faces of the largest AABB
                               // side / h0 (FP32 bits), [2g + 1] the sum of that ratio, fixed point
                               // 2^-16 (zeroed before)
};
int launch_face_bins(const FaceBinArgs& a, cudaStream_t st);
int launch_face_bins(int dim, const float* X, int64_t nf, const BinGrid& g, uint32_t* frange, uint32_t* count,
                     cudaStream_t st);
struct ScatterArgs {
  FaceBinArgs f;
  const uint32_t* offsets;
  uint32_t* ids;
  void* payload;
  const FaceRec3* rec;      // 3D face records (vertices and normal copied into the entries)
};
int launch_scatter(const ScatterArgs& a, cudaStream_t st);

// Exclusive scans (single pass, decoupled look-back).  u32: out[n] = total
// (low 32 bits), *total64 = the full total.  u64: n_dev (nullable) gives the
// element count on the device, n the capacity.
size_t scan_u32_scratch_bytes(int64_t n);
int launch_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint64_t* total64, void* scratch, unsigned* err,
                    cudaStream_t st);
size_t scan_u64_scratch_bytes(int64_t n);
int launch_scan_u64(const uint64_t* in, uint64_t* out, int64_t n, const uint64_t* n_dev, uint64_t* total,
                    void* scratch, unsigned* err, int num_sms, cudaStream_t st);

// Survivor record of a block whose geometry ends at its level: a face that
// meets some cell of the block and the mask of those cells (bit i = cell i).
struct __align__(16) SurvRec {
  uint32_t face;
  uint32_t pad;
  uint64_t cells;
};
constexpr int kRecCap = 64;     // records of a block staged in shared memory
constexpr int kSpillCap = 960;  // more, up to this many, go to the warp's spill area (when given);
                                // a block with still more records is walked again for its lists

struct RefineLevel {
  int dim;
  int level;
  GeomParams g0;
  const GeomParams* table;     // null: every block uses g0
  const uint32_t* gid;         // per-block geometry id (null: 0)
  const int32_t* blocks;
  int64_t n_blocks;            // count, or capacity when n_dev is set
  const uint64_t* n_dev;       // device block count (nullable)
  const uint32_t* offsets;
  const void* payload;
  const float* X;
  const float* nrm;
  int64_t nf;
  uint64_t* mask;
  uint8_t* flag;
  uint16_t* cellcnt;           // per cell face count, blocks whose geometry ends at this level
  uint64_t* blockcnt;          // per block pairs | adjacent cells << 32 (0 for the others)
  SurvRec* recs;               // survivor records (nullable), capacity cap_recs
  int64_t cap_recs;
  uint64_t* rec_count;         // device: records handed out on this level
  uint64_t* rec_desc;          // per block: offset << 16 | count, or ~0 (records incomplete)
  SurvRec* spill;              // nullable: kSpillCap records per warp of the launch (records past kRecCap)
  unsigned long long* counters;
  unsigned* work;              // dynamic work counter (zeroed before launch)
  unsigned* err;
  int warps;                   // warps per CTA (tunable)
  int pred;                    // adjacency predicate: 0 box (SAT of the inflated cell), 1 point (Alg. 1)
  int search;                  // candidates: 0 the bins of the inflated query box, 1 the cell's own bin (point only)
  int batch;                   // consecutive blocks a warp takes per work fetch (1..kMaxBatch)
  int skip_mark_only;          // 1: blocks of geometries with this level's face_levels bit were marked
                               // face by face; the walk takes only the others
};
constexpr int kMaxBatch = 8;
int launch_refine(const RefineLevel& a, int num_sms, cudaStream_t st);
// Levels that launch_refine marks by parent groups (one warp per marked parent's 8
// children): 3D box predicate, whole-query-box search, below the roots.  The
// finest such level then always stages survivor records past shared memory in
// the spill area.
inline bool refine_by_groups(int dim, int level, int pred, int search) {
  return dim == 3 && level > 0 && pred == 0 && search == 0;
}

// Face-by-face marking of the blocks of a level whose only output is the mask
// (box or point predicate, whole-domain search): lv.mask / lv.flag zeroed and
// lv.work zeroed before the launch; blocks found through the level-0 root
// order or, deeper, by descending from the root through the first-child arrays.
// With a geometry table (lv.table) every face reads its row through face_gid;
// only faces whose geometry has this level's face_levels bit are marked.
struct MarkArgs {
  RefineLevel lv;
  const FaceRec3* rec;  // 3D face records (2D reads lv.X)
  const uint32_t* face_gid;
  // per level l < lv.level: the first-child index of each block (-1: none), so that a
  // block of this level is found from its root by one step per level
  const int32_t* first_child[kMaxLevels];
  int batch;            // faces a warp takes per work fetch (1..kFaceBatch)
};
constexpr int kFaceBatch = 8;  // most faces a warp takes per work fetch
int launch_mark_faces(const MarkArgs& m, int num_sms, cudaStream_t st);

// The algorithmic cell-face test count of one level (single geometry): per cell
// of its blocks, the distinct faces in the bins its inflated box overlaps,
// summed into *out.
struct CountArgs {
  int dim;
  int level;
  GeomParams g0;
  const int32_t* blocks;
  int64_t n;                 // blocks of the level
  const uint32_t* offsets;
  const void* payload;
  unsigned long long* out;
};
int launch_count_candidates(const CountArgs& a, int num_sms, cudaStream_t st);

struct EmitArgs {
  RefineLevel lv;
  const uint64_t* block_base;  // exclusive scan of blockcnt over this level
  const uint64_t* run;         // device running totals before this level: [0] cells, [1] pairs
  uint32_t* adj_cell;
  uint32_t* adj_off;
  uint32_t* adj_ids;
  int64_t cap_cells, cap_pairs;
  uint32_t* defer;             // blocks for the second pass (capacity defer_cap) ...
  unsigned* defer_n;           // ... and their count (zeroed before the launch)
  int64_t defer_cap;
};
// Both passes (the work counter zeroed before the launch; it is reused by the second).
int launch_adjacency(const EmitArgs& a, int num_sms, cudaStream_t st);

struct ChildrenArgs {
  int dim;
  int level;
  GeomParams g0;
  const GeomParams* table;
  const uint32_t* gid;
  const int32_t* blocks;
  const uint64_t* mask;
  const uint8_t* flag;         // nullable: marked for refinement (flag != 0) instead of mask != 0
  int64_t n;                   // count, or capacity when n_dev is set
  const uint64_t* n_dev;
  int32_t* child_blocks;
  uint32_t* child_gid;         // nullable
  int32_t* child_parent;
  int32_t* first_child;        // nullable: per block of this level, the index of its first child in the
                               // next level (its children follow in slot order), -1 without children
  int64_t cap_out;
  uint64_t* total;             // device: number of children (next level's count)
  unsigned* err;
};
size_t children_scratch_bytes(int64_t n);

// Node classification of the finest adjacent cells (rows [row0, row0 + n_rows) of
// the adjacency CSR): cls[row] = 1 solid (inside the closed mesh), 0 fluid.
struct ClassifyArgs {
  int dim;
  int level;
  GeomParams g0;
  const int32_t* blocks;       // the finest level's blocks
  const uint32_t* adj_cell;
  int64_t row0, n_rows;
  const uint32_t* offsets;     // exact bins
  const void* payload;
  const float* X;              // faces (SoA), for the winding-number fallback
  int64_t nf;
  uint8_t* cls;
  unsigned long long* counters;
  unsigned* err;
};
int launch_classify(const ClassifyArgs& a, cudaStream_t st);
// Stable compaction of the link arrays to the links of fluid cells.
int64_t fluid_blocks(int64_t n);
int launch_fluid_count(const uint32_t* link_cell, const uint8_t* cls, int64_t n, uint32_t* cnt, cudaStream_t st);
int launch_fluid_move(const uint32_t* link_cell, const uint8_t* link_dir, const float* link_q,
                      const uint32_t* link_face, const uint8_t* cls, int64_t n, const uint32_t* base,
                      uint32_t* o_cell, uint8_t* o_dir, float* o_q, uint32_t* o_face, cudaStream_t st);

// Mark propagation over one level (flags 0/1 in place): `rounds` two-phase rounds
// through a hash of the block coordinates (keys/vals: `slots` entries, a power of
// two >= 2 x capacity, from propagate_hash_slots; coordinates below 2^21).
uint32_t propagate_hash_slots(int64_t cap);
// Hash of a level's blocks (geometry id, coordinates) -> index (the count from n_dev when given,
// bounded by cap); gid nullable (single geometry), cb coordinate bits per axis of the key.
int launch_hash_build(int dim, const int32_t* blocks, const uint32_t* gid, int cb, int64_t cap,
                      const uint64_t* n_dev, unsigned long long* keys, uint32_t* vals, uint32_t slots,
                      unsigned* err, cudaStream_t st);
int launch_propagate(int dim, const int32_t* blocks, int64_t cap, const uint64_t* n_dev, uint8_t* flags,
                     int rounds, unsigned long long* keys, uint32_t* vals, uint32_t slots, unsigned* err,
                     cudaStream_t st);
// out[i] = index of query block i in the reference list, -1 if absent; *n_missing += the absent
// count (hash of `slots` >= 2 x max(n_ref) entries).
int launch_block_map(int dim, const int32_t* ref, int64_t n_ref, const int32_t* query, int64_t n_query,
                     int32_t* out, unsigned long long* n_missing, unsigned long long* keys, uint32_t* vals,
                     uint32_t slots, unsigned* err, cudaStream_t st);
int launch_children(const ChildrenArgs& a, void* scratch, int num_sms, cudaStream_t st);
// Level-0 blocks of every geometry of the table (x fastest within each), with their geometry ids.
int launch_root_blocks(int dim, const int* root, int32_t* blocks, int64_t n, cudaStream_t st);
int launch_root_blocks_multi(int dim, const GeomParams* table, int n_geom, int32_t* blocks, uint32_t* gid,
                             int64_t n, cudaStream_t st);
// Per-face geometry id from the table's face ranges.
int launch_face_gid(const GeomParams* table, int n_geom, int64_t nf, uint32_t* face_gid, cudaStream_t st);

struct LinkArgs {
  int dim;
  int lattice;
  int level;
  GeomParams g0;
  const GeomParams* table;
  const uint32_t* gid;         // per-block geometry ids of this level (nullable)
  const int32_t* blocks;       // this level's blocks
  const uint32_t* adj_cell;
  const uint32_t* adj_off;
  const uint32_t* adj_ids;
  const uint64_t* run;         // device running totals before this level: [0] rows, [2] links
  const uint64_t* level_tot;   // device: this level's pairs | cells << 32
  int64_t cap_rows;
  int64_t cap_pairs;           // capacity of adj_ids
  const float* X;               // 2D faces (SoA)
  const FaceRec3* rec;         // 3D face records
  int64_t nf;
  uint32_t* link_cell;
  uint8_t* link_dir;
  float* link_q;
  uint32_t* link_face;
  int64_t link_cap;
  void* stage;                 // staging area of links_stage_bytes(link_cap) bytes
  uint64_t* n_links;           // device: this level's link count
  unsigned long long* counters;
  unsigned* err;
};
size_t links_scratch_bytes(int64_t n_adj);
size_t links_stage_bytes(int64_t cap_links);
// Three kernels (links, the scan of the tiles' counts, placement); returns the launch count.
int launch_links(const LinkArgs& a, void* scratch, int num_sms, cudaStream_t st);
// close: adj_off[run[0] + cells] = run[1] + pairs (end marker of the level's rows);
// else: run[0] += cells, run[1] += pairs, run[2] += links (n_links nullable).
int launch_advance(const uint64_t* level_tot, const uint64_t* n_links, uint64_t* run, uint32_t* adj_off,
                   int64_t cap_cells, unsigned* err, bool close, cudaStream_t st);

struct AdjointArgs {
  int dim;
  int64_t nf;
  GeomParams g0;
  const GeomParams* table;
  const uint32_t* face_gid;    // nullable
  const int32_t* const* level_blocks;  // device array of per-level block pointers
  const float* X;
  const float* nrm;
  const uint32_t* face_off;    // [nf + 1]
  const uint32_t* face_links;  // link indices grouped by face, ascending within a face
  const float* grad_q;
  const uint32_t* link_cell;
  const uint8_t* link_dir;
  const float* link_q;
  const uint32_t* adj_cell;
  float* grad_face;            // [nf][D][D]
};
size_t radix_sort_scratch_bytes(int64_t n);
// Stable sort of n u32 keys (low key_bits significant); values default to 0..n-1
// (vals_in null); sorted_keys may be null when only the values are wanted.
int launch_stable_sort(const uint32_t* keys, int64_t n, int key_bits, uint32_t* sorted_keys, uint32_t* sorted_vals,
                       const uint32_t* vals_in, void* scratch, uint64_t* total, unsigned* err, cudaStream_t st);
int launch_count_keys(const uint32_t* keys, int64_t n, uint32_t* cnt, cudaStream_t st);
int launch_face_grad(const AdjointArgs& a, cudaStream_t st);
int launch_vertex_grad(int dim, const float* grad_face, const uint32_t* vert_off, const uint32_t* vert_corners,
                       int64_t nv, float* out, cudaStream_t st);

}  // namespace amr
