// api.cu — host side of the C ABI declared in include/amrgeom.h.
//
// A context owns grow-only device buffers (stream-ordered allocations), small
// pinned host staging for the few device->host reads of sizes, and an optional
// per-kernel CUDA-event timing table.  One level engine serves both a single
// geometry and a batch of geometries (a geometry table plus a geometry id per
// block and per face): every level is one refine launch over the blocks of
// all geometries, one child compaction, and, where geometries end, one
// adjacency and one link launch.
//
// Two modes run the engine.  Eager mode learns the data-dependent sizes with a
// few device->host reads and grows the buffers.  Graph mode (after one eager
// call with the same inputs) replays the whole level loop as one captured CUDA
// graph whose kernels read their sizes from device memory and check them
// against the capacities of the eager call; only the final sizes are read
// back.  An overflow re-runs the call eagerly.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <algorithm>
#include <initializer_list>
#include <vector>

#include "amrgeom.h"
#include "internal.cuh"

using namespace amr;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

struct TimedLaunch {
  int slot;
  cudaEvent_t a, b;
};

struct TimingSlot {
  const char* name;
  double ms = 0.0;
  int64_t launches = 0;
};

struct LevelBufs {
  DevBuf blocks, gid, parent, mask, flag, cellcnt, blockcnt, base, desc;
  DevBuf first;           // per block: index of its first child in the next level, -1 without children
  DevBuf prev, n2o, o2n;  // previous call's blocks (kept on request) and the re-adaptation maps
  int64_t n_prev = 0;
  int64_t cap = 0;  // capacity in blocks
};

// device scalar block (u64 slots)
constexpr int SC_N = 0;      // [16] blocks per level
constexpr int SC_TOT = 16;   // [16] adjacency totals per level (pairs | cells << 32)
constexpr int SC_NL = 32;    // [16] links per level
constexpr int SC_RUN = 48;   // [3] running cells, pairs, links
constexpr int SC_REC = 52;   // [16] survivor records handed out per level
constexpr int SC_WORDS = 72;

// A captured graph stays valid while no buffer it uses was reallocated
// (layout generation) and its by-value kernel arguments are unchanged.
struct GraphKey {
  uint64_t layout_gen = 0;
  int64_t nf = 0, n_geom = 0;
  int n_levels = 0, lattice = 0, adjacency = 0, links = 0, warps = 0, B = 0, pred = 0, search = 0, prop = 0;
  uint64_t face_levels = 0;  // signature of the per-geometry choice of face by face
  uint64_t bins = 0;         // signature of the bin grids (every geometry's density, sampled or exact)
  double d_abs = 0, d_rel = 0;
  bool operator==(const GraphKey& o) const {
    return layout_gen == o.layout_gen && nf == o.nf && n_geom == o.n_geom && n_levels == o.n_levels &&
           bins == o.bins &&
           lattice == o.lattice && adjacency == o.adjacency && links == o.links && warps == o.warps && B == o.B &&
           pred == o.pred && search == o.search && prop == o.prop && face_levels == o.face_levels &&
           d_abs == o.d_abs && d_rel == o.d_rel;
  }
};

}  // namespace

struct amr_ctx {
  amr_domain dom{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t gstream = nullptr;  // capture / replay stream of the graph mode
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int device = 0;
  int num_sms = 0;
  std::string err;
  // state
  bool loaded = false, binned = false, refined = false;
  uint64_t load_gen = 0, bin_gen = 0, layout_gen = 0;
  int64_t nf = 0, nv = 0;
  bool indexed = false;
  int B = 0;
  int64_t n_bins = 0, nnz = 0;
  bool count_clean = false;
  // geometry table: one row per geometry; multi = per-block / per-face geometry ids in use
  std::vector<GeomParams> geoms;
  bool multi = false;
  DevBuf table, face_gid;
  // buffers
  DevBuf X, nrm, frec, recs, hkeys, hvals, mkeys, mvals, cls, flbase, tl_cell, tl_dir, tl_q, tl_face, stage_a, stage_b, frange, count, offsets, ids, payload, scratch, misc, scal;
  LevelBufs lv[AMR_MAX_LEVELS];
  DevBuf adj_cell, adj_off, adj_ids, link_cell, link_dir, link_q, link_face, link_stage;
  int64_t cap_cells = 0, cap_pairs = 0, cap_links = 0;
  int64_t cap_recs = 0, want_recs = 0;  // survivor record staging (entries)
  bool sampled_bins = false;             // the last binning used the paper's sampled membership
  bool classified = false;               // cls holds the classes of the last refinement's adjacent cells
  int prev_levels = -1;                  // levels of the kept previous hierarchy (-1: none kept)
  // adjoint
  DevBuf idx, vert_off, vert_corners, face_off, face_links, sort_keys, grad_face, sort_scratch, group_cnt, lvl_ptrs;
  bool vert_groups = false, face_groups = false;
  int64_t n_links = 0;
  // misc layout: [0..CNT_N) u64 counters, then u32 err word, u32 work, u64 totals[4]
  unsigned long long* counters = nullptr;
  unsigned* d_err = nullptr;
  unsigned* d_work = nullptr;
  uint64_t* d_tot = nullptr;
  DevBuf fstat;                           // per geometry: face-size statistics (see FaceBinArgs)
  DevBuf spill;                           // per-warp spill of survivor records (once a call needed it)
  DevBuf calg;                            // per-level algorithmic test counts (amr_candidate_count)
  DevBuf defer;                           // the adjacency's second-pass block list
  bool want_spill = false;
  void* h_stat = nullptr;                 // their mapped pinned copy (h_stat_dev as the device sees it)
  char* h_stat_dev = nullptr;
  size_t h_stat_cap = 0;
  std::vector<double> face_ext_max;       // per geometry, last binning: largest face AABB side / h0
  std::vector<double> face_ext_mean;      // and the mean of that ratio over its faces
  uint64_t* d_scal = nullptr;
  void* h_pinned = nullptr;  // 2 KB
  char* h_dev = nullptr;     // the same block as the device addresses it
  amr_refine_result last{};
  // graph mode
  cudaGraphExec_t gexec = nullptr;
  GraphKey gkey;
  int64_t graph_launches = 0;
  // timing
  bool timing = false;
  bool capturing = false;
  std::vector<TimingSlot> slots;
  std::vector<TimedLaunch> pending;
  std::vector<cudaEvent_t> event_pool;
  int64_t launches = 0;  // kernels launched by this context
};

namespace {

amr_status fail(amr_ctx* c, amr_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return s;
}

#define CK(call)                                                                                    \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) return fail(ctx, AMR_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));   \
  } while (0)

#define TRY(expr)                    \
  do {                               \
    amr_status s_ = (expr);          \
    if (s_ != AMR_OK) return s_;     \
  } while (0)

// Grow a buffer that no captured graph reads (the layout generation stays).
// Hand a device buffer back: in stream order (cudaFreeAsync), or to the caller's
// allocator once the context's stream has finished every use of it.
cudaError_t dev_release(amr_ctx* ctx, void* p) {
  if (!p) return cudaSuccess;
  if (ctx->dom.dev_free) {
    const cudaError_t e = cudaStreamSynchronize(ctx->stream);
    ctx->dom.dev_free(p, ctx->dom.user);
    return e;
  }
  return cudaFreeAsync(p, ctx->stream);
}

amr_status ensure_aux(amr_ctx* ctx, DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.cap >= bytes) return AMR_OK;
  if (b.p) {
    CK(dev_release(ctx, b.p));
    b.p = nullptr;
    b.cap = 0;
  }
  size_t want = bytes + bytes / 4 + 256;
  if (ctx->dom.dev_alloc) {
    b.p = ctx->dom.dev_alloc(want, ctx->dom.user);
    if (!b.p) return fail(ctx, AMR_ENOMEM, "device allocation of %zu bytes failed (caller's allocator)", want);
    b.cap = want;
    return AMR_OK;
  }
  cudaError_t e = cudaMallocAsync(&b.p, want, ctx->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return fail(ctx, AMR_ENOMEM, "device allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
  }
  b.cap = want;
  return AMR_OK;
}

// Grow a buffer; a move invalidates the captured graph (new layout generation).
amr_status ensure(amr_ctx* ctx, DevBuf& b, size_t bytes) {
  if (b.cap >= (bytes == 0 ? 16 : bytes)) return AMR_OK;
  ++ctx->layout_gen;
  return ensure_aux(ctx, b, bytes);
}

// Grow keeping the first `keep` bytes.
amr_status ensure_keep(amr_ctx* ctx, DevBuf& b, size_t bytes, size_t keep) {
  if (b.cap >= bytes) return AMR_OK;
  DevBuf nb;
  TRY(ensure(ctx, nb, bytes));
  if (b.p && keep) CK(cudaMemcpyAsync(nb.p, b.p, keep < b.cap ? keep : b.cap, cudaMemcpyDeviceToDevice, ctx->stream));
  if (b.p) CK(dev_release(ctx, b.p));
  b = nb;
  return AMR_OK;
}

void release(amr_ctx* ctx, DevBuf& b) {
  if (b.p) dev_release(ctx, b.p);
  b.p = nullptr;
  b.cap = 0;
}

int slot_of(amr_ctx* c, const char* name) {
  for (size_t i = 0; i < c->slots.size(); ++i)
    if (std::strcmp(c->slots[i].name, name) == 0) return (int)i;
  c->slots.push_back(TimingSlot{name});
  return (int)c->slots.size() - 1;
}

cudaEvent_t take_event(amr_ctx* c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Times the launches issued inside fn() when timing is on (not while capturing).
template <typename F>
void timed(amr_ctx* c, cudaStream_t st, const char* name, F fn) {
  if (!c->timing || c->capturing) {
    c->launches += fn();
    return;
  }
  TimedLaunch t{slot_of(c, name), take_event(c), take_event(c)};
  cudaEventRecord(t.a, st);
  c->launches += fn();
  cudaEventRecord(t.b, st);
  c->pending.push_back(t);
}

void harvest_timing(amr_ctx* c) {
  for (auto& t : c->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
      c->slots[t.slot].ms += ms;
      c->slots[t.slot].launches += 1;
    }
    c->event_pool.push_back(t.a);
    c->event_pool.push_back(t.b);
  }
  c->pending.clear();
}

// Small transfers between the pinned host block and device memory run as one
// tiny kernel (the block is mapped into the device's address space) instead of
// on a copy engine, where they would queue behind any large copy that another
// stream has in flight.  Up to four pieces of whole 32-bit words.
struct WordCopy {
  const uint32_t* src[4];
  uint32_t* dst[4];
  uint32_t words[4];
};

__global__ void k_copy_words(WordCopy c) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
    for (uint32_t w = threadIdx.x; w < c.words[i]; w += blockDim.x) c.dst[i][w] = c.src[i][w];
}

struct Piece {
  void* dst;
  const void* src;
  size_t bytes;
};

amr_status small_copy(amr_ctx* ctx, cudaStream_t st, std::initializer_list<Piece> pieces) {
  WordCopy c{};
  int i = 0;
  for (const Piece& p : pieces) {
    c.dst[i] = static_cast<uint32_t*>(p.dst);
    c.src[i] = static_cast<const uint32_t*>(p.src);
    c.words[i] = (uint32_t)(p.bytes / 4);
    ++i;
  }
  k_copy_words<<<1, 128, 0, st>>>(c);
  ++ctx->launches;
  CK(cudaGetLastError());
  return AMR_OK;
}

amr_status sync_check(amr_ctx* ctx, cudaStream_t st) {
  CK(cudaStreamSynchronize(st));
  CK(cudaGetLastError());
  harvest_timing(ctx);
  return AMR_OK;
}

// Copy the device error word and the first totals to pinned memory and wait.
amr_status read_back(amr_ctx* ctx, cudaStream_t st, unsigned* err_out, uint64_t* tot_out, int n_tot) {
  char* h = static_cast<char*>(ctx->h_pinned);
  TRY(small_copy(ctx, st, {{ctx->h_dev, ctx->d_tot, sizeof(uint64_t) * 8},  // totals and face stats
                      {ctx->h_dev + 64, ctx->d_err, sizeof(unsigned)}}));
  TRY(sync_check(ctx, st));
  if (tot_out)
    for (int i = 0; i < n_tot; ++i) tot_out[i] = reinterpret_cast<uint64_t*>(h)[i];
  *err_out = *reinterpret_cast<unsigned*>(h + 64);
  return AMR_OK;
}

// One device scalar (u64) and the error word.
amr_status read_scalar(amr_ctx* ctx, cudaStream_t st, int slot, uint64_t* v, unsigned* err_out) {
  char* h = static_cast<char*>(ctx->h_pinned);
  TRY(small_copy(ctx, st, {{ctx->h_dev + 128, ctx->d_scal + slot, sizeof(uint64_t)},
                      {ctx->h_dev + 64, ctx->d_err, sizeof(unsigned)}}));
  TRY(sync_check(ctx, st));
  *v = *reinterpret_cast<uint64_t*>(h + 128);
  *err_out = *reinterpret_cast<unsigned*>(h + 64);
  return AMR_OK;
}

amr_status device_error(amr_ctx* ctx, unsigned e) {
  if (!e) return AMR_OK;
  // clear it so the context stays usable after the report
  cudaMemsetAsync(ctx->d_err, 0, sizeof(unsigned), ctx->stream);
  if (e & ERR_TIMEOUT) return fail(ctx, AMR_ETIMEOUT, "a bounded device-side wait gave up (flags 0x%x)", e);
  if (e & ERR_OVERFLOW) return fail(ctx, AMR_EOVERFLOW, "a device-side size exceeded its range (flags 0x%x)", e);
  if (e & ERR_BADINDEX) return fail(ctx, AMR_EDEVICE_CHECK, "face vertex index out of range");
  if (e & ERR_NONFINITE) return fail(ctx, AMR_EDEVICE_CHECK, "non-finite vertex coordinate");
  return fail(ctx, AMR_EDEVICE_CHECK, "device check failed (flags 0x%x)", e);
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Makes `src` available on the device: device pointers pass through; host
// memory is copied into `stage`.
amr_status to_device(amr_ctx* ctx, const void* src, size_t bytes, DevBuf& stage, const void** dst) {
  if (bytes == 0) {
    *dst = src;
    return AMR_OK;
  }
  if (is_device_ptr(src)) {
    *dst = src;
    return AMR_OK;
  }
  TRY(ensure(ctx, stage, bytes));
  CK(cudaMemcpyAsync(stage.p, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
  *dst = stage.p;
  return AMR_OK;
}

int64_t ipow(int64_t b, int e) {
  int64_t r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

int64_t roots_of(const GeomParams& g, int D) {
  int64_t n = 1;
  for (int a = 0; a < D; ++a) n *= g.root[a];
  return n;
}

void drop_graph(amr_ctx* ctx) {
  if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
  ctx->gexec = nullptr;
}

}  // namespace

// FP32 forms of a row's FP64 fields (hi + lo pairs for h0 and the origin).
void amr_finish_row(GeomParams& g) {
  g.h0_hi = (float)g.h0;
  g.h0_lo = (float)(g.h0 - (double)g.h0_hi);
  for (int a = 0; a < 3; ++a) {
    g.org_hi[a] = (float)g.origin[a];
    g.org_lo[a] = (float)(g.origin[a] - (double)g.org_hi[a]);
    g.scale32[a] = (float)g.bin_scale[a];
  }
  g.d_abs32 = (float)g.d_abs;
  g.d_rel32 = (float)g.d_rel;
}

// Table row of a geometry: domain, bins, levels and near-wall distance.
GeomParams amr_make_row(const amr_domain& d, int B, int n_levels, double d_abs, double d_rel) {
  GeomParams g{};
  for (int a = 0; a < 3; ++a) {
    g.origin[a] = d.origin[a];
    g.root[a] = a < d.dim ? d.root_blocks[a] : 1;
    const double extent = (4.0 * (double)g.root[a]) * d.h0;
    g.bin_scale[a] = B > 0 ? (double)B / extent : 0.0;
  }
  g.h0 = d.h0;
  g.B = B;
  g.n_levels = n_levels;
  g.d_abs = d_abs;
  g.d_rel = d_rel;
  amr_finish_row(g);
  return g;
}

// ---------------------------------------------------------------------------
// context life cycle, binning and the level engine (also used by batch.cu)
// ---------------------------------------------------------------------------
amr_status amr_ctx_init(amr_ctx* ctx) {
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e == cudaSuccess && !ctx->stream) {
    e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
    ctx->own_stream = e == cudaSuccess;
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_pinned, 2048);
  void* hd = nullptr;
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(&hd, ctx->h_pinned, 0);
  ctx->h_dev = static_cast<char*>(hd);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return AMR_ECUDA;
  }
  if (ensure(ctx, ctx->misc, sizeof(unsigned long long) * CNT_N + 64 + 64) != AMR_OK) return AMR_ENOMEM;
  if (ensure(ctx, ctx->scal, sizeof(uint64_t) * SC_WORDS) != AMR_OK) return AMR_ENOMEM;
  char* m = static_cast<char*>(ctx->misc.p);
  ctx->counters = reinterpret_cast<unsigned long long*>(m);
  ctx->d_err = reinterpret_cast<unsigned*>(m + sizeof(unsigned long long) * CNT_N);
  ctx->d_work = ctx->d_err + 1;
  ctx->d_tot = reinterpret_cast<uint64_t*>(m + sizeof(unsigned long long) * CNT_N + 64);
  ctx->d_scal = static_cast<uint64_t*>(ctx->scal.p);
  cudaMemsetAsync(ctx->misc.p, 0, ctx->misc.cap, ctx->stream);
  cudaMemsetAsync(ctx->scal.p, 0, ctx->scal.cap, ctx->stream);
  return AMR_OK;
}

void amr_ctx_free(amr_ctx* ctx) {
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  drop_graph(ctx);
  DevBuf* all[] = {&ctx->X, &ctx->frec, &ctx->recs, &ctx->hkeys, &ctx->hvals, &ctx->mkeys, &ctx->mvals, &ctx->cls, &ctx->flbase,
                   &ctx->tl_cell, &ctx->tl_dir, &ctx->tl_q, &ctx->tl_face, &ctx->nrm,          &ctx->stage_a,    &ctx->stage_b,    &ctx->frange,
                   &ctx->count,     &ctx->offsets,      &ctx->ids,        &ctx->payload,    &ctx->scratch,
                   &ctx->misc,      &ctx->scal,         &ctx->adj_cell,   &ctx->adj_off,    &ctx->adj_ids,
                   &ctx->link_cell, &ctx->link_dir,     &ctx->link_q,     &ctx->link_face,  &ctx->link_stage, &ctx->idx,
                   &ctx->vert_off,  &ctx->vert_corners, &ctx->face_off,   &ctx->face_links, &ctx->sort_keys,
                   &ctx->grad_face, &ctx->sort_scratch, &ctx->group_cnt,  &ctx->lvl_ptrs,   &ctx->table,
                   &ctx->face_gid,  &ctx->fstat,        &ctx->spill,      &ctx->calg,       &ctx->defer};
  for (DevBuf* b : all) release(ctx, *b);
  for (int L = 0; L < AMR_MAX_LEVELS; ++L) {
    LevelBufs& l = ctx->lv[L];
    DevBuf* lb[] = {&l.blocks, &l.gid,  &l.parent, &l.mask, &l.flag, &l.cellcnt,
                    &l.blockcnt, &l.base, &l.desc,   &l.prev, &l.n2o,  &l.o2n, &l.first};
    for (DevBuf* b : lb) release(ctx, *b);
  }
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  for (auto& t : ctx->pending) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  for (auto e : ctx->event_pool) cudaEventDestroy(e);
  if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
  if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
  if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
  if (ctx->h_stat) cudaFreeHost(ctx->h_stat);
}

// Binning of every geometry of the table in one pass (count, scan, scatter).
amr_status amr_bin_all(amr_ctx* ctx) {
  cudaStream_t st = ctx->stream;
  const int D = ctx->dom.dim;
  const int64_t nf = ctx->nf;
  int64_t nb = 0;
  for (auto& g : ctx->geoms) {
    g.bin_base = nb;
    nb += ipow(g.B, D);
  }
  if (ctx->multi) {
    TRY(ensure(ctx, ctx->table, sizeof(GeomParams) * ctx->geoms.size()));
    CK(cudaMemcpyAsync(ctx->table.p, ctx->geoms.data(), sizeof(GeomParams) * ctx->geoms.size(),
                       cudaMemcpyHostToDevice, st));
  }
  if (ctx->count.cap < sizeof(uint32_t) * (size_t)nb) ctx->count_clean = false;
  TRY(ensure(ctx, ctx->count, sizeof(uint32_t) * (size_t)nb));
  if (!ctx->count_clean) {
    CK(cudaMemsetAsync(ctx->count.p, 0, ctx->count.cap, st));
    ctx->count_clean = true;
  }
  TRY(ensure(ctx, ctx->offsets, sizeof(uint32_t) * (size_t)(nb + 1)));
  TRY(ensure(ctx, ctx->frange, sizeof(uint32_t) * 3 * (size_t)(nf > 0 ? nf : 1)));
  TRY(ensure(ctx, ctx->scratch, scan_u32_scratch_bytes(nb)));
  FaceBinArgs fa{};
  fa.dim = D;
  fa.X = static_cast<const float*>(ctx->X.p);
  fa.nf = nf;
  fa.g0 = ctx->geoms[0];
  fa.table = ctx->multi ? static_cast<const GeomParams*>(ctx->table.p) : nullptr;
  fa.face_gid = ctx->multi ? static_cast<const uint32_t*>(ctx->face_gid.p) : nullptr;
  fa.frange = static_cast<uint32_t*>(ctx->frange.p);
  fa.count = static_cast<uint32_t*>(ctx->count.p);
  if (ctx->sampled_bins && !ctx->multi) {
    // the paper's sampled membership: spacing half a bin length (the shortest axis's bin)
    double ext = 1e300;
    for (int a = 0; a < D; ++a) ext = std::min(ext, (4.0 * (double)ctx->dom.root_blocks[a]) * ctx->dom.h0);
    fa.sampled = 1;
    fa.sample_s = 0.5 * (ext / (double)ctx->geoms[0].B);
  }
  const size_t G = ctx->geoms.size(), stat_bytes = 2 * sizeof(unsigned long long) * G;
  TRY(ensure_aux(ctx, ctx->fstat, stat_bytes));
  if (ctx->h_stat_cap < stat_bytes) {
    if (ctx->h_stat) cudaFreeHost(ctx->h_stat);
    ctx->h_stat = nullptr;
    ctx->h_stat_cap = 0;
    void* hd = nullptr;
    cudaError_t e1 = cudaMallocHost(&ctx->h_stat, stat_bytes);
    if (e1 == cudaSuccess) e1 = cudaHostGetDevicePointer(&hd, ctx->h_stat, 0);
    if (e1 != cudaSuccess) {
      cudaGetLastError();
      return fail(ctx, AMR_ENOMEM, "pinned allocation of %zu bytes failed", stat_bytes);
    }
    ctx->h_stat_dev = static_cast<char*>(hd);
    ctx->h_stat_cap = stat_bytes;
  }
  fa.fstat = static_cast<unsigned long long*>(ctx->fstat.p);
  CK(cudaMemsetAsync(ctx->fstat.p, 0, stat_bytes, st));
  uint32_t* offsets = static_cast<uint32_t*>(ctx->offsets.p);
  timed(ctx, st, "bin_count", [&] { return launch_face_bins(fa, st); });
  timed(ctx, st, "bin_scan", [&] {
    return launch_scan_u32(fa.count, offsets, nb, ctx->d_tot, ctx->scratch.p, ctx->d_err, st);
  });
  CK(cudaGetLastError());
  TRY(small_copy(ctx, st, {{ctx->h_stat_dev, ctx->fstat.p, stat_bytes}}));
  unsigned e = 0;
  uint64_t tot = 0;
  TRY(read_back(ctx, st, &e, &tot, 1));
  ctx->face_ext_max.assign(G, 0.0);
  ctx->face_ext_mean.assign(G, 0.0);
  const unsigned long long* hs = static_cast<const unsigned long long*>(ctx->h_stat);
  for (size_t g = 0; g < G; ++g) {
    const int64_t f0 = ctx->multi ? ctx->geoms[g].face_base : 0;
    const int64_t f1 = ctx->multi && g + 1 < G ? ctx->geoms[g + 1].face_base : nf;
    const uint32_t bits = (uint32_t)hs[2 * g];
    float mx;
    std::memcpy(&mx, &bits, sizeof mx);
    ctx->face_ext_max[g] = f1 > f0 ? (double)mx : 0.0;
    ctx->face_ext_mean[g] = f1 > f0 ? (double)hs[2 * g + 1] / 65536.0 / (double)(f1 - f0) : 0.0;
  }
  if (e) {
    ctx->count_clean = false;
    return device_error(ctx, e);
  }
  if (tot > 0xffffffffull) {
    ctx->count_clean = false;
    return fail(ctx, AMR_EOVERFLOW, "%llu (face, bin) entries exceed 2^32 - 1", (unsigned long long)tot);
  }
  const size_t esz = D == 3 ? sizeof(Entry3) : sizeof(Entry2);
  TRY(ensure(ctx, ctx->ids, sizeof(uint32_t) * (size_t)tot));
  TRY(ensure(ctx, ctx->payload, esz * (size_t)tot));
  ScatterArgs sa{};
  sa.f = fa;
  sa.offsets = offsets;
  sa.ids = static_cast<uint32_t*>(ctx->ids.p);
  sa.payload = ctx->payload.p;
  sa.rec = static_cast<const FaceRec3*>(ctx->frec.p);
  timed(ctx, st, "bin_scatter", [&] { return launch_scatter(sa, st); });
  CK(cudaGetLastError());
  ctx->n_bins = nb;
  ctx->nnz = (int64_t)tot;
  ctx->binned = true;
  ++ctx->bin_gen;
  return AMR_OK;
}

namespace {

struct Plan {
  int NL;                           // levels of the deepest geometry
  bool fin_at[AMR_MAX_LEVELS];      // some geometry ends at this level
  bool cont_after[AMR_MAX_LEVELS];  // some geometry continues below this level
  bool face_at[AMR_MAX_LEVELS];     // some geometry's blocks of the level are marked face by face
  bool walk_at[AMR_MAX_LEVELS];     // some geometry's blocks of the level are walked
  bool adjacency, links;
  int lattice, warps, pred, search, propagate;
  int64_t n_roots;
};

// Face-by-face marking applies to a geometry's blocks of a level whose only
// output is the mask, with the whole-domain search, and faces whose cell ranges
// stay small (the geometry's largest face of the last binning, widened by d,
// covers at most kMaxFaceCells cells).
constexpr double kMaxFaceCells = 32768.0;
// Automatic choice: face by face where the geometry's mean face covers at most
// this many cells of the level (the block walk is cheaper once faces span many cells).
constexpr double kAutoFaceCells = 1024.0;

// Cells of level L in the range of a face of geometry g whose largest AABB side
// is ext root cells: (ext 2^L + 2 d_L / h_L + pad) per axis (pad 4 bounds the
// rounding of the range ends and the cell-box reach; pad 1 estimates the typical range).
double face_cells(const amr_ctx* ctx, const GeomParams& g, int L, double ext, double pad) {
  const double hL = std::ldexp(g.h0, -L);
  const double dh = (g.d_abs + g.d_rel * hL) / hL;
  return std::pow(ext * std::ldexp(1.0, L) + 2.0 * dh + pad, (double)ctx->dom.dim);
}

Plan make_plan(const amr_ctx* ctx, const amr_refine_params* p) {
  Plan P{};
  for (const auto& g : ctx->geoms) P.NL = g.n_levels > P.NL ? g.n_levels : P.NL;
  for (const auto& g : ctx->geoms) {
    P.fin_at[g.n_levels - 1] = true;
    for (int L = 0; L < g.n_levels - 1; ++L) P.cont_after[L] = true;
  }
  P.links = p->want_links != 0;
  P.adjacency = p->want_adjacency != 0 || P.links;
  P.lattice = p->lattice;
  P.warps = p->warps_per_cta > 0 ? p->warps_per_cta : 4;
  P.pred = p->predicate;
  P.search = p->search;
  P.propagate = p->propagate;
  for (const auto& g : ctx->geoms) P.n_roots += roots_of(g, ctx->dom.dim);
  return P;
}

// Per geometry and level: face by face or the block walk (face_levels bits of
// the geometry rows, uploaded with the table); the plan's face_at / walk_at say
// which of the two launches a level needs.  Returns a signature of the choice.
uint64_t assign_face_levels(amr_ctx* ctx, Plan& P, const amr_refine_params* p) {
  uint64_t sig = 1469598103934665603ull;
  for (size_t gi = 0; gi < ctx->geoms.size(); ++gi) {
    GeomParams& g = ctx->geoms[gi];
    uint32_t bits = 0;
    const double emax = gi < ctx->face_ext_max.size() ? ctx->face_ext_max[gi] : INFINITY;
    const double emean = gi < ctx->face_ext_mean.size() ? ctx->face_ext_mean[gi] : INFINITY;
    for (int L = 0; L < g.n_levels && p->face_pass != AMR_FACE_PASS_OFF; ++L) {
      bool ok = P.search == AMR_SEARCH_QUERY_BOX && (L < g.n_levels - 1 || !P.adjacency);
      ok = ok && face_cells(ctx, g, L, emax, 4.0) <= kMaxFaceCells;
      if (ok && p->face_pass == AMR_FACE_PASS_AUTO) ok = face_cells(ctx, g, L, emean, 1.0) <= kAutoFaceCells;
      if (ok) bits |= 1u << L;
    }
    g.face_levels = bits;
    for (int L = 0; L < g.n_levels; ++L) {
      if ((bits >> L) & 1u)
        P.face_at[L] = true;
      else
        P.walk_at[L] = true;
    }
    sig = (sig ^ bits) * 1099511628211ull;
  }
  return sig;
}

// Smallest d_L / h_L for which every face a link segment (length up to sqrt(2) h)
// can cross is in the cell's adjacency list: the inflated cell box contains the
// segment once d_L >= h_L / 2; the ball of the point predicate once d_L >= sqrt(2) h_L.
double link_reach(int pred) { return pred == AMR_PRED_POINT ? 1.4142135623730951 : 0.5; }

RefineLevel level_args(amr_ctx* ctx, const Plan& P, int L) {
  RefineLevel a{};
  a.dim = ctx->dom.dim;
  a.level = L;
  a.g0 = ctx->geoms[0];
  a.table = ctx->multi ? static_cast<const GeomParams*>(ctx->table.p) : nullptr;
  a.gid = ctx->multi ? static_cast<const uint32_t*>(ctx->lv[L].gid.p) : nullptr;
  a.blocks = static_cast<const int32_t*>(ctx->lv[L].blocks.p);
  a.n_blocks = ctx->lv[L].cap;
  a.n_dev = ctx->d_scal + SC_N + L;
  a.offsets = static_cast<const uint32_t*>(ctx->offsets.p);
  a.payload = ctx->payload.p;
  a.X = static_cast<const float*>(ctx->X.p);
  a.nrm = static_cast<const float*>(ctx->nrm.p);
  a.nf = ctx->nf;
  a.mask = static_cast<uint64_t*>(ctx->lv[L].mask.p);
  a.flag = static_cast<uint8_t*>(ctx->lv[L].flag.p);
  if (P.fin_at[L] && P.adjacency) {
    a.cellcnt = static_cast<uint16_t*>(ctx->lv[L].cellcnt.p);
    a.blockcnt = static_cast<uint64_t*>(ctx->lv[L].blockcnt.p);
    a.recs = static_cast<SurvRec*>(ctx->recs.p);
    a.cap_recs = ctx->cap_recs;
    a.rec_count = ctx->d_scal + SC_REC + L;
    a.rec_desc = static_cast<uint64_t*>(ctx->lv[L].desc.p);
    a.spill = ctx->want_spill || refine_by_groups(a.dim, L, P.pred, P.search) ? static_cast<SurvRec*>(ctx->spill.p)
                                                                                : nullptr;
  }
  a.counters = ctx->counters;
  a.work = ctx->d_work;
  a.err = ctx->d_err;
  a.warps = P.warps;
  a.pred = P.pred;
  a.search = P.search;
  // blocks per work fetch: batches hide the fetch latency where every warp has many blocks;
  // single blocks keep the load balanced where there are few (and heavy ones cluster)
  const int64_t per_warp = ctx->lv[L].cap / ((int64_t)ctx->num_sms * 16);
  a.batch = per_warp >= 32 ? 4 : (per_warp >= 8 ? 2 : 1);
  return a;
}

__global__ void k_set_u64(uint64_t* p, uint64_t v) { *p = v; }

// Capacity for a size learnt by an eager pass that a captured graph will reuse:
// room for the sizes to drift between calls (a moving wall) without an overflow.
int64_t with_slack(int64_t n) { return n + n / 8 + 256; }

// One pass over all levels.  eager: learn sizes with read-backs and grow
// buffers (with slack when a graph is captured next); otherwise (capture) use
// the capacities as they are.
amr_status engine_pass(amr_ctx* ctx, const Plan& P, bool eager, bool slack, cudaStream_t st) {
  const int D = ctx->dom.dim;
  const int NCH = D == 3 ? 8 : 4;
  const int NCell = D == 3 ? 64 : 16;
  CK(cudaMemsetAsync(ctx->counters, 0, sizeof(unsigned long long) * CNT_N, st));
  CK(cudaMemsetAsync(ctx->d_scal, 0, sizeof(uint64_t) * SC_WORDS, st));
  int64_t run_cells = 0, run_pairs = 0, run_links = 0;
  const int64_t N0 = P.n_roots;
  if (eager) {
    ctx->lv[0].cap = N0;
    TRY(ensure(ctx, ctx->lv[0].blocks, sizeof(int32_t) * D * (size_t)(N0 > 0 ? N0 : 1)));
    if (ctx->multi) TRY(ensure(ctx, ctx->lv[0].gid, sizeof(uint32_t) * (size_t)(N0 > 0 ? N0 : 1)));
  }
  timed(ctx, st, "root_blocks", [&] {
    int k = 0;
    if (ctx->multi)
      k = launch_root_blocks_multi(D, static_cast<const GeomParams*>(ctx->table.p), (int)ctx->geoms.size(),
                                   static_cast<int32_t*>(ctx->lv[0].blocks.p),
                                   static_cast<uint32_t*>(ctx->lv[0].gid.p), N0, st);
    else
      k = launch_root_blocks(D, ctx->geoms[0].root, static_cast<int32_t*>(ctx->lv[0].blocks.p), N0, st);
    k_set_u64<<<1, 1, 0, st>>>(ctx->d_scal + SC_N, (uint64_t)N0);
    return k + 1;
  });
  int64_t N = N0;
  for (int L = 0; L < P.NL; ++L) {
    LevelBufs& lb = ctx->lv[L];
    if (eager) {
      // level 0: the roots; deeper levels: set when their parents were compacted
      if (L == 0) lb.cap = N;
      const size_t n1 = (size_t)(lb.cap > 0 ? lb.cap : 1);
      TRY(ensure(ctx, lb.mask, sizeof(uint64_t) * n1));
      TRY(ensure(ctx, lb.flag, n1));
      if (P.fin_at[L] && P.adjacency) {
        TRY(ensure(ctx, lb.cellcnt, sizeof(uint16_t) * NCell * n1));
        TRY(ensure(ctx, lb.blockcnt, sizeof(uint64_t) * n1));
        TRY(ensure(ctx, lb.base, sizeof(uint64_t) * n1));
        TRY(ensure(ctx, lb.desc, sizeof(uint64_t) * n1));
        // record staging: what the last pass needed, at least a few per block
        int64_t want = ctx->want_recs > 4 * lb.cap + 1024 ? ctx->want_recs : 4 * lb.cap + 1024;
        if (want > ctx->cap_recs) {
          TRY(ensure(ctx, ctx->recs, sizeof(SurvRec) * (size_t)want));
          ctx->cap_recs = want;
        }
        // blocks with more survivor records than shared memory stages were seen: a spill area for
        // every warp the refine launch can hold (32 per SM)
        // (a level marked by parent groups always stages a group's records past shared memory there)
        if (ctx->want_spill || refine_by_groups(D, L, P.pred, P.search))
          TRY(ensure(ctx, ctx->spill, sizeof(SurvRec) * (size_t)kSpillCap * 32 * (size_t)ctx->num_sms));
      }
    }
    RefineLevel a = level_args(ctx, P, L);
    CK(cudaMemsetAsync(ctx->d_work, 0, sizeof(unsigned), st));
    if (P.face_at[L]) {
      // face by face: masks and flags start clear; deeper levels find their blocks by descending
      // from the roots through the upper levels' first-child arrays
      CK(cudaMemsetAsync(a.mask, 0, sizeof(uint64_t) * (size_t)(lb.cap > 0 ? lb.cap : 1), st));
      CK(cudaMemsetAsync(a.flag, 0, (size_t)(lb.cap > 0 ? lb.cap : 1), st));
      MarkArgs m{};
      m.lv = a;
      m.rec = static_cast<const FaceRec3*>(ctx->frec.p);
      m.face_gid = ctx->multi ? static_cast<const uint32_t*>(ctx->face_gid.p) : nullptr;
      for (int l = 0; l < L; ++l) m.first_child[l] = static_cast<const int32_t*>(ctx->lv[l].first.p);
      // faces per work fetch: enough warps to fill the GPU (24 resident per SM)
      const int64_t warps = (int64_t)ctx->num_sms * 24;
      m.batch = (int)std::max<int64_t>(1, std::min<int64_t>(kFaceBatch, ctx->nf / (2 * warps)));
      if (a.blockcnt) CK(cudaMemsetAsync(a.blockcnt, 0, sizeof(uint64_t) * (size_t)(lb.cap > 0 ? lb.cap : 1), st));
      timed(ctx, st, "mark_faces", [&] { return launch_mark_faces(m, ctx->num_sms, st); });
      if (P.walk_at[L]) {
        // the other geometries' blocks: the walk (it also records the faces of those that end here)
        a.skip_mark_only = 1;
        CK(cudaMemsetAsync(ctx->d_work, 0, sizeof(unsigned), st));
        timed(ctx, st, "refine_level", [&] { return launch_refine(a, ctx->num_sms, st); });
      }
    } else {
      timed(ctx, st, "refine_level", [&] { return launch_refine(a, ctx->num_sms, st); });
    }
    if (P.cont_after[L] && P.propagate != 0) {
      // the paper's mark propagation over this level's blocks (flags 0/1 in place)
      const GeomParams& g0 = ctx->geoms[0];
      const double hL = std::ldexp(g0.h0, -L);
      const int rounds = P.propagate > 0 ? P.propagate
                                         : 1 + (int)std::floor((g0.d_abs + g0.d_rel * hL) / (4.0 * hL));
      const uint32_t slots = propagate_hash_slots(lb.cap);
      if (eager) {
        TRY(ensure(ctx, ctx->hkeys, sizeof(unsigned long long) * slots));
        TRY(ensure(ctx, ctx->hvals, sizeof(uint32_t) * slots));
      }
      timed(ctx, st, "propagate", [&] {
        return launch_propagate(D, a.blocks, lb.cap, ctx->d_scal + SC_N + L, a.flag, rounds,
                                static_cast<unsigned long long*>(ctx->hkeys.p), static_cast<uint32_t*>(ctx->hvals.p),
                                slots, ctx->d_err, st);
      });
    }
    if (P.cont_after[L]) {
      LevelBufs& nx = ctx->lv[L + 1];
      if (eager) {
        const int64_t cap = N * NCH;
        nx.cap = cap;
        const size_t c1 = (size_t)(cap > 0 ? cap : 1);
        TRY(ensure(ctx, nx.blocks, sizeof(int32_t) * D * c1));
        TRY(ensure(ctx, nx.parent, sizeof(int32_t) * c1));
        TRY(ensure(ctx, lb.first, sizeof(int32_t) * (size_t)(lb.cap > 0 ? lb.cap : 1)));
        if (ctx->multi) TRY(ensure(ctx, nx.gid, sizeof(uint32_t) * c1));
        TRY(ensure(ctx, ctx->scratch, children_scratch_bytes(lb.cap)));
      }
      ChildrenArgs ca{};
      ca.dim = D;
      ca.level = L;
      ca.g0 = ctx->geoms[0];
      ca.table = a.table;
      ca.gid = a.gid;
      ca.blocks = a.blocks;
      ca.mask = a.mask;
      ca.flag = a.flag;
      ca.n = lb.cap;
      ca.n_dev = ctx->d_scal + SC_N + L;
      ca.child_blocks = static_cast<int32_t*>(nx.blocks.p);
      ca.child_gid = ctx->multi ? static_cast<uint32_t*>(nx.gid.p) : nullptr;
      ca.child_parent = static_cast<int32_t*>(nx.parent.p);
      ca.first_child = static_cast<int32_t*>(lb.first.p);
      ca.cap_out = nx.cap;
      ca.total = ctx->d_scal + SC_N + L + 1;
      ca.err = ctx->d_err;
      timed(ctx, st, "children", [&] { return launch_children(ca, ctx->scratch.p, ctx->num_sms, st); });
      if (eager) {
        CK(cudaGetLastError());
        uint64_t nn = 0;
        unsigned e = 0;
        TRY(read_scalar(ctx, st, SC_N + L + 1, &nn, &e));
        TRY(device_error(ctx, e));
        if ((int64_t)nn > (1ll << 32) / NCell) return fail(ctx, AMR_EOVERFLOW, "level %d has too many blocks", L + 1);
        N = (int64_t)nn;
        const int64_t bound = nx.cap;  // what the child buffers were sized for
        nx.cap = slack ? std::min(with_slack(N), bound) : N;
      }
    }
    if (P.fin_at[L] && P.adjacency) {
      if (eager) TRY(ensure(ctx, ctx->scratch, scan_u64_scratch_bytes(lb.cap)));
      timed(ctx, st, "adj_scan", [&] {
        return launch_scan_u64(static_cast<const uint64_t*>(lb.blockcnt.p), static_cast<uint64_t*>(lb.base.p), lb.cap,
                               ctx->d_scal + SC_N + L, ctx->d_scal + SC_TOT + L, ctx->scratch.p, ctx->d_err,
                               ctx->num_sms, st);
      });
      int64_t cells = 0, pairs = 0;
      if (eager) {
        CK(cudaGetLastError());
        uint64_t tot = 0;
        unsigned e = 0;
        TRY(read_scalar(ctx, st, SC_TOT + L, &tot, &e));
        TRY(device_error(ctx, e));
        cells = (int64_t)(tot >> 32);
        pairs = (int64_t)(tot & 0xffffffffull);
        if (run_pairs + pairs >= (int64_t)0xffffffffll)
          return fail(ctx, AMR_EOVERFLOW, "too many adjacent (cell, face) pairs");
        const int64_t need_c = run_cells + cells, need_p = run_pairs + pairs;
        if (need_c + 1 > ctx->cap_cells) ctx->cap_cells = slack ? with_slack(need_c + 1) : need_c + 1;
        if (need_p > ctx->cap_pairs) ctx->cap_pairs = slack ? with_slack(need_p) : need_p;
        TRY(ensure_keep(ctx, ctx->adj_cell, sizeof(uint32_t) * (size_t)(ctx->cap_cells + 1),
                        sizeof(uint32_t) * (size_t)run_cells));
        TRY(ensure_keep(ctx, ctx->adj_off, sizeof(uint32_t) * (size_t)(ctx->cap_cells + 1),
                        sizeof(uint32_t) * (size_t)(run_cells + 1)));
        TRY(ensure_keep(ctx, ctx->adj_ids, sizeof(uint32_t) * (size_t)(ctx->cap_pairs + 1),
                        sizeof(uint32_t) * (size_t)run_pairs));
      }
      EmitArgs ea{};
      ea.lv = a;
      ea.block_base = static_cast<const uint64_t*>(lb.base.p);
      ea.run = ctx->d_scal + SC_RUN;
      ea.adj_cell = static_cast<uint32_t*>(ctx->adj_cell.p);
      ea.adj_off = static_cast<uint32_t*>(ctx->adj_off.p);
      ea.adj_ids = static_cast<uint32_t*>(ctx->adj_ids.p);
      ea.cap_cells = ctx->cap_cells;
      ea.cap_pairs = ctx->cap_pairs;
      // the second pass's block list: [0] its count, then the blocks (one slot per block of the level)
      if (eager) TRY(ensure(ctx, ctx->defer, sizeof(uint32_t) * (size_t)(lb.cap + 1)));
      ea.defer_n = static_cast<unsigned*>(ctx->defer.p);
      ea.defer = static_cast<uint32_t*>(ctx->defer.p) + 1;
      ea.defer_cap = lb.cap;
      CK(cudaMemsetAsync(ea.defer_n, 0, sizeof(unsigned), st));
      CK(cudaMemsetAsync(ctx->d_work, 0, sizeof(unsigned), st));
      timed(ctx, st, "adjacency", [&] { return launch_adjacency(ea, ctx->num_sms, st); });
      timed(ctx, st, "advance", [&] {
        return launch_advance(ctx->d_scal + SC_TOT + L, nullptr, ctx->d_scal + SC_RUN,
                              static_cast<uint32_t*>(ctx->adj_off.p), ctx->cap_cells, ctx->d_err, true, st);
      });
      if (P.links) {
        LinkArgs la{};
        la.dim = D;
        la.lattice = P.lattice;
        la.level = L;
        la.g0 = ctx->geoms[0];
        la.table = a.table;
        la.gid = a.gid;
        la.blocks = a.blocks;
        la.adj_cell = ea.adj_cell;
        la.adj_off = ea.adj_off;
        la.adj_ids = ea.adj_ids;
        la.run = ctx->d_scal + SC_RUN;
        la.level_tot = ctx->d_scal + SC_TOT + L;
        la.cap_rows = ctx->cap_cells;
        la.cap_pairs = ctx->cap_pairs;
        la.X = a.X;
        la.rec = static_cast<const FaceRec3*>(ctx->frec.p);
        la.nf = ctx->nf;
        la.n_links = ctx->d_scal + SC_NL + L;
        la.counters = ctx->counters;
        la.err = ctx->d_err;
        for (int attempt = 0; attempt < 2; ++attempt) {
          if (eager) {
            // first guess: a quarter more links than (cell, face) pairs (the synthetic spheres have
            // 1.1 per pair); a level with more re-runs once at its exact count
            const int64_t guess = pairs + pairs / 4 + 1024;
            const int64_t want = run_links + (guess > cells ? guess : cells);
            if (want > ctx->cap_links || attempt > 0) {
              const int64_t nc = attempt > 0 ? ctx->cap_links : want;
              const size_t keep = (size_t)run_links;
              TRY(ensure_keep(ctx, ctx->link_cell, sizeof(uint32_t) * (size_t)(nc + 1), sizeof(uint32_t) * keep));
              TRY(ensure_keep(ctx, ctx->link_dir, (size_t)(nc + 1), keep));
              TRY(ensure_keep(ctx, ctx->link_q, sizeof(float) * (size_t)(nc + 1), sizeof(float) * keep));
              TRY(ensure_keep(ctx, ctx->link_face, sizeof(uint32_t) * (size_t)(nc + 1), sizeof(uint32_t) * keep));
              ctx->cap_links = nc;
            }
            TRY(ensure(ctx, ctx->scratch, links_scratch_bytes(ctx->cap_cells)));
            TRY(ensure(ctx, ctx->link_stage, links_stage_bytes(ctx->cap_links)));
          }
          la.link_cell = static_cast<uint32_t*>(ctx->link_cell.p);
          la.link_dir = static_cast<uint8_t*>(ctx->link_dir.p);
          la.link_q = static_cast<float*>(ctx->link_q.p);
          la.link_face = static_cast<uint32_t*>(ctx->link_face.p);
          la.link_cap = ctx->cap_links;
          la.stage = ctx->link_stage.p;
          timed(ctx, st, "links", [&] { return launch_links(la, ctx->scratch.p, ctx->num_sms, st); });
          if (!eager) break;
          CK(cudaGetLastError());
          uint64_t nl = 0;
          unsigned e = 0;
          TRY(read_scalar(ctx, st, SC_NL + L, &nl, &e));
          if (e & ~ERR_OVERFLOW) TRY(device_error(ctx, e));
          if (run_links + (int64_t)nl <= ctx->cap_links) {
            if (e) TRY(device_error(ctx, e));
            run_links += (int64_t)nl;
            break;
          }
          // too small: grow to the exact count and run the level's links again
          CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(unsigned), st));
          ctx->cap_links = run_links + (int64_t)nl;
        }
      }
      timed(ctx, st, "advance", [&] {
        return launch_advance(ctx->d_scal + SC_TOT + L, P.links ? ctx->d_scal + SC_NL + L : nullptr,
                              ctx->d_scal + SC_RUN, static_cast<uint32_t*>(ctx->adj_off.p), ctx->cap_cells,
                              ctx->d_err, false, st);
      });
      run_cells += cells;
      run_pairs += pairs;
    }
  }
  CK(cudaGetLastError());
  return AMR_OK;
}

// Read every size of the last pass (one synchronisation) and fill the result.
amr_status collect(amr_ctx* ctx, const Plan& P, cudaStream_t st, amr_refine_result* out) {
  char* h = static_cast<char*>(ctx->h_pinned);
  // pinned layout: [0, 8 CNT_N) counters, 128 error word, 256 level pointers, 512 scalars
  static_assert(sizeof(unsigned long long) * CNT_N <= 128, "counters overlap the error word");
  static_assert(kMaxLevels == AMR_MAX_LEVELS, "level arrays of the kernels and of the ABI agree");
  TRY(small_copy(ctx, st, {{ctx->h_dev, ctx->counters, sizeof(unsigned long long) * CNT_N},
                      {ctx->h_dev + 128, ctx->d_err, sizeof(unsigned)},
                      {ctx->h_dev + 512, ctx->d_scal, sizeof(uint64_t) * SC_WORDS}}));
  TRY(sync_check(ctx, st));
  const unsigned e = *reinterpret_cast<unsigned*>(h + 128);
  TRY(device_error(ctx, e));
  const uint64_t* sc = reinterpret_cast<const uint64_t*>(h + 512);
  const unsigned long long* cnt = reinterpret_cast<const unsigned long long*>(h);
  // finest blocks whose records did not fit shared memory: keep their records from now on
  if (cnt[CNT_BIG_BLOCKS] > 0 && !ctx->want_spill && P.adjacency) ctx->want_spill = true;
  amr_refine_result r{};
  r.n_levels = P.NL;
  for (int L = 0; L < P.NL; ++L) {
    // record staging that overflowed (those blocks were re-walked): grow it on the next eager pass
    const int64_t nrec = (int64_t)sc[SC_REC + L];
    if (P.adjacency && P.fin_at[L] && nrec > ctx->cap_recs && nrec + nrec / 4 + 1024 > ctx->want_recs)
      ctx->want_recs = nrec + nrec / 4 + 1024;
    r.n_blocks[L] = (int64_t)sc[SC_N + L];
    r.block_coords[L] = static_cast<const int32_t*>(ctx->lv[L].blocks.p);
    r.block_parent[L] = L > 0 ? static_cast<const int32_t*>(ctx->lv[L].parent.p) : nullptr;
    r.cell_mask[L] = static_cast<const uint64_t*>(ctx->lv[L].mask.p);
    r.block_flag[L] = static_cast<const uint8_t*>(ctx->lv[L].flag.p);
  }
  if (P.adjacency) {
    r.n_adj_cells = (int64_t)sc[SC_RUN + 0];
    r.n_adj_pairs = (int64_t)sc[SC_RUN + 1];
    r.adj_cell = static_cast<const uint32_t*>(ctx->adj_cell.p);
    r.adj_off = static_cast<const uint32_t*>(ctx->adj_off.p);
    r.adj_ids = static_cast<const uint32_t*>(ctx->adj_ids.p);
  }
  if (P.links) {
    r.n_links = (int64_t)sc[SC_RUN + 2];
    r.link_cell = static_cast<const uint32_t*>(ctx->link_cell.p);
    r.link_dir = static_cast<const uint8_t*>(ctx->link_dir.p);
    r.link_q = static_cast<const float*>(ctx->link_q.p);
    r.link_face = static_cast<const uint32_t*>(ctx->link_face.p);
  }
  r.n_fallback = (int64_t)(cnt[CNT_FALLBACK] + cnt[CNT_LINK_FALLBACK]);
  r.n_band = (int64_t)(cnt[CNT_BAND] + cnt[CNT_LINK_BAND]);
  r.n_candidates = (int64_t)cnt[CNT_CANDIDATES];
  r.n_survivors = (int64_t)cnt[CNT_SURVIVORS];
  r.n_link_candidates = (int64_t)cnt[CNT_LINK_CAND];
  r.n_face_setups = (int64_t)cnt[CNT_FACE_SETUPS];
  r.n_face_tests = (int64_t)cnt[CNT_FACE_TESTS];
  // per-level block pointers for the adjoint
  TRY(ensure(ctx, ctx->lvl_ptrs, sizeof(void*) * AMR_MAX_LEVELS));
  const int32_t** hp = reinterpret_cast<const int32_t**>(h + 256);
  for (int L = 0; L < AMR_MAX_LEVELS; ++L) hp[L] = L < P.NL ? r.block_coords[L] : nullptr;
  TRY(small_copy(ctx, st, {{ctx->lvl_ptrs.p, ctx->h_dev + 256, sizeof(void*) * AMR_MAX_LEVELS}}));
  CK(cudaStreamSynchronize(st));
  *out = r;
  return AMR_OK;
}

}  // namespace

// Eager pass (or graph replay when the inputs match the captured graph), then
// capture when graph mode is asked for.
amr_status amr_run_refine(amr_ctx* ctx, const amr_refine_params* prm, amr_refine_result* out) {
  Plan P = make_plan(ctx, prm);
  const uint64_t face_sig = assign_face_levels(ctx, P, prm);
  if (ctx->multi)  // the rows now carry the face_levels bits
    CK(cudaMemcpyAsync(ctx->table.p, ctx->geoms.data(), sizeof(GeomParams) * ctx->geoms.size(),
                       cudaMemcpyHostToDevice, ctx->stream));
  GraphKey key;
  key.layout_gen = ctx->layout_gen;
  key.nf = ctx->nf;
  key.n_geom = (int64_t)ctx->geoms.size();
  key.B = ctx->geoms[0].B;
  key.n_levels = prm->n_levels;
  key.lattice = prm->lattice;
  key.adjacency = P.adjacency;
  key.links = P.links;
  key.warps = P.warps;
  key.d_abs = prm->d_abs;
  key.d_rel = prm->d_rel;
  key.pred = prm->predicate;
  key.search = prm->search;
  key.prop = prm->propagate;
  key.face_levels = face_sig;
  key.bins = ctx->sampled_bins ? 1ull : 0ull;
  for (const auto& g : ctx->geoms) key.bins = (key.bins ^ (uint64_t)g.B) * 1099511628211ull;
  const bool want_graph = prm->use_graph != 0;
  if (want_graph && ctx->gexec && ctx->gkey == key) {
    // replay on the graph stream, ordered after the caller's stream
    CK(cudaEventRecord(ctx->ev_in, ctx->stream));
    CK(cudaStreamWaitEvent(ctx->gstream, ctx->ev_in, 0));
    CK(cudaGraphLaunch(ctx->gexec, ctx->gstream));
    ctx->launches += ctx->graph_launches;
    CK(cudaEventRecord(ctx->ev_out, ctx->gstream));
    CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_out, 0));
    amr_refine_result r{};
    const amr_status s = collect(ctx, P, ctx->stream, &r);
    if (s == AMR_OK) {
      r.graph_replay = 1;
      *out = r;
      // next call: an eager pass with more record staging or the spill area
      if (ctx->want_recs > ctx->cap_recs || (ctx->want_spill && !ctx->spill.p)) drop_graph(ctx);
      return AMR_OK;
    }
    if (s != AMR_EOVERFLOW) return s;
    drop_graph(ctx);  // sizes outgrew the capacities: redo eagerly
  }
  TRY(engine_pass(ctx, P, true, want_graph, ctx->stream));
  TRY(collect(ctx, P, ctx->stream, out));
  if (want_graph) {
    drop_graph(ctx);
    key.layout_gen = ctx->layout_gen;
    ctx->capturing = true;
    const int64_t before = ctx->launches;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal);
    amr_status s = AMR_OK;
    if (e == cudaSuccess) s = engine_pass(ctx, P, false, false, ctx->gstream);
    const cudaError_t e2 = cudaStreamEndCapture(ctx->gstream, &graph);
    ctx->capturing = false;
    ctx->graph_launches = ctx->launches - before;
    ctx->launches = before;
    if (e != cudaSuccess || e2 != cudaSuccess || s != AMR_OK) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return fail(ctx, AMR_ECUDA, "graph capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&ctx->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      ctx->gexec = nullptr;
      return fail(ctx, AMR_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    }
    ctx->gkey = key;
  }
  return AMR_OK;
}

extern "C" {

const char* amr_status_str(amr_status s) {
  switch (s) {
    case AMR_OK: return "ok";
    case AMR_EINVAL: return "invalid argument";
    case AMR_ENOMEM: return "out of memory";
    case AMR_ECUDA: return "CUDA error";
    case AMR_EOVERFLOW: return "size overflow";
    case AMR_ETIMEOUT: return "device wait timed out";
    case AMR_ESTATE: return "call out of order";
    case AMR_EDEVICE_CHECK: return "device-side input check failed";
  }
  return "unknown status";
}

const char* amr_last_error(const amr_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

amr_status amr_create(const amr_domain* dom, amr_ctx** out) {
  if (!out) return AMR_EINVAL;
  *out = nullptr;
  if (!dom || (dom->dim != 2 && dom->dim != 3) || !(dom->h0 > 0.0)) return AMR_EINVAL;
  for (int a = 0; a < dom->dim; ++a)
    if (dom->root_blocks[a] < 1 || dom->root_blocks[a] > (1 << 20)) return AMR_EINVAL;
  if (!dom->dev_alloc != !dom->dev_free) return AMR_EINVAL;  // both allocator hooks or neither
  amr_ctx* ctx = new amr_ctx();
  ctx->dom = *dom;
  for (int a = dom->dim; a < 3; ++a) ctx->dom.root_blocks[a] = 1;
  if (dom->stream) ctx->stream = static_cast<cudaStream_t>(dom->stream);
  const amr_status s = amr_ctx_init(ctx);
  if (s != AMR_OK) {
    amr_ctx_free(ctx);
    delete ctx;
    return s;
  }
  ctx->geoms.push_back(amr_make_row(ctx->dom, 1, 1, 0.0, 1.0));
  *out = ctx;
  return AMR_OK;
}

amr_status amr_destroy(amr_ctx* ctx) {
  if (!ctx) return AMR_OK;
  amr_ctx_free(ctx);
  delete ctx;
  return AMR_OK;
}

amr_status amr_set_stream(amr_ctx* ctx, void* stream) {
  if (!ctx) return AMR_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream));
  if (ctx->own_stream && stream) {
    cudaStreamDestroy(ctx->stream);
    ctx->own_stream = false;
  }
  if (stream) {
    ctx->stream = static_cast<cudaStream_t>(stream);
  } else if (!ctx->own_stream) {
    CK(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
    ctx->own_stream = true;
  }
  return AMR_OK;
}

amr_status amr_sync(amr_ctx* ctx) {
  if (!ctx) return AMR_EINVAL;
  unsigned e = 0;
  TRY(read_back(ctx, ctx->stream, &e, nullptr, 0));
  return device_error(ctx, e);
}

amr_status amr_geom_load(amr_ctx* ctx, const float* coords, int64_t n_verts, const int32_t* idx, int64_t n_faces) {
  if (!ctx) return AMR_EINVAL;
  if (ctx->multi) return fail(ctx, AMR_ESTATE, "amr_geom_load on a batch context");
  const int D = ctx->dom.dim;
  if (n_faces < 0 || n_faces >= kMaxFaces) return fail(ctx, AMR_EINVAL, "n_faces must be in [0, 2^29)");
  if (n_faces > 0 && !coords) return fail(ctx, AMR_EINVAL, "null coordinates");
  if (idx && n_verts <= 0 && n_faces > 0) return fail(ctx, AMR_EINVAL, "indexed input needs n_verts > 0");
  ctx->loaded = ctx->binned = ctx->refined = false;
  ctx->vert_groups = ctx->face_groups = false;
  ctx->nf = n_faces;
  ctx->nv = idx ? n_verts : 0;
  ctx->indexed = idx != nullptr;
  TRY(ensure(ctx, ctx->X, sizeof(float) * D * D * (size_t)(n_faces > 0 ? n_faces : 1)));
  if (D == 3) TRY(ensure(ctx, ctx->nrm, sizeof(float) * 6 * (size_t)(n_faces > 0 ? n_faces : 1)));
  if (D == 3) TRY(ensure(ctx, ctx->frec, sizeof(FaceRec3) * (size_t)(n_faces > 0 ? n_faces : 1)));
  cudaStream_t st = ctx->stream;
  if (n_faces > 0) {
    if (idx) {
      const void* dv = nullptr;
      const void* di = nullptr;
      TRY(to_device(ctx, coords, sizeof(float) * D * (size_t)n_verts, ctx->stage_a, &dv));
      TRY(to_device(ctx, idx, sizeof(int32_t) * D * (size_t)n_faces, ctx->stage_b, &di));
      TRY(ensure(ctx, ctx->idx, sizeof(int32_t) * D * (size_t)n_faces));
      CK(cudaMemcpyAsync(ctx->idx.p, di, sizeof(int32_t) * D * (size_t)n_faces, cudaMemcpyDeviceToDevice, st));
      timed(ctx, st, "load_gather", [&] {
        return launch_load_indexed(D, static_cast<const float*>(dv), n_verts, static_cast<const int32_t*>(di),
                                   n_faces, static_cast<float*>(ctx->X.p), ctx->d_err, st);
      });
    } else {
      const void* dc = nullptr;
      TRY(to_device(ctx, coords, sizeof(float) * D * D * (size_t)n_faces, ctx->stage_a, &dc));
      timed(ctx, st, "load_gather", [&] {
        return launch_load_facelist(D, static_cast<const float*>(dc), n_faces, static_cast<float*>(ctx->X.p),
                                    ctx->d_err, st);
      });
    }
    if (D == 3)
      timed(ctx, st, "face_normals", [&] {
        return launch_face_normals(static_cast<const float*>(ctx->X.p), n_faces, static_cast<float*>(ctx->nrm.p),
                                   static_cast<FaceRec3*>(ctx->frec.p), st);
      });
  }
  CK(cudaGetLastError());
  ctx->loaded = true;
  ++ctx->load_gen;
  return AMR_OK;
}

static amr_status bin_faces_impl(amr_ctx* ctx, int B, amr_bins_view* out, bool sampled) {
  if (!ctx || !out) return AMR_EINVAL;
  if (ctx->multi) return fail(ctx, AMR_ESTATE, "amr_bin_faces on a batch context");
  if (!ctx->loaded) return fail(ctx, AMR_ESTATE, "amr_bin_faces before amr_geom_load");
  const int D = ctx->dom.dim;
  if (B < 1 || B > 65535) return fail(ctx, AMR_EINVAL, "bin density must be in [1, 65535]");
  const int64_t nb = ipow(B, D);
  if (nb > (1ll << 30)) return fail(ctx, AMR_EINVAL, "B^dim must not exceed 2^30");
  ctx->binned = ctx->refined = false;
  const GeomParams prev = ctx->geoms[0];
  ctx->geoms[0] = amr_make_row(ctx->dom, B, prev.n_levels, prev.d_abs, prev.d_rel);
  ctx->sampled_bins = sampled;
  TRY(amr_bin_all(ctx));
  ctx->B = B;
  out->B = B;
  out->n_bins = nb;
  out->nnz = ctx->nnz;
  out->offsets = static_cast<const uint32_t*>(ctx->offsets.p);
  out->ids = static_cast<const uint32_t*>(ctx->ids.p);
  out->payload = ctx->payload.p;
  out->payload_bytes = D == 3 ? (int64_t)sizeof(Entry3) : (int64_t)sizeof(Entry2);
  return AMR_OK;
}

amr_status amr_bin_faces(amr_ctx* ctx, int B, amr_bins_view* out) { return bin_faces_impl(ctx, B, out, false); }

amr_status amr_bin_faces_sampled(amr_ctx* ctx, int B, amr_bins_view* out) { return bin_faces_impl(ctx, B, out, true); }

amr_status amr_refine_near_wall(amr_ctx* ctx, const amr_refine_params* prm, amr_refine_result* out) {
  if (!ctx || !prm || !out) return AMR_EINVAL;
  if (ctx->multi) return fail(ctx, AMR_ESTATE, "use amr_batch_run on a batch context");
  if (!ctx->binned) return fail(ctx, AMR_ESTATE, "amr_refine_near_wall before amr_bin_faces");
  const int D = ctx->dom.dim;
  const int NL = prm->n_levels;
  if (NL < 1 || NL > AMR_MAX_LEVELS) return fail(ctx, AMR_EINVAL, "n_levels must be in [1, %d]", AMR_MAX_LEVELS);
  if (!(prm->d_abs >= 0.0) || !(prm->d_rel >= 0.0)) return fail(ctx, AMR_EINVAL, "negative near-wall distance");
  if (prm->warps_per_cta < 0 || prm->warps_per_cta > 8) return fail(ctx, AMR_EINVAL, "warps_per_cta in [0, 8]");
  if (prm->predicate != AMR_PRED_BOX && prm->predicate != AMR_PRED_POINT)
    return fail(ctx, AMR_EINVAL, "predicate must be AMR_PRED_BOX (0) or AMR_PRED_POINT (1)");
  if (prm->search != AMR_SEARCH_QUERY_BOX && prm->search != AMR_SEARCH_OWN_BIN)
    return fail(ctx, AMR_EINVAL, "search must be AMR_SEARCH_QUERY_BOX (0) or AMR_SEARCH_OWN_BIN (1)");
  if (prm->search == AMR_SEARCH_OWN_BIN && (prm->predicate != AMR_PRED_POINT || prm->want_links))
    return fail(ctx, AMR_EINVAL, "the own-bin search needs the point predicate and no links");
  if (ctx->sampled_bins && prm->search != AMR_SEARCH_OWN_BIN)
    return fail(ctx, AMR_EINVAL, "sampled bins only serve the own-bin search");
  if (prm->propagate < -1) return fail(ctx, AMR_EINVAL, "propagate must be >= -1");
  if (prm->face_pass < AMR_FACE_PASS_AUTO || prm->face_pass > AMR_FACE_PASS_ON)
    return fail(ctx, AMR_EINVAL, "face_pass must be AMR_FACE_PASS_AUTO (0), _OFF (1) or _ON (2)");
  if (prm->propagate != 0) {
    for (int a = 0; a < D; ++a)
      if ((int64_t)ctx->dom.root_blocks[a] << (NL - 1) >= (1ll << 21))
        return fail(ctx, AMR_EINVAL, "propagation needs block coordinates below 2^21 on every level");
  }
  if (prm->want_links) {
    if (!((D == 2 && prm->lattice == 9) || (D == 3 && prm->lattice == 19)))
      return fail(ctx, AMR_EINVAL, "lattice must be 9 (D2Q9) in 2D or 19 (D3Q19) in 3D");
    const double hf = ctx->dom.h0 * std::ldexp(1.0, -(NL - 1));
    if (prm->d_abs + prm->d_rel * hf < link_reach(prm->predicate) * hf)
      return fail(ctx, AMR_EINVAL, "links need d_L >= %s h_L on the finest level",
                  prm->predicate == AMR_PRED_POINT ? "sqrt(2)" : "1/2");
  }
  int64_t N0 = 1;
  for (int a = 0; a < D; ++a) N0 *= ctx->dom.root_blocks[a];
  if (N0 > (1ll << 31)) return fail(ctx, AMR_EINVAL, "too many root blocks");
  // keep the previous hierarchy's block lists for amr_adapt_diff_get
  ctx->prev_levels = -1;
  if (prm->keep_previous) {
    // the block lists of the last successful refinement are still in the level buffers
    // (loading and binning do not touch them)
    const int pl = ctx->last.n_levels;
    for (int L = 0; L < pl; ++L) {
      const int64_t n = ctx->last.n_blocks[L];
      LevelBufs& lb = ctx->lv[L];
      TRY(ensure_aux(ctx, lb.prev, sizeof(int32_t) * D * (size_t)(n > 0 ? n : 1)));
      if (n > 0)
        CK(cudaMemcpyAsync(lb.prev.p, lb.blocks.p, sizeof(int32_t) * D * (size_t)n, cudaMemcpyDeviceToDevice,
                           ctx->stream));
      lb.n_prev = n;
    }
    ctx->prev_levels = pl;
  }
  ctx->refined = false;
  ctx->classified = false;
  ctx->face_groups = false;
  ctx->n_links = 0;
  ctx->last.n_levels = 0;  // until this refinement succeeds
  GeomParams& g = ctx->geoms[0];
  g.n_levels = NL;
  g.d_abs = prm->d_abs;
  g.d_rel = prm->d_rel;
  amr_finish_row(g);
  amr_refine_result r{};
  TRY(amr_run_refine(ctx, prm, &r));
  ctx->refined = true;
  ctx->last = r;
  ctx->n_links = prm->want_links ? r.n_links : -1;
  *out = r;
  return AMR_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// adjoint
// ---------------------------------------------------------------------------
namespace {

int key_bits(int64_t n) {
  int b = 1;
  while (b < 32 && ((int64_t)1 << b) < n) ++b;
  return b;
}

// Stable grouping of `n` keys in [0, n_keys): CSR offsets [n_keys + 1] and the
// values (0..n-1) in ascending order within each key.
amr_status group_by_key(amr_ctx* ctx, const uint32_t* keys, int64_t n, int64_t n_keys, DevBuf& off, DevBuf& grouped,
                        const char* name) {
  cudaStream_t st = ctx->stream;
  TRY(ensure(ctx, off, sizeof(uint32_t) * (size_t)(n_keys + 1)));
  TRY(ensure(ctx, grouped, sizeof(uint32_t) * (size_t)(n > 0 ? n : 1)));
  TRY(ensure(ctx, ctx->sort_scratch, radix_sort_scratch_bytes(n)));
  TRY(ensure(ctx, ctx->scratch, scan_u32_scratch_bytes(n_keys)));
  TRY(ensure(ctx, ctx->group_cnt, sizeof(uint32_t) * (size_t)(n_keys > 0 ? n_keys : 1)));
  CK(cudaMemsetAsync(ctx->group_cnt.p, 0, sizeof(uint32_t) * (size_t)(n_keys > 0 ? n_keys : 1), st));
  timed(ctx, st, name, [&] {
    int k = launch_count_keys(keys, n, static_cast<uint32_t*>(ctx->group_cnt.p), st);
    k += launch_scan_u32(static_cast<const uint32_t*>(ctx->group_cnt.p), static_cast<uint32_t*>(off.p), n_keys,
                         ctx->d_tot, ctx->scratch.p, ctx->d_err, st);
    k += launch_stable_sort(keys, n, key_bits(n_keys), nullptr,
                            static_cast<uint32_t*>(grouped.p), nullptr, ctx->sort_scratch.p, ctx->d_tot, ctx->d_err,
                            st);
    return k;
  });
  CK(cudaGetLastError());
  return AMR_OK;
}

}  // namespace

amr_status amr_backward(amr_ctx* ctx, const float* grad_q, float* grad_out) {
  const int D = ctx->dom.dim;
  const int64_t nl = ctx->n_links, nf = ctx->nf;
  if (!ctx->face_groups) {
    TRY(group_by_key(ctx, static_cast<const uint32_t*>(ctx->link_face.p), nl, nf, ctx->face_off, ctx->face_links,
                     "adjoint_group_links"));
    ctx->face_groups = true;
  }
  const bool indexed = ctx->indexed;
  if (indexed && !ctx->vert_groups) {
    TRY(group_by_key(ctx, static_cast<const uint32_t*>(ctx->idx.p), nf * D, ctx->nv, ctx->vert_off,
                     ctx->vert_corners, "adjoint_group_corners"));
    ctx->vert_groups = true;
  }
  float* gface = grad_out;
  if (indexed) {
    TRY(ensure(ctx, ctx->grad_face, sizeof(float) * D * D * (size_t)(nf > 0 ? nf : 1)));
    gface = static_cast<float*>(ctx->grad_face.p);
  }
  AdjointArgs a{};
  a.dim = D;
  a.nf = nf;
  a.g0 = ctx->geoms[0];
  a.table = ctx->multi ? static_cast<const GeomParams*>(ctx->table.p) : nullptr;
  a.face_gid = ctx->multi ? static_cast<const uint32_t*>(ctx->face_gid.p) : nullptr;
  a.level_blocks = static_cast<const int32_t* const*>(ctx->lvl_ptrs.p);
  a.X = static_cast<const float*>(ctx->X.p);
  a.nrm = static_cast<const float*>(ctx->nrm.p);
  a.face_off = static_cast<const uint32_t*>(ctx->face_off.p);
  a.face_links = static_cast<const uint32_t*>(ctx->face_links.p);
  a.grad_q = grad_q;
  a.link_cell = static_cast<const uint32_t*>(ctx->link_cell.p);
  a.link_dir = static_cast<const uint8_t*>(ctx->link_dir.p);
  a.link_q = static_cast<const float*>(ctx->link_q.p);
  a.adj_cell = static_cast<const uint32_t*>(ctx->adj_cell.p);
  a.grad_face = gface;
  cudaStream_t st = ctx->stream;
  timed(ctx, st, "adjoint_face", [&] { return launch_face_grad(a, st); });
  if (indexed)
    timed(ctx, st, "adjoint_vertex", [&] {
      return launch_vertex_grad(D, gface, static_cast<const uint32_t*>(ctx->vert_off.p),
                                static_cast<const uint32_t*>(ctx->vert_corners.p), ctx->nv, grad_out, st);
    });
  CK(cudaGetLastError());
  return AMR_OK;
}

extern "C" {

amr_status amr_q_backward(amr_ctx* ctx, const float* grad_q, float* grad_out) {
  if (!ctx) return AMR_EINVAL;
  if (!ctx->refined || ctx->n_links < 0)
    return fail(ctx, AMR_ESTATE, "amr_q_backward needs a preceding refinement with links");
  const int64_t nl = ctx->n_links;
  if (!grad_out || (nl > 0 && !grad_q)) return fail(ctx, AMR_EINVAL, "null gradient pointer");
  if ((nl > 0 && !is_device_ptr(grad_q)) || !is_device_ptr(grad_out))
    return fail(ctx, AMR_EINVAL, "gradients must be device pointers");
  return amr_backward(ctx, grad_q, grad_out);
}

amr_status amr_classify_nodes(amr_ctx* ctx, const uint8_t** cell_solid, int64_t* n_fallback) {
  if (!ctx || !cell_solid) return AMR_EINVAL;
  if (ctx->multi) return fail(ctx, AMR_ESTATE, "node classification on a batch context");
  if (!ctx->refined || !ctx->last.adj_cell)
    return fail(ctx, AMR_ESTATE, "amr_classify_nodes needs a preceding refinement with adjacency");
  if (ctx->sampled_bins) return fail(ctx, AMR_EINVAL, "node classification needs exact bins");
  const amr_refine_result& r = ctx->last;
  const int64_t n = r.n_adj_cells;
  cudaStream_t st = ctx->stream;
  TRY(ensure(ctx, ctx->cls, (size_t)(n > 0 ? n : 1)));
  CK(cudaMemsetAsync(ctx->counters + CNT_CLASS_FALLBACK, 0, sizeof(unsigned long long), st));
  ClassifyArgs a{};
  a.dim = ctx->dom.dim;
  a.level = r.n_levels - 1;
  a.g0 = ctx->geoms[0];
  a.blocks = r.block_coords[r.n_levels - 1];
  a.adj_cell = r.adj_cell;
  a.row0 = 0;
  a.n_rows = n;
  a.offsets = static_cast<const uint32_t*>(ctx->offsets.p);
  a.payload = ctx->payload.p;
  a.X = static_cast<const float*>(ctx->X.p);
  a.nf = ctx->nf;
  a.cls = static_cast<uint8_t*>(ctx->cls.p);
  a.counters = ctx->counters;
  a.err = ctx->d_err;
  timed(ctx, st, "classify", [&] { return launch_classify(a, st); });
  CK(cudaGetLastError());
  char* h = static_cast<char*>(ctx->h_pinned);
  TRY(small_copy(ctx, st, {{ctx->h_dev, ctx->counters + CNT_CLASS_FALLBACK, sizeof(unsigned long long)},
                      {ctx->h_dev + 64, ctx->d_err, sizeof(unsigned)}}));
  TRY(sync_check(ctx, st));
  TRY(device_error(ctx, *reinterpret_cast<unsigned*>(h + 64)));
  if (n_fallback) *n_fallback = (int64_t)*reinterpret_cast<unsigned long long*>(h);
  ctx->classified = true;
  *cell_solid = static_cast<const uint8_t*>(ctx->cls.p);
  return AMR_OK;
}

amr_status amr_fluid_links(amr_ctx* ctx, amr_refine_result* out) {
  if (!ctx || !out) return AMR_EINVAL;
  if (!ctx->refined || !ctx->classified || ctx->n_links < 0)
    return fail(ctx, AMR_ESTATE, "amr_fluid_links needs links and a preceding amr_classify_nodes");
  const int64_t n = ctx->n_links;
  cudaStream_t st = ctx->stream;
  if (n > 0) {
    const int64_t nb = fluid_blocks(n);
    TRY(ensure(ctx, ctx->group_cnt, sizeof(uint32_t) * (size_t)(nb + 1)));
    TRY(ensure(ctx, ctx->flbase, sizeof(uint32_t) * (size_t)(nb + 1)));
    TRY(ensure(ctx, ctx->scratch, scan_u32_scratch_bytes(nb)));
    TRY(ensure(ctx, ctx->tl_cell, sizeof(uint32_t) * (size_t)n));
    TRY(ensure(ctx, ctx->tl_dir, (size_t)n));
    TRY(ensure(ctx, ctx->tl_q, sizeof(float) * (size_t)n));
    TRY(ensure(ctx, ctx->tl_face, sizeof(uint32_t) * (size_t)n));
    const uint8_t* cls = static_cast<const uint8_t*>(ctx->cls.p);
    auto* lc = static_cast<uint32_t*>(ctx->link_cell.p);
    auto* ld = static_cast<uint8_t*>(ctx->link_dir.p);
    auto* lq = static_cast<float*>(ctx->link_q.p);
    auto* lf = static_cast<uint32_t*>(ctx->link_face.p);
    timed(ctx, st, "fluid_links", [&] {
      int k = launch_fluid_count(lc, cls, n, static_cast<uint32_t*>(ctx->group_cnt.p), st);
      k += launch_scan_u32(static_cast<const uint32_t*>(ctx->group_cnt.p), static_cast<uint32_t*>(ctx->flbase.p), nb,
                           ctx->d_tot, ctx->scratch.p, ctx->d_err, st);
      k += launch_fluid_move(lc, ld, lq, lf, cls, n, static_cast<const uint32_t*>(ctx->flbase.p),
                             static_cast<uint32_t*>(ctx->tl_cell.p), static_cast<uint8_t*>(ctx->tl_dir.p),
                             static_cast<float*>(ctx->tl_q.p), static_cast<uint32_t*>(ctx->tl_face.p), st);
      return k;
    });
    uint64_t kept = 0;
    unsigned e = 0;
    char* h = static_cast<char*>(ctx->h_pinned);
    TRY(small_copy(ctx, st, {{ctx->h_dev + 128, ctx->d_tot, sizeof(uint64_t)},
                        {ctx->h_dev + 64, ctx->d_err, sizeof(unsigned)}}));
    TRY(sync_check(ctx, st));
    kept = *reinterpret_cast<uint64_t*>(h + 128);
    e = *reinterpret_cast<unsigned*>(h + 64);
    TRY(device_error(ctx, e));
    // back into the context's link arrays (graph replays keep writing there)
    CK(cudaMemcpyAsync(lc, ctx->tl_cell.p, sizeof(uint32_t) * kept, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(ld, ctx->tl_dir.p, kept, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(lq, ctx->tl_q.p, sizeof(float) * kept, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(lf, ctx->tl_face.p, sizeof(uint32_t) * kept, cudaMemcpyDeviceToDevice, st));
    ctx->n_links = (int64_t)kept;
  }
  ctx->face_groups = false;
  ctx->last.n_links = ctx->n_links;
  *out = ctx->last;
  return AMR_OK;
}

amr_status amr_adapt_diff_get(amr_ctx* ctx, amr_adapt_diff* out) {
  if (!ctx || !out) return AMR_EINVAL;
  if (ctx->multi) return fail(ctx, AMR_ESTATE, "re-adaptation maps on a batch context");
  if (!ctx->refined || ctx->prev_levels < 0)
    return fail(ctx, AMR_ESTATE, "amr_adapt_diff_get needs a refinement with keep_previous after another");
  const int D = ctx->dom.dim;
  const amr_refine_result& r = ctx->last;
  cudaStream_t st = ctx->stream;
  amr_adapt_diff d{};
  d.n_levels = r.n_levels;
  int64_t cap = 1;
  for (int L = 0; L < AMR_MAX_LEVELS; ++L) {
    const int64_t nn = L < r.n_levels ? r.n_blocks[L] : 0, no = L < ctx->prev_levels ? ctx->lv[L].n_prev : 0;
    cap = std::max(cap, std::max(nn, no));
  }
  const uint32_t slots = propagate_hash_slots(cap);
  TRY(ensure_aux(ctx, ctx->mkeys, sizeof(unsigned long long) * slots));
  TRY(ensure_aux(ctx, ctx->mvals, sizeof(uint32_t) * slots));
  unsigned long long* cnt = ctx->counters;  // [0 .. 2 * levels) as scratch for the missing counts
  const int nl = std::max(r.n_levels, ctx->prev_levels);
  if (2 * nl > CNT_N) {
    TRY(ensure(ctx, ctx->group_cnt, sizeof(unsigned long long) * 2 * (size_t)nl));
    cnt = static_cast<unsigned long long*>(ctx->group_cnt.p);
  }
  CK(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * 2 * (size_t)nl, st));
  for (int L = 0; L < nl; ++L) {
    LevelBufs& lb = ctx->lv[L];
    const int64_t nn = L < r.n_levels ? r.n_blocks[L] : 0;
    const int64_t no = L < ctx->prev_levels ? lb.n_prev : 0;
    TRY(ensure_aux(ctx, lb.n2o, sizeof(int32_t) * (size_t)(nn > 0 ? nn : 1)));
    TRY(ensure_aux(ctx, lb.o2n, sizeof(int32_t) * (size_t)(no > 0 ? no : 1)));
    const int32_t* nb = static_cast<const int32_t*>(lb.blocks.p);
    const int32_t* ob = static_cast<const int32_t*>(lb.prev.p);
    timed(ctx, st, "adapt_diff", [&] {
      int k = launch_block_map(D, ob, no, nb, nn, static_cast<int32_t*>(lb.n2o.p), cnt + 2 * L,
                               static_cast<unsigned long long*>(ctx->mkeys.p), static_cast<uint32_t*>(ctx->mvals.p),
                               slots, ctx->d_err, st);
      k += launch_block_map(D, nb, nn, ob, no, static_cast<int32_t*>(lb.o2n.p), cnt + 2 * L + 1,
                            static_cast<unsigned long long*>(ctx->mkeys.p), static_cast<uint32_t*>(ctx->mvals.p),
                            slots, ctx->d_err, st);
      return k;
    });
    d.n_new[L] = nn;
    d.n_old[L] = no;
    d.new_to_old[L] = static_cast<const int32_t*>(lb.n2o.p);
    d.old_to_new[L] = static_cast<const int32_t*>(lb.o2n.p);
  }
  CK(cudaGetLastError());
  // counts at 1280 of the pinned block (2 x 16 levels at most), the error word at 64
  TRY(small_copy(ctx, st, {{ctx->h_dev + 1280, cnt, sizeof(unsigned long long) * 2 * (size_t)nl},
                      {ctx->h_dev + 64, ctx->d_err, sizeof(unsigned)}}));
  TRY(sync_check(ctx, st));
  const unsigned long long* h = reinterpret_cast<const unsigned long long*>(static_cast<char*>(ctx->h_pinned) + 1280);
  TRY(device_error(ctx, *reinterpret_cast<const unsigned*>(static_cast<char*>(ctx->h_pinned) + 64)));
  for (int L = 0; L < nl; ++L) {
    d.n_created[L] = (int64_t)h[2 * L];
    d.n_removed[L] = (int64_t)h[2 * L + 1];
  }
  *out = d;
  return AMR_OK;
}

amr_status amr_candidate_count(amr_ctx* ctx, int64_t* per_level, int64_t* total) {
  if (!ctx || !per_level) return AMR_EINVAL;
  if (ctx->multi) return fail(ctx, AMR_ESTATE, "amr_candidate_count on a batch context");
  if (!ctx->refined) return fail(ctx, AMR_ESTATE, "amr_candidate_count before amr_refine_near_wall");
  cudaStream_t st = ctx->stream;
  const amr_refine_result& r = ctx->last;
  TRY(ensure_aux(ctx, ctx->calg, sizeof(unsigned long long) * AMR_MAX_LEVELS));
  CK(cudaMemsetAsync(ctx->calg.p, 0, sizeof(unsigned long long) * AMR_MAX_LEVELS, st));
  unsigned long long* out = static_cast<unsigned long long*>(ctx->calg.p);
  for (int L = 0; L < r.n_levels; ++L) {
    if (r.n_blocks[L] <= 0) continue;
    CountArgs a{};
    a.dim = ctx->dom.dim;
    a.level = L;
    a.g0 = ctx->geoms[0];
    a.blocks = r.block_coords[L];
    a.n = r.n_blocks[L];
    a.offsets = static_cast<const uint32_t*>(ctx->offsets.p);
    a.payload = ctx->payload.p;
    a.out = out + L;
    timed(ctx, st, "candidate_count", [&] { return launch_count_candidates(a, ctx->num_sms, st); });
  }
  CK(cudaGetLastError());
  // counts at 1280 of the pinned block (16 levels at most)
  TRY(small_copy(ctx, st, {{ctx->h_dev + 1280, out, sizeof(unsigned long long) * AMR_MAX_LEVELS}}));
  TRY(sync_check(ctx, st));
  const unsigned long long* h = reinterpret_cast<const unsigned long long*>(static_cast<char*>(ctx->h_pinned) + 1280);
  int64_t tot = 0;
  for (int L = 0; L < AMR_MAX_LEVELS; ++L) {
    per_level[L] = L < r.n_levels ? (int64_t)h[L] : 0;
    tot += per_level[L];
  }
  if (total) *total = tot;
  return AMR_OK;
}

amr_status amr_timing_enable(amr_ctx* ctx, int on) {
  if (!ctx) return AMR_EINVAL;
  ctx->timing = on != 0;
  return AMR_OK;
}

amr_status amr_timing_reset(amr_ctx* ctx) {
  if (!ctx) return AMR_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream));
  harvest_timing(ctx);
  for (auto& s : ctx->slots) {
    s.ms = 0.0;
    s.launches = 0;
  }
  return AMR_OK;
}

int amr_timing_get(amr_ctx* ctx, const char** names, double* total_ms, int64_t* launches, int cap) {
  if (!ctx) return -1;
  cudaStreamSynchronize(ctx->stream);
  harvest_timing(ctx);
  const int n = (int)ctx->slots.size();
  for (int i = 0; i < n && i < cap; ++i) {
    if (names) names[i] = ctx->slots[i].name;
    if (total_ms) total_ms[i] = ctx->slots[i].ms;
    if (launches) launches[i] = ctx->slots[i].launches;
  }
  return n;
}

int64_t amr_launch_count(const amr_ctx* ctx) { return ctx ? ctx->launches : -1; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched mode: many geometries, one level engine.
//
// The geometries are gathered into one face array (face ids are batch-global),
// binned in one pass (each geometry with its own bin grid, concatenated bin
// arrays), and refined level by level: one refine launch and one child
// compaction per level cover every geometry still refining; geometries that end
// on a level form their adjacency lists and links there.  Per-geometry views
// are segments of the concatenated outputs.
// ---------------------------------------------------------------------------
namespace {

struct BatchInput {
  amr_domain dom{};
  int64_t nf = 0, nv = 0;
  bool indexed = false;
  DevBuf coords, idx;  // device copies of the caller's arrays
  int n_levels = 1;
  double d_abs = 0.0, d_rel = 1.0;
  int B = 0;
};

// Per geometry: [0,16) first block per level, [16,32) block count per level,
// 32 row start, 33 row end, 34 pair start, 35 pair end, 36 link start, 37 link end.
constexpr int SEG_WORDS = 40;

__device__ int64_t lower_u32(const uint32_t* a, int64_t n, uint32_t v) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (a[mid] < v)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

struct SegArgs {
  int n_geom, n_levels;
  const uint64_t* scal;
  const uint32_t* gid[AMR_MAX_LEVELS];
  const uint64_t* base[AMR_MAX_LEVELS];
  const GeomParams* table;
  const uint32_t* link_cell;
  int64_t* out;
};

__global__ void k_batch_segments(SegArgs a) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= a.n_geom) return;
  int64_t* o = a.out + (int64_t)g * SEG_WORDS;
  const GeomParams P = a.table[g];
  int64_t run_cells = 0, run_pairs = 0;
  for (int L = 0; L < a.n_levels; ++L) {
    const int64_t n = (int64_t)a.scal[SC_N + L];
    int64_t s = 0, e = 0;
    if (a.gid[L] && n > 0) {
      s = lower_u32(a.gid[L], n, (uint32_t)g);
      e = lower_u32(a.gid[L], n, (uint32_t)g + 1);
    }
    o[L] = s;
    o[16 + L] = e - s;
    const uint64_t tot = a.scal[SC_TOT + L];
    if (L == P.n_levels - 1) {
      const uint64_t bs = s < n ? a.base[L][s] : tot;
      const uint64_t be = e < n ? a.base[L][e] : tot;
      o[32] = run_cells + (int64_t)(bs >> 32);
      o[33] = run_cells + (int64_t)(be >> 32);
      o[34] = run_pairs + (int64_t)(bs & 0xffffffffull);
      o[35] = run_pairs + (int64_t)(be & 0xffffffffull);
    }
    run_cells += (int64_t)(tot >> 32);
    run_pairs += (int64_t)(tot & 0xffffffffull);
  }
  const int64_t nl = (int64_t)a.scal[SC_RUN + 2];
  o[36] = a.link_cell ? lower_u32(a.link_cell, nl, (uint32_t)o[32]) : 0;
  o[37] = a.link_cell ? lower_u32(a.link_cell, nl, (uint32_t)o[33]) : 0;
}

__global__ void k_offset_idx(const int32_t* __restrict__ in, int64_t n, int32_t off, int32_t* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i] + off;
}

}  // namespace

struct amr_batch {
  amr_ctx ctx;
  std::vector<BatchInput> in;
  bool prepared = false;
  std::vector<int64_t> seg;  // SEG_WORDS per geometry, filled by amr_batch_run
  amr_refine_result last{};
  int64_t vert_total = 0;
};

namespace {

// Gather every geometry into the batch's face arrays (face ids batch-global)
// and build the geometry table (bins filled in by amr_bin_all).
amr_status batch_gather(amr_batch* b) {
  amr_ctx* ctx = &b->ctx;
  const int D = ctx->dom.dim;
  cudaStream_t st = ctx->stream;
  int64_t nf = 0, nv = 0, roots = 0;
  ctx->geoms.clear();
  for (auto& x : b->in) {
    GeomParams g = amr_make_row(x.dom, x.B, x.n_levels, x.d_abs, x.d_rel);
    g.face_base = nf;
    g.root_base = roots;
    ctx->geoms.push_back(g);
    nf += x.nf;
    nv += x.nv;
    roots += roots_of(g, D);
  }
  ctx->nf = nf;
  ctx->nv = nv;
  b->vert_total = nv;
  TRY(ensure(ctx, ctx->X, sizeof(float) * D * D * (size_t)(nf > 0 ? nf : 1)));
  if (D == 3) TRY(ensure(ctx, ctx->nrm, sizeof(float) * 6 * (size_t)(nf > 0 ? nf : 1)));
  if (D == 3) TRY(ensure(ctx, ctx->frec, sizeof(FaceRec3) * (size_t)(nf > 0 ? nf : 1)));
  TRY(ensure(ctx, ctx->face_gid, sizeof(uint32_t) * (size_t)(nf > 0 ? nf : 1)));
  TRY(ensure(ctx, ctx->table, sizeof(GeomParams) * ctx->geoms.size()));
  CK(cudaMemcpyAsync(ctx->table.p, ctx->geoms.data(), sizeof(GeomParams) * ctx->geoms.size(), cudaMemcpyHostToDevice,
                     st));
  if (ctx->indexed) TRY(ensure(ctx, ctx->idx, sizeof(int32_t) * D * (size_t)(nf > 0 ? nf : 1)));
  int64_t vbase = 0;
  for (size_t i = 0; i < b->in.size(); ++i) {
    const BatchInput& x = b->in[i];
    const int64_t f0 = ctx->geoms[i].face_base;
    timed(ctx, st, "load_gather", [&] {
      if (x.indexed)
        return launch_load_indexed(D, static_cast<const float*>(x.coords.p), x.nv,
                                   static_cast<const int32_t*>(x.idx.p), x.nf, static_cast<float*>(ctx->X.p),
                                   ctx->d_err, st, nf, f0);
      return launch_load_facelist(D, static_cast<const float*>(x.coords.p), x.nf, static_cast<float*>(ctx->X.p),
                                  ctx->d_err, st, nf, f0);
    });
    if (x.indexed && x.nf > 0) {
      k_offset_idx<<<(unsigned)((x.nf * D + 255) / 256 < 4096 ? (x.nf * D + 255) / 256 : 4096), 256, 0, st>>>(
          static_cast<const int32_t*>(x.idx.p), x.nf * D, (int32_t)vbase, static_cast<int32_t*>(ctx->idx.p) + f0 * D);
      ctx->launches += 1;
    }
    vbase += x.nv;
  }
  if (D == 3)
    timed(ctx, st, "face_normals", [&] {
      return launch_face_normals(static_cast<const float*>(ctx->X.p), nf, static_cast<float*>(ctx->nrm.p),
                                 static_cast<FaceRec3*>(ctx->frec.p), st);
    });
  timed(ctx, st, "face_gid", [&] {
    return launch_face_gid(static_cast<const GeomParams*>(ctx->table.p), (int)ctx->geoms.size(), nf,
                           static_cast<uint32_t*>(ctx->face_gid.p), st);
  });
  CK(cudaGetLastError());
  ctx->loaded = true;
  ++ctx->load_gen;
  ctx->vert_groups = ctx->face_groups = false;
  return AMR_OK;
}

amr_status batch_segments(amr_batch* b, int NL) {
  amr_ctx* ctx = &b->ctx;
  const int G = (int)ctx->geoms.size();
  DevBuf d_out;
  TRY(ensure(ctx, d_out, sizeof(int64_t) * SEG_WORDS * (size_t)G));
  SegArgs sa{};
  sa.n_geom = G;
  sa.n_levels = NL;
  sa.scal = ctx->d_scal;
  for (int L = 0; L < NL; ++L) {
    sa.gid[L] = static_cast<const uint32_t*>(ctx->lv[L].gid.p);
    sa.base[L] = static_cast<const uint64_t*>(ctx->lv[L].base.p);
  }
  sa.table = static_cast<const GeomParams*>(ctx->table.p);
  sa.link_cell = static_cast<const uint32_t*>(ctx->link_cell.p);
  sa.out = static_cast<int64_t*>(d_out.p);
  k_batch_segments<<<(G + 63) / 64, 64, 0, ctx->stream>>>(sa);
  ctx->launches += 1;
  b->seg.assign((size_t)SEG_WORDS * G, 0);
  CK(cudaMemcpyAsync(b->seg.data(), d_out.p, sizeof(int64_t) * SEG_WORDS * (size_t)G, cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  release(ctx, d_out);
  return AMR_OK;
}

}  // namespace

extern "C" {

amr_status amr_batch_create(int dim, void* stream, amr_batch** out) {
  if (!out || (dim != 2 && dim != 3)) return AMR_EINVAL;
  *out = nullptr;
  amr_batch* b = new amr_batch();
  amr_ctx* ctx = &b->ctx;
  ctx->dom.dim = dim;
  ctx->dom.h0 = 1.0;
  ctx->multi = true;
  if (stream) ctx->stream = static_cast<cudaStream_t>(stream);
  const amr_status s = amr_ctx_init(ctx);
  if (s != AMR_OK) {
    amr_ctx_free(ctx);
    delete b;
    return s;
  }
  *out = b;
  return AMR_OK;
}

amr_status amr_batch_destroy(amr_batch* b) {
  if (!b) return AMR_OK;
  amr_ctx* ctx = &b->ctx;
  for (auto& x : b->in) {
    release(ctx, x.coords);
    release(ctx, x.idx);
  }
  amr_ctx_free(ctx);
  delete b;
  return AMR_OK;
}

amr_ctx* amr_batch_context(amr_batch* b) { return b ? &b->ctx : nullptr; }

amr_status amr_batch_add(amr_batch* b, const amr_domain* dom, const float* coords, int64_t n_verts,
                         const int32_t* idx, int64_t n_faces, int n_levels, double d_abs, double d_rel,
                         int bin_density, int* index_out) {
  if (!b || !dom) return AMR_EINVAL;
  amr_ctx* ctx = &b->ctx;
  const int D = ctx->dom.dim;
  if (dom->dim != D || !(dom->h0 > 0.0)) return fail(ctx, AMR_EINVAL, "geometry dim must match the batch");
  for (int a = 0; a < D; ++a)
    if (dom->root_blocks[a] < 1 || dom->root_blocks[a] > (1 << 20)) return fail(ctx, AMR_EINVAL, "bad root_blocks");
  if (n_levels < 1 || n_levels > AMR_MAX_LEVELS) return fail(ctx, AMR_EINVAL, "bad n_levels");
  if (!(d_abs >= 0.0) || !(d_rel >= 0.0)) return fail(ctx, AMR_EINVAL, "negative near-wall distance");
  if (bin_density < 0 || bin_density > 65535) return fail(ctx, AMR_EINVAL, "bad bin density");
  if (n_faces < 0 || (n_faces > 0 && !coords) || (idx && n_verts <= 0 && n_faces > 0))
    return fail(ctx, AMR_EINVAL, "bad geometry arrays");
  // an empty geometry takes the batch's input form
  const bool form = n_faces > 0 ? idx != nullptr : (b->in.empty() ? idx != nullptr : ctx->indexed);
  if (!b->in.empty() && n_faces > 0 && form != ctx->indexed) {
    bool any = false;
    for (auto& y : b->in) any = any || y.nf > 0;
    if (any) return fail(ctx, AMR_EINVAL, "all geometries of a batch use the same input form");
    for (auto& y : b->in) y.indexed = form;
  }
  int64_t total = n_faces;
  for (auto& x : b->in) total += x.nf;
  if (total >= kMaxFaces) return fail(ctx, AMR_EINVAL, "a batch holds fewer than 2^29 faces");
  ctx->indexed = form;
  BatchInput x;
  x.dom = *dom;
  for (int a = D; a < 3; ++a) x.dom.root_blocks[a] = 1;
  x.nf = n_faces;
  x.nv = form ? n_verts : 0;
  x.indexed = form;
  x.n_levels = n_levels;
  x.d_abs = d_abs;
  x.d_rel = d_rel;
  x.B = bin_density;
  const size_t cbytes = n_faces > 0 ? sizeof(float) * (idx ? D * (size_t)n_verts : (size_t)D * D * n_faces) : 0;
  TRY(ensure(ctx, x.coords, cbytes));
  if (cbytes) CK(cudaMemcpyAsync(x.coords.p, coords, cbytes, cudaMemcpyDefault, ctx->stream));
  if (idx && n_faces > 0) {
    TRY(ensure(ctx, x.idx, sizeof(int32_t) * D * (size_t)n_faces));
    CK(cudaMemcpyAsync(x.idx.p, idx, sizeof(int32_t) * D * (size_t)n_faces, cudaMemcpyDefault, ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  b->in.push_back(x);
  b->prepared = false;
  if (index_out) *index_out = (int)b->in.size() - 1;
  return AMR_OK;
}

amr_status amr_batch_set_bins(amr_batch* b, int index, int bin_density) {
  if (!b || index < 0 || index >= (int)b->in.size() || bin_density < 1 || bin_density > 65535) return AMR_EINVAL;
  b->in[index].B = bin_density;
  return AMR_OK;
}

amr_status amr_batch_run(amr_batch* b, const amr_refine_params* prm, amr_refine_result* out) {
  if (!b || !prm || !out) return AMR_EINVAL;
  amr_ctx* ctx = &b->ctx;
  const int D = ctx->dom.dim;
  if (b->in.empty()) return fail(ctx, AMR_ESTATE, "empty batch");
  for (auto& x : b->in)
    if (x.B < 1) return fail(ctx, AMR_ESTATE, "a geometry has no bin density (set it or tune it)");
  if (prm->warps_per_cta < 0 || prm->warps_per_cta > 8) return fail(ctx, AMR_EINVAL, "warps_per_cta in [0, 8]");
  if (prm->predicate != AMR_PRED_BOX && prm->predicate != AMR_PRED_POINT)
    return fail(ctx, AMR_EINVAL, "predicate must be AMR_PRED_BOX (0) or AMR_PRED_POINT (1)");
  if (prm->search != AMR_SEARCH_QUERY_BOX || prm->propagate != 0)
    return fail(ctx, AMR_EINVAL, "batches use the query-box search without propagation");
  if (prm->want_links) {
    if (!((D == 2 && prm->lattice == 9) || (D == 3 && prm->lattice == 19)))
      return fail(ctx, AMR_EINVAL, "lattice must be 9 (D2Q9) in 2D or 19 (D3Q19) in 3D");
    for (auto& x : b->in) {
      const double hf = x.dom.h0 * std::ldexp(1.0, -(x.n_levels - 1));
      if (x.d_abs + x.d_rel * hf < link_reach(prm->predicate) * hf)
        return fail(ctx, AMR_EINVAL, "links need d_L >= %s h_L", prm->predicate == AMR_PRED_POINT ? "sqrt(2)" : "1/2");
    }
  }
  ctx->refined = false;
  ctx->face_groups = false;
  TRY(batch_gather(b));
  TRY(amr_bin_all(ctx));
  amr_refine_result r{};
  TRY(amr_run_refine(ctx, prm, &r));
  TRY(batch_segments(b, r.n_levels));
  ctx->refined = true;
  ctx->last = r;
  ctx->n_links = prm->want_links ? r.n_links : -1;
  b->last = r;
  *out = r;
  return AMR_OK;
}

amr_status amr_batch_get_view(amr_batch* b, int index, amr_batch_view* out) {
  if (!b || !out || index < 0 || index >= (int)b->in.size()) return AMR_EINVAL;
  amr_ctx* ctx = &b->ctx;
  if (!ctx->refined || b->seg.empty()) return fail(ctx, AMR_ESTATE, "amr_batch_get_view before amr_batch_run");
  const int D = ctx->dom.dim;
  const int64_t* s = b->seg.data() + (size_t)SEG_WORDS * index;
  const amr_refine_result& R = b->last;
  amr_batch_view v{};
  const int NL = b->in[index].n_levels;
  v.r.n_levels = NL;
  for (int L = 0; L < NL; ++L) {
    v.level_base[L] = s[L];
    v.r.n_blocks[L] = s[16 + L];
    v.r.block_coords[L] = R.block_coords[L] + s[L] * D;
    v.r.block_parent[L] = L > 0 ? R.block_parent[L] + s[L] : nullptr;
    v.r.cell_mask[L] = R.cell_mask[L] + s[L];
    v.r.block_flag[L] = R.block_flag[L] + s[L];
  }
  v.adj_base = s[32];
  v.pair_base = s[34];
  v.link_base = s[36];
  v.face_base = ctx->geoms[index].face_base;
  int64_t vb = 0;
  for (int i = 0; i < index; ++i) vb += b->in[i].nv;
  v.vert_base = vb;
  if (R.adj_cell) {
    v.r.n_adj_cells = s[33] - s[32];
    v.r.n_adj_pairs = s[35] - s[34];
    v.r.adj_cell = R.adj_cell + s[32];
    v.r.adj_off = R.adj_off + s[32];
    v.r.adj_ids = R.adj_ids + s[34];
  }
  if (R.link_cell) {
    v.r.n_links = s[37] - s[36];
    v.r.link_cell = R.link_cell + s[36];
    v.r.link_dir = R.link_dir + s[36];
    v.r.link_q = R.link_q + s[36];
    v.r.link_face = R.link_face + s[36];
  }
  *out = v;
  return AMR_OK;
}

amr_status amr_batch_q_backward(amr_batch* b, const float* grad_q, float* grad_out) {
  if (!b) return AMR_EINVAL;
  return amr_q_backward(&b->ctx, grad_q, grad_out);
}

const char* amr_batch_last_error(const amr_batch* b) { return b ? b->ctx.err.c_str() : "null batch"; }

int64_t amr_batch_launch_count(const amr_batch* b) { return b ? b->ctx.launches : -1; }

// ---------------------------------------------------------------------------
// Autotuner: the paper's trade-off between bin setup (grows with B) and face
// detection (shrinks with B) decides B; the warps per block of the refine
// kernels are tuned for the chosen B.  Objective = CUDA-event time of
// bin + refine (with the caller's adjacency / link options), best of two runs.
// ---------------------------------------------------------------------------
amr_status amr_autotune(amr_ctx* ctx, const amr_refine_params* prm, const int* b_cand, int n_b, const int* w_cand,
                        int n_w, int* best_B, int* best_warps, double* best_ms) {
  if (!ctx || !prm || !best_B || !best_warps) return AMR_EINVAL;
  if (ctx->multi || !ctx->loaded) return fail(ctx, AMR_ESTATE, "amr_autotune needs a loaded single geometry");
  const int D = ctx->dom.dim;
  std::vector<int> bs, ws;
  if (b_cand && n_b > 0) {
    bs.assign(b_cand, b_cand + n_b);
  } else {
    const int def[] = {4, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256};
    for (int B : def)
      if (ipow(B, D) <= (1ll << 24) && (double)B * B <= 16.0 * (double)(ctx->nf > 16 ? ctx->nf : 16)) bs.push_back(B);
  }
  if (w_cand && n_w > 0)
    ws.assign(w_cand, w_cand + n_w);
  else
    ws = {2, 4, 8};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  auto measure = [&](int B, int warps, double* ms) -> amr_status {
    amr_refine_params p = *prm;
    p.use_graph = 0;
    p.warps_per_cta = warps;
    double best = 1e300;
    for (int rep = 0; rep < 2; ++rep) {
      amr_bins_view bv;
      amr_refine_result r;
      CK(cudaEventRecord(e0, ctx->stream));
      TRY(amr_bin_faces(ctx, B, &bv));
      TRY(amr_refine_near_wall(ctx, &p, &r));
      CK(cudaEventRecord(e1, ctx->stream));
      CK(cudaEventSynchronize(e1));
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, e0, e1));
      if (t < best) best = t;
    }
    *ms = best;
    return AMR_OK;
  };
  int bb = bs.empty() ? 1 : bs[0], bw = prm->warps_per_cta > 0 ? prm->warps_per_cta : 4;
  double bt = 1e300;
  for (int B : bs) {
    double t = 0;
    TRY(measure(B, bw, &t));
    if (t < bt) {
      bt = t;
      bb = B;
    }
  }
  for (int w : ws) {
    if (w < 1 || w > 8) continue;
    double t = 0;
    TRY(measure(bb, w, &t));
    if (t < bt) {
      bt = t;
      bw = w;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *best_B = bb;
  *best_warps = bw;
  if (best_ms) *best_ms = bt;
  return AMR_OK;
}

}  // extern "C"
