// api.cu — host side of the C ABI declared in include/amrgeom.h.
//
// The context owns grow-only device buffers (stream-ordered allocations on
// its stream), small pinned host staging for the few device->host reads of
// sizes, and an optional per-kernel CUDA-event timing table.  Every step runs
// as kernels on one stream; the host synchronises only to learn data-dependent
// sizes (bin entries, blocks of the next level, adjacency and link counts).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
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

}  // namespace

struct amr_ctx {
  amr_domain dom{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  int num_sms = 0;
  std::string err;
  // state
  bool loaded = false, binned = false, refined = false;
  int64_t nf = 0, nv = 0;
  bool indexed = false;
  int B = 0;
  int64_t n_bins = 0, nnz = 0;
  bool count_clean = false;
  // buffers
  DevBuf X, nrm, stage_a, stage_b, frange, count, offsets, ids, payload, scratch, misc;
  DevBuf lv_blocks[AMR_MAX_LEVELS], lv_parent[AMR_MAX_LEVELS], lv_mask[AMR_MAX_LEVELS], lv_flag[AMR_MAX_LEVELS];
  DevBuf cellcnt, blockcnt, block_base, adj_cell, adj_off, adj_ids;
  DevBuf link_cell, link_dir, link_q, link_face;
  int64_t link_cap = 0;
  // adjoint: device copy of the index list, vertex -> corner and face -> link groupings
  DevBuf idx, vert_off, vert_corners, face_off, face_links, sort_keys, grad_face, sort_scratch, group_cnt;
  bool vert_groups = false, face_groups = false;
  int64_t n_links = 0;
  double finest_h = 0.0;
  const int32_t* finest_blocks = nullptr;
  // misc layout: [0..CNT_N) u64 counters, then u32 err word, u32 work, u64 totals[4]
  unsigned long long* counters = nullptr;
  unsigned* d_err = nullptr;
  unsigned* d_work = nullptr;
  uint64_t* d_tot = nullptr;
  void* h_pinned = nullptr;  // 256 bytes
  amr_refine_result last{};
  // timing
  bool timing = false;
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

amr_status ensure(amr_ctx* ctx, DevBuf& b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.cap >= bytes) return AMR_OK;
  if (b.p) {
    CK(cudaFreeAsync(b.p, ctx->stream));
    b.p = nullptr;
    b.cap = 0;
  }
  size_t want = bytes + bytes / 4 + 256;
  cudaError_t e = cudaMallocAsync(&b.p, want, ctx->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return fail(ctx, AMR_ENOMEM, "device allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
  }
  b.cap = want;
  return AMR_OK;
}

void release(amr_ctx* ctx, DevBuf& b) {
  if (b.p) cudaFreeAsync(b.p, ctx->stream);
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

// Times the launches issued inside fn() when timing is on.
template <typename F>
void timed(amr_ctx* c, const char* name, F fn) {
  if (!c->timing) {
    c->launches += fn();
    return;
  }
  TimedLaunch t{slot_of(c, name), take_event(c), take_event(c)};
  cudaEventRecord(t.a, c->stream);
  c->launches += fn();
  cudaEventRecord(t.b, c->stream);
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

amr_status sync_check(amr_ctx* ctx) {
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaGetLastError());
  harvest_timing(ctx);
  unsigned e = *reinterpret_cast<volatile unsigned*>(static_cast<char*>(ctx->h_pinned) + 128);
  (void)e;
  return AMR_OK;
}

// Copy the device error word and the requested totals to pinned memory and wait.
amr_status read_back(amr_ctx* ctx, unsigned* err_out, uint64_t* tot_out, int n_tot) {
  char* h = static_cast<char*>(ctx->h_pinned);
  CK(cudaMemcpyAsync(h, ctx->d_tot, sizeof(uint64_t) * 4, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(h + 64, ctx->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
  TRY(sync_check(ctx));
  if (tot_out)
    for (int i = 0; i < n_tot; ++i) tot_out[i] = reinterpret_cast<uint64_t*>(h)[i];
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

BinGrid make_grid(const amr_domain& d, int B) {
  BinGrid g{};
  g.B = B;
  for (int a = 0; a < 3; ++a) {
    g.origin[a] = d.origin[a];
    const double extent = (4.0 * (double)(a < d.dim ? d.root_blocks[a] : 1)) * d.h0;
    g.scale[a] = (double)B / extent;
  }
  return g;
}

}  // namespace

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
  amr_ctx* ctx = new amr_ctx();
  ctx->dom = *dom;
  for (int a = dom->dim; a < 3; ++a) ctx->dom.root_blocks[a] = 1;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e == cudaSuccess) {
    if (dom->stream) {
      ctx->stream = static_cast<cudaStream_t>(dom->stream);
    } else {
      e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
      ctx->own_stream = e == cudaSuccess;
    }
  }
  if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_pinned, 256);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return AMR_ECUDA;
  }
  if (ensure(ctx, ctx->misc, sizeof(unsigned long long) * CNT_N + 64 + 64) != AMR_OK) {
    cudaFreeHost(ctx->h_pinned);
    delete ctx;
    return AMR_ENOMEM;
  }
  char* m = static_cast<char*>(ctx->misc.p);
  ctx->counters = reinterpret_cast<unsigned long long*>(m);
  ctx->d_err = reinterpret_cast<unsigned*>(m + sizeof(unsigned long long) * CNT_N);
  ctx->d_work = ctx->d_err + 1;
  ctx->d_tot = reinterpret_cast<uint64_t*>(m + sizeof(unsigned long long) * CNT_N + 64);
  cudaMemsetAsync(ctx->misc.p, 0, ctx->misc.cap, ctx->stream);
  *out = ctx;
  return AMR_OK;
}

amr_status amr_destroy(amr_ctx* ctx) {
  if (!ctx) return AMR_OK;
  cudaStreamSynchronize(ctx->stream);
  DevBuf* extra[] = {&ctx->idx, &ctx->vert_off, &ctx->vert_corners, &ctx->face_off, &ctx->face_links,
                     &ctx->sort_keys, &ctx->grad_face, &ctx->sort_scratch, &ctx->group_cnt};
  for (DevBuf* b : extra) release(ctx, *b);
  DevBuf* all[] = {&ctx->X,        &ctx->nrm,       &ctx->stage_a,    &ctx->stage_b,  &ctx->frange,
                   &ctx->count,    &ctx->offsets,   &ctx->ids,        &ctx->payload,  &ctx->scratch,
                   &ctx->misc,     &ctx->cellcnt,   &ctx->blockcnt,   &ctx->block_base, &ctx->adj_cell,
                   &ctx->adj_off,  &ctx->adj_ids,   &ctx->link_cell,  &ctx->link_dir, &ctx->link_q,
                   &ctx->link_face};
  for (DevBuf* b : all) release(ctx, *b);
  for (int L = 0; L < AMR_MAX_LEVELS; ++L) {
    release(ctx, ctx->lv_blocks[L]);
    release(ctx, ctx->lv_parent[L]);
    release(ctx, ctx->lv_mask[L]);
    release(ctx, ctx->lv_flag[L]);
  }
  cudaStreamSynchronize(ctx->stream);
  for (auto& t : ctx->pending) {
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  for (auto e : ctx->event_pool) cudaEventDestroy(e);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
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
  TRY(read_back(ctx, &e, nullptr, 0));
  return device_error(ctx, e);
}

amr_status amr_geom_load(amr_ctx* ctx, const float* coords, int64_t n_verts, const int32_t* idx, int64_t n_faces) {
  if (!ctx) return AMR_EINVAL;
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
  if (n_faces > 0) {
    if (idx) {
      const void* dv = nullptr;
      const void* di = nullptr;
      TRY(to_device(ctx, coords, sizeof(float) * D * (size_t)n_verts, ctx->stage_a, &dv));
      TRY(to_device(ctx, idx, sizeof(int32_t) * D * (size_t)n_faces, ctx->stage_b, &di));
      TRY(ensure(ctx, ctx->idx, sizeof(int32_t) * D * (size_t)n_faces));
      CK(cudaMemcpyAsync(ctx->idx.p, di, sizeof(int32_t) * D * (size_t)n_faces, cudaMemcpyDeviceToDevice,
                         ctx->stream));
      timed(ctx, "load_gather", [&] {
        return launch_load_indexed(D, static_cast<const float*>(dv), n_verts, static_cast<const int32_t*>(di), n_faces,
                            static_cast<float*>(ctx->X.p), ctx->d_err, ctx->stream);
      });
    } else {
      const void* dc = nullptr;
      TRY(to_device(ctx, coords, sizeof(float) * D * D * (size_t)n_faces, ctx->stage_a, &dc));
      timed(ctx, "load_gather", [&] {
        return launch_load_facelist(D, static_cast<const float*>(dc), n_faces, static_cast<float*>(ctx->X.p), ctx->d_err,
                             ctx->stream);
      });
    }
    if (D == 3)
      timed(ctx, "face_normals", [&] {
        return launch_face_normals(static_cast<const float*>(ctx->X.p), n_faces, static_cast<float*>(ctx->nrm.p),
                            ctx->stream);
      });
  }
  CK(cudaGetLastError());
  ctx->loaded = true;
  return AMR_OK;
}

amr_status amr_bin_faces(amr_ctx* ctx, int B, amr_bins_view* out) {
  if (!ctx || !out) return AMR_EINVAL;
  if (!ctx->loaded) return fail(ctx, AMR_ESTATE, "amr_bin_faces before amr_geom_load");
  const int D = ctx->dom.dim;
  if (B < 1 || B > 65535) return fail(ctx, AMR_EINVAL, "bin density must be in [1, 65535]");
  int64_t nb = 1;
  for (int a = 0; a < D; ++a) nb *= B;
  if (nb > (1ll << 30)) return fail(ctx, AMR_EINVAL, "B^dim must not exceed 2^30");
  ctx->binned = ctx->refined = false;
  const int64_t nf = ctx->nf;
  if (ctx->count.cap < sizeof(uint32_t) * (size_t)nb) ctx->count_clean = false;
  TRY(ensure(ctx, ctx->count, sizeof(uint32_t) * (size_t)nb));
  if (!ctx->count_clean) {
    CK(cudaMemsetAsync(ctx->count.p, 0, ctx->count.cap, ctx->stream));
    ctx->count_clean = true;
  }
  TRY(ensure(ctx, ctx->offsets, sizeof(uint32_t) * (size_t)(nb + 1)));
  TRY(ensure(ctx, ctx->frange, sizeof(uint32_t) * 3 * (size_t)(nf > 0 ? nf : 1)));
  TRY(ensure(ctx, ctx->scratch, scan_u32_scratch_bytes(nb)));
  const BinGrid g = make_grid(ctx->dom, B);
  uint32_t* count = static_cast<uint32_t*>(ctx->count.p);
  uint32_t* offsets = static_cast<uint32_t*>(ctx->offsets.p);
  timed(ctx, "bin_count", [&] {
    return launch_face_bins(D, static_cast<const float*>(ctx->X.p), nf, g, static_cast<uint32_t*>(ctx->frange.p), count,
                     ctx->stream);
  });
  timed(ctx, "bin_scan", [&] {
    return launch_scan_u32(count, offsets, nb, ctx->d_tot, ctx->scratch.p, ctx->d_err, ctx->stream);
  });
  CK(cudaGetLastError());
  unsigned e = 0;
  uint64_t tot = 0;
  TRY(read_back(ctx, &e, &tot, 1));
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
  timed(ctx, "bin_scatter", [&] {
    return launch_scatter(D, static_cast<const float*>(ctx->X.p), nf, static_cast<const uint32_t*>(ctx->frange.p), offsets,
                   count, static_cast<uint32_t*>(ctx->ids.p), ctx->payload.p, B, ctx->stream);
  });
  CK(cudaGetLastError());
  ctx->B = B;
  ctx->n_bins = nb;
  ctx->nnz = (int64_t)tot;
  ctx->binned = true;
  out->B = B;
  out->n_bins = nb;
  out->nnz = (int64_t)tot;
  out->offsets = offsets;
  out->ids = static_cast<const uint32_t*>(ctx->ids.p);
  return AMR_OK;
}

amr_status amr_refine_near_wall(amr_ctx* ctx, const amr_refine_params* prm, amr_refine_result* out) {
  if (!ctx || !prm || !out) return AMR_EINVAL;
  if (!ctx->binned) return fail(ctx, AMR_ESTATE, "amr_refine_near_wall before amr_bin_faces");
  const int D = ctx->dom.dim;
  const int NL = prm->n_levels;
  if (NL < 1 || NL > AMR_MAX_LEVELS) return fail(ctx, AMR_EINVAL, "n_levels must be in [1, %d]", AMR_MAX_LEVELS);
  if (!(prm->d_abs >= 0.0) || !(prm->d_rel >= 0.0)) return fail(ctx, AMR_EINVAL, "negative near-wall distance");
  const bool links = prm->want_links != 0;
  const bool adjacency = prm->want_adjacency != 0 || links;
  if (links) {
    if (!((D == 2 && prm->lattice == 9) || (D == 3 && prm->lattice == 19)))
      return fail(ctx, AMR_EINVAL, "lattice must be 9 (D2Q9) in 2D or 19 (D3Q19) in 3D");
    const double hf = ctx->dom.h0 * std::ldexp(1.0, -(NL - 1));
    if (prm->d_abs + prm->d_rel * hf < 0.5 * hf)
      return fail(ctx, AMR_EINVAL, "links need d_L >= h_L/2 on the finest level");
  }
  ctx->refined = false;
  ctx->face_groups = false;
  ctx->n_links = 0;
  amr_refine_result r{};
  r.n_levels = NL;
  CK(cudaMemsetAsync(ctx->counters, 0, sizeof(unsigned long long) * CNT_N, ctx->stream));
  int64_t N = 1;
  for (int a = 0; a < D; ++a) N *= ctx->dom.root_blocks[a];
  if (N > (1ll << 31)) return fail(ctx, AMR_EINVAL, "too many root blocks");
  TRY(ensure(ctx, ctx->lv_blocks[0], sizeof(int32_t) * D * (size_t)N));
  timed(ctx, "root_blocks", [&] {
    return launch_root_blocks(D, ctx->dom.root_blocks, static_cast<int32_t*>(ctx->lv_blocks[0].p), N, ctx->stream);
  });
  const int NCell = D == 3 ? 64 : 16;
  RefineLevel lv{};
  for (int L = 0; L < NL; ++L) {
    const bool finest = L == NL - 1;
    const double h = ctx->dom.h0 * std::ldexp(1.0, -L);
    const double d = prm->d_abs + prm->d_rel * h;
    r.n_blocks[L] = N;
    TRY(ensure(ctx, ctx->lv_mask[L], sizeof(uint64_t) * (size_t)N));
    TRY(ensure(ctx, ctx->lv_flag[L], (size_t)N));
    lv = RefineLevel{};
    lv.dim = D;
    lv.blocks = static_cast<const int32_t*>(ctx->lv_blocks[L].p);
    lv.n_blocks = N;
    lv.offsets = static_cast<const uint32_t*>(ctx->offsets.p);
    lv.payload = ctx->payload.p;
    lv.X = static_cast<const float*>(ctx->X.p);
    lv.nrm = static_cast<const float*>(ctx->nrm.p);
    lv.nf = ctx->nf;
    lv.grid = make_grid(ctx->dom, ctx->B);
    for (int a = 0; a < 3; ++a) lv.origin[a] = ctx->dom.origin[a];
    lv.h = h;
    lv.d = d;
    lv.mask = static_cast<uint64_t*>(ctx->lv_mask[L].p);
    lv.flag = static_cast<uint8_t*>(ctx->lv_flag[L].p);
    lv.counters = ctx->counters;
    lv.work = ctx->d_work;
    lv.err = ctx->d_err;
    if (finest && adjacency) {
      TRY(ensure(ctx, ctx->cellcnt, sizeof(uint16_t) * NCell * (size_t)N));
      TRY(ensure(ctx, ctx->blockcnt, sizeof(uint64_t) * (size_t)N));
      lv.cellcnt = static_cast<uint16_t*>(ctx->cellcnt.p);
      lv.blockcnt = static_cast<uint64_t*>(ctx->blockcnt.p);
    }
    CK(cudaMemsetAsync(ctx->d_work, 0, sizeof(unsigned), ctx->stream));
    timed(ctx, "refine_level", [&] { return launch_refine(lv, ctx->num_sms, ctx->stream); });
    r.block_coords[L] = static_cast<const int32_t*>(ctx->lv_blocks[L].p);
    r.block_parent[L] = L > 0 ? static_cast<const int32_t*>(ctx->lv_parent[L].p) : nullptr;
    r.cell_mask[L] = lv.mask;
    r.block_flag[L] = lv.flag;
    if (!finest) {
      // children of the marked blocks -> next level (worst case 2^D per block)
      TRY(ensure(ctx, ctx->scratch, children_scratch_bytes(N)));
      const int64_t cap = N * (D == 3 ? 8 : 4);
      TRY(ensure(ctx, ctx->lv_blocks[L + 1], sizeof(int32_t) * D * (size_t)(cap > 0 ? cap : 1)));
      TRY(ensure(ctx, ctx->lv_parent[L + 1], sizeof(int32_t) * (size_t)(cap > 0 ? cap : 1)));
      timed(ctx, "children", [&] {
        return launch_children(D, lv.blocks, lv.mask, N, static_cast<int32_t*>(ctx->lv_blocks[L + 1].p),
                        static_cast<int32_t*>(ctx->lv_parent[L + 1].p), ctx->d_tot, ctx->scratch.p, ctx->d_err,
                        ctx->stream);
      });
      CK(cudaGetLastError());
      unsigned e = 0;
      uint64_t tot = 0;
      TRY(read_back(ctx, &e, &tot, 1));
      TRY(device_error(ctx, e));
      N = (int64_t)tot;
      if (N > (1ll << 32) / NCell) return fail(ctx, AMR_EOVERFLOW, "level %d has too many blocks", L + 1);
    }
  }
  // finest level: adjacent-face lists
  if (adjacency) {
    const int64_t Nf = N;
    TRY(ensure(ctx, ctx->block_base, sizeof(uint64_t) * (size_t)(Nf > 0 ? Nf : 1)));
    TRY(ensure(ctx, ctx->scratch, scan_u64_scratch_bytes(Nf)));
    timed(ctx, "adj_scan", [&] {
      return launch_scan_u64(static_cast<const uint64_t*>(ctx->blockcnt.p), static_cast<uint64_t*>(ctx->block_base.p), Nf,
                      ctx->d_tot, ctx->scratch.p, ctx->d_err, ctx->stream);
    });
    CK(cudaGetLastError());
    unsigned e = 0;
    uint64_t tot = 0;
    TRY(read_back(ctx, &e, &tot, 1));
    TRY(device_error(ctx, e));
    const uint64_t pairs = tot & 0xffffffffull, cells = tot >> 32;
    if (Nf > 0 && (pairs >= 0xffffffffull)) return fail(ctx, AMR_EOVERFLOW, "too many adjacent (cell, face) pairs");
    TRY(ensure(ctx, ctx->adj_cell, sizeof(uint32_t) * (size_t)(cells + 1)));
    TRY(ensure(ctx, ctx->adj_off, sizeof(uint32_t) * (size_t)(cells + 1)));
    TRY(ensure(ctx, ctx->adj_ids, sizeof(uint32_t) * (size_t)(pairs + 1)));
    EmitArgs ea{};
    ea.lv = lv;
    ea.block_base = static_cast<const uint64_t*>(ctx->block_base.p);
    ea.adj_cell = static_cast<uint32_t*>(ctx->adj_cell.p);
    ea.adj_off = static_cast<uint32_t*>(ctx->adj_off.p);
    ea.adj_ids = static_cast<uint32_t*>(ctx->adj_ids.p);
    uint32_t* hp = reinterpret_cast<uint32_t*>(static_cast<char*>(ctx->h_pinned) + 192);
    *hp = (uint32_t)pairs;
    CK(cudaMemcpyAsync(static_cast<uint32_t*>(ctx->adj_off.p) + cells, hp, sizeof(uint32_t), cudaMemcpyHostToDevice,
                       ctx->stream));
    CK(cudaMemsetAsync(ctx->d_work, 0, sizeof(unsigned), ctx->stream));
    timed(ctx, "adjacency", [&] { return launch_adjacency(ea, ctx->num_sms, ctx->stream); });
    CK(cudaGetLastError());
    r.n_adj_cells = (int64_t)cells;
    r.n_adj_pairs = (int64_t)pairs;
    r.adj_cell = ea.adj_cell;
    r.adj_off = ea.adj_off;
    r.adj_ids = ea.adj_ids;
    if (links) {
      LinkArgs la{};
      la.dim = D;
      la.lattice = prm->lattice;
      la.blocks = lv.blocks;
      la.adj_cell = ea.adj_cell;
      la.adj_off = ea.adj_off;
      la.adj_ids = ea.adj_ids;
      la.n_adj = (int64_t)cells;
      la.X = static_cast<const float*>(ctx->X.p);
      la.nrm = static_cast<const float*>(ctx->nrm.p);
      la.nf = ctx->nf;
      for (int a = 0; a < 3; ++a) la.origin[a] = ctx->dom.origin[a];
      la.h = ctx->dom.h0 * std::ldexp(1.0, -(NL - 1));
      la.n_links = ctx->d_tot;
      la.counters = ctx->counters;
      la.err = ctx->d_err;
      int64_t want = ctx->link_cap;
      if (want < (int64_t)cells * 4) want = (int64_t)cells * 4;
      for (int attempt = 0; attempt < 2; ++attempt) {
        TRY(ensure(ctx, ctx->link_cell, sizeof(uint32_t) * (size_t)(want + 1)));
        TRY(ensure(ctx, ctx->link_dir, (size_t)(want + 1)));
        TRY(ensure(ctx, ctx->link_q, sizeof(float) * (size_t)(want + 1)));
        TRY(ensure(ctx, ctx->link_face, sizeof(uint32_t) * (size_t)(want + 1)));
        ctx->link_cap = want;
        la.link_cell = static_cast<uint32_t*>(ctx->link_cell.p);
        la.link_dir = static_cast<uint8_t*>(ctx->link_dir.p);
        la.link_q = static_cast<float*>(ctx->link_q.p);
        la.link_face = static_cast<uint32_t*>(ctx->link_face.p);
        la.link_cap = want;
        TRY(ensure(ctx, ctx->scratch, links_scratch_bytes(la.n_adj)));
        timed(ctx, "links", [&] { return launch_links(la, ctx->scratch.p, ctx->stream); });
        CK(cudaGetLastError());
        uint64_t nl = 0;
        TRY(read_back(ctx, &e, &nl, 1));
        TRY(device_error(ctx, e));
        if ((int64_t)nl <= want) {
          r.n_links = (int64_t)nl;
          break;
        }
        want = (int64_t)nl;  // capacity too small: grow to the exact count and run again
      }
      r.link_cell = la.link_cell;
      r.link_dir = la.link_dir;
      r.link_q = la.link_q;
      r.link_face = la.link_face;
    }
  }
  // counters and the final error check
  char* h = static_cast<char*>(ctx->h_pinned);
  CK(cudaMemcpyAsync(h, ctx->counters, sizeof(unsigned long long) * CNT_N, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(h + 128, ctx->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
  TRY(sync_check(ctx));
  const unsigned long long* cnt = reinterpret_cast<const unsigned long long*>(h);
  r.n_fallback = (int64_t)(cnt[CNT_FALLBACK] + cnt[CNT_LINK_FALLBACK]);
  r.n_band = (int64_t)(cnt[CNT_BAND] + cnt[CNT_LINK_BAND]);
  r.n_candidates = (int64_t)cnt[CNT_CANDIDATES];
  r.n_survivors = (int64_t)cnt[CNT_SURVIVORS];
  TRY(device_error(ctx, *reinterpret_cast<unsigned*>(h + 128)));
  ctx->refined = true;
  ctx->last = r;
  ctx->n_links = links ? r.n_links : -1;
  ctx->finest_h = ctx->dom.h0 * std::ldexp(1.0, -(NL - 1));
  ctx->finest_blocks = r.block_coords[NL - 1];
  *out = r;
  return AMR_OK;
}

namespace {

int key_bits(int64_t n) {
  int b = 1;
  while (b < 32 && ((int64_t)1 << b) < n) ++b;
  return b;
}

// Stable grouping of `n` keys in [0, n_keys): CSR offsets [n_keys + 1] and the
// values (default 0..n-1) in ascending order within each key.
amr_status group_by_key(amr_ctx* ctx, const uint32_t* keys, int64_t n, int64_t n_keys, const uint32_t* vals,
                        DevBuf& off, DevBuf& grouped, const char* name) {
  TRY(ensure(ctx, off, sizeof(uint32_t) * (size_t)(n_keys + 1)));
  TRY(ensure(ctx, grouped, sizeof(uint32_t) * (size_t)(n > 0 ? n : 1)));
  TRY(ensure(ctx, ctx->sort_keys, sizeof(uint32_t) * (size_t)(n > 0 ? n : 1)));
  TRY(ensure(ctx, ctx->sort_scratch, radix_sort_scratch_bytes(n)));
  TRY(ensure(ctx, ctx->scratch, scan_u32_scratch_bytes(n_keys)));
  TRY(ensure(ctx, ctx->group_cnt, sizeof(uint32_t) * (size_t)(n_keys > 0 ? n_keys : 1)));
  CK(cudaMemsetAsync(ctx->group_cnt.p, 0, sizeof(uint32_t) * (size_t)(n_keys > 0 ? n_keys : 1), ctx->stream));
  timed(ctx, name, [&] {
    int k = launch_count_keys(keys, n, static_cast<uint32_t*>(ctx->group_cnt.p), ctx->stream);
    k += launch_scan_u32(static_cast<const uint32_t*>(ctx->group_cnt.p), static_cast<uint32_t*>(off.p), n_keys,
                         ctx->d_tot, ctx->scratch.p, ctx->d_err, ctx->stream);
    k += launch_stable_sort(keys, n, key_bits(n_keys), static_cast<uint32_t*>(ctx->sort_keys.p),
                            static_cast<uint32_t*>(grouped.p), vals, ctx->sort_scratch.p, ctx->d_tot, ctx->d_err,
                            ctx->stream);
    return k;
  });
  CK(cudaGetLastError());
  return AMR_OK;
}

}  // namespace

extern "C" {

amr_status amr_q_backward(amr_ctx* ctx, const float* grad_q, float* grad_out) {
  if (!ctx) return AMR_EINVAL;
  if (!ctx->refined || ctx->n_links < 0)
    return fail(ctx, AMR_ESTATE, "amr_q_backward needs a preceding amr_refine_near_wall with links");
  const int D = ctx->dom.dim;
  const int64_t nl = ctx->n_links, nf = ctx->nf;
  if (!grad_out || (nl > 0 && !grad_q)) return fail(ctx, AMR_EINVAL, "null gradient pointer");
  if ((nl > 0 && !is_device_ptr(grad_q)) || !is_device_ptr(grad_out))
    return fail(ctx, AMR_EINVAL, "gradients must be device pointers");
  if (!ctx->face_groups) {
    TRY(group_by_key(ctx, static_cast<const uint32_t*>(ctx->link_face.p), nl, nf, nullptr, ctx->face_off,
                     ctx->face_links, "adjoint_group_links"));
    ctx->face_groups = true;
  }
  const bool indexed = ctx->indexed;
  if (indexed && !ctx->vert_groups) {
    TRY(group_by_key(ctx, static_cast<const uint32_t*>(ctx->idx.p), nf * D, ctx->nv, nullptr, ctx->vert_off,
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
  a.X = static_cast<const float*>(ctx->X.p);
  a.nrm = static_cast<const float*>(ctx->nrm.p);
  a.face_off = static_cast<const uint32_t*>(ctx->face_off.p);
  a.face_links = static_cast<const uint32_t*>(ctx->face_links.p);
  a.grad_q = grad_q;
  a.link_cell = static_cast<const uint32_t*>(ctx->link_cell.p);
  a.link_dir = static_cast<const uint8_t*>(ctx->link_dir.p);
  a.link_q = static_cast<const float*>(ctx->link_q.p);
  a.adj_cell = static_cast<const uint32_t*>(ctx->adj_cell.p);
  a.blocks = ctx->finest_blocks;
  for (int c = 0; c < 3; ++c) a.origin[c] = ctx->dom.origin[c];
  a.h = ctx->finest_h;
  a.grad_face = gface;
  timed(ctx, "adjoint_face", [&] { return launch_face_grad(a, ctx->stream); });
  if (indexed)
    timed(ctx, "adjoint_vertex", [&] {
      return launch_vertex_grad(D, gface, static_cast<const uint32_t*>(ctx->vert_off.p),
                                static_cast<const uint32_t*>(ctx->vert_corners.p), ctx->nv, grad_out, ctx->stream);
    });
  CK(cudaGetLastError());
  return AMR_OK;
}

}  // extern "C"

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
