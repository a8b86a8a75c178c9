/* amrgeom.h — C ABI of the GB300 geometry-to-AMR near-wall refinement library.
 *
 * The library implements the data-parallel hot path of the geometry module in
 * Jaber, Essel & Sullivan, "Towards a GPU-native adaptive mesh refinement scheme
 * for the Lattice Boltzmann Method in complex geometries" (2025), whose
 * procedure has three steps (Abstract; Sec. "Methodology"):
 *   1. import the faces (edges in 2D, triangles in 3D) as an index list or a
 *      face-vertex coordinate list            -> amr_geom_load
 *   2. spatially bin the faces into B^D bins   -> amr_bin_faces
 *   3. near-wall refinement of a forest of octrees (blocks of 4^D cells): every
 *      cell detects adjacency to the faces of the bins around it, marked blocks
 *      are split, and the finest cells list their faces and form wall links
 *      along the lattice directions         -> amr_refine_near_wall
 * plus the vertex adjoint of the link fractions q (amr_q_backward).
 *
 * Conventions
 *   - Domain box: origin[a] + [0, 4*root_blocks[a]*h0] per axis.  Level-L cell
 *     size h_L = h0 * 2^-L.  Block (b0,b1,b2) of level L holds cells 4b..4b+3.
 *   - Cell bit within a block: i + 4j (+ 16k), x fastest.  Level-0 blocks in
 *     x-fastest lexicographic order; the children of the marked blocks of level
 *     L follow in parent order, child slot s = bx + 2by (+ 4bz).
 *   - Adjacency (Sec. "Face Detection", box form): a cell is adjacent to a face
 *     when its box inflated by d_L = d_abs + d_rel*h_L meets the closed face.
 *   - Bins (Sec. "Spatial Binning Algorithm"): a face is stored in every bin its
 *     axis-aligned bounding box overlaps (bins half-open, outer bins unbounded).
 *   - Lattice directions: D2Q9 1..8 = (1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),
 *     (-1,-1),(1,-1); D3Q19 1..6 = +x,-x,+y,-y,+z,-z, 7..18 = xy, xz, yz plane
 *     diagonals, each (+,+),(-,-),(+,-),(-,+).
 *
 * Ownership and threading
 *   - The caller owns every input it passes; inputs are copied before the call
 *     returns its status.  Pointers may be host or device memory (detected).
 *   - Output views are BORROWED device pointers owned by the context, valid
 *     until the next call of the same step or amr_destroy.
 *   - All work is ordered on the context's stream.  A context is not
 *     thread-safe; use one context per host thread.
 *   - Every call returns a status and never aborts.  A failed device-side check
 *     (bad index, non-finite coordinate, a bounded wait that ran out) is reported
 *     by the call that synchronises after it.
 */
#ifndef AMRGEOM_H
#define AMRGEOM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AMR_MAX_LEVELS 16

#if defined(__GNUC__)
#define AMR_API __attribute__((visibility("default")))
#else
#define AMR_API
#endif

typedef struct amr_ctx amr_ctx;

typedef enum {
  AMR_OK = 0,
  AMR_EINVAL = 1,        /* invalid argument or input data */
  AMR_ENOMEM = 2,        /* device or host allocation failed */
  AMR_ECUDA = 3,         /* a CUDA runtime call failed (see amr_last_error) */
  AMR_EOVERFLOW = 4,     /* a size exceeded its representable range (e.g. > 2^32 bin entries) */
  AMR_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
  AMR_ESTATE = 6,        /* calls out of order (load -> bin -> refine -> backward) */
  AMR_EDEVICE_CHECK = 7  /* a device-side input check failed */
} amr_status;

typedef struct {
  int dim;               /* 2 or 3 */
  int root_blocks[3];    /* root blocks per axis (entries beyond dim ignored), each >= 1 */
  double origin[3];      /* domain origin */
  double h0;             /* level-0 cell size, > 0 */
  void* stream;          /* cudaStream_t to order all work on; NULL = a stream the context creates */
  /* Optional device allocator (give both or neither; NULL = cudaMallocAsync /
   * cudaFreeAsync on the context's stream).  Every device buffer the context owns
   * is taken from dev_alloc(bytes, user), which returns device memory of the
   * current device usable on the context's stream (NULL = out of memory: the
   * call fails with ENOMEM), and is handed back with dev_free(ptr, user) once the
   * context's stream has finished every use of it (the library synchronises the
   * stream first).  Both are called on the host thread that calls the library;
   * buffers grow only in eager calls, never while a graph is replayed.  Pinned
   * host staging (a few KB) is not taken from it.  amr_bin_faces_static ignores
   * these fields. */
  void* (*dev_alloc)(size_t bytes, void* user);
  void (*dev_free)(void* ptr, void* user);
  void* user;
} amr_domain;

/* Create a context on the current CUDA device.  *out receives the handle.
 * EINVAL: bad dim / root_blocks / h0.  ECUDA: no usable device. */
AMR_API amr_status amr_create(const amr_domain* dom, amr_ctx** out);

/* Free every device and host buffer of the context.  NULL is accepted. */
AMR_API amr_status amr_destroy(amr_ctx* ctx);

/* Static description of a status code. */
AMR_API const char* amr_status_str(amr_status s);

/* Detail text of the last error raised on this context ("" if none). */
AMR_API const char* amr_last_error(const amr_ctx* ctx);

/* Replace the stream all later work is ordered on (NULL = the context's own). */
AMR_API amr_status amr_set_stream(amr_ctx* ctx, void* stream);

/* Step 1 — import (Sec. "Representation of the Complex Boundary Geometry").
 * idx == NULL: `coords` is a face-vertex list f32[n_faces][dim][dim].
 * idx != NULL: `coords` = vertices f32[n_verts][dim], idx = i32[n_faces][dim].
 * The faces are gathered into a resident structure-of-arrays copy on the device
 * (the paper's geom_f_face_X) together with per-face double-float normals.
 * 0 <= n_faces < 2^29.  EINVAL: bad sizes, null pointers; EDEVICE_CHECK: an index
 * out of [0, n_verts) or a non-finite coordinate (detected on the device). */
AMR_API amr_status amr_geom_load(amr_ctx* ctx, const float* coords, int64_t n_verts, const int32_t* idx,
                         int64_t n_faces);

/* Step 2 — binning (Sec. "Spatial Binning Algorithm": binned_face_ids_N,
 * binned_face_ids).  B = bin_density bins per axis over the domain box, B >= 1
 * (B = 1 is the paper's naive scheme), B^dim <= 2^30.  Bin b = bx + B*by (+ B^2*bz).
 * offsets[b]..offsets[b+1] index the face ids of bin b in `ids`; the order
 * within a bin is unspecified (atomic scatter).  EOVERFLOW: more than 2^32 - 1
 * (face, bin) entries.
 * payload: one entry per (face, bin) entry, in the order of `ids` (entry k
 * belongs to ids[k]), so that a bin's faces with their coordinates are one
 * contiguous run of memory; payload_bytes per entry, 16-byte aligned:
 *   3D (64 B): f32 v[9] (vertex-major coordinates), f32 n[3] (the normal
 *              (v1-v0)x(v2-v0) formed in FP64, rounded to FP32), u32 id, u32 bin[3];
 *   2D (32 B): f32 v[4], u32 id, u32 bin[3] (bin[2] = 0);
 * id = face id in bits 0..28, bit 29 / 30 / 31 set when this bin is the first
 * of the face's bin range along x / y / z; bin = this entry's bin coordinates. */
typedef struct {
  int B;
  int64_t n_bins;             /* B^dim */
  int64_t nnz;                /* total (face, bin) entries */
  const uint32_t* offsets;    /* device [n_bins + 1] */
  const uint32_t* ids;        /* device [nnz] */
  const void* payload;        /* device [nnz] entries of payload_bytes (see above) */
  int64_t payload_bytes;      /* 64 (3D) or 32 (2D) */
} amr_bins_view;
AMR_API amr_status amr_bin_faces(amr_ctx* ctx, int bin_density, amr_bins_view* out);

/* Step 2, the paper's own membership (Sec. "Spatial Binning Algorithm", Fig.
 * "Discretization of edges and triangles"): each face is discretised into points
 * (its first edge into n + 1 points, n = ceil(length / s); in 3D every segment
 * from such a point to the opposite vertex likewise; s = half a bin length) and
 * belongs to every bin that holds one of them.  A subset of amr_bin_faces' bins;
 * meant for the paper's binned search (amr_refine_params.search =
 * AMR_SEARCH_OWN_BIN), which requires it or exact bins.  Same view and errors as
 * amr_bin_faces; single-geometry contexts only. */
AMR_API amr_status amr_bin_faces_sampled(amr_ctx* ctx, int bin_density, amr_bins_view* out);

/* Step 3 — near-wall refinement (Sec. "Cell-Face Identification Algorithms").
 * n_levels total levels (n_levels - 1 refinement passes), 1 <= n_levels <= AMR_MAX_LEVELS.
 * lattice: 0 (no links), 9 (D2Q9, dim 2) or 19 (D3Q19, dim 3).
 * predicate: when a cell is adjacent to a face (Sec. "Face Detection"):
 *   AMR_PRED_BOX   (0, default) the cell box inflated by d_L meets the closed face
 *                  (separating-axis test);
 *   AMR_PRED_POINT (1) the cell centre lies within distance d_L of the closed face
 *                  (the paper's Alg. 1: spheres, cylinders and prism of radius d_spec;
 *                  the paper's absolute d_spec is d_abs with d_rel = 0).
 * want_links requires want_adjacency and, on the finest level, d_L >= h_L/2 (box)
 * or d_L >= sqrt(2) h_L (point), so that every face a link crosses is in the
 * cell's adjacency list; otherwise AMR_EINVAL.
 * Eager calls read back each level's size; graph calls read back once at the end
 * and re-run eagerly (transparently) if a size outgrew the captured capacities. */
typedef struct {
  int n_levels;
  double d_abs;               /* near-wall distance d_L = d_abs + d_rel * h_L, >= 0 */
  double d_rel;
  int lattice;
  int want_adjacency;
  int want_links;
  int use_graph;              /* 1: replay the level loop as one captured CUDA graph when the inputs match
                                 the previous call (the first call runs eagerly and captures) */
  int warps_per_cta;          /* warps per thread block of the refine kernels, 0 = default (4), max 8 */
  int predicate;              /* AMR_PRED_BOX (0) or AMR_PRED_POINT (1) */
  int search;                 /* AMR_SEARCH_QUERY_BOX (0): every bin the cell's test region overlaps (exact
                                 for any bin density); AMR_SEARCH_OWN_BIN (1): only the bin holding the cell
                                 centre, the paper's binned face detection (needs AMR_PRED_POINT, no links) */
  int propagate;              /* refinement-mark propagation rounds after each level that is refined further
                                 (Sec. "Spatial Binning Algorithm"): 0 none, -1 the paper's
                                 1 + floor(d_L / block length), k > 0 exactly k; each round marks the existing
                                 neighbour blocks (3^D - 1) of every marked block; single-geometry only */
  int keep_previous;          /* 1: keep the previous call's block lists for amr_adapt_diff (re-adaptation of
                                 a moving or changing geometry); single-geometry only */
  int face_pass;              /* levels whose only output is the mask (every level above the finest, and the
                                 finest without adjacency): AMR_FACE_PASS_AUTO (0) marks them face by face where
                                 that is expected to be cheaper than the block walk, _OFF (1) never, _ON (2)
                                 wherever it applies (single geometry, AMR_SEARCH_QUERY_BOX, block coordinates
                                 below 2^21).  Results are identical either way. */
} amr_refine_params;
enum { AMR_PRED_BOX = 0, AMR_PRED_POINT = 1 };
enum { AMR_SEARCH_QUERY_BOX = 0, AMR_SEARCH_OWN_BIN = 1 };
enum { AMR_FACE_PASS_AUTO = 0, AMR_FACE_PASS_OFF = 1, AMR_FACE_PASS_ON = 2 };

/* Results.  Level arrays are per level 0..n_levels-1.
 *   block_coords[L]  device i32 [N_L][dim]
 *   block_parent[L]  device i32 [N_L], index of the parent in level L-1 (NULL for L = 0)
 *   cell_mask[L]     device u64 [N_L], adjacency bit per cell (low 16 bits in 2D)
 *   block_flag[L]    device u8  [N_L], 1 when the block is marked (mask != 0)
 * Finest level (when want_adjacency):
 *   adj_cell   device u32 [n_adj_cells]: block index * 4^dim + cell bit, ascending
 *   adj_off    device u32 [n_adj_cells + 1]: CSR offsets into adj_ids
 *   adj_ids    device u32 [n_adj_pairs]: adjacent face ids, ascending per cell
 * Links (when want_links), sorted by (cell, direction):
 *   link_cell  device u32 [n_links]: row of the adjacent cell in adj_cell
 *   link_dir   device u8  [n_links]: lattice direction 1..Q-1
 *   link_q     device f32 [n_links]: smallest t in [0,1] with centre + t*c_i*h on a face
 *   link_face  device u32 [n_links]: the face hit at q (smallest id on ties)
 * Diagnostics: n_fallback = close decisions re-evaluated in FP64; n_band = those
 * whose FP64 margin was within 1e-6*h (adjacency) or 1e-6 (links) of the boundary. */
typedef struct {
  int n_levels;
  int64_t n_blocks[AMR_MAX_LEVELS];
  const int32_t* block_coords[AMR_MAX_LEVELS];
  const int32_t* block_parent[AMR_MAX_LEVELS];
  const uint64_t* cell_mask[AMR_MAX_LEVELS];
  const uint8_t* block_flag[AMR_MAX_LEVELS];
  int64_t n_adj_cells;
  int64_t n_adj_pairs;
  const uint32_t* adj_cell;
  const uint32_t* adj_off;
  const uint32_t* adj_ids;
  int64_t n_links;
  const uint32_t* link_cell;
  const uint8_t* link_dir;
  const float* link_q;
  const uint32_t* link_face;
  int64_t n_fallback;
  int64_t n_band;
  int64_t n_candidates;       /* (block, face) candidate pairs read from the bins, all levels */
  int64_t n_survivors;        /* candidates that passed the block-level test */
  int64_t n_link_candidates;  /* (cell, face, direction) triples that passed the plane-range filter */
  int64_t n_face_setups;      /* faces set up by the face-by-face marking (face_pass), all its levels */
  int64_t n_face_tests;       /* (face, cell) tests it ran */
  int graph_replay;           /* 1: the level loop ran as a replay of the captured graph; 0: eagerly (first
                                 call, changed inputs or layout, or sizes beyond the graph's capacities) */
} amr_refine_result;
AMR_API amr_status amr_refine_near_wall(amr_ctx* ctx, const amr_refine_params* params, amr_refine_result* out);

/* Vertex adjoint of the link fractions q (not part of the paper: it lets a
 * training loop differentiate a loss of q with respect to the geometry).
 * grad_q: DEVICE f32 [n_links] aligned with the link arrays of the last
 * amr_refine_near_wall (which must have formed links).  grad_out: DEVICE f32,
 * overwritten: [n_verts][dim] when the geometry was loaded as an index list,
 * else [n_faces][dim][dim].  Gradients flow through q of the hit face only
 * (dt/dv of the plane / line through that face); flags, masks and adjacency are
 * not differentiated.  Deterministic: links are grouped by face with a stable
 * radix sort and summed in ascending link order, face corners by vertex in
 * ascending (face, corner) order, without float atomics, so repeated calls give
 * bitwise identical results.  ESTATE without links; EINVAL for host pointers. */
AMR_API amr_status amr_q_backward(amr_ctx* ctx, const float* grad_q, float* grad_out);

/* Node classification (not in the paper's method: the next step it names towards
 * the LBM boundary conditions).  After amr_refine_near_wall with adjacency on an
 * exactly binned single-geometry context: for every adjacent cell of the finest
 * level (row i of adj_cell), *cell_solid[i] = 1 when its centre lies inside the
 * closed boundary mesh, else 0 (fluid).  Decided by the parity of the faces a ray
 * from the centre along +x crosses (each face once; FP32 box cull, FP64 crossing
 * test); a ray through an edge or vertex, or a centre on a face, falls back to the
 * generalized winding number of the whole mesh (|w| > 1/2 = solid), counted in
 * *n_fallback (nullable).  The mesh must be closed (either orientation).
 * cell_solid: BORROWED device u8 [n_adj_cells], valid until the next refinement.
 * Errors: ESTATE (no refinement with adjacency, batch context), EINVAL (sampled bins). */
AMR_API amr_status amr_classify_nodes(amr_ctx* ctx, const uint8_t** cell_solid, int64_t* n_fallback);

/* Restricts the wall links of the last refinement to fluid cells (after
 * amr_classify_nodes): a stable compaction of link_cell / link_dir / link_q /
 * link_face in place; *out is the updated result (n_links and the same borrowed
 * arrays).  The q adjoint then applies to the kept links.  Errors: ESTATE. */
AMR_API amr_status amr_fluid_links(amr_ctx* ctx, amr_refine_result* out);

/* Re-adaptation bookkeeping (not in the paper's method: its dynamic re-adaptation
 * and coarsening are future work).  After two successive amr_refine_near_wall
 * calls on one context, the second with keep_previous = 1, per level L:
 *   new_to_old[L][i] = index of the new block i in the previous call's level-L
 *                      list, -1 when it did not exist (a block created by refinement);
 *   old_to_new[L][j] = index of the previous block j in the new list, -1 when it
 *                      is gone (a block removed by coarsening);
 * with the counts.  Levels beyond either hierarchy's depth map to -1.  All
 * device arrays are BORROWED until the next refinement.  Errors: ESTATE (no
 * kept previous hierarchy). */
typedef struct {
  int n_levels;                            /* levels of the new hierarchy */
  int64_t n_new[AMR_MAX_LEVELS], n_old[AMR_MAX_LEVELS];
  int64_t n_created[AMR_MAX_LEVELS], n_removed[AMR_MAX_LEVELS];
  const int32_t* new_to_old[AMR_MAX_LEVELS];  /* device [n_new[L]] */
  const int32_t* old_to_new[AMR_MAX_LEVELS];  /* device [n_old[L]] */
} amr_adapt_diff;
AMR_API amr_status amr_adapt_diff_get(amr_ctx* ctx, amr_adapt_diff* out);

/* Algorithmic cell-face test count of the last refinement (a measurement; Sec. "Spatial Binning
 * Algorithm": every cell checks the faces of the bins around it).  Per level L, per_level[L] =
 * sum over the cells of its blocks of the number of distinct faces stored in the bins that the
 * cell's inflated box (centre +- (h_L / 2 + d_L)) overlaps; the bin range is formed in FP64, so
 * the count is exact and fixed by the geometry and the bin density, whatever the kernels execute.
 * per_level: host array of AMR_MAX_LEVELS (levels past n_levels get 0); total: nullable host.
 * Single-geometry contexts after amr_refine_near_wall (else AMR_ESTATE). */
AMR_API amr_status amr_candidate_count(amr_ctx* ctx, int64_t* per_level, int64_t* total);

/* Wait for all work of the context; report device-side check failures. */
AMR_API amr_status amr_sync(amr_ctx* ctx);

/* Per-kernel timing with CUDA events on the context stream (off by default).
 * amr_timing_get fills up to `cap` entries in launch-table order and returns
 * how many kernels have been timed; names are static strings. */
AMR_API amr_status amr_timing_enable(amr_ctx* ctx, int on);
AMR_API amr_status amr_timing_reset(amr_ctx* ctx);
AMR_API int amr_timing_get(amr_ctx* ctx, const char** names, double* total_ms, int64_t* launches, int cap);

/* Autotuner (not in the paper; it automates the paper's bin-density study,
 * where bin setup grows and face detection shrinks with B).  On the loaded
 * geometry, times bin + refine (with the caller's adjacency / link options,
 * eager mode, best of two runs, CUDA events) for each candidate bin density,
 * then each candidate warps-per-block for the best density.  Candidates NULL =
 * defaults (B in 4..256 with B^dim <= 2^24; warps 2, 4, 8).  Leaves the context
 * binned with the last candidate: bin again with *best_B before refining. */
AMR_API amr_status amr_autotune(amr_ctx* ctx, const amr_refine_params* params, const int* b_candidates, int n_b,
                                const int* w_candidates, int n_w, int* best_B, int* best_warps, double* best_ms);

/* Batched mode (not in the paper): many geometries of uneven size and depth
 * refined together.  Per level, one refine launch and one child compaction
 * cover every geometry still refining; geometries that end on a level form
 * their adjacency lists and links there.  With use_graph the whole level loop
 * is one CUDA graph replay.  Results are concatenations with batch-global
 * indices; amr_batch_get_view gives one geometry's segments and the bases to
 * subtract from its indices. */
typedef struct amr_batch amr_batch;
typedef struct {
  amr_refine_result r;                    /* pointers into the batch's arrays, this geometry's segments */
  int64_t level_base[AMR_MAX_LEVELS];     /* first block of the geometry in each level's batch list:
                                             block_parent values and adj_cell / 4^dim are batch-global */
  int64_t adj_base;                       /* first adjacent-cell row: subtract from link_cell */
  int64_t pair_base;                      /* first adjacency pair: subtract from adj_off */
  int64_t link_base;                      /* first link */
  int64_t face_base;                      /* first face: subtract from adj_ids and link_face */
  int64_t vert_base;                      /* first vertex (indexed input) */
} amr_batch_view;
/* Create an empty batch of dimension dim on `stream` (NULL: its own stream). */
AMR_API amr_status amr_batch_create(int dim, void* stream, amr_batch** out);
AMR_API amr_status amr_batch_destroy(amr_batch* b);
/* Add one geometry (copied to the device now; host or device pointers): its own
 * domain (dom->stream ignored), levels, near-wall distance and bin density
 * (0 = set later with amr_batch_set_bins, e.g. from amr_autotune).  All
 * geometries use the same input form (index list or face-vertex list). */
AMR_API amr_status amr_batch_add(amr_batch* b, const amr_domain* dom, const float* coords, int64_t n_verts,
                                 const int32_t* idx, int64_t n_faces, int n_levels, double d_abs, double d_rel,
                                 int bin_density, int* index_out);
AMR_API amr_status amr_batch_set_bins(amr_batch* b, int index, int bin_density);
/* Gather, bin and refine every geometry.  params: lattice, want_adjacency,
 * want_links, use_graph, warps_per_cta (n_levels and distances are per geometry). */
AMR_API amr_status amr_batch_run(amr_batch* b, const amr_refine_params* params, amr_refine_result* out);
AMR_API amr_status amr_batch_get_view(amr_batch* b, int index, amr_batch_view* out);
/* Adjoint of all links of the last run: grad_out [sum n_verts][dim] (indexed) or
 * [sum n_faces][dim][dim]; device pointers. */
AMR_API amr_status amr_batch_q_backward(amr_batch* b, const float* grad_q, float* grad_out);
AMR_API const char* amr_batch_last_error(const amr_batch* b);
AMR_API int64_t amr_batch_launch_count(const amr_batch* b);

/* Number of CUDA kernels this context has launched since its creation. */
AMR_API int64_t amr_launch_count(const amr_ctx* ctx);

/* Binning that allocates nothing.  The paper has no counterpart: this is a
 * service for callers that cannot allocate device memory — e.g. a solver that
 * reserved the device's memory for its own arena up front, a plugin whose host
 * owns every device allocation, or a time-critical loop that must not pay the
 * implicit synchronisation of cudaMalloc / cudaFree.  It computes the same CSR
 * bins as amr_bin_faces without a context and without any allocation: its
 * scratch (bin counts, per-face bin ranges, scan tile states; about 2.6 MB) is a
 * fixed array in device global memory that every GPU loading this library holds
 * until the process exits.
 *   dom        domain (dim, root_blocks, origin, h0) and the stream to run on
 *              (NULL = the legacy default stream); no context is needed.
 *   faces      DEVICE f32 [dim*dim][n_faces]: vertex-major, then coordinate, then
 *              face (the structure-of-arrays form geom_f_face_X); caller-owned.
 *   n_faces    0 <= n_faces <= AMR_STATIC_MAX_FACES.
 *   bin_density B >= 1 with B^dim <= AMR_STATIC_MAX_BINS.
 *   offsets    DEVICE u32 [B^dim + 1], written (CSR start of every bin).
 *   ids        DEVICE u32 [ids_capacity], written (face ids grouped by bin; order
 *              within a bin unspecified).
 *   nnz        HOST, receives the number of (face, bin) entries.
 * Returns EINVAL for sizes beyond the maxima or pointers that are not device
 * (or managed) memory of the current device (nothing is launched), EINVAL too
 * when a coordinate is NaN or infinite (checked on the device; offsets, ids and
 * *nnz are then not valid), EOVERFLOW when nnz > ids_capacity (offsets and *nnz
 * are still valid, ids is untouched).  The call waits on its stream for the
 * count and the scan before it returns; the ids are written asynchronously on
 * the stream after that.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) and keeps it for the life of the
 * process; make that first call before any stream capture, and do not use this
 * entry point after a cudaDeviceReset of that device.  Every call shares the one
 * array per device, so calls whose work overlaps on the GPU (other streams or
 * threads) race: serialise them. */
#define AMR_STATIC_MAX_BINS (1 << 18)
#define AMR_STATIC_MAX_FACES (1 << 17)
AMR_API amr_status amr_bin_faces_static(const amr_domain* dom, const float* faces, int64_t n_faces, int bin_density,
                                        uint32_t* offsets, uint32_t* ids, int64_t ids_capacity, int64_t* nnz);

#ifdef __cplusplus
}
#endif
#endif
