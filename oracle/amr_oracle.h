/* amr_oracle.h — plain serial FP64 oracle of the geometry-to-AMR hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * bench's CPU-baseline leg load this library.  It shares no code with the CUDA
 * path and is not part of the product.
 *
 * It computes the plain definitions of the three steps of the paper
 * (Jaber, Essel, Sullivan 2025, Sec. "Methodology"):
 *   1. import:  faces as an index list or a face-vertex coordinate list
 *               (Sec. "Representation of the Complex Boundary Geometry");
 *   2. binning: every face goes to every bin its axis-aligned bounding box
 *               overlaps, B bins per axis over the domain
 *               (Sec. "Spatial Binning Algorithm");
 *   3. near-wall refinement: a cell is adjacent to a face when the cell box,
 *               inflated by the near-wall distance, intersects the closed face
 *               (pred 0, box), or when the cell centre lies within the
 *               near-wall distance of the closed face (pred 1, point: Alg. 1);
 *               flagged blocks split into 2^D children; adjacent cells of the
 *               finest level list their faces and form wall links with the
 *               lattice directions (Sec. "Cell-Face Identification Algorithms").
 *
 * Everything is FP64; FP32 inputs are promoted exactly.
 * Conventions (shared by the definition, not by code):
 *   - domain box: origin[a] + [0, 4*root[a]*h0] per axis; level-L cell size h_L = h0 * 2^-L;
 *   - block (b0,b1,b2) at level L covers cells 4*b .. 4*b+3 per axis;
 *   - cell bit within a block: i + 4*j (+ 16*k), x fastest;
 *   - root blocks in x-fastest lexicographic order; children in parent order,
 *     child slot s = bx + 2*by (+ 4*bz);
 *   - cell centre: origin + (c + 1/2) * h_L;
 *   - inflated half-width r_L = h_L/2 + d_L, d_L = d_abs + d_rel * h_L.
 */
#ifndef AMR_ORACLE_H
#define AMR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_geom orc_geom;

typedef struct {
  int dim;          /* 2 or 3 */
  int root[3];      /* root blocks per axis */
  double origin[3]; /* domain origin */
  double h0;        /* level-0 cell size */
} orc_domain;

/* Import.  idx == NULL: coords is a face-vertex list f32[n_faces][dim][dim];
 * else coords = verts f32[n_verts][dim] and idx = i32[n_faces][dim].
 * Returns NULL and fills err on invalid input. */
orc_geom* orc_geom_new(int dim, const float* coords, int64_t n_verts, const int32_t* idx,
                       int64_t n_faces, char* err, int errlen);
void orc_geom_free(orc_geom* g);
int64_t orc_geom_nfaces(const orc_geom* g);

/* Binning with B bins per axis over the domain box. */
int orc_bins_build(orc_geom* g, const orc_domain* dom, int B);
int64_t orc_bins_nnz(const orc_geom* g);

/* The paper's sampled binning (Sec. "Spatial Binning Algorithm"): the face is
 * discretised into points (first edge, then segments to the opposite vertex,
 * spacing at most half a bin length) and belongs to every bin holding one of
 * them.  Replaces the bins like orc_bins_build. */
int orc_bins_build_sampled(orc_geom* g, const orc_domain* dom, int B);

/* The sample points of face f at the given spacing (pts[cap][dim], may be NULL);
 * returns their number. */
int64_t orc_face_samples(const orc_geom* g, int64_t f, double spacing, double* pts, int64_t cap);

/* Refinement-mark propagation: `rounds` two-phase rounds in which every block with
 * flags == 1 marks (flags = 1) the existing blocks of the list among its 3^D - 1
 * neighbours of the same level. */
int orc_propagate(int dim, const int32_t* blocks, int64_t n, uint8_t* flags, int rounds);
void orc_bins_copy(const orc_geom* g, uint32_t* offsets, uint32_t* ids);
void orc_face_bin_range(const orc_geom* g, int64_t f, int32_t* lo, int32_t* hi);

/* Separating-axis margin of the closed box [-r, r]^dim and a closed face whose
 * vertices are given relative to the box centre (verts_local[dim][dim]).
 * Positive = separated by that distance along the best axis, <= 0 = intersect. */
double orc_sat_margin(int dim, const double* verts_local, double r);

/* Euclidean distance from the origin to the closed face whose vertices are
 * given relative to it (verts_local[dim][dim]); the point predicate of Alg. 1. */
double orc_point_face_dist(int dim, const double* verts_local);

/* Refinement of a list of blocks of one level: per block the adjacency bit of
 * every cell (mask) and the cells whose decision lies within the 1e-6*h_L
 * margin band (band).  pred: 0 = box predicate, 1 = point predicate (margin =
 * distance - d_L).  search: 0 = the faces of every bin the cell's inflated box
 * overlaps, 1 = the faces of the bin holding the cell centre (the paper's binned
 * search).  Counters may be NULL. */
int orc_refine_blocks(const orc_geom* g, const orc_domain* dom, int level, double d_abs, double d_rel, int pred,
                      int search,
                      const int32_t* blocks, int64_t n, uint64_t* mask, uint64_t* band,
                      int64_t* n_band_pairs, int64_t* n_candidates);

/* Node classification: generalized winding number of the closed mesh at x
 * (+-1 inside a closed, consistently oriented mesh, 0 outside), and per cell
 * centre solid = |w| > 1/2, band = the centre lies within 1e-6*h_L of the mesh. */
double orc_winding_number(const orc_geom* g, const double* x);
int orc_classify(const orc_geom* g, const orc_domain* dom, int level, const int32_t* cells, int64_t n,
                 uint8_t* solid, uint8_t* band);

/* Children of the flagged blocks (mask != 0), canonical order.  child_* may be
 * NULL to only count. Returns the number of children. */
int64_t orc_children(int dim, const int32_t* blocks, int64_t n, const uint64_t* mask,
                     int32_t* child_blocks, int32_t* child_parent);

/* Adjacent faces of given cells (global cell coords [n][dim] at `level`),
 * ascending face ids.  counts[n]; ids/band written up to `cap` entries
 * (band[e] = 1 when that pair's margin is within the band).  Returns total entries. */
int64_t orc_cell_faces(const orc_geom* g, const orc_domain* dom, int level, double d_abs, double d_rel, int pred,
                       int search,
                       const int32_t* cells, int64_t n, int64_t* counts, uint32_t* ids, uint8_t* band,
                       int64_t cap);

/* Wall links of given cells along lattice (9 = D2Q9, 19 = D3Q19) directions 1..Q-1:
 * q[n][Q-1] (NaN = no hit), face[n][Q-1] (-1 = no hit), band[n][Q-1] (1 = the
 * hit/miss or q is within the 1e-6 margin band).  */
int orc_cell_links(const orc_geom* g, const orc_domain* dom, int level, int lattice,
                   const int32_t* cells, int64_t n, double* q, int64_t* face, uint8_t* band);

/* Velocity-set direction i (0..Q-1) of a lattice. Returns 0 on success. */
int orc_lattice_dir(int lattice, int i, int* c);

/* q of one (cell, direction, face) triple, with the face vertices taken from
 * `verts_override` ([dim][dim], NULL = the stored face).  NaN = no hit. */
double orc_link_q(const orc_geom* g, const orc_domain* dom, int level, int lattice, const int32_t* cell,
                  int dir, int64_t face, const double* verts_override);

/* Analytic gradient of L = sum_k grad_q[k] * q_k over the given links with
 * respect to the face-vertex coordinates: grad[n_faces][dim][dim] (accumulated). */
int orc_q_grad(const orc_geom* g, const orc_domain* dom, int level, int lattice, const int32_t* cells,
               const int32_t* dirs, const int64_t* faces, const double* grad_q, int64_t n_links,
               double* grad);

#ifdef __cplusplus
}
#endif
#endif
