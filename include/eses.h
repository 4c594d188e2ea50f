/*
 * eses.h -- C ABI of the GB300 ESES library (libeses.so).
 *
 * Eulerian solvent excluded surface: given atoms (centres c_i, van der Waals
 * radii r_i; Eq. 1), a probe radius r_p, a grid spacing h and a margin, the
 * library labels every point of a Cartesian grid as inside or outside the
 * solvent excluded surface (Eq. 2), computes the intersection of every grid
 * edge whose end labels differ with the surface (Eq. 3-4) together with the
 * surface normal there, and the surface area and enclosed volume.
 *
 * The SES is the boundary of the union of all probe balls of radius r_p whose
 * centres are at distance >= r_i + r_p from every atom (§1).  A grid point x
 * is inside (label 1) iff dist(x, free probe centres) >= r_p.  r_p must be
 * > 0: at r_p = 0 that set is the whole space and the surface degenerates to
 * the van der Waals surface.
 *
 * Grid (Eq. 2, §2.3): point (i,j,k) sits at origin + h*(i,j,k) with
 *   origin_a = min_i(c_ia - r_i) - margin,
 *   dims_a   = ceil((max_i(c_ia + r_i) + margin - origin_a) / h) + 1.
 * Labels are stored C order, k fastest: index = (i*dims[1] + j)*dims[2] + k.
 *
 * Intersections (Eq. 3-4): for each axis a, one record per edge
 * (p, p + e_a) with different labels: lower point linear index, tau in
 * [0,1] such that the surface point is p + tau*h*e_a (the paper's lambda is
 * 1 - tau), and the unit normal pointing into the solvent.  When an edge
 * holds several roots the first one from the lower point is reported.
 * Records are ordered by tile (8x8x8-point tiles in C order of the tile
 * index), then by lower index within the tile; the order is deterministic.
 *
 * Area  = h^2 * sum over all crossing edges of |n_a| (a = the edge's axis).
 * Volume = h^2/3 * sum over the three axes of the inside length along grid
 * lines (an edge with both ends inside counts h; a crossing edge counts the
 * part on the inside end's side of the root).
 *
 * Blocks (§2.3-2.5, Algorithm 1): the paper splits the grid into cubic
 * blocks computed independently, each with the atoms near it.  Here the
 * blocks are the unit of eses_set_blocks (block selections for streaming or
 * for sharding one molecule over processes): block b along an axis owns the
 * points [b B, min((b+1) B, dims)) and the edges leaving them in +
 * directions, B = ESES_OPT_BLOCK_PTS.  (The paper's blocks share their faces,
 * B - 1 cells; these own B points each, so that a block is whole 8x8x8
 * tiles.)  Results never depend on B or on the selection.
 *
 * Conventions for every function below:
 *   - return value 0 on success, a negative ESES_E* code on failure; on
 *     failure eses_last_error() describes the cause;
 *   - no exception crosses the ABI; no call aborts the process;
 *   - pointers documented "host" must be host memory, "device" must be
 *     memory of the context's device; all sizes are element counts;
 *   - a context is used by one host thread at a time.
 */
#ifndef ESES_H
#define ESES_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct eses_ctx eses_ctx;

#define ESES_OK 0
#define ESES_EINVAL (-1)    /* invalid argument (sizes, non-finite input, r <= 0, r_p <= 0, h <= 0, margin < h,
                                a molecule's grid of 2^31 or more 8x8x8-point tiles) */
#define ESES_ENOMEM (-2)    /* host or device allocation failed */
#define ESES_ECUDA (-3)     /* a CUDA call failed */
#define ESES_ETIMEOUT (-4)  /* a bounded device wait expired */
#define ESES_ECAPACITY (-5) /* a per-tile list exceeded its capacity (even in global memory, see eses_stats [15]) */
#define ESES_ESTATE (-6)    /* call out of order (e.g. results before eses_run) */
#define ESES_EROOT (-7)     /* a crossing edge had no surface root (numerical failure) */

/* option keys for eses_set_option */
#define ESES_OPT_BLOCK_PTS 1   /* B, points per block edge for eses_set_blocks: a multiple of 8 in [8, 2^20]
                                  (default 64); changing it clears a block selection */
#define ESES_OPT_PRECISION 2   /* ESES_PREC_* (default ESES_PREC_FP32_FILTERED) */
#define ESES_OPT_STREAM 3      /* cudaStream_t cast to int64 (0 = the context's own stream) */
#define ESES_OPT_SYNC 4        /* 1 (default): eses_run waits for the device; 0: returns after enqueueing */
#define ESES_OPT_PROFILE 5     /* 1: time every stage of eses_run with CUDA events (eses_stage_times) */
#define ESES_OPT_GRAPH 6       /* 1: after the first (planning) run, capture the device path in one CUDA graph
                                  and replay it on every later eses_run (default 0) */
#define ESES_OPT_QUEUE 7       /* 1 (default): persistent tile kernels take tiles from a device work queue;
                                  0: fixed grid-stride order */
#define ESES_OPT_CLS_CTAS 8    /* classification CTAs per SM (0 = occupancy limit, default) */
#define ESES_OPT_CLS_TILES 9   /* classification tiles per queue pop (default 4) */
#define ESES_OPT_EDGE_CTAS 10  /* root-solve staging pass: CTAs per SM (0 = occupancy limit, default) */
#define ESES_OPT_EDGE_TILES 11 /* root-solve staging pass: tiles per queue pop (default 4) */
#define ESES_OPT_ROOT_THREADS 12 /* root solve: threads per block of the per-candidate root kernels
                                    (0 = 256, default; 64, 128 or 256) */
#define ESES_OPT_EXTERIOR 13   /* 1: exterior-only surface -- outside points that no path of outside grid points
                                  (6-neighbour steps) joins to the domain boundary lie in cavities and are labelled
                                  inside before the crossing edges are found (default 0: every free probe position
                                  is solvent, §1).  Its sweeps are synchronised from the host, so a run with this
                                  option is never captured in a CUDA graph.  Timed in the "band" stage; the number
                                  of filled points is eses_stats [13]. */
#define ESES_OPT_TC_WAIT 14    /* for tests of the failure path: polls of each tensor-core wait of the proposer's
                                  scoring (-1 = the default limit, 2^22).  A wait that runs out makes eses_run return
                                  ESES_ETIMEOUT with exact labels (the tiles go to the exact classification); 0 makes
                                  every scoring wait give up at once.  The wait before the tensor memory is freed
                                  always uses the default limit, so no memory is freed under work in flight. */
#define ESES_OPT_CULL 16       /* 1 (default): buried-patch pre-culling (the paper's proposed improvement, §5):
                                  only the circles that keep a free arc, the expanded spheres that keep a free face
                                  and the free triple points carry witnesses into the tiles; 0: every circle and
                                  every face does (results are identical; for measuring what the culling saves) */
#define ESES_OPT_FAIL_ALLOC 15 /* for tests of the failure path: N >= 1 makes the N-th device allocation that the
                                  context's next eses_run, eses_autotune, eses_set_proposer or eses_mesh_count calls
                                  attempt fail with ESES_ENOMEM before cudaMalloc is called (the count runs across
                                  calls until it fires; 0 = never, the default).  The context stays valid: the next
                                  run plans again, and eses_destroy releases every buffer. */

#define ESES_PROPOSER_OFF 0      /* classify every tile (default) */
#define ESES_PROPOSER_MLP 1      /* the MLP scores tiles; those scored far are certified and filled */
#define ESES_PROPOSER_CERTIFY 2  /* the certificate on every tile (no network) */

#define ESES_MLP_NPARAM 6337     /* parameters of the proposer MLP (layout at eses_set_proposer) */

#define ESES_PREC_FP64 0           /* every step in FP64 */
#define ESES_PREC_FP32_FILTERED 1  /* FP32 with a forward-error filter, FP64 inside the filter band */

/* Create a context for one molecule.  xyz: host, n_atoms*3 doubles (x,y,z per
 * atom, Angstrom); radii: host, n_atoms doubles.  Both are copied; the caller
 * keeps ownership.  Uses the current CUDA device.  *out receives the context
 * (NULL on failure).  Coincident atoms (equal centre and radius) are one
 * ball: repeats are dropped (the union of balls, hence the surface, is the
 * same); atom indices reported by the library are input indices. */
int eses_create(const double *xyz, const double *radii, int64_t n_atoms, double r_p, double h, double margin,
                eses_ctx **out);

/* As eses_create, for one molecule on a grid the caller gives instead of the
 * grid of Eq. 2: point (i,j,k) at origin + h*(i,j,k), dims[a] points per axis
 * (host, 3 values each; dims in [1, 2^30], at most 2^40 points).  The atoms
 * need not lie inside the grid.  This is for the ranks of one molecule split
 * over processes: each holds only the atoms near its blocks and all must use
 * the molecule's own grid.  The labels and intersections of every point
 * equal those of a context holding all atoms on the same grid as long as
 * the atoms within r_i + 2 r_p (+ 1e-6 A) of the computed box (see
 * eses_set_blocks) are present (§2.2: nothing farther can change a point). */
int eses_create_on_grid(const double *xyz, const double *radii, int64_t n_atoms, double r_p, double h,
                        const double origin[3], const int64_t dims[3], eses_ctx **out);

/* As eses_create, with xyz and radii in device memory (copied on the device). */
int eses_create_device(const double *xyz, const double *radii, int64_t n_atoms, double r_p, double h, double margin,
                       eses_ctx **out);

/* Create a context for a batch of n_mol molecules that share r_p, h and
 * margin.  xyz: host, 3 doubles per atom, the molecules' atoms one after the
 * other; radii: host, one double per atom, same order; n_atoms: host, n_mol
 * counts (each >= 1).  Every molecule gets its own grid (Eq. 2 on its own
 * atoms) and its own results, equal to what eses_create on that molecule
 * alone gives; a run processes all molecules together (one launch per stage,
 * persistent tile kernels with a device work queue).  Results are read with
 * the eses_mol_* functions (the single-molecule accessors below return
 * ESES_EINVAL on a context with more than one molecule).  This batching has
 * no counterpart in the paper, which runs one molecule at a time. */
int eses_create_batch(const double *xyz, const double *radii, const int64_t *n_atoms, int n_mol, double r_p,
                      double h, double margin, eses_ctx **out);

/* Create a batch context from one host array per molecule (xyz[m]: 3 *
 * n_atoms[m] doubles, radii[m]: n_atoms[m] doubles; copied) and run it once.
 * On failure *out is NULL and eses_last_error(NULL) describes the cause. */
int eses_run_batch(int n_mol, const double *const *xyz, const double *const *radii, const int64_t *n_atoms,
                   double r_p, double h, double margin, eses_ctx **out);

/* Set an option (ESES_OPT_*).  Takes effect at the next eses_run. */
int eses_set_option(eses_ctx *ctx, int key, int64_t value);

/* Read an option's current value (host output). */
int eses_get_option(const eses_ctx *ctx, int key, int64_t *value);

/* Autotuner: runs the context once, then times the persistent kernels
 * (classification; root solve) over their launch shapes -- CTAs per SM from 1
 * to the occupancy limit, tiles per queue pop, threads per block of the
 * root kernels -- on
 * the context's own workload, `reps` timed launches each (1..100), keeps the
 * fastest (readable with eses_get_option) and runs once more with it.
 * ms_out (host, 2 doubles, may be NULL): mean milliseconds of the chosen
 * classification and root-solve launches. */
int eses_autotune(eses_ctx *ctx, int reps, double *ms_out);

/* Learned tile proposer (a GPU-side addition; the paper classifies every
 * point).  Tiles are 8x8x8 points; a tile is "far" when all its labels are
 * equal.  mode ESES_PROPOSER_MLP: a multilayer perceptron 32 -> 64 -> 64 -> 1
 * (ReLU) scores every tile from 32 atom-density features (eses_tile_data) and
 * a tile whose score sigmoid(z) < p_far is checked by an exact certificate
 * from nearest-atom distance bounds around the tile centre t (points within
 * delta of t): all points outside if min_i(|t - c_i| - r_i - r_p) >= delta,
 * all inside if max_i(r_i - |t - c_i|) > delta.  Certified tiles are filled;
 * all other tiles are classified exactly, so labels never depend on the
 * network.  ESES_PROPOSER_CERTIFY applies the certificate to every tile.
 * params: host, ESES_MLP_NPARAM floats, copied (NULL keeps the previous
 * ones): W1[32][64] (input-major), b1[64], W2[64][64], b2[64], w3[64], b3.
 * eses_stats [11] counts the tiles proposed far, [12] the tiles certified. */
int eses_set_proposer(eses_ctx *ctx, int mode, const float *params, double p_far);

/* Number of 8x8x8-point tiles of the context, all molecules (host output). */
int eses_num_tiles(const eses_ctx *ctx, int64_t *n);

/* Training data of the proposer from the last run: device outputs, either may
 * be NULL: features (n_tiles * 32 floats, tile-major, the proposer's
 * features) and targets (n_tiles bytes, 1 where the tile's labels are not
 * all equal).  Tiles are numbered molecule by molecule, C order within one. */
int eses_tile_data(const eses_ctx *ctx, float *features, uint8_t *targets);

/* Training kernels of the proposer MLP (device pointers; stream = cudaStream_t
 * or NULL; they enqueue and return).  eses_mlp_forward: z[s] = MLP(X[s]) for
 * n samples of 32 features.  eses_mlp_grad: grad (ESES_MLP_NPARAM floats) and
 * loss (1 float) of L = sum_s w[s] * BCE(z_s, y[s]) (binary cross entropy on
 * the logit z); scratch holds eses_mlp_grad_scratch(n) floats; the result is
 * deterministic.  eses_mlp_adam: one Adam step (beta 0.9, 0.999, eps 1e-8,
 * step >= 1) on params with moments m, v.  Errors: ESES_EINVAL, ESES_ECUDA
 * (eses_last_error(NULL)). */
int eses_mlp_forward(const float *X, int64_t n, const float *params, float *z, void *stream);
int64_t eses_mlp_grad_scratch(int64_t n);
/* The proposer's scoring path on n rows: BF16 weights and activations on the
 * tensor cores (tcgen05.mma, FP32 accumulation in tensor memory); *err
 * (device int) gets bit 16 when a bounded wait ran out (those rows score
 * +inf). */
int eses_mlp_forward_tc(const float *X, int64_t n, const float *params, float *z, int *err, void *stream);
int eses_mlp_grad(const float *X, const float *y, const float *w, int64_t n, const float *params, float *grad,
                  float *loss, float *scratch, void *stream);
int eses_mlp_adam(float *params, const float *grad, float *m, float *v, int step, float lr, void *stream);

/* Triangle mesh of the surface from the last run's labels and intersections
 * (one molecule; ESES_EINVAL on a batch context, ESES_ESTATE before a run).
 * Cube by cube (lower corner in C order within 8x8x8 tiles, tiles in order),
 * each cube's triangles from a 256-case table built by this rule: corner i of
 * a cube sits at offset ((i >> 2) & 1, (i >> 1) & 1, i & 1); cube edge 4 a + j
 * runs along axis a from the j-th corner (increasing corner number) with axis-a
 * offset 0 and is cut when its labels differ; on each face two cut edges make
 * one segment and four make two, each joining the edges at one inside corner;
 * the segments close into loops, each started at its smallest edge, walked
 * first to the smaller neighbour, reversed after its first vertex when its
 * Newell normal (edge midpoints) points on the whole from outside corners to
 * inside ones, and cut into the fan (v0, v_k, v_k+1).  The mesh is closed and
 * its triangles face the solvent.  eses_mesh_count makes the mesh (device
 * buffers owned by the context, kept until the next run) and returns the
 * number of triangles (below 2^31).  eses_mesh copies it to host buffers,
 * either may be NULL: keys (n * 3 int64: per vertex 3 * (linear index of the
 * lower point of its edge) + axis) and xyz (n * 9 doubles: the three vertices,
 * each its edge's intersection point).  eses_mesh_table (no device needed)
 * writes the case table: tri[case * 3 * ESES_MESH_MAXT + 3 k + v] cube edges
 * (-1 past the last triangle), ntri[case] triangles, for the 256 cases (bit i
 * of the case: corner i inside). */
#define ESES_MESH_MAXT 5
int eses_mesh_count(eses_ctx *ctx, int64_t *n_tri);
int eses_mesh(eses_ctx *ctx, int64_t *keys, double *xyz);
int eses_mesh_table(int8_t *tri, uint8_t *ntri);

/* Number of molecules of the context (host output). */
int eses_num_molecules(const eses_ctx *ctx, int *n);

/* Per-molecule results of a batch context (molecule m in [0, n_mol)); the
 * same layout and semantics as the single-molecule functions below. */
int eses_mol_grid(const eses_ctx *ctx, int m, int64_t dims[3], double origin[3]);
int eses_mol_labels(const eses_ctx *ctx, int m, int8_t *out);
int eses_mol_labels_device(const eses_ctx *ctx, int m, const int8_t **dptr);
int eses_mol_num_intersections(const eses_ctx *ctx, int m, int axis, int64_t *n);
int eses_mol_intersections(const eses_ctx *ctx, int m, int axis, int64_t *lower_idx, double *tau, double *normal,
                           float *tau32, float *normal32);
int eses_mol_intersections_device(const eses_ctx *ctx, int m, int axis, const int64_t **lower_idx,
                                  const double **tau, const double **normal, const float **tau32,
                                  const float **normal32);
int eses_mol_area_volume(const eses_ctx *ctx, int m, double *area, double *volume);
int eses_mol_intersection_patches(const eses_ctx *ctx, int m, int axis, int8_t *kind, int32_t *atoms);

/* Run the whole path: cell binning, patch construction, classification,
 * crossing edges, root solve, area and volume.  Results stay in device memory
 * owned by the context until the next eses_run or eses_destroy.  Limits of
 * one context: fewer than 2^27 atoms, circle pairs and free triple points
 * (ESES_EINVAL), and fewer than 2^31 crossing edges over all molecules (their
 * offsets are 32-bit; 2^31 edges would take about 200 GB of outputs). */
int eses_run(eses_ctx *ctx);

/* Block selections of a one-molecule context (§2.3-2.5, Algorithm 1 runs
 * blocks one by one; here a selection is one run).  eses_num_blocks: blocks
 * per axis, ceil(dims / B) (host output).  eses_set_blocks: the next runs
 * compute only the blocks [block_lo[a], block_hi[a]) per axis (host, 3
 * values each; 0 <= lo < hi <= eses_num_blocks); NULL, NULL restores the
 * whole grid.  A selection owns the points of its blocks; the run also
 * labels one 8-point layer of tiles beyond them in + directions (the other
 * ends of the owned edges) but reports only owned points: eses_labels copies
 * the owned box (eses_owned_box: its first point lo[3] and extent dims[3] in
 * grid points), the intersections are the owned edges with lower indices of
 * the full grid (eses_grid), in tile order within the selection, and area,
 * volume and eses_stats [0] cover the owned part, so the results of disjoint
 * selections add up to the whole grid's.  Device memory follows the
 * selection's size: a grid larger than the device is run in selections.
 * Under a selection eses_labels_device, eses_mesh_count and the
 * exterior-only option return an error (they need the whole grid).  One run
 * computes fewer than 2^29 tiles of 8x8x8 points (about 2.7e11 points);
 * eses_run returns ESES_EINVAL for a larger grid without a selection. */
int eses_num_blocks(const eses_ctx *ctx, int64_t nblocks[3]);
int eses_set_blocks(eses_ctx *ctx, const int64_t block_lo[3], const int64_t block_hi[3]);
int eses_owned_box(const eses_ctx *ctx, int64_t lo[3], int64_t dims[3]);

/* Grid dimensions and origin (host outputs, 3 values each). */
int eses_grid(const eses_ctx *ctx, int64_t dims[3], double origin[3]);

/* Copy the labels (int8, dims[0]*dims[1]*dims[2], C order) to host memory. */
int eses_labels(const eses_ctx *ctx, int8_t *out);

/* Borrow the device pointer of the labels; valid until the next eses_run or
 * eses_destroy. */
int eses_labels_device(const eses_ctx *ctx, const int8_t **dptr);

/* Number of crossing edges along axis (0,1,2). */
int eses_num_intersections(const eses_ctx *ctx, int axis, int64_t *n);

/* Copy the intersections of one axis to host memory.  Every output is
 * caller-allocated for eses_num_intersections() records and may be NULL:
 * lower_idx (int64), tau (double), normal (3 doubles per record), tau32 and
 * normal32 (the same in float). */
int eses_intersections(const eses_ctx *ctx, int axis, int64_t *lower_idx, double *tau, double *normal,
                       float *tau32, float *normal32);

/* Borrow the device pointers of one axis' intersections (valid until the next
 * eses_run or eses_destroy); any output pointer may be NULL. */
int eses_intersections_device(const eses_ctx *ctx, int axis, const int64_t **lower_idx, const double **tau,
                              const double **normal, const float **tau32, const float **normal32);

/* The surface patch of every intersection of one axis and the atoms that
 * generate it -- the "nearby atoms" of each surface point that the paper's
 * chain colouring uses (§4.1).  Host outputs, caller-allocated for
 * eses_num_intersections() records, in the order of eses_intersections, each
 * may be NULL: kind (int8: 0 convex patch of a van der Waals sphere, 1 saddle
 * patch of a pair torus, 2 concave patch of a probe sphere at a free triple
 * point, -1 an edge with no root, see ESES_EROOT) and atoms (3 int32 per
 * record: the input indices of the patch's one, two or three atoms in
 * ascending order, padded with -1).  The patch is the one whose witness is
 * the nearest free probe centre at the intersection; where two patches meet
 * at an intersection (a crease, measure zero) either may be reported. */
int eses_intersection_patches(const eses_ctx *ctx, int axis, int8_t *kind, int32_t *atoms);

/* Surface area (A^2) and enclosed volume (A^3), host outputs. */
int eses_area_volume(const eses_ctx *ctx, double *area, double *volume);

/* Diagnostics of the last run, host output of up to n int64 values:
 * [0] points, [1] tiles, [2] tiles with work, [3] circle pairs, [4] pairs
 * with a free arc, [5] free triple points, [6] points re-evaluated in FP64
 * (filter band), [7] crossing edges (all axes), [8] edges with a reported
 * root failure, [9] inside points, [10] kernels launched by the run,
 * [11] tiles proposed far, [12] tiles certified far (eses_set_proposer),
 * [13] cavity points labelled inside (ESES_OPT_EXTERIOR), [14] flood-fill
 * sweeps, [15] tile stagings that overflowed the shared-memory lists (256
 * atoms, 384 free-arc pairs, 384 free triple points in the classification
 * and the root solve's staging pass; 320, 512, 640 in the FP64
 * re-evaluation) and were redone with lists in global memory (1024, 2048,
 * 2048; beyond those ESES_ECAPACITY),
 * summed over the classification, the FP64 re-evaluation and the root solve;
 * [16] atom tests of the classification's witness freeness checks (each
 * convex or saddle witness of a shell point is tested against the staged
 * atoms whose expanded spheres meet its atoms' ones, one test per atom);
 * [17] (edge, sphere) and [18] (edge, torus) candidates of the root solve's
 * prefilter, [19] crossing edges that took the warp selection. */
int eses_stats(const eses_ctx *ctx, int64_t *out, int n);

/* Device time in milliseconds of every stage of the last eses_run, measured
 * with CUDA events on the context's stream (requires ESES_OPT_PROFILE = 1),
 * host output of up to n values: [0] cell binning, [1] neighbours and circle
 * pairs, [2] free arcs, triple points and patch bins, [3] classification,
 * [4] FP64 band re-evaluation, [5] crossing-edge counts and offsets,
 * [6] root solve (first root and its patch per crossing edge), [7] FP64 root
 * polish, normals and area/volume terms, [8] area/volume reduction.  Stages
 * that wait for a host read of a list total include that wait. */
int eses_stage_times(const eses_ctx *ctx, double *ms, int n);

/* Records of crossing edges whose root solve failed in the last run (at most
 * 8 are kept), host output of max_records * 24 int64: [0] axis, [1..3] lower
 * point (i,j,k), [4] label of the lower point, [5..7] staged atoms, circle
 * pairs and triple points of its tile, [8] candidate roots of the edge,
 * [9..15] the first candidates' root distance from the lower point in 1e-9 A,
 * [16..22] their patch kinds (0 convex, 1 saddle, 2 concave), [23] the
 * molecule.  *n_out receives the number of records copied. */
int eses_root_failures(const eses_ctx *ctx, int64_t *records, int max_records, int *n_out);

/* Patch model of the last run (§1: saddle patches lie on the circles where
 * two expanded spheres meet, concave patches are centred on free triple
 * points): number of circle pairs, of pairs whose circle keeps a free arc,
 * and of free triple points (host outputs). */
int eses_patch_counts(const eses_ctx *ctx, int64_t *n_pairs, int64_t *n_free_pairs, int64_t *n_vertices);

/* Copy the patch model to host memory; every output may be NULL and is sized
 * from eses_patch_counts: pair_atoms (2 int32 per pair, input atom indices,
 * first < second), pair_free (1 per pair), pair_circle (7 doubles per pair:
 * centre, unit axis from the first to the second atom, radius), vertices (3
 * doubles per free triple point).  A circle is always computed from its atom
 * with the smaller input index, so its bits do not depend on the order in
 * which the library sorts the atoms. */
int eses_patch_data(const eses_ctx *ctx, int32_t *pair_atoms, uint8_t *pair_free, double *pair_circle,
                    double *vertices);

/* List the crossing edges of a label grid without allocating any memory.
 * There is no counterpart in the paper: this entry point exists for callers
 * that cannot call cudaMalloc -- code whose device memory is owned by a
 * framework allocator or a fixed budget, or work issued where allocation is
 * not allowed.
 * labels: device, int8 (0/1), dims[0]*dims[1]*dims[2], C order (as from
 * eses_labels_device); dims: host, 3 values.  idx0, idx1, idx2: device,
 * caller-allocated int64 outputs of capacity[0..2] entries: the lower point's
 * linear index of every edge along axis 0, 1, 2 whose end labels differ, in
 * the order of eses_intersections.  counts: host output, the number of such
 * edges per axis.  stream: a cudaStream_t (NULL: the default stream); the
 * call waits for that stream before returning.
 * Its working memory (per-tile counts and offsets) is one file-scope device
 * array sized for 131,072 tiles of 8x8x8 points (at most 67,108,864 grid
 * points, about 3 MiB, held by every GPU that loads the library until the
 * process exits).  Larger grids return ESES_EINVAL.  The first call on a
 * device looks up that array's address (make it before any stream capture)
 * and keeps it for the life of the process: after cudaDeviceReset do not call
 * this entry point again on that device.
 * Calls share the array: calls that overlap on the GPU race.  Returns
 * ESES_ECAPACITY when a count exceeds its capacity (the first capacity[a]
 * entries are written), ESES_EINVAL for NULL pointers or bad sizes,
 * ESES_ECUDA when a CUDA call fails.  It does not set eses_last_error. */
int eses_crossing_edges_noalloc(const int8_t *labels, const int64_t dims[3], int64_t *idx0, int64_t *idx1,
                                int64_t *idx2, const int64_t capacity[3], int64_t counts[3], void *stream);

/* Last error message of the context (or of the last failed create when ctx
 * is NULL).  Never NULL. */
const char *eses_last_error(const eses_ctx *ctx);

/* Release every resource of the context.  NULL is accepted. */
void eses_destroy(eses_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* ESES_H */
