// eses_kernels.h -- host-side launchers of the libeses kernels (internal).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "eses_internal.cuh"

namespace eses {

// ---- exclusive scan (eses_scan.cu) ---------------------------------------
// out[0..n] = exclusive prefix sums of in[0..n-1]; out[n] = total.  `tmp`
// must hold scan_tmp_ints(n) ints.  in and out may not alias.
long long scan_tmp_ints(long long n);
int scan_exclusive(const int *in, int *out, long long n, int *tmp, cudaStream_t st);

// ---- model construction (eses_model.cu) ----------------------------------
struct ModelBuf;  // owned by the context
int launch_cell_count(const double *xyz, const int *in_mol, int n, const CellGrid *cg, double cell, int *cell_id,
                      int *cell_count, cudaStream_t st);
int launch_cell_scatter(const double *xyz, const double *r, int n, const int *cell_id, const int *cell_start,
                         int *cursor, int *sorted_orig, cudaStream_t st);
int launch_cell_finish(const double *xyz, const double *r, const int *in_mol, int ncell, const int *cell_start,
                       int *sorted_orig, double4 *atom, int *atom_mol, cudaStream_t st);
int launch_nb_count(const Model &M, int *nb_count, int *circle_count, uint8_t *contained, cudaStream_t st);
int launch_nb_fill(const Model &M, int *nb_list, cudaStream_t st);
int launch_pair_count(const Model &M, int *pair_count, cudaStream_t st);
int launch_pair_fill(const Model &M, const int *pair_start, double4 *pair_o, double4 *pair_u, int2 *pair_ij,
                      cudaStream_t st);
int launch_arcs(const Model &M, uint8_t *pair_free, int *vert_count, cudaStream_t st);
int launch_arcs_emit(const Model &M, const int *vert_start, double4 *vert, int *vert_mol, int4 *vert_atoms,
                     cudaStream_t st);
int launch_faces(const Model &M, const int *circle_count, const uint8_t *contained, uint8_t *face, cudaStream_t st);
int launch_bin_count(const Model &M, int which, bool cull, int *count, int *item_cell, cudaStream_t st);
// FP32 double-float copies: which 0 atoms (hi, lo), 1 circles (hi, lo, axis), 2 triple points (hi, lo)
int launch_model_f32(const Model &M, int which, const Grid *grids, float4 *hi, float4 *lo_, float4 *u32,
                     cudaStream_t st);
int launch_bin_scatter(const Model &M, int which, const int *item_cell, const int *start, int *cursor, int *list,
                        cudaStream_t st);

// ---- classification (eses_classify.cu) -----------------------------------
// persistent: `grid` CTAs take tiles in the order of Q (labels of the whole batch)
void classify_init();
int classify_ctas_per_sm(int precision);
// ovf: int[2 + tiles] scratch (tiles sent to the global-memory tier over the
// run, the stage's count, then the tiles that overflowed the shared-memory
// staging); big: classify_big_bytes() of global scratch for that tier
// n_tests (may be null): adds up the atom tests of the shell points' witness freeness
int launch_classify(const Model &M, const Batch &B, int precision, const TileSched &Q, int grid, int8_t *labels,
                    int *tile_band, int *err, int *ovf, unsigned char *big, unsigned long long *n_tests,
                    cudaStream_t st);
size_t classify_big_bytes();
int launch_band(const Model &M, const Batch &B, int8_t *labels, const int *tile_band, int *err, int *ovf,
                unsigned char *big, cudaStream_t st);
// exterior-only surface (eses_exterior.cu): state init, one sweep (sets *changed
// when it reached new points), cavity points relabelled inside (counted)
int launch_ext_init(const Batch &B, const int8_t *labels, uint8_t *ext, uint8_t *tile_open, cudaStream_t st);
int launch_ext_sweep(const Batch &B, uint8_t *ext, uint8_t *tile_open, int *changed, int grid, cudaStream_t st);
int launch_ext_fill(const Batch &B, uint8_t *ext, uint8_t *tile_open, int *flags, long long max_sweeps,
                    cudaStream_t st);
int launch_ext_apply(const Batch &B, int8_t *labels, const uint8_t *ext, unsigned long long *filled, cudaStream_t st);

// ---- crossing edges, roots, area/volume (eses_edges.cu) ------------------
int launch_edge_count(const Batch &B, const int8_t *labels, int *tile_edges, int *tile_inside_edges,
                      cudaStream_t st);
// medge[a * (n_mol + 1) + m]: first edge of molecule m in axis a's output
int launch_mol_edges(const Batch &B, const int *edge_start, long long *medge, cudaStream_t st);
struct EdgeOut {
    long long *idx[3];
    double *tau[3];
    double *nrm[3];
    float *tau32[3];
    float *nrm32[3];
    int2 *code[3];  // chosen piece per edge, from the warp solve to the FP64 polish
};
// failed-edge log: FAIL_LOG records of FAIL_REC int64 (axis, i, j, k, label,
// staged atoms/pairs/vertices, then the 16 edge_root debug counters)
constexpr int FAIL_LOG = 8;
constexpr int FAIL_REC = 24;
long long polish_blocks(long long n_edges);
// The root solve runs in phases linked by lists in HBM (eses_edges.cu):
// staging (per tile: staged lists, edge records, prefiltered (edge, piece)
// candidates), roots per sphere and per torus candidate, the easy picks, the
// warp selections.  RootRec: one accepted root of a candidate.
struct RootRec {
    double t64;    // exact root once computed (NaN before)
    float t, err;  // FP32 root and its error bound (A)
};
// buffers of the phased root solve; the capacities are planned by the caller
// from the totals the staging pass adds up in ctr ([0] slab bytes, [1] sphere
// and [2] torus candidates; [3] edges listed for the warp selection; [4] torus
// candidates listed for FP64 work)
struct RootWork {
    int4 *einfo;            // per crossing edge: slab (16-byte units), packed point/axis/label/dropped,
                            // first sphere and first torus candidate
    int *ecnt;              // per crossing edge: sphere candidates | torus candidates << 16
    int2 *csph, *ctor;      // candidates: (edge, staged item) and (edge, staged pair)
    uint8_t *nsph, *ntor;   // accepted roots per candidate
    RootRec *rsph, *rtor;   // their roots: 2 slots per sphere candidate, 4 per torus candidate
    unsigned char *slab;    // staged tiles
    unsigned long long *ctr;  // 8 counters, [4] the torus candidates listed for FP64 work
    int *hard;              // edges listed for the warp selection (at most one per edge)
    int2 *jobs;             // torus candidates with FP64 work: (candidate, 1 pending slots / 2 whole)
    long long cap_slab, cap_sph, cap_tor, cap_jobs;
    long long n_edges;      // crossing edges of the run (all axes)
};
void edges_init();
int edge_ctas_per_sm(int precision);
bool root_threads_valid(int threads);  // 0 (the default, 256), 64, 128 or 256
long long slab_bytes_max(int precision);  // one tile's slab at the global tier's capacities
// staging pass: persistent, `grid` CTAs take tiles in the order of Q (its head
// and W.ctr are reset first); then the global-memory tier over the tiles ovf lists
int launch_edge_stage(const Model &M, const Batch &B, int precision, const TileSched &Q, int grid,
                      const int8_t *labels, const int *edge_start, EdgeOut out, int *err, int *ovf,
                      unsigned char *big, const RootWork &W, cudaStream_t st);
// roots of the candidates, picks and warp selections (`threads` per block of the root kernels)
int launch_edge_roots(const Model &M, const Batch &B, int precision, int threads, EdgeOut out,
                      const int *edge_start, long long ne_all, int *n_fail, int *err, long long *fail_log,
                      const RootWork &W, cudaStream_t st);
size_t edges_big_bytes();
int launch_edge_polish(const Model &M, const Batch &B, EdgeOut out, long long n_edges_total, const long long *medge,
                       double2 *term, cudaStream_t st);
// triangle mesh of a one-molecule run (eses_mesh.cu): the case table to constant
// memory (once per device), the host copy of it, crossing-edge masks per tile,
// triangles per tile, and the triangles (keys and FP64 points)
int mesh_init();
int mesh_table_host(int8_t *tri, uint8_t *n, int max_tri);
int launch_mesh_masks(const Batch &B, const int8_t *labels, uint32_t *mask, cudaStream_t st);
int launch_mesh_count(const Batch &B, const int8_t *labels, int *tile_tri, cudaStream_t st);
int launch_mesh_emit(const Batch &B, const int8_t *labels, const uint32_t *mask, const int *edge_start,
                     const EdgeOut &out, const int *tile_off, long long *keys, double *xyz, int *err, cudaStream_t st);
// part_d / part_i: reduce_scratch(n_mol) doubles / int64 each
long long reduce_scratch(int n_mol);
int launch_reduce(const Batch &B, const double2 *term, const long long *medge, const int *tile_inside, double *part_d,
                  long long *part_i, double *out2, long long *counts, cudaStream_t st);

// ---- learned tile proposer (eses_mlp.cu) ---------------------------------
// MLP 32 -> 64 -> 64 -> 1 with ReLU; parameters in one float vector:
// W1[32][64] (in x out), b1[64], W2[64][64], b2[64], w3[64], b3
constexpr int MLP_IN = 32, MLP_H = 64;
constexpr int P_W1 = 0;
constexpr int P_B1 = P_W1 + MLP_IN * MLP_H;
constexpr int P_W2 = P_B1 + MLP_H;
constexpr int P_B2 = P_W2 + MLP_H * MLP_H;
constexpr int P_W3 = P_B2 + MLP_H;
constexpr int P_B3 = P_W3 + MLP_H;
constexpr int MLP_NPARAM = P_B3 + 1;
void mlp_init();
int launch_mlp_forward(const float *X, int n, const float *P, float *z, cudaStream_t st);
long long mlp_grad_scratch(int n);  // floats
int launch_mlp_grad(const float *X, const float *y, const float *w, int n, const float *P, float *part, float *grad,
                    float *loss, cudaStream_t st);
int launch_adam(float *P, const float *g, float *m, float *v, int step, float lr, cudaStream_t st);
int launch_tile_features(const Model &M, const Batch &B, float *feat, cudaStream_t st);
int launch_tile_targets(const Batch &B, const int8_t *labels, uint8_t *target, cudaStream_t st);
// mode 1: MLP + certificate, 2: certificate on every tile; need[t] = 1 for
// tiles left to the exact classification; counts[0..1] += proposed, certified;
// wait_limit: polls of each tensor-core wait (< 0: the default limit)
int launch_propose(const Model &M, const Batch &B, int mode, const float *P, float z_far, int8_t *labels,
                   int *tile_band, int *need, int *counts, int *err, long long wait_limit, cudaStream_t st);
// the proposer's tensor-core MLP on n rows of features (err |= ERR_TIMEOUT on a wait that ran out)
int launch_mlp_forward_tc(const float *X, int n, const float *P, float *z, int *err, cudaStream_t st);
int launch_compact(long long n, const int *need, const int *pos, int *list, cudaStream_t st);

}  // namespace eses
