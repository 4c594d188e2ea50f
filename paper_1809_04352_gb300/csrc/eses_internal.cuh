// eses_internal.cuh -- data layout shared by the kernels of libeses.
//
// Everything lives in device memory owned by one context:
//   atoms       sorted by cell (counting sort), double4 (x, y, z, r)
//   cell grid   uniform cells of edge 2*R_max, CSR cell_start
//   neighbours  CSR: j with |c_i - c_j| < R_i + R_j (R = r + r_p)
//   pairs       i < j with an intersection circle of the expanded spheres
//               (saddle patch carrier, §1): centre o, axis u, radius rho,
//               flag "has a free arc"
//   vertices    free triple points (concave patch centres, §1)
//   patch bins  free-arc pairs binned by o, vertices binned by position
// Tiles of 8x8x8 grid points are the unit of work; every tile stages the
// atoms, free-arc pairs and free vertices that can influence its points into
// shared memory (§2.2: the classification of a point depends only on atoms
// within r_max + 2 r_p).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace eses {

constexpr int TILE = 8;          // points per tile edge
constexpr int TILE_PTS = TILE * TILE * TILE;

// Per-tile staging capacities: the shared-memory tier every tile uses, and
// the larger tier in global memory for the tiles that overflow it (very
// dense atom sets); only a tile that overflows both is an error.
struct CapSmall {
    static constexpr int A = 320, P = 512, V = 640;
};
struct CapBig {
    static constexpr int A = 1024, P = 2048, V = 2048;
};
// the shared-memory tier of the classification and of the root solve's
// staging pass: lists sized so that four CTAs fit an SM (the tiles past them
// take the global-memory tier)
struct CapMid {
    static constexpr int A = 256, P = 384, V = 384;
};
constexpr int ERR_CAP_ANY = 1 | 2 | 4;  // ERR_CAP_ATOMS | ERR_CAP_PAIRS | ERR_CAP_VERTS

// device error bits (OR-ed into ctx->d_err)
enum : int {
    ERR_CAP_ATOMS = 1,
    ERR_CAP_PAIRS = 2,
    ERR_CAP_VERTS = 4,
    ERR_ROOT = 8,
    ERR_TIMEOUT = 16,
    ERR_CAP_EDGES = 32,
    ERR_CAP_CAND = 64,
};

// label codes in the label array
constexpr int8_t LABEL_OUT = 0;
constexpr int8_t LABEL_IN = 1;
constexpr int8_t LABEL_BAND = 2;  // FP32 filter undecided: re-evaluated in FP64

// Cell grid of one molecule: its cells hold ids coff .. coff + cn0*cn1*cn2 - 1
// of the cell arrays shared by all molecules of a batch.
struct CellGrid {
    double clo[3];                // cell grid origin
    int cn[3];                    // cells per axis
    int coff;                     // first cell id
};

// The patch model of every molecule of a batch.  Items of different molecules
// never interact: every cell-list query stays in the item's own molecule's
// cells, so all lists (neighbours, pairs, triple points) are built in one
// pass over the whole batch.
struct Model {
    int n_atoms;                  // all molecules
    int n_mol;
    const CellGrid *cg;           // per molecule
    const int *atom_mol;          // molecule of each sorted atom
    const double4 *atom;          // sorted atoms (x, y, z, r)
    const int *atom_orig;         // original index of each sorted atom (in the batch)
    const uint8_t *atom_face;     // 1: expanded sphere keeps a free face
    double cell;                  // cell edge (all molecules)
    const int *cell_start;        // ncell + 1
    const int *nb_start;          // n_atoms + 1
    const int *nb_list;
    int n_pairs;
    const double4 *pair_o;        // o.xyz, rho
    const double4 *pair_u;        // u.xyz, 0
    const int2 *pair_ij;          // sorted atom indices i < j
    const uint8_t *pair_free;     // 1: the circle keeps a free arc
    const int *pcell_start;       // free-arc pairs binned by o
    const int *pcell_list;
    int n_verts;
    const double4 *vert;          // free triple points (xyz, third atom of the triple as a double)
    const int *vert_mol;          // molecule of each triple point
    const int *vcell_start;
    const int *vcell_list;
    double rp, rmax, Rmax;
    // FP32 double-float copies relative to the grid origin (value = hi + lo):
    // staging in FP32 keeps the FP64 frame's accuracy without FP64 arithmetic
    const float4 *atom_hi;        // (x, y, z, r)
    const float4 *atom_lo;        // (x, y, z, 0)
    const float4 *pair_hi;        // (o, rho)
    const float4 *pair_lo;        // (o, 0)
    const float4 *pair_u32;       // (u, 0)
    const float4 *vert_hi;
    const float4 *vert_lo;
};

// The grid of one molecule (Eq. 2 with the origin of its reading), or the box
// of it that a block selection computes: the box starts at tile toff of the
// molecule's full grid (point 8 toff), holds dims points (its labels, C
// order), and owns the first own[a] points along each axis -- only owned
// points give edges, intersections and area/volume terms; the rest of the
// box is the layer of neighbours the owned edges need.  Without a selection
// toff = 0 and own = dims = full.
struct Grid {
    double lo[3];                 // origin of the full grid
    double h;
    long long dims[3];            // points of the computed box
    long long own[3];             // owned points from the box origin
    long long full[3];            // points of the full grid (output lower indices index it)
    int toff[3];                  // first tile of the box in the full grid
    int tiles[3];
    long long n_tiles;
    long long tile0;              // index of its first tile in the batch
    long long lab0;               // offset of its labels in the batch's label array
    double rp;
    double halo;                  // r_max + 2 r_p
    float d0;                     // FP32 error bound of a staged position difference
    float hl[TILE + 1];           // k * h rounded to FP32, k = 0..8 (tile-frame point coordinates)
    float ht_hi, ht_lo;           // TILE * h as a double-float
};

// The tiles of a batch: molecule m owns global tiles tile_off[m] .. tile_off[m+1]-1.
struct Batch {
    int n_mol;
    long long n_tiles;            // all molecules
    const Grid *grid;             // per molecule
    const long long *tile_off;    // n_mol + 1
};

__host__ __device__ inline long long ceil_div_ll(long long a, long long b) { return (a + b - 1) / b; }

// Order in which a persistent kernel's CTAs take tiles: `per` consecutive
// global tiles at a time, popped from the device counter `head` (dynamic load
// balance over molecules and tiles of uneven cost), or in grid-stride order
// when head is null.
struct TileSched {
    unsigned long long *head;
    int per;
    const int *list;    // optional: the global tiles to process (else every tile)
    const int *list_n;  // device count of `list`
};

// number of queue positions and the global tile at a position
__device__ __forceinline__ long long sched_count(const TileSched &Q, long long n_tiles)
{
    return Q.list ? (long long)*Q.list_n : n_tiles;
}
__device__ __forceinline__ long long sched_tile(const TileSched &Q, long long pos)
{
    return Q.list ? (long long)Q.list[pos] : pos;
}

// first global tile of the CTA's next batch of Q.per tiles (whole block)
__device__ __forceinline__ long long next_tiles(const TileSched &Q, long long &iter, long long *sh)
{
    if (threadIdx.x == 0)
        *sh = Q.head ? (long long)atomicAdd(Q.head, (unsigned long long)Q.per)
                     : ((long long)blockIdx.x + iter * (long long)gridDim.x) * Q.per;
    __syncthreads();
    const long long b = *sh;
    __syncthreads();
    ++iter;
    return b;
}

// The molecule's grid into shared memory, for a whole block working on one of
// its tiles (uniform, cheap reads instead of a struct in registers).  Ends
// with a barrier.
__device__ __forceinline__ void load_grid(const Batch &B, int mol, Grid &sG)
{
    static_assert(sizeof(Grid) % 4 == 0, "Grid copied as words");
    constexpr int W = (int)(sizeof(Grid) / 4);
    const int *src = reinterpret_cast<const int *>(B.grid + mol);
    int *dst = reinterpret_cast<int *>(&sG);
    for (int k = threadIdx.x; k < W; k += blockDim.x) dst[k] = src[k];
    __syncthreads();
}

// molecule owning global tile gt (binary search of the tile offsets)
__device__ __forceinline__ int mol_of_tile(const Batch &B, long long gt)
{
    int lo = 0, hi = B.n_mol;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (B.tile_off[mid] <= gt) lo = mid;
        else hi = mid;
    }
    return lo;
}

}  // namespace eses
