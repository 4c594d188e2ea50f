// eses_exterior.cu -- exterior-only surface (cavities filled).
//
// §1 counts every free probe position as solvent; the exterior-only variant
// keeps only the solvent a probe can reach from outside the molecule.  On the
// grid (reading X1): an outside point is exterior iff a path of outside
// points, each step between 6-neighbours, joins it to the domain boundary
// (whose points are all outside, reading C2); every other outside point is in
// a cavity and becomes inside.  The crossing edges, roots and area/volume are
// then computed from the relabelled grid by the usual stages.
//
// State per point (one byte): 0 inside, 1 outside not reached yet, 2 reached.
//   k_ext_init:  boundary outside points reached, other outside points 1;
//                a tile is open while it holds points in state 1;
//   k_ext_sweep: per 8x8x8 tile with a one-point halo in shared memory, the
//                reached set grows inside the tile until it stops (a bounded
//                loop: a path inside the tile has fewer than 512 steps); the
//                tile's new points are written back and a flag set; a
//                tile left without state-1 points closes and is not read
//                again.  Sweeps repeat until one changes nothing (the
//                reached set only grows, so neighbours read mid-sweep are
//                either state and the fixed point is the same): k_ext_fill
//                runs them all in one cooperative launch with a grid-wide
//                barrier after each sweep (k_ext_sweep, one sweep per launch
//                driven from the host, where cooperative launch is missing);
//   k_ext_apply: points still 1 are cavity points: label 1, counted.
#include <cooperative_groups.h>

#include "eses_kernels.h"
#include "eses_tile.cuh"

namespace eses {

constexpr int EXT_WARPS = 8;
constexpr int EXT_THREADS = 256;
constexpr int HALO_W = TILE + 2;  // 10 points per axis

// the tile's points: warp per tile, 16 points per lane
__global__ void __launch_bounds__(EXT_WARPS * 32) k_ext_init(Batch B, const int8_t *__restrict__ labels_all,
                                                            uint8_t *__restrict__ ext_all,
                                                            uint8_t *__restrict__ tile_open)
{
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * EXT_WARPS;
    for (long long gt = (long long)blockIdx.x * EXT_WARPS + (threadIdx.x >> 5); gt < B.n_tiles; gt += nw) {
        const Grid &G = B.grid[mol_of_tile(B, gt)];
        const long long d[3] = {G.dims[0], G.dims[1], G.dims[2]};
        int t[3];
        tile_coords(G, gt - G.tile0, t);
        bool open = false;
        for (int p = lane; p < TILE_PTS; p += 32) {
            const long long g[3] = {(long long)TILE * t[0] + (p >> 6), (long long)TILE * t[1] + ((p >> 3) & 7),
                                    (long long)TILE * t[2] + (p & 7)};
            if (g[0] >= d[0] || g[1] >= d[1] || g[2] >= d[2]) continue;
            const long long idx = G.lab0 + (g[0] * d[1] + g[1]) * d[2] + g[2];
            const bool face = g[0] == 0 || g[1] == 0 || g[2] == 0 || g[0] == d[0] - 1 || g[1] == d[1] - 1 ||
                              g[2] == d[2] - 1;
            const uint8_t v = labels_all[idx] != 0 ? 0 : (face ? 2 : 1);
            ext_all[idx] = v;
            open = open || v == 1;
        }
        open = __any_sync(0xffffffffu, open);
        if (lane == 0) tile_open[gt] = open ? 1 : 0;
    }
}

// one sweep over the block's tiles gt = blockIdx.x, + gridDim.x, ... (whole block)
__device__ void sweep_tiles(const Batch &B, uint8_t *__restrict__ ext_all, uint8_t *__restrict__ tile_open,
                            int *__restrict__ changed, uint8_t *s, uint8_t *s0)
{
    for (long long gt = blockIdx.x; gt < B.n_tiles; gt += gridDim.x) {
        if (!tile_open[gt]) continue;  // uniform: every thread reads the same byte
        const Grid &G = B.grid[mol_of_tile(B, gt)];
        const long long d[3] = {G.dims[0], G.dims[1], G.dims[2]};
        int t[3];
        tile_coords(G, gt - G.tile0, t);
        uint8_t *ext = ext_all + G.lab0;
        // the tile and its halo; points off the grid are walls
        bool open = false;
        for (int q = threadIdx.x; q < HALO_W * HALO_W * HALO_W; q += EXT_THREADS) {
            const int li = q / (HALO_W * HALO_W) - 1, lj = (q / HALO_W) % HALO_W - 1, lk = q % HALO_W - 1;
            const long long g[3] = {(long long)TILE * t[0] + li, (long long)TILE * t[1] + lj,
                                    (long long)TILE * t[2] + lk};
            uint8_t v = 0;
            if (g[0] >= 0 && g[1] >= 0 && g[2] >= 0 && g[0] < d[0] && g[1] < d[1] && g[2] < d[2])
                v = *(volatile const uint8_t *)&ext[(g[0] * d[1] + g[1]) * d[2] + g[2]];
            s[q] = v;
            const bool mine = li >= 0 && lj >= 0 && lk >= 0 && li < TILE && lj < TILE && lk < TILE;
            if (mine) {
                s0[(li * TILE + lj) * TILE + lk] = v;
                if (v == 1) open = true;
            }
        }
        if (!__syncthreads_or(open)) {  // nothing left to reach in this tile
            if (threadIdx.x == 0) tile_open[gt] = 0;
            continue;
        }
        // grow the reached set inside the tile until it stops
        for (int it = 0; it < TILE_PTS; ++it) {
            bool grew = false;
            for (int p = threadIdx.x; p < TILE_PTS; p += EXT_THREADS) {
                const int li = p >> 6, lj = (p >> 3) & 7, lk = p & 7;
                const int q = ((li + 1) * HALO_W + (lj + 1)) * HALO_W + (lk + 1);
                if (s[q] != 1) continue;
                if (s[q - 1] == 2 || s[q + 1] == 2 || s[q - HALO_W] == 2 || s[q + HALO_W] == 2 ||
                    s[q - HALO_W * HALO_W] == 2 || s[q + HALO_W * HALO_W] == 2) {
                    s[q] = 2;
                    grew = true;
                }
            }
            if (!__syncthreads_or(grew)) break;
        }
        bool any = false, left = false;
        for (int p = threadIdx.x; p < TILE_PTS; p += EXT_THREADS) {
            const int li = p >> 6, lj = (p >> 3) & 7, lk = p & 7;
            const int q = ((li + 1) * HALO_W + (lj + 1)) * HALO_W + (lk + 1);
            left = left || s[q] == 1;
            if (s[q] == 2 && s0[p] == 1) {
                const long long g[3] = {(long long)TILE * t[0] + li, (long long)TILE * t[1] + lj,
                                        (long long)TILE * t[2] + lk};
                ext[(g[0] * d[1] + g[1]) * d[2] + g[2]] = 2;
                any = true;
            }
        }
        left = __syncthreads_or(left);
        if (__syncthreads_or(any) && threadIdx.x == 0) atomicExch(changed, 1);
        if (!left && threadIdx.x == 0) tile_open[gt] = 0;
    }
}

__global__ void __launch_bounds__(EXT_THREADS) k_ext_sweep(Batch B, uint8_t *__restrict__ ext_all,
                                                          uint8_t *__restrict__ tile_open, int *__restrict__ changed)
{
    __shared__ uint8_t s[HALO_W * HALO_W * HALO_W];
    __shared__ uint8_t s0[TILE_PTS];  // the tile's states before the sweep
    sweep_tiles(B, ext_all, tile_open, changed, s, s0);
}

// Every sweep in one cooperative launch (all blocks resident): after each
// sweep a grid-wide barrier, then every block reads that sweep's changed flag
// and all stop together when it is clear.  Three flags rotate: block 0 clears
// the next sweep's flag, which every block last read before the previous
// barrier.  At most max_sweeps sweeps (the host loop's bound); flags[3]
// receives the number of sweeps run.
__global__ void __launch_bounds__(EXT_THREADS) k_ext_fill(Batch B, uint8_t *__restrict__ ext_all,
                                                         uint8_t *__restrict__ tile_open, int *__restrict__ flags,
                                                         long long max_sweeps)
{
    __shared__ uint8_t s[HALO_W * HALO_W * HALO_W];
    __shared__ uint8_t s0[TILE_PTS];
    cooperative_groups::grid_group grid = cooperative_groups::this_grid();
    long long it = 0;
    for (; it < max_sweeps; ++it) {
        if (blockIdx.x == 0 && threadIdx.x == 0) flags[(it + 1) % 3] = 0;
        sweep_tiles(B, ext_all, tile_open, &flags[it % 3], s, s0);
        grid.sync();
        if (*(volatile int *)&flags[it % 3] == 0) break;  // the same value in every block
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) flags[3] = (int)(it < max_sweeps ? it + 1 : it);
}

__global__ void __launch_bounds__(EXT_WARPS * 32) k_ext_apply(Batch B, int8_t *__restrict__ labels_all,
                                                             const uint8_t *__restrict__ ext_all,
                                                             unsigned long long *__restrict__ filled)
{
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * EXT_WARPS;
    unsigned long long n = 0;
    for (long long gt = (long long)blockIdx.x * EXT_WARPS + (threadIdx.x >> 5); gt < B.n_tiles; gt += nw) {
        const Grid &G = B.grid[mol_of_tile(B, gt)];
        const long long d[3] = {G.dims[0], G.dims[1], G.dims[2]};
        int t[3];
        tile_coords(G, gt - G.tile0, t);
        for (int p = lane; p < TILE_PTS; p += 32) {
            const long long g[3] = {(long long)TILE * t[0] + (p >> 6), (long long)TILE * t[1] + ((p >> 3) & 7),
                                    (long long)TILE * t[2] + (p & 7)};
            if (g[0] >= d[0] || g[1] >= d[1] || g[2] >= d[2]) continue;
            const long long idx = G.lab0 + (g[0] * d[1] + g[1]) * d[2] + g[2];
            if (ext_all[idx] == 1) {
                labels_all[idx] = LABEL_IN;
                ++n;
            }
        }
    }
    n = __reduce_add_sync(0xffffffffu, (unsigned)n);
    if (lane == 0 && n) atomicAdd(filled, n);
}

static int warp_grid(long long n_tiles)
{
    const long long g = (n_tiles + EXT_WARPS - 1) / EXT_WARPS;
    return (int)(g < 1 ? 1 : (g > 1048576 ? 1048576 : g));
}

int launch_ext_init(const Batch &B, const int8_t *labels, uint8_t *ext, uint8_t *tile_open, cudaStream_t st)
{
    k_ext_init<<<warp_grid(B.n_tiles), EXT_WARPS * 32, 0, st>>>(B, labels, ext, tile_open);
    return 1;
}

int launch_ext_sweep(const Batch &B, uint8_t *ext, uint8_t *tile_open, int *changed, int grid, cudaStream_t st)
{
    k_ext_sweep<<<grid < 1 ? 1 : grid, EXT_THREADS, 0, st>>>(B, ext, tile_open, changed);
    return 1;
}

// all sweeps in one cooperative launch; returns 0 when the device cannot
// launch cooperatively (the caller then drives k_ext_sweep from the host)
int launch_ext_fill(const Batch &B, uint8_t *ext, uint8_t *tile_open, int *flags, long long max_sweeps,
                    cudaStream_t st)
{
    int dev = 0, coop = 0, n_sm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return 0;
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ext_fill, EXT_THREADS, 0);
    if (per_sm < 1) return 0;
    long long grid = (long long)per_sm * n_sm;
    if (grid > B.n_tiles) grid = B.n_tiles < 1 ? 1 : B.n_tiles;
    Batch b = B;
    void *args[] = {&b, &ext, &tile_open, &flags, &max_sweeps};
    if (cudaLaunchCooperativeKernel((void *)k_ext_fill, dim3((unsigned)grid), dim3(EXT_THREADS), args, 0, st) !=
        cudaSuccess)
        return -1;
    return 1;
}

int launch_ext_apply(const Batch &B, int8_t *labels, const uint8_t *ext, unsigned long long *filled, cudaStream_t st)
{
    k_ext_apply<<<warp_grid(B.n_tiles), EXT_WARPS * 32, 0, st>>>(B, labels, ext, filled);
    return 1;
}

}  // namespace eses
