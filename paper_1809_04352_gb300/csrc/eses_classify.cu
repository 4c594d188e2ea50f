// eses_classify.cu -- grid-point classification kernels (the second ESES
// stage, Eq. 2), one CTA per 8x8x8 tile.
//
// k_classify<T, FILT>: stages the tile's atoms and patches in shared memory
// and labels its 512 points.  T = double, FILT = false is the plain FP64
// form; T = float, FILT = true is the filtered form, whose undecided points
// get LABEL_BAND and are counted per tile.  Warp-uniform early outs: a warp
// whose points all lie in no expanded ball, or all inside one van der Waals
// ball, never enters the patch loops.
// k_band: re-labels the undecided points of the tiles that have any, in FP64.
#include "eses_kernels.h"
#include "eses_tile.cuh"

namespace eses {

constexpr int CLS_THREADS = 256;

template <class T, bool FILT>
__global__ void __launch_bounds__(CLS_THREADS) k_classify(Model M, Grid G, int8_t *__restrict__ labels,
                                                          int *__restrict__ tile_band, int *__restrict__ err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileS<T> &S = *reinterpret_cast<TileS<T> *>(smem_raw);
    __shared__ int band;
    for (long long tile = blockIdx.x; tile < G.n_tiles; tile += gridDim.x) {
        double x0[3];
        stage_tile<T>(M, G, tile, S, x0);
        if (threadIdx.x == 0) {
            band = 0;
            if (S.flags) atomicOr(err, S.flags);
        }
        __syncthreads();
        int t[3];
        tile_coords(G, tile, t);
        const T rp = (T)M.rp;
        const T d0 = FILT ? (T)G.d0 : T(0);
        for (int p = threadIdx.x; p < TILE_PTS; p += CLS_THREADS) {
            int li = p >> 6, lj = (p >> 3) & 7, lk = p & 7;
            long long gi = (long long)TILE * t[0] + li, gj = (long long)TILE * t[1] + lj,
                      gk = (long long)TILE * t[2] + lk;
            if (gi >= G.dims[0] || gj >= G.dims[1] || gk >= G.dims[2]) continue;
            T x = (T)((double)li * G.h), y = (T)((double)lj * G.h), z = (T)((double)lk * G.h);
            int lab = classify_pt<T, FILT>(x, y, z, S, rp, rp, d0);
            labels[(gi * G.dims[1] + gj) * G.dims[2] + gk] = (int8_t)lab;
            if (FILT && lab == LABEL_BAND) atomicAdd(&band, 1);
        }
        __syncthreads();
        if (threadIdx.x == 0 && tile_band) tile_band[tile] = band;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(CLS_THREADS) k_band(Model M, Grid G, int8_t *__restrict__ labels,
                                                      const int *__restrict__ tile_band, int *__restrict__ err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileS<double> &S = *reinterpret_cast<TileS<double> *>(smem_raw);
    for (long long tile = blockIdx.x; tile < G.n_tiles; tile += gridDim.x) {
        if (tile_band[tile] == 0) continue;  // uniform across the block
        double x0[3];
        stage_tile<double>(M, G, tile, S, x0);
        if (threadIdx.x == 0 && S.flags) atomicOr(err, S.flags);
        int t[3];
        tile_coords(G, tile, t);
        for (int p = threadIdx.x; p < TILE_PTS; p += CLS_THREADS) {
            int li = p >> 6, lj = (p >> 3) & 7, lk = p & 7;
            long long gi = (long long)TILE * t[0] + li, gj = (long long)TILE * t[1] + lj,
                      gk = (long long)TILE * t[2] + lk;
            if (gi >= G.dims[0] || gj >= G.dims[1] || gk >= G.dims[2]) continue;
            long long idx = (gi * G.dims[1] + gj) * G.dims[2] + gk;
            if (labels[idx] != LABEL_BAND) continue;
            int lab = classify_pt<double, false>((double)li * G.h, (double)lj * G.h, (double)lk * G.h, S, M.rp, M.rp,
                                                 0.0);
            labels[idx] = (int8_t)lab;
        }
        __syncthreads();
    }
}

static int grid_size(long long n_tiles)
{
    long long g = n_tiles < 1 ? 1 : n_tiles;
    return (int)(g > 2147483647LL ? 2147483647LL : g);
}

int launch_classify(const Model &M, const Grid &G, int precision, int8_t *labels, int *tile_band, int *err,
                     cudaStream_t st)
{
    if (precision == 0) {
        size_t sm = sizeof(TileS<double>);
        cudaFuncSetAttribute(k_classify<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_classify<double, false><<<grid_size(G.n_tiles), CLS_THREADS, sm, st>>>(M, G, labels, tile_band, err);
    } else {
        size_t sm = sizeof(TileS<float>);
        cudaFuncSetAttribute(k_classify<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_classify<float, true><<<grid_size(G.n_tiles), CLS_THREADS, sm, st>>>(M, G, labels, tile_band, err);
    }
    return 1;
}

int launch_band(const Model &M, const Grid &G, int8_t *labels, const int *tile_band, int *err, cudaStream_t st)
{
    size_t sm = sizeof(TileS<double>);
    cudaFuncSetAttribute(k_band, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_band<<<grid_size(G.n_tiles), CLS_THREADS, sm, st>>>(M, G, labels, tile_band, err);
    return 1;
}

}  // namespace eses
