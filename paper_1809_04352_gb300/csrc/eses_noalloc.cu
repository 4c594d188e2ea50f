// eses_noalloc.cu -- crossing-edge extraction that allocates no memory.
//
// eses_crossing_edges_noalloc() lists, for each axis, the lower point of every
// grid edge whose two end labels differ, in the same order as
// eses_intersections() (8x8x8 tiles in C order, then lower index).  It is for
// callers that cannot call cudaMalloc: code whose device memory is owned by a
// framework allocator or a fixed budget, or work issued where an allocation
// call is not allowed.  The caller passes the labels and the output arrays;
// the per-tile counts and offsets it needs live in one file-scope __device__
// array of NAL_MAX_TILES tiles, which every GPU that loads the library holds
// until the process exits.
//
// The first call on a device looks up that array's device address with
// cudaGetSymbolAddress (with the device current) and caches it; make that
// first call before any stream capture.  The cached address belongs to the
// device's current context: after cudaDeviceReset the process must not call
// this entry point again on that device.  Every call reuses the same array and
// leaves its contents behind; each call rewrites every entry it reads, so no
// state carries over, but two calls that overlap on the GPU (different
// streams, or one launched before the previous has finished on another
// stream) race on the array.
#include <mutex>

#include "../../include/eses.h"
#include "eses_internal.cuh"

namespace eses {

constexpr long long NAL_MAX_TILES = 1LL << 17;  // 131,072 tiles = 67,108,864 points
constexpr int NAL_THREADS = 256;
// layout: counts [3][NAL_MAX_TILES], offsets [3 * NAL_MAX_TILES + 1]
constexpr long long NAL_SCRATCH_INTS = 6 * NAL_MAX_TILES + 1;
// k_nal_write gives each thread points 2*tid and 2*tid+1, and nal_flag splits a local point index
// into (p >> 6, (p >> 3) & 7, p & 7): both hold for 8x8x8 tiles only
static_assert(TILE == 8 && TILE_PTS == 2 * NAL_THREADS, "noalloc kernels assume 8^3 tiles and 256 threads");

static __device__ __align__(256) int g_nal_scratch[NAL_SCRATCH_INTS];

struct NalGrid {
    long long dims[3];
    int tiles[3];
    long long nt;
};

__device__ __forceinline__ void nal_tile(const NalGrid &G, long long tile, int t[3])
{
    t[2] = (int)(tile % G.tiles[2]);
    t[1] = (int)((tile / G.tiles[2]) % G.tiles[1]);
    t[0] = (int)(tile / ((long long)G.tiles[1] * G.tiles[2]));
}

// 1 if the edge (p, p + e_a) crosses; local point p = (li, lj, lk)
__device__ __forceinline__ int nal_flag(const NalGrid &G, const int8_t *labels, const int t[3], int p, int a,
                                        long long *gidx)
{
    long long g[3] = {(long long)TILE * t[0] + (p >> 6), (long long)TILE * t[1] + ((p >> 3) & 7),
                      (long long)TILE * t[2] + (p & 7)};
    if (g[0] >= G.dims[0] || g[1] >= G.dims[1] || g[2] >= G.dims[2]) return 0;
    if (g[a] + 1 >= G.dims[a]) return 0;
    const long long str[3] = {G.dims[1] * G.dims[2], G.dims[2], 1};
    long long idx = g[0] * str[0] + g[1] * str[1] + g[2];
    *gidx = idx;
    return labels[idx] != labels[idx + str[a]] ? 1 : 0;
}

__device__ __forceinline__ int nal_block_excl(int v, int *sh, int *total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    __syncthreads();
    if (lane == 31) sh[wid] = inc;
    __syncthreads();
    int base = 0, tot = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
        if (k < wid) base += sh[k];
        tot += sh[k];
    }
    __syncthreads();
    *total = tot;
    return base + inc - v;
}

// per tile and axis: number of crossing edges -> counts[a * max + tile]
__global__ void __launch_bounds__(NAL_THREADS) k_nal_count(NalGrid G, const int8_t *__restrict__ labels,
                                                           int *__restrict__ scratch)
{
    __shared__ int sh[NAL_THREADS / 32];
    for (long long tile = blockIdx.x; tile < G.nt; tile += gridDim.x) {
        int t[3];
        nal_tile(G, tile, t);
        for (int a = 0; a < 3; ++a) {
            int c = 0;
            long long gi;
            for (int p = threadIdx.x; p < TILE_PTS; p += NAL_THREADS) c += nal_flag(G, labels, t, p, a, &gi);
            int tot;
            nal_block_excl(c, sh, &tot);
            if (threadIdx.x == 0) scratch[a * NAL_MAX_TILES + tile] = tot;
        }
    }
}

// one block: exclusive scan of the 3 * nt counts (axis-major) into the offsets
__global__ void __launch_bounds__(1024) k_nal_scan(long long nt, int *__restrict__ scratch)
{
    __shared__ int sh[32];
    int *counts = scratch;
    int *offs = scratch + 3 * NAL_MAX_TILES;
    const long long n = 3 * nt;
    const long long per = (n + blockDim.x - 1) / blockDim.x;
    const long long b = (long long)threadIdx.x * per;
    int s = 0;
    for (long long k = b; k < b + per && k < n; ++k) s += counts[(k / nt) * NAL_MAX_TILES + (k % nt)];
    int tot;
    int run = nal_block_excl(s, sh, &tot);
    for (long long k = b; k < b + per && k < n; ++k) {
        offs[k] = run;
        run += counts[(k / nt) * NAL_MAX_TILES + (k % nt)];
    }
    if (threadIdx.x == 0) offs[n] = tot;
}

// per tile: write the lower indices at the tile's offset, in point order
__global__ void __launch_bounds__(NAL_THREADS) k_nal_write(NalGrid G, const int8_t *__restrict__ labels,
                                                           const int *__restrict__ scratch, long long *out0,
                                                           long long *out1, long long *out2, long long cap0,
                                                           long long cap1, long long cap2)
{
    __shared__ int sh[NAL_THREADS / 32];
    const int *offs = scratch + 3 * NAL_MAX_TILES;
    long long *outs[3] = {out0, out1, out2};
    const long long caps[3] = {cap0, cap1, cap2};
    for (long long tile = blockIdx.x; tile < G.nt; tile += gridDim.x) {
        int t[3];
        nal_tile(G, tile, t);
        for (int a = 0; a < 3; ++a) {
            const long long base = (long long)offs[a * G.nt + tile] - offs[a * G.nt];
            long long g0 = 0, g1 = 0;
            int f0 = nal_flag(G, labels, t, 2 * threadIdx.x, a, &g0);
            int f1 = nal_flag(G, labels, t, 2 * threadIdx.x + 1, a, &g1);
            int tot;
            long long r = base + nal_block_excl(f0 + f1, sh, &tot);
            if (f0) {
                if (r < caps[a]) outs[a][r] = g0;
                ++r;
            }
            if (f1 && r < caps[a]) outs[a][r] = g1;
        }
    }
}

static std::mutex g_nal_mutex;
static int *g_nal_ptr[64] = {nullptr};

}  // namespace eses

using namespace eses;

extern "C" int eses_crossing_edges_noalloc(const int8_t *labels, const int64_t dims[3], int64_t *idx0, int64_t *idx1,
                                           int64_t *idx2, const int64_t capacity[3], int64_t counts[3], void *stream)
{
    if (!labels || !dims || !capacity || !counts || !idx0 || !idx1 || !idx2) return ESES_EINVAL;
    NalGrid G;
    G.nt = 1;
    for (int a = 0; a < 3; ++a) {
        if (dims[a] < 1 || capacity[a] < 0) return ESES_EINVAL;
        G.dims[a] = dims[a];
        // tile count in 64 bits, compared before it is narrowed (a wrapped int would pass the check)
        const long long ta = (dims[a] - 1) / TILE + 1;
        if (ta > NAL_MAX_TILES) return ESES_EINVAL;
        G.tiles[a] = (int)ta;
        G.nt *= ta;
        if (G.nt > NAL_MAX_TILES) return ESES_EINVAL;  // grid larger than the scratch array covers
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return ESES_ECUDA;
    int *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_nal_mutex);
        if (!g_nal_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_nal_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return ESES_ECUDA;
            }
            g_nal_ptr[dev] = (int *)p;
        }
        scratch = g_nal_ptr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    int grid = (int)(G.nt < 65535 * 16 ? G.nt : 65535 * 16);
    k_nal_count<<<grid, NAL_THREADS, 0, st>>>(G, labels, scratch);
    k_nal_scan<<<1, 1024, 0, st>>>(G.nt, scratch);
    k_nal_write<<<grid, NAL_THREADS, 0, st>>>(G, labels, scratch, (long long *)idx0, (long long *)idx1,
                                              (long long *)idx2, capacity[0], capacity[1], capacity[2]);
    int tot[4] = {0, 0, 0, 0};
    const int *offs = scratch + 3 * NAL_MAX_TILES;
    bool ok = cudaGetLastError() == cudaSuccess;
    for (int a = 0; a < 3 && ok; ++a)
        ok = cudaMemcpyAsync(&tot[a], offs + a * G.nt, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess;
    if (ok) ok = cudaMemcpyAsync(&tot[3], offs + 3 * G.nt, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess;
    if (ok) ok = cudaStreamSynchronize(st) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        return ESES_ECUDA;
    }
    int over = 0;
    for (int a = 0; a < 3; ++a) {
        counts[a] = (int64_t)tot[a + 1] - tot[a];
        if (counts[a] > capacity[a]) over = 1;
    }
    return over ? ESES_ECAPACITY : ESES_OK;
}
