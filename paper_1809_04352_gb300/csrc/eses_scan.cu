// eses_scan.cu -- device-wide exclusive prefix sum of int32 counts.
//
// Reduce-then-scan: chunks of SCAN_CHUNK elements are reduced to partial sums,
// the partials are scanned (recursively when there are many), and every
// chunk is scanned again with its base.  Used for the counting sorts of the
// cell binning, the neighbour/pair/vertex lists and the per-tile edge counts.
#include "eses_kernels.h"

namespace eses {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_CHUNK = SCAN_THREADS * SCAN_ITEMS;

__device__ __forceinline__ int warp_incl_scan(int v)
{
    const unsigned lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= (unsigned)o) v += t;
    }
    return v;
}

// exclusive block scan of one int per thread; returns the block total in *total
__device__ __forceinline__ int block_excl_scan(int v, int *total)
{
    __shared__ int wsum[SCAN_THREADS / 32 + 1];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = warp_incl_scan(v);
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int w = (lane < SCAN_THREADS / 32) ? wsum[lane] : 0;
        int wi = warp_incl_scan(w);
        if (lane < SCAN_THREADS / 32) wsum[lane] = wi - w;
        if (lane == SCAN_THREADS / 32 - 1) wsum[SCAN_THREADS / 32] = wi;  // slot after the last warp
    }
    __syncthreads();
    int res = inc - v + wsum[wid];
    *total = wsum[SCAN_THREADS / 32];
    __syncthreads();
    return res;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan_reduce(const int *__restrict__ in, long long n,
                                                              int *__restrict__ partial)
{
    long long base = (long long)blockIdx.x * SCAN_CHUNK;
    int s = 0;
    for (int i = threadIdx.x; i < SCAN_CHUNK; i += SCAN_THREADS) {
        long long g = base + i;
        if (g < n) s += in[g];
    }
    int tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// scan a chunk with an optional base from `partial` (already exclusive-scanned)
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_down(const int *__restrict__ in, long long n,
                                                            const int *__restrict__ partial, int *__restrict__ out)
{
    long long base = (long long)blockIdx.x * SCAN_CHUNK;
    int v[SCAN_ITEMS];
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        long long g = base + (long long)threadIdx.x * SCAN_ITEMS + k;
        v[k] = (g < n) ? in[g] : 0;
        s += v[k];
    }
    int tot;
    int ex = block_excl_scan(s, &tot);
    int off = (partial ? partial[blockIdx.x] : 0) + ex;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        long long g = base + (long long)threadIdx.x * SCAN_ITEMS + k;
        if (g < n) out[g] = off;
        off += v[k];
    }
    // the thread that owns element n-1 (or the last thread) writes the total
    long long last = n - 1;
    if (last >= base && last < base + SCAN_CHUNK && (last - base) / SCAN_ITEMS == threadIdx.x) out[n] = off;
}

long long scan_tmp_ints(long long n)
{
    long long t = 0;
    while (n > SCAN_CHUNK) {
        long long m = ceil_div_ll(n, SCAN_CHUNK);
        t += 2 * (m + 1);
        n = m;
    }
    return t + 1;
}

int scan_exclusive(const int *in, int *out, long long n, int *tmp, cudaStream_t st)
{
    if (n <= 0) {
        cudaMemsetAsync(out, 0, sizeof(int), st);
        return 0;
    }
    if (n <= SCAN_CHUNK) {
        k_scan_down<<<1, SCAN_THREADS, 0, st>>>(in, n, nullptr, out);
        return 1;
    }
    long long m = ceil_div_ll(n, SCAN_CHUNK);
    int *partial = tmp;
    int *partial_scan = tmp + (m + 1);
    k_scan_reduce<<<(unsigned)m, SCAN_THREADS, 0, st>>>(in, n, partial);
    int nl = scan_exclusive(partial, partial_scan, m, tmp + 2 * (m + 1), st);
    k_scan_down<<<(unsigned)m, SCAN_THREADS, 0, st>>>(in, n, partial_scan, out);
    return nl + 2;
}

}  // namespace eses
