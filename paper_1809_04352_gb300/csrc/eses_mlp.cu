// eses_mlp.cu -- the learned tile proposer: per-tile features, the MLP
// 32 -> 64 -> 64 -> 1 (ReLU), its training kernels (forward, backward, Adam)
// and the exact far-tile certificate.
//
// A tile whose labels are all equal (no surface crossing inside it) is "far".
// The proposer scores every tile from cheap atom-density features; a tile it
// scores far is checked by an exact certificate built from nearest-atom
// distance bounds around the tile's centre t (the tile's points lie within
// delta = 3.5 h sqrt(3) of t):
//   all points free (label 0) if  min_i (|t - c_i| - R_i) >= delta
//     (then |x - c_i| >= R_i for every point x and atom i: x is a free probe
//      position, at distance 0 < r_p from the free set);
//   all points inside (label 1) if  max_i (r_i - |t - c_i|) > delta
//     (then every point lies inside van der Waals ball i).
// A certified tile is filled with its label; every other tile (a miss, or a
// tile scored near) goes to the exact classification, so the labels do not
// depend on the network.  Features of a tile (molecule cell grid, cells of
// edge `cell` around the cell holding t):
//   f[0..26]  log(1 + atoms) in the 27 cells around t's cell
//   f[27..29] position of t in its cell, in cell units, minus 1/2
//   f[30]     log(1 + atoms in the 27 cells)
//   f[31]     tile edge (8 h) over the cell edge
#include <math.h>

#include <algorithm>

#include "eses_kernels.h"
#include "eses_mlp_tc.cuh"
#include "eses_tile.cuh"

namespace eses {

constexpr int GRAD_S = 64;        // samples per block of the gradient kernel
constexpr int GRAD_THREADS = 256;
constexpr int PROP_THREADS = 128;  // tiles per block of the proposer kernel

// ---------------------------------------------------------------------------
// MLP forward (FP32), one thread per sample
// ---------------------------------------------------------------------------
__device__ __forceinline__ float mlp_eval(const float *P, const float *x)
{
    float h2[MLP_H];
#pragma unroll
    for (int k = 0; k < MLP_H; ++k) h2[k] = P[P_B2 + k];
    for (int j = 0; j < MLP_H; ++j) {
        float a = P[P_B1 + j];
#pragma unroll
        for (int i = 0; i < MLP_IN; ++i) a = fmaf(x[i], P[P_W1 + i * MLP_H + j], a);
        a = fmaxf(a, 0.0f);
#pragma unroll
        for (int k = 0; k < MLP_H; ++k) h2[k] = fmaf(a, P[P_W2 + j * MLP_H + k], h2[k]);
    }
    float z = P[P_B3];
#pragma unroll
    for (int k = 0; k < MLP_H; ++k) z = fmaf(fmaxf(h2[k], 0.0f), P[P_W3 + k], z);
    return z;
}

__global__ void __launch_bounds__(256) k_mlp_forward(const float *__restrict__ X, int n, const float *__restrict__ Pg,
                                                     float *__restrict__ z)
{
    __shared__ float P[MLP_NPARAM];
    for (int k = threadIdx.x; k < MLP_NPARAM; k += blockDim.x) P[k] = Pg[k];
    __syncthreads();
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    float x[MLP_IN];
#pragma unroll
    for (int i = 0; i < MLP_IN; ++i) x[i] = X[(size_t)s * MLP_IN + i];
    z[s] = mlp_eval(P, x);
}

// ---------------------------------------------------------------------------
// gradient of L = sum_s w_s * BCE(z_s, y_s) (BCE with logits) with respect to
// every parameter; per-block partial sums in fixed order, then a fixed-order
// reduction over blocks (deterministic)
// ---------------------------------------------------------------------------
struct GradSmem {
    float P[MLP_NPARAM];
    float X[GRAD_S][MLP_IN];
    float H1[GRAD_S][MLP_H];
    float H2[GRAD_S][MLP_H];
    float D1[GRAD_S][MLP_H];
    float D2[GRAD_S][MLP_H];
    float dz[GRAD_S];
    float loss[GRAD_S];
};

__global__ void __launch_bounds__(GRAD_THREADS) k_mlp_grad_part(const float *__restrict__ X,
                                                                const float *__restrict__ y,
                                                                const float *__restrict__ w, int n,
                                                                const float *__restrict__ Pg,
                                                                float *__restrict__ part)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GradSmem &G = *reinterpret_cast<GradSmem *>(smem_raw);
    const int tid = threadIdx.x;
    const int s0 = blockIdx.x * GRAD_S;
    const int ns = min(GRAD_S, n - s0);
    for (int k = tid; k < MLP_NPARAM; k += GRAD_THREADS) G.P[k] = Pg[k];
    for (int k = tid; k < GRAD_S * MLP_IN; k += GRAD_THREADS) {
        const int s = k / MLP_IN, i = k % MLP_IN;
        G.X[s][i] = s < ns ? X[(size_t)(s0 + s) * MLP_IN + i] : 0.0f;
    }
    __syncthreads();
    for (int k = tid; k < GRAD_S * MLP_H; k += GRAD_THREADS) {
        const int s = k / MLP_H, j = k % MLP_H;
        float a = G.P[P_B1 + j];
        for (int i = 0; i < MLP_IN; ++i) a = fmaf(G.X[s][i], G.P[P_W1 + i * MLP_H + j], a);
        G.H1[s][j] = fmaxf(a, 0.0f);
    }
    __syncthreads();
    for (int k = tid; k < GRAD_S * MLP_H; k += GRAD_THREADS) {
        const int s = k / MLP_H, j = k % MLP_H;
        float a = G.P[P_B2 + j];
        for (int i = 0; i < MLP_H; ++i) a = fmaf(G.H1[s][i], G.P[P_W2 + i * MLP_H + j], a);
        G.H2[s][j] = fmaxf(a, 0.0f);
    }
    __syncthreads();
    if (tid < GRAD_S) {
        const int s = tid;
        float dz = 0.0f, l = 0.0f;
        if (s < ns) {
            float z = G.P[P_B3];
            for (int k = 0; k < MLP_H; ++k) z = fmaf(G.H2[s][k], G.P[P_W3 + k], z);
            const float yy = y[s0 + s], ww = w[s0 + s];
            const float sg = 1.0f / (1.0f + expf(-z));
            dz = ww * (sg - yy);
            l = ww * (fmaxf(z, 0.0f) - z * yy + log1pf(expf(-fabsf(z))));
        }
        G.dz[s] = dz;
        G.loss[s] = l;
    }
    __syncthreads();
    for (int k = tid; k < GRAD_S * MLP_H; k += GRAD_THREADS) {
        const int s = k / MLP_H, j = k % MLP_H;
        G.D2[s][j] = G.H2[s][j] > 0.0f ? G.dz[s] * G.P[P_W3 + j] : 0.0f;
    }
    __syncthreads();
    for (int k = tid; k < GRAD_S * MLP_H; k += GRAD_THREADS) {
        const int s = k / MLP_H, j = k % MLP_H;
        float a = 0.0f;
        if (G.H1[s][j] > 0.0f)
            for (int q = 0; q < MLP_H; ++q) a = fmaf(G.D2[s][q], G.P[P_W2 + j * MLP_H + q], a);
        G.D1[s][j] = a;
    }
    __syncthreads();
    float *out = part + (size_t)blockIdx.x * (MLP_NPARAM + 1);
    for (int q = tid; q < MLP_NPARAM; q += GRAD_THREADS) {
        float g = 0.0f;
        if (q < P_B1) {
            const int i = q / MLP_H, j = q % MLP_H;
            for (int s = 0; s < GRAD_S; ++s) g = fmaf(G.X[s][i], G.D1[s][j], g);
        } else if (q < P_W2) {
            const int j = q - P_B1;
            for (int s = 0; s < GRAD_S; ++s) g += G.D1[s][j];
        } else if (q < P_B2) {
            const int j = (q - P_W2) / MLP_H, k = (q - P_W2) % MLP_H;
            for (int s = 0; s < GRAD_S; ++s) g = fmaf(G.H1[s][j], G.D2[s][k], g);
        } else if (q < P_W3) {
            const int k = q - P_B2;
            for (int s = 0; s < GRAD_S; ++s) g += G.D2[s][k];
        } else if (q < P_B3) {
            const int k = q - P_W3;
            for (int s = 0; s < GRAD_S; ++s) g = fmaf(G.dz[s], G.H2[s][k], g);
        } else {
            for (int s = 0; s < GRAD_S; ++s) g += G.dz[s];
        }
        out[q] = g;
    }
    if (tid == 0) {
        float l = 0.0f;
        for (int s = 0; s < GRAD_S; ++s) l += G.loss[s];
        out[MLP_NPARAM] = l;
    }
}

__global__ void k_mlp_grad_reduce(const float *__restrict__ part, int nblocks, float *__restrict__ grad,
                                  float *__restrict__ loss)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q > MLP_NPARAM) return;
    float g = 0.0f;
    for (int b = 0; b < nblocks; ++b) g += part[(size_t)b * (MLP_NPARAM + 1) + q];
    if (q < MLP_NPARAM) grad[q] = g;
    else if (loss) *loss = g;
}

__global__ void k_adam(float *__restrict__ P, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= MLP_NPARAM) return;
    const float gq = g[q];
    const float mq = b1 * m[q] + (1.0f - b1) * gq;
    const float vq = b2 * v[q] + (1.0f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    P[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
}

// ---------------------------------------------------------------------------
// tile features, targets, certificate
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tile_centre(const Grid &G, long long tile, double t[3])
{
    int tc[3];
    tile_coords(G, tile, tc);
    for (int a = 0; a < 3; ++a) t[a] = G.lo[a] + G.h * ((double)(TILE * (tc[a] + G.toff[a])) + 0.5 * (TILE - 1));
}

__device__ __forceinline__ long long floor_ll(double v) { return (long long)floor(v); }

__device__ void tile_features(const Model &M, const Grid &G, int mol, long long tile, float *f)
{
    const CellGrid cg = M.cg[mol];
    double t[3];
    tile_centre(G, tile, t);
    long long ci[3];
    for (int a = 0; a < 3; ++a) {
        const double u = (t[a] - cg.clo[a]) / M.cell;
        ci[a] = floor_ll(u);
        f[27 + a] = fminf(fmaxf((float)(u - (double)ci[a]) - 0.5f, -1.5f), 1.5f);
    }
    int tot = 0, k = 0;
    for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dz = -1; dz <= 1; ++dz, ++k) {
                const long long a = ci[0] + dx, b = ci[1] + dy, c = ci[2] + dz;
                int n = 0;
                if (a >= 0 && b >= 0 && c >= 0 && a < cg.cn[0] && b < cg.cn[1] && c < cg.cn[2]) {
                    const int id = cg.coff + (int)((a * cg.cn[1] + b) * cg.cn[2] + c);
                    n = M.cell_start[id + 1] - M.cell_start[id];
                }
                tot += n;
                f[k] = log1pf((float)n);
            }
    f[30] = log1pf((float)tot);
    f[31] = (float)(TILE * G.h / M.cell);
}

__global__ void k_tile_features(Model M, Batch B, float *__restrict__ feat)
{
    for (long long base = (long long)blockIdx.x * blockDim.x; base < B.n_tiles; base += (long long)gridDim.x * blockDim.x) {
        const long long gt = base + threadIdx.x;
        if (gt < B.n_tiles) {
            const int mol = mol_of_tile(B, gt);
            const Grid &G = B.grid[mol];
            float f[MLP_IN];
            tile_features(M, G, mol, gt - G.tile0, f);
            for (int i = 0; i < MLP_IN; ++i) feat[(size_t)gt * MLP_IN + i] = f[i];
        }
    }
}

// 1 when the tile's labels are not all equal (the tile holds surface)
__global__ void k_tile_targets(Batch B, const int8_t *__restrict__ labels_all, uint8_t *__restrict__ target)
{
    const int lane = threadIdx.x & 31;
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long gt = w; gt < B.n_tiles; gt += nw) {
        const int mol = mol_of_tile(B, gt);
        const Grid &G = B.grid[mol];
        const int8_t *labels = labels_all + G.lab0;
        int tc[3];
        tile_coords(G, gt - G.tile0, tc);
        int mn = 127, mx = -128;
        for (int p = lane; p < TILE_PTS; p += 32) {
            const long long g0 = (long long)TILE * tc[0] + (p >> 6), g1 = (long long)TILE * tc[1] + ((p >> 3) & 7),
                            g2 = (long long)TILE * tc[2] + (p & 7);
            if (g0 >= G.dims[0] || g1 >= G.dims[1] || g2 >= G.dims[2]) continue;
            const int v = labels[(g0 * G.dims[1] + g1) * G.dims[2] + g2];
            mn = min(mn, v);
            mx = max(mx, v);
        }
        for (int o = 16; o > 0; o >>= 1) {
            mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (lane == 0) target[gt] = mn != mx ? 1 : 0;
    }
}

// Certificate of one tile (whole warp): 0 all points outside, 1 all inside,
// -1 neither proven.  FP32 on the double-float atom copies (relative to the
// grid origin) and squared distances, with the rounding covered: a squared
// distance carries a relative error below 1e-6, the thresholds get 1e-4 A of
// slack, so a certified answer is exact.
__device__ int certify_tile(const Model &M, const Grid &G, int mol, long long tile)
{
    const int lane = threadIdx.x & 31;
    const CellGrid cg = M.cg[mol];
    int tc[3];
    tile_coords(G, tile, tc);
    float th[3], tl[3];
    int c0[3], c1[3];
    const float delta = (float)(0.5 * (TILE - 1) * G.h * 1.7320508075688772);
    const float slack = 1e-4f, rel_lo = 1.0f - 2e-6f, rel_hi = 1.0f + 2e-6f;
    const float rp = (float)M.rp;
    // every atom that can matter lies within delta + R_max of t: the cells that
    // ball meets, indices in FP32 with 1e-2 A of room for their rounding (no
    // FP64 division: a handful per tile would bound the whole kernel)
    const float icell = 1.0f / (float)M.cell;
    const float reach = (delta + (float)M.Rmax + 1e-2f) * icell;
    for (int a = 0; a < 3; ++a) {
        const double rel = G.h * ((double)(TILE * (tc[a] + G.toff[a])) + 0.5 * (TILE - 1));
        th[a] = (float)rel;
        tl[a] = (float)(rel - (double)th[a]);
        const float u = ((float)(G.lo[a] - cg.clo[a]) + th[a]) * icell;  // centre in cell units
        c0[a] = max((int)floorf(u - reach), 0);
        c1[a] = min((int)floorf(u + reach), cg.cn[a] - 1);
    }
    bool not_out = false, in = false;
    // per (x, y) cell column, the atoms of its z cells are contiguous
    for (int a = c0[0]; a <= c1[0]; ++a)
        for (int b = c0[1]; b <= c1[1]; ++b) {
            if (c0[2] > c1[2]) continue;
            const int id0 = cg.coff + (a * cg.cn[1] + b) * cg.cn[2];
            const int e = M.cell_start[id0 + c1[2] + 1];
            for (int k = M.cell_start[id0 + c0[2]] + lane; k < e; k += 32) {
                const float4 hi = M.atom_hi[k], lo = M.atom_lo[k];
                const float dx = (hi.x - th[0]) + (lo.x - tl[0]);
                const float dy = (hi.y - th[1]) + (lo.y - tl[1]);
                const float dz = (hi.z - th[2]) + (lo.z - tl[2]);
                const float d2 = dx * dx + dy * dy + dz * dz;
                const float to = hi.w + rp + delta + slack;  // outside needs d >= R + delta
                if (d2 * rel_lo < to * to) not_out = true;
                const float ti = hi.w - delta - slack;  // inside needs d < r - delta
                if (ti > 0.0f && d2 * rel_hi < ti * ti) in = true;
            }
        }
    if (!__any_sync(0xffffffffu, not_out)) return 0;
    if (__any_sync(0xffffffffu, in)) return 1;
    return -1;
}

// Proposer: features and tensor-core score per tile (thread per tile, 128
// tiles per CTA step), then the certificate for the tiles scored far (warp
// per tile); certified tiles are filled, the others flagged for the exact
// classification.  mode 1: MLP + certificate; mode 2: certificate on every tile.
__global__ void __launch_bounds__(PROP_THREADS) k_propose(Model M, Batch B, int mode, const float *__restrict__ Pg,
                                                          float z_far, int8_t *__restrict__ labels_all,
                                                          int *__restrict__ tile_band, int *__restrict__ need,
                                                          int *__restrict__ counts, int *__restrict__ err,
                                                          long long wait_limit)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TcSmem &T = *reinterpret_cast<TcSmem *>(smem_raw);
    __shared__ int far_list[PROP_THREADS];
    __shared__ int n_far;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t phase = 0;
    if (mode == 1) tc_setup(T, Pg, wait_limit);
    for (long long base = (long long)blockIdx.x * PROP_THREADS; base < B.n_tiles;
         base += (long long)gridDim.x * PROP_THREADS) {
        if (threadIdx.x == 0) n_far = 0;
        __syncthreads();
        const long long gt = base + threadIdx.x;
        const bool valid = gt < B.n_tiles;
        bool far = valid;
        if (mode == 1) {
            float f[MLP_IN];
            if (valid) {
                const int mol = mol_of_tile(B, gt);
                const Grid &G = B.grid[mol];
                tile_features(M, G, mol, gt - G.tile0, f);
            }
            const float zt = tc_score(T, f, valid, phase, err);  // every thread: block-wide barriers inside
            far = valid && zt < z_far;
        }
        if (valid) need[gt] = 1;
        if (far) far_list[atomicAdd(&n_far, 1)] = (int)threadIdx.x;
        __syncthreads();
        const int nf = n_far;
        for (int k = warp; k < nf; k += PROP_THREADS / 32) {
            const long long g2 = base + far_list[k];
            const int mol = mol_of_tile(B, g2);
            const Grid &G = B.grid[mol];
            const long long tile = g2 - G.tile0;
            const int r = certify_tile(M, G, mol, tile);
            if (r >= 0) {
                int8_t *labels = labels_all + G.lab0;
                int tc[3];
                tile_coords(G, tile, tc);
                for (int p = lane; p < TILE_PTS; p += 32) {
                    const long long g0 = (long long)TILE * tc[0] + (p >> 6),
                                    g1 = (long long)TILE * tc[1] + ((p >> 3) & 7), gz = (long long)TILE * tc[2] + (p & 7);
                    if (g0 < G.dims[0] && g1 < G.dims[1] && gz < G.dims[2])
                        labels[(g0 * G.dims[1] + g1) * G.dims[2] + gz] = (int8_t)r;
                }
                if (lane == 0) {
                    need[g2] = 0;
                    if (tile_band) tile_band[g2] = 0;
                }
            }
            if (lane == 0) {
                atomicAdd(&counts[0], 1);                // tiles proposed far
                if (r >= 0) atomicAdd(&counts[1], 1);    // certified
            }
        }
        __syncthreads();
    }
    if (mode == 1) tc_teardown(T, phase);
}

// The tensor-core MLP on arbitrary rows (n x 32 features): z = MLP(X), BF16
// weights and activations, FP32 accumulation (the proposer's scoring path).
__global__ void __launch_bounds__(PROP_THREADS) k_mlp_forward_tc(const float *__restrict__ X, int n,
                                                                 const float *__restrict__ Pg, float *__restrict__ z,
                                                                 int *__restrict__ err)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TcSmem &T = *reinterpret_cast<TcSmem *>(smem_raw);
    uint32_t phase = 0;
    tc_setup(T, Pg);
    for (long long base = (long long)blockIdx.x * PROP_THREADS; base < n; base += (long long)gridDim.x * PROP_THREADS) {
        const long long s = base + threadIdx.x;
        const bool valid = s < n;
        float x[MLP_IN];
#pragma unroll
        for (int i = 0; i < MLP_IN; ++i) x[i] = valid ? X[s * MLP_IN + i] : 0.0f;
        const float v = tc_score(T, x, valid, phase, err);
        if (valid) z[s] = v;
    }
    tc_teardown(T, phase);
}

// list of the tiles flagged in `need`, from their exclusive scan
__global__ void k_compact(long long n, const int *__restrict__ need, const int *__restrict__ pos,
                          int *__restrict__ list)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && need[i]) list[pos[i]] = (int)i;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static size_t grad_smem() { return sizeof(GradSmem); }

void mlp_init()
{
    cudaFuncSetAttribute(k_mlp_grad_part, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem());
    cudaFuncSetAttribute(k_propose, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TcSmem));
    cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TcSmem));
}

int launch_mlp_forward(const float *X, int n, const float *P, float *z, cudaStream_t st)
{
    if (n <= 0) return 0;
    k_mlp_forward<<<(n + 255) / 256, 256, 0, st>>>(X, n, P, z);
    return 1;
}

long long mlp_grad_scratch(int n) { return (long long)((n + GRAD_S - 1) / GRAD_S) * (MLP_NPARAM + 1); }

int launch_mlp_grad(const float *X, const float *y, const float *w, int n, const float *P, float *part, float *grad,
                    float *loss, cudaStream_t st)
{
    if (n <= 0) return 0;
    const int nb = (n + GRAD_S - 1) / GRAD_S;
    k_mlp_grad_part<<<nb, GRAD_THREADS, grad_smem(), st>>>(X, y, w, n, P, part);
    k_mlp_grad_reduce<<<(MLP_NPARAM + 1 + 255) / 256, 256, 0, st>>>(part, nb, grad, loss);
    return 2;
}

int launch_adam(float *P, const float *g, float *m, float *v, int step, float lr, cudaStream_t st)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    k_adam<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(P, g, m, v, lr, b1, b2, eps, c1, c2);
    return 1;
}

int launch_tile_features(const Model &M, const Batch &B, float *feat, cudaStream_t st)
{
    const long long g = std::min<long long>((B.n_tiles + 127) / 128, 1 << 20);
    k_tile_features<<<(unsigned)std::max(g, 1LL), 128, 0, st>>>(M, B, feat);
    return 1;
}

int launch_tile_targets(const Batch &B, const int8_t *labels, uint8_t *target, cudaStream_t st)
{
    const long long g = std::min<long long>((B.n_tiles + 7) / 8, 1 << 20);
    k_tile_targets<<<(unsigned)std::max(g, 1LL), 256, 0, st>>>(B, labels, target);
    return 1;
}

// persistent grids: at most 4 CTAs per SM, so every CTA's 128 TMEM columns fit (512 per SM)
static int tc_grid(long long rows)
{
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long need = (rows + PROP_THREADS - 1) / PROP_THREADS;
    return (int)std::max(1LL, std::min(need, 4LL * nsm));
}

int launch_propose(const Model &M, const Batch &B, int mode, const float *P, float z_far, int8_t *labels,
                   int *tile_band, int *need, int *counts, int *err, long long wait_limit, cudaStream_t st)
{
    k_propose<<<tc_grid(B.n_tiles), PROP_THREADS, sizeof(TcSmem), st>>>(M, B, mode, P, z_far, labels, tile_band, need,
                                                                       counts, err, wait_limit);
    return 1;
}

int launch_mlp_forward_tc(const float *X, int n, const float *P, float *z, int *err, cudaStream_t st)
{
    if (n <= 0) return 0;
    k_mlp_forward_tc<<<tc_grid(n), PROP_THREADS, sizeof(TcSmem), st>>>(X, n, P, z, err);
    return 1;
}

int launch_compact(long long n, const int *need, const int *pos, int *list, cudaStream_t st)
{
    if (n <= 0) return 0;
    k_compact<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, need, pos, list);
    return 1;
}

}  // namespace eses
