// eses_tile.cuh -- tile staging and point classification (device code).
//
// A tile is 8x8x8 grid points.  Its "region" is the box [x0, x0 + 8h]^3,
// which holds the tile's points and the first points of the next tiles, so
// the edges leaving the tile in + directions lie inside it.  Staged into
// shared memory, in coordinates relative to x0 (FP64 differences, then
// rounded to the working type):
//   atoms     with dist(c, region) < r + 2 r_p  (§2.2 locality radius; the
//             paper's r_p + r_max is too small -- an atom within r + 2 r_p
//             of x can cover a probe centre that would reach x)
//   pairs     with a free arc and dist(o, region) < rho + r_p
//   vertices  free triple points with dist(v, region) < r_p
// Every staged item keeps its index in the model, so exact FP64 values in
// the same tile frame can be fetched from HBM (ExactAcc) when an FP32 test
// is undecided.
//
// Classification of a point x (Eq. 2): x is outside M iff some free probe
// centre lies at distance < r_p.  The nearest free point, when it is that
// close, is the radial projection on a containing expanded sphere (convex
// patch), the nearest point of a pair circle (saddle) -- and then x lies in
// one of the pair's two expanded balls, since x is in the triangle of the two
// centres and that point -- or a free triple point (concave); each candidate
// counts only if it is free.  Inside a van der Waals ball x is always in M;
// outside every expanded ball x is free.
//
// FP32 filtering: every comparison of a computed squared distance with a
// threshold t^2 is accepted only if it clears an error bound
//     e = 2 ((2 t + delta) delta + 1e-6 t^2)
// where delta bounds the error of the compared vector (positions staged in
// FP32 carry at most d0, derived points carry the propagated error).  A
// comparison inside the band leaves the point undecided; undecided points
// are re-evaluated by the same code in FP64.
#pragma once

#include <math.h>

#include "eses_internal.cuh"

namespace eses {

template <class T>
struct alignas(16) P4 {
    T x, y, z, w;
};

constexpr int STAGE_CELLS = 128;  // cells staged with item-parallel scan (else one thread per cell)
// words of a set of staged atoms (bit k: staged slot k) for capacity C
template <class C>
__host__ __device__ constexpr int atom_words() { return (C::A + 31) / 32; }

template <class T, class C = CapSmall>
struct TileS {
    P4<T> atom[C::A];       // centre (tile frame), vdW radius
    P4<T> po[C::P];         // circle centre (tile frame), rho
    P4<T> pu[C::P];         // circle axis
    P4<T> vq[C::V];         // free triple point (tile frame)
    int agid[C::A];         // sorted atom index
    int2 pij[C::P];         // sorted atom indices of the pair
    int pidx[C::P];         // pair index in the model
    int vidx[C::V];         // triple point index in the model
    uint8_t aface[C::A];    // expanded sphere keeps a free face
    int cid[STAGE_CELLS];           // cells of the staging range
    int cs[3][STAGE_CELLS + 1];     // prefix of their atoms / pairs / vertices
    double fx0[3], fx1[3];          // tile region (absolute), computed once per tile
    float fh0[3], fl0[3];           // region origin in the grid frame, double-float
    int fc0[3], fc1[3];             // cell range of the region plus halo
    int na, np, nv, flags;
};

// ---------------------------------------------------------------------------
// accessors: staged (shared memory) or exact (FP64 from HBM, same tile frame)
// ---------------------------------------------------------------------------
template <class T, class C = CapSmall>
struct SmemAcc {
    using real = T;
    const TileS<T, C> &S;
    __device__ SmemAcc(const TileS<T, C> &s) : S(s) {}
    __device__ int na() const { return S.na; }
    __device__ int np() const { return S.np; }
    __device__ int nv() const { return S.nv; }
    __device__ P4<T> atom(int a) const { return S.atom[a]; }
    __device__ int agid(int a) const { return S.agid[a]; }
    __device__ bool face(int a) const { return S.aface[a] != 0; }
    __device__ P4<T> po(int p) const { return S.po[p]; }
    __device__ P4<T> pu(int p) const { return S.pu[p]; }
    __device__ int2 pij(int p) const { return S.pij[p]; }
    __device__ P4<T> vq(int v) const { return S.vq[v]; }
};

template <class TS, class C = CapSmall>
struct ExactAcc {
    using real = double;
    const TileS<TS, C> &S;
    const Model &M;
    double x0, y0, z0;
    __device__ ExactAcc(const TileS<TS, C> &s, const Model &m, const double *o)
        : S(s), M(m), x0(o[0]), y0(o[1]), z0(o[2]) {}
    __device__ int na() const { return S.na; }
    __device__ int np() const { return S.np; }
    __device__ int nv() const { return S.nv; }
    __device__ P4<double> atom(int a) const
    {
        double4 g = M.atom[S.agid[a]];
        return P4<double>{g.x - x0, g.y - y0, g.z - z0, g.w};
    }
    __device__ int agid(int a) const { return S.agid[a]; }
    __device__ bool face(int a) const { return S.aface[a] != 0; }
    __device__ P4<double> po(int p) const
    {
        double4 g = M.pair_o[S.pidx[p]];
        return P4<double>{g.x - x0, g.y - y0, g.z - z0, g.w};
    }
    __device__ P4<double> pu(int p) const
    {
        double4 g = M.pair_u[S.pidx[p]];
        return P4<double>{g.x, g.y, g.z, 0.0};
    }
    __device__ int2 pij(int p) const { return S.pij[p]; }
    __device__ P4<double> vq(int v) const
    {
        double4 g = M.vert[S.vidx[v]];
        return P4<double>{g.x - x0, g.y - y0, g.z - z0, 0.0};
    }
};

__device__ __forceinline__ double box_dist2(double x, double y, double z, const double *b0, const double *b1)
{
    double ex = x < b0[0] ? b0[0] - x : (x > b1[0] ? x - b1[0] : 0.0);
    double ey = y < b0[1] ? b0[1] - y : (y > b1[1] ? y - b1[1] : 0.0);
    double ez = z < b0[2] ? b0[2] - z : (z > b1[2] ? z - b1[2] : 0.0);
    return ex * ex + ey * ey + ez * ez;
}

// tile index within its molecule -> tile coordinates (fewer than 2^31 tiles
// per molecule, checked at create: 32-bit division)
__device__ __forceinline__ void tile_coords(const Grid &G, long long tile, int t[3])
{
    const unsigned tt = (unsigned)tile, n2 = (unsigned)G.tiles[2], n1 = (unsigned)G.tiles[1];
    const unsigned q = tt / n2;
    t[2] = (int)(tt - q * n2);
    t[1] = (int)(q % n1);
    t[0] = (int)(q / n1);
}

// Test one cell item against the region and append it (atoms, pairs, vertices).
// FP64 staging: FP64 box test, FP64 difference to the tile origin, rounded
// once.  FP32 staging: the double-float copies (hi + lo, grid frame); the box
// test uses hi with a 1e-3 A margin, and the tile-frame coordinate is
// (hi - x0_hi) + (lo - x0_lo), whose error is a rounding of the result only.
struct StageFrame {
    double x0[3], x1[3];   // region, absolute (FP64)
    float h0[3], l0[3];    // region origin, grid frame, double-float
    float b0[3], b1[3];    // region in the grid frame (hi parts), for FP32 box tests
};

__device__ __forceinline__ float box_dist2f(float x, float y, float z, const float *b0, const float *b1)
{
    float ex = x < b0[0] ? b0[0] - x : (x > b1[0] ? x - b1[0] : 0.0f);
    float ey = y < b0[1] ? b0[1] - y : (y > b1[1] ? y - b1[1] : 0.0f);
    float ez = z < b0[2] ? b0[2] - z : (z > b1[2] ? z - b1[2] : 0.0f);
    return ex * ex + ey * ey + ez * ez;
}

template <class T, class C>
__device__ __forceinline__ void stage_item(const Model &M, TileS<T, C> &S, int list, int k, const StageFrame &F)
{
    const double rp = M.rp;
    if constexpr (sizeof(T) == sizeof(float)) {
        const float rpf = (float)rp, tol = 1e-3f;
        if (list == 0) {
            float4 a = M.atom_hi[k];
            float reach = a.w + 2.0f * rpf + tol;
            if (box_dist2f(a.x, a.y, a.z, F.b0, F.b1) < reach * reach) {
                int s = atomicAdd(&S.na, 1);
                if (s < C::A) {
                    float4 l = M.atom_lo[k];
                    S.atom[s] = P4<T>{(a.x - F.h0[0]) + (l.x - F.l0[0]), (a.y - F.h0[1]) + (l.y - F.l0[1]),
                                      (a.z - F.h0[2]) + (l.z - F.l0[2]), a.w};
                    S.agid[s] = k;
                    S.aface[s] = M.atom_face[k];
                }
            }
        } else if (list == 1) {
            int p = M.pcell_list[k];
            float4 o = M.pair_hi[p];
            float reach = o.w + rpf + tol;
            if (box_dist2f(o.x, o.y, o.z, F.b0, F.b1) < reach * reach) {
                int s = atomicAdd(&S.np, 1);
                if (s < C::P) {
                    float4 l = M.pair_lo[p];
                    float4 u = M.pair_u32[p];
                    S.po[s] = P4<T>{(o.x - F.h0[0]) + (l.x - F.l0[0]), (o.y - F.h0[1]) + (l.y - F.l0[1]),
                                    (o.z - F.h0[2]) + (l.z - F.l0[2]), o.w};
                    S.pu[s] = P4<T>{u.x, u.y, u.z, 0.0f};
                    S.pij[s] = M.pair_ij[p];
                    S.pidx[s] = p;
                }
            }
        } else {
            int v = M.vcell_list[k];
            float4 q = M.vert_hi[v];
            float reach = rpf + tol;
            if (box_dist2f(q.x, q.y, q.z, F.b0, F.b1) < reach * reach) {
                int s = atomicAdd(&S.nv, 1);
                if (s < C::V) {
                    float4 l = M.vert_lo[v];
                    S.vq[s] = P4<T>{(q.x - F.h0[0]) + (l.x - F.l0[0]), (q.y - F.h0[1]) + (l.y - F.l0[1]),
                                    (q.z - F.h0[2]) + (l.z - F.l0[2]), 0.0f};
                    S.vidx[s] = v;
                }
            }
        }
    } else {
        const double tol = 1e-6;
        const double *x0 = F.x0, *x1 = F.x1;
        if (list == 0) {
            double4 a = M.atom[k];
            double reach = a.w + 2.0 * rp + tol;
            if (box_dist2(a.x, a.y, a.z, x0, x1) < reach * reach) {
                int s = atomicAdd(&S.na, 1);
                if (s < C::A) {
                    S.atom[s] = P4<T>{(T)(a.x - x0[0]), (T)(a.y - x0[1]), (T)(a.z - x0[2]), (T)a.w};
                    S.agid[s] = k;
                    S.aface[s] = M.atom_face[k];
                }
            }
        } else if (list == 1) {
            int p = M.pcell_list[k];
            double4 o = M.pair_o[p];
            double reach = o.w + rp + tol;
            if (box_dist2(o.x, o.y, o.z, x0, x1) < reach * reach) {
                int s = atomicAdd(&S.np, 1);
                if (s < C::P) {
                    double4 u = M.pair_u[p];
                    S.po[s] = P4<T>{(T)(o.x - x0[0]), (T)(o.y - x0[1]), (T)(o.z - x0[2]), (T)o.w};
                    S.pu[s] = P4<T>{(T)u.x, (T)u.y, (T)u.z, (T)0};
                    S.pij[s] = M.pair_ij[p];
                    S.pidx[s] = p;
                }
            }
        } else {
            int v = M.vcell_list[k];
            double4 q = M.vert[v];
            double reach = rp + tol;
            if (box_dist2(q.x, q.y, q.z, x0, x1) < reach * reach) {
                int s = atomicAdd(&S.nv, 1);
                if (s < C::V) {
                    S.vq[s] = P4<T>{(T)(q.x - x0[0]), (T)(q.y - x0[1]), (T)(q.z - x0[2]), (T)0};
                    S.vidx[s] = v;
                }
            }
        }
    }
}

// Stage the tile's atoms, free-arc pairs and free vertices (whole block of at
// least 96 threads).
// The items of every cell in range are numbered by a prefix over the cells
// and tested one per thread, so all threads share the work.
template <class T, class C>
__device__ void stage_tile(const Model &M, const Grid &G, int mol, long long tile, TileS<T, C> &S, double x0[3])
{
    const CellGrid &CG = M.cg[mol];
    if (threadIdx.x < 6) {  // the tile frame, once per tile: one thread per axis and end
        int t[3];
        tile_coords(G, tile, t);
        const int a = threadIdx.x < 3 ? threadIdx.x : threadIdx.x - 3;
        const double rel = G.h * (double)(TILE * (t[a] + G.toff[a]));  // region origin in the grid frame
        const double fx0 = G.lo[a] + rel, fx1 = fx0 + G.h * (double)TILE;
        // cell range of the region plus halo: FP32 indices with 1e-2 A of room
        // for their rounding (an FP64 division costs more than the rest)
        const float icell = 1.0f / (float)M.cell, halo = (float)G.halo + 1e-2f;
        if (threadIdx.x < 3) {
            S.fx0[a] = fx0;
            S.fx1[a] = fx1;
            S.fh0[a] = (float)rel;
            S.fl0[a] = (float)(rel - (double)S.fh0[a]);
            const int c = (int)floorf(((float)(fx0 - CG.clo[a]) - halo) * icell);
            S.fc0[a] = c < 0 ? 0 : (c >= CG.cn[a] ? CG.cn[a] - 1 : c);
        } else {
            const int c = (int)floorf(((float)(fx1 - CG.clo[a]) + halo) * icell);
            S.fc1[a] = c < 0 ? 0 : (c >= CG.cn[a] ? CG.cn[a] - 1 : c);
        }
    }
    if (threadIdx.x == 32) {
        S.na = 0;
        S.np = 0;
        S.nv = 0;
        S.flags = 0;
    }
    __syncthreads();
    StageFrame F;
    int c0[3], nc[3];
    for (int a = 0; a < 3; ++a) {
        x0[a] = S.fx0[a];
        F.x0[a] = S.fx0[a];
        F.x1[a] = S.fx1[a];
        F.h0[a] = S.fh0[a];
        F.l0[a] = S.fl0[a];
        F.b0[a] = F.h0[a];
        F.b1[a] = F.h0[a] + G.ht_hi;
        c0[a] = S.fc0[a];
        nc[a] = S.fc1[a] - S.fc0[a] + 1;
    }
    const int ncell = nc[0] * nc[1] * nc[2];
    if (ncell <= STAGE_CELLS) {
        for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
            int cz = c % nc[2], cy = (c / nc[2]) % nc[1], cx = c / (nc[1] * nc[2]);
            int id = CG.coff + ((c0[0] + cx) * CG.cn[1] + (c0[1] + cy)) * CG.cn[2] + (c0[2] + cz);
            S.cid[c] = id;
            S.cs[0][c + 1] = M.cell_start[id + 1] - M.cell_start[id];
            S.cs[1][c + 1] = M.pcell_start[id + 1] - M.pcell_start[id];
            S.cs[2][c + 1] = M.vcell_start[id + 1] - M.vcell_start[id];
        }
        __syncthreads();
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (warp < 3) {  // inclusive scan of each list's counts
            int *cs = S.cs[warp];
            int carry = 0;
            if (lane == 0) cs[0] = 0;
            for (int base = 1; base <= ncell; base += 32) {
                int k = base + lane;
                int v = k <= ncell ? cs[k] : 0;
                for (int o = 1; o < 32; o <<= 1) {
                    int u = __shfl_up_sync(0xffffffffu, v, o);
                    if (lane >= o) v += u;
                }
                if (k <= ncell) cs[k] = v + carry;
                carry += __shfl_sync(0xffffffffu, v, 31);
            }
        }
        __syncthreads();
        const int n0 = S.cs[0][ncell], n1 = S.cs[1][ncell], n2 = S.cs[2][ncell];
        for (int it = threadIdx.x; it < n0 + n1 + n2; it += blockDim.x) {
            int list = it < n0 ? 0 : (it < n0 + n1 ? 1 : 2);
            int k = it - (list == 0 ? 0 : (list == 1 ? n0 : n0 + n1));
            const int *cs = S.cs[list];
            int lo = 0, hi = ncell;
            while (hi - lo > 1) {
                int mid = (lo + hi) >> 1;
                if (cs[mid] <= k) lo = mid;
                else hi = mid;
            }
            int id = S.cid[lo];
            int off = k - cs[lo];
            int item = list == 0 ? M.cell_start[id] + off : (list == 1 ? M.pcell_start[id] + off : M.vcell_start[id] + off);
            stage_item<T>(M, S, list, item, F);
        }
    } else {
        __syncthreads();
        for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
            int cz = c % nc[2], cy = (c / nc[2]) % nc[1], cx = c / (nc[1] * nc[2]);
            int id = CG.coff + ((c0[0] + cx) * CG.cn[1] + (c0[1] + cy)) * CG.cn[2] + (c0[2] + cz);
            for (int k = M.cell_start[id]; k < M.cell_start[id + 1]; ++k) stage_item<T>(M, S, 0, k, F);
            for (int k = M.pcell_start[id]; k < M.pcell_start[id + 1]; ++k) stage_item<T>(M, S, 1, k, F);
            for (int k = M.vcell_start[id]; k < M.vcell_start[id + 1]; ++k) stage_item<T>(M, S, 2, k, F);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (S.na > C::A) { S.flags |= ERR_CAP_ATOMS; S.na = C::A; }
        if (S.np > C::P) { S.flags |= ERR_CAP_PAIRS; S.np = C::P; }
        if (S.nv > C::V) { S.flags |= ERR_CAP_VERTS; S.nv = C::V; }
    }
    __syncthreads();
}

// 1: d2 < t2 for certain; 0: d2 >= t2 for certain; -1: undecided (FP32 only).
// t is the threshold distance, delta the error bound of the compared vector.
template <bool FILT, class T>
__device__ __forceinline__ int lt_sq(T d2, T t2, T t, T delta)
{
    if (!FILT) return d2 < t2 ? 1 : 0;
    T e = T(2) * ((T(2) * t + delta) * delta + T(1e-6) * t2);
    if (d2 < t2 - e) return 1;
    if (d2 >= t2 + e) return 0;
    return -1;
}

// 1: a < b for certain; 0: a >= b for certain; -1 undecided (error bound e).
template <bool FILT, class T>
__device__ __forceinline__ int lt_lin(T a, T b, T e)
{
    if (!FILT) return a < b ? 1 : 0;
    if (a < b - T(2) * e) return 1;
    if (a >= b + T(2) * e) return 0;
    return -1;
}

// Freeness of q against every staged atom but e0, e1 (sorted indices of the
// atoms whose spheres carry q).  1 free, 0 covered, -1 undecided.
template <bool FILT, class Acc, class T>
__device__ __noinline__ int free_pt(const Acc &A, T qx, T qy, T qz, int e0, int e1, T rp, T delta)
{
    int res = 1;
    const int na = A.na();
    for (int k = 0; k < na; ++k) {
        int g = A.agid(k);
        if (g == e0 || g == e1) continue;
        P4<T> c = A.atom(k);
        T dx = qx - c.x, dy = qy - c.y, dz = qz - c.z;
        T R = c.w + rp;
        int t = lt_sq<FILT>(dx * dx + dy * dy + dz * dz, R * R, R, delta);
        if (t == 1) return 0;
        if (t < 0) res = -1;
    }
    return res;
}

// Freeness of q against the staged atoms in the set m0 & m1 (m1 may be
// null): 1 free, 0 covered, -1 undecided.  A witness q on the expanded
// sphere of atom a (and, for a saddle, of atom b too) can only be covered by
// an atom whose expanded sphere meets a's (and b's): |q - c_k| < R_k and
// |q - c_a| = R_a give |c_a - c_k| < R_a + R_k.  So the neighbour sets of a
// (and b) hold every atom that can cover q, and the answer is the one of
// every staged atom but a and b; an atom outside the sets could only have
// left an FP32 test undecided, never covered q.  nt counts the atom tests.
template <bool FILT, class Acc, class T>
__device__ __noinline__ int free_set(const Acc &A, T qx, T qy, T qz, const unsigned *m0, const unsigned *m1, T rp,
                                     T delta, int &nt)
{
    int res = 1;
    const int nw = (A.na() + 31) >> 5;
    for (int w = 0; w < nw; ++w) {
        unsigned bits = m1 ? (m0[w] & m1[w]) : m0[w];
        while (bits) {
            const int k = (w << 5) + __ffs(bits) - 1;
            bits &= bits - 1;
            ++nt;
            const P4<T> c = A.atom(k);
            const T dx = qx - c.x, dy = qy - c.y, dz = qz - c.z;
            const T R = c.w + rp;
            const int t = lt_sq<FILT>(dx * dx + dy * dy + dz * dz, R * R, R, delta);
            if (t == 1) return 0;
            if (t < 0) res = -1;
        }
    }
    return res;
}

// Staged slots of every staged pair's two atoms (-1: atom not staged), by an
// open-addressing hash of the staged atoms' model indices (hkey[slot_hash_size],
// hval[slot_hash_size] scratch).  Whole block; ends with a barrier.
template <class C>
__host__ __device__ constexpr int slot_hash_size()  // a power of two > 2 C::A
{
    int n = 1;
    while (n <= 2 * C::A) n <<= 1;
    return n;
}

template <class T, class C>
__device__ void pair_slots(const TileS<T, C> &S, int *hkey, short *hval, short2 *pslot)
{
    constexpr int HS = slot_hash_size<C>();
    auto slot_hash = [](int key) { return ((unsigned)key * 2654435761u) & (unsigned)(HS - 1); };
    for (int k = threadIdx.x; k < HS; k += blockDim.x) hkey[k] = -1;
    __syncthreads();
    for (int a = threadIdx.x; a < S.na; a += blockDim.x) {
        const int key = S.agid[a];
        for (unsigned h = slot_hash(key);; h = (h + 1) & (HS - 1)) {
            const int prev = atomicCAS(&hkey[h], -1, key);
            if (prev == -1 || prev == key) {
                hval[h] = (short)a;
                break;
            }
        }
    }
    __syncthreads();
    for (int p = threadIdx.x; p < S.np; p += blockDim.x) {
        const int2 ij = S.pij[p];
        short si = -1, sj = -1;
        for (unsigned h = slot_hash(ij.x);; h = (h + 1) & (HS - 1)) {
            const int k = hkey[h];
            if (k == ij.x) { si = hval[h]; break; }
            if (k == -1) break;
        }
        for (unsigned h = slot_hash(ij.y);; h = (h + 1) & (HS - 1)) {
            const int k = hkey[h];
            if (k == ij.y) { sj = hval[h]; break; }
            if (k == -1) break;
        }
        pslot[p] = make_short2(si, sj);
    }
    __syncthreads();
}

// Neighbour sets of the staged atoms (whole block): bit b of nbm[a * aw + w]
// (b = 32 w + bit) is set when the expanded spheres of staged atoms a != b
// come within 1e-3 A of meeting (the margin covers the rounding of staged
// FP32 positions, so no true neighbour is left out).
template <class T, class C>
__device__ __forceinline__ void build_neighbour_sets(const TileS<T, C> &S, unsigned *nbm, T rp)
{
    constexpr int aw = atom_words<C>();
    const int na = S.na, nw = (na + 31) >> 5;
    for (int it = threadIdx.x; it < na * nw; it += blockDim.x) {
        const int a = it / nw, w = it - a * nw;
        const P4<T> ca = S.atom[a];
        const T Ra = ca.w + rp + T(1e-3);
        unsigned bits = 0u;
        const int b0 = w << 5, b1 = min(na, b0 + 32);
        for (int b = b0; b < b1; ++b) {
            const P4<T> cb = S.atom[b];
            const T dx = ca.x - cb.x, dy = ca.y - cb.y, dz = ca.z - cb.z;
            const T reach = Ra + cb.w + rp;
            if (b != a && dx * dx + dy * dy + dz * dz < reach * reach) bits |= 1u << (b - b0);
        }
        nbm[a * aw + w] = bits;
    }
}

// Direction from a circle's axis towards y (y relative to the centre, u the
// unit axis): the part of y normal to u, with the rounding left along u
// removed, so it is normal to u even next to the axis; on the axis (to 1e-12
// relative) any unit normal to u -- every circle point is then nearest.
// Returns |w| before normalisation (0 on the axis) and w as a unit vector.
__device__ __forceinline__ double axis_normal(const double *y, const double *u, double *w)
{
    const double z = y[0] * u[0] + y[1] * u[1] + y[2] * u[2];
    for (int a = 0; a < 3; ++a) w[a] = y[a] - z * u[a];
    const double zr = w[0] * u[0] + w[1] * u[1] + w[2] * u[2];
    for (int a = 0; a < 3; ++a) w[a] -= zr * u[a];
    const double nw = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    if (nw > 1e-12 * (1.0 + sqrt(y[0] * y[0] + y[1] * y[1] + y[2] * y[2]))) {
        const double inw = 1.0 / nw;  // one FP64 division, not three
        for (int a = 0; a < 3; ++a) w[a] *= inw;
        return nw;
    }
    const double ax = fabs(u[0]) > 0.6 ? 0.0 : 1.0, ay = fabs(u[0]) > 0.6 ? 1.0 : 0.0;
    w[0] = -u[2] * ay;
    w[1] = u[2] * ax;
    w[2] = u[0] * ay - u[1] * ax;
    const double nv = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    for (int a = 0; a < 3; ++a) w[a] /= nv;
    return 0.0;
}

// Witness proposals.  A convex proposal of atom a at x is the radial
// projection q of x on a's expanded sphere, a saddle proposal of pair p the
// nearest point q of p's circle; each counts when q is free and closer than
// thr.  Return: 0 no proposal (certain), 1 proposal within thr (certain),
// -1 proposal with the distance test undecided, -2 undecided without a
// proposal; dq bounds the error of q, e0/e1 are the atoms that carry q.
template <bool FILT, class Acc, class T>
__device__ __forceinline__ int face_proposal(const Acc &A, int a, T x, T y, T z, T rp, T thr, T d0, T &qx, T &qy,
                                             T &qz, T &dq, int &e0, int &e1)
{
    if (!A.face(a)) return 0;
    P4<T> c = A.atom(a);
    T dx = x - c.x, dy = y - c.y, dz = z - c.z;
    T d2 = dx * dx + dy * dy + dz * dz;
    T R = c.w + rp;
    if (lt_sq<FILT>(d2, R * R, R, d0) == 0) return 0;
    T d = sqrt(d2);
    if (d <= T(1e-3)) return FILT ? -2 : 0;  // x at a centre is inside its vdW ball
    T wd = fabs(R - d);                        // distance to the projection
    int tw = lt_lin<FILT>(wd, thr, d0 + T(1e-6) * R);
    if (tw == 0) return 0;
    T s = R / d;
    qx = c.x + s * dx;
    qy = c.y + s * dy;
    qz = c.z + s * dz;
    dq = FILT ? d0 * (T(1) + T(2) * R / d) + T(1e-6) * R : T(0);
    e0 = A.agid(a);
    e1 = -1;
    return tw;
}

template <bool FILT, class Acc, class T>
__device__ __forceinline__ int saddle_proposal(const Acc &A, int p, T x, T y, T z, T rp, T thr, T d0, T &qx, T &qy,
                                               T &qz, T &dq, int &e0, int &e1)
{
    P4<T> o = A.po(p);
    P4<T> u = A.pu(p);
    T yx = x - o.x, yy = y - o.y, yz = z - o.z;
    T zc = yx * u.x + yy * u.y + yz * u.z;
    T wx = yx - zc * u.x, wy = yy - zc * u.y, wz = yz - zc * u.z;
    T w2 = wx * wx + wy * wy + wz * wz;
    T nw = sqrt(w2);
    T e1d = nw - o.w;
    T dist2 = e1d * e1d + zc * zc;
    T dw = FILT ? T(2) * d0 + T(2e-6) * (nw + fabs(zc)) : T(0);
    int t = lt_sq<FILT>(dist2, thr * thr, thr, T(1.5) * dw + T(1e-6));
    if (t == 0) return 0;
    if (FILT && nw < T(1e-3)) return -2;  // near the circle's axis the nearest point is ill-conditioned
    if constexpr (FILT) {
        T k = o.w / nw;
        qx = o.x + k * wx; qy = o.y + k * wy; qz = o.z + k * wz;
    } else {
        const double yv[3] = {(double)yx, (double)yy, (double)yz}, uv[3] = {(double)u.x, (double)u.y, (double)u.z};
        double wn[3];
        axis_normal(yv, uv, wn);
        qx = o.x + o.w * (T)wn[0]; qy = o.y + o.w * (T)wn[1]; qz = o.z + o.w * (T)wn[2];
    }
    dq = FILT ? o.w * T(2) * dw / nw + d0 + T(1e-6) * o.w : T(0);
    int2 ij = A.pij(p);
    e0 = ij.x;
    e1 = ij.y;
    return t;
}

// Convex witness of staged atom a at x: 1 free projection at distance < thr,
// 0 none, -1 undecided.  nbm: the staged atoms' neighbour sets; the
// projection's freeness is tested against a's neighbours (free_set).
template <bool FILT, class Acc, class T>
__device__ __noinline__ int face_witness(const Acc &A, int a, T x, T y, T z, T rp, T thr, T d0, const unsigned *nbm,
                                         int aw, int &nt)
{
    T qx, qy, qz, dq;
    int e0, e1;
    const int tw = face_proposal<FILT>(A, a, x, y, z, rp, thr, d0, qx, qy, qz, dq, e0, e1);
    if (tw == 0) return 0;
    if (tw == -2) return -1;
    int f = free_set<FILT>(A, qx, qy, qz, nbm + a * aw, (const unsigned *)nullptr, rp, dq + d0, nt);
    if (f == 1 && tw == 1) return 1;
    return f == 0 ? 0 : -1;
}

// Saddle witness of pair p at x: nearest point of its circle; its freeness
// is tested against the common neighbours of the pair's staged atoms (slots
// sa, sb).
template <bool FILT, class Acc, class T>
__device__ __noinline__ int saddle_witness(const Acc &A, int p, T x, T y, T z, T rp, T thr, T d0, const unsigned *nbm,
                                           int aw, int sa, int sb, int &nt)
{
    T qx, qy, qz, dq;
    int e0, e1;
    const int t = saddle_proposal<FILT>(A, p, x, y, z, rp, thr, d0, qx, qy, qz, dq, e0, e1);
    if (t == 0) return 0;
    if (t == -2) return -1;
    int f = free_set<FILT>(A, qx, qy, qz, nbm + sa * aw, nbm + sb * aw, rp, dq + d0, nt);
    if (f == 1 && t == 1) return 1;
    return f == 0 ? 0 : -1;
}

// Freeness of q (the same on every lane) against every staged atom but e0,
// e1, lanes over the atoms: 1 free, 0 covered, -1 undecided.
template <bool FILT, class Acc, class T>
__device__ __forceinline__ int warp_free(const Acc &A, T qx, T qy, T qz, int e0, int e1, T rp, T delta)
{
    const unsigned full = 0xffffffffu;
    bool cov = false, und = false;
    for (int k = threadIdx.x & 31; k < A.na(); k += 32) {
        int g = A.agid(k);
        if (g == e0 || g == e1) continue;
        P4<T> c = A.atom(k);
        T dx = qx - c.x, dy = qy - c.y, dz = qz - c.z;
        T R = c.w + rp;
        int t = lt_sq<FILT>(dx * dx + dy * dy + dz * dz, R * R, R, delta);
        if (t == 1) cov = true;
        else if (t < 0) und = true;
    }
    if (__any_sync(full, cov)) return 0;
    return __any_sync(full, und) ? -1 : 1;
}

// Proposals held by the lanes in `mask`, tested one after the other by the
// whole warp: 1 as soon as one is free and certainly within thr; else
// und is set when one could be, and `mine` on the lanes whose proposal could be.
template <bool FILT, class Acc, class T>
__device__ __forceinline__ int warp_test_proposals(const Acc &A, unsigned mask, int tw, T qx, T qy, T qz, T dq, int e0,
                                                   int e1, T rp, T d0, bool &und, bool &mine)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    while (mask) {
        const int b = __ffs(mask) - 1;
        mask &= mask - 1;
        const int btw = __shfl_sync(full, tw, b);
        if (btw == -2) {
            und = true;
            if (lane == b) mine = true;
            continue;
        }
        const T bx = __shfl_sync(full, qx, b), by = __shfl_sync(full, qy, b), bz = __shfl_sync(full, qz, b);
        const T bd = __shfl_sync(full, dq, b);
        const int b0 = __shfl_sync(full, e0, b), b1 = __shfl_sync(full, e1, b);
        const int f = warp_free<FILT>(A, bx, by, bz, b0, b1, rp, bd + d0);
        if (f == 1 && btw == 1) return 1;
        if (f != 0) {
            und = true;
            if (lane == b) mine = true;
        }
    }
    return 0;
}

// Warp-cooperative witness search at one point (all 32 lanes call it with the
// same point): 1 if a free probe centre lies at distance < thr (certain),
// 0 if none does (certain), -1 undecided with the undecided triple points and
// proposals flagged (um_vert, um_prop: on the lane that holds the item, bit r
// for item r * 32 + lane; proposals are numbered atoms first, then pairs),
// -2 undecided whether the point lies in an expanded ball (nothing flagged).
// Items (exclude_kind, exclude_id) are skipped: kind 0 atom (convex witness),
// 1 pair, 2 vertex, -1 none.
template <bool FILT, class Acc, class T>
__device__ __noinline__ int warp_witness(const Acc &A, T x, T y, T z, T rp, T thr, T d0, int exclude_kind,
                                         int exclude_id, unsigned &um_prop, unsigned &um_vert)
{
    um_prop = 0u;
    um_vert = 0u;
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int na = A.na(), np = A.np(), nv = A.nv();
    bool vdw = false, sas = false, sas_u = false;
    for (int a = lane; a < na; a += 32) {
        P4<T> c = A.atom(a);
        T dx = x - c.x, dy = y - c.y, dz = z - c.z;
        T d2 = dx * dx + dy * dy + dz * dz;
        T r = c.w, R = c.w + rp;
        if (lt_sq<FILT>(d2, r * r, r, d0) == 1) vdw = true;
        int s = lt_sq<FILT>(d2, R * R, R, d0);
        if (s == 1) sas = true;
        else if (s < 0) sas_u = true;
    }
    if (__any_sync(full, vdw)) return 0;
    if (!__any_sync(full, sas)) return __any_sync(full, sas_u) ? -2 : 1;
    bool found = false, und = false;
    const T thr2 = thr * thr;
    for (int v = lane; v < nv; v += 32) {
        if (exclude_kind == 2 && v == exclude_id) continue;
        P4<T> q = A.vq(v);
        T dx = x - q.x, dy = y - q.y, dz = z - q.z;
        int t = lt_sq<FILT>(dx * dx + dy * dy + dz * dz, thr2, thr, d0);
        if (t == 1) found = true;
        else if (t < 0) {
            und = true;
            if ((v >> 5) < 32) um_vert |= 1u << (v >> 5);
            else um_vert = ~0u, um_prop = ~0u;  // beyond the masks: the retest takes every item
        }
    }
    if (__any_sync(full, found)) return 1;
    und = __any_sync(full, und);
    // convex and saddle proposals: lanes propose, the warp tests freeness
    for (int i0 = 0; i0 < na + np; i0 += 32) {
        const int i = i0 + lane;
        T qx = T(0), qy = T(0), qz = T(0), dq = T(0);
        int e0 = -1, e1 = -1, tw = 0;
        if (i < na) {
            if (!(exclude_kind == 0 && i == exclude_id))
                tw = face_proposal<FILT>(A, i, x, y, z, rp, thr, d0, qx, qy, qz, dq, e0, e1);
        } else if (i < na + np) {
            if (!(exclude_kind == 1 && i - na == exclude_id))
                tw = saddle_proposal<FILT>(A, i - na, x, y, z, rp, thr, d0, qx, qy, qz, dq, e0, e1);
        }
        const unsigned m = __ballot_sync(full, tw != 0);
        bool mine = false;
        if (warp_test_proposals<FILT>(A, m, tw, qx, qy, qz, dq, e0, e1, rp, d0, und, mine) == 1) return 1;
        if (mine) {
            if ((i0 >> 5) < 32) um_prop |= 1u << (i0 >> 5);
            else um_vert = ~0u, um_prop = ~0u;  // beyond the masks: the retest takes every item
        }
    }
    return und ? -1 : 0;
}

// FP64 re-test of the items that a warp_witness<true> pass at the same point
// left undecided (um_prop, um_vert from that pass).  Its other items were
// decided for every position within its error bound, the exact point among
// them, so this gives the FP64 search's answer: 1 if a free probe centre lies
// at distance < thr, else 0.
template <class Acc>
__device__ __noinline__ int warp_witness_retest(const Acc &X, double x, double y, double z, double rp, double thr,
                                                unsigned um_prop, unsigned um_vert)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int na = X.na(), np = X.np(), nv = X.nv();
    bool found = false;
    // items past the masks' 32 words are retested when the lane's masks are
    // the "every item" mark that warp_witness leaves for them
    const bool all = um_vert == ~0u && um_prop == ~0u;
    for (int v = lane; v < nv; v += 32) {
        if (!((v >> 5) < 32 ? ((um_vert >> (v >> 5)) & 1u) : all)) continue;
        const P4<double> q = X.vq(v);
        const double dx = x - q.x, dy = y - q.y, dz = z - q.z;
        if (dx * dx + dy * dy + dz * dz < thr * thr) found = true;
    }
    if (__any_sync(full, found)) return 1;
    for (int i0 = 0; i0 < na + np; i0 += 32) {
        const int i = i0 + lane;
        double qx = 0.0, qy = 0.0, qz = 0.0, dq = 0.0;
        int e0 = -1, e1 = -1, tw = 0;
        if (i < na + np && ((i0 >> 5) < 32 ? ((um_prop >> (i0 >> 5)) & 1u) : all)) {
            if (i < na) tw = face_proposal<false>(X, i, x, y, z, rp, thr, 0.0, qx, qy, qz, dq, e0, e1);
            else tw = saddle_proposal<false>(X, i - na, x, y, z, rp, thr, 0.0, qx, qy, qz, dq, e0, e1);
        }
        bool und = false, mine = false;
        if (warp_test_proposals<false>(X, __ballot_sync(full, tw != 0), tw, qx, qy, qz, dq, e0, e1, rp, 0.0, und,
                                       mine) == 1)
            return 1;
    }
    return 0;
}

}  // namespace eses
