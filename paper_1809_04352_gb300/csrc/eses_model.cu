// eses_model.cu -- analytic patch construction (the first ESES stage, §2.2).
//
// From the atoms this builds, in FP64:
//   1. a counting sort of the atoms into uniform cells (cell edge 2 R_max, so
//      every overlapping pair of expanded balls sits in adjacent cells);
//   2. neighbour lists: j with |c_i - c_j| < R_i + R_j;
//   3. circle pairs: i < j whose expanded spheres meet in a circle
//      (|R_i - R_j| < D < R_i + R_j), carrier of the saddle (toroidal) patch;
//   4. for every circle, the arcs covered by the other expanded balls: a ball k
//      covers the arc where cos(phi - psi_k) > T_k; the circle keeps a free
//      arc unless one ball covers it whole or every covered-arc end point is
//      itself covered.  A free end point lies on three expanded spheres and in
//      no other ball: it is a free triple point (concave patch centre; the
//      probe-clash test of the north-star is this freeness test, in FP64);
//   5. a per-atom flag "the expanded sphere keeps a free face";
//   6. free-arc pairs and free triple points binned into the cells.
// The paper builds patches from all atom pairs under a distance threshold
// (§5) -- the same set as step 3.
#include <math.h>

#include "eses_kernels.h"

namespace eses {

// double-float split of a grid-frame coordinate
__device__ __forceinline__ void split_df(double v, float &hi, float &lo)
{
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

__device__ __forceinline__ int cell_coord(double v, double lo, double cell, int n)
{
    int k = (int)floor((v - lo) / cell);
    return k < 0 ? 0 : (k >= n ? n - 1 : k);
}

// cell id of a point of molecule m
__device__ __forceinline__ int cell_of(const CellGrid &g, double cell, double x, double y, double z)
{
    int a = cell_coord(x, g.clo[0], cell, g.cn[0]);
    int b = cell_coord(y, g.clo[1], cell, g.cn[1]);
    int c = cell_coord(z, g.clo[2], cell, g.cn[2]);
    return g.coff + (a * g.cn[1] + b) * g.cn[2] + c;
}

__global__ void k_cell_count(const double *__restrict__ xyz, const int *__restrict__ in_mol, int n,
                             const CellGrid *__restrict__ cg, double cell, int *__restrict__ cell_id,
                             int *__restrict__ cell_count)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int id = cell_of(cg[in_mol[i]], cell, xyz[3 * i + 0], xyz[3 * i + 1], xyz[3 * i + 2]);
    cell_id[i] = id;
    atomicAdd(&cell_count[id], 1);
}

int launch_cell_count(const double *xyz, const int *in_mol, int n, const CellGrid *cg, double cell, int *cell_id,
                      int *cell_count, cudaStream_t st)
{
    if (n <= 0) return 0;
    k_cell_count<<<(n + 255) / 256, 256, 0, st>>>(xyz, in_mol, n, cg, cell, cell_id, cell_count);
    return 1;
}

__global__ void k_cell_scatter(int n, const int *__restrict__ cell_id, const int *__restrict__ cell_start,
                               int *__restrict__ cursor, int *__restrict__ sorted_orig)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int id = cell_id[i];
    sorted_orig[cell_start[id] + atomicAdd(&cursor[id], 1)] = i;
}

int launch_cell_scatter(const double *, const double *, int n, const int *cell_id, const int *cell_start, int *cursor,
                         int *sorted_orig, cudaStream_t st)
{
    if (n <= 0) return 0;
    k_cell_scatter<<<(n + 255) / 256, 256, 0, st>>>(n, cell_id, cell_start, cursor, sorted_orig);
    return 1;
}

// order every cell by original atom index (deterministic layout), then gather
__global__ void k_cell_finish(const double *__restrict__ xyz, const double *__restrict__ r,
                              const int *__restrict__ in_mol, int ncell, const int *__restrict__ cell_start,
                              int *__restrict__ sorted_orig, double4 *__restrict__ atom, int *__restrict__ atom_mol)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    int s = cell_start[c], e = cell_start[c + 1];
    for (int a = s + 1; a < e; ++a) {
        int v = sorted_orig[a];
        int b = a - 1;
        while (b >= s && sorted_orig[b] > v) {
            sorted_orig[b + 1] = sorted_orig[b];
            --b;
        }
        sorted_orig[b + 1] = v;
    }
    for (int a = s; a < e; ++a) {
        int o = sorted_orig[a];
        atom[a] = make_double4(xyz[3 * o], xyz[3 * o + 1], xyz[3 * o + 2], r[o]);
        atom_mol[a] = in_mol[o];
    }
}

int launch_cell_finish(const double *xyz, const double *r, const int *in_mol, int ncell, const int *cell_start,
                       int *sorted_orig, double4 *atom, int *atom_mol, cudaStream_t st)
{
    k_cell_finish<<<(ncell + 255) / 256, 256, 0, st>>>(xyz, r, in_mol, ncell, cell_start, sorted_orig, atom, atom_mol);
    return 1;
}

// --------------------------------------------------------------------------
// neighbour iteration over the 27 cells around a sorted atom (in the cells of
// its own molecule), one warp: f(j, valid) on every lane for 32 consecutive
// atoms of a cell at a time, so the lanes visit the atoms in cell order and
// ballots over `valid` keep that order
// --------------------------------------------------------------------------
template <class F>
__device__ __forceinline__ void warp_neighbour_cells(const Model &M, int mol, double px, double py, double pz, F f)
{
    const int lane = threadIdx.x & 31;
    const CellGrid g = M.cg[mol];
    const int ca = cell_coord(px, g.clo[0], M.cell, g.cn[0]);
    const int cb = cell_coord(py, g.clo[1], M.cell, g.cn[1]);
    const int cc = cell_coord(pz, g.clo[2], M.cell, g.cn[2]);
    for (int a = max(ca - 1, 0); a <= min(ca + 1, g.cn[0] - 1); ++a)
        for (int b = max(cb - 1, 0); b <= min(cb + 1, g.cn[1] - 1); ++b)
            for (int c = max(cc - 1, 0); c <= min(cc + 1, g.cn[2] - 1); ++c) {
                const int id = g.coff + (a * g.cn[1] + b) * g.cn[2] + c;
                const int s0 = M.cell_start[id], s1 = M.cell_start[id + 1];
                for (int j0 = s0; j0 < s1; j0 += 32) f(j0 + lane, j0 + lane < s1);
            }
}

constexpr int NB_WARPS = 4;  // warps (atoms) per block of the neighbour and pair kernels

// the circle where expanded spheres (ci, Ri) and (cj, Rj) meet, if any.  Every
// operation is an explicit round-to-nearest intrinsic, so no multiply-add is
// contracted and every inlined copy (count and fill kernels, any path)
// computes the same bits: counts and fills agree, and a circle's bits do not
// depend on where it was computed.  frame_of and cover_of are kept out of
// line for the same reason.
__device__ __forceinline__ bool circle_of(double4 ci, double Ri, double4 cj, double Rj, double3 &o, double3 &u,
                                          double &rho)
{
    const double dx = __dsub_rn(cj.x, ci.x), dy = __dsub_rn(cj.y, ci.y), dz = __dsub_rn(cj.z, ci.z);
    const double D2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    const double S = __dadd_rn(Ri, Rj);
    if (!(D2 < __dmul_rn(S, S))) return false;
    const double D = __dsqrt_rn(D2);
    if (!(D > fabs(__dsub_rn(Ri, Rj)))) return false;
    const double a = __ddiv_rn(__dsub_rn(__dadd_rn(D2, __dmul_rn(Ri, Ri)), __dmul_rn(Rj, Rj)), __dmul_rn(2.0, D));
    const double rho2 = __dsub_rn(__dmul_rn(Ri, Ri), __dmul_rn(a, a));
    if (!(rho2 > 0.0)) return false;
    u = make_double3(__ddiv_rn(dx, D), __ddiv_rn(dy, D), __ddiv_rn(dz, D));
    o = make_double3(__dadd_rn(ci.x, __dmul_rn(a, u.x)), __dadd_rn(ci.y, __dmul_rn(a, u.y)),
                     __dadd_rn(ci.z, __dmul_rn(a, u.z)));
    rho = __dsqrt_rn(rho2);
    return true;
}

// The circle of atoms i and j, computed from the one with the smaller input
// index (axis from it to the other): the same bits whatever the atoms' places
// in the cell sort, so any model holding both atoms -- a subset of the atoms
// on the same grid included -- has the same circle.
__device__ __forceinline__ bool circle_canon(const Model &M, int i, int j, const double4 &ci, double Ri,
                                             const double4 &cj, double Rj, double3 &o, double3 &u, double &rho)
{
    const bool sw = M.atom_orig[i] > M.atom_orig[j];
    return circle_of(sw ? cj : ci, sw ? Rj : Ri, sw ? ci : cj, sw ? Ri : Rj, o, u, rho);
}

// One warp per atom: neighbours (expanded spheres that overlap), circles, and
// whether the expanded ball lies inside another one.
__global__ void __launch_bounds__(NB_WARPS * 32) k_nb_count(Model M, int *__restrict__ nb_count,
                                                           int *__restrict__ circle_count,
                                                           uint8_t *__restrict__ contained)
{
    const int i = blockIdx.x * NB_WARPS + (threadIdx.x >> 5);
    if (i >= M.n_atoms) return;  // uniform per warp
    const double4 ci = M.atom[i];
    const double Ri = ci.w + M.rp;
    int nb = 0, nc = 0;
    bool inside = false;
    warp_neighbour_cells(M, M.atom_mol[i], ci.x, ci.y, ci.z, [&](int j, bool valid) {
        if (!valid || j == i) return;
        const double4 cj = M.atom[j];
        const double Rj = cj.w + M.rp;
        const double dx = cj.x - ci.x, dy = cj.y - ci.y, dz = cj.z - ci.z;
        const double D2 = dx * dx + dy * dy + dz * dz;
        const double S = Ri + Rj;
        if (D2 < S * S) {
            ++nb;
            double3 o, u;
            double rho;
            if (circle_canon(M, i, j, ci, Ri, cj, Rj, o, u, rho)) ++nc;
            else if (Rj >= Ri && sqrt(D2) <= Rj - Ri) inside = true;  // ball i inside ball j
        }
    });
    for (int o = 16; o > 0; o >>= 1) {
        nb += __shfl_xor_sync(0xffffffffu, nb, o);
        nc += __shfl_xor_sync(0xffffffffu, nc, o);
    }
    inside = __any_sync(0xffffffffu, inside);
    if ((threadIdx.x & 31) == 0) {
        nb_count[i] = nb;
        circle_count[i] = nc;
        contained[i] = inside ? 1 : 0;
    }
}

int launch_nb_count(const Model &M, int *nb_count, int *circle_count, uint8_t *contained, cudaStream_t st)
{
    if (M.n_atoms <= 0) return 0;
    k_nb_count<<<(M.n_atoms + NB_WARPS - 1) / NB_WARPS, NB_WARPS * 32, 0, st>>>(M, nb_count, circle_count, contained);
    return 1;
}

// One warp per atom: the neighbour list in cell order (the same order as a
// serial walk over the 27 cells).
__global__ void __launch_bounds__(NB_WARPS * 32) k_nb_fill(Model M, int *__restrict__ nb_list)
{
    const int i = blockIdx.x * NB_WARPS + (threadIdx.x >> 5);
    if (i >= M.n_atoms) return;
    const int lane = threadIdx.x & 31;
    const double4 ci = M.atom[i];
    const double Ri = ci.w + M.rp;
    int w = M.nb_start[i];
    warp_neighbour_cells(M, M.atom_mol[i], ci.x, ci.y, ci.z, [&](int j, bool valid) {
        bool keep = false;
        if (valid && j != i) {
            const double4 cj = M.atom[j];
            const double Rj = cj.w + M.rp;
            const double dx = cj.x - ci.x, dy = cj.y - ci.y, dz = cj.z - ci.z;
            const double S = Ri + Rj;
            keep = dx * dx + dy * dy + dz * dz < S * S;
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) nb_list[w + __popc(m & ((1u << lane) - 1))] = j;
        w += __popc(m);
    });
}

int launch_nb_fill(const Model &M, int *nb_list, cudaStream_t st)
{
    if (M.n_atoms <= 0) return 0;
    k_nb_fill<<<(M.n_atoms + NB_WARPS - 1) / NB_WARPS, NB_WARPS * 32, 0, st>>>(M, nb_list);
    return 1;
}

// One warp per atom i: circles with neighbours j > i.
__global__ void __launch_bounds__(NB_WARPS * 32) k_pair_count(Model M, int *__restrict__ pair_count)
{
    const int i = blockIdx.x * NB_WARPS + (threadIdx.x >> 5);
    if (i >= M.n_atoms) return;
    const double4 ci = M.atom[i];
    const double Ri = ci.w + M.rp;
    int c = 0;
    for (int t = M.nb_start[i] + (threadIdx.x & 31); t < M.nb_start[i + 1]; t += 32) {
        const int j = M.nb_list[t];
        if (j <= i) continue;
        const double4 cj = M.atom[j];
        double3 o, u;
        double rho;
        if (circle_canon(M, i, j, ci, Ri, cj, cj.w + M.rp, o, u, rho)) ++c;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) pair_count[i] = c;
}

int launch_pair_count(const Model &M, int *pair_count, cudaStream_t st)
{
    if (M.n_atoms <= 0) return 0;
    k_pair_count<<<(M.n_atoms + NB_WARPS - 1) / NB_WARPS, NB_WARPS * 32, 0, st>>>(M, pair_count);
    return 1;
}

// One warp per atom i: the circles with neighbours j > i, in neighbour-list order.
__global__ void __launch_bounds__(NB_WARPS * 32) k_pair_fill(Model M, const int *__restrict__ pair_start,
                                                            double4 *__restrict__ pair_o, double4 *__restrict__ pair_u,
                                                            int2 *__restrict__ pair_ij)
{
    const int i = blockIdx.x * NB_WARPS + (threadIdx.x >> 5);
    if (i >= M.n_atoms) return;
    const int lane = threadIdx.x & 31;
    const double4 ci = M.atom[i];
    const double Ri = ci.w + M.rp;
    int w = pair_start[i];
    const int t1 = M.nb_start[i + 1];
    for (int t0 = M.nb_start[i]; t0 < t1; t0 += 32) {
        const int t = t0 + lane;
        bool keep = false;
        double3 o, u;
        double rho = 0.0;
        int j = -1;
        if (t < t1) {
            j = M.nb_list[t];
            if (j > i) {
                const double4 cj = M.atom[j];
                keep = circle_canon(M, i, j, ci, Ri, cj, cj.w + M.rp, o, u, rho);
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const int k = w + __popc(m & ((1u << lane) - 1));
            pair_o[k] = make_double4(o.x, o.y, o.z, rho);
            pair_u[k] = make_double4(u.x, u.y, u.z, 0.0);
            pair_ij[k] = make_int2(i, j);
        }
        w += __popc(m);
    }
}

int launch_pair_fill(const Model &M, const int *pair_start, double4 *pair_o, double4 *pair_u, int2 *pair_ij,
                      cudaStream_t st)
{
    if (M.n_atoms <= 0) return 0;
    k_pair_fill<<<(M.n_atoms + NB_WARPS - 1) / NB_WARPS, NB_WARPS * 32, 0, st>>>(M, pair_start, pair_o, pair_u,
                                                                               pair_ij);
    return 1;
}

// --------------------------------------------------------------------------
// free arcs and free triple points
// --------------------------------------------------------------------------
struct CircleFrame {
    double3 o, u, v1, v2;
    double rho;
};

__device__ __noinline__ CircleFrame frame_of(double4 po, double4 pu)
{
    CircleFrame f;
    f.o = make_double3(po.x, po.y, po.z);
    f.u = make_double3(pu.x, pu.y, pu.z);
    f.rho = po.w;
    // a unit vector normal to u
    double3 t = fabs(f.u.x) > 0.6 ? make_double3(0.0, 1.0, 0.0) : make_double3(1.0, 0.0, 0.0);
    double3 v = make_double3(f.u.y * t.z - f.u.z * t.y, f.u.z * t.x - f.u.x * t.z, f.u.x * t.y - f.u.y * t.x);
    double nv = sqrt(v.x * v.x + v.y * v.y + v.z * v.z);
    f.v1 = make_double3(v.x / nv, v.y / nv, v.z / nv);
    f.v2 = make_double3(f.u.y * f.v1.z - f.u.z * f.v1.y, f.u.z * f.v1.x - f.u.x * f.v1.z,
                        f.u.x * f.v1.y - f.u.y * f.v1.x);
    return f;
}

// Coverage of the circle by ball (ck, Rk): 0 none, 1 partial (end points
// qa, qb returned), 2 the whole circle.
__device__ __noinline__ int cover_of(const CircleFrame &f, double4 ck, double Rk, double3 &qa, double3 &qb)
{
    double dx = ck.x - f.o.x, dy = ck.y - f.o.y, dz = ck.z - f.o.z;
    double d1 = dx * f.v1.x + dy * f.v1.y + dz * f.v1.z;
    double d2 = dx * f.v2.x + dy * f.v2.y + dz * f.v2.z;
    double dd = dx * dx + dy * dy + dz * dz;
    double A = sqrt(d1 * d1 + d2 * d2);
    // |q(phi) - c_k|^2 = rho^2 + |d|^2 - 2 rho A cos(phi - psi); covered iff < R_k^2
    double num = f.rho * f.rho + dd - Rk * Rk;
    double den = 2.0 * f.rho * A;
    if (num >= den) return 0;
    if (num < -den) return 2;
    double T = num / den;
    double s = sqrt(fmax(0.0, 1.0 - T * T));
    double3 ep = make_double3((d1 * f.v1.x + d2 * f.v2.x) / A, (d1 * f.v1.y + d2 * f.v2.y) / A,
                              (d1 * f.v1.z + d2 * f.v2.z) / A);
    double3 en = make_double3(f.u.y * ep.z - f.u.z * ep.y, f.u.z * ep.x - f.u.x * ep.z, f.u.x * ep.y - f.u.y * ep.x);
    qa = make_double3(f.o.x + f.rho * (T * ep.x + s * en.x), f.o.y + f.rho * (T * ep.y + s * en.y),
                      f.o.z + f.rho * (T * ep.z + s * en.z));
    qb = make_double3(f.o.x + f.rho * (T * ep.x - s * en.x), f.o.y + f.rho * (T * ep.y - s * en.y),
                      f.o.z + f.rho * (T * ep.z - s * en.z));
    return 1;
}

__device__ __forceinline__ bool common_nb(const Model &M, int k, int i, int j, double4 cj, double Rj)
{
    if (k == i || k == j) return false;
    double4 ck = M.atom[k];
    double Rk = ck.w + M.rp;
    double dx = ck.x - cj.x, dy = ck.y - cj.y, dz = ck.z - cj.z;
    double S = Rk + Rj;
    return dx * dx + dy * dy + dz * dz < S * S;
}

// the end point q (on sphere k) is free iff no other common neighbour covers it
__device__ __forceinline__ bool endpoint_free(const Model &M, int i, int j, int k, double4 cj, double Rj, double3 q)
{
    for (int t = M.nb_start[i]; t < M.nb_start[i + 1]; ++t) {
        int m = M.nb_list[t];
        if (m == k || !common_nb(M, m, i, j, cj, Rj)) continue;
        double4 cm = M.atom[m];
        double Rm = cm.w + M.rp;
        double dx = q.x - cm.x, dy = q.y - cm.y, dz = q.z - cm.z;
        if (dx * dx + dy * dy + dz * dz < Rm * Rm) return false;
    }
    return true;
}

template <bool EMIT>
__device__ void arcs_of_pair(const Model &M, int p, uint8_t *pair_free, int *vert_count, const int *vert_start,
                             double4 *vert)
{
    int2 ij = M.pair_ij[p];
    const int i = ij.x, j = ij.y;
    CircleFrame f = frame_of(M.pair_o[p], M.pair_u[p]);
    double4 cj = M.atom[j];
    double Rj = cj.w + M.rp;
    bool full = false;
    int n_partial = 0, n_free_end = 0, n_emit = 0;
    int w = EMIT ? vert_start[p] : 0;
    for (int t = M.nb_start[i]; t < M.nb_start[i + 1] && !full; ++t) {
        int k = M.nb_list[t];
        if (!common_nb(M, k, i, j, cj, Rj)) continue;
        double4 ck = M.atom[k];
        double3 qa, qb;
        int c = cover_of(f, ck, ck.w + M.rp, qa, qb);
        if (c == 2) {
            full = true;
        } else if (c == 1) {
            ++n_partial;
            bool fa = endpoint_free(M, i, j, k, cj, Rj, qa);
            bool fb = endpoint_free(M, i, j, k, cj, Rj, qb);
            n_free_end += (int)fa + (int)fb;
            // each triple point is emitted once: from the circle of the triple's two
            // atoms with the smaller input indices (any cell order gives the same bits)
            if (M.atom_orig[k] > M.atom_orig[i] && M.atom_orig[k] > M.atom_orig[j]) {
                if (fa) {
                    if (EMIT) vert[w + n_emit] = make_double4(qa.x, qa.y, qa.z, (double)k);
                    ++n_emit;
                }
                if (fb) {
                    if (EMIT) vert[w + n_emit] = make_double4(qb.x, qb.y, qb.z, (double)k);
                    ++n_emit;
                }
            }
        }
    }
    if (!EMIT) {
        bool has_free = !full && (n_partial == 0 || n_free_end > 0);
        pair_free[p] = has_free ? 1 : 0;
        vert_count[p] = full ? 0 : n_emit;
    }
}

// FP32-filtered form of arcs_of_pair, one warp per circle: the common
// neighbours are cached in FP32 in the circle's frame (from the double-float
// copies: two roundings of the offset), and every decision -- common neighbour, no/partial/full cover,
// end point covered -- is taken in FP32 when it clears its error bound and in
// FP64 otherwise, so the decisions are those of the FP64 form.  FP32 end
// points carry a propagated error bound (the FP64 end point is used when that
// bound exceeds 2e-4 A); emitted triple points are always computed in FP64.
constexpr int ARC_MAXN = 256;

// 1: d2 < t^2 certain, 0: d2 >= t^2 certain, -1 undecided (delta: error of the vector)
__device__ __forceinline__ int arc_lt(float d2, float t, float delta)
{
    float t2 = t * t;
    float e = 2.0f * ((2.0f * t + delta) * delta + 1e-6f * t2);
    if (d2 < t2 - e) return 1;
    if (d2 >= t2 + e) return 0;
    return -1;
}

// The lanes gather the common neighbours (ballot compaction, list order;
// circles with more than ARC_MAXN take the FP64 form on one lane), then each
// lane takes candidates a = lane, lane + 32, ...: its cover of the circle, its
// end points and their freeness against every other candidate.  Emitted triple points keep the order (a, end point).
constexpr int ARC_WARPS = 4;

struct ArcWarp {
    float4 nb[ARC_MAXN];
    int nbk[ARC_MAXN];
};

template <bool EMIT>
__device__ void arcs_of_pair_warp(const Model &M, int p, ArcWarp &W, uint8_t *pair_free, int *vert_count,
                                  const int *vert_start, double4 *vert)
{
    const unsigned full_mask = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int2 ij = M.pair_ij[p];
    const int i = ij.x, j = ij.y;
    const float4 oh = M.pair_hi[p], ol = M.pair_lo[p], u4 = M.pair_u32[p];
    const float rho = oh.w;
    const float ux = u4.x, uy = u4.y, uz = u4.z;
    const float tx = fabsf(ux) > 0.6f ? 0.0f : 1.0f, ty = fabsf(ux) > 0.6f ? 1.0f : 0.0f;
    float v1x = -uz * ty, v1y = uz * tx, v1z = ux * ty - uy * tx;
    const float iv1 = 1.0f / sqrtf(v1x * v1x + v1y * v1y + v1z * v1z);
    v1x *= iv1; v1y *= iv1; v1z *= iv1;
    const float v2x = uy * v1z - uz * v1y, v2y = uz * v1x - ux * v1z, v2z = ux * v1y - uy * v1x;
    const float dlt = 3e-6f;
    const float4 jh = M.atom_hi[j], jl = M.atom_lo[j];
    const float djx = (jh.x - oh.x) + (jl.x - ol.x), djy = (jh.y - oh.y) + (jl.y - ol.y),
                djz = (jh.z - oh.z) + (jl.z - ol.z);
    const float rpf = (float)M.rp;
    const float Rj = jh.w + rpf;
    const double4 cj = M.atom[j];
    const double Rj64 = cj.w + M.rp;
    // 1. common neighbours, in list order
    int n = 0;
    const int t_end = M.nb_start[i + 1];
    for (int t0 = M.nb_start[i]; t0 < t_end; t0 += 32) {
        const int t = t0 + lane;
        bool keep = false;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        int k = -1;
        if (t < t_end) {
            k = M.nb_list[t];
            if (k != j) {
                const float4 kh = M.atom_hi[k], kl = M.atom_lo[k];
                const float dx = (kh.x - oh.x) + (kl.x - ol.x), dy = (kh.y - oh.y) + (kl.y - ol.y),
                            dz = (kh.z - oh.z) + (kl.z - ol.z);
                const float Rk = kh.w + rpf;
                const float ex = dx - djx, ey = dy - djy, ez = dz - djz;
                const int c = arc_lt(ex * ex + ey * ey + ez * ez, Rk + Rj, 2.0f * dlt);
                keep = c == 1 || (c < 0 && common_nb(M, k, i, j, cj, Rj64));
                v = make_float4(dx, dy, dz, Rk);
            }
        }
        const unsigned m = __ballot_sync(full_mask, keep);
        const int pos = n + __popc(m & ((1u << lane) - 1));
        if (keep && pos < ARC_MAXN) {
            W.nb[pos] = v;
            W.nbk[pos] = k;
        }
        n += __popc(m);
    }
    __syncwarp();
    if (n > ARC_MAXN) {  // very crowded circle: the FP64 form, one lane
        if (lane == 0) arcs_of_pair<EMIT>(M, p, pair_free, vert_count, vert_start, vert);
        __syncwarp();
        return;
    }
    CircleFrame f;
    bool have64 = false;
    // 2. a candidate that covers the whole circle ends the work before any
    //    end point is tested (at protein packing most circles are buried
    //    this way): the same cover decisions as below, FP64 when undecided
    bool full = false;
    for (int r = 0; r * 32 < n && !full; ++r) {
        const int a = r * 32 + lane;
        bool whole = false;
        if (a < n) {
            const float4 c = W.nb[a];
            const float d1 = c.x * v1x + c.y * v1y + c.z * v1z;
            const float d2 = c.x * v2x + c.y * v2y + c.z * v2z;
            const float dd = c.x * c.x + c.y * c.y + c.z * c.z;
            const float A = sqrtf(d1 * d1 + d2 * d2);
            const float num = rho * rho + dd - c.w * c.w, den = 2.0f * rho * A;
            const float dk = sqrtf(dd);
            const float en = 2.0f * dk * dlt + 2e-6f * (rho * rho + dd + c.w * c.w);
            const float ed = 2.0f * rho * (dlt + 3e-7f * dk) + 2e-6f * den;
            const float err = 2.0f * (en + ed);
            if (num < -den - err) {
                whole = true;
            } else if (num < -den + err) {  // undecided near a whole cover: FP64
                if (!have64) {
                    f = frame_of(M.pair_o[p], M.pair_u[p]);
                    have64 = true;
                }
                const double4 ck = M.atom[W.nbk[a]];
                double3 qa, qb;
                whole = cover_of(f, ck, ck.w + M.rp, qa, qb) == 2;
            }
        }
        full = __any_sync(full_mask, whole);
    }
    if (full) {
        if (!EMIT && lane == 0) {
            pair_free[p] = 0;
            vert_count[p] = 0;
        }
        __syncwarp();
        return;
    }
    // 3. candidates a = lane + 32 r: covers, end points and their freeness
    int n_partial = 0, n_free_end = 0, n_emit_total = 0;
    const int w0 = EMIT ? vert_start[p] : 0;
    for (int r = 0; r * 32 < n; ++r) {
        const int a = r * 32 + lane;
        int status = 0;  // 0 none, 1 partial, 2 full
        bool fr[2] = {false, false};
        double3 qe[2];
        bool e64 = false;
        if (a < n) {
            const float4 c = W.nb[a];
            const float d1 = c.x * v1x + c.y * v1y + c.z * v1z;
            const float d2 = c.x * v2x + c.y * v2y + c.z * v2z;
            const float dd = c.x * c.x + c.y * c.y + c.z * c.z;
            const float A = sqrtf(d1 * d1 + d2 * d2);
            const float num = rho * rho + dd - c.w * c.w, den = 2.0f * rho * A;
            const float dk = sqrtf(dd);
            const float en = 2.0f * dk * dlt + 2e-6f * (rho * rho + dd + c.w * c.w);
            const float ed = 2.0f * rho * (dlt + 3e-7f * dk) + 2e-6f * den;
            const float err = 2.0f * (en + ed);
            float qf[2][3];
            float dq = 1.0f;
            if (num >= den + err) {
                status = 0;
            } else if (num < -den - err) {
                status = 2;
            } else {
                status = 1;
                if (num < den - err && num > -den + err) {  // partial for certain: FP32 end points
                    const float T = num / den;
                    const float sT = sqrtf(fmaxf(0.0f, 1.0f - T * T));
                    const float iA = 1.0f / A;
                    const float epx = (d1 * v1x + d2 * v2x) * iA, epy = (d1 * v1y + d2 * v2y) * iA,
                                epz = (d1 * v1z + d2 * v2z) * iA;
                    const float enx = uy * epz - uz * epy, eny = uz * epx - ux * epz, enz = ux * epy - uy * epx;
                    for (int e = 0; e < 2; ++e) {
                        const float sg = e == 0 ? 1.0f : -1.0f;
                        qf[e][0] = rho * (T * epx + sg * sT * enx);
                        qf[e][1] = rho * (T * epy + sg * sT * eny);
                        qf[e][2] = rho * (T * epz + sg * sT * enz);
                    }
                    const float dT = (en + fabsf(T) * ed) / den;
                    dq = rho * (dT * (1.0f + fabsf(T) / fmaxf(sT, 1e-6f)) + 2.0f * (dlt / fmaxf(A, 1e-6f) + 3e-7f)) +
                         1e-6f;
                }
                if (dq > 2e-4f) {  // undecided cover or loose FP32 end points: FP64
                    if (!have64) {
                        f = frame_of(M.pair_o[p], M.pair_u[p]);
                        have64 = true;
                    }
                    const double4 ck = M.atom[W.nbk[a]];
                    const int cov = cover_of(f, ck, ck.w + M.rp, qe[0], qe[1]);
                    status = cov;
                    if (cov == 1) {
                        for (int e = 0; e < 2; ++e) {
                            qf[e][0] = (float)(qe[e].x - f.o.x);
                            qf[e][1] = (float)(qe[e].y - f.o.y);
                            qf[e][2] = (float)(qe[e].z - f.o.z);
                        }
                        dq = 1e-6f;
                        e64 = true;
                    }
                }
            }
            if (status == 1) {
                for (int e = 0; e < 2; ++e) {
                    bool free_ = true;
                    for (int b = 0; b < n && free_; ++b) {
                        if (b == a) continue;
                        const float4 cb = W.nb[b];
                        const float ex = qf[e][0] - cb.x, ey = qf[e][1] - cb.y, ez = qf[e][2] - cb.z;
                        int t = arc_lt(ex * ex + ey * ey + ez * ez, cb.w, dq + dlt);
                        if (t < 0) {  // FP64: the exact end point against the exact ball
                            if (!e64) {
                                if (!have64) {
                                    f = frame_of(M.pair_o[p], M.pair_u[p]);
                                    have64 = true;
                                }
                                const double4 ck = M.atom[W.nbk[a]];
                                cover_of(f, ck, ck.w + M.rp, qe[0], qe[1]);
                                e64 = true;
                            }
                            const double4 c64 = M.atom[W.nbk[b]];
                            const double Rb = c64.w + M.rp;
                            const double gx = qe[e].x - c64.x, gy = qe[e].y - c64.y, gz = qe[e].z - c64.z;
                            t = (gx * gx + gy * gy + gz * gz < Rb * Rb) ? 1 : 0;
                        }
                        if (t == 1) free_ = false;
                    }
                    fr[e] = free_;
                }
            }
        }
        full = full || __any_sync(full_mask, status == 2);
        if (full) break;  // uniform
        int np_ = status == 1 ? 1 : 0, nf_ = (int)fr[0] + (int)fr[1];
        // emitted once: from the circle of the two atoms with the smaller input indices
        const bool emits = status == 1 && a < n && M.atom_orig[W.nbk[a]] > M.atom_orig[i] &&
                           M.atom_orig[W.nbk[a]] > M.atom_orig[j];
        int ne_ = emits ? nf_ : 0;
        // inclusive scan of ne_ over the lanes (the serial order a = 0, 1, ...)
        int inc = ne_;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(full_mask, inc, o);
            if (lane >= o) inc += u;
        }
        const int tot = __shfl_sync(full_mask, inc, 31);
        if (EMIT && ne_ > 0) {
            if (!e64) {
                if (!have64) {
                    f = frame_of(M.pair_o[p], M.pair_u[p]);
                    have64 = true;
                }
                const double4 ck = M.atom[W.nbk[a]];
                cover_of(f, ck, ck.w + M.rp, qe[0], qe[1]);
            }
            int wpos = w0 + n_emit_total + inc - ne_;
            const double kw = (double)W.nbk[a];  // the triple's third atom
            for (int e = 0; e < 2; ++e)
                if (fr[e]) vert[wpos++] = make_double4(qe[e].x, qe[e].y, qe[e].z, kw);
        }
        n_emit_total += tot;
        for (int o = 16; o > 0; o >>= 1) {
            np_ += __shfl_xor_sync(full_mask, np_, o);
            nf_ += __shfl_xor_sync(full_mask, nf_, o);
        }
        n_partial += np_;
        n_free_end += nf_;
    }
    if (!EMIT && lane == 0) {
        const bool has_free = !full && (n_partial == 0 || n_free_end > 0);
        pair_free[p] = has_free ? 1 : 0;
        vert_count[p] = full ? 0 : n_emit_total;
    }
    __syncwarp();
}

__global__ void __launch_bounds__(ARC_WARPS * 32) k_arcs(Model M, uint8_t *__restrict__ pair_free,
                                                         int *__restrict__ vert_count)
{
    __shared__ ArcWarp W[ARC_WARPS];
    const int warp = threadIdx.x >> 5;
    const int p = blockIdx.x * ARC_WARPS + warp;
    if (p >= M.n_pairs) return;  // uniform per warp
    arcs_of_pair_warp<false>(M, p, W[warp], pair_free, vert_count, nullptr, nullptr);
}

// emits the free triple points of circle p (xyz, third atom in w), their
// molecule and their three atoms (i, j of the circle, k; sorted indices)
__global__ void __launch_bounds__(ARC_WARPS * 32) k_arcs_emit(Model M, const int *__restrict__ vert_start,
                                                              double4 *__restrict__ vert, int *__restrict__ vert_mol,
                                                              int4 *__restrict__ vert_atoms)
{
    __shared__ ArcWarp W[ARC_WARPS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int p = blockIdx.x * ARC_WARPS + warp;
    if (p >= M.n_pairs) return;
    if (vert_start[p + 1] == vert_start[p]) return;
    arcs_of_pair_warp<true>(M, p, W[warp], nullptr, nullptr, vert_start, vert);
    __syncwarp();
    const int2 ij = M.pair_ij[p];
    const int mol = M.atom_mol[ij.x];
    for (int k = vert_start[p] + lane; k < vert_start[p + 1]; k += 32) {
        vert_mol[k] = mol;
        vert_atoms[k] = make_int4(ij.x, ij.y, (int)vert[k].w, 0);
    }
}

int launch_arcs(const Model &M, uint8_t *pair_free, int *vert_count, cudaStream_t st)
{
    if (M.n_pairs <= 0) return 0;
    k_arcs<<<(M.n_pairs + ARC_WARPS - 1) / ARC_WARPS, ARC_WARPS * 32, 0, st>>>(M, pair_free, vert_count);
    return 1;
}

int launch_arcs_emit(const Model &M, const int *vert_start, double4 *vert, int *vert_mol, int4 *vert_atoms,
                     cudaStream_t st)
{
    if (M.n_pairs <= 0) return 0;
    k_arcs_emit<<<(M.n_pairs + ARC_WARPS - 1) / ARC_WARPS, ARC_WARPS * 32, 0, st>>>(M, vert_start, vert, vert_mol,
                                                                                  vert_atoms);
    return 1;
}

__global__ void k_faces_init(int n, const int *__restrict__ circle_count, const uint8_t *__restrict__ contained,
                             uint8_t *__restrict__ face)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    face[i] = (circle_count[i] == 0 && !contained[i]) ? 1 : 0;
}

__global__ void k_faces_pairs(Model M, uint8_t *__restrict__ face)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M.n_pairs) return;
    if (M.pair_free[p]) {
        int2 ij = M.pair_ij[p];
        face[ij.x] = 1;
        face[ij.y] = 1;
    }
}

int launch_faces(const Model &M, const int *circle_count, const uint8_t *contained, uint8_t *face, cudaStream_t st)
{
    int nl = 0;
    if (M.n_atoms > 0) ++nl, k_faces_init<<<(M.n_atoms + 255) / 256, 256, 0, st>>>(M.n_atoms, circle_count, contained, face);
    if (M.n_pairs > 0) ++nl, k_faces_pairs<<<(M.n_pairs + 255) / 256, 256, 0, st>>>(M, face);
    return nl;
}

// which = 0: free-arc pairs by circle centre; which = 1: free triple points
// cull: bin only the circles that keep a free arc (buried saddle patches are
// culled before the classification); without it every circle is binned
__global__ void k_bin_count(Model M, int which, bool cull, int *__restrict__ count, int *__restrict__ item_cell)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    int n = which == 0 ? M.n_pairs : M.n_verts;
    if (p >= n) return;
    double x, y, z;
    int mol;
    if (which == 0) {
        if (cull && !M.pair_free[p]) {
            item_cell[p] = -1;
            return;
        }
        double4 o = M.pair_o[p];
        x = o.x; y = o.y; z = o.z;
        mol = M.atom_mol[M.pair_ij[p].x];
    } else {
        double4 v = M.vert[p];
        x = v.x; y = v.y; z = v.z;
        mol = M.vert_mol[p];
    }
    int id = cell_of(M.cg[mol], M.cell, x, y, z);
    item_cell[p] = id;
    atomicAdd(&count[id], 1);
}

__global__ void k_bin_scatter(int n, const int *__restrict__ item_cell, const int *__restrict__ start,
                              int *__restrict__ cursor, int *__restrict__ list)
{
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int id = item_cell[p];
    if (id < 0) return;
    list[start[id] + atomicAdd(&cursor[id], 1)] = p;
}

__global__ void k_f32_atoms(Model M, const Grid *__restrict__ grids, float4 *__restrict__ hi, float4 *__restrict__ lo)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M.n_atoms) return;
    const double *L = grids[M.atom_mol[k]].lo;
    const double lx = L[0], ly = L[1], lz = L[2];
    float hx, hy, hz, ex, ey, ez;
    double4 a = M.atom[k];
    split_df(a.x - lx, hx, ex);
    split_df(a.y - ly, hy, ey);
    split_df(a.z - lz, hz, ez);
    hi[k] = make_float4(hx, hy, hz, (float)a.w);
    lo[k] = make_float4(ex, ey, ez, 0.0f);
}

__global__ void k_f32_pairs(Model M, const Grid *__restrict__ grids, float4 *__restrict__ hi, float4 *__restrict__ lo,
                            float4 *__restrict__ u32)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M.n_pairs) return;
    const double *L = grids[M.atom_mol[M.pair_ij[k].x]].lo;
    const double lx = L[0], ly = L[1], lz = L[2];
    float hx, hy, hz, ex, ey, ez;
    double4 o = M.pair_o[k];
    double4 u = M.pair_u[k];
    split_df(o.x - lx, hx, ex);
    split_df(o.y - ly, hy, ey);
    split_df(o.z - lz, hz, ez);
    hi[k] = make_float4(hx, hy, hz, (float)o.w);
    lo[k] = make_float4(ex, ey, ez, 0.0f);
    u32[k] = make_float4((float)u.x, (float)u.y, (float)u.z, 0.0f);
}

__global__ void k_f32_verts(Model M, const Grid *__restrict__ grids, float4 *__restrict__ hi, float4 *__restrict__ lo)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= M.n_verts) return;
    const double *L = grids[M.vert_mol[k]].lo;
    const double lx = L[0], ly = L[1], lz = L[2];
    float hx, hy, hz, ex, ey, ez;
    double4 v = M.vert[k];
    split_df(v.x - lx, hx, ex);
    split_df(v.y - ly, hy, ey);
    split_df(v.z - lz, hz, ez);
    hi[k] = make_float4(hx, hy, hz, 0.0f);
    lo[k] = make_float4(ex, ey, ez, 0.0f);
}

// which: 0 atoms, 1 circles (centre and axis), 2 triple points; relative to
// the grid origin of each item's molecule
int launch_model_f32(const Model &M, int which, const Grid *grids, float4 *hi, float4 *lo_, float4 *u32,
                     cudaStream_t st)
{
    int n = which == 0 ? M.n_atoms : (which == 1 ? M.n_pairs : M.n_verts);
    if (n <= 0) return 0;
    if (which == 0) k_f32_atoms<<<(n + 255) / 256, 256, 0, st>>>(M, grids, hi, lo_);
    else if (which == 1) k_f32_pairs<<<(n + 255) / 256, 256, 0, st>>>(M, grids, hi, lo_, u32);
    else k_f32_verts<<<(n + 255) / 256, 256, 0, st>>>(M, grids, hi, lo_);
    return 1;
}

int launch_bin_count(const Model &M, int which, bool cull, int *count, int *item_cell, cudaStream_t st)
{
    int n = which == 0 ? M.n_pairs : M.n_verts;
    if (n <= 0) return 0;
    k_bin_count<<<(n + 255) / 256, 256, 0, st>>>(M, which, cull, count, item_cell);
    return 1;
}

int launch_bin_scatter(const Model &M, int which, const int *item_cell, const int *start, int *cursor, int *list,
                        cudaStream_t st)
{
    int n = which == 0 ? M.n_pairs : M.n_verts;
    if (n <= 0) return 0;
    k_bin_scatter<<<(n + 255) / 256, 256, 0, st>>>(n, item_cell, start, cursor, list);
    return 1;
}

}  // namespace eses
