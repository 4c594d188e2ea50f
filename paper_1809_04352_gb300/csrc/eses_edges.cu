// eses_edges.cu -- crossing edges, surface roots and normals, area and volume
// (the third and fourth ESES stages, Eq. 3-4).
//
// k_edge_count: per tile and axis, the edges (p, p + e_a) leaving the tile's
//   points whose end labels differ, and the edges with both ends inside.
// (exclusive scan of the counts -> every tile's output offset per axis; the
//   paper serialises this output step in a critical section, Algorithm 1)
// k_edge_solve: per tile, stages the patches and solves every crossing edge.
//   The surface along an edge is made of pieces of van der Waals spheres
//   (convex), tori around pair circles (saddle) and probe spheres around free
//   triple points (concave).  Every root of every such piece in [0, h] whose
//   witness (projection on the expanded sphere / nearest circle point / the
//   triple point) is free, and whose witness distance crosses r_p in the
//   direction that leaves the end point's side (falling from an inside end,
//   rising from an outside end), is a candidate.  From an inside end point
//   the first candidate is the first root; from an outside end point the
//   first candidate that is not strictly outside M is.  Sphere roots come from the
//   quadratic, torus roots from the quartic
//     (|y-o|^2 + rho^2 - r_p^2)^2 = 4 rho^2 (|y-o|^2 - ((y-o).u)^2)
//   solved on [0, h] by root isolation on the derivative chain (quadratic ->
//   cubic -> quartic, monotone pieces) and safeguarded Newton-bisection,
//   keeping the near branch (|w| - rho)^2 + z^2 = r_p^2.  All in FP64.
// k_reduce: area = h^2 sum |n_a|, volume = h^2/3 sum of inside lengths.
#include <math.h>

#include "eses_kernels.h"
#include "eses_tile.cuh"

namespace eses {

constexpr int EDGE_THREADS = 256;

// --------------------------------------------------------------------------
// polynomial roots on an interval
// --------------------------------------------------------------------------
template <int DEG>
__device__ __forceinline__ double horner(const double *c, double t)
{
    double v = c[DEG];
#pragma unroll
    for (int k = DEG - 1; k >= 0; --k) v = fma(v, t, c[k]);
    return v;
}

// root of c on [a, b], where c is monotone and f(a) (= fa) and f(b) differ in sign
template <int DEG>
__device__ double mono_root(const double *c, double a, double b, double fa)
{
    double dc[DEG];
#pragma unroll
    for (int k = 0; k < DEG; ++k) dc[k] = (double)(k + 1) * c[k + 1];
    double t = 0.5 * (a + b);
    for (int it = 0; it < 100; ++it) {
        double f = horner<DEG>(c, t);
        if (f == 0.0) return t;
        if ((f < 0.0) == (fa < 0.0)) a = t;
        else b = t;
        double df = horner<DEG - 1>(dc, t);
        double tn = (df != 0.0) ? t - f / df : 0.5 * (a + b);
        if (!(tn > a && tn < b)) tn = 0.5 * (a + b);
        if (fabs(tn - t) <= 1e-15 * fmax(1.0, fabs(t))) return tn;
        t = tn;
        if (b - a <= 1e-15 * fmax(1.0, fabs(a))) return 0.5 * (a + b);
    }
    return t;
}

// roots of c[0] + c[1] t + ... + c[DEG] t^DEG in [lo, hi], ascending
template <int DEG>
struct PolyRoots {
    __device__ static int run(const double *c, double lo, double hi, double *out)
    {
        double dc[DEG];
#pragma unroll
        for (int k = 0; k < DEG; ++k) dc[k] = (double)(k + 1) * c[k + 1];
        double crit[DEG - 1];
        int ncr = PolyRoots<DEG - 1>::run(dc, lo, hi, crit);
        double pts[DEG + 1];
        int np = 0;
        pts[np++] = lo;
        for (int k = 0; k < ncr; ++k)
            if (crit[k] > pts[np - 1] && crit[k] < hi) pts[np++] = crit[k];
        pts[np++] = hi;
        int n = 0;
        double fprev = horner<DEG>(c, pts[0]);
        if (fprev == 0.0) out[n++] = pts[0];
        for (int k = 0; k + 1 < np; ++k) {
            double fnext = horner<DEG>(c, pts[k + 1]);
            if (fnext == 0.0) {
                if (n == 0 || out[n - 1] != pts[k + 1]) out[n++] = pts[k + 1];
            } else if (fprev != 0.0 && ((fprev < 0.0) != (fnext < 0.0))) {
                out[n++] = mono_root<DEG>(c, pts[k], pts[k + 1], fprev);
            }
            fprev = fnext;
        }
        return n;
    }
};

template <>
struct PolyRoots<1> {
    __device__ static int run(const double *c, double lo, double hi, double *out)
    {
        if (c[1] == 0.0) return 0;
        double t = -c[0] / c[1];
        if (t >= lo && t <= hi) {
            out[0] = t;
            return 1;
        }
        return 0;
    }
};

template <>
struct PolyRoots<2> {
    __device__ static int run(const double *c, double lo, double hi, double *out)
    {
        double a = c[2], b = c[1], cc = c[0];
        if (a == 0.0) return PolyRoots<1>::run(c, lo, hi, out);
        double disc = b * b - 4.0 * a * cc;
        if (disc < 0.0) return 0;
        double sq = sqrt(disc);
        double q = -0.5 * (b + (b >= 0.0 ? sq : -sq));
        double r1 = q / a;
        double r2 = (q != 0.0) ? cc / q : r1;
        if (r1 > r2) {
            double tmp = r1;
            r1 = r2;
            r2 = tmp;
        }
        int n = 0;
        if (r1 >= lo && r1 <= hi) out[n++] = r1;
        if (r2 >= lo && r2 <= hi && (n == 0 || r2 != out[0])) out[n++] = r2;
        return n;
    }
};

// --------------------------------------------------------------------------
// edge root
// --------------------------------------------------------------------------
// --------------------------------------------------------------------------
// edge root, one warp per edge
// --------------------------------------------------------------------------
constexpr int EDGE_WARPS = EDGE_THREADS / 32;
constexpr int WCAND = 64;  // candidate roots per warp

struct WCand {
    double t, qx, qy, qz;
    int kind, id;  // kind 0: van der Waals sphere (atom slot), 1: torus (pair slot), 2: probe sphere (vertex slot)
};

struct EdgeSmem {
    int8_t lab[9 * 9 * 9];
    short eptr[3 * TILE_PTS];  // crossing edges of the tile (local point), grouped by axis
    int estart[4];
    long long ebase[3];
    int sh[EDGE_WARPS];
    double shd[EDGE_WARPS];
    WCand cand[EDGE_WARPS][WCAND];
    int ncand[EDGE_WARPS];
};

__device__ __forceinline__ void warp_push(EdgeSmem &E, int warp, double t, double qx, double qy, double qz, int kind,
                                          int id)
{
    int slot = atomicAdd(&E.ncand[warp], 1);
    if (slot < WCAND) {
        WCand &c = E.cand[warp][slot];
        c.t = t;
        c.qx = qx;
        c.qy = qy;
        c.qz = qz;
        c.kind = kind;
        c.id = id;
    }
}

// index of the smallest t (ties: smaller index), -1 if every t is +inf
__device__ __forceinline__ int warp_argmin(const WCand *c, int n)
{
    const int lane = threadIdx.x & 31;
    double bt = INFINITY;
    int bk = -1;
    for (int k = lane; k < n; k += 32)
        if (c[k].t < bt) {
            bt = c[k].t;
            bk = k;
        }
    for (int o = 16; o > 0; o >>= 1) {
        double ot = __shfl_xor_sync(0xffffffffu, bt, o);
        int ok = __shfl_xor_sync(0xffffffffu, bk, o);
        if (ot < bt || (ot == bt && ok >= 0 && (bk < 0 || ok < bk))) {
            bt = ot;
            bk = ok;
        }
    }
    return bk;
}

// Candidate roots of one crossing edge (lower point s, local index p, +axis,
// length h), then the first root.  Sphere and torus roots are solved in FP64
// only for the pieces that an FP32 test (with a margin) lets through; the
// freeness of a witness is decided in FP32 when the filter allows and in FP64
// otherwise.  From an inside end point the answer is the first candidate; from
// an outside end point it is the first candidate at which no free probe centre
// lies strictly closer than r_p (within 1e-11 A).
template <class T, bool FILT>
__device__ int warp_edge(const Model &M, const TileS<T> &S, const double *x0, EdgeSmem &E, int warp, int axis, int p,
                         int lab_s, double h, double rp, T d0, double &t_out, double q_out[3])
{
    const int lane = threadIdx.x & 31;
    const int li = p >> 6, lj = (p >> 3) & 7, lk = p & 7;
    const double s64[3] = {(double)li * h, (double)lj * h, (double)lk * h};
    const T s[3] = {(T)s64[0], (T)s64[1], (T)s64[2]};
    SmemAcc<T> A(S);
    ExactAcc<T> X(S, M, x0);
    if (lane == 0) E.ncand[warp] = 0;
    __syncwarp();
    const int na = S.na, nv = S.nv, np = S.np;
    const T hT = (T)h, rpT = (T)rp;
    const T mg = FILT ? T(2e-3) : T(0);  // margin of the FP32 prefilters (A)
    const T fd = d0 + T(2e-6);            // error of an FP64 witness rounded into the tile frame
    const bool inside = lab_s == LABEL_IN;
    for (int it = lane; it < na + nv + np; it += 32) {
        if (it < na) {  // convex: van der Waals sphere, witness = projection on the expanded sphere
            P4<T> c = S.atom[it];
            T d[3] = {s[0] - c.x, s[1] - c.y, s[2] - c.z};
            T dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            T reach = c.w + hT + mg;
            if (dd > reach * reach) continue;
            T b = d[axis], disc = b * b - (dd - c.w * c.w);
            if (disc < -mg) continue;
            T sq = sqrt(fmax(disc, T(0)) + mg);
            if (-b + sq < -mg || -b - sq > hT + mg) continue;
            P4<double> ce = X.atom(it);
            double de[3] = {s64[0] - ce.x, s64[1] - ce.y, s64[2] - ce.z};
            double co[3] = {de[0] * de[0] + de[1] * de[1] + de[2] * de[2] - ce.w * ce.w, 2.0 * de[axis], 1.0};
            double rt[2];
            int nr = PolyRoots<2>::run(co, 0.0, h, rt);
            for (int k = 0; k < nr; ++k) {
                double v[3] = {de[0], de[1], de[2]};
                v[axis] += rt[k];
                double nvv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
                if (!(nvv > 0.0)) continue;
                // the witness distance R - |y - c| must fall from an inside end point
                // and rise from an outside one
                double rate = -v[axis] / nvv;
                if (inside ? rate > 1e-9 : rate < -1e-9) continue;
                double R = ce.w + rp;
                double q[3] = {ce.x + R * v[0] / nvv, ce.y + R * v[1] / nvv, ce.z + R * v[2] / nvv};
                int f = FILT ? free_pt<true>(A, (T)q[0], (T)q[1], (T)q[2], S.agid[it], -1, rpT, fd) : -1;
                if (f < 0) f = free_pt<false>(X, q[0], q[1], q[2], S.agid[it], -1, rp, 0.0);
                if (f == 1) warp_push(E, warp, rt[k], q[0], q[1], q[2], 0, it);
            }
        } else if (it < na + nv) {  // concave: probe sphere around a free triple point
            const int vi = it - na;
            P4<T> c = S.vq[vi];
            T d[3] = {s[0] - c.x, s[1] - c.y, s[2] - c.z};
            T dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            T reach = rpT + hT + mg;
            if (dd > reach * reach) continue;
            T b = d[axis], disc = b * b - (dd - rpT * rpT);
            if (disc < -mg) continue;
            T sq = sqrt(fmax(disc, T(0)) + mg);
            if (-b + sq < -mg || -b - sq > hT + mg) continue;
            P4<double> ce = X.vq(vi);
            double de[3] = {s64[0] - ce.x, s64[1] - ce.y, s64[2] - ce.z};
            double co[3] = {de[0] * de[0] + de[1] * de[1] + de[2] * de[2] - rp * rp, 2.0 * de[axis], 1.0};
            double rt[2];
            int nr = PolyRoots<2>::run(co, 0.0, h, rt);
            for (int k = 0; k < nr; ++k) {
                double rate = (de[axis] + rt[k]) / rp;  // d|y - v|/dt
                if (inside ? rate > 1e-9 : rate < -1e-9) continue;
                warp_push(E, warp, rt[k], ce.x, ce.y, ce.z, 2, vi);
            }
        } else {  // saddle: torus around a free-arc circle
            const int pi = it - na - nv;
            P4<T> o = S.po[pi];
            P4<T> u = S.pu[pi];
            // 1-Lipschitz distance to the circle, checked at the edge midpoint
            T m[3] = {s[0] - o.x, s[1] - o.y, s[2] - o.z};
            m[axis] += T(0.5) * hT;
            T zc = m[0] * u.x + m[1] * u.y + m[2] * u.z;
            T w2 = fmax(m[0] * m[0] + m[1] * m[1] + m[2] * m[2] - zc * zc, T(0));
            T e1 = sqrt(w2) - o.w;
            T gm = sqrt(e1 * e1 + zc * zc) - rpT;
            if (fabs(gm) > T(0.5) * hT + mg) continue;
            P4<double> oe = X.po(pi);
            P4<double> ue = X.pu(pi);
            const double rho = oe.w;
            double p0[3] = {s64[0] - oe.x, s64[1] - oe.y, s64[2] - oe.z};
            double uu[3] = {ue.x, ue.y, ue.z};
            double P = p0[0] * p0[0] + p0[1] * p0[1] + p0[2] * p0[2];
            double z0 = p0[0] * uu[0] + p0[1] * uu[1] + p0[2] * uu[2];
            double pe = p0[axis], eu = uu[axis];
            double K = P + rho * rho - rp * rp;
            double r2 = rho * rho;
            double co[5];
            co[4] = 1.0;
            co[3] = 4.0 * pe;
            co[2] = 4.0 * pe * pe + 2.0 * K - 4.0 * r2 * (1.0 - eu * eu);
            co[1] = 4.0 * pe * K - 8.0 * r2 * (pe - z0 * eu);
            co[0] = K * K - 4.0 * r2 * (P - z0 * z0);
            double rt[4];
            int nr = PolyRoots<4>::run(co, 0.0, h, rt);
            for (int k = 0; k < nr; ++k) {
                double y[3] = {p0[0], p0[1], p0[2]};
                y[axis] += rt[k];
                double zy = y[0] * uu[0] + y[1] * uu[1] + y[2] * uu[2];
                double w[3] = {y[0] - zy * uu[0], y[1] - zy * uu[1], y[2] - zy * uu[2]};
                double nw = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
                double near2 = (nw - rho) * (nw - rho) + zy * zy;
                if (fabs(near2 - rp * rp) > 1e-7 * rp * rp) continue;  // far branch of the quartic
                if (!(nw > 0.0)) continue;
                double rate = ((nw - rho) * w[axis] / nw + zy * uu[axis]) / rp;
                if (inside ? rate > 1e-9 : rate < -1e-9) continue;
                double q[3] = {oe.x + rho * w[0] / nw, oe.y + rho * w[1] / nw, oe.z + rho * w[2] / nw};
                int2 ij = S.pij[pi];
                int f = FILT ? free_pt<true>(A, (T)q[0], (T)q[1], (T)q[2], ij.x, ij.y, rpT, fd) : -1;
                if (f < 0) f = free_pt<false>(X, q[0], q[1], q[2], ij.x, ij.y, rp, 0.0);
                if (f == 1) warp_push(E, warp, rt[k], q[0], q[1], q[2], 1, pi);
            }
        }
    }
    __syncwarp();
    int n = E.ncand[warp];
    int status = n > WCAND ? 2 : 0;  // 2: candidate buffer overflow
    if (n > WCAND) n = WCAND;
    WCand *c = E.cand[warp];
    int pick = -1;
    if (inside) {
        pick = warp_argmin(c, n);
    } else {
        for (int iter = 0; iter < n; ++iter) {
            int k = warp_argmin(c, n);
            if (k < 0) break;
            double y[3] = {s64[0], s64[1], s64[2]};
            y[axis] += c[k].t;
            int r;
            if (FILT) {
                r = warp_witness<true>(A, (T)y[0], (T)y[1], (T)y[2], rpT, rpT, d0, c[k].kind, c[k].id);
                if (r < 0) r = warp_witness<false>(X, y[0], y[1], y[2], rp, rp - 1e-11, 0.0, -1, -1);
            } else {
                r = warp_witness<false>(X, y[0], y[1], y[2], rp, rp - 1e-11, 0.0, -1, -1);
            }
            if (r == 0) {
                pick = k;
                break;
            }
            __syncwarp();
            if (lane == 0) c[k].t = INFINITY;  // strictly outside M: not the root
            __syncwarp();
        }
    }
    if (pick < 0) return 1;
    t_out = c[pick].t;
    q_out[0] = c[pick].qx;
    q_out[1] = c[pick].qy;
    q_out[2] = c[pick].qz;
    return status;
}

// --------------------------------------------------------------------------
// kernels
// --------------------------------------------------------------------------
__device__ __forceinline__ int block_sum_int(int v, int *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    int tot = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tot += sh[k];
    __syncthreads();
    return tot;
}

__device__ __forceinline__ double block_sum_double(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double tot = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tot += sh[k];  // fixed order: deterministic
    __syncthreads();
    return tot;
}

__global__ void __launch_bounds__(EDGE_THREADS) k_edge_count(Grid G, const int8_t *__restrict__ labels,
                                                             int *__restrict__ tile_edges,
                                                             int *__restrict__ tile_inside)
{
    __shared__ int sh[EDGE_THREADS / 32];
    const long long nt = G.n_tiles;
    const long long st1 = G.dims[2], st0 = G.dims[1] * G.dims[2];
    for (long long tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        int t[3];
        tile_coords(G, tile, t);
        int ce[3] = {0, 0, 0}, ci[3] = {0, 0, 0}, npin = 0;
        for (int p = threadIdx.x; p < TILE_PTS; p += EDGE_THREADS) {
            long long g[3] = {(long long)TILE * t[0] + (p >> 6), (long long)TILE * t[1] + ((p >> 3) & 7),
                              (long long)TILE * t[2] + (p & 7)};
            if (g[0] >= G.dims[0] || g[1] >= G.dims[1] || g[2] >= G.dims[2]) continue;
            long long idx = g[0] * st0 + g[1] * st1 + g[2];
            int l0 = labels[idx];
            npin += l0;
            const long long str[3] = {st0, st1, 1};
            for (int a = 0; a < 3; ++a) {
                if (g[a] + 1 >= G.dims[a]) continue;
                int l1 = labels[idx + str[a]];
                if (l0 != l1) ++ce[a];
                else if (l0) ++ci[a];
            }
        }
        for (int a = 0; a < 3; ++a) {
            int e = block_sum_int(ce[a], sh);
            int i = block_sum_int(ci[a], sh);
            if (threadIdx.x == 0) {
                tile_edges[a * nt + tile] = e;
                tile_inside[a * nt + tile] = i;
            }
        }
        int pin = block_sum_int(npin, sh);
        if (threadIdx.x == 0) tile_inside[3 * nt + tile] = pin;
    }
}

__device__ __forceinline__ int block_excl_scan_e(int v, int *sh, int *total)
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

template <class T, bool FILT>
__global__ void __launch_bounds__(EDGE_THREADS) k_edge_solve(Model M, Grid G, const int8_t *__restrict__ labels,
                                                             const int *__restrict__ edge_start, EdgeOut out,
                                                             double *__restrict__ tile_area,
                                                             double *__restrict__ tile_vol, int *__restrict__ n_fail,
                                                             int *__restrict__ err, long long *__restrict__ fail_log)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileS<T> &S = *reinterpret_cast<TileS<T> *>(smem_raw);
    EdgeSmem &E = *reinterpret_cast<EdgeSmem *>(smem_raw + ((sizeof(TileS<T>) + 15) & ~(size_t)15));
    const long long nt = G.n_tiles;
    const long long st1 = G.dims[2], st0 = G.dims[1] * G.dims[2];
    const double h = G.h, rp = M.rp;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const T d0 = FILT ? (T)G.d0 : T(0);
    for (long long tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        int tot = 0;
        for (int a = 0; a < 3; ++a) tot += edge_start[a * nt + tile + 1] - edge_start[a * nt + tile];
        if (tot == 0) {
            if (threadIdx.x == 0) {
                tile_area[tile] = 0.0;
                tile_vol[tile] = 0.0;
            }
            continue;
        }
        double x0[3];
        stage_tile<T>(M, G, tile, S, x0);
        if (threadIdx.x == 0 && S.flags) atomicOr(err, S.flags);
        int t[3];
        tile_coords(G, tile, t);
        // labels of the tile and of the next layer (9^3), -1 outside the grid
        for (int q = threadIdx.x; q < 729; q += EDGE_THREADS) {
            int li = q / 81, lj = (q / 9) % 9, lk = q % 9;
            long long g[3] = {(long long)TILE * t[0] + li, (long long)TILE * t[1] + lj, (long long)TILE * t[2] + lk};
            int8_t v = -1;
            if (g[0] < G.dims[0] && g[1] < G.dims[1] && g[2] < G.dims[2]) v = labels[g[0] * st0 + g[1] * st1 + g[2]];
            E.lab[q] = v;
        }
        if (threadIdx.x == 0) E.estart[0] = 0;
        __syncthreads();
        // the tile's crossing edges, axis by axis, in point order
        for (int a = 0; a < 3; ++a) {
            int flag[2];
            for (int k = 0; k < 2; ++k) {
                int q = 2 * threadIdx.x + k;
                int l[3] = {q >> 6, (q >> 3) & 7, q & 7};
                int8_t l0 = E.lab[(l[0] * 9 + l[1]) * 9 + l[2]];
                l[a] += 1;
                int8_t l1 = E.lab[(l[0] * 9 + l[1]) * 9 + l[2]];
                flag[k] = (l0 >= 0 && l1 >= 0 && l0 != l1) ? 1 : 0;
            }
            int tsum;
            int rank = block_excl_scan_e(flag[0] + flag[1], E.sh, &tsum);
            const int base = E.estart[a];
            for (int k = 0; k < 2; ++k)
                if (flag[k]) E.eptr[base + rank++] = (short)(2 * threadIdx.x + k);
            if (threadIdx.x == 0) {
                E.estart[a + 1] = base + tsum;
                E.ebase[a] = (long long)edge_start[a * nt + tile] - edge_start[a * nt];
            }
            __syncthreads();
        }
        double area = 0.0, vol = 0.0;
        const int ne = E.estart[3];
        for (int e = warp; e < ne; e += EDGE_WARPS) {
            const int a = e < E.estart[1] ? 0 : (e < E.estart[2] ? 1 : 2);
            const int q = E.eptr[e];
            const int li = q >> 6, lj = (q >> 3) & 7, lk = q & 7;
            const int lab_s = E.lab[(li * 9 + lj) * 9 + lk];
            double tr = 0.5 * h, qq[3] = {0.0, 0.0, 0.0};
            int status = warp_edge<T, FILT>(M, S, x0, E, warp, a, q, lab_s, h, rp, d0, tr, qq);
            if (lane == 0) {
                double nrm[3] = {0.0, 0.0, 0.0};
                if (status != 1) {
                    double y[3] = {(double)li * h, (double)lj * h, (double)lk * h};
                    y[a] += tr;
                    double v[3] = {qq[0] - y[0], qq[1] - y[1], qq[2] - y[2]};
                    double nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
                    if (nv > 0.0) {
                        nrm[0] = v[0] / nv;
                        nrm[1] = v[1] / nv;
                        nrm[2] = v[2] / nv;
                    }
                }
                if (status != 0) {
                    atomicOr(err, status == 1 ? ERR_ROOT : ERR_CAP_CAND);
                    if (status == 1) {
                        int slot = atomicAdd(n_fail, 1);
                        if (slot < FAIL_LOG) {
                            long long *rec = fail_log + FAIL_REC * slot;
                            for (int z = 0; z < FAIL_REC; ++z) rec[z] = 0;
                            rec[0] = a;
                            rec[1] = (long long)TILE * t[0] + li;
                            rec[2] = (long long)TILE * t[1] + lj;
                            rec[3] = (long long)TILE * t[2] + lk;
                            rec[4] = lab_s;
                            rec[5] = S.na;
                            rec[6] = S.np;
                            rec[7] = S.nv;
                            rec[8] = E.ncand[warp];
                            for (int z = 0; z < 7 && z < E.ncand[warp] && z < WCAND; ++z) {
                                rec[9 + z] = (long long)(E.cand[warp][z].t * 1e9);
                                rec[16 + z] = E.cand[warp][z].kind;
                            }
                        }
                    }
                }
                const long long o = E.ebase[a] + (e - E.estart[a]);
                out.idx[a][o] = (long long)(TILE * t[0] + li) * st0 + (long long)(TILE * t[1] + lj) * st1 +
                                (TILE * t[2] + lk);
                out.tau[a][o] = tr / h;
                out.nrm[a][3 * o + 0] = nrm[0];
                out.nrm[a][3 * o + 1] = nrm[1];
                out.nrm[a][3 * o + 2] = nrm[2];
                out.tau32[a][o] = (float)(tr / h);
                out.nrm32[a][3 * o + 0] = (float)nrm[0];
                out.nrm32[a][3 * o + 1] = (float)nrm[1];
                out.nrm32[a][3 * o + 2] = (float)nrm[2];
                area += h * h * fabs(nrm[a]);
                vol += lab_s == LABEL_IN ? tr : h - tr;
            }
            __syncwarp();
        }
        double ta = block_sum_double(area, E.shd);
        double tv = block_sum_double(vol, E.shd);
        if (threadIdx.x == 0) {
            tile_area[tile] = ta;
            tile_vol[tile] = tv;
        }
        __syncthreads();
    }
}

// single-block deterministic reduction: out2 = {area, volume};
// counts = {inside points, inside edges (all axes), crossing edges}
__global__ void __launch_bounds__(1024) k_reduce(Grid G, const double *__restrict__ tile_area,
                                                 const double *__restrict__ tile_vol,
                                                 const int *__restrict__ tile_inside, double *__restrict__ out2,
                                                 long long *__restrict__ counts)
{
    __shared__ double sa[32], sv[32];
    __shared__ long long si[32], sp[32];
    const long long nt = G.n_tiles;
    double a = 0.0, v = 0.0;
    long long ie = 0, pin = 0;
    for (long long k = threadIdx.x; k < nt; k += blockDim.x) {
        a += tile_area[k];
        v += tile_vol[k];
        ie += (long long)tile_inside[k] + tile_inside[nt + k] + tile_inside[2 * nt + k];
        pin += tile_inside[3 * nt + k];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        v += __shfl_down_sync(0xffffffffu, v, o);
        ie += __shfl_down_sync(0xffffffffu, ie, o);
        pin += __shfl_down_sync(0xffffffffu, pin, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sa[wid] = a;
        sv[wid] = v;
        si[wid] = ie;
        sp[wid] = pin;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double A = 0.0, V = 0.0;
        long long IE = 0, P = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            A += sa[k];
            V += sv[k];
            IE += si[k];
            P += sp[k];
        }
        out2[0] = A;
        out2[1] = G.h * G.h * (V + G.h * (double)IE) / 3.0;
        counts[0] = P;
        counts[1] = IE;
    }
}

static int grid_tiles(long long n)
{
    long long g = n < 1 ? 1 : n;
    return (int)(g > 2147483647LL ? 2147483647LL : g);
}

int launch_edge_count(const Grid &G, const int8_t *labels, int *tile_edges, int *tile_inside, cudaStream_t st)
{
    k_edge_count<<<grid_tiles(G.n_tiles), EDGE_THREADS, 0, st>>>(G, labels, tile_edges, tile_inside);
    return 1;
}

template <class T, bool FILT>
static void edge_solve_launch(const Model &M, const Grid &G, const int8_t *labels, const int *edge_start, EdgeOut out,
                              double *tile_area, double *tile_vol, int *n_fail, int *err, long long *fail_log,
                              cudaStream_t st)
{
    size_t sm = ((sizeof(TileS<T>) + 15) & ~(size_t)15) + sizeof(EdgeSmem);
    cudaFuncSetAttribute(k_edge_solve<T, FILT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_edge_solve<T, FILT><<<grid_tiles(G.n_tiles), EDGE_THREADS, sm, st>>>(M, G, labels, edge_start, out, tile_area,
                                                                           tile_vol, n_fail, err, fail_log);
}

int launch_edge_solve(const Model &M, const Grid &G, int precision, const int8_t *labels, const int *edge_start,
                      EdgeOut out, double *tile_area, double *tile_vol, int *n_fail, int *err, long long *fail_log,
                      cudaStream_t st)
{
    if (precision == 0)
        edge_solve_launch<double, false>(M, G, labels, edge_start, out, tile_area, tile_vol, n_fail, err, fail_log, st);
    else
        edge_solve_launch<float, true>(M, G, labels, edge_start, out, tile_area, tile_vol, n_fail, err, fail_log, st);
    return 1;
}

int launch_reduce(const Grid &G, const double *tile_area, const double *tile_vol, const int *tile_inside,
                   const int8_t *, double *out2, long long *counts, cudaStream_t st)
{
    k_reduce<<<1, 1024, 0, st>>>(G, tile_area, tile_vol, tile_inside, out2, counts);
    return 1;
}

}  // namespace eses
