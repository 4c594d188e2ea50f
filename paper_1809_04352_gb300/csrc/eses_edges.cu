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
constexpr int MAX_CAND = 32;

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
struct Cand {
    double t, qx, qy, qz;
};

__device__ __forceinline__ void push_cand(Cand *c, int &nc, double t, double qx, double qy, double qz)
{
    // keep the MAX_CAND smallest t, ascending
    int k = nc < MAX_CAND ? nc : MAX_CAND - 1;
    if (nc >= MAX_CAND && t >= c[MAX_CAND - 1].t) return;
    while (k > 0 && c[k - 1].t > t) {
        c[k] = c[k - 1];
        --k;
    }
    c[k].t = t;
    c[k].qx = qx;
    c[k].qy = qy;
    c[k].qz = qz;
    if (nc < MAX_CAND) ++nc;
}

// First surface root on the edge from s (tile frame) along +axis, length h.
// lab_s is the label of s.  Returns false when no root is found.
// dbg (optional, 16 counters): [0] sphere roots, [1] sphere witness covered,
// [2] probe-sphere roots, [3] tori tested, [4] quartic roots, [5] far-branch
// roots, [6] torus witness covered, [7] candidates, [8] candidates rejected by
// validation, [9..15] t of the first candidates (x 1e9, truncated)
__device__ bool edge_root(const TileS<double> &S, const double s[3], int axis, double h, double rp, int lab_s,
                          double &t_out, double q_out[3], long long *dbg = nullptr)
{
    Cand c[MAX_CAND];
    int nc = 0;
    // convex: van der Waals spheres, witness = projection on the expanded sphere
    for (int a = 0; a < S.na; ++a) {
        P4<double> at = S.atom[a];
        double d[3] = {s[0] - at.x, s[1] - at.y, s[2] - at.z};
        double b = d[axis];
        double cc = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] - at.w * at.w;
        double disc = b * b - cc;
        if (disc < 0.0) continue;
        double co[3] = {cc, 2.0 * b, 1.0};
        double rt[2];
        int nr = PolyRoots<2>::run(co, 0.0, h, rt);
        for (int k = 0; k < nr; ++k) {
            double y[3] = {s[0], s[1], s[2]};
            y[axis] += rt[k];
            double v[3] = {y[0] - at.x, y[1] - at.y, y[2] - at.z};
            double nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            if (!(nv > 0.0)) continue;
            // the witness distance R - |y - c| must cross r_p the right way:
            // rising (leaving the outside of M) from an outside end point,
            // falling from an inside one
            double rate = -v[axis] / nv;
            if (lab_s == LABEL_IN ? rate > 1e-9 : rate < -1e-9) continue;
            double R = at.w + rp;
            double qx = at.x + R * v[0] / nv, qy = at.y + R * v[1] / nv, qz = at.z + R * v[2] / nv;
            if (dbg) dbg[0]++;
            if (free_pt<double, false>(qx, qy, qz, S, S.agid[a], -1, rp, 0.0) == 1) push_cand(c, nc, rt[k], qx, qy, qz);
            else if (dbg) dbg[1]++;
        }
    }
    // concave: probe spheres around free triple points
    for (int v = 0; v < S.nv; ++v) {
        P4<double> q = S.vq[v];
        double d[3] = {s[0] - q.x, s[1] - q.y, s[2] - q.z};
        double b = d[axis];
        double cc = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] - rp * rp;
        if (b * b - cc < 0.0) continue;
        double co[3] = {cc, 2.0 * b, 1.0};
        double rt[2];
        int nr = PolyRoots<2>::run(co, 0.0, h, rt);
        if (dbg) dbg[2] += nr;
        for (int k = 0; k < nr; ++k) {
            double rate = (d[axis] + rt[k]) / rp;  // d|y - v|/dt at the root
            if (lab_s == LABEL_IN ? rate > 1e-9 : rate < -1e-9) continue;
            push_cand(c, nc, rt[k], q.x, q.y, q.z);
        }
    }
    // saddle: tori around free-arc circles
    for (int p = 0; p < S.np; ++p) {
        P4<double> o = S.po[p];
        P4<double> u = S.pu[p];
        const double rho = o.w;
        double p0[3] = {s[0] - o.x, s[1] - o.y, s[2] - o.z};
        double uu[3] = {u.x, u.y, u.z};
        double P = p0[0] * p0[0] + p0[1] * p0[1] + p0[2] * p0[2];
        double z0 = p0[0] * u.x + p0[1] * u.y + p0[2] * u.z;
        // quick reject: the tube around the circle must come within reach of the edge
        double w0 = sqrt(fmax(P - z0 * z0, 0.0));
        double dmid = sqrt((w0 - rho) * (w0 - rho) + z0 * z0);
        if (dmid - rp > h + 1e-9 || rp - dmid > h + 1e-9) continue;  // 1-Lipschitz along the edge
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
        if (dbg) {
            dbg[3]++;
            dbg[4] += nr;
        }
        for (int k = 0; k < nr; ++k) {
            double y[3] = {p0[0], p0[1], p0[2]};
            y[axis] += rt[k];
            double zc = y[0] * u.x + y[1] * u.y + y[2] * u.z;
            double w[3] = {y[0] - zc * u.x, y[1] - zc * u.y, y[2] - zc * u.z};
            double nw = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
            double near2 = (nw - rho) * (nw - rho) + zc * zc;
            if (fabs(near2 - rp * rp) > 1e-7 * rp * rp) {  // far branch of the quartic
                if (dbg) dbg[5]++;
                continue;
            }
            if (!(nw > 0.0)) continue;
            // d/dt of the distance to the circle: ((|w| - rho) w_a / |w| + z u_a) / r_p
            double rate = ((nw - rho) * w[axis] / nw + zc * uu[axis]) / rp;
            if (lab_s == LABEL_IN ? rate > 1e-9 : rate < -1e-9) continue;
            double qx = o.x + rho * w[0] / nw, qy = o.y + rho * w[1] / nw, qz = o.z + rho * w[2] / nw;
            int2 ij = S.pij[p];
            if (free_pt<double, false>(qx, qy, qz, S, ij.x, ij.y, rp, 0.0) == 1) push_cand(c, nc, rt[k], qx, qy, qz);
            else if (dbg) dbg[6]++;
        }
    }
    if (dbg) {
        dbg[7] = nc;
        for (int k = 0; k < nc && k < 7; ++k) dbg[9 + k] = (long long)(c[k].t * 1e9);
    }
    if (nc == 0) return false;
    int pick = -1;
    if (lab_s == LABEL_IN) {
        pick = 0;
    } else {
        for (int k = 0; k < nc; ++k) {
            double y[3] = {s[0], s[1], s[2]};
            y[axis] += c[k].t;
            // not strictly outside M: no free centre closer than r_p - 1e-11
            if (classify_pt<double, false>(y[0], y[1], y[2], S, rp, rp - 1e-11, 0.0) == 1) {
                pick = k;
                break;
            }
            if (dbg) dbg[8]++;
        }
    }
    if (pick < 0) return false;
    t_out = c[pick].t;
    q_out[0] = c[pick].qx;
    q_out[1] = c[pick].qy;
    q_out[2] = c[pick].qz;
    return true;
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

struct EdgeSmem {
    int8_t lab[9 * 9 * 9];
    int sh[EDGE_THREADS / 32];
    double shd[EDGE_THREADS / 32];
};

__global__ void __launch_bounds__(EDGE_THREADS) k_edge_solve(Model M, Grid G, const int8_t *__restrict__ labels,
                                                             const int *__restrict__ edge_start, EdgeOut out,
                                                             double *__restrict__ tile_area,
                                                             double *__restrict__ tile_vol, int *__restrict__ n_fail,
                                                             int *__restrict__ err, long long *__restrict__ fail_log)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileS<double> &S = *reinterpret_cast<TileS<double> *>(smem_raw);
    __shared__ EdgeSmem E;
    const long long nt = G.n_tiles;
    const long long st1 = G.dims[2], st0 = G.dims[1] * G.dims[2];
    const double h = G.h, rp = M.rp;
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
        stage_tile<double>(M, G, tile, S, x0);
        if (threadIdx.x == 0 && S.flags) atomicOr(err, S.flags);
        int t[3];
        tile_coords(G, tile, t);
        // labels of the tile and of the next layer (9^3), -1 outside the grid
        for (int p = threadIdx.x; p < 729; p += EDGE_THREADS) {
            int li = p / 81, lj = (p / 9) % 9, lk = p % 9;
            long long g[3] = {(long long)TILE * t[0] + li, (long long)TILE * t[1] + lj, (long long)TILE * t[2] + lk};
            int8_t v = -1;
            if (g[0] < G.dims[0] && g[1] < G.dims[1] && g[2] < G.dims[2]) v = labels[g[0] * st0 + g[1] * st1 + g[2]];
            E.lab[p] = v;
        }
        __syncthreads();
        double area = 0.0, vol = 0.0;
        for (int a = 0; a < 3; ++a) {
            const long long base = (long long)edge_start[a * nt + tile] - edge_start[a * nt];
            // two consecutive points per thread keep the output in point order
            int flag[2];
            for (int k = 0; k < 2; ++k) {
                int p = 2 * threadIdx.x + k;
                int li = p >> 6, lj = (p >> 3) & 7, lk = p & 7;
                int l[3] = {li, lj, lk};
                int8_t l0 = E.lab[(li * 9 + lj) * 9 + lk];
                l[a] += 1;
                int8_t l1 = E.lab[(l[0] * 9 + l[1]) * 9 + l[2]];
                flag[k] = (l0 >= 0 && l1 >= 0 && l0 != l1) ? 1 : 0;
            }
            int tsum;
            int rank = block_excl_scan_e(flag[0] + flag[1], E.sh, &tsum);
            for (int k = 0; k < 2; ++k) {
                if (!flag[k]) continue;
                int p = 2 * threadIdx.x + k;
                int li = p >> 6, lj = (p >> 3) & 7, lk = p & 7;
                int lab_s = E.lab[(li * 9 + lj) * 9 + lk];
                double s[3] = {(double)li * h, (double)lj * h, (double)lk * h};
                double tr = 0.5 * h, q[3] = {0.0, 0.0, 0.0};
                double nrm[3] = {0.0, 0.0, 0.0};
                if (edge_root(S, s, a, h, rp, lab_s, tr, q)) {
                    double y[3] = {s[0], s[1], s[2]};
                    y[a] += tr;
                    double v[3] = {q[0] - y[0], q[1] - y[1], q[2] - y[2]};
                    double nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
                    if (nv > 0.0) {
                        nrm[0] = v[0] / nv;
                        nrm[1] = v[1] / nv;
                        nrm[2] = v[2] / nv;
                    }
                } else {
                    int slot = atomicAdd(n_fail, 1);
                    atomicOr(err, ERR_ROOT);
                    if (slot < FAIL_LOG) {
                        long long *rec = fail_log + FAIL_REC * slot;
                        for (int z = 0; z < FAIL_REC; ++z) rec[z] = 0;
                        double tt, qq[3];
                        edge_root(S, s, a, h, rp, lab_s, tt, qq, rec + 8);
                        rec[0] = a;
                        rec[1] = (long long)TILE * t[0] + li;
                        rec[2] = (long long)TILE * t[1] + lj;
                        rec[3] = (long long)TILE * t[2] + lk;
                        rec[4] = lab_s;
                        rec[5] = S.na;
                        rec[6] = S.np;
                        rec[7] = S.nv;
                    }
                }
                long long g[3] = {(long long)TILE * t[0] + li, (long long)TILE * t[1] + lj,
                                  (long long)TILE * t[2] + lk};
                long long o = base + rank;
                out.idx[a][o] = g[0] * st0 + g[1] * st1 + g[2];
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
                ++rank;
            }
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

int launch_edge_solve(const Model &M, const Grid &G, const int8_t *labels, const int *edge_start, EdgeOut out,
                       double *tile_area, double *tile_vol, int *n_fail, int *err, long long *fail_log,
                       cudaStream_t st)
{
    size_t sm = sizeof(TileS<double>);
    cudaFuncSetAttribute(k_edge_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_edge_solve<<<grid_tiles(G.n_tiles), EDGE_THREADS, sm, st>>>(M, G, labels, edge_start, out, tile_area, tile_vol,
                                                                  n_fail, err, fail_log);
    return 1;
}

int launch_reduce(const Grid &G, const double *tile_area, const double *tile_vol, const int *tile_inside,
                   const int8_t *, double *out2, long long *counts, cudaStream_t st)
{
    k_reduce<<<1, 1024, 0, st>>>(G, tile_area, tile_vol, tile_inside, out2, counts);
    return 1;
}

}  // namespace eses
