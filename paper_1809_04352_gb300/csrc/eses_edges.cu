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
template <class R>
__device__ __forceinline__ R root_eps();
template <>
__device__ __forceinline__ double root_eps<double>() { return 1e-15; }
template <>
__device__ __forceinline__ float root_eps<float>() { return 2e-7f; }

template <class R, int DEG>
__device__ __forceinline__ R horner(const R *c, R t)
{
    R v = c[DEG];
#pragma unroll
    for (int k = DEG - 1; k >= 0; --k) v = fma(v, t, c[k]);
    return v;
}

// root of c on [a, b], where c is monotone and f(a) (= fa) and f(b) differ in sign
template <class R, int DEG>
__device__ R mono_root(const R *c, R a, R b, R fa)
{
    R dc[DEG];
#pragma unroll
    for (int k = 0; k < DEG; ++k) dc[k] = (R)(k + 1) * c[k + 1];
    R t = R(0.5) * (a + b);
    for (int it = 0; it < 100; ++it) {
        R f = horner<R, DEG>(c, t);
        if (f == R(0)) return t;
        if ((f < R(0)) == (fa < R(0))) a = t;
        else b = t;
        R df = horner<R, DEG - 1>(dc, t);
        R tn = (df != R(0)) ? t - f / df : R(0.5) * (a + b);
        if (!(tn > a && tn < b)) tn = R(0.5) * (a + b);
        if (fabs(tn - t) <= root_eps<R>() * fmax(R(1), fabs(t))) return tn;
        t = tn;
        if (b - a <= root_eps<R>() * fmax(R(1), fabs(a))) return R(0.5) * (a + b);
    }
    return t;
}

// roots of c[0] + c[1] t + ... + c[DEG] t^DEG in [lo, hi], ascending: the
// derivative's roots split [lo, hi] into monotone pieces, each holding at most
// one root, found by safeguarded Newton-bisection
template <class R, int DEG>
struct PolyRoots {
    __device__ static int run(const R *c, R lo, R hi, R *out)
    {
        R dc[DEG];
#pragma unroll
        for (int k = 0; k < DEG; ++k) dc[k] = (R)(k + 1) * c[k + 1];
        R crit[DEG - 1];
        int ncr = PolyRoots<R, DEG - 1>::run(dc, lo, hi, crit);
        R pts[DEG + 1];
        int np = 0;
        pts[np++] = lo;
        for (int k = 0; k < ncr; ++k)
            if (crit[k] > pts[np - 1] && crit[k] < hi) pts[np++] = crit[k];
        pts[np++] = hi;
        int n = 0;
        R fprev = horner<R, DEG>(c, pts[0]);
        if (fprev == R(0)) out[n++] = pts[0];
        for (int k = 0; k + 1 < np; ++k) {
            R fnext = horner<R, DEG>(c, pts[k + 1]);
            if (fnext == R(0)) {
                if (n == 0 || out[n - 1] != pts[k + 1]) out[n++] = pts[k + 1];
            } else if (fprev != R(0) && ((fprev < R(0)) != (fnext < R(0)))) {
                out[n++] = mono_root<R, DEG>(c, pts[k], pts[k + 1], fprev);
            }
            fprev = fnext;
        }
        return n;
    }
};

template <class R>
struct PolyRoots<R, 1> {
    __device__ static int run(const R *c, R lo, R hi, R *out)
    {
        if (c[1] == R(0)) return 0;
        R t = -c[0] / c[1];
        if (t >= lo && t <= hi) {
            out[0] = t;
            return 1;
        }
        return 0;
    }
};

template <class R>
struct PolyRoots<R, 2> {
    __device__ static int run(const R *c, R lo, R hi, R *out)
    {
        R a = c[2], b = c[1], cc = c[0];
        if (a == R(0)) return PolyRoots<R, 1>::run(c, lo, hi, out);
        R disc = b * b - R(4) * a * cc;
        if (disc < R(0)) return 0;
        R sq = sqrt(disc);
        R q = R(-0.5) * (b + (b >= R(0) ? sq : -sq));
        R r1 = q / a;
        R r2 = (q != R(0)) ? cc / q : r1;
        if (r1 > r2) {
            R tmp = r1;
            r1 = r2;
            r2 = tmp;
        }
        int n = 0;
        if (r1 >= lo && r1 <= hi) out[n++] = r1;
        if (r2 >= lo && r2 <= hi && (n == 0 || r2 != out[0])) out[n++] = r2;
        return n;
    }
};

// two FP64 Newton steps on c from t (the step's divisor in FP32: the error of
// the start point, about 1e-6 of the edge, shrinks below 1e-12 either way)
template <int DEG>
__device__ __forceinline__ double polish(const double *c, double t)
{
    double dc[DEG];
#pragma unroll
    for (int k = 0; k < DEG; ++k) dc[k] = (double)(k + 1) * c[k + 1];
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        double f = horner<double, DEG>(c, t);
        float df = (float)horner<double, DEG - 1>(dc, t);
        if (df != 0.0f) t -= f * (double)(1.0f / df);
    }
    return t;
}

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
// length h), then the first root.  Every piece the FP32 prefilter lets
// through has its roots isolated in FP32 on [-m, h + m] (quadratic for the
// spheres, the torus quartic on its derivative chain) and polished by two FP64
// Newton steps on the exact FP64 polynomial; the freeness of a witness is
// decided in FP32 when the filter allows and in FP64 otherwise.  From an
// inside end point the answer is the first candidate; from an outside end
// point it is the first candidate at which no free probe centre lies strictly
// closer than r_p (within 1e-11 A).  On success t_out is the root and n_out
// the unit normal (FP64); returns 0, 1 (no root) or 2 (candidate overflow).
template <class T, bool FILT>
__device__ int warp_edge(const Model &M, const TileS<T> &S, const double *x0, EdgeSmem &E, int warp, int axis, int p,
                         int lab_s, double h, double rp, T d0, double &t_out, double n_out[3])
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
    const T fd = d0 + T(4e-6);            // error of an FP32 witness built from an FP64 root
    const bool inside = lab_s == LABEL_IN;
    const T lo = FILT ? T(-1e-4) : T(0), hi = hT + (FILT ? T(1e-4) : T(0));
    for (int it = lane; it < na + nv + np; it += 32) {
        if (it < na) {  // convex: van der Waals sphere, witness = projection on the expanded sphere
            P4<T> c = S.atom[it];
            T d[3] = {s[0] - c.x, s[1] - c.y, s[2] - c.z};
            T dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            T reach = c.w + hT + mg;
            if (dd > reach * reach) continue;
            T b = d[axis], disc = b * b - (dd - c.w * c.w);
            if (disc < -mg) continue;
            T co32[3] = {dd - c.w * c.w, T(2) * b, T(1)};
            T rt32[2];
            int nr = PolyRoots<T, 2>::run(co32, lo, hi, rt32);
            if (FILT && nr == 0 && disc < mg) {  // grazing: let FP64 decide
                rt32[0] = -b;
                nr = (-b >= lo && -b <= hi) ? 1 : 0;
            }
            if (nr == 0) continue;
            P4<double> ce = X.atom(it);
            double de[3] = {s64[0] - ce.x, s64[1] - ce.y, s64[2] - ce.z};
            double co[3] = {de[0] * de[0] + de[1] * de[1] + de[2] * de[2] - ce.w * ce.w, 2.0 * de[axis], 1.0};
            for (int k = 0; k < nr; ++k) {
                double t = polish<2>(co, (double)rt32[k]);
                if (!(t >= 0.0 && t <= h) || fabs(horner<double, 2>(co, t)) > 1e-9 * ce.w) continue;
                double v[3] = {de[0], de[1], de[2]};
                v[axis] += t;
                // the witness distance R - |y - c| must fall from an inside end point
                // and rise from an outside one: its rate has the sign of -v_axis
                if (inside ? -v[axis] > 1e-9 * ce.w : -v[axis] < -1e-9 * ce.w) continue;
                T v32[3] = {(T)v[0], (T)v[1], (T)v[2]};
                T R = c.w + rpT;
                T sc = R / sqrt(v32[0] * v32[0] + v32[1] * v32[1] + v32[2] * v32[2]);
                int f = FILT ? free_pt<true>(A, c.x + sc * v32[0], c.y + sc * v32[1], c.z + sc * v32[2], S.agid[it], -1,
                                             rpT, fd)
                             : -1;
                if (f < 0) {
                    double nvv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
                    double R64 = ce.w + rp;
                    f = free_pt<false>(X, ce.x + R64 * v[0] / nvv, ce.y + R64 * v[1] / nvv, ce.z + R64 * v[2] / nvv,
                                       S.agid[it], -1, rp, 0.0);
                }
                if (f == 1) warp_push(E, warp, t, 0.0, 0.0, 0.0, 0, it);
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
            T co32[3] = {dd - rpT * rpT, T(2) * b, T(1)};
            T rt32[2];
            int nr = PolyRoots<T, 2>::run(co32, lo, hi, rt32);
            if (FILT && nr == 0 && disc < mg) {
                rt32[0] = -b;
                nr = (-b >= lo && -b <= hi) ? 1 : 0;
            }
            if (nr == 0) continue;
            P4<double> ce = X.vq(vi);
            double de[3] = {s64[0] - ce.x, s64[1] - ce.y, s64[2] - ce.z};
            double co[3] = {de[0] * de[0] + de[1] * de[1] + de[2] * de[2] - rp * rp, 2.0 * de[axis], 1.0};
            for (int k = 0; k < nr; ++k) {
                double t = polish<2>(co, (double)rt32[k]);
                if (!(t >= 0.0 && t <= h) || fabs(horner<double, 2>(co, t)) > 1e-9 * rp) continue;
                double rate = de[axis] + t;  // sign of d|y - v|/dt
                if (inside ? rate > 1e-9 * rp : rate < -1e-9 * rp) continue;
                warp_push(E, warp, t, 0.0, 0.0, 0.0, 2, vi);
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
            // quartic (|y-o|^2 + rho^2 - r_p^2)^2 - 4 rho^2 |w|^2 in t
            T q0[3] = {s[0] - o.x, s[1] - o.y, s[2] - o.z};
            T uu32[3] = {u.x, u.y, u.z};
            T P = q0[0] * q0[0] + q0[1] * q0[1] + q0[2] * q0[2];
            T z0 = q0[0] * u.x + q0[1] * u.y + q0[2] * u.z;
            T pe = q0[axis], eu = uu32[axis];
            T K = P + o.w * o.w - rpT * rpT, r2 = o.w * o.w;
            T co32[5] = {K * K - T(4) * r2 * (P - z0 * z0), T(4) * pe * K - T(8) * r2 * (pe - z0 * eu),
                         T(4) * pe * pe + T(2) * K - T(4) * r2 * (T(1) - eu * eu), T(4) * pe, T(1)};
            T rt32[4];
            int nr = PolyRoots<T, 4>::run(co32, lo, hi, rt32);
            if (nr == 0) continue;
            P4<double> oe = X.po(pi);
            P4<double> ue = X.pu(pi);
            const double rho = oe.w;
            double p0[3] = {s64[0] - oe.x, s64[1] - oe.y, s64[2] - oe.z};
            double uu[3] = {ue.x, ue.y, ue.z};
            double Pd = p0[0] * p0[0] + p0[1] * p0[1] + p0[2] * p0[2];
            double z0d = p0[0] * uu[0] + p0[1] * uu[1] + p0[2] * uu[2];
            double ped = p0[axis], eud = uu[axis];
            double Kd = Pd + rho * rho - rp * rp;
            double r2d = rho * rho;
            double co[5];
            co[4] = 1.0;
            co[3] = 4.0 * ped;
            co[2] = 4.0 * ped * ped + 2.0 * Kd - 4.0 * r2d * (1.0 - eud * eud);
            co[1] = 4.0 * ped * Kd - 8.0 * r2d * (ped - z0d * eud);
            co[0] = Kd * Kd - 4.0 * r2d * (Pd - z0d * z0d);
            for (int k = 0; k < nr; ++k) {
                double t = polish<4>(co, (double)rt32[k]);
                if (!(t >= 0.0 && t <= h)) continue;
                double y[3] = {p0[0], p0[1], p0[2]};
                y[axis] += t;
                // near branch (|w| - rho)^2 + z^2 = r_p^2  <=>  |y-o|^2 + rho^2 - r_p^2 >= 0
                double Ay = y[0] * y[0] + y[1] * y[1] + y[2] * y[2] + rho * rho - rp * rp;
                if (Ay < 0.0) continue;
                double zy = y[0] * uu[0] + y[1] * uu[1] + y[2] * uu[2];
                double w[3] = {y[0] - zy * uu[0], y[1] - zy * uu[1], y[2] - zy * uu[2]};
                double w2d = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
                if (!(w2d > 0.0)) continue;
                // rate of the distance to the circle: ((|w| - rho) w_a / |w| + z u_a) / r_p
                float nwf = sqrtf((float)w2d);
                float rate = ((nwf - (float)rho) * (float)w[axis] / nwf + (float)(zy * uu[axis])) / (float)rp;
                if (fabsf(rate) < 1e-4f) {
                    double nw = sqrt(w2d);
                    double rd = ((nw - rho) * w[axis] / nw + zy * uu[axis]) / rp;
                    rate = rd > 1e-9 ? 1.0f : (rd < -1e-9 ? -1.0f : 0.0f);
                }
                if (inside ? rate > 0.0f : rate < 0.0f) continue;
                T kk = (T)(rho / (double)nwf);
                int2 ij = S.pij[pi];
                int f = FILT ? free_pt<true>(A, o.x + kk * (T)w[0], o.y + kk * (T)w[1], o.z + kk * (T)w[2], ij.x, ij.y,
                                             rpT, fd)
                             : -1;
                if (f < 0) {
                    double nw = sqrt(w2d);
                    f = free_pt<false>(X, oe.x + rho * w[0] / nw, oe.y + rho * w[1] / nw, oe.z + rho * w[2] / nw, ij.x,
                                       ij.y, rp, 0.0);
                }
                if (f == 1) warp_push(E, warp, t, 0.0, 0.0, 0.0, 1, pi);
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
    // normal at the root: unit vector from the surface point to its witness
    const double t = c[pick].t;
    double y[3] = {s64[0], s64[1], s64[2]};
    y[axis] += t;
    double v[3];
    const int kind = c[pick].kind, id = c[pick].id;
    if (kind == 0) {  // convex: radial, outward
        P4<double> ce = X.atom(id);
        v[0] = y[0] - ce.x; v[1] = y[1] - ce.y; v[2] = y[2] - ce.z;
    } else if (kind == 2) {  // concave: towards the probe centre
        P4<double> ce = X.vq(id);
        v[0] = ce.x - y[0]; v[1] = ce.y - y[1]; v[2] = ce.z - y[2];
    } else {  // saddle: towards the nearest circle point
        P4<double> oe = X.po(id);
        P4<double> ue = X.pu(id);
        double yo[3] = {y[0] - oe.x, y[1] - oe.y, y[2] - oe.z};
        double zy = yo[0] * ue.x + yo[1] * ue.y + yo[2] * ue.z;
        double w[3] = {yo[0] - zy * ue.x, yo[1] - zy * ue.y, yo[2] - zy * ue.z};
        double nw = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
        double k2 = oe.w / nw;
        v[0] = k2 * w[0] - yo[0]; v[1] = k2 * w[1] - yo[1]; v[2] = k2 * w[2] - yo[2];
    }
    double vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    t_out = t;
    n_out[0] = v[0] / vn;
    n_out[1] = v[1] / vn;
    n_out[2] = v[2] / vn;
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
    const double h = G.h, rp = M.rp, inv_h = 1.0 / G.h;
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
            double tr = 0.5 * h, nrm[3] = {0.0, 0.0, 0.0};
            int status = warp_edge<T, FILT>(M, S, x0, E, warp, a, q, lab_s, h, rp, d0, tr, nrm);
            if (lane == 0) {
                if (status == 1) nrm[0] = nrm[1] = nrm[2] = 0.0;
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
                out.tau[a][o] = tr * inv_h;
                out.nrm[a][3 * o + 0] = nrm[0];
                out.nrm[a][3 * o + 1] = nrm[1];
                out.nrm[a][3 * o + 2] = nrm[2];
                out.tau32[a][o] = (float)(tr * inv_h);
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
