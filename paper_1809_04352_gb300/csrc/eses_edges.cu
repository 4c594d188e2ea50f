// eses_edges.cu -- crossing edges, surface roots and normals, area and volume
// (the third and fourth ESES stages, Eq. 3-4).
//
// k_edge_count: per tile and axis, the edges (p, p + e_a) leaving the tile's
//   points whose end labels differ, and the edges with both ends inside.
// (exclusive scan of the counts -> every tile's output offset per axis; the
//   paper serialises this output step in a critical section, Algorithm 1)
// The root solve: the surface along an edge is made of pieces of van der
//   Waals spheres (convex), tori around pair circles (saddle) and probe
//   spheres around free triple points (concave).  Every root of every such
//   piece in [0, h] whose witness (projection on the expanded sphere /
//   nearest circle point / the triple point) is free, and whose witness
//   distance crosses r_p in the direction that leaves the end point's side
//   (falling from an inside end, rising from an outside end), is a candidate.
//   From an inside end point the first candidate is the first root; from an
//   outside end point the first candidate that is not strictly outside M is.
//   Five launches linked by lists in HBM:
//   k_edge_stage: persistent CTAs take tiles from the work queue; per tile
//     the pieces are staged (shared memory, or the global-memory tier for a
//     tile that overflows it), the crossing edges listed, and written out:
//     the staged lists (the tile's slab), an edge record per edge, and the
//     (edge, piece) pairs that pass a prefilter (one warp per edge, lanes over
//     the staged pieces), spheres and tori in separate lists;
//   k_roots_sphere / k_roots_torus: one thread per pair, no block barrier:
//     sphere roots from the quadratic; torus roots of
//          (|y-o|^2 + rho^2 - r_p^2)^2 = 4 rho^2 (|y-o|^2 - ((y-o).u)^2)
//     on the near branch (|w| - rho)^2 + z^2 = r_p^2, isolated in FP32 on
//     eight sub-intervals with certified exclusion and monotonicity tests and
//     refined by Newton (undecided: the quartic on its derivative chain, then
//     FP64); every FP32 root carries an error bound; the accepted roots go to
//     the pair's slots;
//   k_edge_pick: one thread per edge: the first root when the end point is
//     inside or one candidate is left and the FP32 bounds order the
//     candidates; the other edges are listed;
//   k_edge_hard: one warp per listed edge: near ties broken on FP64 roots; at
//     an outside end point each earlier candidate tested first against the
//     later candidates' witnesses, then by the full witness search, whose
//     undecided items are re-tested in FP64.
//   The chosen piece and its FP32 root are recorded for the polish.
// k_edge_polish: one thread per crossing edge (full warps of FP64 work): the
//   FP64 root of the chosen piece next to the recorded one, the normal, the
//   outputs and the area/volume terms.
// k_reduce: per molecule, area = h^2 sum |n_a|, volume = h^2/3 sum of
//   inside lengths.
// Every tile kernel runs over the tiles of all molecules of a batch.
#include <math.h>

#include <algorithm>

#include "eses_kernels.h"
#include "eses_tile.cuh"

namespace eses {

constexpr int EDGE_THREADS = 256;
constexpr int EDGE_WARPS = EDGE_THREADS / 32;
constexpr int WCAND = 64;        // candidate roots of one edge in the selection buffer
constexpr int ROOT_THREADS_MAX = 256;  // per-candidate root kernels: threads per block (at most, the default)
constexpr int PICK_THREADS = 256;
constexpr int HARD_THREADS = 256;
constexpr int HMASK_WORDS = 1536;  // prefilter hit masks kept between the staging pass's two sweeps
constexpr int POLISH_THREADS = 256;

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
    __device__ static __noinline__ int run(const R *c, R lo, R hi, R *out)
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

// --------------------------------------------------------------------------
// exact (FP64) roots and normals of one piece, any common frame
// --------------------------------------------------------------------------
// root of |s + t e_axis - c| = rad nearest t0 (t0 returned when none is real)
__device__ __forceinline__ double exact_root_sphere(const double *c, double rad, const double *s, int axis, double t0)
{
    double d[3] = {s[0] - c[0], s[1] - c[1], s[2] - c[2]};
    double b = d[axis];
    double cc = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] - rad * rad;
    double disc = b * b - cc;
    if (disc < 0.0) return t0;
    double sq = sqrt(disc);
    double q = -(b + (b >= 0.0 ? sq : -sq));
    double r1 = q, r2 = (q != 0.0) ? cc / q : q;
    return fabs(r1 - t0) <= fabs(r2 - t0) ? r1 : r2;
}

__device__ __forceinline__ void torus_coeffs(const double *o, const double *u, double rho, double rp, const double *s,
                                             int axis, double *co)
{
    double p0[3] = {s[0] - o[0], s[1] - o[1], s[2] - o[2]};
    double P = p0[0] * p0[0] + p0[1] * p0[1] + p0[2] * p0[2];
    double z0 = p0[0] * u[0] + p0[1] * u[1] + p0[2] * u[2];
    double pe = p0[axis], eu = u[axis];
    double K = P + rho * rho - rp * rp;
    double r2 = rho * rho;
    co[4] = 1.0;
    co[3] = 4.0 * pe;
    co[2] = 4.0 * pe * pe + 2.0 * K - 4.0 * r2 * (1.0 - eu * eu);
    co[1] = 4.0 * pe * K - 8.0 * r2 * (pe - z0 * eu);
    co[0] = K * K - 4.0 * r2 * (P - z0 * z0);
}

// FP64 Newton steps on the torus quartic from t0, at most four (the FP32 root
// is within 1e-3 A and the root simple, else the warp solve already took it in
// FP64): quadratic convergence, so the steps stop once one moves t by less
// than 1e-13 A (the next would move it by about the square of that)
__device__ __noinline__ double exact_root_torus(const double *o, const double *u, double rho, double rp,
                                                   const double *s, int axis, double t0)
{
    double co[5];
    torus_coeffs(o, u, rho, rp, s, axis, co);
    double dc[4] = {co[1], 2.0 * co[2], 3.0 * co[3], 4.0};
    double t = t0;
    for (int it = 0; it < 4; ++it) {
        double f = horner<double, 4>(co, t);
        double df = horner<double, 3>(dc, t);
        if (df == 0.0) break;
        const double dt = f / df;
        t -= dt;
        if (fabs(dt) < 1e-13) break;
    }
    return t;
}

// unit normal at y (towards the witness, i.e. into the solvent)
__device__ __forceinline__ void exact_normal(int kind, const double *c, const double *u, double rho, const double *y,
                                             double *n)
{
    double v[3];
    if (kind == 0) {  // convex: radial, outward
        v[0] = y[0] - c[0]; v[1] = y[1] - c[1]; v[2] = y[2] - c[2];
    } else if (kind == 2) {  // concave: towards the probe centre
        v[0] = c[0] - y[0]; v[1] = c[1] - y[1]; v[2] = c[2] - y[2];
    } else {  // saddle: towards the nearest point of the circle
        double yo[3] = {y[0] - c[0], y[1] - c[1], y[2] - c[2]};
        double w[3];
        axis_normal(yo, u, w);
        v[0] = rho * w[0] - yo[0]; v[1] = rho * w[1] - yo[1]; v[2] = rho * w[2] - yo[2];
    }
    double vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double iv = vn > 0.0 ? 1.0 / vn : 0.0;
    n[0] = v[0] * iv;
    n[1] = v[1] * iv;
    n[2] = v[2] * iv;
}

// exact root of a staged piece (tile frame, FP64 data from HBM) near t0
template <class XA>
__device__ __noinline__ double staged_exact_root(const XA &X, int kind, int slot, const double *s,
                                                    int axis, double rp, double t0)
{
    if (kind == 0) {
        P4<double> c = X.atom(slot);
        double cc[3] = {c.x, c.y, c.z};
        return exact_root_sphere(cc, c.w, s, axis, t0);
    }
    if (kind == 2) {
        P4<double> c = X.vq(slot);
        double cc[3] = {c.x, c.y, c.z};
        return exact_root_sphere(cc, rp, s, axis, t0);
    }
    P4<double> o = X.po(slot);
    P4<double> u = X.pu(slot);
    double oo[3] = {o.x, o.y, o.z}, uu[3] = {u.x, u.y, u.z};
    return exact_root_torus(oo, uu, o.w, rp, s, axis, t0);
}

// --------------------------------------------------------------------------
// the phased root solve: data between the launches
// --------------------------------------------------------------------------
// A candidate root of one crossing edge during the selection.
struct WCand {
    double t64;    // exact root once computed (NaN before)
    float t, err;  // FP32 root and its error bound (A)
    int kind, id;  // kind 0: van der Waals sphere (atom slot), 1: torus (pair slot), 2: probe sphere (vertex slot)
};

// Accepted roots of one (edge, piece) candidate, written to the candidate's
// slots in HBM (at most SPH_SLOTS for a sphere, whose two roots cross in
// opposite directions; at most TOR_SLOTS, the quartic's degree, for a torus).
constexpr int SPH_SLOTS = 2;
constexpr int TOR_SLOTS = 4;
struct RootSink {
    RootRec *r;
    int n, cap;
    __device__ __forceinline__ void push(float t, float err, double t64)
    {
        if (n < cap) {
            RootRec q;
            q.t64 = t64;
            q.t = t;
            q.err = err;
            r[n] = q;
        }
        ++n;
    }
    // a slot kept for a root whose decision needs FP64 (err < 0: pending; the
    // FP32 root kept in t), settled by k_roots_torus_exact
    __device__ __forceinline__ void pend(float t) { push(t, -1.0f, __longlong_as_double(0x7ff8000000000000LL)); }
};
// a settled slot whose root was rejected
__device__ __forceinline__ RootRec no_root()
{
    RootRec q;
    q.t64 = __longlong_as_double(0x7ff8000000000000LL);
    q.t = INFINITY;
    q.err = 0.0f;
    return q;
}

// Lower point p (local index) of an edge in the tile frame, and the spacing,
// in T: for FP32 the molecule's table of k * h rounded to FP32 (the same
// values as rounding the FP64 products), so no FP64 arithmetic is spent.
template <class T>
__device__ __forceinline__ void edge_point(const Grid &G, int p, T *s, T &hT)
{
    if constexpr (sizeof(T) == sizeof(float)) {
        s[0] = G.hl[p >> 6];
        s[1] = G.hl[(p >> 3) & 7];
        s[2] = G.hl[p & 7];
        hT = G.hl[1];
    } else {
        s[0] = (double)(p >> 6) * G.h;
        s[1] = (double)((p >> 3) & 7) * G.h;
        s[2] = (double)(p & 7) * G.h;
        hT = G.h;
    }
}

// einfo[].y: lower point (local index), axis, end label, dropped (a buffer of
// the staging pass was full)
__host__ __device__ constexpr int edge_pack(int p, int axis, int lab, int dropped)
{
    return p | (axis << 9) | (lab << 11) | (dropped << 12);
}
__device__ __forceinline__ int pk_point(int pk) { return pk & 511; }
__device__ __forceinline__ int pk_axis(int pk) { return (pk >> 9) & 3; }
__device__ __forceinline__ int pk_label(int pk) { return (pk >> 11) & 1; }
__device__ __forceinline__ bool pk_dropped(int pk) { return ((pk >> 12) & 1) != 0; }

// A staged tile in HBM (its slab): this header, then the staged lists in the
// tile frame, each segment 16-byte aligned.  Written once by the staging pass
// and read (through L1/L2) by every root and selection thread of the tile.
struct alignas(16) SlabHdr {
    int na, np, nv, mol;
    double x0[3];  // tile frame origin (absolute)
    int t[3];      // tile coordinates in the run's grid
    int gt;        // batch tile
};

__host__ __device__ constexpr long long align16(long long b) { return (b + 15) & ~15LL; }

template <class T>
struct SlabLayout {
    long long atom, po, pu, vq, agid, pij, pidx, vidx, face, nbm, pslot, bytes;
    __host__ __device__ SlabLayout(int na, int np, int nv)
    {
        const long long nw = (na + 31) / 32;  // words of a set of staged atoms
        const long long P = (long long)sizeof(P4<T>);
        atom = (long long)sizeof(SlabHdr);
        po = atom + na * P;
        pu = po + np * P;
        vq = pu + np * P;
        agid = vq + nv * P;
        pij = align16(agid + 4LL * na);
        pidx = align16(pij + 8LL * np);
        vidx = align16(pidx + 4LL * np);
        face = align16(vidx + 4LL * nv);
        nbm = align16(face + na);
        pslot = align16(nbm + 4LL * na * nw);
        bytes = align16(pslot + 4LL * np);
    }
};

__device__ __forceinline__ P4<float> ldg4(const P4<float> *p)
{
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    return P4<float>{v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ P4<double> ldg4(const P4<double> *p)
{
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    return P4<double>{a.x, a.y, b.x, b.y};
}

// the staged lists of a slab (same interface as SmemAcc)
template <class T>
struct SlabAcc {
    using real = T;
    const P4<T> *a_, *po_, *pu_, *vq_;
    const int *agid_, *pidx_, *vidx_;
    const int2 *pij_;
    const uint8_t *face_;
    const unsigned *nbm_;
    const short2 *pslot_;
    int na_, np_, nv_, nw_;
    __device__ explicit SlabAcc(const unsigned char *s)
    {
        const int4 h = __ldg(reinterpret_cast<const int4 *>(s));
        na_ = h.x;
        np_ = h.y;
        nv_ = h.z;
        const SlabLayout<T> L(na_, np_, nv_);
        a_ = reinterpret_cast<const P4<T> *>(s + L.atom);
        po_ = reinterpret_cast<const P4<T> *>(s + L.po);
        pu_ = reinterpret_cast<const P4<T> *>(s + L.pu);
        vq_ = reinterpret_cast<const P4<T> *>(s + L.vq);
        agid_ = reinterpret_cast<const int *>(s + L.agid);
        pij_ = reinterpret_cast<const int2 *>(s + L.pij);
        pidx_ = reinterpret_cast<const int *>(s + L.pidx);
        vidx_ = reinterpret_cast<const int *>(s + L.vidx);
        face_ = reinterpret_cast<const uint8_t *>(s + L.face);
        nbm_ = reinterpret_cast<const unsigned *>(s + L.nbm);
        pslot_ = reinterpret_cast<const short2 *>(s + L.pslot);
        nw_ = (na_ + 31) >> 5;
    }
    __device__ int na() const { return na_; }
    __device__ int np() const { return np_; }
    __device__ int nv() const { return nv_; }
    __device__ P4<T> atom(int a) const { return ldg4(a_ + a); }
    __device__ int agid(int a) const { return __ldg(agid_ + a); }
    __device__ bool face(int a) const { return __ldg(face_ + a) != 0; }
    __device__ P4<T> po(int p) const { return ldg4(po_ + p); }
    __device__ P4<T> pu(int p) const { return ldg4(pu_ + p); }
    __device__ int2 pij(int p) const { return __ldg(pij_ + p); }
    __device__ P4<T> vq(int v) const { return ldg4(vq_ + v); }
    __device__ int pidx(int p) const { return __ldg(pidx_ + p); }
    __device__ int vidx(int v) const { return __ldg(vidx_ + v); }
    // neighbour set of staged atom a (staged atoms whose expanded spheres
    // come within 1e-3 A of meeting a's), ceil(na / 32) words
    __device__ const unsigned *nb(int a) const { return nbm_ + (size_t)a * nw_; }
    // staged slots of pair p's atoms (-1: not staged)
    __device__ short2 pslot(int p) const { return __ldg(pslot_ + p); }
    // model index of a staged piece (kind as in WCand)
    __device__ int model_index(int kind, int slot) const
    {
        return kind == 0 ? agid(slot) : (kind == 1 ? pidx(slot) : vidx(slot));
    }
};

// FP64 data of a slab's pieces from HBM, in the same tile frame (as ExactAcc)
template <class T>
struct SlabExact {
    using real = double;
    const SlabAcc<T> &S;
    const Model &M;
    double x0, y0, z0;
    __device__ SlabExact(const SlabAcc<T> &s, const Model &m, const double *o)
        : S(s), M(m), x0(o[0]), y0(o[1]), z0(o[2]) {}
    __device__ int na() const { return S.na(); }
    __device__ int np() const { return S.np(); }
    __device__ int nv() const { return S.nv(); }
    __device__ P4<double> atom(int a) const
    {
        const double4 g = M.atom[S.agid(a)];
        return P4<double>{g.x - x0, g.y - y0, g.z - z0, g.w};
    }
    __device__ int agid(int a) const { return S.agid(a); }
    __device__ bool face(int a) const { return S.face(a); }
    __device__ P4<double> po(int p) const
    {
        const double4 g = M.pair_o[S.pidx(p)];
        return P4<double>{g.x - x0, g.y - y0, g.z - z0, g.w};
    }
    __device__ P4<double> pu(int p) const
    {
        const double4 g = M.pair_u[S.pidx(p)];
        return P4<double>{g.x, g.y, g.z, 0.0};
    }
    __device__ int2 pij(int p) const { return S.pij(p); }
    __device__ P4<double> vq(int v) const
    {
        const double4 g = M.vert[S.vidx(v)];
        return P4<double>{g.x - x0, g.y - y0, g.z - z0, 0.0};
    }
    __device__ const unsigned *nb(int a) const { return S.nb(a); }
    __device__ short2 pslot(int p) const { return S.pslot(p); }
};

// Freeness of a witness on the expanded sphere of staged atom a (and, for a
// saddle witness, of staged atom b too): only the atoms whose expanded
// spheres meet a's (and b's) can cover it, so the neighbour sets decide the
// same as a test against every staged atom but a and b (free_set).  A pair
// whose atoms are not both staged is tested against every staged atom.
template <bool FILT, class Acc, class T>
__device__ __forceinline__ int free_witness(const Acc &A, T qx, T qy, T qz, int sa, int sb, int ga, int gb, T rp,
                                            T delta)
{
    int nt = 0;
    if (sa >= 0 && (gb < 0 || sb >= 0))
        return free_set<FILT>(A, qx, qy, qz, A.nb(sa), gb < 0 ? (const unsigned *)nullptr : A.nb(sb), rp, delta, nt);
    return free_pt<FILT>(A, qx, qy, qz, ga, gb, rp, delta);
}

// shared memory of the staging pass (beside the staged tile)
struct StageSmem {
    int8_t lab[9 * 9 * 9];
    short eptr[3 * TILE_PTS];  // crossing edges of the tile (local point), grouped by axis
    int cs[3 * TILE_PTS + 1];  // per edge: sphere candidates, then their offset in the tile's run
    int ct[3 * TILE_PTS + 1];  // the same for tori
    int estart[4];
    int gbase[3];  // global id of the tile's first edge per axis (all axes numbered in one run)
    int abase[3];  // its index in the axis' output
    int sh[EDGE_WARPS], sh2[EDGE_WARPS];
    long long slab;    // slab offset (16-byte units), -1 when the slab buffer is full
    long long sb, tb;  // the tile's first sphere / torus candidate, -1 when a buffer is full
    long long sb0, tb0;  // the same as reserved (also when a buffer is full)
    unsigned hmask[HMASK_WORDS];  // prefilter hits, ceil(items / 32) words per edge (when they fit)
};

// items [0, nsph) are spheres: the bits of 32-item word w that are spheres
__device__ __forceinline__ unsigned sphere_bits(int w, int nsph)
{
    const int r = nsph - 32 * w;
    return r >= 32 ? 0xffffffffu : (r <= 0 ? 0u : (1u << r) - 1u);
}

// axis, lower point (local index) and its label of crossing edge e of the tile
struct EdgeRef {
    int axis, p, lab;
};
__device__ __forceinline__ EdgeRef edge_ref(const StageSmem &E, int e)
{
    EdgeRef r;
    r.axis = e < E.estart[1] ? 0 : (e < E.estart[2] ? 1 : 2);
    r.p = E.eptr[e];
    r.lab = E.lab[((r.p >> 6) * 9 + ((r.p >> 3) & 7)) * 9 + (r.p & 7)];
    return r;
}

// index of the smallest key (ties: smaller index), -1 if every key is +inf
__device__ __forceinline__ int warp_argmin_key(float key, int k)
{
    float bt = key;
    int bk = (key < INFINITY) ? k : -1;
    for (int o = 16; o > 0; o >>= 1) {
        float ot = __shfl_xor_sync(0xffffffffu, bt, o);
        int ok = __shfl_xor_sync(0xffffffffu, bk, o);
        if (ok >= 0 && (bk < 0 || ot < bt || (ot == bt && ok < bk))) {
            bt = ot;
            bk = ok;
        }
    }
    return bk;
}

__device__ __forceinline__ int warp_argmin(const WCand *c, int n)
{
    const int lane = threadIdx.x & 31;
    float bt = INFINITY;
    int bk = -1;
    for (int k = lane; k < n; k += 32)
        if (c[k].t < bt) {
            bt = c[k].t;
            bk = k;
        }
    return warp_argmin_key(bt, bk);
}

// --------------------------------------------------------------------------
// torus pieces: near-branch roots of g(t) = D(t) - r_p, D the distance from
// y(t) = q0 + t e_axis to the circle (centre at the frame origin, axis u,
// radius rho).  These are the roots of the quartic whose nearest circle point
// is the witness.
// --------------------------------------------------------------------------
// D, dD/dt, the distance |w| to the circle's axis, |y|^2, z = y.u and w at t
__device__ __forceinline__ void circle_dist32(const float *q0, const float *u, float rho, int axis, float t, float &D,
                                              float &dD, float &nw, float &yy, float &z, float *w)
{
    float y0 = q0[0], y1 = q0[1], y2 = q0[2];
    if (axis == 0) y0 += t;
    else if (axis == 1) y1 += t;
    else y2 += t;
    z = y0 * u[0] + y1 * u[1] + y2 * u[2];
    yy = y0 * y0 + y1 * y1 + y2 * y2;
    w[0] = y0 - z * u[0];
    w[1] = y1 - z * u[1];
    w[2] = y2 - z * u[2];
    nw = sqrtf(fmaxf(yy - z * z, 0.0f));
    const float e = nw - rho;
    D = sqrtf(e * e + z * z);
    const float wa = axis == 0 ? w[0] : (axis == 1 ? w[1] : w[2]);
    dD = (nw > 0.0f && D > 0.0f) ? (e * wa / nw + z * u[axis]) / D : 0.0f;
}

// error bound of the FP32 D: staged positions (d0) and rounding of |y|^2 - z^2
// (relative 2^-24 per operation, amplified by |y|^2 / |w| in |w|)
__device__ __forceinline__ float circle_dist_err(float d0, float yy, float nw, float rho, float rp)
{
    return 2.0f * d0 + 4e-7f * (yy / fmaxf(nw, 1e-3f) + sqrtf(yy) + rho + rp);
}

// g along the edge from its quadratic pieces: |y|^2 = yy0 + 2 qa t + t^2 and
// z = z0 + ua t (qa, ua the edge-axis components of q0 and u)
struct LineCircle32 {
    float yy0, qa, z0, ua, rho, rp;
    __device__ __forceinline__ void eval(float t, float &g, float &dg, float &nw, float &yy) const
    {
        yy = fmaf(t, t + 2.0f * qa, yy0);
        const float z = fmaf(t, ua, z0);
        nw = sqrtf(fmaxf(yy - z * z, 0.0f));
        const float e = nw - rho;
        const float D = sqrtf(e * e + z * z);
        g = D - rp;
        const float wa = qa + t - z * ua;  // edge-axis component of w
        dg = (nw > 0.0f && D > 0.0f) ? __fdividef(e * __fdividef(wa, nw) + z * ua, D) : 0.0f;
    }
};

// Certified FP32 isolation of the roots of g on [lo, hi].  g is 1-Lipschitz
// and |g''| <= C = max(1/D, 1/|w|) (the distance to a circle has Hessian
// eigenvalues 0 and 1/D in the meridian plane and (dD/d|w|)/|w| around the
// axis; D and |w| are 1-Lipschitz too, so on a sub-interval of length l they
// stay above their smaller end value minus l/2).  On 8 sub-intervals: none
// holds a root when |g| at its ends adds up to more than its length; g' keeps
// its sign when g' has the same sign at both ends and |g'| there adds up to
// more than C l, and then the sub-interval holds one root if g changes sign,
// else none.  Each root is refined by Newton from the secant point inside its
// bracket.  Returns false when a sign or the monotonicity cannot be decided.
__device__ __noinline__ bool torus_roots32(const float *q0, const float *u, float rho, float rp, int axis, float lo,
                                           float hi, float d0, float *rt, int &nr)
{
    constexpr int K = 8;
    const float dl = (hi - lo) / (float)K;
    LineCircle32 L;
    L.yy0 = q0[0] * q0[0] + q0[1] * q0[1] + q0[2] * q0[2];
    L.qa = q0[axis];
    L.z0 = q0[0] * u[0] + q0[1] * u[1] + q0[2] * u[2];
    L.ua = u[axis];
    L.rho = rho;
    L.rp = rp;
    unsigned rootmask = 0;
    float gp = 0.0f, dgp = 0.0f, egp = 0.0f, mwp = 0.0f;
#pragma unroll
    for (int k = 0; k <= K; ++k) {
        const float t = k == K ? hi : lo + (float)k * dl;
        float g, dg, nw, yy;
        L.eval(t, g, dg, nw, yy);
        const float eg = circle_dist_err(d0, yy, nw, rho, rp);
        const float mw = fminf(g + rp, nw);
        if (k > 0) {
            const bool sc = (gp <= 0.0f) != (g <= 0.0f);
            if (sc || fabsf(gp) + fabsf(g) <= dl + egp + eg) {
                if (fabsf(gp) <= egp || fabsf(g) <= eg) return false;
                const float low = fminf(mwp, mw) - 0.5f * dl;
                if (!(low > 1e-2f)) return false;
                if (!((dgp > 0.0f) == (dg > 0.0f) && fabsf(dgp) + fabsf(dg) > dl / low + 2e-4f)) return false;
                if (sc) rootmask |= 1u << (k - 1);
            }
        }
        gp = g;
        dgp = dg;
        egp = eg;
        mwp = mw;
    }
    nr = 0;
    while (rootmask) {
        const int k = __ffs(rootmask) - 1;
        rootmask &= rootmask - 1;
        if (nr == 4) return false;
        float a = lo + (float)k * dl, b = k + 1 == K ? hi : lo + (float)(k + 1) * dl;
        float ga, gb, dga, dgb, nwa, yya;
        L.eval(a, ga, dga, nwa, yya);
        L.eval(b, gb, dgb, nwa, yya);
        const bool neg_a = ga <= 0.0f;
        float t = a + (b - a) * __fdividef(ga, ga - gb);
        for (int itn = 0; itn < 5; ++itn) {  // Newton, bisection when it leaves the bracket
            float f, df, nw, yy;
            L.eval(t, f, df, nw, yy);
            if (f == 0.0f) break;
            if ((f <= 0.0f) == neg_a) a = t;
            else b = t;
            float tn = df != 0.0f ? t - __fdividef(f, df) : 0.5f * (a + b);
            if (!(tn > a && tn < b)) tn = 0.5f * (a + b);
            t = tn;
        }
        rt[nr++] = t;
    }
    return true;
}

// One FP64 root t64 of a torus piece: kept if it lies on the near branch in
// [0, h], its witness distance crosses r_p in the direction that leaves the
// end point's side, and its witness (nearest circle point) is free.
template <class Acc>
__device__ __noinline__ void torus_root_exact(const Acc &X, RootSink &out, int pi, const double *s64, int axis,
                                              double h, double rp, bool inside, double t64)
{
    if (!(t64 >= 0.0 && t64 <= h)) return;
    const P4<double> oe = X.po(pi);
    const P4<double> ue = X.pu(pi);
    const double oo[3] = {oe.x, oe.y, oe.z}, u64[3] = {ue.x, ue.y, ue.z};
    double yd[3] = {s64[0] - oo[0], s64[1] - oo[1], s64[2] - oo[2]};
    yd[axis] += t64;
    const double Ad = yd[0] * yd[0] + yd[1] * yd[1] + yd[2] * yd[2] + oe.w * oe.w - rp * rp;
    const double zd = yd[0] * u64[0] + yd[1] * u64[1] + yd[2] * u64[2];
    double wd[3];
    const double nwd = axis_normal(yd, u64, wd);  // unit direction
    const double near2 = (nwd - oe.w) * (nwd - oe.w) + zd * zd;
    if (fabs(near2 - rp * rp) > 1e-7 * rp * rp || !(nwd > 0.0) || !(Ad >= 0.0)) return;
    const double rd = ((nwd - oe.w) * wd[axis] + zd * u64[axis]) / rp;
    const double rate = fabs(rd) <= 1e-9 ? 0.0 : rd;
    if (inside ? rate > 0.0 : rate < 0.0) return;
    const int2 ij = X.pij(pi);
    const short2 sl = X.pslot(pi);
    const int f = free_witness<false>(X, oo[0] + oe.w * wd[0], oo[1] + oe.w * wd[1], oo[2] + oe.w * wd[2], (int)sl.x,
                                      (int)sl.y, ij.x, ij.y, rp, 0.0);
    if (f == 1) out.push((float)t64, 0.0f, t64);
}

// Every root of a torus piece in [0, h] from the quartic, each decided in FP64.
template <class Acc>
__device__ __noinline__ void torus_piece_exact(const Acc &X, RootSink &out, int pi, const double *s64, int axis,
                                               double h, double rp, bool inside)
{
    const P4<double> oe = X.po(pi);
    const P4<double> ue = X.pu(pi);
    const double oo[3] = {oe.x, oe.y, oe.z}, u64[3] = {ue.x, ue.y, ue.z};
    double co[5], r64[4];
    torus_coeffs(oo, u64, oe.w, rp, s64, axis, co);
    const int n = PolyRoots<double, 4>::run(co, 0.0, h, r64);
    for (int k = 0; k < n; ++k) torus_root_exact(X, out, pi, s64, axis, h, rp, inside, r64[k]);
}

// Can item `it` (staged atom, vertex or pair, in that order) put a root on the
// edge from s along axis?  Spheres |y - c| = rad: only if the distance from c
// to the segment takes the value rad (its minimum and maximum over the
// segment bracket rad); tori: the 1-Lipschitz distance to the circle is
// within h/2 of r_p at the edge's midpoint.  mg widens both for FP32.
template <class T, class CP>
__device__ __forceinline__ bool cand_test(const TileS<T, CP> &S, const T *s, int axis, int it, T hT, T rpT, T mg)
{
    const int na = S.na, nv = S.nv;
    if (it < na + nv) {
        const P4<T> c = it < na ? S.atom[it] : S.vq[it - na];
        const T rad = it < na ? c.w : rpT;
        const T d0 = s[0] - c.x, d1 = s[1] - c.y, d2 = s[2] - c.z;
        const T dd = d0 * d0 + d1 * d1 + d2 * d2;
        const T da = axis == 0 ? d0 : (axis == 1 ? d1 : d2);
        const T tc = fmin(fmax(-da, T(0)), hT);         // nearest point of the segment
        const T dmin2 = dd + tc * (tc + T(2) * da);
        const T dmax2 = dd + fmax(T(0), hT * (hT + T(2) * da));
        const T rhi = rad + mg, rlo = fmax(rad - mg, T(0));
        return dmin2 <= rhi * rhi && dmax2 >= rlo * rlo;
    }
    const int pi = it - na - nv;
    const P4<T> o = S.po[pi];
    const P4<T> u = S.pu[pi];
    T m[3] = {s[0] - o.x, s[1] - o.y, s[2] - o.z};
    m[axis] += T(0.5) * hT;
    const T zc = m[0] * u.x + m[1] * u.y + m[2] * u.z;
    const T w2 = fmax(m[0] * m[0] + m[1] * m[1] + m[2] * m[2] - zc * zc, T(0));
    const T e1 = sqrt(w2) - o.w;
    const T gm = sqrt(e1 * e1 + zc * zc) - rpT;
    return fabs(gm) <= T(0.5) * hT + mg;
}

// Roots of one (edge, piece) candidate that can be the surface on that edge:
// every root in [0, h] of the piece whose witness distance crosses r_p in the
// direction that leaves the end point's side (falling from an inside end,
// rising from an outside end) and whose witness is free.  FP32 roots carry an
// error bound; a decision the bound cannot make goes to FP64.  A: the staged
// lists (tile frame), X: the same pieces in FP64; s64 the edge's lower point
// in the tile frame.
//
// Spheres (item < na: van der Waals sphere of staged atom `item`, convex,
// witness = projection on the expanded sphere; else the probe sphere of staged
// triple point item - na, concave, witness = the triple point).
template <class T, bool FILT, class AccT, class AccX>
__device__ void sphere_roots(const AccT &A, const AccX &X, int item, const T *s, const double *s64, int axis,
                             bool inside, T hT, T rpT, double h, double rp, T d0, RootSink &out)
{
    const int na = A.na();
    const T lo = FILT ? T(-1e-4) : T(0), hi = hT + (FILT ? T(1e-4) : T(0));
    const T tmax = T(1e-3);  // FP32 root error beyond which FP64 decides (grazing pieces)
    const double NaN = __longlong_as_double(0x7ff8000000000000LL);
    const bool vdw = item < na;
    const int slot = vdw ? item : item - na;
    const P4<T> c = vdw ? A.atom(slot) : A.vq(slot);
    const T rad = vdw ? c.w : rpT;
    const T d[3] = {s[0] - c.x, s[1] - c.y, s[2] - c.z};
    const T dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const T b = d[axis], disc = b * b - (dd - rad * rad);
    const T co32[3] = {dd - rad * rad, T(2) * b, T(1)};
    T rt32[2];
    int nr = PolyRoots<T, 2>::run(co32, lo, hi, rt32);
    if (FILT && nr == 0 && disc < T(2e-3)) {  // grazing: let FP64 decide
        rt32[0] = -b;
        nr = (-b >= lo && -b <= hi) ? 1 : 0;
    }
    for (int k = 0; k < nr; ++k) {
        T t = rt32[k];
        T vA = d[axis] + t;  // +-sqrt(disc) at a root: the rate of |y - c|
        T terr = T(0);
        if (FILT) {
            const T derr = T(2) * (fabs(b) + sqrt(dd)) * d0 + T(2e-6) * (dd + rad * rad);
            terr = d0 + derr / (T(2) * fmax(fabs(vA), T(1e-20)));
        }
        double t64 = NaN;
        const bool exact = FILT && (terr > tmax || t < terr + T(1e-6) || t > hT - terr - T(1e-6));
        if (exact) {
            const P4<double> ce = vdw ? X.atom(slot) : X.vq(slot);
            const double cc[3] = {ce.x, ce.y, ce.z};
            const double r64 = vdw ? ce.w : rp;
            t64 = exact_root_sphere(cc, r64, s64, axis, (double)t);
            double dv[3] = {s64[0] - cc[0], s64[1] - cc[1], s64[2] - cc[2]};
            dv[axis] += t64;
            const double f = dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2] - r64 * r64;
            if (!(t64 >= 0.0 && t64 <= h) || fabs(f) > 1e-9 * r64) continue;
            vA = (T)dv[axis];
            if (fabs(dv[axis]) <= 1e-9 * r64) vA = T(0);  // tangent: either way
            t = (T)t64;
            terr = T(0);
        }
        // witness distance: R - |y - c| (convex) falls iff vA > 0; |y - v| (concave) rises iff vA > 0
        const bool rises = vdw ? (vA < T(0)) : (vA > T(0));
        const bool falls = vdw ? (vA > T(0)) : (vA < T(0));
        if (inside ? rises : falls) continue;
        if (vdw) {
            T v32[3] = {d[0], d[1], d[2]};
            v32[axis] += t;
            const T nvv = sqrt(v32[0] * v32[0] + v32[1] * v32[1] + v32[2] * v32[2]);
            const T Rr = c.w + rpT;
            const T sc = Rr / nvv;
            int f = -1;
            if (FILT) {
                const T delta = d0 + terr * (T(1) + sc) + T(2e-6);
                f = free_witness<true>(A, c.x + sc * v32[0], c.y + sc * v32[1], c.z + sc * v32[2], slot, -1,
                                       A.agid(slot), -1, rpT, delta);
            }
            if (f < 0) {
                const P4<double> ce = X.atom(slot);
                const double cc[3] = {ce.x, ce.y, ce.z};
                if (t64 != t64) t64 = exact_root_sphere(cc, ce.w, s64, axis, (double)t);
                double v[3] = {s64[0] - cc[0], s64[1] - cc[1], s64[2] - cc[2]};
                v[axis] += t64;
                const double nv64 = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
                const double R64 = ce.w + rp;
                f = free_witness<false>(X, cc[0] + R64 * v[0] / nv64, cc[1] + R64 * v[1] / nv64,
                                        cc[2] + R64 * v[2] / nv64, slot, -1, A.agid(slot), -1, rp, 0.0);
            }
            if (f != 1) continue;
        }
        out.push((float)t, (float)terr, t64);
    }
}

// Tori (saddle pieces) around the free-arc circle of staged pair pi: roots on
// the near branch, isolated in FP32 (certified) with the quartic on its
// derivative chain and FP64 where that cannot decide.
template <class T, bool FILT, class AccT, class AccX>
__device__ void torus_roots(const AccT &A, const AccX &X, int pi, const double *s64, int axis, bool inside, double h,
                            double rp, T d0, RootSink &out)
{
    if constexpr (!FILT) {
        torus_piece_exact(A, out, pi, s64, axis, h, rp, inside);
    } else {
        const T s[3] = {(T)s64[0], (T)s64[1], (T)s64[2]};
        const T hT = (T)h, rpT = (T)rp;
        const T lo = T(-1e-4), hi = hT + T(1e-4);
        const T tmax = T(1e-3);
        const double NaN = __longlong_as_double(0x7ff8000000000000LL);
        const P4<T> o = A.po(pi);
        const P4<T> u = A.pu(pi);
        const float q0[3] = {s[0] - o.x, s[1] - o.y, s[2] - o.z};
        const float uu[3] = {u.x, u.y, u.z};
        float rt[4];
        int nr = 0;
        if (!torus_roots32(q0, uu, o.w, rpT, axis, lo, hi, d0, rt, nr)) {
            // sampling undecided (near-tangent line, or close to the circle's axis): the
            // quartic's roots on the derivative chain
            const float P = q0[0] * q0[0] + q0[1] * q0[1] + q0[2] * q0[2];
            const float z0 = q0[0] * uu[0] + q0[1] * uu[1] + q0[2] * uu[2];
            const float pe = q0[axis], eu = uu[axis];
            const float K = P + o.w * o.w - rpT * rpT, r2 = o.w * o.w;
            const float co32[5] = {K * K - 4.0f * r2 * (P - z0 * z0), 4.0f * pe * K - 8.0f * r2 * (pe - z0 * eu),
                                   4.0f * pe * pe + 2.0f * K - 4.0f * r2 * (1.0f - eu * eu), 4.0f * pe, 1.0f};
            float rq[4];
            const int nq = PolyRoots<float, 4>::run(co32, lo, hi, rq);
            nr = 0;
            for (int k = 0; k < nq; ++k) {
                float D, dD, nw, yy, zy, wv[3];
                circle_dist32(q0, uu, o.w, axis, rq[k], D, dD, nw, yy, zy, wv);
                // near branch: A = |y|^2 + rho^2 - r_p^2 >= 0; undecided signs go to FP64
                const float Ay = yy + r2 - rpT * rpT;
                if (fabsf(Ay) < 1e-3f * (yy + r2 + rpT * rpT)) nr = -1;
                else if (Ay > 0.0f && nr >= 0) rt[nr++] = rq[k];
            }
            if (nr < 0) {
                torus_piece_exact(X, out, pi, s64, axis, h, rp, inside);
                return;
            }
        }
        const int2 ij = A.pij(pi);
        const short2 sl = A.pslot(pi);
        for (int k = 0; k < nr; ++k) {
            const float t = rt[k];
            float D, rate, nw, yy, zy, wv[3];
            circle_dist32(q0, uu, o.w, axis, t, D, rate, nw, yy, zy, wv);
            // root error: residual plus rounding of g over |g'| (g' varies little within terr)
            const float terr =
                (fabsf(D - rpT) + circle_dist_err(d0, yy, nw, o.w, rpT)) / fmax(fabs(rate), 1e-20f) + d0;
            if (terr > tmax || t < terr + 1e-6f || t > hT - terr - 1e-6f || fabs(rate) < 1e-3f ||
                nw < 1e-3f) {  // grazing or at an end point: the FP64 root decides
                const P4<double> oe = X.po(pi);
                const P4<double> ue = X.pu(pi);
                const double oo[3] = {oe.x, oe.y, oe.z}, u64[3] = {ue.x, ue.y, ue.z};
                const double t64 = exact_root_torus(oo, u64, oe.w, rp, s64, axis, (double)t);
                torus_root_exact(X, out, pi, s64, axis, h, rp, inside, t64);
                continue;
            }
            if (inside ? rate > 0.0f : rate < 0.0f) continue;
            const float kk = o.w / nw;
            const float delta = d0 + terr * (1.0f + 2.0f * o.w / nw) + 2e-6f;
            const int f = free_witness<true>(A, o.x + kk * wv[0], o.y + kk * wv[1], o.z + kk * wv[2], (int)sl.x,
                                             (int)sl.y, ij.x, ij.y, rpT, delta);
            if (f == 1) {
                out.push(t, terr, NaN);
            } else if (f < 0) {
                const P4<double> oe = X.po(pi);
                const P4<double> ue = X.pu(pi);
                const double oo[3] = {oe.x, oe.y, oe.z}, u64[3] = {ue.x, ue.y, ue.z};
                const double t64 = exact_root_torus(oo, u64, oe.w, rp, s64, axis, (double)t);
                torus_root_exact(X, out, pi, s64, axis, h, rp, inside, t64);
            }
        }
    }
}

// First root of one crossing edge from its candidates c[0, n) (whole warp; c
// in shared memory, updated in place).  Returns 0 with the chosen piece (kind,
// staged slot) and its root, 1 when no root is found, 2 when the candidates
// overflowed the buffer (the first WCAND are used).
template <class T, bool FILT, class AccT, class AccX>
__device__ int warp_select(const AccT &A, const AccX &X, WCand *c, int n, const T *s, const double *s64, int axis,
                           bool inside, float hf, T rpT, double rp, T d0, float &t_out, int &kind_out, int &slot_out)
{
    const int lane = threadIdx.x & 31;
    const float tie = 1e-6f * hf;  // FP32 rounding of a root
    int status = n > WCAND ? 2 : 0;
    if (n > WCAND) n = WCAND;
    int pick = -1;
    for (int iter = 0; iter <= n; ++iter) {
        int k = warp_argmin(c, n);
        if (k < 0) break;
        // candidates that the FP32 bounds cannot order against k: settle with FP64 roots
        const float tk = c[k].t, ek = c[k].err;
        bool tied = false;
        for (int j = lane; j < n; j += 32)
            if (j != k && c[j].t < INFINITY && c[j].t - tk <= c[j].err + ek + tie) tied = true;
        if (__any_sync(0xffffffffu, tied)) {
            for (int j = lane; j < n; j += 32)
                if (c[j].t < INFINITY && c[j].t - tk <= c[j].err + ek + tie && c[j].t64 != c[j].t64)
                    c[j].t64 = staged_exact_root(X, c[j].kind, c[j].id, s64, axis, rp, (double)c[j].t);
            __syncwarp();
            double bt = INFINITY;
            int bk = -1;
            for (int j = lane; j < n; j += 32)
                if (c[j].t < INFINITY && c[j].t - tk <= c[j].err + ek + tie && c[j].t64 < bt) {
                    bt = c[j].t64;
                    bk = j;
                }
            for (int o = 16; o > 0; o >>= 1) {
                double ot = __shfl_xor_sync(0xffffffffu, bt, o);
                int ok = __shfl_xor_sync(0xffffffffu, bk, o);
                if (ok >= 0 && (bk < 0 || ot < bt || (ot == bt && ok < bk))) {
                    bt = ot;
                    bk = ok;
                }
            }
            k = bk;
        }
        if (inside) {
            pick = k;
            break;
        }
        // outside end point: the root must not be strictly outside M.  The
        // surface crossing is always a candidate (the nearest free point at
        // it is a piece's free witness) and every candidate before it lies
        // strictly outside, so the last candidate left needs no test.
        bool others = false;
        for (int j = lane; j < n; j += 32)
            if (j != k && c[j].t < INFINITY) others = true;
        if (!__any_sync(0xffffffffu, others)) {
            pick = k;
            break;
        }
        int r;
        unsigned um_prop = 0u, um_vert = 0u;
        if (FILT) {
            // FP32 position: the FP32 root and its bound, or the exact root
            // rounded (its rounding and that of the sum within 2e-7 A)
            const bool ex = c[k].t64 == c[k].t64;
            T y0 = s[0], y1 = s[1], y2 = s[2];
            T tt = ex ? (T)c[k].t64 : (T)c[k].t;
            if (axis == 0) y0 += tt;
            else if (axis == 1) y1 += tt;
            else y2 += tt;
            const T dk = d0 + (ex ? T(2e-7) : (T)c[k].err);
            // First the witnesses of the other remaining candidates' pieces at
            // y_k: the crossing is a later candidate, whose witness at y_k is
            // usually free and closer than r_p (then y_k is strictly outside M).
            // Only a certain answer counts; otherwise the full search decides.
            T qx = T(0), qy = T(0), qz = T(0), dq = T(0);
            int e0 = -1, e1 = -1, tw = 0;
            bool vnear = false;
            if (lane < n && lane != k && c[lane].t < INFINITY &&
                !(c[lane].kind == c[k].kind && c[lane].id == c[k].id)) {
                const int id = c[lane].id;
                if (c[lane].kind == 0) {
                    tw = face_proposal<true>(A, id, y0, y1, y2, rpT, rpT, dk, qx, qy, qz, dq, e0, e1);
                } else if (c[lane].kind == 1) {
                    tw = saddle_proposal<true>(A, id, y0, y1, y2, rpT, rpT, dk, qx, qy, qz, dq, e0, e1);
                } else {  // a free triple point closer than r_p
                    const P4<T> v = A.vq(id);
                    const T dx = y0 - v.x, dy = y1 - v.y, dz = y2 - v.z;
                    vnear = lt_sq<true>(dx * dx + dy * dy + dz * dz, rpT * rpT, rpT, dk) == 1;
                }
            }
            bool und = false, mine = false;
            if (__any_sync(0xffffffffu, vnear) ||
                warp_test_proposals<true>(A, __ballot_sync(0xffffffffu, tw == 1), tw, qx, qy, qz, dq, e0, e1, rpT,
                                          dk, und, mine) == 1)
                r = 1;
            else
                r = warp_witness<true>(A, y0, y1, y2, rpT, rpT, dk, c[k].kind, c[k].id, um_prop, um_vert);
        } else {
            r = -2;
        }
        if (r < 0) {  // FP64 at the exact root: the undecided items only, or the whole search
            double t64 = c[k].t64;
            if (t64 != t64) t64 = staged_exact_root(X, c[k].kind, c[k].id, s64, axis, rp, (double)c[k].t);
            double y[3] = {s64[0], s64[1], s64[2]};
            y[axis] += t64;
            if (r == -1)
                r = warp_witness_retest(X, y[0], y[1], y[2], rp, rp - 1e-11, um_prop, um_vert);
            else
                r = warp_witness<false>(X, y[0], y[1], y[2], rp, rp - 1e-11, 0.0, -1, -1, um_prop, um_vert);
        }
        if (r == 0) {
            pick = k;
            break;
        }
        __syncwarp();
        if (lane == 0) c[k].t = INFINITY;  // strictly outside M: not the root
        __syncwarp();
    }
    if (pick < 0) return 1;
    t_out = c[pick].t64 == c[pick].t64 ? (float)c[pick].t64 : c[pick].t;
    kind_out = c[pick].kind;
    slot_out = c[pick].id;
    return status;
}

// Per tile and axis: crossing edges (end labels differ) and inside edges (both
// ends inside) leaving the tile's points in + direction, and the tile's inside
// points.  One warp per tile, 16 points per lane, warp sums (no block barrier).
constexpr int COUNT_WARPS = 8;

__global__ void __launch_bounds__(COUNT_WARPS * 32) k_edge_count(Batch B, const int8_t *__restrict__ labels_all,
                                                                int *__restrict__ tile_edges,
                                                                int *__restrict__ tile_inside)
{
    const int lane = threadIdx.x & 31;
    const long long nt = B.n_tiles;
    const long long nw = (long long)gridDim.x * COUNT_WARPS;
    for (long long gt = (long long)blockIdx.x * COUNT_WARPS + (threadIdx.x >> 5); gt < nt; gt += nw) {
        const Grid &G = B.grid[mol_of_tile(B, gt)];
        const long long dims[3] = {G.dims[0], G.dims[1], G.dims[2]};
        const long long own[3] = {G.own[0], G.own[1], G.own[2]};
        const int8_t *__restrict__ labels = labels_all + G.lab0;
        const long long st1 = dims[2], st0 = dims[1] * dims[2];
        int t[3];
        tile_coords(G, gt - G.tile0, t);
        int ce[3] = {0, 0, 0}, ci[3] = {0, 0, 0}, npin = 0;
        for (int p = lane; p < TILE_PTS; p += 32) {
            const long long g[3] = {(long long)TILE * t[0] + (p >> 6), (long long)TILE * t[1] + ((p >> 3) & 7),
                                    (long long)TILE * t[2] + (p & 7)};
            if (g[0] >= own[0] || g[1] >= own[1] || g[2] >= own[2]) continue;  // not owned (or not in the grid)
            const long long idx = g[0] * st0 + g[1] * st1 + g[2];
            const int l0 = labels[idx];
            npin += l0;
            const long long str[3] = {st0, st1, 1};
            for (int a = 0; a < 3; ++a) {
                if (g[a] + 1 >= dims[a]) continue;
                const int l1 = labels[idx + str[a]];
                if (l0 != l1) ++ce[a];
                else if (l0) ++ci[a];
            }
        }
        for (int a = 0; a < 3; ++a) {
            ce[a] = __reduce_add_sync(0xffffffffu, ce[a]);
            ci[a] = __reduce_add_sync(0xffffffffu, ci[a]);
        }
        npin = __reduce_add_sync(0xffffffffu, npin);
        if (lane < 3) {
            tile_edges[lane * nt + gt] = lane == 0 ? ce[0] : (lane == 1 ? ce[1] : ce[2]);
            tile_inside[lane * nt + gt] = lane == 0 ? ci[0] : (lane == 1 ? ci[1] : ci[2]);
        } else if (lane == 3) {
            tile_inside[3 * nt + gt] = npin;
        }
    }
}

// per axis, the first crossing edge of every molecule in the axis' output
// (medge[a * (n_mol + 1) + m]; m = n_mol gives the axis total)
__global__ void k_mol_edges(Batch B, const int *__restrict__ edge_start, long long *__restrict__ medge)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= 3 * (B.n_mol + 1)) return;
    const int a = k / (B.n_mol + 1), m = k % (B.n_mol + 1);
    const long long nt = B.n_tiles;
    medge[k] = (long long)edge_start[a * nt + B.tile_off[m]] - edge_start[a * nt];
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

template <class T, class CP>
__host__ __device__ constexpr size_t edge_tile_bytes()  // rounded to 256: aligned slices in global memory
{
    return (sizeof(TileS<T, CP>) + 255) & ~(size_t)255;
}

// exclusive prefix sums of v[0..n) and w[0..n) in place (whole block), the
// totals at v[n] and w[n]; each thread sums a contiguous run of entries
__device__ __forceinline__ void block_scan_runs(int *v, int *w, int n, int *sh, int *sh2)
{
    const int per = (n + EDGE_THREADS - 1) / EDGE_THREADS;
    const int b = threadIdx.x * per, e = min(n, b + per);
    int sv = 0, sw = 0;
    for (int k = b; k < e; ++k) {
        sv += v[k];
        sw += w[k];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int iv = sv, iw = sw;
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(0xffffffffu, iv, o);
        const int c = __shfl_up_sync(0xffffffffu, iw, o);
        if (lane >= o) {
            iv += a;
            iw += c;
        }
    }
    if (lane == 31) {
        sh[wid] = iv;
        sh2[wid] = iw;
    }
    __syncthreads();
    int bv = 0, bw = 0, tv = 0, tw = 0;
    for (int k = 0; k < EDGE_WARPS; ++k) {
        if (k < wid) {
            bv += sh[k];
            bw += sh2[k];
        }
        tv += sh[k];
        tw += sh2[k];
    }
    int rv = bv + iv - sv, rw = bw + iw - sw;
    for (int k = b; k < e; ++k) {
        const int a = v[k], c = w[k];
        v[k] = rv;
        w[k] = rw;
        rv += a;
        rw += c;
    }
    if (threadIdx.x == 0) {
        v[n] = tv;
        w[n] = tw;
    }
    __syncthreads();
}

// 1. Staging pass.  Persistent CTAs take tiles from the work queue.  Per tile
// with crossing edges: the pieces are staged (CP = CapMid: in shared memory,
// a tile that overflows it goes to ovf; CP = CapBig (BIG): the tiles listed in
// ovf, staged in this CTA's slice of the global scratch `big`, lists cut at
// capacity with the error bit set), the crossing edges listed per axis in
// point order, and written to HBM: the staged lists (the tile's slab), per
// edge its output point index and its record (einfo, ecnt), and the (edge,
// piece) pairs that pass the prefilter, spheres and tori in separate lists,
// each edge's run in item order.  A buffer that is full drops the tile's
// edges (flagged); the counters still add up what was needed.
template <class T, bool FILT, class CP, bool BIG>
__global__ void __launch_bounds__(EDGE_THREADS) k_edge_stage(Model M, Batch B, TileSched Q,
                                                             const int8_t *__restrict__ labels_all,
                                                             const int *__restrict__ edge_start, EdgeOut out,
                                                             int *__restrict__ err, int *__restrict__ ovf,
                                                             unsigned char *__restrict__ big, RootWork W)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileS<T, CP> &S = *reinterpret_cast<TileS<T, CP> *>(BIG ? big + (size_t)blockIdx.x * edge_tile_bytes<T, CP>()
                                                             : smem_raw);
    StageSmem &E = *reinterpret_cast<StageSmem *>(BIG ? smem_raw : smem_raw + edge_tile_bytes<T, CP>());
    __shared__ long long q_base;
    __shared__ Grid sG;
    const long long nt = B.n_tiles;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const T rpT = (T)M.rp, mg = FILT ? T(2e-3) : T(0);
    long long iter = 0;
    const long long npos = sched_count(Q, nt);
    for (;;) {
      const long long base = next_tiles(Q, iter, &q_base);
      if (base >= npos) break;
      const long long bend = min(base + (long long)Q.per, npos);
      for (long long pos = base; pos < bend; ++pos) {
        const long long gt = sched_tile(Q, pos);
        int tot = 0;
        for (int a = 0; a < 3; ++a) tot += edge_start[a * nt + gt + 1] - edge_start[a * nt + gt];
        if (tot == 0) continue;
        const int mol = mol_of_tile(B, gt);
        load_grid(B, mol, sG);
        const Grid &G = sG;
        const long long tile = gt - G.tile0;
        const int8_t *__restrict__ labels = labels_all + G.lab0;
        const long long st1 = G.dims[2], st0 = G.dims[1] * G.dims[2];
        const long long fst1 = G.full[2], fst0 = G.full[1] * G.full[2];  // strides of the output indices
        const double h = G.h;
        const T hT = (T)h;
        double x0[3];
        stage_tile<T>(M, G, mol, tile, S, x0);
        if (!BIG && (S.flags & ERR_CAP_ANY)) {  // uniform: set before stage_tile's last barrier
            if (threadIdx.x == 0) {  // to the global-memory tier (ovf: run total, stage count, tiles)
                atomicAdd(&ovf[0], 1);
                const int k = atomicAdd(&ovf[1], 1);
                ovf[2 + k] = (int)gt;
            }
            __syncthreads();
            continue;
        }
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
                const bool owned = TILE * t[0] + l[0] < G.own[0] && TILE * t[1] + l[1] < G.own[1] &&
                                   TILE * t[2] + l[2] < G.own[2];
                int8_t l0 = E.lab[(l[0] * 9 + l[1]) * 9 + l[2]];
                l[a] += 1;
                int8_t l1 = E.lab[(l[0] * 9 + l[1]) * 9 + l[2]];
                flag[k] = (owned && l0 >= 0 && l1 >= 0 && l0 != l1) ? 1 : 0;
            }
            int tsum;
            int rank = block_excl_scan_e(flag[0] + flag[1], E.sh, &tsum);
            const int eb = E.estart[a];
            for (int k = 0; k < 2; ++k)
                if (flag[k]) E.eptr[eb + rank++] = (short)(2 * threadIdx.x + k);
            if (threadIdx.x == 0) {
                E.estart[a + 1] = eb + tsum;
                E.gbase[a] = edge_start[a * nt + gt];
                E.abase[a] = edge_start[a * nt + gt] - edge_start[a * nt];
            }
            __syncthreads();
        }
        const int ne = E.estart[3];
        const int na = S.na, np = S.np, nv = S.nv, nsph = na + nv, nitem = nsph + np;
        if (threadIdx.x == 0) {  // the tile's slab
            const unsigned long long bytes = (unsigned long long)SlabLayout<T>(na, np, nv).bytes;
            const unsigned long long off = atomicAdd(W.ctr, bytes);
            E.slab = off + bytes <= (unsigned long long)W.cap_slab ? (long long)(off >> 4) : -1LL;
        }
        // output point index of every edge (full grid)
        for (int e = threadIdx.x; e < ne; e += EDGE_THREADS) {
            const EdgeRef R = edge_ref(E, e);
            const int li = R.p >> 6, lj = (R.p >> 3) & 7, lk = R.p & 7;
            out.idx[R.axis][E.abase[R.axis] + (e - E.estart[R.axis])] =
                (long long)(TILE * (t[0] + G.toff[0]) + li) * fst0 + (long long)(TILE * (t[1] + G.toff[1]) + lj) * fst1 +
                (TILE * (t[2] + G.toff[2]) + lk);
        }
        // (edge, item) pairs that pass the prefilter, counted: one warp per edge,
        // lanes over items; the hit masks kept when they fit
        const int nwd = (nitem + 31) >> 5;
        const bool keep = (long long)ne * nwd <= HMASK_WORDS;
        for (int e = warp; e < ne; e += EDGE_WARPS) {
            const EdgeRef R = edge_ref(E, e);
            T s[3], hs;
            edge_point<T>(G, R.p, s, hs);
            int cs = 0, ct = 0;
            for (int i0 = 0; i0 < nitem; i0 += 32) {
                const int it = i0 + lane;
                const bool hit = it < nitem && cand_test<T, CP>(S, s, R.axis, it, hT, rpT, mg);
                const unsigned m = __ballot_sync(0xffffffffu, hit), sm = sphere_bits(i0 >> 5, nsph);
                cs += __popc(m & sm);
                ct += __popc(m & ~sm);
                if (keep && lane == 0) E.hmask[e * nwd + (i0 >> 5)] = m;
            }
            if (lane == 0) {
                E.cs[e] = cs;
                E.ct[e] = ct;
            }
        }
        __syncthreads();
        block_scan_runs(E.cs, E.ct, ne, E.sh, E.sh2);
        if (threadIdx.x == 0) {
            const unsigned long long ns = (unsigned long long)E.cs[ne], nq = (unsigned long long)E.ct[ne];
            const unsigned long long sb = atomicAdd(W.ctr + 1, ns);
            const unsigned long long tb = atomicAdd(W.ctr + 2, nq);
            const bool ok = E.slab >= 0 && sb + ns <= (unsigned long long)W.cap_sph &&
                            tb + nq <= (unsigned long long)W.cap_tor;
            E.sb = ok ? (long long)sb : -1LL;
            E.tb = ok ? (long long)tb : -1LL;
            E.sb0 = (long long)sb;
            E.tb0 = (long long)tb;
        }
        __syncthreads();
        const bool ok = E.sb >= 0;
        if (ok) {  // the slab: header and staged lists
            unsigned char *sl = W.slab + ((size_t)E.slab << 4);
            const SlabLayout<T> L(na, np, nv);
            if (threadIdx.x == 0) {
                SlabHdr hd;
                hd.na = na;
                hd.np = np;
                hd.nv = nv;
                hd.mol = mol;
                for (int a = 0; a < 3; ++a) {
                    hd.x0[a] = x0[a];
                    hd.t[a] = t[a];
                }
                hd.gt = (int)gt;
                *reinterpret_cast<SlabHdr *>(sl) = hd;
            }
            P4<T> *pa = reinterpret_cast<P4<T> *>(sl + L.atom);
            P4<T> *po = reinterpret_cast<P4<T> *>(sl + L.po);
            P4<T> *pu = reinterpret_cast<P4<T> *>(sl + L.pu);
            P4<T> *pv = reinterpret_cast<P4<T> *>(sl + L.vq);
            int *ag = reinterpret_cast<int *>(sl + L.agid);
            int2 *pj = reinterpret_cast<int2 *>(sl + L.pij);
            int *px = reinterpret_cast<int *>(sl + L.pidx);
            int *vx = reinterpret_cast<int *>(sl + L.vidx);
            uint8_t *fc = reinterpret_cast<uint8_t *>(sl + L.face);
            for (int k = threadIdx.x; k < na; k += EDGE_THREADS) {
                pa[k] = S.atom[k];
                ag[k] = S.agid[k];
                fc[k] = S.aface[k];
            }
            for (int k = threadIdx.x; k < np; k += EDGE_THREADS) {
                po[k] = S.po[k];
                pu[k] = S.pu[k];
                pj[k] = S.pij[k];
                px[k] = S.pidx[k];
            }
            for (int k = threadIdx.x; k < nv; k += EDGE_THREADS) {
                pv[k] = S.vq[k];
                vx[k] = S.vidx[k];
            }
            // neighbour sets (expanded spheres within 1e-3 A of meeting; the
            // margin covers the rounding of the staged FP32 positions)
            unsigned *nbm = reinterpret_cast<unsigned *>(sl + L.nbm);
            const int nw = (na + 31) >> 5;
            for (int it = threadIdx.x; it < na * nw; it += EDGE_THREADS) {
                const int a = it / nw, w = it - a * nw;
                const P4<T> ca = S.atom[a];
                const T Ra = ca.w + rpT + T(1e-3);
                unsigned bits = 0u;
                const int b0 = w << 5, b1 = min(na, b0 + 32);
                for (int b = b0; b < b1; ++b) {
                    const P4<T> cb = S.atom[b];
                    const T dx = ca.x - cb.x, dy = ca.y - cb.y, dz = ca.z - cb.z;
                    const T reach = Ra + cb.w + rpT;
                    if (b != a && dx * dx + dy * dy + dz * dz < reach * reach) bits |= 1u << (b - b0);
                }
                nbm[it] = bits;
            }
            // staged slots of every pair's atoms
            short2 *ps = reinterpret_cast<short2 *>(sl + L.pslot);
            for (int k = threadIdx.x; k < np; k += EDGE_THREADS) {
                const int2 ij = S.pij[k];
                int si = -1, sj = -1;
                for (int a = 0; a < na; ++a) {
                    const int g = S.agid[a];
                    si = g == ij.x ? a : si;
                    sj = g == ij.y ? a : sj;
                }
                ps[k] = make_short2((short)si, (short)sj);
            }
        }
        // edge records
        for (int e = threadIdx.x; e < ne; e += EDGE_THREADS) {
            const EdgeRef R = edge_ref(E, e);
            const long long g = (long long)E.gbase[R.axis] + (e - E.estart[R.axis]);
            W.einfo[g] = make_int4(ok ? (int)E.slab : 0, edge_pack(R.p, R.axis, R.lab, ok ? 0 : 1),
                                   ok ? (int)(E.sb + E.cs[e]) : 0, ok ? (int)(E.tb + E.ct[e]) : 0);
            W.ecnt[g] = ok ? ((E.cs[e + 1] - E.cs[e]) | ((E.ct[e + 1] - E.ct[e]) << 16)) : 0;
        }
        // the pairs themselves, in item order.  Every slot of the reserved runs
        // below the capacities is written: a slot no pair fills (a dropped tile,
        // or a second prefilter pass that disagreed with the count) gets a dead
        // record (edge -1), so the root kernels never read an unwritten slot.
        if (ok) {
            for (int e = warp; e < ne; e += EDGE_WARPS) {
                const EdgeRef R = edge_ref(E, e);
                const int g = E.gbase[R.axis] + (e - E.estart[R.axis]);
                T s[3], hs;
            edge_point<T>(G, R.p, s, hs);
                long long ps = E.sb + E.cs[e], pt = E.tb + E.ct[e];
                const long long ps1 = E.sb + E.cs[e + 1], pt1 = E.tb + E.ct[e + 1];
                const unsigned below = (1u << lane) - 1;
                for (int i0 = 0; i0 < nitem; i0 += 32) {
                    const int it = i0 + lane;
                    const unsigned m =
                        keep ? E.hmask[e * nwd + (i0 >> 5)]
                             : __ballot_sync(0xffffffffu, it < nitem && cand_test<T, CP>(S, s, R.axis, it, hT, rpT, mg));
                    const bool hit = (m >> lane) & 1u;
                    const unsigned sm = sphere_bits(i0 >> 5, nsph), ms = m & sm, mt = m & ~sm;
                    const long long qs = ps + __popc(ms & below), qt = pt + __popc(mt & below);
                    if (hit && it < nsph && qs < ps1) W.csph[qs] = make_int2(g, it);
                    if (hit && it >= nsph && qt < pt1) W.ctor[qt] = make_int2(g, it - nsph);
                    ps += __popc(ms);
                    pt += __popc(mt);
                }
                for (long long q = ps + lane; q < ps1; q += 32) W.csph[q] = make_int2(-1, 0);
                for (long long q = pt + lane; q < pt1; q += 32) W.ctor[q] = make_int2(-1, 0);
            }
        } else {
            const long long s1 = min(E.sb0 + E.cs[ne], W.cap_sph), t1 = min(E.tb0 + E.ct[ne], W.cap_tor);
            for (long long q = E.sb0 + threadIdx.x; q < s1; q += EDGE_THREADS) W.csph[q] = make_int2(-1, 0);
            for (long long q = E.tb0 + threadIdx.x; q < t1; q += EDGE_THREADS) W.ctor[q] = make_int2(-1, 0);
        }
        __syncthreads();
      }
    }
}

// slab, grid and edge geometry of global edge g's record
struct EdgeView {
    const unsigned char *slab;
    int axis, p, lab;
    double s64[3];  // lower point in the tile frame
};

// 2. Roots of the sphere candidates, one thread each (grid-stride).
template <class T, bool FILT>
__global__ void __launch_bounds__(ROOT_THREADS_MAX) k_roots_sphere(Model M, Batch B, RootWork W,
                                                                   int *__restrict__ err)
{
    const long long n = min((long long)W.ctr[1], W.cap_sph);
    const double rp = M.rp;
    const T rpT = (T)rp;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int2 c = W.csph[k];
        if (c.x < 0 || c.x >= W.n_edges) {  // dead record
            W.nsph[k] = 0;
            continue;
        }
        const int4 inf = W.einfo[c.x];
        const unsigned char *sl = W.slab + ((size_t)(unsigned)inf.x << 4);
        const SlabHdr *hd = reinterpret_cast<const SlabHdr *>(sl);
        const int mol = __ldg(&hd->mol);
        const double x0[3] = {__ldg(&hd->x0[0]), __ldg(&hd->x0[1]), __ldg(&hd->x0[2])};
        const double h = B.grid[mol].h;
        const T d0 = FILT ? (T)B.grid[mol].d0 : T(0);
        const int pk = inf.y, p = pk_point(pk);
        const double s64[3] = {(double)(p >> 6) * h, (double)((p >> 3) & 7) * h, (double)(p & 7) * h};
        T s[3], hT;
        edge_point<T>(B.grid[mol], p, s, hT);
        const SlabAcc<T> A(sl);
        const SlabExact<T> X(A, M, x0);
        RootSink out{W.rsph + (size_t)SPH_SLOTS * k, 0, SPH_SLOTS};
        sphere_roots<T, FILT>(A, X, c.y, s, s64, pk_axis(pk), pk_label(pk) == LABEL_IN, hT, rpT, h, rp, d0, out);
        if (out.n > SPH_SLOTS) atomicOr(err, ERR_CAP_CAND);
        W.nsph[k] = (uint8_t)min(out.n, SPH_SLOTS);
    }
}

// The FP32 part of torus_roots (FILT): the certified isolation and, per
// root, the FP32 decisions.  A root whose decision needs FP64 keeps a pending
// slot; a candidate whose isolation is undecided is left whole to the exact
// kernel.  Returns 0 (done), 1 (pending slots) or 2 (whole candidate).
template <class AccT>
__device__ int torus_roots_fp32(const AccT &A, int pi, const float *s, int axis, bool inside, float hT, float rpT,
                                float d0, RootSink &out)
{
    const float lo = -1e-4f, hi = hT + 1e-4f;
    const float tmax = 1e-3f;
    const double NaN = __longlong_as_double(0x7ff8000000000000LL);
    const P4<float> o = A.po(pi);
    const P4<float> u = A.pu(pi);
    const float q0[3] = {s[0] - o.x, s[1] - o.y, s[2] - o.z};
    const float uu[3] = {u.x, u.y, u.z};
    float rt[4];
    int nr = 0;
    if (!torus_roots32(q0, uu, o.w, rpT, axis, lo, hi, d0, rt, nr)) return 2;
    int job = 0;
    const int2 ij = A.pij(pi);
    const short2 sl = A.pslot(pi);
    for (int k = 0; k < nr; ++k) {
        const float t = rt[k];
        float D, rate, nw, yy, zy, wv[3];
        circle_dist32(q0, uu, o.w, axis, t, D, rate, nw, yy, zy, wv);
        const float terr = (fabsf(D - rpT) + circle_dist_err(d0, yy, nw, o.w, rpT)) / fmax(fabs(rate), 1e-20f) + d0;
        if (terr > tmax || t < terr + 1e-6f || t > hT - terr - 1e-6f || fabs(rate) < 1e-3f || nw < 1e-3f) {
            out.pend(t);  // grazing or at an end point: the FP64 root decides
            job = 1;
            continue;
        }
        if (inside ? rate > 0.0f : rate < 0.0f) continue;
        const float kk = o.w / nw;
        const float delta = d0 + terr * (1.0f + 2.0f * o.w / nw) + 2e-6f;
        const int f = free_witness<true>(A, o.x + kk * wv[0], o.y + kk * wv[1], o.z + kk * wv[2], (int)sl.x,
                                         (int)sl.y, ij.x, ij.y, rpT, delta);
        if (f == 1) {
            out.push(t, terr, NaN);
        } else if (f < 0) {
            out.pend(t);
            job = 1;
        }
    }
    return job;
}

// 3. Roots of the torus candidates, one thread each (grid-stride, the lanes
// of a warp together).  FP32 form: torus_roots_fp32, and the candidates with
// FP64 work listed for k_roots_torus_exact (one warp-aggregated append per
// iteration); FP64 form: every root in FP64 here.
template <class T, bool FILT>
__global__ void __launch_bounds__(ROOT_THREADS_MAX) k_roots_torus(Model M, Batch B, RootWork W,
                                                                  int *__restrict__ err)
{
    const long long n = min((long long)W.ctr[2], W.cap_tor);
    const double rp = M.rp;
    const float rpf = (float)rp;
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); k0 < n; k0 += stride) {
        const long long k = k0 + lane;
        int job = 0;
        if (k < n) {
        const int2 c = W.ctor[k];
        if (c.x < 0 || c.x >= W.n_edges) {  // dead record
            W.ntor[k] = 0;
        } else {
        const int4 inf = W.einfo[c.x];
        const unsigned char *sl = W.slab + ((size_t)(unsigned)inf.x << 4);
        const SlabHdr *hd = reinterpret_cast<const SlabHdr *>(sl);
        const int mol = __ldg(&hd->mol);
        const double x0[3] = {__ldg(&hd->x0[0]), __ldg(&hd->x0[1]), __ldg(&hd->x0[2])};
        const double h = B.grid[mol].h;
        const T d0 = FILT ? (T)B.grid[mol].d0 : T(0);
        const int pk = inf.y, p = pk_point(pk);
        const SlabAcc<T> A(sl);
        RootSink out{W.rtor + (size_t)TOR_SLOTS * k, 0, TOR_SLOTS};
        if constexpr (FILT) {
            float s[3], hT;
            edge_point<float>(B.grid[mol], p, s, hT);
            job = torus_roots_fp32(A, c.y, s, pk_axis(pk), pk_label(pk) == LABEL_IN, hT, rpf, (float)d0, out);
        } else {
            const double s64[3] = {(double)(p >> 6) * h, (double)((p >> 3) & 7) * h, (double)(p & 7) * h};
            const SlabExact<T> X(A, M, x0);
            torus_roots<T, FILT>(A, X, c.y, s64, pk_axis(pk), pk_label(pk) == LABEL_IN, h, rp, d0, out);
        }
        if (out.n > TOR_SLOTS) atomicOr(err, ERR_CAP_CAND);
        W.ntor[k] = (uint8_t)min(out.n, TOR_SLOTS);
        }
        }
        if constexpr (FILT) {  // list the candidates with FP64 work: (candidate, whole)
            const unsigned m = __ballot_sync(0xffffffffu, job != 0);
            if (m) {
                unsigned long long b = 0;
                if (lane == 0) b = atomicAdd(W.ctr + 4, (unsigned long long)__popc(m));
                b = __shfl_sync(0xffffffffu, b, 0);
                if (job != 0) {
                    const unsigned long long q = b + __popc(m & ((1u << lane) - 1));
                    // (a full list is reported by the run from the count)
                    if (q < (unsigned long long)W.cap_jobs) W.jobs[q] = make_int2((int)k, job);
                }
            }
        }
    }
}

// 3b. The listed torus candidates' FP64 work, one thread each (FP32 form
// only): job 1 settles the pending slots (the FP64 root next to the FP32 one,
// kept or rejected as torus_roots does), job 2 solves the whole candidate
// with torus_roots (the quartic on its derivative chain, FP64 where needed).
template <class T, bool FILT>
__global__ void __launch_bounds__(ROOT_THREADS_MAX) k_roots_torus_exact(Model M, Batch B, RootWork W,
                                                                        int *__restrict__ err)
{
    const long long n = min((long long)W.ctr[4], W.cap_jobs);
    const double rp = M.rp;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int2 jb = W.jobs[q];
        const long long k = jb.x;
        const int2 c = W.ctor[k];
        const int4 inf = W.einfo[c.x];
        const unsigned char *sl = W.slab + ((size_t)(unsigned)inf.x << 4);
        const SlabHdr *hd = reinterpret_cast<const SlabHdr *>(sl);
        const int mol = __ldg(&hd->mol);
        const double x0[3] = {__ldg(&hd->x0[0]), __ldg(&hd->x0[1]), __ldg(&hd->x0[2])};
        const double h = B.grid[mol].h;
        const T d0 = FILT ? (T)B.grid[mol].d0 : T(0);
        const int pk = inf.y, p = pk_point(pk), axis = pk_axis(pk);
        const bool inside = pk_label(pk) == LABEL_IN;
        const double s64[3] = {(double)(p >> 6) * h, (double)((p >> 3) & 7) * h, (double)(p & 7) * h};
        const SlabAcc<T> A(sl);
        const SlabExact<T> X(A, M, x0);
        RootRec *slots = W.rtor + (size_t)TOR_SLOTS * k;
        if (jb.y == 2) {
            RootSink out{slots, 0, TOR_SLOTS};
            torus_roots<T, FILT>(A, X, c.y, s64, axis, inside, h, rp, d0, out);
            if (out.n > TOR_SLOTS) atomicOr(err, ERR_CAP_CAND);
            W.ntor[k] = (uint8_t)min(out.n, TOR_SLOTS);
        } else {
            const P4<double> oe = X.po(c.y);
            const P4<double> ue = X.pu(c.y);
            const double oo[3] = {oe.x, oe.y, oe.z}, u64[3] = {ue.x, ue.y, ue.z};
            const int nr = W.ntor[k];
            for (int j = 0; j < nr; ++j) {
                const RootRec r = slots[j];
                if (!(r.err < 0.0f)) continue;
                const double t64 = exact_root_torus(oo, u64, oe.w, rp, s64, axis, (double)r.t);
                RootSink one{slots + j, 0, 1};
                torus_root_exact(X, one, c.y, s64, axis, h, rp, inside, t64);
                if (one.n == 0) slots[j] = no_root();
            }
        }
    }
}

// chosen piece of an edge for the FP64 polish: FP32 root, kind, model index,
// end label, failure
__device__ __forceinline__ void code_out(EdgeOut &out, int axis, long long o, int failed, float tr, int kind, int mid,
                                         int lab)
{
    out.code[axis][o] = make_int2(__float_as_int(tr), (kind << 29) | (lab << 28) | (failed << 27) | mid);
}

// 4. The first root of every edge whose choice needs neither a witness test
// nor an FP64 tie break -- an inside end point, or a single candidate (the
// last candidate needs no test) -- with no candidate the FP32 bounds cannot
// order: one thread per edge, candidates in order (spheres by item, then
// tori); the other edges are listed for the warp selection.  A dropped edge
// is recorded as failed (and the run as over capacity).
template <class T>
__global__ void __launch_bounds__(PICK_THREADS) k_edge_pick(Batch B, RootWork W, const int *__restrict__ edge_start,
                                                            long long ne_all, EdgeOut out, int *__restrict__ err)
{
    const long long nt = B.n_tiles;
    const int lane = threadIdx.x & 31;
    const long long nwarp = (long long)gridDim.x * (PICK_THREADS / 32);
    for (long long w0 = ((long long)blockIdx.x * (PICK_THREADS / 32) + (threadIdx.x >> 5)) * 32; w0 < ne_all;
         w0 += nwarp * 32) {
        const long long g = w0 + lane;
        bool hard = false;
        if (g < ne_all) {
            const int4 inf = W.einfo[g];
            const int cnt = W.ecnt[g];
            const int ns = cnt & 0xffff, nq = (cnt >> 16) & 0xffff;
            // the axis from the edge's place in the output (all axes in one run)
            const int axis = g < edge_start[nt] ? 0 : (g < edge_start[2 * nt] ? 1 : 2);
            const int pk = inf.y, lab = pk_label(pk);
            const long long o = g - edge_start[axis * nt];
            // a record that is not the staging pass's (never expected) counts as dropped
            const bool bad = pk_axis(pk) != axis || inf.x < 0 || 16LL * inf.x >= W.cap_slab || inf.z < 0 ||
                             inf.w < 0 || (long long)inf.z + ns > W.cap_sph || (long long)inf.w + nq > W.cap_tor;
            if (pk_dropped(pk) || bad) {
                atomicOr(err, ERR_CAP_CAND);
                code_out(out, axis, o, 1, 0.0f, 0, 0, lab);
            } else {
                const unsigned char *sl = W.slab + ((size_t)(unsigned)inf.x << 4);
                const SlabHdr *hd = reinterpret_cast<const SlabHdr *>(sl);
                const int na = __ldg(&hd->na);
                // smallest FP32 root (ties to the first), its record, and the count
                int n = 0, kind = -1, slot = 0, kn = -1;
                float tk = INFINITY, ek = 0.0f;
                double t64k = 0.0;
                for (int j = 0; j < ns; ++j) {
                    const int nr = W.nsph[inf.z + j];
                    for (int r = 0; r < nr; ++r) {
                        const RootRec q = W.rsph[(size_t)SPH_SLOTS * (inf.z + j) + r];
                        if (!(q.t < INFINITY)) continue;
                        if (q.t < tk) {
                            const int it = W.csph[inf.z + j].y;
                            tk = q.t;
                            ek = q.err;
                            t64k = q.t64;
                            kind = it < na ? 0 : 2;
                            slot = it < na ? it : it - na;
                            kn = n;
                        }
                        ++n;
                    }
                }
                for (int j = 0; j < nq; ++j) {
                    const int nr = W.ntor[inf.w + j];
                    for (int r = 0; r < nr; ++r) {
                        const RootRec q = W.rtor[(size_t)TOR_SLOTS * (inf.w + j) + r];
                        if (!(q.t < INFINITY) || q.err < 0.0f) continue;  // rejected (or never settled)
                        if (q.t < tk) {
                            tk = q.t;
                            ek = q.err;
                            t64k = q.t64;
                            kind = 1;
                            slot = W.ctor[inf.w + j].y;
                            kn = n;
                        }
                        ++n;
                    }
                }
                hard = !(n >= 1 && n <= WCAND && (lab == LABEL_IN || n == 1) && kn >= 0);
                if (!hard) {  // every other candidate ordered after it by the FP32 bounds
                    const float tie = 1e-6f * B.grid[__ldg(&hd->mol)].hl[1];
                    int m = 0;
                    for (int j = 0; j < ns && !hard; ++j) {
                        const int nr = W.nsph[inf.z + j];
                        for (int r = 0; r < nr; ++r) {
                            const RootRec q = W.rsph[(size_t)SPH_SLOTS * (inf.z + j) + r];
                            if (!(q.t < INFINITY)) continue;
                            if (m != kn && q.t - tk <= q.err + ek + tie) hard = true;
                            ++m;
                        }
                    }
                    for (int j = 0; j < nq && !hard; ++j) {
                        const int nr = W.ntor[inf.w + j];
                        for (int r = 0; r < nr; ++r) {
                            const RootRec q = W.rtor[(size_t)TOR_SLOTS * (inf.w + j) + r];
                            if (!(q.t < INFINITY) || q.err < 0.0f) continue;
                            if (m != kn && q.t - tk <= q.err + ek + tie) hard = true;
                            ++m;
                        }
                    }
                }
                if (!hard) {
                    const SlabAcc<T> A(sl);
                    const float tr = t64k == t64k ? (float)t64k : tk;
                    code_out(out, axis, o, 0, tr, kind, A.model_index(kind, slot), lab);
                }
            }
        }
        const unsigned m = __ballot_sync(0xffffffffu, hard);
        int base = 0;
        if (lane == 0 && m) base = (int)atomicAdd(W.ctr + 3, (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (hard) W.hard[base + __popc(m & ((1u << lane) - 1))] = (int)g;
    }
}

// 5. The listed edges: one warp per edge (grid-stride over the list).  The
// edge's accepted roots are gathered in candidate order into the warp's
// buffer in shared memory (at most WCAND; more is a capacity error), then
// chosen by warp_select.  A failure is logged with its candidates.
template <class T, bool FILT>
__global__ void __launch_bounds__(HARD_THREADS) k_edge_hard(Model M, Batch B, RootWork W,
                                                            const int *__restrict__ edge_start, EdgeOut out,
                                                            int *__restrict__ n_fail, int *__restrict__ err,
                                                            long long *__restrict__ fail_log)
{
    __shared__ WCand cand[HARD_THREADS / 32][WCAND];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long nt = B.n_tiles;
    const long long nh = (long long)W.ctr[3];
    const double rp = M.rp;
    const T rpT = (T)rp;
    WCand *c = cand[warp];
    for (long long q = (long long)blockIdx.x * (HARD_THREADS / 32) + warp; q < nh;
         q += (long long)gridDim.x * (HARD_THREADS / 32)) {
        const int g = W.hard[q];
        const int4 inf = W.einfo[g];
        const int cnt = W.ecnt[g];
        const int ns = cnt & 0xffff, nq = (cnt >> 16) & 0xffff;
        const int pk = inf.y, axis = pk_axis(pk), lab = pk_label(pk), p = pk_point(pk);
        const long long o = (long long)g - edge_start[axis * nt];
        const unsigned char *sl = W.slab + ((size_t)(unsigned)inf.x << 4);
        const SlabHdr *hd = reinterpret_cast<const SlabHdr *>(sl);
        const int mol = __ldg(&hd->mol);
        const double x0[3] = {__ldg(&hd->x0[0]), __ldg(&hd->x0[1]), __ldg(&hd->x0[2])};
        const double h = B.grid[mol].h;
        const T d0 = FILT ? (T)B.grid[mol].d0 : T(0);
        const double s64[3] = {(double)(p >> 6) * h, (double)((p >> 3) & 7) * h, (double)(p & 7) * h};
        T s[3], hT;
        edge_point<T>(B.grid[mol], p, s, hT);
        const SlabAcc<T> A(sl);
        const SlabExact<T> X(A, M, x0);
        const int na = A.na();
        // gather: lanes over candidates, each lane's roots at its prefix of the counts
        int n = 0;
        for (int j0 = 0; j0 < ns + nq; j0 += 32) {
            const int j = j0 + lane;
            const bool sph = j < ns;
            int nr = 0;
            if (j < ns + nq) nr = sph ? W.nsph[inf.z + j] : W.ntor[inf.w + (j - ns)];
            int inc = nr;
            for (int d = 1; d < 32; d <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, inc, d);
                if (lane >= d) inc += u;
            }
            const int at = n + inc - nr;
            if (nr > 0) {
                int kind, slot;
                if (sph) {
                    const int it = W.csph[inf.z + j].y;
                    kind = it < na ? 0 : 2;
                    slot = it < na ? it : it - na;
                } else {
                    kind = 1;
                    slot = W.ctor[inf.w + (j - ns)].y;
                }
                for (int r = 0; r < nr; ++r) {
                    if (at + r >= WCAND) break;
                    const RootRec qr = sph ? W.rsph[(size_t)SPH_SLOTS * (inf.z + j) + r]
                                           : W.rtor[(size_t)TOR_SLOTS * (inf.w + (j - ns)) + r];
                    WCand &w = c[at + r];
                    w.t64 = qr.t64;
                    w.t = qr.err < 0.0f ? INFINITY : qr.t;  // a rejected (or unsettled) slot: no candidate
                    w.err = qr.err;
                    w.kind = kind;
                    w.id = slot;
                }
            }
            n += __shfl_sync(0xffffffffu, inc, 31);
        }
        __syncwarp();
        float tr = 0.5f * (float)h;
        int kind = 0, slot = 0;
        int status = pk_dropped(pk) ? 2 : warp_select<T, FILT>(A, X, c, n, s, s64, axis, lab == LABEL_IN, (float)hT, rpT, rp, d0, tr,
                                                               kind, slot);
        if (lane == 0) {
            const int mid = status == 1 || pk_dropped(pk) ? 0 : A.model_index(kind, slot);
            if (status != 0) atomicOr(err, status == 1 ? ERR_ROOT : ERR_CAP_CAND);
            if (status == 1) {
                const int fs = atomicAdd(n_fail, 1);
                if (fs < FAIL_LOG) {
                    long long *rec = fail_log + FAIL_REC * fs;
                    for (int z = 0; z < FAIL_REC; ++z) rec[z] = 0;
                    rec[0] = axis;
                    rec[1] = (long long)TILE * __ldg(&hd->t[0]) + (p >> 6);
                    rec[2] = (long long)TILE * __ldg(&hd->t[1]) + ((p >> 3) & 7);
                    rec[3] = (long long)TILE * __ldg(&hd->t[2]) + (p & 7);
                    rec[4] = lab;
                    rec[5] = na;
                    rec[6] = A.np();
                    rec[7] = A.nv();
                    rec[8] = n;
                    for (int z = 0; z < 7 && z < n && z < WCAND; ++z) {
                        rec[9 + z] = (long long)((double)c[z].t * 1e9);
                        rec[16 + z] = c[z].kind;
                    }
                    rec[23] = mol;
                }
            }
            code_out(out, axis, o, status == 1 || pk_dropped(pk) ? 1 : 0, tr, kind, mid, lab);
        }
        __syncwarp();
    }
}

// One thread per crossing edge, over the three axes: FP64 root of the chosen
// piece next to the recorded FP32 root, normal, outputs, area/volume terms
// (block partial sums in fixed order).
__global__ void __launch_bounds__(POLISH_THREADS) k_edge_polish(Model M, Batch B, EdgeOut out,
                                                                const long long *__restrict__ medge,
                                                                double2 *__restrict__ term)
{
    const long long e = (long long)blockIdx.x * POLISH_THREADS + threadIdx.x;
    const int nm = B.n_mol;
    const long long n0 = medge[nm], n1 = medge[2 * nm + 1], n2 = medge[3 * nm + 2];
    const double rp = M.rp;
    if (e < n0 + n1 + n2) {
        const int a = e < n0 ? 0 : (e < n0 + n1 ? 1 : 2);
        const long long o = e - (a == 0 ? 0 : (a == 1 ? n0 : n0 + n1));
        // molecule of the edge: its axis output is molecule-major
        const long long *me = medge + a * (nm + 1);
        int lo = 0, hi = nm;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (me[mid] <= o) lo = mid;
            else hi = mid;
        }
        const Grid &G = B.grid[lo];
        const double h = G.h;
        const long long idx = out.idx[a][o];
        const int2 code = out.code[a][o];
        const float t32 = __int_as_float(code.x);
        const int kind = (code.y >> 29) & 3, lab_s = (code.y >> 28) & 1, failed = (code.y >> 27) & 1;
        const int mid = code.y & ((1 << 27) - 1);
        // the recorded piece must exist (a kind and index out of range is treated as a failed root)
        const bool bad = kind == 3 || (kind == 0 && mid >= M.n_atoms) || (kind == 1 && mid >= M.n_pairs) ||
                         (kind == 2 && mid >= M.n_verts);
        long long gi, gj, gk;  // full-grid point of the lower index
        if (idx < (1LL << 32) && G.full[1] * G.full[2] < (1LL << 32)) {  // 32-bit division where it fits
            const unsigned i32 = (unsigned)idx, d2 = (unsigned)G.full[2], d1 = (unsigned)G.full[1];
            const unsigned q = i32 / d2;
            gk = i32 - q * d2;
            gj = q % d1;
            gi = q / d1;
        } else {
            gi = idx / (G.full[1] * G.full[2]);
            gj = (idx / G.full[2]) % G.full[1];
            gk = idx % G.full[2];
        }
        const double s[3] = {G.lo[0] + h * (double)gi, G.lo[1] + h * (double)gj, G.lo[2] + h * (double)gk};
        double t = 0.5 * h, n[3] = {0.0, 0.0, 0.0};
        if (!failed && !bad) {
            double c[3], u[3] = {0.0, 0.0, 0.0}, rho = 0.0;
            if (kind == 0) {
                double4 g = M.atom[mid];
                c[0] = g.x; c[1] = g.y; c[2] = g.z;
                t = exact_root_sphere(c, g.w, s, a, (double)t32);
            } else if (kind == 2) {
                double4 g = M.vert[mid];
                c[0] = g.x; c[1] = g.y; c[2] = g.z;
                t = exact_root_sphere(c, rp, s, a, (double)t32);
            } else {
                double4 g = M.pair_o[mid];
                double4 q = M.pair_u[mid];
                c[0] = g.x; c[1] = g.y; c[2] = g.z;
                u[0] = q.x; u[1] = q.y; u[2] = q.z;
                rho = g.w;
                t = exact_root_torus(c, u, rho, rp, s, a, (double)t32);
            }
            t = fmin(fmax(t, 0.0), h);
            double y[3] = {s[0], s[1], s[2]};
            y[a] += t;
            exact_normal(kind, c, u, rho, y, n);
        }
        const double tau = t * (1.0 / h);
        out.tau[a][o] = tau;
        out.nrm[a][3 * o + 0] = n[0];
        out.nrm[a][3 * o + 1] = n[1];
        out.nrm[a][3 * o + 2] = n[2];
        out.tau32[a][o] = (float)tau;
        out.nrm32[a][3 * o + 0] = (float)n[0];
        out.nrm32[a][3 * o + 1] = (float)n[1];
        out.nrm32[a][3 * o + 2] = (float)n[2];
        // Crofton area term and the inside length of the edge (C9)
        term[e] = make_double2(h * h * fabs(n[a]), lab_s ? t : h - t);
    }
}

// Area/volume reduction in two fixed-order levels (deterministic): block
// (m, g) of k_reduce_part sums the terms of molecule m whose index within the
// molecule's range is g (mod RED_PARTS * blockDim), in a fixed tree;
// k_reduce_final adds the RED_PARTS partials of each molecule in order.
constexpr int RED_PARTS = 16;
constexpr int RED_THREADS = 512;

__global__ void __launch_bounds__(RED_THREADS) k_reduce_part(Batch B, const double2 *__restrict__ term,
                                                             const long long *__restrict__ medge,
                                                             const int *__restrict__ tile_inside,
                                                             double *__restrict__ part_d,
                                                             long long *__restrict__ part_i)
{
    __shared__ double sa[32], sv[32];
    __shared__ long long si[32], sp[32];
    const int m = blockIdx.x / RED_PARTS, g = blockIdx.x % RED_PARTS, nm = B.n_mol;
    const long long nt = B.n_tiles;
    const long long stride = (long long)RED_PARTS * RED_THREADS;
    const long long first = (long long)g * RED_THREADS + threadIdx.x;
    double a = 0.0, v = 0.0;
    long long ie = 0, pin = 0;
    long long axis_base = 0;
    for (int ax = 0; ax < 3; ++ax) {
        const long long *me = medge + ax * (nm + 1);
        for (long long k = me[m] + first; k < me[m + 1]; k += stride) {
            const double2 w = term[axis_base + k];
            a += w.x;
            v += w.y;
        }
        axis_base += me[nm];
    }
    for (long long k = B.tile_off[m] + first; k < B.tile_off[m + 1]; k += stride) {
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
        for (int k = 0; k < RED_THREADS / 32; ++k) {
            A += sa[k];
            V += sv[k];
            IE += si[k];
            P += sp[k];
        }
        part_d[2 * blockIdx.x] = A;
        part_d[2 * blockIdx.x + 1] = V;
        part_i[2 * blockIdx.x] = P;
        part_i[2 * blockIdx.x + 1] = IE;
    }
}

// out2[2m..] = {area, volume}; counts[2m..] = {inside points, inside edges (all axes)}
__global__ void k_reduce_final(Batch B, const double *__restrict__ part_d, const long long *__restrict__ part_i,
                               double *__restrict__ out2, long long *__restrict__ counts)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= B.n_mol) return;
    double A = 0.0, V = 0.0;
    long long P = 0, IE = 0;
    for (int g = 0; g < RED_PARTS; ++g) {
        const int k = m * RED_PARTS + g;
        A += part_d[2 * k];
        V += part_d[2 * k + 1];
        P += part_i[2 * k];
        IE += part_i[2 * k + 1];
    }
    const double h = B.grid[m].h;
    out2[2 * m] = A;
    out2[2 * m + 1] = h * h * (V + h * (double)IE) / 3.0;
    counts[2 * m] = P;
    counts[2 * m + 1] = IE;
}

static int grid_tiles(long long n)
{
    long long g = n < 1 ? 1 : n;
    return (int)(g > 2147483647LL ? 2147483647LL : g);
}

int launch_edge_count(const Batch &B, const int8_t *labels, int *tile_edges, int *tile_inside, cudaStream_t st)
{
    k_edge_count<<<grid_tiles((B.n_tiles + COUNT_WARPS - 1) / COUNT_WARPS), COUNT_WARPS * 32, 0, st>>>(
        B, labels, tile_edges, tile_inside);
    return 1;
}

int launch_mol_edges(const Batch &B, const int *edge_start, long long *medge, cudaStream_t st)
{
    const int n = 3 * (B.n_mol + 1);
    k_mol_edges<<<(n + 255) / 256, 256, 0, st>>>(B, edge_start, medge);
    return 1;
}

template <class T>
static size_t stage_smem()
{
    return edge_tile_bytes<T, CapMid>() + sizeof(StageSmem);
}

static int g_edge_n_sm = 1;  // SMs: the grid of the global-memory tier and of the persistent root kernels
// resident blocks per SM: [FP64, FP32][sphere roots, torus roots][64, 128, 256 threads]; hard selection
static int g_occ_roots[2][2][3];
static int g_occ_hard[2];
static int g_occ_exact[2];

static int threads_slot(int threads) { return threads <= 64 ? 0 : (threads <= 128 ? 1 : 2); }

// dynamic shared memory limits and occupancies (once per device, before any launch or capture)
void edges_init()
{
    cudaFuncSetAttribute(k_edge_stage<double, false, CapMid, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)stage_smem<double>());
    cudaFuncSetAttribute(k_edge_stage<float, true, CapMid, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)stage_smem<float>());
    cudaFuncSetAttribute(k_edge_stage<double, false, CapBig, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(StageSmem));
    cudaFuncSetAttribute(k_edge_stage<float, true, CapBig, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(StageSmem));
    int dev = 0, n_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    g_edge_n_sm = n_sm > 0 ? n_sm : 1;
    const int tb[3] = {64, 128, 256};
    for (int k = 0; k < 3; ++k) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_occ_roots[0][0][k], k_roots_sphere<double, false>, tb[k], 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_occ_roots[0][1][k], k_roots_torus<double, false>, tb[k], 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_occ_roots[1][0][k], k_roots_sphere<float, true>, tb[k], 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_occ_roots[1][1][k], k_roots_torus<float, true>, tb[k], 0);
    }
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_occ_exact[1], k_roots_torus_exact<float, true>, 256, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_occ_hard[0], k_edge_hard<double, false>, HARD_THREADS, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_occ_hard[1], k_edge_hard<float, true>, HARD_THREADS, 0);
}

// bytes of global scratch the staging pass's global-memory tier needs
size_t edges_big_bytes()
{
    size_t per = edge_tile_bytes<double, CapBig>();
    if (edge_tile_bytes<float, CapBig>() > per) per = edge_tile_bytes<float, CapBig>();
    return per * (size_t)g_edge_n_sm;
}

int edge_ctas_per_sm(int precision)
{
    int n = 0;
    if (precision == 0)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_edge_stage<double, false, CapMid, false>, EDGE_THREADS,
                                                      stage_smem<double>());
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_edge_stage<float, true, CapMid, false>, EDGE_THREADS,
                                                      stage_smem<float>());
    return n > 0 ? n : 1;
}

bool root_threads_valid(int threads) { return threads == 0 || threads == 64 || threads == 128 || threads == 256; }

long long slab_bytes_max(int precision)
{
    return precision == 0 ? SlabLayout<double>(CapBig::A, CapBig::P, CapBig::V).bytes
                          : SlabLayout<float>(CapBig::A, CapBig::P, CapBig::V).bytes;
}

template <class T, bool FILT>
static void stage_launch(const Model &M, const Batch &B, const TileSched &Q, int grid, const int8_t *labels,
                         const int *edge_start, EdgeOut out, int *err, int *ovf, unsigned char *big,
                         const RootWork &W, cudaStream_t st)
{
    cudaMemsetAsync(W.ctr, 0, 8 * sizeof(unsigned long long), st);
    if (Q.head) cudaMemsetAsync(Q.head, 0, sizeof(unsigned long long), st);
    cudaMemsetAsync(ovf + 1, 0, sizeof(int), st);
    k_edge_stage<T, FILT, CapMid, false><<<grid, EDGE_THREADS, stage_smem<T>(), st>>>(M, B, Q, labels, edge_start,
                                                                                       out, err, ovf, nullptr, W);
    TileSched QB{nullptr, 1, ovf + 2, ovf + 1};
    k_edge_stage<T, FILT, CapBig, true><<<g_edge_n_sm, EDGE_THREADS, sizeof(StageSmem), st>>>(
        M, B, QB, labels, edge_start, out, err, ovf, big, W);
}

template <class T, bool FILT>
static void roots_launch(const Model &M, const Batch &B, int threads, EdgeOut out, const int *edge_start,
                         long long ne_all, int *n_fail, int *err, long long *fail_log, const RootWork &W,
                         cudaStream_t st)
{
    const int P = FILT ? 1 : 0, ts = threads_slot(threads), tb = 64 << ts;
    const int gs = std::max(g_occ_roots[P][0][ts], 1) * g_edge_n_sm;
    const int gq = std::max(g_occ_roots[P][1][ts], 1) * g_edge_n_sm;
    k_roots_sphere<T, FILT><<<gs, tb, 0, st>>>(M, B, W, err);
    cudaMemsetAsync(W.ctr + 3, 0, 2 * sizeof(unsigned long long), st);  // hard edges, FP64 jobs
    k_roots_torus<T, FILT><<<gq, tb, 0, st>>>(M, B, W, err);
    if (FILT)
        k_roots_torus_exact<T, FILT><<<std::max(g_occ_exact[P], 1) * g_edge_n_sm, tb, 0, st>>>(M, B, W, err);
    const long long pb = std::min<long long>(std::max<long long>(ceil_div_ll(ne_all, PICK_THREADS), 1),
                                             8LL * g_edge_n_sm);
    k_edge_pick<T><<<(unsigned)pb, PICK_THREADS, 0, st>>>(B, W, edge_start, ne_all, out, err);
    k_edge_hard<T, FILT><<<std::max(g_occ_hard[P], 1) * g_edge_n_sm, HARD_THREADS, 0, st>>>(
        M, B, W, edge_start, out, n_fail, err, fail_log);
}

int launch_edge_stage(const Model &M, const Batch &B, int precision, const TileSched &Q, int grid,
                      const int8_t *labels, const int *edge_start, EdgeOut out, int *err, int *ovf,
                      unsigned char *big, const RootWork &W, cudaStream_t st)
{
    if (grid < 1) grid = 1;
    if (precision == 0)
        stage_launch<double, false>(M, B, Q, grid, labels, edge_start, out, err, ovf, big, W, st);
    else
        stage_launch<float, true>(M, B, Q, grid, labels, edge_start, out, err, ovf, big, W, st);
    return 2;
}

int launch_edge_roots(const Model &M, const Batch &B, int precision, int threads, EdgeOut out,
                      const int *edge_start, long long ne_all, int *n_fail, int *err, long long *fail_log,
                      const RootWork &W, cudaStream_t st)
{
    if (!root_threads_valid(threads) || threads == 0) threads = ROOT_THREADS_MAX;
    if (precision == 0)
        roots_launch<double, false>(M, B, threads, out, edge_start, ne_all, n_fail, err, fail_log, W, st);
    else
        roots_launch<float, true>(M, B, threads, out, edge_start, ne_all, n_fail, err, fail_log, W, st);
    return precision == 0 ? 4 : 5;
}

long long polish_blocks(long long n_edges) { return n_edges > 0 ? ceil_div_ll(n_edges, POLISH_THREADS) : 0; }

int launch_edge_polish(const Model &M, const Batch &B, EdgeOut out, long long n_edges_total,
                       const long long *medge, double2 *term, cudaStream_t st)
{
    long long nb = polish_blocks(n_edges_total);
    if (nb > 0) k_edge_polish<<<(unsigned)nb, POLISH_THREADS, 0, st>>>(M, B, out, medge, term);
    return nb > 0 ? 1 : 0;
}

long long reduce_scratch(int n_mol) { return 2LL * RED_PARTS * n_mol; }

int launch_reduce(const Batch &B, const double2 *term, const long long *medge, const int *tile_inside, double *part_d,
                  long long *part_i, double *out2, long long *counts, cudaStream_t st)
{
    k_reduce_part<<<B.n_mol * RED_PARTS, RED_THREADS, 0, st>>>(B, term, medge, tile_inside, part_d, part_i);
    k_reduce_final<<<(B.n_mol + 127) / 128, 128, 0, st>>>(B, part_d, part_i, out2, counts);
    return 2;
}

}  // namespace eses
