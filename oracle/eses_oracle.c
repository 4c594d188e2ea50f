/*
 * eses_oracle.c -- plain, slow FP64 CPU oracle for the Eulerian solvent
 * excluded surface (ESES).  TEST INFRASTRUCTURE ONLY: it is built and called by
 * the tests, by the package's smoke check and by the benchmark's CPU-baseline
 * leg.  The GPU library never links or calls it, and it shares no code with it.
 *
 * What it computes (the definitions, written out):
 *
 *   Atoms A = {(c_i, r_i)} (Eq. 1).  Probe radius r_p.  Expanded radii
 *   R_i = r_i + r_p.  Free probe centres
 *        Omega_free = { p : |p - c_i| >= R_i  for every i }.
 *   The SES is the boundary of the union of all probe balls of radius r_p
 *   centred in Omega_free (§1); the enclosed volume is
 *        M = { x : dist(x, Omega_free) >= r_p }.
 *   Inside[i,j,k] = 1 iff grid point (i,j,k) lies in M (Eq. 2).
 *   For every grid edge whose two end labels differ, the intersection with the
 *   SES is the first root, from the lower-index end point s, of
 *        g(tau) = dist(s + tau*h*e_a, Omega_free) - r_p ,  tau in [0,1]
 *   (Eq. 3-4; lambda of Eq. 4 equals 1 - tau).
 *
 * dist(x, Omega_free) is evaluated exactly as a minimum over candidate free
 * points.  The nearest free point q* of a point x outside Omega_free lies on
 * the boundary of Omega_free, which is made of pieces of expanded spheres
 * (faces), arcs of pair-intersection circles and triple points (vertices) --
 * the convex, saddle and concave patches of §1.  Hence q* is one of
 *   F  (convex):  for a ball i containing x, the radial projection of x onto
 *                 sphere (c_i, R_i), at distance R_i - |x - c_i|;
 *   E  (saddle):  for a pair (i,j) of intersecting expanded spheres, the point
 *                 of their intersection circle nearest to x;
 *   V  (concave): a point lying on three expanded spheres;
 * and a candidate counts only if it is itself free.  The minimum over the
 * free candidates is therefore dist(x, Omega_free): every candidate is a free
 * point (so the minimum cannot undershoot) and q* is among them.
 *
 * Two facts shorten the label test and are proved from the definition:
 *   - x inside a van der Waals ball (|x - c_i| < r_i): every free p has
 *     |p - x| >= |p - c_i| - |x - c_i| > R_i - r_i = r_p, so x is in M;
 *   - x in Omega_free: dist = 0, x is not in M.
 *
 * Intersections: g is 1-Lipschitz in arc length, so sphere tracing from s
 * (step |g|/h in tau) never passes a root and converges to the first one.
 *
 * Block decomposition follows Algorithm 1 and §2.3-2.5: blocks of B points
 * per edge (B-1 cells, shared face), each block gathers its relevant atoms,
 * builds its own patch model, classifies its points, computes the
 * intersections on its edges, and keeps only the points and edges it owns
 * (the half-open rule of §2.5).  The last block along an axis also owns the
 * domain's + face, so the output covers the whole grid.
 *
 * Readings where the paper is silent (grid origin and extent, ties, first
 * root, area and volume estimators) are stated beside the code that takes
 * them.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no fused
 * multiply-add, so the arithmetic is the plain IEEE sequence written here).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define EO_TYPE_NONE (-1)
#define EO_TYPE_F 0
#define EO_TYPE_E 1
#define EO_TYPE_V 2
#define EO_TYPE_FREE 3 /* the point itself is free */

/* ------------------------------------------------------------------------ */
/* small vector helpers                                                      */
/* ------------------------------------------------------------------------ */
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double dist2(const double *a, const double *b)
{
    double d0 = a[0] - b[0], d1 = a[1] - b[1], d2 = a[2] - b[2];
    return d0 * d0 + d1 * d1 + d2 * d2;
}
static void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* growable arrays */
typedef struct { double *v; int64_t n, cap; } dvec;
typedef struct { int64_t *v; int64_t n, cap; } ivec;
static void dpush(dvec *a, double x)
{
    if (a->n == a->cap) { a->cap = a->cap ? 2 * a->cap : 64; a->v = (double *)realloc(a->v, (size_t)a->cap * sizeof(double)); }
    a->v[a->n++] = x;
}
static void ipush(ivec *a, int64_t x)
{
    if (a->n == a->cap) { a->cap = a->cap ? 2 * a->cap : 64; a->v = (int64_t *)realloc(a->v, (size_t)a->cap * sizeof(int64_t)); }
    a->v[a->n++] = x;
}

/* ------------------------------------------------------------------------ */
/* grid (Eq. 2 with the origin and extent readings)                          */
/* ------------------------------------------------------------------------ */
/* Grid point (i,j,k) sits at lo + h*(i,j,k).  lo_a = min_i(c_ia - r_i) - margin
 * and n_a = ceil((max_i(c_ia + r_i) + margin - lo_a)/h) + 1: the tight van der
 * Waals box padded by the margin (§2.3), so the + faces lie at least `margin`
 * beyond every atom and hold no inside point (§2.5). */
int eo_grid(const double *xyz, const double *r, int64_t n, double h, double margin, int64_t dims[3], double lo[3])
{
    if (n < 1 || !(h > 0.0) || !(margin >= h)) return -1;
    for (int a = 0; a < 3; ++a) {
        double mn = xyz[a] - r[0], mx = xyz[a] + r[0];
        for (int64_t i = 1; i < n; ++i) {
            double v0 = xyz[3 * i + a] - r[i], v1 = xyz[3 * i + a] + r[i];
            if (v0 < mn) mn = v0;
            if (v1 > mx) mx = v1;
        }
        lo[a] = mn - margin;
        dims[a] = (int64_t)ceil((mx + margin - lo[a]) / h) + 1;
    }
    return 0;
}

/* Number of blocks along an axis of n points when a block has B points per
 * edge and neighbouring blocks share a face (B-1 cells per block). */
int64_t eo_block_count(int64_t n, int64_t B)
{
    int64_t cells = B - 1;
    if (n <= 1) return 1;
    return (n - 1 + cells - 1) / cells;
}

/* ------------------------------------------------------------------------ */
/* patch model of a set of atoms                                             */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n;
    double *c;      /* 3n centres */
    double *r;      /* n vdW radii */
    double *R;      /* n expanded radii */
    int64_t *gid;   /* n global atom ids (tie order) */
    double rp, Rmax;
    /* pairs with an intersection circle: centre o, unit axis u (c_i -> c_j),
     * radius rho, one unit vector v1 normal to u */
    int np;
    int *pi, *pj;
    double *po, *pu, *prho, *pv1;
    /* free triple points */
    int nv;
    int *vi, *vj, *vk;
    double *vq;
    /* uniform cell grid (cell edge >= Rmax + cap) */
    int brute;
    double cell, clo[3];
    int cn[3];
    int *a_start, *a_list, *p_start, *p_list, *v_start, *v_list;
} Model;

static void model_free(Model *m)
{
    free(m->c); free(m->r); free(m->R); free(m->gid);
    free(m->pi); free(m->pj); free(m->po); free(m->pu); free(m->prho); free(m->pv1);
    free(m->vi); free(m->vj); free(m->vk); free(m->vq);
    free(m->a_start); free(m->a_list); free(m->p_start); free(m->p_list); free(m->v_start); free(m->v_list);
    memset(m, 0, sizeof(*m));
}

static int cell_of(const Model *m, const double *x, int *ci)
{
    for (int a = 0; a < 3; ++a) {
        int k = (int)floor((x[a] - m->clo[a]) / m->cell);
        if (k < 0) k = 0;
        if (k >= m->cn[a]) k = m->cn[a] - 1;
        ci[a] = k;
    }
    return (ci[0] * m->cn[1] + ci[1]) * m->cn[2] + ci[2];
}

/* counting-sort items (positions pos[3*k]) into the cell grid */
static void bin_items(const Model *m, const double *pos, int cnt, int **start_out, int **list_out)
{
    int ncell = m->cn[0] * m->cn[1] * m->cn[2];
    int *start = (int *)calloc((size_t)ncell + 1, sizeof(int));
    int *list = (int *)malloc(sizeof(int) * (size_t)(cnt > 0 ? cnt : 1));
    int *cid = (int *)malloc(sizeof(int) * (size_t)(cnt > 0 ? cnt : 1));
    int ci[3];
    for (int k = 0; k < cnt; ++k) { cid[k] = cell_of(m, pos + 3 * k, ci); start[cid[k] + 1]++; }
    for (int c = 0; c < ncell; ++c) start[c + 1] += start[c];
    int *fill = (int *)malloc(sizeof(int) * (size_t)ncell);
    memcpy(fill, start, sizeof(int) * (size_t)ncell);
    for (int k = 0; k < cnt; ++k) list[fill[cid[k]]++] = k;   /* ascending k within a cell */
    free(fill); free(cid);
    *start_out = start; *list_out = list;
}

/* Iterate the items of the 27 cells around x (or all items in brute mode). */
#define FOR_NEAR(m, x, start, list, cnt, k, ...)                                        \
    do {                                                                                 \
        if ((m)->brute) {                                                                \
            for (int k = 0; k < (cnt); ++k) { __VA_ARGS__ }                                     \
        } else {                                                                         \
            int ci_[3];                                                                  \
            cell_of((m), (x), ci_);                                                      \
            for (int dx_ = -1; dx_ <= 1; ++dx_)                                          \
                for (int dy_ = -1; dy_ <= 1; ++dy_)                                      \
                    for (int dz_ = -1; dz_ <= 1; ++dz_) {                                \
                        int a_ = ci_[0] + dx_, b_ = ci_[1] + dy_, c_ = ci_[2] + dz_;     \
                        if (a_ < 0 || b_ < 0 || c_ < 0 || a_ >= (m)->cn[0] ||            \
                            b_ >= (m)->cn[1] || c_ >= (m)->cn[2]) continue;              \
                        int cc_ = (a_ * (m)->cn[1] + b_) * (m)->cn[2] + c_;              \
                        for (int t_ = (start)[cc_]; t_ < (start)[cc_ + 1]; ++t_) {       \
                            int k = (list)[t_];                                          \
                            __VA_ARGS__                                                  \
                        }                                                                \
                    }                                                                    \
        }                                                                                \
    } while (0)

/* q is free iff |q - c_k| >= R_k for every atom k other than the excluded
 * generating atoms (which carry q on their own sphere by construction). */
static int is_free(const Model *m, const double *q, int e0, int e1, int e2)
{
    int ok = 1;
    FOR_NEAR(m, q, m->a_start, m->a_list, m->n, k, {
        if (ok && k != e0 && k != e1 && k != e2) {
            if (dist2(q, m->c + 3 * k) < m->R[k] * m->R[k]) ok = 0;
        }
    });
    return ok;
}

/* Build the patch model of the given atoms: all pairs with an intersection
 * circle (saddle patches) and all free triple points (concave patches).  The
 * probe-clash test of a triple point is the freeness test above. */
/* Coincident atoms (the same centre and radius) are one ball: the union of
 * balls, hence Omega_free and M (§1), does not change when one is dropped,
 * and keeping both would make each one's sphere "cover" the other's surface
 * points in floating point.  keep[i] = 0 for every repeat of an earlier atom. */
typedef struct { double x, y, z, r; int i; } AtomKey;
static int cmp_atomkey(const void *a, const void *b)
{
    const AtomKey *p = (const AtomKey *)a, *q = (const AtomKey *)b;
    if (p->x != q->x) return p->x < q->x ? -1 : 1;
    if (p->y != q->y) return p->y < q->y ? -1 : 1;
    if (p->z != q->z) return p->z < q->z ? -1 : 1;
    if (p->r != q->r) return p->r < q->r ? -1 : 1;
    return (p->i > q->i) - (p->i < q->i);
}
static int unique_atoms(const double *xyz, const double *r, int n, char *keep)
{
    AtomKey *k = (AtomKey *)malloc(sizeof(AtomKey) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        k[i].x = xyz[3 * i]; k[i].y = xyz[3 * i + 1]; k[i].z = xyz[3 * i + 2]; k[i].r = r[i]; k[i].i = i;
        keep[i] = 1;
    }
    qsort(k, (size_t)n, sizeof(AtomKey), cmp_atomkey);
    int kept = n;
    for (int t = 1; t < n; ++t)
        if (k[t].x == k[t - 1].x && k[t].y == k[t - 1].y && k[t].z == k[t - 1].z && k[t].r == k[t - 1].r) {
            keep[k[t].i] = 0;
            --kept;
        }
    free(k);
    return kept;
}

static void model_build(Model *m, const double *xyz_in, const double *r_in, const int64_t *gid_in, int n_in,
                        double rp, double cap, int brute)
{
    char *keep = (char *)malloc((size_t)(n_in > 0 ? n_in : 1));
    const int n = unique_atoms(xyz_in, r_in, n_in, keep);
    double *xyz = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *r = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int64_t *gid = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int i = 0, k = 0; i < n_in; ++i) {
        if (!keep[i]) continue;
        for (int a = 0; a < 3; ++a) xyz[3 * k + a] = xyz_in[3 * i + a];
        r[k] = r_in[i];
        gid[k] = gid_in ? gid_in[i] : i;
        ++k;
    }
    free(keep);
    memset(m, 0, sizeof(*m));
    m->n = n; m->rp = rp; m->brute = brute;
    m->c = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    m->r = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    m->R = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    m->gid = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    m->Rmax = 0.0;
    double bmin[3] = {1e300, 1e300, 1e300}, bmax[3] = {-1e300, -1e300, -1e300};
    for (int i = 0; i < n; ++i) {
        for (int a = 0; a < 3; ++a) {
            m->c[3 * i + a] = xyz[3 * i + a];
            if (xyz[3 * i + a] < bmin[a]) bmin[a] = xyz[3 * i + a];
            if (xyz[3 * i + a] > bmax[a]) bmax[a] = xyz[3 * i + a];
        }
        m->r[i] = r[i];
        m->R[i] = r[i] + rp;
        m->gid[i] = gid ? gid[i] : i;
        if (m->R[i] > m->Rmax) m->Rmax = m->R[i];
    }
    if (n == 0) { bmin[0] = bmin[1] = bmin[2] = 0.0; bmax[0] = bmax[1] = bmax[2] = 0.0; }
    /* cell edge covers every query radius used below: F candidates (R_max),
     * E candidates (rho + cap <= R_max + cap), V (cap), freeness (R_max);
     * pair search needs R_i + R_j <= 2 R_max, done by brute force over cells
     * within two cells when cap < R_max (handled by a wider loop below). */
    m->cell = m->Rmax + cap;
    if (m->cell < 1e-3) m->cell = 1e-3;
    long long total = 1;
    for (int a = 0; a < 3; ++a) {
        m->clo[a] = bmin[a] - m->cell;
        m->cn[a] = (int)floor((bmax[a] + m->cell - m->clo[a]) / m->cell) + 1;
        total *= m->cn[a];
    }
    if (total > 50000000LL) m->brute = 1; /* pathological extent: fall back to brute force */
    if (m->brute) { m->cn[0] = m->cn[1] = m->cn[2] = 1; m->cell = 1e300; }
    bin_items(m, m->c, n, &m->a_start, &m->a_list);

    /* neighbour lists: j with |c_i - c_j| < R_i + R_j (every pair of
     * overlapping expanded balls, whether or not a circle exists) */
    int *nb_start = (int *)calloc((size_t)n + 1, sizeof(int));
    ivec NB = {0};
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            double Rs = m->R[i] + m->R[j];
            if (dist2(m->c + 3 * i, m->c + 3 * j) < Rs * Rs) ipush(&NB, j);
        }
        nb_start[i + 1] = (int)NB.n;
    }

    /* pairs: |c_i - c_j| < R_i + R_j and |c_i - c_j| > |R_i - R_j| */
    ivec PI = {0}, PJ = {0};
    dvec PO = {0}, PU = {0}, PR = {0}, PV = {0};
    for (int i = 0; i < n; ++i) {
        for (int t = nb_start[i]; t < nb_start[i + 1]; ++t) {
            int j = (int)NB.v[t];
            if (j <= i) continue;
            double D = sqrt(dist2(m->c + 3 * i, m->c + 3 * j));
            if (D <= fabs(m->R[i] - m->R[j])) continue; /* one ball inside the other: no circle */
            double u[3], o[3];
            for (int a = 0; a < 3; ++a) u[a] = (m->c[3 * j + a] - m->c[3 * i + a]) / D;
            double aa = (D * D + m->R[i] * m->R[i] - m->R[j] * m->R[j]) / (2.0 * D);
            double rho2 = m->R[i] * m->R[i] - aa * aa;
            if (!(rho2 > 0.0)) continue;
            for (int a = 0; a < 3; ++a) o[a] = m->c[3 * i + a] + aa * u[a];
            /* a unit vector normal to u */
            double t3[3] = {1.0, 0.0, 0.0};
            if (fabs(u[0]) > 0.6) { t3[0] = 0.0; t3[1] = 1.0; }
            double v1[3];
            cross3(u, t3, v1);
            double nv1 = sqrt(dot3(v1, v1));
            for (int a = 0; a < 3; ++a) v1[a] /= nv1;
            ipush(&PI, i); ipush(&PJ, j);
            for (int a = 0; a < 3; ++a) { dpush(&PO, o[a]); dpush(&PU, u[a]); dpush(&PV, v1[a]); }
            dpush(&PR, sqrt(rho2));
        }
    }
    m->np = (int)PI.n;
    m->pi = (int *)malloc(sizeof(int) * (size_t)(m->np > 0 ? m->np : 1));
    m->pj = (int *)malloc(sizeof(int) * (size_t)(m->np > 0 ? m->np : 1));
    for (int k = 0; k < m->np; ++k) { m->pi[k] = (int)PI.v[k]; m->pj[k] = (int)PJ.v[k]; }
    m->po = PO.v; m->pu = PU.v; m->prho = PR.v; m->pv1 = PV.v;
    free(PI.v); free(PJ.v);
    if (m->np == 0) { m->po = (double *)malloc(24); m->pu = (double *)malloc(24); m->prho = (double *)malloc(8); m->pv1 = (double *)malloc(24); }
    bin_items(m, m->po, m->np, &m->p_start, &m->p_list);

    /* triple points of every triple i < j < k of mutually overlapping
     * expanded spheres, by trilateration; kept iff free (probe-clash test) */
    ivec VI = {0}, VJ = {0}, VK = {0};
    dvec VQ = {0};
    for (int i = 0; i < n; ++i) {
        for (int t1 = nb_start[i]; t1 < nb_start[i + 1]; ++t1) {
            int j = (int)NB.v[t1];
            if (j <= i) continue;
            for (int t2 = nb_start[i]; t2 < nb_start[i + 1]; ++t2) {
                int k = (int)NB.v[t2];
                if (k <= j) continue;
                double Sjk = m->R[j] + m->R[k];
                if (dist2(m->c + 3 * j, m->c + 3 * k) >= Sjk * Sjk) continue;
                const double *c1 = m->c + 3 * i, *c2 = m->c + 3 * j, *c3 = m->c + 3 * k;
                double R1 = m->R[i], R2 = m->R[j], R3 = m->R[k];
                double ex[3], ey[3], ez[3], d21[3], d31[3];
                for (int a = 0; a < 3; ++a) { d21[a] = c2[a] - c1[a]; d31[a] = c3[a] - c1[a]; }
                double d = sqrt(dot3(d21, d21));
                for (int a = 0; a < 3; ++a) ex[a] = d21[a] / d;
                double ii = dot3(ex, d31);
                for (int a = 0; a < 3; ++a) ey[a] = d31[a] - ii * ex[a];
                double ny = sqrt(dot3(ey, ey));
                if (!(ny > 1e-12)) continue; /* collinear centres */
                for (int a = 0; a < 3; ++a) ey[a] /= ny;
                cross3(ex, ey, ez);
                double jj = dot3(ey, d31);
                double X = (R1 * R1 - R2 * R2 + d * d) / (2.0 * d);
                double Y = (R1 * R1 - R3 * R3 + ii * ii + jj * jj) / (2.0 * jj) - (ii / jj) * X;
                double Z2 = R1 * R1 - X * X - Y * Y;
                if (!(Z2 > 0.0)) continue; /* the three spheres share no point */
                double Z = sqrt(Z2);
                for (int s = -1; s <= 1; s += 2) {
                    double q[3];
                    for (int a = 0; a < 3; ++a) q[a] = c1[a] + X * ex[a] + Y * ey[a] + s * Z * ez[a];
                    if (!is_free(m, q, i, j, k)) continue;
                    ipush(&VI, i); ipush(&VJ, j); ipush(&VK, k);
                    for (int a = 0; a < 3; ++a) dpush(&VQ, q[a]);
                }
            }
        }
    }
    free(nb_start); free(NB.v);
    m->nv = (int)VI.n;
    m->vi = (int *)malloc(sizeof(int) * (size_t)(m->nv > 0 ? m->nv : 1));
    m->vj = (int *)malloc(sizeof(int) * (size_t)(m->nv > 0 ? m->nv : 1));
    m->vk = (int *)malloc(sizeof(int) * (size_t)(m->nv > 0 ? m->nv : 1));
    for (int k = 0; k < m->nv; ++k) { m->vi[k] = (int)VI.v[k]; m->vj[k] = (int)VJ.v[k]; m->vk[k] = (int)VK.v[k]; }
    m->vq = VQ.v;
    if (m->nv == 0) m->vq = (double *)malloc(24);
    free(VI.v); free(VJ.v); free(VK.v);
    bin_items(m, m->vq, m->nv, &m->v_start, &m->v_list);
    free(xyz); free(r); free(gid);
}

/* ------------------------------------------------------------------------ */
/* distance to Omega_free, capped                                            */
/* ------------------------------------------------------------------------ */
typedef struct {
    int type;         /* EO_TYPE_F/E/V or NONE (no free point closer than cap) */
    int64_t ids[3];   /* global ids of the generating atoms */
    int loc;          /* model index of the witness' patch: atom (F), pair (E), triple point (V) */
    double q[3];      /* the witness (nearest free point) */
    /* instrumentation for the flop model (counts of candidate work) */
    long n_reach;     /* atoms with |x - c| < r + 2 r_p */
    long n_face;      /* face candidates (balls containing x) */
    long n_face_tests;/* freeness tests of face candidates (atoms tested) */
    long n_arc;       /* saddle candidates within cap */
    long n_vert;      /* vertex candidates examined */
} Witness;

/* min(cap, dist(x, Omega_free)).  Candidates are examined in the order
 * F (atom order), E (pair order), V (triple order) with a strict "<", so the
 * first candidate wins a tie: the tie rule F < E < V, then atom order. */
static double dist_free(const Model *m, const double *x, double cap, Witness *w)
{
    double best = cap;
    if (w) { memset(w, 0, sizeof(*w)); w->type = EO_TYPE_NONE; }
    const double rp = m->rp;
    int in_some_ball = 0;
    /* F: radial projections onto spheres of balls that contain x */
    FOR_NEAR(m, x, m->a_start, m->a_list, m->n, i, {
        double dd2 = dist2(x, m->c + 3 * i);
        if (w) { double rr = m->r[i] + 2.0 * rp; if (dd2 < rr * rr) w->n_reach++; }
        if (dd2 < m->R[i] * m->R[i]) {
            in_some_ball = 1;
            double dx = sqrt(dd2);
            double dist = m->R[i] - dx;
            if (w) w->n_face++;
            if (dist < best) {
                double q[3], dir[3];
                if (dx > 0.0) {
                    for (int a = 0; a < 3; ++a) dir[a] = (x[a] - m->c[3 * i + a]) / dx;
                } else {
                    dir[0] = 1.0; dir[1] = 0.0; dir[2] = 0.0; /* x at the centre: any direction */
                }
                for (int a = 0; a < 3; ++a) q[a] = m->c[3 * i + a] + m->R[i] * dir[a];
                if (w) w->n_face_tests++;
                if (is_free(m, q, i, -1, -1)) {
                    best = dist;
                    if (w) { w->type = EO_TYPE_F; w->loc = i; w->ids[0] = m->gid[i]; w->ids[1] = w->ids[2] = -1; memcpy(w->q, q, sizeof q); }
                }
            }
        }
    });
    /* x in no expanded ball: x itself is free, dist = 0 */
    if (!in_some_ball) {
        if (w) { w->type = EO_TYPE_FREE; memcpy(w->q, x, 3 * sizeof(double)); w->ids[0] = w->ids[1] = w->ids[2] = -1; }
        return 0.0;
    }
    /* E: nearest point of each pair circle */
    FOR_NEAR(m, x, m->p_start, m->p_list, m->np, p, {
        const double *o = m->po + 3 * p, *u = m->pu + 3 * p;
        double y[3] = {x[0] - o[0], x[1] - o[1], x[2] - o[2]};
        double z = dot3(y, u);
        double wv[3] = {y[0] - z * u[0], y[1] - z * u[1], y[2] - z * u[2]};
        /* the nearest circle point lies along the part of y normal to the
         * axis; remove the rounding left along u, so that the direction is
         * normal to u even when x is (numerically) on the axis */
        double zr = dot3(wv, u);
        for (int a = 0; a < 3; ++a) wv[a] -= zr * u[a];
        double nw = sqrt(dot3(wv, wv));
        double q[3];
        if (nw > 1e-12 * (1.0 + sqrt(dot3(y, y)))) {
            for (int a = 0; a < 3; ++a) q[a] = o[a] + m->prho[p] * wv[a] / nw;
        } else {
            for (int a = 0; a < 3; ++a) q[a] = o[a] + m->prho[p] * m->pv1[3 * p + a]; /* x on the axis */
        }
        double dist = sqrt(dist2(x, q));
        if (dist < cap && w) w->n_arc++;
        if (dist < best && is_free(m, q, m->pi[p], m->pj[p], -1)) {
            best = dist;
            if (w) { w->type = EO_TYPE_E; w->loc = p; w->ids[0] = m->gid[m->pi[p]]; w->ids[1] = m->gid[m->pj[p]]; w->ids[2] = -1; memcpy(w->q, q, sizeof q); }
        }
    });
    /* V: free triple points */
    FOR_NEAR(m, x, m->v_start, m->v_list, m->nv, v, {
        double dist = sqrt(dist2(x, m->vq + 3 * v));
        if (w && dist < cap) w->n_vert++;
        if (dist < best) {
            best = dist;
            if (w) { w->type = EO_TYPE_V; w->loc = v; w->ids[0] = m->gid[m->vi[v]]; w->ids[1] = m->gid[m->vj[v]]; w->ids[2] = m->gid[m->vk[v]]; memcpy(w->q, m->vq + 3 * v, 3 * sizeof(double)); }
        }
    });
    return best;
}

/* Eq. 2: 1 iff x in M, i.e. dist(x, Omega_free) >= r_p.  Ties (dist == r_p)
 * count as inside: M is closed. */
static int label_of(const Model *m, const double *x, Witness *w, int *near_tie)
{
    int in_sas = 0;
    if (w) { memset(w, 0, sizeof(*w)); w->type = EO_TYPE_NONE; }
    int inside_vdw = 0;
    FOR_NEAR(m, x, m->a_start, m->a_list, m->n, i, {
        double dd2 = dist2(x, m->c + 3 * i);
        if (dd2 < m->r[i] * m->r[i]) inside_vdw = 1;
        if (dd2 < m->R[i] * m->R[i]) in_sas = 1;
    });
    if (inside_vdw) return 1;
    if (!in_sas) return 0;
    double d = dist_free(m, x, m->rp, w);
    if (near_tie && fabs(d - m->rp) < 1e-10 && d < m->rp) *near_tie += 1;
    return d >= m->rp ? 1 : 0;
}

/* ------------------------------------------------------------------------ */
/* public point queries (for tests)                                          */
/* ------------------------------------------------------------------------ */
int eo_distance_points(const double *xyz, const double *r, int64_t n, double rp, const double *pts, int64_t m_pts,
                       double cap, int brute, double *d_out, double *q_out, int32_t *type_out, int64_t *ids_out,
                       int64_t *counts_out)
{
    Model m;
    model_build(&m, xyz, r, NULL, (int)n, rp, cap, brute);
    for (int64_t k = 0; k < m_pts; ++k) {
        Witness w;
        d_out[k] = dist_free(&m, pts + 3 * k, cap, &w);
        if (q_out) memcpy(q_out + 3 * k, w.q, 3 * sizeof(double));
        if (type_out) type_out[k] = w.type;
        if (ids_out) { ids_out[3 * k] = w.ids[0]; ids_out[3 * k + 1] = w.ids[1]; ids_out[3 * k + 2] = w.ids[2]; }
        if (counts_out) {
            counts_out[5 * k + 0] = w.n_reach; counts_out[5 * k + 1] = w.n_face; counts_out[5 * k + 2] = w.n_face_tests;
            counts_out[5 * k + 3] = w.n_arc; counts_out[5 * k + 4] = w.n_vert;
        }
    }
    model_free(&m);
    return 0;
}

int eo_label_points(const double *xyz, const double *r, int64_t n, double rp, const double *pts, int64_t m_pts,
                    int brute, int8_t *out)
{
    Model m;
    model_build(&m, xyz, r, NULL, (int)n, rp, rp, brute);
    for (int64_t k = 0; k < m_pts; ++k) out[k] = (int8_t)label_of(&m, pts + 3 * k, NULL, NULL);
    model_free(&m);
    return 0;
}

/* model statistics: number of circle pairs and free triple points */
int eo_model_stats(const double *xyz, const double *r, int64_t n, double rp, int64_t *n_pairs, int64_t *n_free_vertices,
                   double *vertices_out, int64_t cap_vertices, int64_t *pairs_out, int64_t cap_pairs)
{
    Model m;
    model_build(&m, xyz, r, NULL, (int)n, rp, rp, 0);
    *n_pairs = m.np;
    *n_free_vertices = m.nv;
    if (vertices_out) {
        for (int v = 0; v < m.nv && v < cap_vertices; ++v) memcpy(vertices_out + 3 * v, m.vq + 3 * v, 3 * sizeof(double));
    }
    if (pairs_out) {
        for (int p = 0; p < m.np && p < cap_pairs; ++p) { pairs_out[2 * p] = m.pi[p]; pairs_out[2 * p + 1] = m.pj[p]; }
    }
    model_free(&m);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* full run (Algorithm 1)                                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t dims[3];
    double lo[3], h, rp;
    int8_t *labels;
    /* sparse runs: labels hold only the listed blocks' owned points, block
     * after block, C order within a block */
    int sparse;
    int64_t nblk;
    int64_t *blk_lo, *blk_hi, *blk_off;
    ivec idx[3];
    dvec tau[3], nrm[3];
    ivec ptype[3];
    ivec wid[3];               /* 3 per edge: the witness' generating atoms (-1 unused) */
    double area, volume_lines, volume_count;
    int64_t near_ties, slow_edges;
    /* instrumentation sums over the owned points / edges */
    int64_t sum_reach, sum_face, sum_face_tests, sum_arc, sum_vert, n_shell, n_points_done;
} eo_result;

/* Root of the witness' patch next to tau (in [0, 1] units of h): the van der
 * Waals sphere |y - c_i| = r_i (F: dist = R_i - |y - c_i|), the probe sphere
 * |y - q_v| = r_p (V), or the torus (|w| - rho)^2 + z^2 = r_p^2 (E, Newton
 * from tau).  A grazing sphere (discriminant <= 0) touches at its vertex. */
static double refine_on_patch(const Model *m, const double *s, int axis, double h, double tau, const Witness *w)
{
    if (w->type == EO_TYPE_F || w->type == EO_TYPE_V) {
        const double *c = w->type == EO_TYPE_F ? m->c + 3 * w->loc : m->vq + 3 * w->loc;
        const double rad = w->type == EO_TYPE_F ? m->r[w->loc] : m->rp;
        double d[3] = {s[0] - c[0], s[1] - c[1], s[2] - c[2]};
        double b = d[axis];
        double disc = b * b - (dot3(d, d) - rad * rad);
        double t0 = tau * h;
        if (disc <= 0.0) return -b / h;
        double sq = sqrt(disc);
        double r1 = -b - sq, r2 = -b + sq;
        return (fabs(r1 - t0) <= fabs(r2 - t0) ? r1 : r2) / h;
    }
    /* E: Newton on f(t) = (|w| - rho)^2 + z^2 - r_p^2 along the edge */
    const double *o = m->po + 3 * w->loc, *u = m->pu + 3 * w->loc;
    const double rho = m->prho[w->loc], rp = m->rp;
    double t = tau * h;
    for (int it = 0; it < 100; ++it) {
        double y[3] = {s[0] - o[0], s[1] - o[1], s[2] - o[2]};
        y[axis] += t;
        double z = dot3(y, u);
        double wv[3] = {y[0] - z * u[0], y[1] - z * u[1], y[2] - z * u[2]};
        double nw = sqrt(dot3(wv, wv));
        if (!(nw > 0.0)) break;
        double f = (nw - rho) * (nw - rho) + z * z - rp * rp;
        double df = 2.0 * (nw - rho) * wv[axis] / nw + 2.0 * z * u[axis];
        if (df == 0.0) break;
        double step = f / df;
        t -= step;
        if (fabs(step) <= 1e-16 * (1.0 + fabs(t))) break;
    }
    return t / h;
}

/* Sphere tracing of g(tau) = min(cap, dist(s + tau h e_a)) - r_p from tau = 0
 * (the lower-index end point): step |g|/h never passes a root of the
 * 1-Lipschitz g, so the sequence converges to the first root (Eq. 3-4 with
 * the first-root reading for edges that hold several roots). */
static double first_root(const Model *m, const double *s, int axis, double h, double cap, Witness *w, int *slow)
{
    double tau = 0.0, y[3];
    const double tol = 1e-11; /* Angstrom; g at the reported root */
    int it;
    for (it = 0; it < 2000000; ++it) {
        y[0] = s[0]; y[1] = s[1]; y[2] = s[2];
        y[axis] = s[axis] + tau * h;
        double g = dist_free(m, y, cap, w) - m->rp;
        double ag = fabs(g);
        if (ag <= tol) break;
        tau += ag / h;
        if (tau >= 1.0) { tau = 1.0; break; }
    }
    if (it >= 2000000 && slow) *slow += 1;
    /* witness at the final point */
    y[0] = s[0]; y[1] = s[1]; y[2] = s[2];
    y[axis] = s[axis] + tau * h;
    double g0 = fabs(dist_free(m, y, cap, w) - m->rp);
    /* |g| <= tol bounds the root's position only by tol / |g'|, which is
     * large where the edge grazes the surface: finish on the equation of the
     * witness' own patch (the surface there), solved next to tau */
    if (w && w->type != EO_TYPE_NONE && w->type != EO_TYPE_FREE) {
        double t = refine_on_patch(m, s, axis, h, tau, w);
        if (t >= tau - 1e-7 && t <= 1.0 && fabs(t - tau) <= 1e-3) {
            Witness w2;
            double y2[3] = {s[0], s[1], s[2]};
            y2[axis] = s[axis] + t * h;
            double g2 = fabs(dist_free(m, y2, cap, &w2) - m->rp);
            if (g2 <= (g0 > 1e-12 ? g0 : 1e-12)) { tau = t; *w = w2; }
        }
    }
    return tau;
}

typedef struct {
    int64_t b[3];              /* block coordinates */
    int64_t own_lo[3], own_hi[3];   /* owned points [lo, hi) */
    int64_t cmp_hi[3];         /* computed points [own_lo, cmp_hi) */
    ivec idx[3];
    dvec tau[3], nrm[3];
    ivec ptype[3];
    ivec wid[3];               /* 3 per edge: the witness' generating atoms (-1 unused) */
    double area, vol_lines, vol_count;
    int64_t near_ties, slow;
    int64_t sum_reach, sum_face, sum_face_tests, sum_arc, sum_vert, n_shell, n_points;
} BlockOut;

static void run_block(const double *xyz, const double *r, const int64_t *gid, int64_t n, double rp, double h,
                      const int64_t *dims, const double *lo, BlockOut *bo, int8_t *labels, int8_t *own_out, int brute,
                      int instrument)
{
    const double cap = rp + 2.0 * h; /* enough for the sphere tracing of a crossing edge */
    /* block box in space (computed points) */
    double bmin[3], bmax[3];
    for (int a = 0; a < 3; ++a) {
        bmin[a] = lo[a] + h * (double)bo->own_lo[a];
        bmax[a] = lo[a] + h * (double)(bo->cmp_hi[a] - 1);
    }
    /* AssembleRelevantAtoms: atoms whose expanded sphere + cap reaches the box */
    int64_t cnt = 0;
    int64_t *sel = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) {
        double e2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            double v = xyz[3 * i + a], e = 0.0;
            if (v < bmin[a]) e = bmin[a] - v;
            else if (v > bmax[a]) e = v - bmax[a];
            e2 += e * e;
        }
        double reach = r[i] + rp + cap + 1e-9;
        if (e2 < reach * reach) sel[cnt++] = i;
    }
    double *bx = (double *)malloc(sizeof(double) * 3 * (size_t)(cnt > 0 ? cnt : 1));
    double *br = (double *)malloc(sizeof(double) * (size_t)(cnt > 0 ? cnt : 1));
    for (int64_t k = 0; k < cnt; ++k) {
        for (int a = 0; a < 3; ++a) bx[3 * k + a] = xyz[3 * sel[k] + a];
        br[k] = r[sel[k]];
    }
    if (gid) /* the caller's atom ids (a subset of a larger input) */
        for (int64_t k = 0; k < cnt; ++k) sel[k] = gid[sel[k]];
    Model m;
    model_build(&m, bx, br, sel, (int)cnt, rp, cap, brute);

    /* classify the computed points (owned points plus the shared + face) */
    int64_t ex[3];
    for (int a = 0; a < 3; ++a) ex[a] = bo->cmp_hi[a] - bo->own_lo[a];
    int8_t *loc = (int8_t *)malloc((size_t)(ex[0] * ex[1] * ex[2]));
    for (int64_t i = 0; i < ex[0]; ++i)
        for (int64_t j = 0; j < ex[1]; ++j)
            for (int64_t k = 0; k < ex[2]; ++k) {
                int64_t g[3] = {bo->own_lo[0] + i, bo->own_lo[1] + j, bo->own_lo[2] + k};
                double x[3];
                for (int a = 0; a < 3; ++a) x[a] = lo[a] + h * (double)g[a];
                int nt = 0;
                int lab = label_of(&m, x, NULL, &nt);
                loc[(i * ex[1] + j) * ex[2] + k] = (int8_t)lab;
                int owned = g[0] < bo->own_hi[0] && g[1] < bo->own_hi[1] && g[2] < bo->own_hi[2];
                if (owned) {
                    bo->near_ties += nt;
                    if (own_out) /* sparse run: the block's own array */
                        own_out[((g[0] - bo->own_lo[0]) * (bo->own_hi[1] - bo->own_lo[1]) + (g[1] - bo->own_lo[1])) *
                                    (bo->own_hi[2] - bo->own_lo[2]) + (g[2] - bo->own_lo[2])] = (int8_t)lab;
                    else
                        labels[(g[0] * dims[1] + g[1]) * dims[2] + g[2]] = (int8_t)lab; /* LocalToGlobal, Eq. 5 */
                    bo->n_points++;
                    if (lab) bo->vol_count += 1.0;
                }
            }
    /* owned edges: from owned point p to p + e_a (RemoveDuplicates, §2.5) */
    for (int axis = 0; axis < 3; ++axis) {
        for (int64_t i = 0; i < ex[0]; ++i)
            for (int64_t j = 0; j < ex[1]; ++j)
                for (int64_t k = 0; k < ex[2]; ++k) {
                    int64_t g[3] = {bo->own_lo[0] + i, bo->own_lo[1] + j, bo->own_lo[2] + k};
                    if (!(g[0] < bo->own_hi[0] && g[1] < bo->own_hi[1] && g[2] < bo->own_hi[2])) continue;
                    int64_t l[3] = {i, j, k};
                    if (g[axis] + 1 >= dims[axis]) continue;
                    int64_t l2[3] = {i, j, k};
                    l2[axis] += 1;
                    int ls = loc[(l[0] * ex[1] + l[1]) * ex[2] + l[2]];
                    int lt = loc[(l2[0] * ex[1] + l2[1]) * ex[2] + l2[2]];
                    if (ls == lt) {
                        if (ls) bo->vol_lines += h; /* edge entirely inside */
                        continue;
                    }
                    double s[3];
                    for (int a = 0; a < 3; ++a) s[a] = lo[a] + h * (double)g[a];
                    Witness w;
                    int slow = 0;
                    double tau = first_root(&m, s, axis, h, cap, &w, &slow);
                    bo->slow += slow;
                    double p[3] = {s[0], s[1], s[2]};
                    p[axis] = s[axis] + tau * h;
                    double nrm[3] = {0.0, 0.0, 0.0};
                    if (w.type != EO_TYPE_NONE) {
                        double v[3] = {w.q[0] - p[0], w.q[1] - p[1], w.q[2] - p[2]};
                        double nv = sqrt(dot3(v, v));
                        if (nv > 0.0) for (int a = 0; a < 3; ++a) nrm[a] = v[a] / nv;
                    }
                    int64_t gidx = (g[0] * dims[1] + g[1]) * dims[2] + g[2];
                    ipush(&bo->idx[axis], gidx);
                    dpush(&bo->tau[axis], tau);
                    for (int a = 0; a < 3; ++a) dpush(&bo->nrm[axis], nrm[a]);
                    ipush(&bo->ptype[axis], w.type);
                    for (int q = 0; q < 3; ++q) ipush(&bo->wid[axis], w.type == EO_TYPE_NONE ? -1 : w.ids[q]);
                    /* C9 readings: area by the Crofton-type sum of |n_a|,
                     * volume by the inside length along grid lines */
                    bo->area += h * h * fabs(nrm[axis]);
                    bo->vol_lines += ls ? tau * h : (1.0 - tau) * h;
                }
    }
    free(loc);
    model_free(&m);
    free(sel); free(bx); free(br);
}

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* Run the whole grid (block_pts == 0: one block) or a subset of blocks
 * (block_ids != NULL: only those blocks, for timing samples; labels of other
 * points are left at -1).  nthreads <= 0: OpenMP default. */
static eo_result *run_impl(const double *xyz, const double *r, int64_t n, double rp, double h, double margin,
                           int64_t block_pts, int nthreads, int brute, int instrument, const int64_t *block_ids,
                           int64_t n_block_ids, int sparse, const int64_t *gid, const double *glo,
                           const int64_t *gdims)
{
    if (!(rp > 0.0)) return NULL; /* at r_p = 0 the closed set M is the whole space */
    if (sparse && !block_ids) return NULL;
    eo_result *res = (eo_result *)calloc(1, sizeof(eo_result));
    if (glo) { /* the caller's grid */
        if (!(h > 0.0)) { free(res); return NULL; }
        for (int a = 0; a < 3; ++a) {
            if (gdims[a] < 1) { free(res); return NULL; }
            res->dims[a] = gdims[a];
            res->lo[a] = glo[a];
        }
    } else if (eo_grid(xyz, r, n, h, margin, res->dims, res->lo) != 0) { free(res); return NULL; }
    res->h = h; res->rp = rp;
    res->sparse = sparse;
    const int64_t *dims = res->dims;
    int64_t npts = dims[0] * dims[1] * dims[2];
    if (!sparse) {
        res->labels = (int8_t *)malloc((size_t)npts);
        memset(res->labels, 0xff, (size_t)npts);
    }
    int64_t cells[3], nb[3];
    for (int a = 0; a < 3; ++a) {
        if (block_pts <= 1) { cells[a] = dims[a]; nb[a] = 1; }
        else { cells[a] = block_pts - 1; nb[a] = eo_block_count(dims[a], block_pts); }
    }
    int64_t nblocks = nb[0] * nb[1] * nb[2];
    int64_t nrun = block_ids ? n_block_ids : nblocks;
    BlockOut *bos = (BlockOut *)calloc((size_t)(nrun > 0 ? nrun : 1), sizeof(BlockOut));
    for (int64_t t = 0; t < nrun; ++t) {
        int64_t id = block_ids ? block_ids[t] : t;
        BlockOut *bo = &bos[t];
        bo->b[0] = id / (nb[1] * nb[2]);
        bo->b[1] = (id / nb[2]) % nb[1];
        bo->b[2] = id % nb[2];
        for (int a = 0; a < 3; ++a) {
            bo->own_lo[a] = cells[a] * bo->b[a];                       /* Eq. 5 */
            bo->own_hi[a] = (bo->b[a] == nb[a] - 1) ? dims[a] : bo->own_lo[a] + cells[a];
            bo->cmp_hi[a] = bo->own_hi[a] + 1 < dims[a] ? bo->own_hi[a] + 1 : dims[a];
        }
    }
    if (sparse) {
        res->nblk = nrun;
        res->blk_lo = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)(nrun > 0 ? nrun : 1));
        res->blk_hi = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)(nrun > 0 ? nrun : 1));
        res->blk_off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nrun + 1));
        res->blk_off[0] = 0;
        for (int64_t t = 0; t < nrun; ++t) {
            int64_t e = 1;
            for (int a = 0; a < 3; ++a) {
                res->blk_lo[3 * t + a] = bos[t].own_lo[a];
                res->blk_hi[3 * t + a] = bos[t].own_hi[a];
                e *= bos[t].own_hi[a] - bos[t].own_lo[a];
            }
            res->blk_off[t + 1] = res->blk_off[t] + e;
        }
        res->labels = (int8_t *)malloc((size_t)(res->blk_off[nrun] > 0 ? res->blk_off[nrun] : 1));
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t t = 0; t < nrun; ++t)
        run_block(xyz, r, gid, n, rp, h, dims, res->lo, &bos[t], res->labels,
                  sparse ? res->labels + res->blk_off[t] : NULL, brute, instrument);
    /* OutputInfo: concatenate in block order, then order edges by lower index */
    for (int64_t t = 0; t < nrun; ++t) {
        BlockOut *bo = &bos[t];
        for (int axis = 0; axis < 3; ++axis) {
            for (int64_t e = 0; e < bo->idx[axis].n; ++e) {
                ipush(&res->idx[axis], bo->idx[axis].v[e]);
                dpush(&res->tau[axis], bo->tau[axis].v[e]);
                for (int a = 0; a < 3; ++a) dpush(&res->nrm[axis], bo->nrm[axis].v[3 * e + a]);
                ipush(&res->ptype[axis], bo->ptype[axis].v[e]);
                for (int q = 0; q < 3; ++q) ipush(&res->wid[axis], bo->wid[axis].v[3 * e + q]);
            }
            free(bo->idx[axis].v); free(bo->tau[axis].v); free(bo->nrm[axis].v); free(bo->ptype[axis].v);
            free(bo->wid[axis].v);
        }
        res->area += bo->area;
        res->volume_lines += bo->vol_lines;
        res->volume_count += bo->vol_count;
        res->near_ties += bo->near_ties;
        res->slow_edges += bo->slow;
        res->sum_reach += bo->sum_reach; res->sum_face += bo->sum_face; res->sum_face_tests += bo->sum_face_tests;
        res->sum_arc += bo->sum_arc; res->sum_vert += bo->sum_vert; res->n_shell += bo->n_shell;
        res->n_points_done += bo->n_points;
    }
    free(bos);
    /* sort each axis' edges by lower index (a permutation sort) */
    for (int axis = 0; axis < 3; ++axis) {
        int64_t ne = res->idx[axis].n;
        if (ne < 2) continue;
        int64_t *key = (int64_t *)malloc(sizeof(int64_t) * 2 * (size_t)ne);
        for (int64_t e = 0; e < ne; ++e) { key[2 * e] = res->idx[axis].v[e]; key[2 * e + 1] = e; }
        qsort(key, (size_t)ne, 2 * sizeof(int64_t), cmp_i64);
        int64_t *ni = (int64_t *)malloc(sizeof(int64_t) * (size_t)ne);
        double *nt = (double *)malloc(sizeof(double) * (size_t)ne);
        double *nn = (double *)malloc(sizeof(double) * 3 * (size_t)ne);
        int64_t *np = (int64_t *)malloc(sizeof(int64_t) * (size_t)ne);
        int64_t *nw = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)ne);
        for (int64_t e = 0; e < ne; ++e) {
            int64_t src = key[2 * e + 1];
            ni[e] = res->idx[axis].v[src];
            nt[e] = res->tau[axis].v[src];
            for (int a = 0; a < 3; ++a) nn[3 * e + a] = res->nrm[axis].v[3 * src + a];
            np[e] = res->ptype[axis].v[src];
            for (int q = 0; q < 3; ++q) nw[3 * e + q] = res->wid[axis].v[3 * src + q];
        }
        free(res->idx[axis].v); free(res->tau[axis].v); free(res->nrm[axis].v); free(res->ptype[axis].v);
        free(res->wid[axis].v);
        res->idx[axis].v = ni; res->tau[axis].v = nt; res->nrm[axis].v = nn; res->ptype[axis].v = np;
        res->wid[axis].v = nw;
        res->idx[axis].cap = res->tau[axis].cap = res->ptype[axis].cap = ne;
        res->nrm[axis].cap = res->wid[axis].cap = 3 * ne;
        free(key);
    }
    /* C9: V = mean over the three axes of h^2 * (inside length along lines);
     * the three per-axis sums were accumulated together above */
    res->area = res->area;
    res->volume_lines = h * h * res->volume_lines / 3.0;
    res->volume_count = h * h * h * res->volume_count;
    return res;
}

eo_result *eo_run(const double *xyz, const double *r, int64_t n, double rp, double h, double margin, int64_t block_pts,
                  int nthreads, int brute, int instrument, const int64_t *block_ids, int64_t n_block_ids)
{
    return run_impl(xyz, r, n, rp, h, margin, block_pts, nthreads, brute, instrument, block_ids, n_block_ids, 0, NULL,
                    NULL, NULL);
}

/* As eo_run over the listed blocks only, storing only their owned points'
 * labels (for grids too large to hold whole on the host). */
eo_result *eo_run_sparse(const double *xyz, const double *r, int64_t n, double rp, double h, double margin,
                         int64_t block_pts, int nthreads, const int64_t *block_ids, int64_t n_block_ids)
{
    return run_impl(xyz, r, n, rp, h, margin, block_pts, nthreads, 0, 0, block_ids, n_block_ids, 1, NULL, NULL, NULL);
}

/* As eo_run on a grid given by the caller (point (i,j,k) at origin +
 * h (i,j,k), dims points per axis) instead of the grid of Eq. 2, for atoms
 * that carry the caller's ids (gid: one per atom, or NULL for 0..n-1): the
 * oracle of one rank of a molecule split over processes, which holds only
 * the atoms near its part of the grid. */
eo_result *eo_run_grid(const double *xyz, const double *r, const int64_t *gid, int64_t n, double rp, double h,
                       const double origin[3], const int64_t dims[3], int64_t block_pts, int nthreads)
{
    return run_impl(xyz, r, n, rp, h, h, block_pts, nthreads, 0, 0, NULL, 0, 0, gid, origin, dims);
}

/* sparse runs: owned region [lo, hi) of block t and its label count; labels of block t */
int64_t eo_result_block_region(const eo_result *res, int64_t t, int64_t lo[3], int64_t hi[3])
{
    if (!res->sparse || t < 0 || t >= res->nblk) return -1;
    for (int a = 0; a < 3; ++a) { lo[a] = res->blk_lo[3 * t + a]; hi[a] = res->blk_hi[3 * t + a]; }
    return res->blk_off[t + 1] - res->blk_off[t];
}
void eo_result_block_labels(const eo_result *res, int64_t t, int8_t *out)
{
    memcpy(out, res->labels + res->blk_off[t], (size_t)(res->blk_off[t + 1] - res->blk_off[t]));
}

void eo_result_grid(const eo_result *res, int64_t dims[3], double lo[3])
{
    for (int a = 0; a < 3; ++a) { dims[a] = res->dims[a]; lo[a] = res->lo[a]; }
}
void eo_result_labels(const eo_result *res, int8_t *out)
{
    if (res->sparse) return;
    memcpy(out, res->labels, (size_t)(res->dims[0] * res->dims[1] * res->dims[2]));
}
int64_t eo_result_num_intersections(const eo_result *res, int axis) { return res->idx[axis].n; }
/* the generating atoms of each intersection's witness patch (§4.1's "nearby
 * atoms"): 3 input ids per edge -- one for a convex patch, the pair for a
 * saddle, the triple for a concave patch -- padded with -1 */
void eo_result_intersection_atoms(const eo_result *res, int axis, int64_t *ids)
{
    for (int64_t k = 0; k < res->wid[axis].n; ++k) ids[k] = res->wid[axis].v[k];
}
void eo_result_intersections(const eo_result *res, int axis, int64_t *idx, double *tau, double *normal, int32_t *ptype)
{
    int64_t ne = res->idx[axis].n;
    for (int64_t e = 0; e < ne; ++e) {
        idx[e] = res->idx[axis].v[e];
        tau[e] = res->tau[axis].v[e];
        for (int a = 0; a < 3; ++a) normal[3 * e + a] = res->nrm[axis].v[3 * e + a];
        if (ptype) ptype[e] = (int32_t)res->ptype[axis].v[e];
    }
}
/* stats[0..9] = area, volume(lines), volume(count), near ties, slow edges,
 * sum reach, sum face, sum face tests, sum arc, sum vert; stats2 = shell, points */
void eo_result_stats(const eo_result *res, double *stats)
{
    stats[0] = res->area; stats[1] = res->volume_lines; stats[2] = res->volume_count;
    stats[3] = (double)res->near_ties; stats[4] = (double)res->slow_edges;
    stats[5] = (double)res->sum_reach; stats[6] = (double)res->sum_face; stats[7] = (double)res->sum_face_tests;
    stats[8] = (double)res->sum_arc; stats[9] = (double)res->sum_vert; stats[10] = (double)res->n_shell;
    stats[11] = (double)res->n_points_done;
}
void eo_result_free(eo_result *res)
{
    if (!res) return;
    free(res->labels);
    free(res->blk_lo); free(res->blk_hi); free(res->blk_off);
    for (int a = 0; a < 3; ++a) {
        free(res->idx[a].v); free(res->tau[a].v); free(res->nrm[a].v); free(res->ptype[a].v); free(res->wid[a].v);
    }
    free(res);
}

/* ------------------------------------------------------------------------ */
/* exterior-only surface (cavities filled)                                    */
/* ------------------------------------------------------------------------ */
/* Reading X1.  §1 counts every free probe position as solvent (reading C4);
 * the exterior-only variant keeps only the solvent that a probe can reach
 * from outside the molecule.  On the grid: an outside point is exterior iff a
 * path of outside points, each step between 6-neighbours, joins it to the
 * domain boundary (whose points are all outside, reading C2).  Every other
 * outside point lies in a cavity and becomes inside.  Plain breadth-first
 * search from the boundary.  Returns the number of relabelled points. */
int64_t eo_exterior_labels(int8_t *labels, const int64_t dims[3])
{
    const int64_t d0 = dims[0], d1 = dims[1], d2 = dims[2], n = d0 * d1 * d2;
    if (n <= 0) return 0;
    uint8_t *seen = (uint8_t *)calloc((size_t)n, 1);
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t head = 0, tail = 0;
    for (int64_t i = 0; i < d0; ++i)
        for (int64_t j = 0; j < d1; ++j)
            for (int64_t k = 0; k < d2; ++k) {
                int on_face = i == 0 || j == 0 || k == 0 || i == d0 - 1 || j == d1 - 1 || k == d2 - 1;
                int64_t p = (i * d1 + j) * d2 + k;
                if (on_face && labels[p] == 0) { seen[p] = 1; queue[tail++] = p; }
            }
    while (head < tail) {
        int64_t p = queue[head++];
        int64_t g[3] = {p / (d1 * d2), (p / d2) % d1, p % d2};
        for (int a = 0; a < 3; ++a)
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                int64_t q[3] = {g[0], g[1], g[2]};
                q[a] += sgn;
                if (q[a] < 0 || q[a] >= dims[a]) continue;
                int64_t pq = (q[0] * d1 + q[1]) * d2 + q[2];
                if (labels[pq] == 0 && !seen[pq]) { seen[pq] = 1; queue[tail++] = pq; }
            }
    }
    int64_t filled = 0;
    for (int64_t p = 0; p < n; ++p)
        if (labels[p] == 0 && !seen[p]) { labels[p] = 1; ++filled; }
    free(seen);
    free(queue);
    return filled;
}

/* Exterior-only form of a whole-grid result: cavity points relabelled inside
 * (eo_exterior_labels), the crossing edges that touch them dropped -- their
 * other end is inside, since an outside neighbour would have joined the
 * cavity to the exterior, so the edges left keep their first roots -- and the
 * area and volume recomputed from what is left with the estimators of C9.
 * Returns the number of relabelled points, -1 for a sparse result. */
int64_t eo_result_exterior(eo_result *res)
{
    if (res->sparse) return -1;
    const int64_t *dims = res->dims;
    const double h = res->h;
    int64_t filled = eo_exterior_labels(res->labels, dims);
    const int64_t str[3] = {dims[1] * dims[2], dims[2], 1};
    double area = 0.0, lines = 0.0;
    for (int axis = 0; axis < 3; ++axis) {
        int64_t keep = 0;
        for (int64_t e = 0; e < res->idx[axis].n; ++e) {
            int64_t p = res->idx[axis].v[e];
            int ls = res->labels[p], lt = res->labels[p + str[axis]];
            if (ls == lt) continue;
            res->idx[axis].v[keep] = p;
            res->tau[axis].v[keep] = res->tau[axis].v[e];
            for (int a = 0; a < 3; ++a) res->nrm[axis].v[3 * keep + a] = res->nrm[axis].v[3 * e + a];
            res->ptype[axis].v[keep] = res->ptype[axis].v[e];
            for (int q = 0; q < 3; ++q) res->wid[axis].v[3 * keep + q] = res->wid[axis].v[3 * e + q];
            double tau = res->tau[axis].v[e];
            area += h * h * fabs(res->nrm[axis].v[3 * e + axis]);
            lines += ls ? tau * h : (1.0 - tau) * h;
            ++keep;
        }
        res->idx[axis].n = res->tau[axis].n = res->ptype[axis].n = keep;
        res->nrm[axis].n = res->wid[axis].n = 3 * keep;
    }
    int64_t inside = 0;
    for (int64_t i = 0; i < dims[0]; ++i)
        for (int64_t j = 0; j < dims[1]; ++j)
            for (int64_t k = 0; k < dims[2]; ++k) {
                int64_t g[3] = {i, j, k}, p = (i * dims[1] + j) * dims[2] + k;
                if (!res->labels[p]) continue;
                ++inside;
                for (int axis = 0; axis < 3; ++axis)
                    if (g[axis] + 1 < dims[axis] && res->labels[p + str[axis]]) lines += h; /* edge inside */
            }
    res->area = area;
    res->volume_lines = h * h * lines / 3.0;
    res->volume_count = h * h * h * (double)inside;
    return filled;
}

int eo_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* algorithmic flop model (instrumentation)                                  */
/* ------------------------------------------------------------------------ */
/* Counts, over every grid point x, the candidate work that the definition of
 * Eq. 2 implies, with fixed unit costs:
 *   8  per atom within reach (|x - c| < r + 2 r_p: the atoms that decide x);
 * and for shell points (inside some expanded ball, outside every van der
 * Waals ball):
 *   12 per face candidate (expanded ball containing x) plus 8 per freeness
 *      test of its projection against each atom within reach,
 *   30 per saddle candidate (pair circle passing within r_p of x, with x
 *      inside one of the pair's expanded balls),
 *   8  per concave candidate (free triple point within r_p of x).
 * out[0] = points, out[1] = sum n_reach, out[2] = shell points,
 * out[3] = sum over shell points of n_face, out[4] = sum of n_face * n_reach,
 * out[5] = sum n_arc, out[6] = sum n_vert, out[7] = total model flops. */
int eo_flop_counts(const double *xyz, const double *r, int64_t n, double rp, double h, double margin, int nthreads,
                   int64_t *out)
{
    int64_t dims[3];
    double lo[3];
    if (eo_grid(xyz, r, n, h, margin, dims, lo) != 0) return -1;
    Model m;
    model_build(&m, xyz, r, NULL, (int)n, rp, rp, 0);
    /* saddle candidates: circles within r_p of x whose pair has a ball that
     * contains x (the nearest free point of x lies on such a circle's arc
     * only then: x is in the triangle of the two centres and that point) */
    int64_t s_reach = 0, s_shell = 0, s_face = 0, s_fr = 0, s_arc = 0, s_vert = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : s_reach, s_shell, s_face, s_fr, s_arc, s_vert)
#endif
    for (int64_t i = 0; i < dims[0]; ++i)
        for (int64_t j = 0; j < dims[1]; ++j)
            for (int64_t k = 0; k < dims[2]; ++k) {
                double x[3] = {lo[0] + h * (double)i, lo[1] + h * (double)j, lo[2] + h * (double)k};
                long reach = 0, face = 0;
                int in_vdw = 0;
                FOR_NEAR(&m, x, m.a_start, m.a_list, m.n, a, {
                    double d2 = dist2(x, m.c + 3 * a);
                    double rr = m.r[a] + 2.0 * rp;
                    if (d2 < rr * rr) reach++;
                    if (d2 < m.R[a] * m.R[a]) face++;
                    if (d2 < m.r[a] * m.r[a]) in_vdw = 1;
                });
                s_reach += reach;
                if (face == 0 || in_vdw) continue;
                s_shell++;
                s_face += face;
                s_fr += face * reach;
                long arc = 0, vert = 0;
                FOR_NEAR(&m, x, m.p_start, m.p_list, m.np, p, {
                    const double *o = m.po + 3 * p, *u = m.pu + 3 * p;
                    double y[3] = {x[0] - o[0], x[1] - o[1], x[2] - o[2]};
                    double z = dot3(y, u);
                    double w2 = dot3(y, y) - z * z;
                    double nw = sqrt(w2 > 0.0 ? w2 : 0.0);
                    double e = nw - m.prho[p];
                    if (e * e + z * z < rp * rp) {
                        int pi_ = m.pi[p], pj_ = m.pj[p];
                        if (dist2(x, m.c + 3 * pi_) < m.R[pi_] * m.R[pi_] || dist2(x, m.c + 3 * pj_) < m.R[pj_] * m.R[pj_])
                            arc++;
                    }
                });
                FOR_NEAR(&m, x, m.v_start, m.v_list, m.nv, v, {
                    if (dist2(x, m.vq + 3 * v) < rp * rp) vert++;
                });
                s_arc += arc;
                s_vert += vert;
            }
    model_free(&m);
    out[0] = dims[0] * dims[1] * dims[2];
    out[1] = s_reach;
    out[2] = s_shell;
    out[3] = s_face;
    out[4] = s_fr;
    out[5] = s_arc;
    out[6] = s_vert;
    out[7] = 8 * s_reach + 12 * s_face + 8 * s_fr + 30 * s_arc + 8 * s_vert;
    return 0;
}

/* Edge terms of the flop model, over given crossing edges (lower point
 * linear index per axis): per edge, 20 flops per sphere-patch candidate (van
 * der Waals sphere or probe sphere of a free triple point that the edge
 * segment meets) and 150 per torus candidate (circle whose tube of radius r_p
 * the segment meets: the distance to the circle takes r_p on the segment,
 * judged on 33 samples with the 1-Lipschitz slack).
 * out[0] = edges, out[1] = van der Waals spheres, out[2] = probe spheres,
 * out[3] = tori, out[4] = model flops. */
static double seg_dist2(const double *s, int axis, double h, const double *c)
{
    double t = c[axis] - s[axis];
    if (t < 0.0) t = 0.0;
    if (t > h) t = h;
    double y[3] = {s[0], s[1], s[2]};
    y[axis] += t;
    return dist2(y, c);
}

int eo_edge_flop_counts(const double *xyz, const double *r, int64_t n, double rp, double h, double margin,
                        const int64_t *n_edges, const int64_t *const *idx, int nthreads, int64_t *out)
{
    int64_t dims[3];
    double lo[3];
    if (eo_grid(xyz, r, n, h, margin, dims, lo) != 0) return -1;
    Model m;
    model_build(&m, xyz, r, NULL, (int)n, rp, rp + h, 0);
    int64_t s_e = 0, s_v = 0, s_p = 0, s_t = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    for (int axis = 0; axis < 3; ++axis) {
        const int64_t ne = n_edges[axis];
        const int64_t *ix = idx[axis];
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : s_e, s_v, s_p, s_t)
#endif
        for (int64_t e = 0; e < ne; ++e) {
            int64_t g = ix[e];
            int64_t gi = g / (dims[1] * dims[2]), gj = (g / dims[2]) % dims[1], gk = g % dims[2];
            double s[3] = {lo[0] + h * (double)gi, lo[1] + h * (double)gj, lo[2] + h * (double)gk};
            double mid[3] = {s[0], s[1], s[2]};
            mid[axis] += 0.5 * h;
            s_e++;
            FOR_NEAR(&m, mid, m.a_start, m.a_list, m.n, a, {
                if (seg_dist2(s, axis, h, m.c + 3 * a) < m.r[a] * m.r[a]) s_v++;
            });
            FOR_NEAR(&m, mid, m.v_start, m.v_list, m.nv, v, {
                if (seg_dist2(s, axis, h, m.vq + 3 * v) < rp * rp) s_p++;
            });
            FOR_NEAR(&m, mid, m.p_start, m.p_list, m.np, p, {
                const double *o = m.po + 3 * p, *u = m.pu + 3 * p;
                double dmin = 1e300, dmax = -1e300;
                for (int k = 0; k <= 32; ++k) {
                    double y[3] = {s[0] - o[0], s[1] - o[1], s[2] - o[2]};
                    y[axis] += h * (double)k / 32.0;
                    double z = dot3(y, u);
                    double w2 = dot3(y, y) - z * z;
                    double ee = sqrt(w2 > 0.0 ? w2 : 0.0) - m.prho[p];
                    double d = sqrt(ee * ee + z * z);
                    if (d < dmin) dmin = d;
                    if (d > dmax) dmax = d;
                }
                double slack = h / 64.0;
                if (dmin - slack <= rp && dmax + slack >= rp) s_t++;
            });
        }
    }
    model_free(&m);
    out[0] = s_e;
    out[1] = s_v;
    out[2] = s_p;
    out[3] = s_t;
    out[4] = 20 * (s_v + s_p) + 150 * s_t;
    return 0;
}
