// eses_api.cu -- the C ABI (include/eses.h) and the host orchestration of one
// run: cell binning -> neighbours -> circle pairs -> free arcs and triple
// points -> patch bins -> classification (+ FP64 band) -> crossing edges ->
// roots -> area/volume.  Every step runs on the device; the host only sizes
// buffers (it reads four list totals per run) and launches.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/eses.h"
#include "eses_kernels.h"

using namespace eses;

// stages timed with CUDA events when ESES_OPT_PROFILE is set
enum { NSTAT = 11 };
enum { ST_BIN = 0, ST_PAIRS, ST_ARCS, ST_CLASSIFY, ST_BAND, ST_EDGE_COUNT, ST_EDGE_SOLVE, ST_EDGE_POLISH, ST_REDUCE, NSTAGE };

namespace {

struct DBuf {
    void *p = nullptr;
    size_t cap = 0;
};

struct CudaError {
    cudaError_t e;
    const char *what;
};

void ck(cudaError_t e, const char *what)
{
    if (e != cudaSuccess) throw CudaError{e, what};
}

template <class T>
T *ensure(DBuf &b, size_t count)
{
    size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    if (b.cap < bytes) {
        if (b.p) cudaFree(b.p);
        b.p = nullptr;
        b.cap = 0;
        size_t want = bytes + bytes / 4;
        cudaError_t e = cudaMalloc(&b.p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            b.p = nullptr;
            throw std::bad_alloc();
        }
        b.cap = want;
    }
    return (T *)b.p;
}

thread_local std::string g_create_error;

}  // namespace

struct eses_ctx {
    int device = 0;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    bool sync = true;
    int precision = ESES_PREC_FP32_FILTERED;
    int block_pts = 64;
    long long n_atoms = 0;
    double rp = 0, h = 0, margin = 0;
    double lo[3] = {0, 0, 0};
    long long dims[3] = {0, 0, 0};
    double rmax = 0, Rmax = 0;
    double amin[3], amax[3];
    Model M{};
    Grid G{};
    // device buffers
    DBuf xyz, rad, cell_id, cell_count, cell_start, cursor, atom_orig, atom;
    DBuf nb_count, nb_start, nb_list, circle_count, contained, face;
    DBuf pair_count, pair_start, pair_o, pair_u, pair_ij, pair_free;
    DBuf vert_count, vert_start, vert;
    DBuf pbin_count, pbin_start, pbin_cursor, pbin_cell, pbin_list;
    DBuf vbin_count, vbin_start, vbin_cursor, vbin_cell, vbin_list;
    DBuf labels, tile_band, tile_edges, edge_start, tile_inside, tile_area, tile_vol;
    DBuf out_idx[3], out_tau[3], out_nrm[3], out_tau32[3], out_nrm32[3], out_code[3];
    DBuf scan_tmp, misc;  // misc: err, n_fail, area/vol, counts
    DBuf fail_log;
    DBuf atom_hi, atom_lo, pair_hi, pair_lo, pair_u32, vert_hi, vert_lo;
    // results
    bool ran = false;
    long long n_edges[3] = {0, 0, 0};
    double area = 0, volume = 0;
    long long stats[NSTAT] = {0};
    std::string err;
    // stage timing (ESES_OPT_PROFILE)
    bool profile = false;
    cudaEvent_t ev[NSTAGE + 1] = {};
    float stage_ms[NSTAGE] = {0};
};

namespace {

int fail(eses_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    else g_create_error = msg;
    return code;
}

int scan(eses_ctx *c, const int *in, int *out, long long n)
{
    int *tmp = ensure<int>(c->scan_tmp, (size_t)scan_tmp_ints(n));
    return scan_exclusive(in, out, n, tmp, c->stream);
}

int read_total(eses_ctx *c, const int *start, long long n)
{
    int v = 0;
    ck(cudaMemcpyAsync(&v, start + n, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "read list total");
    ck(cudaStreamSynchronize(c->stream), "synchronize");
    return v;
}

int validate(const double *xyz, const double *r, int64_t n, double rp, double h, double margin, std::string &msg)
{
    if (n < 1 || n > (int64_t)1 << 30) { msg = "n_atoms must be in [1, 2^30]"; return ESES_EINVAL; }
    if (!(rp > 0.0) || !isfinite(rp)) { msg = "r_p must be finite and > 0"; return ESES_EINVAL; }
    if (!(h > 0.0) || !isfinite(h)) { msg = "h must be finite and > 0"; return ESES_EINVAL; }
    if (!(margin >= h) || !isfinite(margin)) { msg = "margin must be finite and >= h"; return ESES_EINVAL; }
    for (int64_t i = 0; i < n; ++i) {
        if (!isfinite(xyz[3 * i]) || !isfinite(xyz[3 * i + 1]) || !isfinite(xyz[3 * i + 2])) {
            msg = "non-finite atom coordinate at index " + std::to_string(i);
            return ESES_EINVAL;
        }
        if (!(r[i] > 0.0) || !isfinite(r[i])) {
            msg = "atom radius must be finite and > 0 (index " + std::to_string(i) + ")";
            return ESES_EINVAL;
        }
    }
    return ESES_OK;
}

// grid of Eq. 2 and the cell/tile layout; xyz/r on the host
int setup(eses_ctx *c, const double *xyz, const double *r)
{
    const long long n = c->n_atoms;
    c->rmax = 0.0;
    for (int a = 0; a < 3; ++a) {
        double mn = xyz[a] - r[0], mx = xyz[a] + r[0];
        c->amin[a] = xyz[a];
        c->amax[a] = xyz[a];
        for (long long i = 1; i < n; ++i) {
            double v0 = xyz[3 * i + a] - r[i], v1 = xyz[3 * i + a] + r[i];
            if (v0 < mn) mn = v0;
            if (v1 > mx) mx = v1;
            c->amin[a] = std::min(c->amin[a], xyz[3 * i + a]);
            c->amax[a] = std::max(c->amax[a], xyz[3 * i + a]);
        }
        c->lo[a] = mn - c->margin;
        c->dims[a] = (long long)ceil((mx + c->margin - c->lo[a]) / c->h) + 1;
    }
    for (long long i = 0; i < n; ++i) c->rmax = std::max(c->rmax, r[i]);
    c->Rmax = c->rmax + c->rp;
    long long npts = c->dims[0] * c->dims[1] * c->dims[2];
    if (c->dims[0] > (1LL << 30) || c->dims[1] > (1LL << 30) || c->dims[2] > (1LL << 30) || npts > (1LL << 40))
        return fail(c, ESES_EINVAL, "grid too large");
    Model &M = c->M;
    M.n_atoms = (int)n;
    M.rp = c->rp;
    M.rmax = c->rmax;
    M.Rmax = c->Rmax;
    // cubic cells of edge >= 2 R_max: overlapping expanded balls sit in adjacent cells
    M.cell = std::max(2.0 * c->Rmax, 1e-3);
    for (int a = 0; a < 3; ++a) M.clo[a] = c->amin[a] - 1e-6;
    long long ncell = 0;
    for (int it = 0; it < 200; ++it) {
        ncell = 1;
        for (int a = 0; a < 3; ++a) {
            long long k = (long long)floor((c->amax[a] - M.clo[a]) / M.cell) + 1;
            M.cn[a] = (int)std::min(k, 1LL << 20);
            ncell *= k;
        }
        if (ncell <= (1LL << 26)) break;
        M.cell *= 1.25;  // very sparse extents: coarser cells stay correct
    }
    if (ncell > (1LL << 26)) return fail(c, ESES_EINVAL, "cell grid too large");
    Grid &G = c->G;
    for (int a = 0; a < 3; ++a) {
        G.lo[a] = c->lo[a];
        G.dims[a] = c->dims[a];
        G.tiles[a] = (int)ceil_div_ll(c->dims[a], TILE);
    }
    G.h = c->h;
    G.n_tiles = (long long)G.tiles[0] * G.tiles[1] * G.tiles[2];
    G.rp = c->rp;
    G.halo = c->rmax + 2.0 * c->rp;
    double L = 8.0 * c->h * sqrt(3.0) + G.halo + 1.0;
    // staged FP32 coordinates carry two roundings of at most 2^-24 L each, a grid
    // point one, a difference of two of them one more: 5 * 2^-24 L per
    // coordinate, 5.2e-7 L for the vector; d0 rounds that up
    G.d0 = (float)(6e-7 * L);
    for (int k = 0; k <= TILE; ++k) G.hl[k] = (float)((double)k * c->h);
    G.ht_hi = (float)(TILE * c->h);
    G.ht_lo = (float)(TILE * c->h - (double)G.ht_hi);
    return ESES_OK;
}

int create_common(const double *hxyz, const double *hr, int64_t n, double rp, double h, double margin,
                  const double *dxyz, const double *dr, eses_ctx **out)
{
    if (!out) return fail(nullptr, ESES_EINVAL, "out is NULL");
    *out = nullptr;
    std::string msg;
    int rc = validate(hxyz, hr, n, rp, h, margin, msg);
    if (rc) return fail(nullptr, rc, msg);
    eses_ctx *c = new (std::nothrow) eses_ctx();
    if (!c) return fail(nullptr, ESES_ENOMEM, "host allocation failed");
    c->n_atoms = n;
    c->rp = rp;
    c->h = h;
    c->margin = margin;
    try {
        ck(cudaGetDevice(&c->device), "cudaGetDevice");
        ck(cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking), "cudaStreamCreate");
        c->stream = c->own_stream;
        rc = setup(c, hxyz, hr);
        if (rc) {
            g_create_error = c->err;
            eses_destroy(c);
            return rc;
        }
        double *x = ensure<double>(c->xyz, 3 * (size_t)n);
        double *r = ensure<double>(c->rad, (size_t)n);
        if (dxyz) {
            ck(cudaMemcpyAsync(x, dxyz, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, c->stream), "copy atoms");
            ck(cudaMemcpyAsync(r, dr, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream), "copy radii");
        } else {
            ck(cudaMemcpyAsync(x, hxyz, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, c->stream), "copy atoms");
            ck(cudaMemcpyAsync(r, hr, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream), "copy radii");
        }
        ck(cudaStreamSynchronize(c->stream), "synchronize");
    } catch (const CudaError &e) {
        std::string m = std::string(e.what) + ": " + cudaGetErrorString(e.e);
        eses_destroy(c);
        return fail(nullptr, ESES_ECUDA, m);
    } catch (const std::bad_alloc &) {
        eses_destroy(c);
        return fail(nullptr, ESES_ENOMEM, "device allocation failed");
    }
    *out = c;
    return ESES_OK;
}

void free_buf(DBuf &b)
{
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
}

void mark(eses_ctx *c, int k)
{
    if (c->profile) ck(cudaEventRecord(c->ev[k], c->stream), "cudaEventRecord");
}

int run_impl(eses_ctx *c)
{
    cudaStream_t st = c->stream;
    int nl = 0;  // kernels launched by this run
    if (c->profile && !c->ev[0])
        for (int k = 0; k <= NSTAGE; ++k) ck(cudaEventCreate(&c->ev[k]), "cudaEventCreate");
    Model &M = c->M;
    Grid &G = c->G;
    const int n = M.n_atoms;
    const long long ncell = (long long)M.cn[0] * M.cn[1] * M.cn[2];
    int *misc = ensure<int>(c->misc, 64);
    int *d_err = misc, *d_fail = misc + 1;
    double *d_av = (double *)(misc + 8);
    long long *d_counts = (long long *)(misc + 16);
    ck(cudaMemsetAsync(misc, 0, 64 * sizeof(int), st), "memset");

    mark(c, ST_BIN);
    // 1. cell binning (counting sort, deterministic within a cell)
    int *cell_id = ensure<int>(c->cell_id, n);
    int *cell_count = ensure<int>(c->cell_count, ncell);
    int *cell_start = ensure<int>(c->cell_start, ncell + 1);
    int *cursor = ensure<int>(c->cursor, ncell);
    int *orig = ensure<int>(c->atom_orig, n);
    double4 *atom = ensure<double4>(c->atom, n);
    ck(cudaMemsetAsync(cell_count, 0, sizeof(int) * ncell, st), "memset");
    ck(cudaMemsetAsync(cursor, 0, sizeof(int) * ncell, st), "memset");
    nl += launch_cell_count((const double *)c->xyz.p, (const double *)c->rad.p, n, M.clo, M.cell, M.cn, cell_id, cell_count,
                      st);
    nl += scan(c, cell_count, cell_start, ncell);
    nl += launch_cell_scatter(nullptr, nullptr, n, cell_id, cell_start, cursor, orig, st);
    nl += launch_cell_finish((const double *)c->xyz.p, (const double *)c->rad.p, n, (int)ncell, cell_start, orig, atom, st);
    M.atom = atom;
    M.atom_orig = orig;
    M.cell_start = cell_start;
    float4 *ahi = ensure<float4>(c->atom_hi, n), *alo = ensure<float4>(c->atom_lo, n);
    nl += launch_model_f32(M, 0, G.lo, ahi, alo, nullptr, st);
    M.atom_hi = ahi;
    M.atom_lo = alo;

    mark(c, ST_PAIRS);
    // 2. neighbours
    int *nb_count = ensure<int>(c->nb_count, n);
    int *circle_count = ensure<int>(c->circle_count, n);
    uint8_t *contained = ensure<uint8_t>(c->contained, n);
    int *nb_start = ensure<int>(c->nb_start, n + 1);
    nl += launch_nb_count(M, nb_count, circle_count, contained, st);
    nl += scan(c, nb_count, nb_start, n);
    int n_nb = read_total(c, nb_start, n);
    int *nb_list = ensure<int>(c->nb_list, std::max(n_nb, 1));
    M.nb_start = nb_start;
    M.nb_list = nb_list;
    nl += launch_nb_fill(M, nb_list, st);

    // 3. circle pairs
    int *pair_count = ensure<int>(c->pair_count, n);
    int *pair_start = ensure<int>(c->pair_start, n + 1);
    nl += launch_pair_count(M, pair_count, st);
    nl += scan(c, pair_count, pair_start, n);
    int np = read_total(c, pair_start, n);
    M.n_pairs = np;
    double4 *pair_o = ensure<double4>(c->pair_o, std::max(np, 1));
    double4 *pair_u = ensure<double4>(c->pair_u, std::max(np, 1));
    int2 *pair_ij = ensure<int2>(c->pair_ij, std::max(np, 1));
    nl += launch_pair_fill(M, pair_start, pair_o, pair_u, pair_ij, st);
    M.pair_o = pair_o;
    M.pair_u = pair_u;
    M.pair_ij = pair_ij;
    float4 *phi = ensure<float4>(c->pair_hi, std::max(np, 1)), *plo = ensure<float4>(c->pair_lo, std::max(np, 1));
    float4 *pu32 = ensure<float4>(c->pair_u32, std::max(np, 1));
    nl += launch_model_f32(M, 1, G.lo, phi, plo, pu32, st);
    M.pair_hi = phi;
    M.pair_lo = plo;
    M.pair_u32 = pu32;

    mark(c, ST_ARCS);
    // 4. free arcs and free triple points
    uint8_t *pair_free = ensure<uint8_t>(c->pair_free, std::max(np, 1));
    int *vert_count = ensure<int>(c->vert_count, std::max(np, 1));
    int *vert_start = ensure<int>(c->vert_start, np + 1);
    nl += launch_arcs(M, pair_free, vert_count, st);
    M.pair_free = pair_free;
    nl += scan(c, vert_count, vert_start, np);
    int nv = read_total(c, vert_start, np);
    M.n_verts = nv;
    double4 *vert = ensure<double4>(c->vert, std::max(nv, 1));
    nl += launch_arcs_emit(M, vert_start, vert, st);
    M.vert = vert;

    if (n >= (1 << 27) || np >= (1 << 27) || nv >= (1 << 27))
        return fail(c, ESES_EINVAL, "more than 2^27 atoms, circle pairs or triple points");
    // 5. free faces
    uint8_t *face = ensure<uint8_t>(c->face, n);
    nl += launch_faces(M, circle_count, contained, face, st);
    M.atom_face = face;

    // 6. patch bins
    int *pcnt = ensure<int>(c->pbin_count, ncell);
    int *pstart = ensure<int>(c->pbin_start, ncell + 1);
    int *pcur = ensure<int>(c->pbin_cursor, ncell);
    int *pcell = ensure<int>(c->pbin_cell, std::max(np, 1));
    int *plist = ensure<int>(c->pbin_list, std::max(np, 1));
    ck(cudaMemsetAsync(pcnt, 0, sizeof(int) * ncell, st), "memset");
    ck(cudaMemsetAsync(pcur, 0, sizeof(int) * ncell, st), "memset");
    nl += launch_bin_count(M, 0, pcnt, pcell, st);
    nl += scan(c, pcnt, pstart, ncell);
    nl += launch_bin_scatter(M, 0, pcell, pstart, pcur, plist, st);
    int *vcnt = ensure<int>(c->vbin_count, ncell);
    int *vstart = ensure<int>(c->vbin_start, ncell + 1);
    int *vcur = ensure<int>(c->vbin_cursor, ncell);
    int *vcell = ensure<int>(c->vbin_cell, std::max(nv, 1));
    int *vlist = ensure<int>(c->vbin_list, std::max(nv, 1));
    ck(cudaMemsetAsync(vcnt, 0, sizeof(int) * ncell, st), "memset");
    ck(cudaMemsetAsync(vcur, 0, sizeof(int) * ncell, st), "memset");
    nl += launch_bin_count(M, 1, vcnt, vcell, st);
    nl += scan(c, vcnt, vstart, ncell);
    nl += launch_bin_scatter(M, 1, vcell, vstart, vcur, vlist, st);
    M.pcell_start = pstart;
    M.pcell_list = plist;
    M.vcell_start = vstart;
    M.vcell_list = vlist;
    float4 *vhi = ensure<float4>(c->vert_hi, std::max(nv, 1)), *vlo = ensure<float4>(c->vert_lo, std::max(nv, 1));
    nl += launch_model_f32(M, 2, G.lo, vhi, vlo, nullptr, st);
    M.vert_hi = vhi;
    M.vert_lo = vlo;

    // 7. classification (+ FP64 band re-evaluation)
    const long long npts = G.dims[0] * G.dims[1] * G.dims[2];
    const long long nt = G.n_tiles;
    int8_t *labels = ensure<int8_t>(c->labels, npts);
    int *tile_band = ensure<int>(c->tile_band, nt);
    mark(c, ST_CLASSIFY);
    nl += launch_classify(M, G, c->precision, labels, c->precision == ESES_PREC_FP64 ? nullptr : tile_band, d_err, st);
    mark(c, ST_BAND);
    if (c->precision != ESES_PREC_FP64) nl += launch_band(M, G, labels, tile_band, d_err, st);

    // 8. crossing edges, roots, area and volume
    int *tile_edges = ensure<int>(c->tile_edges, 3 * nt);
    int *edge_start = ensure<int>(c->edge_start, 3 * nt + 1);
    int *tile_inside = ensure<int>(c->tile_inside, 4 * nt);
    mark(c, ST_EDGE_COUNT);
    nl += launch_edge_count(G, labels, tile_edges, tile_inside, st);
    nl += scan(c, tile_edges, edge_start, 3 * nt);
    std::vector<int> tot(4);
    for (int a = 0; a < 3; ++a)
        ck(cudaMemcpyAsync(&tot[a], edge_start + a * nt, sizeof(int), cudaMemcpyDeviceToHost, st), "read");
    ck(cudaMemcpyAsync(&tot[3], edge_start + 3 * nt, sizeof(int), cudaMemcpyDeviceToHost, st), "read");
    ck(cudaStreamSynchronize(st), "synchronize");
    EdgeOut eo;
    for (int a = 0; a < 3; ++a) {
        long long ne = (long long)tot[a + 1] - tot[a];
        c->n_edges[a] = ne;
        eo.idx[a] = ensure<long long>(c->out_idx[a], std::max(ne, 1LL));
        eo.tau[a] = ensure<double>(c->out_tau[a], std::max(ne, 1LL));
        eo.nrm[a] = ensure<double>(c->out_nrm[a], 3 * std::max(ne, 1LL));
        eo.tau32[a] = ensure<float>(c->out_tau32[a], std::max(ne, 1LL));
        eo.nrm32[a] = ensure<float>(c->out_nrm32[a], 3 * std::max(ne, 1LL));
        eo.code[a] = ensure<int2>(c->out_code[a], std::max(ne, 1LL));
    }
    const long long nparts = polish_blocks(c->n_edges[0] + c->n_edges[1] + c->n_edges[2]);
    double *part = ensure<double>(c->tile_area, 2 * std::max(nparts, 1LL));
    mark(c, ST_EDGE_SOLVE);
    long long *fail_log = ensure<long long>(c->fail_log, FAIL_LOG * FAIL_REC);
    nl += launch_edge_solve(M, G, c->precision, labels, edge_start, eo, d_fail, d_err, fail_log, st);
    mark(c, ST_EDGE_POLISH);
    nl += launch_edge_polish(M, G, eo, c->n_edges, part, st);
    mark(c, ST_REDUCE);
    nl += launch_reduce(G, part, nparts, tile_inside, d_av, d_counts, st);
    mark(c, NSTAGE);
    ck(cudaGetLastError(), "kernel launch");

    // results
    int hmisc[64];
    ck(cudaMemcpyAsync(hmisc, misc, sizeof(hmisc), cudaMemcpyDeviceToHost, st), "read results");
    ck(cudaStreamSynchronize(st), "synchronize");
    if (c->profile)
        for (int k = 0; k < NSTAGE; ++k) ck(cudaEventElapsedTime(&c->stage_ms[k], c->ev[k], c->ev[k + 1]), "elapsed");
    double av[2];
    memcpy(av, hmisc + 8, sizeof(av));
    long long cnt[2];
    memcpy(cnt, hmisc + 16, sizeof(cnt));
    c->area = av[0];
    c->volume = av[1];
    c->stats[0] = npts;
    c->stats[1] = nt;
    c->stats[2] = 0;
    c->stats[3] = np;
    c->stats[4] = -1;  // filled on demand by eses_patch_counts
    c->stats[5] = nv;
    c->stats[6] = 0;
    c->stats[7] = c->n_edges[0] + c->n_edges[1] + c->n_edges[2];
    c->stats[8] = hmisc[1];
    c->stats[9] = cnt[0];
    c->stats[10] = nl;
    c->ran = true;
    int derr = hmisc[0];
    if (derr & (ERR_CAP_ATOMS | ERR_CAP_PAIRS | ERR_CAP_VERTS | ERR_CAP_CAND)) {
        c->ran = false;
        return fail(c, ESES_ECAPACITY, (derr & ERR_CAP_CAND) ? "an edge had more candidate roots than its buffer holds"
                                                             : "a tile's staged list exceeded its shared-memory capacity");
    }
    if (hmisc[1] > 0)
        return fail(c, ESES_EROOT, std::to_string(hmisc[1]) + " crossing edges had no surface root");
    return ESES_OK;
}

}  // namespace

extern "C" {

int eses_create(const double *xyz, const double *radii, int64_t n_atoms, double r_p, double h, double margin,
                eses_ctx **out)
{
    if (!xyz || !radii) return fail(nullptr, ESES_EINVAL, "xyz or radii is NULL");
    return create_common(xyz, radii, n_atoms, r_p, h, margin, nullptr, nullptr, out);
}

int eses_create_device(const double *xyz, const double *radii, int64_t n_atoms, double r_p, double h, double margin,
                       eses_ctx **out)
{
    if (!xyz || !radii) return fail(nullptr, ESES_EINVAL, "xyz or radii is NULL");
    if (n_atoms < 1 || n_atoms > (int64_t)1 << 30) return fail(nullptr, ESES_EINVAL, "n_atoms must be in [1, 2^30]");
    std::vector<double> hx(3 * (size_t)n_atoms), hr((size_t)n_atoms);
    if (cudaMemcpy(hx.data(), xyz, sizeof(double) * 3 * n_atoms, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(hr.data(), radii, sizeof(double) * n_atoms, cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, ESES_EINVAL, "xyz/radii are not readable device memory");
    }
    return create_common(hx.data(), hr.data(), n_atoms, r_p, h, margin, xyz, radii, out);
}

int eses_set_option(eses_ctx *c, int key, int64_t value)
{
    if (!c) return fail(nullptr, ESES_EINVAL, "ctx is NULL");
    switch (key) {
    case ESES_OPT_BLOCK_PTS:
        if (value < 9 || value > (1 << 20)) return fail(c, ESES_EINVAL, "block points must be in [9, 2^20]");
        c->block_pts = (int)value;
        return ESES_OK;
    case ESES_OPT_PRECISION:
        if (value != ESES_PREC_FP64 && value != ESES_PREC_FP32_FILTERED) return fail(c, ESES_EINVAL, "bad precision");
        c->precision = (int)value;
        return ESES_OK;
    case ESES_OPT_STREAM:
        c->stream = value ? (cudaStream_t)(intptr_t)value : c->own_stream;
        return ESES_OK;
    case ESES_OPT_SYNC:
        c->sync = value != 0;
        return ESES_OK;
    case ESES_OPT_PROFILE:
        c->profile = value != 0;
        return ESES_OK;
    default:
        return fail(c, ESES_EINVAL, "unknown option key " + std::to_string(key));
    }
}

int eses_run(eses_ctx *c)
{
    if (!c) return fail(nullptr, ESES_EINVAL, "ctx is NULL");
    c->ran = false;
    try {
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        return run_impl(c);
    } catch (const CudaError &e) {
        return fail(c, ESES_ECUDA, std::string(e.what) + ": " + cudaGetErrorString(e.e));
    } catch (const std::bad_alloc &) {
        return fail(c, ESES_ENOMEM, "device allocation failed");
    }
}

int eses_grid(const eses_ctx *c, int64_t dims[3], double origin[3])
{
    if (!c || !dims || !origin) return fail(nullptr, ESES_EINVAL, "NULL argument");
    for (int a = 0; a < 3; ++a) {
        dims[a] = c->dims[a];
        origin[a] = c->lo[a];
    }
    return ESES_OK;
}

int eses_labels(const eses_ctx *cc, int8_t *out)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!c || !out) return fail(c, ESES_EINVAL, "NULL argument");
    if (!c->ran) return fail(c, ESES_ESTATE, "no results: call eses_run first");
    size_t n = (size_t)(c->dims[0] * c->dims[1] * c->dims[2]);
    if (cudaMemcpyAsync(out, c->labels.p, n, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        return fail(c, ESES_ECUDA, "label copy failed");
    return ESES_OK;
}

int eses_labels_device(const eses_ctx *cc, const int8_t **dptr)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!c || !dptr) return fail(c, ESES_EINVAL, "NULL argument");
    if (!c->ran) return fail(c, ESES_ESTATE, "no results: call eses_run first");
    *dptr = (const int8_t *)c->labels.p;
    return ESES_OK;
}

int eses_num_intersections(const eses_ctx *cc, int axis, int64_t *n)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!c || !n || axis < 0 || axis > 2) return fail(c, ESES_EINVAL, "bad argument");
    if (!c->ran) return fail(c, ESES_ESTATE, "no results: call eses_run first");
    *n = c->n_edges[axis];
    return ESES_OK;
}

int eses_intersections(const eses_ctx *cc, int axis, int64_t *lower_idx, double *tau, double *normal, float *tau32,
                       float *normal32)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!c || axis < 0 || axis > 2) return fail(c, ESES_EINVAL, "bad argument");
    if (!c->ran) return fail(c, ESES_ESTATE, "no results: call eses_run first");
    size_t ne = (size_t)c->n_edges[axis];
    if (ne == 0) return ESES_OK;
    cudaStream_t st = c->stream;
    bool ok = true;
    if (lower_idx) ok &= cudaMemcpyAsync(lower_idx, c->out_idx[axis].p, ne * 8, cudaMemcpyDeviceToHost, st) == cudaSuccess;
    if (tau) ok &= cudaMemcpyAsync(tau, c->out_tau[axis].p, ne * 8, cudaMemcpyDeviceToHost, st) == cudaSuccess;
    if (normal) ok &= cudaMemcpyAsync(normal, c->out_nrm[axis].p, ne * 24, cudaMemcpyDeviceToHost, st) == cudaSuccess;
    if (tau32) ok &= cudaMemcpyAsync(tau32, c->out_tau32[axis].p, ne * 4, cudaMemcpyDeviceToHost, st) == cudaSuccess;
    if (normal32)
        ok &= cudaMemcpyAsync(normal32, c->out_nrm32[axis].p, ne * 12, cudaMemcpyDeviceToHost, st) == cudaSuccess;
    ok &= cudaStreamSynchronize(st) == cudaSuccess;
    if (!ok) return fail(c, ESES_ECUDA, "intersection copy failed");
    return ESES_OK;
}

int eses_intersections_device(const eses_ctx *cc, int axis, const int64_t **lower_idx, const double **tau,
                              const double **normal, const float **tau32, const float **normal32)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!c || axis < 0 || axis > 2) return fail(c, ESES_EINVAL, "bad argument");
    if (!c->ran) return fail(c, ESES_ESTATE, "no results: call eses_run first");
    if (lower_idx) *lower_idx = (const int64_t *)c->out_idx[axis].p;
    if (tau) *tau = (const double *)c->out_tau[axis].p;
    if (normal) *normal = (const double *)c->out_nrm[axis].p;
    if (tau32) *tau32 = (const float *)c->out_tau32[axis].p;
    if (normal32) *normal32 = (const float *)c->out_nrm32[axis].p;
    return ESES_OK;
}

int eses_area_volume(const eses_ctx *cc, double *area, double *volume)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!c || !area || !volume) return fail(c, ESES_EINVAL, "NULL argument");
    if (!c->ran) return fail(c, ESES_ESTATE, "no results: call eses_run first");
    *area = c->area;
    *volume = c->volume;
    return ESES_OK;
}

int eses_stats(const eses_ctx *cc, int64_t *out, int n)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!c || !out || n < 0) return fail(c, ESES_EINVAL, "bad argument");
    for (int k = 0; k < n && k < NSTAT; ++k) out[k] = c->stats[k];
    return ESES_OK;
}

int eses_root_failures(const eses_ctx *cc, int64_t *records, int max_records, int *n_out)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!c || !n_out || max_records < 0 || (max_records > 0 && !records)) return fail(c, ESES_EINVAL, "bad argument");
    if (!c->ran) return fail(c, ESES_ESTATE, "no results: call eses_run first");
    int nf = (int)c->stats[8];
    int n = std::min(std::min(nf, FAIL_LOG), max_records);
    *n_out = n;
    if (n > 0 &&
        cudaMemcpy(records, c->fail_log.p, sizeof(int64_t) * FAIL_REC * n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(c, ESES_ECUDA, "failure log copy failed");
    return ESES_OK;
}

int eses_patch_counts(const eses_ctx *cc, int64_t *n_pairs, int64_t *n_free_pairs, int64_t *n_vertices)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!c || !n_pairs || !n_free_pairs || !n_vertices) return fail(c, ESES_EINVAL, "NULL argument");
    if (!c->ran) return fail(c, ESES_ESTATE, "no results: call eses_run first");
    const int np = c->M.n_pairs;
    std::vector<uint8_t> fr((size_t)std::max(np, 1));
    if (np > 0 && cudaMemcpy(fr.data(), c->pair_free.p, np, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(c, ESES_ECUDA, "copy failed");
    long long nf = 0;
    for (int p = 0; p < np; ++p) nf += fr[p] ? 1 : 0;
    *n_pairs = np;
    *n_free_pairs = nf;
    *n_vertices = c->M.n_verts;
    c->stats[4] = nf;
    return ESES_OK;
}

int eses_patch_data(const eses_ctx *cc, int32_t *pair_atoms, uint8_t *pair_free, double *pair_circle,
                    double *vertices)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!c) return fail(c, ESES_EINVAL, "NULL argument");
    if (!c->ran) return fail(c, ESES_ESTATE, "no results: call eses_run first");
    const int np = c->M.n_pairs, nv = c->M.n_verts, n = c->M.n_atoms;
    std::vector<int> orig((size_t)n);
    std::vector<int2> ij((size_t)std::max(np, 1));
    std::vector<double4> po((size_t)std::max(np, 1)), pu((size_t)std::max(np, 1)), vq((size_t)std::max(nv, 1));
    bool ok = cudaMemcpy(orig.data(), c->atom_orig.p, sizeof(int) * n, cudaMemcpyDeviceToHost) == cudaSuccess;
    if (np > 0) {
        ok &= cudaMemcpy(ij.data(), c->pair_ij.p, sizeof(int2) * np, cudaMemcpyDeviceToHost) == cudaSuccess;
        ok &= cudaMemcpy(po.data(), c->pair_o.p, sizeof(double4) * np, cudaMemcpyDeviceToHost) == cudaSuccess;
        ok &= cudaMemcpy(pu.data(), c->pair_u.p, sizeof(double4) * np, cudaMemcpyDeviceToHost) == cudaSuccess;
        if (pair_free) ok &= cudaMemcpy(pair_free, c->pair_free.p, np, cudaMemcpyDeviceToHost) == cudaSuccess;
    }
    if (nv > 0) ok &= cudaMemcpy(vq.data(), c->vert.p, sizeof(double4) * nv, cudaMemcpyDeviceToHost) == cudaSuccess;
    if (!ok) return fail(c, ESES_ECUDA, "patch copy failed");
    for (int p = 0; p < np; ++p) {
        if (pair_atoms) {
            pair_atoms[2 * p] = orig[ij[p].x];
            pair_atoms[2 * p + 1] = orig[ij[p].y];
        }
        if (pair_circle) {
            double *o = pair_circle + 7 * p;
            o[0] = po[p].x; o[1] = po[p].y; o[2] = po[p].z;
            o[3] = pu[p].x; o[4] = pu[p].y; o[5] = pu[p].z;
            o[6] = po[p].w;
        }
    }
    if (vertices)
        for (int v = 0; v < nv; ++v) {
            vertices[3 * v] = vq[v].x;
            vertices[3 * v + 1] = vq[v].y;
            vertices[3 * v + 2] = vq[v].z;
        }
    return ESES_OK;
}

int eses_stage_times(const eses_ctx *cc, double *ms, int n)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!c || !ms || n < 0) return fail(c, ESES_EINVAL, "bad argument");
    if (!c->profile) return fail(c, ESES_ESTATE, "stage timing is off (ESES_OPT_PROFILE)");
    if (!c->ran) return fail(c, ESES_ESTATE, "no results: call eses_run first");
    for (int k = 0; k < n && k < NSTAGE; ++k) ms[k] = c->stage_ms[k];
    return ESES_OK;
}

const char *eses_last_error(const eses_ctx *c)
{
    if (!c) return g_create_error.c_str();
    return c->err.c_str();
}

void eses_destroy(eses_ctx *c)
{
    if (!c) return;
    DBuf *bufs[] = {&c->xyz, &c->rad, &c->cell_id, &c->cell_count, &c->cell_start, &c->cursor, &c->atom_orig,
                    &c->atom, &c->nb_count, &c->nb_start, &c->nb_list, &c->circle_count, &c->contained, &c->face,
                    &c->pair_count, &c->pair_start, &c->pair_o, &c->pair_u, &c->pair_ij, &c->pair_free,
                    &c->vert_count, &c->vert_start, &c->vert, &c->pbin_count, &c->pbin_start, &c->pbin_cursor,
                    &c->pbin_cell, &c->pbin_list, &c->vbin_count, &c->vbin_start, &c->vbin_cursor, &c->vbin_cell,
                    &c->vbin_list, &c->labels, &c->tile_band, &c->tile_edges, &c->edge_start, &c->tile_inside,
                    &c->tile_area, &c->tile_vol, &c->scan_tmp, &c->misc, &c->fail_log,
                    &c->atom_hi, &c->atom_lo, &c->pair_hi, &c->pair_lo, &c->pair_u32, &c->vert_hi, &c->vert_lo};
    if (c->own_stream) cudaStreamSynchronize(c->own_stream);
    for (DBuf *b : bufs) free_buf(*b);
    for (int a = 0; a < 3; ++a) {
        free_buf(c->out_idx[a]);
        free_buf(c->out_tau[a]);
        free_buf(c->out_nrm[a]);
        free_buf(c->out_tau32[a]);
        free_buf(c->out_nrm32[a]);
        free_buf(c->out_code[a]);
    }
    for (int k = 0; k <= NSTAGE; ++k)
        if (c->ev[k]) cudaEventDestroy(c->ev[k]);
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    delete c;
}

}  // extern "C"
