// eses_api.cu -- the C ABI (include/eses.h) and the host orchestration of one
// run over a batch of molecules (one molecule is a batch of one):
// cell binning -> neighbours -> circle pairs -> free arcs and triple points ->
// patch bins -> classification (+ FP64 band) -> crossing edges -> roots ->
// area/volume.  Every step runs on the device over all molecules at once:
// the model lists are built in one pass (each molecule keeps its own cells),
// and the tile kernels are persistent, taking tiles of every molecule from a
// device work queue.
//
// The first run of a context plans it: the host reads four list totals to
// size the buffers.  With ESES_OPT_GRAPH the next run captures the whole
// device path, with those sizes, in one CUDA graph, and every later run
// replays it (the inputs of a context never change, so neither do the sizes).
// eses_autotune times the persistent kernels' launch shapes on the context's
// own workload and keeps the fastest.
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

static_assert(MLP_NPARAM == ESES_MLP_NPARAM, "proposer parameter count");

// stages timed with CUDA events when ESES_OPT_PROFILE is set
enum { NSTAT = 20 };
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

struct CaptureGrow {};  // a buffer would have to grow during graph capture

thread_local bool g_capturing = false;
// allocation-failure injection (ESES_OPT_FAIL_ALLOC): the calling context's
// countdown while one of its entry points runs; the allocation that brings it
// to zero fails before cudaMalloc is called
thread_local long long *g_fail_countdown = nullptr;

template <class T>
T *ensure(DBuf &b, size_t count)
{
    size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    if (b.cap < bytes) {
        if (g_capturing) throw CaptureGrow{};
        if (b.p) cudaFree(b.p);
        b.p = nullptr;
        b.cap = 0;
        size_t want = bytes + bytes / 4;
        if (g_fail_countdown && *g_fail_countdown > 0 && --*g_fail_countdown == 0) throw std::bad_alloc();
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

struct MolInfo {
    long long atom0 = 0, n_atoms = 0;  // range in the batch input
    double lo[3] = {0, 0, 0};
    long long dims[3] = {0, 0, 0};
    double rmax = 0;
    double amin[3] = {0, 0, 0}, amax[3] = {0, 0, 0};
};

// launch shape of a persistent tile kernel
struct Shape {
    int ctas_per_sm = 0;  // 0: the occupancy limit
    int tiles_per_pop = 4;
    int threads = 0;      // root solve: threads per block of the per-candidate root kernels (0: 256)
};

}  // namespace

struct eses_ctx {
    int device = 0;
    int n_sm = 1;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    bool sync = true;
    int precision = ESES_PREC_FP32_FILTERED;
    int block_pts = 64;
    int n_mol = 1;
    long long n_atoms = 0;  // all molecules, coincident repeats dropped
    std::vector<int64_t> kept;  // input index of every atom of the model
    std::vector<int64_t> in_off;  // first input index of every molecule (n_mol + 1)
    double rp = 0, h = 0, margin = 0;
    double rmax = 0, Rmax = 0;
    std::vector<MolInfo> mol;
    std::vector<Grid> grids;
    std::vector<CellGrid> cgs;
    std::vector<long long> tile_off;
    long long n_tiles = 0, n_points = 0, ncell = 0;
    Model M{};
    Batch B{};
    // device buffers
    DBuf xyz, rad, in_mol, grid_d, cg_d, tile_off_d, atom_mol, vert_mol, medge, term, queue;
    DBuf cell_id, cell_count, cell_start, cursor, atom_orig, atom;
    DBuf nb_count, nb_start, nb_list, circle_count, contained, face;
    DBuf pair_count, pair_start, pair_o, pair_u, pair_ij, pair_free;
    DBuf vert_count, vert_start, vert, vert_atoms;
    DBuf pbin_count, pbin_start, pbin_cursor, pbin_cell, pbin_list;
    DBuf vbin_count, vbin_start, vbin_cursor, vbin_cell, vbin_list;
    DBuf labels, tile_band, tile_edges, edge_start, tile_inside;
    DBuf out_idx[3], out_tau[3], out_nrm[3], out_tau32[3], out_nrm32[3], out_code[3];
    DBuf scan_tmp, misc, av, counts, red_d, red_i;  // misc: err, n_fail
    DBuf fail_log;
    DBuf ovf, big;  // tiles that overflow the shared-memory staging, and the global-memory tier's scratch
    // phased root solve: edge records, candidates, their roots, staged tiles (slabs), counters, hard edges
    DBuf r_einfo, r_ecnt, r_csph, r_ctor, r_nsph, r_ntor, r_rsph, r_rtor, r_slab, r_ctr, r_hard, r_jobs;
    long long cap_sph = 0, cap_tor = 0, cap_slab = 0, cap_jobs = 0;  // planned capacities
    DBuf atom_hi, atom_lo, pair_hi, pair_lo, pair_u32, vert_hi, vert_lo;
    // plan: list sizes of the first run (the inputs never change)
    bool planned = false;
    int plan_precision = -1;
    int n_nb = 0, n_pairs = 0, n_verts = 0;
    long long n_edges[3] = {0, 0, 0};
    // results
    bool ran = false;
    std::vector<long long> medge_h;  // 3 * (n_mol + 1)
    std::vector<double> av_h;        // 2 per molecule
    std::vector<long long> cnt_h;    // 2 per molecule
    long long stats[NSTAT] = {0};
    std::string err;
    // launch shapes (eses_autotune, ESES_OPT_*)
    Shape cls, edge;
    bool use_queue = true;
    // exterior-only surface (ESES_OPT_EXTERIOR)
    bool exterior = false;
    DBuf ext, ext_open, ext_misc;
    // triangle mesh of the last run (eses_mesh_count / eses_mesh)
    DBuf mesh_mask, mesh_tile, mesh_off, mesh_keys, mesh_xyz, mesh_err;
    long long n_tri = -1;  // -1: not made for the current results
    long long n_cavity = 0;
    int ext_sweeps = 0;
    // learned tile proposer
    int proposer = 0;  // ESES_PROPOSER_*
    float z_far = 0.0f;
    bool have_params = false;
    DBuf mlp_params, need, need_pos, tile_list, prop_counts, features, targets;
    // CUDA graph of the device path
    bool graph_on = false;
    cudaGraphExec_t gexec = nullptr;
    int graph_launches = 0;  // kernels in the graph
    // block selection (eses_set_blocks): blocks [sel_lo, sel_hi) of block_pts points per axis
    bool sel = false;
    long long sel_lo[3] = {0, 0, 0}, sel_hi[3] = {0, 0, 0};
    // grid given by the caller (eses_create_on_grid)
    bool grid_given = false;
    double given_lo[3] = {0, 0, 0};
    long long given_dims[3] = {0, 0, 0};
    // buried-patch pre-culling (ESES_OPT_CULL)
    bool cull = true;
    // failure injection for tests (ESES_OPT_TC_WAIT, ESES_OPT_FAIL_ALLOC)
    long long tc_wait = -1;      // polls of each tensor-core scoring wait (-1: the default limit)
    long long fail_alloc = 0;    // countdown to the device allocation that fails (0: none)
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

void drop_graph(eses_ctx *c)
{
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
}

int scan(eses_ctx *c, const int *in, int *out, long long n)
{
    int *tmp = ensure<int>(c->scan_tmp, (size_t)scan_tmp_ints(n));
    return scan_exclusive(in, out, n, tmp, c->stream);
}

// list total at start[n]: read when planning, the planned value when capturing
int list_total(eses_ctx *c, const int *start, long long n, int &planned)
{
    if (g_capturing) return planned;
    int v = 0;
    ck(cudaMemcpyAsync(&v, start + n, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "read list total");
    ck(cudaStreamSynchronize(c->stream), "synchronize");
    planned = v;
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

// Grids of Eq. 2, cell grids and the tile layout of every molecule; xyz/r on the host
int setup(eses_ctx *c, const double *xyz, const double *r, const int64_t *counts)
{
    const int nm = c->n_mol;
    c->mol.assign(nm, MolInfo());
    c->rmax = 0.0;
    long long a0 = 0;
    for (int m = 0; m < nm; ++m) {
        MolInfo &I = c->mol[m];
        I.atom0 = a0;
        I.n_atoms = counts[m];
        a0 += counts[m];
        const double *X = xyz + 3 * I.atom0;
        const double *R = r + I.atom0;
        for (int a = 0; a < 3; ++a) {
            double mn = X[a] - R[0], mx = X[a] + R[0];
            I.amin[a] = X[a];
            I.amax[a] = X[a];
            for (long long i = 1; i < I.n_atoms; ++i) {
                double v0 = X[3 * i + a] - R[i], v1 = X[3 * i + a] + R[i];
                if (v0 < mn) mn = v0;
                if (v1 > mx) mx = v1;
                I.amin[a] = std::min(I.amin[a], X[3 * i + a]);
                I.amax[a] = std::max(I.amax[a], X[3 * i + a]);
            }
            I.lo[a] = mn - c->margin;
            I.dims[a] = (long long)ceil((mx + c->margin - I.lo[a]) / c->h) + 1;
            if (c->grid_given) {  // one molecule on the caller's grid
                I.lo[a] = c->given_lo[a];
                I.dims[a] = c->given_dims[a];
            }
        }
        I.rmax = 0.0;
        for (long long i = 0; i < I.n_atoms; ++i) I.rmax = std::max(I.rmax, R[i]);
        c->rmax = std::max(c->rmax, I.rmax);
        if (I.dims[0] > (1LL << 30) || I.dims[1] > (1LL << 30) || I.dims[2] > (1LL << 30) ||
            I.dims[0] * I.dims[1] * I.dims[2] > (1LL << 40))
            return fail(c, ESES_EINVAL, "grid too large (molecule " + std::to_string(m) + ")");
    }
    c->Rmax = c->rmax + c->rp;
    Model &M = c->M;
    M.n_atoms = (int)c->n_atoms;
    M.n_mol = nm;
    M.rp = c->rp;
    M.rmax = c->rmax;
    M.Rmax = c->Rmax;
    // cubic cells of edge >= 2 R_max: overlapping expanded balls sit in adjacent cells
    M.cell = std::max(2.0 * c->Rmax, 1e-3);
    c->cgs.assign(nm, CellGrid());
    for (int it = 0; it < 200; ++it) {
        long long total = 0;
        bool ok = true;
        for (int m = 0; m < nm; ++m) {
            CellGrid &g = c->cgs[m];
            long long n = 1;
            for (int a = 0; a < 3; ++a) {
                g.clo[a] = c->mol[m].amin[a] - 1e-6;
                long long k = (long long)floor((c->mol[m].amax[a] - g.clo[a]) / M.cell) + 1;
                if (k > (1LL << 20)) ok = false;
                g.cn[a] = (int)std::min(k, 1LL << 20);
                n *= k;
            }
            g.coff = (int)std::min(total, (long long)INT32_MAX);
            total += n;
        }
        c->ncell = total;
        if (ok && total <= (1LL << 26)) break;
        M.cell *= 1.25;  // very sparse extents: coarser cells stay correct
    }
    if (c->ncell > (1LL << 26)) return fail(c, ESES_EINVAL, "cell grid too large");
    c->grids.assign(nm, Grid());
    c->tile_off.assign(nm + 1, 0);
    long long lab0 = 0;
    for (int m = 0; m < nm; ++m) {
        Grid &G = c->grids[m];
        const MolInfo &I = c->mol[m];
        for (int a = 0; a < 3; ++a) {
            G.lo[a] = I.lo[a];
            G.dims[a] = I.dims[a];
            G.own[a] = I.dims[a];
            G.full[a] = I.dims[a];
            G.toff[a] = 0;
            G.tiles[a] = (int)ceil_div_ll(I.dims[a], TILE);
        }
        G.h = c->h;
        G.n_tiles = (long long)G.tiles[0] * G.tiles[1] * G.tiles[2];
        if (G.n_tiles >= (1LL << 31)) return fail(c, ESES_EINVAL, "grid too large (2^31 tiles in one molecule)");
        G.tile0 = c->tile_off[m];
        G.lab0 = lab0;
        c->tile_off[m + 1] = c->tile_off[m] + G.n_tiles;
        lab0 += I.dims[0] * I.dims[1] * I.dims[2];
        G.rp = c->rp;
        G.halo = I.rmax + 2.0 * c->rp;
        double L = 8.0 * c->h * sqrt(3.0) + G.halo + 1.0;
        // staged FP32 coordinates carry two roundings of at most 2^-24 L each, a grid
        // point one, a difference of two of them one more: 5 * 2^-24 L per
        // coordinate, 5.2e-7 L for the vector; d0 rounds that up
        G.d0 = (float)(6e-7 * L);
        for (int k = 0; k <= TILE; ++k) G.hl[k] = (float)((double)k * c->h);
        G.ht_hi = (float)(TILE * c->h);
        G.ht_lo = (float)(TILE * c->h - (double)G.ht_hi);
    }
    c->n_tiles = c->tile_off[nm];
    c->n_points = lab0;
    return ESES_OK;
}

int create_common(const double *hxyz, const double *hr, const int64_t *counts, int n_mol, double rp, double h,
                  double margin, const double *dxyz, const double *dr, eses_ctx **out,
                  const double *grid_lo = nullptr, const int64_t *grid_dims = nullptr)
{
    if (!out) return fail(nullptr, ESES_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_mol < 1 || n_mol > (1 << 20)) return fail(nullptr, ESES_EINVAL, "n_mol must be in [1, 2^20]");
    long long total = 0;
    for (int m = 0; m < n_mol; ++m) {
        if (counts[m] < 1) return fail(nullptr, ESES_EINVAL, "every molecule needs at least one atom");
        total += counts[m];
    }
    std::string msg;
    int rc = validate(hxyz, hr, total, rp, h, margin, msg);
    if (rc) return fail(nullptr, rc, msg);
    // Coincident atoms (the same centre and radius, within one molecule) are
    // one ball: the union of balls (§1) does not change without the repeats,
    // and keeping them would let each sphere "cover" the other's surface.
    std::vector<int64_t> in_off((size_t)n_mol + 1, 0);  // first input index of every molecule
    for (int m = 0; m < n_mol; ++m) in_off[(size_t)m + 1] = in_off[(size_t)m] + counts[m];
    std::vector<int64_t> kept;  // input index of every atom the model uses
    std::vector<int64_t> kcounts(counts, counts + n_mol);
    {
        kept.reserve((size_t)total);
        long long a0 = 0;
        std::vector<int64_t> idx;
        for (int m = 0; m < n_mol; ++m) {
            idx.resize((size_t)counts[m]);
            for (long long i = 0; i < counts[m]; ++i) idx[(size_t)i] = a0 + i;
            auto key_less = [&](int64_t a, int64_t b) {
                for (int q = 0; q < 3; ++q)
                    if (hxyz[3 * a + q] != hxyz[3 * b + q]) return hxyz[3 * a + q] < hxyz[3 * b + q];
                if (hr[a] != hr[b]) return hr[a] < hr[b];
                return a < b;
            };
            std::sort(idx.begin(), idx.end(), key_less);
            std::vector<char> keep((size_t)counts[m], 1);
            for (size_t t = 1; t < idx.size(); ++t) {
                const int64_t a = idx[t - 1], b = idx[t];
                if (hxyz[3 * a] == hxyz[3 * b] && hxyz[3 * a + 1] == hxyz[3 * b + 1] &&
                    hxyz[3 * a + 2] == hxyz[3 * b + 2] && hr[a] == hr[b])
                    keep[(size_t)(b - a0)] = 0;
            }
            int64_t nk = 0;
            for (long long i = 0; i < counts[m]; ++i)
                if (keep[(size_t)i]) {
                    kept.push_back(a0 + i);
                    ++nk;
                }
            kcounts[(size_t)m] = nk;
            a0 += counts[m];
        }
    }
    const bool has_repeats = (long long)kept.size() != total;
    std::vector<double> cx, cr;
    if (has_repeats) {
        cx.resize(3 * kept.size());
        cr.resize(kept.size());
        for (size_t k = 0; k < kept.size(); ++k) {
            for (int q = 0; q < 3; ++q) cx[3 * k + q] = hxyz[3 * kept[k] + q];
            cr[k] = hr[kept[k]];
        }
        hxyz = cx.data();
        hr = cr.data();
        counts = kcounts.data();
        total = (long long)kept.size();
        dxyz = nullptr;  // upload the de-duplicated host copy
        dr = nullptr;
    }
    eses_ctx *c = new (std::nothrow) eses_ctx();
    if (!c) return fail(nullptr, ESES_ENOMEM, "host allocation failed");
    c->kept = std::move(kept);
    c->in_off = std::move(in_off);
    c->n_atoms = total;
    c->n_mol = n_mol;
    c->rp = rp;
    c->h = h;
    c->margin = margin;
    if (grid_lo) {
        c->grid_given = true;
        for (int a = 0; a < 3; ++a) {
            c->given_lo[a] = grid_lo[a];
            c->given_dims[a] = grid_dims[a];
        }
    }
    try {
        ck(cudaGetDevice(&c->device), "cudaGetDevice");
        ck(cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device), "device attribute");
        classify_init();
        edges_init();
        mlp_init();
        if (mesh_init() != 0) throw CudaError{cudaErrorInvalidValue, "mesh case table"};
        ck(cudaGetLastError(), "kernel attributes");
        ck(cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking), "cudaStreamCreate");
        c->stream = c->own_stream;
        rc = setup(c, hxyz, hr, counts);
        if (rc) {
            g_create_error = c->err;
            eses_destroy(c);
            return rc;
        }
        double *x = ensure<double>(c->xyz, 3 * (size_t)total);
        double *r = ensure<double>(c->rad, (size_t)total);
        if (dxyz) {
            ck(cudaMemcpyAsync(x, dxyz, sizeof(double) * 3 * total, cudaMemcpyDeviceToDevice, c->stream), "copy atoms");
            ck(cudaMemcpyAsync(r, dr, sizeof(double) * total, cudaMemcpyDeviceToDevice, c->stream), "copy radii");
        } else {
            ck(cudaMemcpyAsync(x, hxyz, sizeof(double) * 3 * total, cudaMemcpyHostToDevice, c->stream), "copy atoms");
            ck(cudaMemcpyAsync(r, hr, sizeof(double) * total, cudaMemcpyHostToDevice, c->stream), "copy radii");
        }
        std::vector<int> im((size_t)total);
        for (int m = 0; m < n_mol; ++m)
            for (long long i = 0; i < c->mol[m].n_atoms; ++i) im[(size_t)(c->mol[m].atom0 + i)] = m;
        int *imd = ensure<int>(c->in_mol, (size_t)total);
        Grid *gd = ensure<Grid>(c->grid_d, (size_t)n_mol);
        CellGrid *cgd = ensure<CellGrid>(c->cg_d, (size_t)n_mol);
        long long *tod = ensure<long long>(c->tile_off_d, (size_t)n_mol + 1);
        ck(cudaMemcpyAsync(imd, im.data(), sizeof(int) * total, cudaMemcpyHostToDevice, c->stream), "copy");
        ck(cudaMemcpyAsync(gd, c->grids.data(), sizeof(Grid) * n_mol, cudaMemcpyHostToDevice, c->stream), "copy");
        ck(cudaMemcpyAsync(cgd, c->cgs.data(), sizeof(CellGrid) * n_mol, cudaMemcpyHostToDevice, c->stream), "copy");
        ck(cudaMemcpyAsync(tod, c->tile_off.data(), sizeof(long long) * (n_mol + 1), cudaMemcpyHostToDevice, c->stream),
           "copy");
        ck(cudaStreamSynchronize(c->stream), "synchronize");
        c->M.cg = cgd;
        c->B.n_mol = n_mol;
        c->B.n_tiles = c->n_tiles;
        c->B.grid = gd;
        c->B.tile_off = tod;
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
    if (!c->profile) return;
    // under capture an external record becomes a node of the graph, replayed every launch
    if (g_capturing) ck(cudaEventRecordWithFlags(c->ev[k], c->stream, cudaEventRecordExternal), "cudaEventRecord");
    else ck(cudaEventRecord(c->ev[k], c->stream), "cudaEventRecord");
}

int grid_of(const eses_ctx *c, const Shape &s, int max_per_sm)
{
    int k = s.ctas_per_sm > 0 ? std::min(s.ctas_per_sm, max_per_sm) : max_per_sm;
    long long g = (long long)std::max(k, 1) * c->n_sm;
    long long need = ceil_div_ll(std::max(c->n_tiles, 1LL), std::max(s.tiles_per_pop, 1));
    return (int)std::max(1LL, std::min(g, need));
}

TileSched sched_of(eses_ctx *c, const Shape &s, int which)
{
    TileSched q;
    q.head = c->use_queue ? (unsigned long long *)c->queue.p + which : nullptr;
    q.per = std::max(s.tiles_per_pop, 1);
    q.list = nullptr;
    q.list_n = nullptr;
    return q;
}

// Buffers of the phased root solve.  Planning: capacities from a first
// estimate per crossing edge (grown by run_device when the staging pass needs
// more); capturing: the planned capacities.
constexpr long long SLAB_CAP_MAX = 16LL * 2147483647LL;  // slab offsets are 16-byte units in an int
RootWork root_work(eses_ctx *c, long long ne_all)
{
    const long long ne = std::max(ne_all, 1LL);
    if (!g_capturing) {
        c->cap_sph = std::max(c->cap_sph, 3 * ne + 1024);
        c->cap_tor = std::max(c->cap_tor, 4 * ne + 1024);
        c->cap_slab = std::max(c->cap_slab, 96 * ne + (1LL << 20));
        c->cap_slab = std::min(c->cap_slab, SLAB_CAP_MAX);
        c->cap_jobs = std::max(c->cap_jobs, c->cap_tor / 4 + 4096);
    }
    RootWork W;
    W.einfo = ensure<int4>(c->r_einfo, (size_t)ne);
    W.ecnt = ensure<int>(c->r_ecnt, (size_t)ne);
    W.hard = ensure<int>(c->r_hard, (size_t)ne);
    W.csph = ensure<int2>(c->r_csph, (size_t)c->cap_sph);
    W.nsph = ensure<uint8_t>(c->r_nsph, (size_t)c->cap_sph);
    W.rsph = ensure<RootRec>(c->r_rsph, 2 * (size_t)c->cap_sph);
    W.ctor = ensure<int2>(c->r_ctor, (size_t)c->cap_tor);
    W.ntor = ensure<uint8_t>(c->r_ntor, (size_t)c->cap_tor);
    W.rtor = ensure<RootRec>(c->r_rtor, 4 * (size_t)c->cap_tor);
    W.slab = ensure<unsigned char>(c->r_slab, (size_t)c->cap_slab);
    W.ctr = ensure<unsigned long long>(c->r_ctr, 8);
    W.jobs = ensure<int2>(c->r_jobs, (size_t)c->cap_jobs);
    W.cap_slab = c->cap_slab;
    W.cap_sph = c->cap_sph;
    W.cap_tor = c->cap_tor;
    W.cap_jobs = c->cap_jobs;
    W.n_edges = ne_all;
    return W;
}

// The device path of one run.  Planning (not capturing): reads list totals
// and sizes every buffer; capturing: uses the planned sizes and touches no
// host memory.  Returns the number of kernels launched.
int run_device(eses_ctx *c)
{
    cudaStream_t st = c->stream;
    int nl = 0;
    Model &M = c->M;
    Batch &B = c->B;
    const int n = M.n_atoms;
    const long long ncell = c->ncell;
    const long long nt = c->n_tiles;
    int *misc = ensure<int>(c->misc, 64);
    int *d_err = misc, *d_fail = misc + 1;
    unsigned long long *d_tests = reinterpret_cast<unsigned long long *>(misc + 8);  // classification atom tests
    unsigned long long *queue = ensure<unsigned long long>(c->queue, 4);
    ck(cudaMemsetAsync(misc, 0, 64 * sizeof(int), st), "memset");
    ck(cudaMemsetAsync(queue, 0, 4 * sizeof(unsigned long long), st), "memset");

    mark(c, ST_BIN);
    // 1. cell binning (counting sort, deterministic within a cell)
    int *cell_id = ensure<int>(c->cell_id, n);
    int *cell_count = ensure<int>(c->cell_count, ncell);
    int *cell_start = ensure<int>(c->cell_start, ncell + 1);
    int *cursor = ensure<int>(c->cursor, ncell);
    int *orig = ensure<int>(c->atom_orig, n);
    double4 *atom = ensure<double4>(c->atom, n);
    int *atom_mol = ensure<int>(c->atom_mol, n);
    ck(cudaMemsetAsync(cell_count, 0, sizeof(int) * ncell, st), "memset");
    ck(cudaMemsetAsync(cursor, 0, sizeof(int) * ncell, st), "memset");
    nl += launch_cell_count((const double *)c->xyz.p, (const int *)c->in_mol.p, n, M.cg, M.cell, cell_id, cell_count,
                            st);
    nl += scan(c, cell_count, cell_start, ncell);
    nl += launch_cell_scatter(nullptr, nullptr, n, cell_id, cell_start, cursor, orig, st);
    nl += launch_cell_finish((const double *)c->xyz.p, (const double *)c->rad.p, (const int *)c->in_mol.p, (int)ncell,
                             cell_start, orig, atom, atom_mol, st);
    M.atom = atom;
    M.atom_orig = orig;
    M.atom_mol = atom_mol;
    M.cell_start = cell_start;
    float4 *ahi = ensure<float4>(c->atom_hi, n), *alo = ensure<float4>(c->atom_lo, n);
    nl += launch_model_f32(M, 0, B.grid, ahi, alo, nullptr, st);
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
    const int n_nb = list_total(c, nb_start, n, c->n_nb);
    int *nb_list = ensure<int>(c->nb_list, std::max(n_nb, 1));
    M.nb_start = nb_start;
    M.nb_list = nb_list;
    nl += launch_nb_fill(M, nb_list, st);

    // 3. circle pairs
    int *pair_count = ensure<int>(c->pair_count, n);
    int *pair_start = ensure<int>(c->pair_start, n + 1);
    nl += launch_pair_count(M, pair_count, st);
    nl += scan(c, pair_count, pair_start, n);
    const int np = list_total(c, pair_start, n, c->n_pairs);
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
    nl += launch_model_f32(M, 1, B.grid, phi, plo, pu32, st);
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
    const int nv = list_total(c, vert_start, np, c->n_verts);
    M.n_verts = nv;
    double4 *vert = ensure<double4>(c->vert, std::max(nv, 1));
    int *vert_mol = ensure<int>(c->vert_mol, std::max(nv, 1));
    int4 *vert_atoms = ensure<int4>(c->vert_atoms, std::max(nv, 1));
    nl += launch_arcs_emit(M, vert_start, vert, vert_mol, vert_atoms, st);
    M.vert = vert;
    M.vert_mol = vert_mol;

    if (n >= (1 << 27) || np >= (1 << 27) || nv >= (1 << 27))
        throw std::string("more than 2^27 atoms, circle pairs or triple points");
    // 5. free faces
    uint8_t *face = ensure<uint8_t>(c->face, n);
    nl += launch_faces(M, circle_count, contained, face, st);
    if (!c->cull) ck(cudaMemsetAsync(face, 1, n, st), "memset");  // every face a witness carrier
    M.atom_face = face;

    // 6. patch bins
    int *pcnt = ensure<int>(c->pbin_count, ncell);
    int *pstart = ensure<int>(c->pbin_start, ncell + 1);
    int *pcur = ensure<int>(c->pbin_cursor, ncell);
    int *pcell = ensure<int>(c->pbin_cell, std::max(np, 1));
    int *plist = ensure<int>(c->pbin_list, std::max(np, 1));
    ck(cudaMemsetAsync(pcnt, 0, sizeof(int) * ncell, st), "memset");
    ck(cudaMemsetAsync(pcur, 0, sizeof(int) * ncell, st), "memset");
    nl += launch_bin_count(M, 0, c->cull, pcnt, pcell, st);
    nl += scan(c, pcnt, pstart, ncell);
    nl += launch_bin_scatter(M, 0, pcell, pstart, pcur, plist, st);
    int *vcnt = ensure<int>(c->vbin_count, ncell);
    int *vstart = ensure<int>(c->vbin_start, ncell + 1);
    int *vcur = ensure<int>(c->vbin_cursor, ncell);
    int *vcell = ensure<int>(c->vbin_cell, std::max(nv, 1));
    int *vlist = ensure<int>(c->vbin_list, std::max(nv, 1));
    ck(cudaMemsetAsync(vcnt, 0, sizeof(int) * ncell, st), "memset");
    ck(cudaMemsetAsync(vcur, 0, sizeof(int) * ncell, st), "memset");
    nl += launch_bin_count(M, 1, true, vcnt, vcell, st);
    nl += scan(c, vcnt, vstart, ncell);
    nl += launch_bin_scatter(M, 1, vcell, vstart, vcur, vlist, st);
    M.pcell_start = pstart;
    M.pcell_list = plist;
    M.vcell_start = vstart;
    M.vcell_list = vlist;
    float4 *vhi = ensure<float4>(c->vert_hi, std::max(nv, 1)), *vlo = ensure<float4>(c->vert_lo, std::max(nv, 1));
    nl += launch_model_f32(M, 2, B.grid, vhi, vlo, nullptr, st);
    M.vert_hi = vhi;
    M.vert_lo = vlo;

    // 7. classification (+ FP64 band re-evaluation), persistent over all tiles;
    //    with the proposer, certified far tiles are filled first and only the
    //    others are classified
    int8_t *labels = ensure<int8_t>(c->labels, c->n_points);
    int *tile_band = ensure<int>(c->tile_band, nt);
    int *prop_counts = ensure<int>(c->prop_counts, 4);
    ck(cudaMemsetAsync(prop_counts, 0, 4 * sizeof(int), st), "memset");
    mark(c, ST_CLASSIFY);
    TileSched cq = sched_of(c, c->cls, 0);
    if (c->proposer != ESES_PROPOSER_OFF) {
        int *need = ensure<int>(c->need, nt);
        int *pos = ensure<int>(c->need_pos, nt + 1);
        int *list = ensure<int>(c->tile_list, nt);
        nl += launch_propose(M, B, c->proposer, (const float *)c->mlp_params.p, c->z_far, labels,
                             c->precision == ESES_PREC_FP64 ? nullptr : tile_band, need, prop_counts, d_err,
                             c->tc_wait, st);
        nl += scan(c, need, pos, nt);
        nl += launch_compact(nt, need, pos, list, st);
        cq.list = list;
        cq.list_n = pos + nt;
    }
    int *ovf = ensure<int>(c->ovf, (size_t)nt + 2);
    ck(cudaMemsetAsync(ovf, 0, sizeof(int), st), "memset");
    unsigned char *big = ensure<unsigned char>(c->big, std::max(classify_big_bytes(), edges_big_bytes()));
    nl += launch_classify(M, B, c->precision, cq, grid_of(c, c->cls, classify_ctas_per_sm(c->precision)), labels,
                          c->precision == ESES_PREC_FP64 ? nullptr : tile_band, d_err, ovf, big, d_tests, st);
    mark(c, ST_BAND);
    if (c->precision != ESES_PREC_FP64) nl += launch_band(M, B, labels, tile_band, d_err, ovf, big, st);
    c->n_cavity = 0;
    c->ext_sweeps = 0;
    if (c->exterior) {  // cavities filled: sweeps until one reaches nothing new (never under capture)
        if (g_capturing) throw std::string("the exterior-only surface is not captured in a graph");
        uint8_t *ext = ensure<uint8_t>(c->ext, c->n_points);
        uint8_t *open = ensure<uint8_t>(c->ext_open, nt);
        // em[0..1]: four ints (three sweep flags, the sweep count), em[2]: filled points
        unsigned long long *em = ensure<unsigned long long>(c->ext_misc, 3);
        int *flags = reinterpret_cast<int *>(em);
        ck(cudaMemsetAsync(em, 0, 3 * sizeof(unsigned long long), st), "memset");
        nl += launch_ext_init(B, labels, ext, open, st);
        // a sweep reaches at least one more tile, or nothing: at most nt + 1 sweeps
        const int coop = launch_ext_fill(B, ext, open, flags, nt + 1, st);
        if (coop < 0) throw CudaError{cudaGetLastError(), "cooperative launch"};
        if (coop == 1) {  // one launch for every sweep
            ++nl;
        } else {  // no cooperative launch on this device: one launch per sweep, driven from the host
            const int sweep_grid = (int)std::min<long long>(std::max<long long>(nt, 1), 8LL * c->n_sm);
            for (long long it = 0; it <= nt; ++it) {
                ck(cudaMemsetAsync(flags, 0, sizeof(int), st), "memset");
                nl += launch_ext_sweep(B, ext, open, flags, sweep_grid, st);
                int changed = 0;
                ck(cudaMemcpyAsync(&changed, flags, sizeof(changed), cudaMemcpyDeviceToHost, st), "read");
                ck(cudaStreamSynchronize(st), "synchronize");
                ++c->ext_sweeps;
                if (!changed) break;
            }
        }
        nl += launch_ext_apply(B, labels, ext, em + 2, st);
        unsigned long long misc[3] = {0, 0, 0};
        ck(cudaMemcpyAsync(misc, em, sizeof(misc), cudaMemcpyDeviceToHost, st), "read");
        ck(cudaStreamSynchronize(st), "synchronize");
        if (coop == 1) c->ext_sweeps = reinterpret_cast<const int *>(misc)[3];
        c->n_cavity = (long long)misc[2];
    }

    // 8. crossing edges, roots, area and volume
    int *tile_edges = ensure<int>(c->tile_edges, 3 * nt);
    int *edge_start = ensure<int>(c->edge_start, 3 * nt + 1);
    int *tile_inside = ensure<int>(c->tile_inside, 4 * nt);
    long long *medge = ensure<long long>(c->medge, 3 * ((size_t)c->n_mol + 1));
    mark(c, ST_EDGE_COUNT);
    nl += launch_edge_count(B, labels, tile_edges, tile_inside, st);
    nl += scan(c, tile_edges, edge_start, 3 * nt);
    nl += launch_mol_edges(B, edge_start, medge, st);
    if (!g_capturing) {
        std::vector<int> tot(4);
        for (int a = 0; a < 3; ++a)
            ck(cudaMemcpyAsync(&tot[a], edge_start + a * nt, sizeof(int), cudaMemcpyDeviceToHost, st), "read");
        ck(cudaMemcpyAsync(&tot[3], edge_start + 3 * nt, sizeof(int), cudaMemcpyDeviceToHost, st), "read");
        ck(cudaStreamSynchronize(st), "synchronize");
        for (int a = 0; a < 3; ++a) c->n_edges[a] = (long long)tot[a + 1] - tot[a];
    }
    EdgeOut eo;
    for (int a = 0; a < 3; ++a) {
        const long long ne = c->n_edges[a];
        eo.idx[a] = ensure<long long>(c->out_idx[a], std::max(ne, 1LL));
        eo.tau[a] = ensure<double>(c->out_tau[a], std::max(ne, 1LL));
        eo.nrm[a] = ensure<double>(c->out_nrm[a], 3 * std::max(ne, 1LL));
        eo.tau32[a] = ensure<float>(c->out_tau32[a], std::max(ne, 1LL));
        eo.nrm32[a] = ensure<float>(c->out_nrm32[a], 3 * std::max(ne, 1LL));
        eo.code[a] = ensure<int2>(c->out_code[a], std::max(ne, 1LL));
    }
    const long long ne_all = c->n_edges[0] + c->n_edges[1] + c->n_edges[2];
    double2 *term = ensure<double2>(c->term, std::max(ne_all, 1LL));
    double *av = ensure<double>(c->av, 2 * (size_t)c->n_mol);
    long long *cnt = ensure<long long>(c->counts, 2 * (size_t)c->n_mol);
    long long *fail_log = ensure<long long>(c->fail_log, FAIL_LOG * FAIL_REC);
    mark(c, ST_EDGE_SOLVE);
    RootWork W = root_work(c, ne_all);
    const TileSched eq = sched_of(c, c->edge, 1);
    const int eg = grid_of(c, c->edge, edge_ctas_per_sm(c->precision));
    nl += launch_edge_stage(M, B, c->precision, eq, eg, labels, edge_start, eo, d_err, ovf, big, W, st);
    if (!g_capturing) {  // planning: the totals the staging pass needed; a full buffer is grown and the pass rerun
        unsigned long long need[3] = {0, 0, 0};
        int ov[2] = {0, 0};
        ck(cudaMemcpyAsync(need, W.ctr, sizeof(need), cudaMemcpyDeviceToHost, st), "read");
        ck(cudaMemcpyAsync(ov, ovf, sizeof(ov), cudaMemcpyDeviceToHost, st), "read");
        ck(cudaStreamSynchronize(st), "synchronize");
        if ((long long)need[0] > W.cap_slab || (long long)need[1] > W.cap_sph || (long long)need[2] > W.cap_tor) {
            c->cap_slab = std::max(c->cap_slab, (long long)(need[0] + need[0] / 8));
            c->cap_sph = std::max(c->cap_sph, (long long)(need[1] + need[1] / 8));
            c->cap_tor = std::max(c->cap_tor, (long long)(need[2] + need[2] / 8));
            W = root_work(c, ne_all);
            // the tiles the first pass gave the global-memory tier are counted again
            const int run_total = ov[0] - ov[1];
            ck(cudaMemcpyAsync(ovf, &run_total, sizeof(int), cudaMemcpyHostToDevice, st), "write");
            nl += launch_edge_stage(M, B, c->precision, eq, eg, labels, edge_start, eo, d_err, ovf, big, W, st);
        }
    }
    nl += launch_edge_roots(M, B, c->precision, c->edge.threads, eo, edge_start, ne_all, d_fail, d_err, fail_log, W,
                            st);
    if (!g_capturing) {  // planning: a full FP64 job list is grown and the root launches rerun
        unsigned long long jobs = 0;
        ck(cudaMemcpyAsync(&jobs, W.ctr + 4, sizeof(jobs), cudaMemcpyDeviceToHost, st), "read");
        ck(cudaStreamSynchronize(st), "synchronize");
        if ((long long)jobs > W.cap_jobs) {
            c->cap_jobs = (long long)(jobs + jobs / 8);
            W = root_work(c, ne_all);
            nl += launch_edge_roots(M, B, c->precision, c->edge.threads, eo, edge_start, ne_all, d_fail, d_err,
                                    fail_log, W, st);
        }
    }
    mark(c, ST_EDGE_POLISH);
    nl += launch_edge_polish(M, B, eo, ne_all, medge, term, st);
    mark(c, ST_REDUCE);
    double *part_d = ensure<double>(c->red_d, (size_t)reduce_scratch(c->n_mol));
    long long *part_i = ensure<long long>(c->red_i, (size_t)reduce_scratch(c->n_mol));
    nl += launch_reduce(B, term, medge, tile_inside, part_d, part_i, av, cnt, st);
    mark(c, NSTAGE);
    ck(cudaGetLastError(), "kernel launch");
    return nl;
}

// results of the run just enqueued (host reads; waits for the device)
int finish(eses_ctx *c, int nl)
{
    cudaStream_t st = c->stream;
    const int nm = c->n_mol;
    int hmisc[64];
    c->medge_h.assign(3 * ((size_t)nm + 1), 0);
    c->av_h.assign(2 * (size_t)nm, 0.0);
    c->cnt_h.assign(2 * (size_t)nm, 0);
    ck(cudaMemcpyAsync(hmisc, c->misc.p, sizeof(hmisc), cudaMemcpyDeviceToHost, st), "read results");
    int hprop[4] = {0, 0, 0, 0};
    ck(cudaMemcpyAsync(hprop, c->prop_counts.p, sizeof(hprop), cudaMemcpyDeviceToHost, st), "read results");
    int hovf = 0;  // tiles the global-memory staging tier took
    ck(cudaMemcpyAsync(&hovf, c->ovf.p, sizeof(int), cudaMemcpyDeviceToHost, st), "read results");
    // root solve: slab bytes, sphere and torus candidates, hard edges, torus candidates with FP64 work
    unsigned long long rctr[5] = {0, 0, 0, 0, 0};
    if (c->r_ctr.p) ck(cudaMemcpyAsync(rctr, c->r_ctr.p, sizeof(rctr), cudaMemcpyDeviceToHost, st), "read results");
    ck(cudaMemcpyAsync(c->medge_h.data(), c->medge.p, sizeof(long long) * c->medge_h.size(), cudaMemcpyDeviceToHost, st),
       "read results");
    ck(cudaMemcpyAsync(c->av_h.data(), c->av.p, sizeof(double) * c->av_h.size(), cudaMemcpyDeviceToHost, st),
       "read results");
    ck(cudaMemcpyAsync(c->cnt_h.data(), c->counts.p, sizeof(long long) * c->cnt_h.size(), cudaMemcpyDeviceToHost, st),
       "read results");
    ck(cudaStreamSynchronize(st), "synchronize");
    if (c->profile)
        for (int k = 0; k < NSTAGE; ++k) ck(cudaEventElapsedTime(&c->stage_ms[k], c->ev[k], c->ev[k + 1]), "elapsed");
    long long inside = 0;
    for (int m = 0; m < nm; ++m) inside += c->cnt_h[2 * m];
    c->stats[0] = c->sel ? c->grids[0].own[0] * c->grids[0].own[1] * c->grids[0].own[2] : c->n_points;
    c->stats[1] = c->n_tiles;
    c->stats[2] = 0;
    c->stats[3] = c->n_pairs;
    c->stats[4] = -1;  // filled on demand by eses_patch_counts
    c->stats[5] = c->n_verts;
    c->stats[6] = 0;
    c->stats[7] = c->n_edges[0] + c->n_edges[1] + c->n_edges[2];
    c->stats[8] = hmisc[1];
    c->stats[9] = inside;
    c->stats[10] = nl;
    c->stats[11] = hprop[0];
    c->stats[12] = hprop[1];
    c->stats[13] = c->n_cavity;
    c->stats[14] = c->ext_sweeps;
    c->stats[15] = hovf;
    unsigned long long tests = 0;
    memcpy(&tests, hmisc + 8, sizeof(tests));
    c->stats[16] = (long long)tests;
    c->stats[17] = (long long)rctr[1];
    c->stats[18] = (long long)rctr[2];
    c->stats[19] = (long long)rctr[3];
    c->ran = true;
    int derr = hmisc[0];
    if ((long long)rctr[4] > c->cap_jobs) derr |= ERR_CAP_CAND;  // the FP64 job list was full (never planned so)
    if (derr & (ERR_CAP_ATOMS | ERR_CAP_PAIRS | ERR_CAP_VERTS | ERR_CAP_CAND)) {
        c->ran = false;
        return fail(c, ESES_ECAPACITY, (derr & ERR_CAP_CAND) ? "an edge had more candidate roots than its buffer holds"
                                                             : "a tile's staged list exceeded its shared-memory capacity");
    }
    if (hmisc[1] > 0)
        return fail(c, ESES_EROOT, std::to_string(hmisc[1]) + " crossing edges had no surface root");
    if (derr & ERR_TIMEOUT)
        return fail(c, ESES_ETIMEOUT, "a bounded device wait ran out (the proposer fell back to the exact path)");
    return ESES_OK;
}

int run_impl(eses_ctx *c)
{
    if (c->profile && !c->ev[0])
        for (int k = 0; k <= NSTAGE; ++k) ck(cudaEventCreate(&c->ev[k]), "cudaEventCreate");
    const bool replay = c->graph_on && !c->exterior && c->planned && c->plan_precision == c->precision;
    if (!replay) {
        drop_graph(c);
        const int nl = run_device(c);
        c->planned = true;
        c->plan_precision = c->precision;
        return finish(c, nl);
    }
    if (!c->gexec) {
        cudaGraph_t g = nullptr;
        ck(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
        g_capturing = true;
        int nl = 0;
        try {
            nl = run_device(c);
        } catch (...) {
            g_capturing = false;
            cudaStreamEndCapture(c->stream, &g);
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            throw;
        }
        g_capturing = false;
        ck(cudaStreamEndCapture(c->stream, &g), "end capture");
        cudaError_t e = cudaGraphInstantiate(&c->gexec, g, 0);
        cudaGraphDestroy(g);
        ck(e, "graph instantiate");
        c->graph_launches = nl;
    }
    ck(cudaGraphLaunch(c->gexec, c->stream), "graph launch");
    return finish(c, c->graph_launches);
}

// The box that the next runs of a one-molecule context compute: the whole
// grid, or the tiles of a block selection plus one tile layer in + directions
// (the neighbours of the owned points' edges), clipped to the grid.  Sets the
// grid, the tile layout and their device copies; the next run plans again.
void apply_box(eses_ctx *c)
{
    Grid &G = c->grids[0];
    const MolInfo &I = c->mol[0];
    long long nt = 1, np = 1;
    for (int a = 0; a < 3; ++a) {
        const long long full = I.dims[a], ftiles = ceil_div_ll(full, TILE);
        G.full[a] = full;
        if (!c->sel) {
            G.toff[a] = 0;
            G.dims[a] = G.own[a] = full;
            G.tiles[a] = (int)ftiles;
        } else {
            const long long B = c->block_pts;
            const long long lo = c->sel_lo[a] * B, hi = std::min(c->sel_hi[a] * B, full);
            const long long tend = std::min(ceil_div_ll(hi, TILE) + 1, ftiles);
            G.toff[a] = (int)(lo / TILE);
            G.tiles[a] = (int)(tend - lo / TILE);
            G.dims[a] = std::min(tend * TILE, full) - lo;
            G.own[a] = hi - lo;
        }
        nt *= G.tiles[a];
        np *= G.dims[a];
    }
    G.n_tiles = nt;
    G.tile0 = 0;
    G.lab0 = 0;
    c->tile_off.assign(2, 0);
    c->tile_off[1] = nt;
    c->n_tiles = nt;
    c->n_points = np;
    c->B.n_tiles = nt;
    ck(cudaMemcpyAsync(c->grid_d.p, &G, sizeof(Grid), cudaMemcpyHostToDevice, c->stream), "copy grid");
    ck(cudaMemcpyAsync(c->tile_off_d.p, c->tile_off.data(), 2 * sizeof(long long), cudaMemcpyHostToDevice, c->stream),
       "copy tile offsets");
    ck(cudaStreamSynchronize(c->stream), "synchronize");
    drop_graph(c);
    c->planned = false;
    c->ran = false;
}

// points the allocation-failure countdown at the context for one entry point
struct AllocScope {
    explicit AllocScope(eses_ctx *c) { g_fail_countdown = &c->fail_alloc; }
    ~AllocScope() { g_fail_countdown = nullptr; }
};

int run_guarded(eses_ctx *c)
{
    c->ran = false;
    c->n_tri = -1;
    if (c->sel && c->exterior)
        return fail(c, ESES_EINVAL, "the exterior-only surface needs the whole grid (no block selection)");
    // per-tile arrays are indexed in 32 bits (4 ints per tile): a larger grid runs in block selections
    if (c->n_tiles >= (1LL << 31) / 4)
        return fail(c, ESES_EINVAL, "too many tiles in one run: select blocks (eses_set_blocks)");
    AllocScope scope(c);
    try {
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        return run_impl(c);
    } catch (const CudaError &e) {
        return fail(c, ESES_ECUDA, std::string(e.what) + ": " + cudaGetErrorString(e.e));
    } catch (const std::bad_alloc &) {
        // buffers may be half sized: the next run plans again
        drop_graph(c);
        c->planned = false;
        return fail(c, ESES_ENOMEM, "device allocation failed");
    } catch (const CaptureGrow &) {
        // a buffer the plan did not size: plan again (eagerly), capture next time
        drop_graph(c);
        c->planned = false;
        return run_guarded(c);
    } catch (const std::string &m) {
        return fail(c, ESES_EINVAL, m);
    }
}

bool mol_ok(const eses_ctx *c, int m) { return c && m >= 0 && m < c->n_mol; }

long long mol_points(const eses_ctx *c, int m)
{
    const MolInfo &I = c->mol[m];
    return I.dims[0] * I.dims[1] * I.dims[2];
}

// first record and count of molecule m in axis a's output
void mol_range(const eses_ctx *c, int m, int a, long long &off, long long &n)
{
    const long long *me = c->medge_h.data() + a * (c->n_mol + 1);
    off = me[m];
    n = me[m + 1] - me[m];
}

int single(eses_ctx *c)
{
    if (c && c->n_mol != 1) return fail(c, ESES_EINVAL, "batch context: use the eses_mol_* accessors");
    return ESES_OK;
}

}  // namespace

extern "C" {

int eses_create(const double *xyz, const double *radii, int64_t n_atoms, double r_p, double h, double margin,
                eses_ctx **out)
{
    if (!xyz || !radii) return fail(nullptr, ESES_EINVAL, "xyz or radii is NULL");
    if (n_atoms < 1 || n_atoms > (int64_t)1 << 30) return fail(nullptr, ESES_EINVAL, "n_atoms must be in [1, 2^30]");
    return create_common(xyz, radii, &n_atoms, 1, r_p, h, margin, nullptr, nullptr, out);
}

int eses_create_on_grid(const double *xyz, const double *radii, int64_t n_atoms, double r_p, double h,
                        const double origin[3], const int64_t dims[3], eses_ctx **out)
{
    if (!xyz || !radii || !origin || !dims) return fail(nullptr, ESES_EINVAL, "NULL argument");
    if (n_atoms < 1 || n_atoms > (int64_t)1 << 30) return fail(nullptr, ESES_EINVAL, "n_atoms must be in [1, 2^30]");
    for (int a = 0; a < 3; ++a) {
        if (!isfinite(origin[a])) return fail(nullptr, ESES_EINVAL, "origin must be finite");
        if (dims[a] < 1 || dims[a] > (1LL << 30)) return fail(nullptr, ESES_EINVAL, "dims must be in [1, 2^30]");
    }
    if (dims[0] * dims[1] * dims[2] > (1LL << 40)) return fail(nullptr, ESES_EINVAL, "grid too large");
    // margin = h passes the argument check; the caller's grid replaces the one it would give
    return create_common(xyz, radii, &n_atoms, 1, r_p, h, h, nullptr, nullptr, out, origin, dims);
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
    return create_common(hx.data(), hr.data(), &n_atoms, 1, r_p, h, margin, xyz, radii, out);
}

int eses_create_batch(const double *xyz, const double *radii, const int64_t *n_atoms, int n_mol, double r_p, double h,
                      double margin, eses_ctx **out)
{
    if (!xyz || !radii || !n_atoms) return fail(nullptr, ESES_EINVAL, "xyz, radii or n_atoms is NULL");
    return create_common(xyz, radii, n_atoms, n_mol, r_p, h, margin, nullptr, nullptr, out);
}

int eses_run_batch(int n_mol, const double *const *xyz, const double *const *radii, const int64_t *n_atoms,
                   double r_p, double h, double margin, eses_ctx **out)
{
    if (!out) return fail(nullptr, ESES_EINVAL, "out is NULL");
    *out = nullptr;
    if (!xyz || !radii || !n_atoms || n_mol < 1) return fail(nullptr, ESES_EINVAL, "bad argument");
    std::vector<double> X, R;
    for (int m = 0; m < n_mol; ++m) {
        if (!xyz[m] || !radii[m] || n_atoms[m] < 1)
            return fail(nullptr, ESES_EINVAL, "bad molecule " + std::to_string(m));
        X.insert(X.end(), xyz[m], xyz[m] + 3 * n_atoms[m]);
        R.insert(R.end(), radii[m], radii[m] + n_atoms[m]);
    }
    eses_ctx *c = nullptr;
    int rc = eses_create_batch(X.data(), R.data(), n_atoms, n_mol, r_p, h, margin, &c);
    if (rc) return rc;
    rc = run_guarded(c);
    if (rc) {
        g_create_error = c->err;
        eses_destroy(c);
        return rc;
    }
    *out = c;
    return ESES_OK;
}

int eses_set_option(eses_ctx *c, int key, int64_t value)
{
    if (!c) return fail(nullptr, ESES_EINVAL, "ctx is NULL");
    switch (key) {
    case ESES_OPT_BLOCK_PTS:
        if (value < TILE || value > (1 << 20) || value % TILE)
            return fail(c, ESES_EINVAL, "block points must be a multiple of 8 in [8, 2^20]");
        if (value != c->block_pts && c->sel) {  // the selection was in blocks of the old size: whole grid again
            c->sel = false;
            try {
                apply_box(c);
            } catch (const CudaError &e) {
                return fail(c, ESES_ECUDA, std::string(e.what) + ": " + cudaGetErrorString(e.e));
            }
        }
        c->block_pts = (int)value;
        return ESES_OK;
    case ESES_OPT_PRECISION:
        if (value != ESES_PREC_FP64 && value != ESES_PREC_FP32_FILTERED) return fail(c, ESES_EINVAL, "bad precision");
        c->precision = (int)value;
        return ESES_OK;
    case ESES_OPT_STREAM:
        drop_graph(c);
        c->stream = value ? (cudaStream_t)(intptr_t)value : c->own_stream;
        return ESES_OK;
    case ESES_OPT_SYNC:
        c->sync = value != 0;
        return ESES_OK;
    case ESES_OPT_PROFILE:
        drop_graph(c);
        c->profile = value != 0;
        return ESES_OK;
    case ESES_OPT_GRAPH:
        drop_graph(c);
        c->graph_on = value != 0;
        return ESES_OK;
    case ESES_OPT_QUEUE:
        drop_graph(c);
        c->use_queue = value != 0;
        return ESES_OK;
    case ESES_OPT_CLS_CTAS:
    case ESES_OPT_EDGE_CTAS:
        if (value < 0 || value > 64) return fail(c, ESES_EINVAL, "CTAs per SM must be in [0, 64]");
        drop_graph(c);
        (key == ESES_OPT_CLS_CTAS ? c->cls : c->edge).ctas_per_sm = (int)value;
        return ESES_OK;
    case ESES_OPT_CLS_TILES:
    case ESES_OPT_EDGE_TILES:
        if (value < 1 || value > 64) return fail(c, ESES_EINVAL, "tiles per pop must be in [1, 64]");
        drop_graph(c);
        (key == ESES_OPT_CLS_TILES ? c->cls : c->edge).tiles_per_pop = (int)value;
        return ESES_OK;
    case ESES_OPT_ROOT_THREADS:
        if (value < 0 || value > 256 || !root_threads_valid((int)value))
            return fail(c, ESES_EINVAL, "root threads must be 0, 64, 128 or 256");
        drop_graph(c);
        c->edge.threads = (int)value;
        return ESES_OK;
    case ESES_OPT_CULL:
        if (value != 0 && value != 1) return fail(c, ESES_EINVAL, "cull must be 0 or 1");
        if ((value != 0) != c->cull) {  // other staging lists: plan again
            drop_graph(c);
            c->planned = false;
        }
        c->cull = value != 0;
        return ESES_OK;
    case ESES_OPT_TC_WAIT:
        if (value < -1) return fail(c, ESES_EINVAL, "wait limit must be >= -1");
        drop_graph(c);
        c->tc_wait = value;
        return ESES_OK;
    case ESES_OPT_FAIL_ALLOC:
        if (value < 0) return fail(c, ESES_EINVAL, "allocation countdown must be >= 0");
        c->fail_alloc = value;
        return ESES_OK;
    case ESES_OPT_EXTERIOR:
        if (value != 0 && value != 1) return fail(c, ESES_EINVAL, "exterior must be 0 or 1");
        if (value && c->sel) return fail(c, ESES_EINVAL, "the exterior-only surface needs the whole grid");
        if ((value != 0) != c->exterior) {  // other list sizes: plan again (buffers may move)
            drop_graph(c);
            c->planned = false;
        }
        c->exterior = value != 0;
        return ESES_OK;
    default:
        return fail(c, ESES_EINVAL, "unknown option key " + std::to_string(key));
    }
}

int eses_get_option(const eses_ctx *cc, int key, int64_t *value)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!c || !value) return fail(c, ESES_EINVAL, "NULL argument");
    switch (key) {
    case ESES_OPT_BLOCK_PTS: *value = c->block_pts; return ESES_OK;
    case ESES_OPT_PRECISION: *value = c->precision; return ESES_OK;
    case ESES_OPT_STREAM: *value = (int64_t)(intptr_t)c->stream; return ESES_OK;
    case ESES_OPT_SYNC: *value = c->sync ? 1 : 0; return ESES_OK;
    case ESES_OPT_PROFILE: *value = c->profile ? 1 : 0; return ESES_OK;
    case ESES_OPT_TC_WAIT: *value = c->tc_wait; return ESES_OK;
    case ESES_OPT_CULL: *value = c->cull ? 1 : 0; return ESES_OK;
    case ESES_OPT_FAIL_ALLOC: *value = c->fail_alloc; return ESES_OK;
    case ESES_OPT_GRAPH: *value = c->graph_on ? 1 : 0; return ESES_OK;
    case ESES_OPT_QUEUE: *value = c->use_queue ? 1 : 0; return ESES_OK;
    case ESES_OPT_CLS_CTAS: *value = c->cls.ctas_per_sm; return ESES_OK;
    case ESES_OPT_EDGE_CTAS: *value = c->edge.ctas_per_sm; return ESES_OK;
    case ESES_OPT_CLS_TILES: *value = c->cls.tiles_per_pop; return ESES_OK;
    case ESES_OPT_EDGE_TILES: *value = c->edge.tiles_per_pop; return ESES_OK;
    case ESES_OPT_ROOT_THREADS: *value = c->edge.threads; return ESES_OK;
    case ESES_OPT_EXTERIOR: *value = c->exterior ? 1 : 0; return ESES_OK;
    default: return fail(c, ESES_EINVAL, "unknown option key " + std::to_string(key));
    }
}

int eses_run(eses_ctx *c)
{
    if (!c) return fail(nullptr, ESES_EINVAL, "ctx is NULL");
    return run_guarded(c);
}

int eses_autotune(eses_ctx *c, int reps, double *ms_out)
{
    if (!c) return fail(nullptr, ESES_EINVAL, "ctx is NULL");
    if (reps < 1 || reps > 100) return fail(c, ESES_EINVAL, "reps must be in [1, 100]");
    const bool graph = c->graph_on;
    c->graph_on = false;
    drop_graph(c);
    int rc = run_guarded(c);  // plans and leaves valid inputs for every stage
    if (rc) {
        c->graph_on = graph;
        return rc;
    }
    AllocScope scope(c);
    try {
        cudaStream_t st = c->stream;
        cudaEvent_t e0, e1;
        ck(cudaEventCreate(&e0), "event");
        ck(cudaEventCreate(&e1), "event");
        Model &M = c->M;
        Batch &B = c->B;
        int *misc = (int *)c->misc.p;
        int8_t *labels = (int8_t *)c->labels.p;
        int *tile_band = (int *)c->tile_band.p;
        auto time_it = [&](auto &&launch) {
            launch();
            ck(cudaEventRecord(e0, st), "record");
            for (int r = 0; r < reps; ++r) launch();
            ck(cudaEventRecord(e1, st), "record");
            ck(cudaEventSynchronize(e1), "sync");
            float ms = 0.0f;
            ck(cudaEventElapsedTime(&ms, e0, e1), "elapsed");
            return ms / reps;
        };
        const int cls_max = classify_ctas_per_sm(c->precision), edge_max = edge_ctas_per_sm(c->precision);
        // classification: CTAs per SM x tiles per pop (labels are rewritten identically)
        Shape best_cls = c->cls;
        float best_cls_ms = INFINITY;
        for (int k = 1; k <= cls_max; ++k)
            for (int per : {1, 4, 16}) {
                Shape s;
                s.ctas_per_sm = k;
                s.tiles_per_pop = per;
                float ms = time_it([&] {
                    ck(cudaMemsetAsync(c->queue.p, 0, 4 * sizeof(unsigned long long), st), "memset");
                    launch_classify(M, B, c->precision, sched_of(c, s, 0), grid_of(c, s, cls_max), labels,
                                    c->precision == ESES_PREC_FP64 ? nullptr : tile_band, misc, (int *)c->ovf.p,
                                    (unsigned char *)c->big.p, nullptr, st);
                });
                if (ms < best_cls_ms) best_cls_ms = ms, best_cls = s;
            }
        if (c->precision != ESES_PREC_FP64)
            launch_band(M, B, labels, tile_band, misc, (int *)c->ovf.p, (unsigned char *)c->big.p, st);
        // root solve: staging CTAs per SM x tiles per pop x root-kernel threads per block
        Shape best_edge = c->edge;
        float best_edge_ms = INFINITY;
        EdgeOut eo;
        for (int a = 0; a < 3; ++a) {
            eo.idx[a] = (long long *)c->out_idx[a].p;
            eo.tau[a] = (double *)c->out_tau[a].p;
            eo.nrm[a] = (double *)c->out_nrm[a].p;
            eo.tau32[a] = (float *)c->out_tau32[a].p;
            eo.nrm32[a] = (float *)c->out_nrm32[a].p;
            eo.code[a] = (int2 *)c->out_code[a].p;
        }
        RootWork W;  // the planned buffers of the run above
        W.einfo = (int4 *)c->r_einfo.p;
        W.ecnt = (int *)c->r_ecnt.p;
        W.hard = (int *)c->r_hard.p;
        W.csph = (int2 *)c->r_csph.p;
        W.nsph = (uint8_t *)c->r_nsph.p;
        W.rsph = (RootRec *)c->r_rsph.p;
        W.ctor = (int2 *)c->r_ctor.p;
        W.ntor = (uint8_t *)c->r_ntor.p;
        W.rtor = (RootRec *)c->r_rtor.p;
        W.slab = (unsigned char *)c->r_slab.p;
        W.ctr = (unsigned long long *)c->r_ctr.p;
        W.jobs = (int2 *)c->r_jobs.p;
        W.cap_jobs = c->cap_jobs;
        W.cap_slab = c->cap_slab;
        W.cap_sph = c->cap_sph;
        W.cap_tor = c->cap_tor;
        const long long ne_all = c->n_edges[0] + c->n_edges[1] + c->n_edges[2];
        W.n_edges = ne_all;
        for (int k = 1; k <= edge_max; ++k)
            for (int per : {1, 4})
                for (int threads : {128, 256}) {
                    Shape s;
                    s.ctas_per_sm = k;
                    s.tiles_per_pop = per;
                    s.threads = threads;
                    float ms = time_it([&] {
                        launch_edge_stage(M, B, c->precision, sched_of(c, s, 1), grid_of(c, s, edge_max), labels,
                                          (const int *)c->edge_start.p, eo, misc, (int *)c->ovf.p,
                                          (unsigned char *)c->big.p, W, st);
                        launch_edge_roots(M, B, c->precision, threads, eo, (const int *)c->edge_start.p, ne_all,
                                          misc + 1, misc, (long long *)c->fail_log.p, W, st);
                    });
                    if (ms < best_edge_ms) best_edge_ms = ms, best_edge = s;
                }
        ck(cudaGetLastError(), "autotune launch");
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        c->cls = best_cls;
        c->edge = best_edge;
        if (ms_out) {
            ms_out[0] = best_cls_ms;
            ms_out[1] = best_edge_ms;
        }
    } catch (const CudaError &e) {
        c->graph_on = graph;
        return fail(c, ESES_ECUDA, std::string(e.what) + ": " + cudaGetErrorString(e.e));
    }
    c->graph_on = graph;
    return run_guarded(c);  // fresh results with the chosen shapes
}

int eses_set_proposer(eses_ctx *c, int mode, const float *params, double p_far)
{
    if (!c) return fail(nullptr, ESES_EINVAL, "ctx is NULL");
    if (mode != ESES_PROPOSER_OFF && mode != ESES_PROPOSER_MLP && mode != ESES_PROPOSER_CERTIFY)
        return fail(c, ESES_EINVAL, "bad proposer mode");
    if (mode == ESES_PROPOSER_MLP) {
        if (!(p_far > 0.0 && p_far < 1.0)) return fail(c, ESES_EINVAL, "p_far must be in (0, 1)");
        if (!params && !c->have_params) return fail(c, ESES_EINVAL, "the MLP proposer needs parameters");
    }
    AllocScope scope(c);
    try {
        if (params) {
            for (int k = 0; k < MLP_NPARAM; ++k)
                if (!isfinite(params[k])) return fail(c, ESES_EINVAL, "non-finite proposer parameter");
            float *d = ensure<float>(c->mlp_params, MLP_NPARAM);
            ck(cudaMemcpy(d, params, sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice), "copy parameters");
            c->have_params = true;
        }
    } catch (const CudaError &e) {
        return fail(c, ESES_ECUDA, std::string(e.what) + ": " + cudaGetErrorString(e.e));
    } catch (const std::bad_alloc &) {
        return fail(c, ESES_ENOMEM, "device allocation failed");
    }
    drop_graph(c);
    if (mode != c->proposer) c->planned = false;  // its buffers join the plan
    c->proposer = mode;
    if (mode == ESES_PROPOSER_MLP) c->z_far = (float)log(p_far / (1.0 - p_far));
    return ESES_OK;
}

int eses_num_tiles(const eses_ctx *c, int64_t *n)
{
    if (!c || !n) return fail(const_cast<eses_ctx *>(c), ESES_EINVAL, "NULL argument");
    *n = c->n_tiles;
    return ESES_OK;
}

int eses_tile_data(const eses_ctx *cc, float *features, uint8_t *targets)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!c) return fail(c, ESES_EINVAL, "NULL argument");
    if (!c->ran) return fail(c, ESES_ESTATE, "no results: call eses_run first");
    try {
        if (features) launch_tile_features(c->M, c->B, features, c->stream);
        if (targets) launch_tile_targets(c->B, (const int8_t *)c->labels.p, targets, c->stream);
        ck(cudaGetLastError(), "tile data");
        ck(cudaStreamSynchronize(c->stream), "synchronize");
    } catch (const CudaError &e) {
        return fail(c, ESES_ECUDA, std::string(e.what) + ": " + cudaGetErrorString(e.e));
    }
    return ESES_OK;
}

int eses_num_molecules(const eses_ctx *c, int *n)
{
    if (!c || !n) return fail(const_cast<eses_ctx *>(c), ESES_EINVAL, "NULL argument");
    *n = c->n_mol;
    return ESES_OK;
}

int eses_mol_grid(const eses_ctx *cc, int m, int64_t dims[3], double origin[3])
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!mol_ok(c, m) || !dims || !origin) return fail(c, ESES_EINVAL, "bad argument");
    for (int a = 0; a < 3; ++a) {
        dims[a] = c->mol[m].dims[a];
        origin[a] = c->mol[m].lo[a];
    }
    return ESES_OK;
}

int eses_mol_labels(const eses_ctx *cc, int m, int8_t *out)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!mol_ok(c, m) || !out) return fail(c, ESES_EINVAL, "bad argument");
    if (!c->ran) return fail(c, ESES_ESTATE, "no results: call eses_run first");
    const Grid &G = c->grids[m];
    const int8_t *src = (const int8_t *)c->labels.p + G.lab0;
    bool ok = true;
    if (!c->sel) {
        const size_t n = (size_t)mol_points(c, m);
        ok = cudaMemcpyAsync(out, src, n, cudaMemcpyDeviceToHost, c->stream) == cudaSuccess;
    } else {  // the owned box out of the computed box, one plane at a time
        for (long long i = 0; i < G.own[0] && ok; ++i)
            ok = cudaMemcpy2DAsync(out + i * G.own[1] * G.own[2], (size_t)G.own[2], src + i * G.dims[1] * G.dims[2],
                                   (size_t)G.dims[2], (size_t)G.own[2], (size_t)G.own[1], cudaMemcpyDeviceToHost,
                                   c->stream) == cudaSuccess;
    }
    if (!ok || cudaStreamSynchronize(c->stream) != cudaSuccess) return fail(c, ESES_ECUDA, "label copy failed");
    return ESES_OK;
}

int eses_mol_labels_device(const eses_ctx *cc, int m, const int8_t **dptr)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!mol_ok(c, m) || !dptr) return fail(c, ESES_EINVAL, "bad argument");
    if (!c->ran) return fail(c, ESES_ESTATE, "no results: call eses_run first");
    if (c->sel) return fail(c, ESES_ESTATE, "a block selection's labels are read with eses_labels");
    *dptr = (const int8_t *)c->labels.p + c->grids[m].lab0;
    return ESES_OK;
}

int eses_mol_num_intersections(const eses_ctx *cc, int m, int axis, int64_t *n)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!mol_ok(c, m) || !n || axis < 0 || axis > 2) return fail(c, ESES_EINVAL, "bad argument");
    if (!c->ran) return fail(c, ESES_ESTATE, "no results: call eses_run first");
    long long off, cnt;
    mol_range(c, m, axis, off, cnt);
    *n = cnt;
    return ESES_OK;
}

int eses_mol_intersections(const eses_ctx *cc, int m, int axis, int64_t *lower_idx, double *tau, double *normal,
                           float *tau32, float *normal32)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!mol_ok(c, m) || axis < 0 || axis > 2) return fail(c, ESES_EINVAL, "bad argument");
    if (!c->ran) return fail(c, ESES_ESTATE, "no results: call eses_run first");
    long long off, cnt;
    mol_range(c, m, axis, off, cnt);
    const size_t ne = (size_t)cnt;
    if (ne == 0) return ESES_OK;
    cudaStream_t st = c->stream;
    bool ok = true;
    if (lower_idx)
        ok &= cudaMemcpyAsync(lower_idx, (const long long *)c->out_idx[axis].p + off, ne * 8, cudaMemcpyDeviceToHost,
                              st) == cudaSuccess;
    if (tau)
        ok &= cudaMemcpyAsync(tau, (const double *)c->out_tau[axis].p + off, ne * 8, cudaMemcpyDeviceToHost, st) ==
              cudaSuccess;
    if (normal)
        ok &= cudaMemcpyAsync(normal, (const double *)c->out_nrm[axis].p + 3 * off, ne * 24, cudaMemcpyDeviceToHost,
                              st) == cudaSuccess;
    if (tau32)
        ok &= cudaMemcpyAsync(tau32, (const float *)c->out_tau32[axis].p + off, ne * 4, cudaMemcpyDeviceToHost, st) ==
              cudaSuccess;
    if (normal32)
        ok &= cudaMemcpyAsync(normal32, (const float *)c->out_nrm32[axis].p + 3 * off, ne * 12,
                              cudaMemcpyDeviceToHost, st) == cudaSuccess;
    ok &= cudaStreamSynchronize(st) == cudaSuccess;
    if (!ok) return fail(c, ESES_ECUDA, "intersection copy failed");
    return ESES_OK;
}

int eses_mol_intersections_device(const eses_ctx *cc, int m, int axis, const int64_t **lower_idx, const double **tau,
                                  const double **normal, const float **tau32, const float **normal32)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!mol_ok(c, m) || axis < 0 || axis > 2) return fail(c, ESES_EINVAL, "bad argument");
    if (!c->ran) return fail(c, ESES_ESTATE, "no results: call eses_run first");
    long long off, cnt;
    mol_range(c, m, axis, off, cnt);
    if (lower_idx) *lower_idx = (const int64_t *)c->out_idx[axis].p + off;
    if (tau) *tau = (const double *)c->out_tau[axis].p + off;
    if (normal) *normal = (const double *)c->out_nrm[axis].p + 3 * off;
    if (tau32) *tau32 = (const float *)c->out_tau32[axis].p + off;
    if (normal32) *normal32 = (const float *)c->out_nrm32[axis].p + 3 * off;
    return ESES_OK;
}

int eses_mol_intersection_patches(const eses_ctx *cc, int m, int axis, int8_t *kind, int32_t *atoms)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!mol_ok(c, m) || axis < 0 || axis > 2) return fail(c, ESES_EINVAL, "bad argument");
    if (!c->ran) return fail(c, ESES_ESTATE, "no results: call eses_run first");
    long long off, n;
    mol_range(c, m, axis, off, n);
    if (n == 0) return ESES_OK;
    if (!kind && !atoms) return ESES_OK;
    const int na = c->M.n_atoms, np = c->M.n_pairs, nv = c->M.n_verts;
    std::vector<int2> code((size_t)n);
    std::vector<int> orig((size_t)na);
    std::vector<int2> ij((size_t)std::max(np, 1));
    std::vector<int4> va((size_t)std::max(nv, 1));
    bool ok = cudaMemcpy(code.data(), (const int2 *)c->out_code[axis].p + off, sizeof(int2) * (size_t)n,
                         cudaMemcpyDeviceToHost) == cudaSuccess;
    ok &= cudaMemcpy(orig.data(), c->atom_orig.p, sizeof(int) * (size_t)na, cudaMemcpyDeviceToHost) == cudaSuccess;
    if (np > 0) ok &= cudaMemcpy(ij.data(), c->pair_ij.p, sizeof(int2) * np, cudaMemcpyDeviceToHost) == cudaSuccess;
    if (nv > 0) ok &= cudaMemcpy(va.data(), c->vert_atoms.p, sizeof(int4) * nv, cudaMemcpyDeviceToHost) == cudaSuccess;
    if (!ok) return fail(c, ESES_ECUDA, "patch id copy failed");
    const int64_t base = c->in_off[(size_t)m];
    auto input_id = [&](int sorted) { return (int32_t)(c->kept[(size_t)orig[(size_t)sorted]] - base); };
    for (long long e = 0; e < n; ++e) {
        const int y = code[(size_t)e].y;
        const int k = (y >> 29) & 3, failed = (y >> 27) & 1, mid = y & ((1 << 27) - 1);
        int32_t id[3] = {-1, -1, -1};
        int nid = 0;
        if (!failed) {
            if (k == 0) {
                id[nid++] = input_id(mid);
            } else if (k == 1) {
                id[nid++] = input_id(ij[(size_t)mid].x);
                id[nid++] = input_id(ij[(size_t)mid].y);
            } else {
                id[nid++] = input_id(va[(size_t)mid].x);
                id[nid++] = input_id(va[(size_t)mid].y);
                id[nid++] = input_id(va[(size_t)mid].z);
            }
            std::sort(id, id + nid);
        }
        if (kind) kind[e] = failed ? (int8_t)-1 : (int8_t)k;
        if (atoms)
            for (int q = 0; q < 3; ++q) atoms[3 * e + q] = id[q];
    }
    return ESES_OK;
}

int eses_mol_area_volume(const eses_ctx *cc, int m, double *area, double *volume)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!mol_ok(c, m) || !area || !volume) return fail(c, ESES_EINVAL, "bad argument");
    if (!c->ran) return fail(c, ESES_ESTATE, "no results: call eses_run first");
    *area = c->av_h[2 * m];
    *volume = c->av_h[2 * m + 1];
    return ESES_OK;
}

int eses_num_blocks(const eses_ctx *cc, int64_t nblocks[3])
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!c || !nblocks) return fail(c, ESES_EINVAL, "NULL argument");
    if (int rc = single(c)) return rc;
    for (int a = 0; a < 3; ++a) nblocks[a] = ceil_div_ll(c->mol[0].dims[a], c->block_pts);
    return ESES_OK;
}

int eses_set_blocks(eses_ctx *c, const int64_t block_lo[3], const int64_t block_hi[3])
{
    if (!c) return fail(nullptr, ESES_EINVAL, "ctx is NULL");
    if (int rc = single(c)) return rc;
    if ((block_lo == nullptr) != (block_hi == nullptr)) return fail(c, ESES_EINVAL, "give both block bounds or neither");
    if (block_lo) {
        if (c->exterior) return fail(c, ESES_EINVAL, "the exterior-only surface needs the whole grid");
        for (int a = 0; a < 3; ++a) {
            const long long nb = ceil_div_ll(c->mol[0].dims[a], c->block_pts);
            if (block_lo[a] < 0 || block_hi[a] <= block_lo[a] || block_hi[a] > nb)
                return fail(c, ESES_EINVAL, "block range must satisfy 0 <= lo < hi <= eses_num_blocks");
        }
    }
    c->sel = block_lo != nullptr;
    for (int a = 0; a < 3; ++a) {
        c->sel_lo[a] = c->sel ? block_lo[a] : 0;
        c->sel_hi[a] = c->sel ? block_hi[a] : 0;
    }
    try {
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        apply_box(c);
    } catch (const CudaError &e) {
        return fail(c, ESES_ECUDA, std::string(e.what) + ": " + cudaGetErrorString(e.e));
    }
    return ESES_OK;
}

int eses_owned_box(const eses_ctx *cc, int64_t lo[3], int64_t dims[3])
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!c || !lo || !dims) return fail(c, ESES_EINVAL, "NULL argument");
    if (int rc = single(c)) return rc;
    const Grid &G = c->grids[0];
    for (int a = 0; a < 3; ++a) {
        lo[a] = (int64_t)TILE * G.toff[a];
        dims[a] = G.own[a];
    }
    return ESES_OK;
}

int eses_grid(const eses_ctx *cc, int64_t dims[3], double origin[3])
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!c || !dims || !origin) return fail(c, ESES_EINVAL, "NULL argument");
    if (int rc = single(c)) return rc;
    return eses_mol_grid(c, 0, dims, origin);
}

int eses_labels(const eses_ctx *cc, int8_t *out)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!c || !out) return fail(c, ESES_EINVAL, "NULL argument");
    if (int rc = single(c)) return rc;
    return eses_mol_labels(c, 0, out);
}

int eses_labels_device(const eses_ctx *cc, const int8_t **dptr)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!c || !dptr) return fail(c, ESES_EINVAL, "NULL argument");
    if (int rc = single(c)) return rc;
    return eses_mol_labels_device(c, 0, dptr);
}

int eses_num_intersections(const eses_ctx *cc, int axis, int64_t *n)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!c || !n || axis < 0 || axis > 2) return fail(c, ESES_EINVAL, "bad argument");
    if (int rc = single(c)) return rc;
    return eses_mol_num_intersections(c, 0, axis, n);
}

int eses_intersections(const eses_ctx *cc, int axis, int64_t *lower_idx, double *tau, double *normal, float *tau32,
                       float *normal32)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!c || axis < 0 || axis > 2) return fail(c, ESES_EINVAL, "bad argument");
    if (int rc = single(c)) return rc;
    return eses_mol_intersections(c, 0, axis, lower_idx, tau, normal, tau32, normal32);
}

int eses_intersections_device(const eses_ctx *cc, int axis, const int64_t **lower_idx, const double **tau,
                              const double **normal, const float **tau32, const float **normal32)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!c || axis < 0 || axis > 2) return fail(c, ESES_EINVAL, "bad argument");
    if (int rc = single(c)) return rc;
    return eses_mol_intersections_device(c, 0, axis, lower_idx, tau, normal, tau32, normal32);
}

int eses_intersection_patches(const eses_ctx *cc, int axis, int8_t *kind, int32_t *atoms)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!c) return fail(c, ESES_EINVAL, "NULL argument");
    if (int rc = single(c)) return rc;
    return eses_mol_intersection_patches(c, 0, axis, kind, atoms);
}

int eses_area_volume(const eses_ctx *cc, double *area, double *volume)
{
    eses_ctx *c = const_cast<eses_ctx *>(cc);
    if (!c || !area || !volume) return fail(c, ESES_EINVAL, "NULL argument");
    if (int rc = single(c)) return rc;
    return eses_mol_area_volume(c, 0, area, volume);
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
            const int32_t a = (int32_t)c->kept[(size_t)orig[ij[p].x]], b = (int32_t)c->kept[(size_t)orig[ij[p].y]];
            pair_atoms[2 * p] = std::min(a, b);  // the circle's axis points from this atom to the other
            pair_atoms[2 * p + 1] = std::max(a, b);
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

int eses_mesh_count(eses_ctx *c, int64_t *n_tri)
{
    if (!c || !n_tri) return fail(c, ESES_EINVAL, "NULL argument");
    if (int rc = single(c)) return rc;
    if (!c->ran) return fail(c, ESES_ESTATE, "no results: call eses_run first");
    if (c->sel) return fail(c, ESES_ESTATE, "the mesh needs the whole grid (no block selection)");
    AllocScope scope(c);
    try {
        ck(cudaSetDevice(c->device), "cudaSetDevice");
        if (c->n_tri < 0) {
            cudaStream_t st = c->stream;
            const long long nt = c->n_tiles;
            const Batch &B = c->B;
            uint32_t *mask = ensure<uint32_t>(c->mesh_mask, (size_t)nt * 3 * (TILE_PTS / 32));
            int *tile = ensure<int>(c->mesh_tile, nt);
            int *off = ensure<int>(c->mesh_off, nt + 1);
            int *derr = ensure<int>(c->mesh_err, 1);
            launch_mesh_masks(B, (const int8_t *)c->labels.p, mask, st);
            launch_mesh_count(B, (const int8_t *)c->labels.p, tile, st);
            // the total in 64 bits first: the offsets are 32-bit
            std::vector<int> per_tile((size_t)nt);
            ck(cudaMemcpyAsync(per_tile.data(), tile, sizeof(int) * (size_t)nt, cudaMemcpyDeviceToHost, st), "read");
            ck(cudaStreamSynchronize(st), "synchronize");
            long long total = 0;
            for (int v : per_tile) total += v;
            if (total >= (1LL << 31)) return fail(c, ESES_EINVAL, "mesh of 2^31 triangles or more");
            scan(c, tile, off, nt);
            const int tot = (int)total;
            EdgeOut eo{};
            for (int a = 0; a < 3; ++a) eo.tau[a] = (double *)c->out_tau[a].p;
            long long *keys = ensure<long long>(c->mesh_keys, 3 * (size_t)std::max(tot, 1));
            double *xyz = ensure<double>(c->mesh_xyz, 9 * (size_t)std::max(tot, 1));
            ck(cudaMemsetAsync(derr, 0, sizeof(int), st), "memset");
            launch_mesh_emit(B, (const int8_t *)c->labels.p, mask, (const int *)c->edge_start.p, eo, off, keys, xyz,
                             derr, st);
            int herr = 0;
            ck(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, st), "read");
            ck(cudaStreamSynchronize(st), "synchronize");
            ck(cudaGetLastError(), "mesh kernels");
            if (herr) return fail(c, ESES_ESTATE, "a cut cube edge has no intersection in the run's output");
            c->n_tri = tot;
        }
    } catch (const CudaError &e) {
        return fail(c, ESES_ECUDA, std::string(e.what) + ": " + cudaGetErrorString(e.e));
    } catch (const std::bad_alloc &) {
        return fail(c, ESES_ENOMEM, "device allocation failed");
    }
    *n_tri = c->n_tri;
    return ESES_OK;
}

int eses_mesh(eses_ctx *c, int64_t *keys, double *xyz)
{
    if (!c || (!keys && !xyz)) return fail(c, ESES_EINVAL, "NULL argument");
    int64_t n = 0;
    if (int rc = eses_mesh_count(c, &n)) return rc;
    if (n == 0) return ESES_OK;
    if (keys && cudaMemcpy(keys, c->mesh_keys.p, sizeof(int64_t) * 3 * (size_t)n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(c, ESES_ECUDA, "copy mesh keys");
    if (xyz && cudaMemcpy(xyz, c->mesh_xyz.p, sizeof(double) * 9 * (size_t)n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(c, ESES_ECUDA, "copy mesh points");
    return ESES_OK;
}

int eses_mesh_table(int8_t *tri, uint8_t *ntri)
{
    if (!tri || !ntri) return fail(nullptr, ESES_EINVAL, "NULL argument");
    if (mesh_table_host(tri, ntri, ESES_MESH_MAXT) != 0) return fail(nullptr, ESES_EINVAL, "mesh case table");
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

int eses_mlp_forward(const float *X, int64_t n, const float *params, float *z, void *stream)
{
    if (!X || !params || !z || n < 0 || n > (1LL << 30)) return fail(nullptr, ESES_EINVAL, "bad argument");
    launch_mlp_forward(X, (int)n, params, z, (cudaStream_t)stream);
    if (cudaGetLastError() != cudaSuccess) return fail(nullptr, ESES_ECUDA, "mlp forward launch failed");
    return ESES_OK;
}

int eses_mlp_forward_tc(const float *X, int64_t n, const float *params, float *z, int *err, void *stream)
{
    if (!X || !params || !z || !err || n < 0 || n > (1LL << 30)) return fail(nullptr, ESES_EINVAL, "bad argument");
    mlp_init();
    launch_mlp_forward_tc(X, (int)n, params, z, err, (cudaStream_t)stream);
    if (cudaGetLastError() != cudaSuccess) return fail(nullptr, ESES_ECUDA, "tensor-core mlp launch failed");
    return ESES_OK;
}

int64_t eses_mlp_grad_scratch(int64_t n) { return n > 0 && n <= (1LL << 30) ? mlp_grad_scratch((int)n) : 0; }

int eses_mlp_grad(const float *X, const float *y, const float *w, int64_t n, const float *params, float *grad,
                  float *loss, float *scratch, void *stream)
{
    if (!X || !y || !w || !params || !grad || !loss || !scratch || n < 1 || n > (1LL << 30))
        return fail(nullptr, ESES_EINVAL, "bad argument");
    mlp_init();
    launch_mlp_grad(X, y, w, (int)n, params, scratch, grad, loss, (cudaStream_t)stream);
    if (cudaGetLastError() != cudaSuccess) return fail(nullptr, ESES_ECUDA, "mlp gradient launch failed");
    return ESES_OK;
}

int eses_mlp_adam(float *params, const float *grad, float *m, float *v, int step, float lr, void *stream)
{
    if (!params || !grad || !m || !v || step < 1 || !(lr > 0.0f)) return fail(nullptr, ESES_EINVAL, "bad argument");
    launch_adam(params, grad, m, v, step, lr, (cudaStream_t)stream);
    if (cudaGetLastError() != cudaSuccess) return fail(nullptr, ESES_ECUDA, "adam launch failed");
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
    DBuf *bufs[] = {&c->xyz, &c->rad, &c->in_mol, &c->grid_d, &c->cg_d, &c->tile_off_d, &c->atom_mol, &c->vert_mol,
                    &c->medge, &c->term, &c->queue, &c->cell_id, &c->cell_count, &c->cell_start, &c->cursor,
                    &c->atom_orig, &c->atom, &c->nb_count, &c->nb_start, &c->nb_list, &c->circle_count,
                    &c->contained, &c->face, &c->pair_count, &c->pair_start, &c->pair_o, &c->pair_u, &c->pair_ij,
                    &c->pair_free, &c->vert_count, &c->vert_start, &c->vert, &c->vert_atoms, &c->pbin_count, &c->pbin_start,
                    &c->pbin_cursor, &c->pbin_cell, &c->pbin_list, &c->vbin_count, &c->vbin_start, &c->vbin_cursor,
                    &c->vbin_cell, &c->vbin_list, &c->labels, &c->tile_band, &c->tile_edges, &c->edge_start,
                    &c->tile_inside, &c->scan_tmp, &c->misc, &c->av, &c->counts, &c->red_d, &c->red_i, &c->fail_log,
                    &c->ovf, &c->big, &c->r_einfo, &c->r_ecnt, &c->r_csph, &c->r_ctor, &c->r_nsph, &c->r_ntor,
                    &c->r_rsph, &c->r_rtor, &c->r_slab, &c->r_ctr, &c->r_hard, &c->r_jobs, &c->atom_hi,
                    &c->atom_lo, &c->pair_hi, &c->pair_lo, &c->pair_u32, &c->vert_hi, &c->vert_lo,
                    &c->mlp_params, &c->need, &c->need_pos, &c->tile_list, &c->prop_counts, &c->features,
                    &c->targets, &c->ext, &c->ext_open, &c->ext_misc, &c->mesh_mask, &c->mesh_tile, &c->mesh_off,
                    &c->mesh_keys, &c->mesh_xyz, &c->mesh_err};
    if (c->own_stream) cudaStreamSynchronize(c->own_stream);
    drop_graph(c);
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
