// eses_mesh.cu -- triangle mesh of the surface from the labels and the edge
// intersections of a run, cube by cube (the next item after the hot path;
// the paper stops at the labels and intersections, Eq. 2-4).
//
// The cube rule (reading M1).  Corner i of a grid cube sits at offset
// ((i >> 2) & 1, (i >> 1) & 1, i & 1) from the cube's lower corner.  Cube edge
// 4 a + j runs along axis a from the j-th corner, in increasing corner number,
// whose axis-a offset is 0; it is cut when its corner labels differ, and its
// surface point is that edge's intersection.  On each face the cut edges pair
// into segments: two cut edges make one; four (inside corners on a diagonal)
// make two, each joining the two edges at one inside corner.  The rule sees
// only the face's labels, so cubes sharing a face agree and the mesh closes.
// The segments form loops (each cut edge is on two faces); a loop starts at
// its smallest edge, walks first towards the smaller of its two neighbours,
// is reversed after its first vertex if its Newell normal (from the edge
// midpoints) points on the whole from outside corners to inside ones, and is
// cut into the fan (v0, v_k, v_k+1).  The 256-case table is built on the host
// at library set-up.
//
// Kernels (one warp per 8x8x8 tile, cubes by their lower corner):
//   k_mesh_masks  per tile and axis, a 512-bit mask of the crossing edges
//                 leaving its points (their rank in the tile's run of the
//                 axis' output is a prefix popcount);
//   k_mesh_count  triangles per tile;
//   k_mesh_emit   after an exclusive scan, the triangles: per vertex the key
//                 3 * (lower point of its edge) + axis and the intersection
//                 point (FP64), read from the run's outputs.
#include <cstring>
#include <vector>

#include "eses_kernels.h"
#include "eses_tile.cuh"

namespace eses {

constexpr int MESH_WARPS = 8;
constexpr int MC_MAXT = 12;  // triangles per cube at most (the rule gives at most 5)

__constant__ int8_t c_mc_tri[256][3 * MC_MAXT];
__constant__ uint8_t c_mc_n[256];
__constant__ int8_t c_mc_edge[12][4];  // axis, offsets of the lower corner

// ---------------------------------------------------------------------------
// the case table (host)
// ---------------------------------------------------------------------------
static int corner_off(int i, int a) { return (i >> (2 - a)) & 1; }

struct CubeEdge {
    int axis, lo, hi;
};

static std::vector<CubeEdge> cube_edges()
{
    std::vector<CubeEdge> out;
    for (int a = 0; a < 3; ++a)
        for (int i = 0; i < 8; ++i)
            if (corner_off(i, a) == 0) out.push_back({a, i, i | (1 << (2 - a))});
    return out;
}

// one case: triangles as cube-edge triples; false if the rule fails (never expected)
static bool mc_case(int cs, const std::vector<CubeEdge> &E, std::vector<int> &tris)
{
    tris.clear();
    int in[8];
    for (int i = 0; i < 8; ++i) in[i] = (cs >> i) & 1;
    bool cut[12];
    for (int e = 0; e < 12; ++e) cut[e] = in[E[e].lo] != in[E[e].hi];
    int nb[12][2], nn[12] = {0};
    auto link = [&](int x, int y) {
        if (nn[x] < 2) nb[x][nn[x]] = y;
        if (nn[y] < 2) nb[y][nn[y]] = x;
        ++nn[x];
        ++nn[y];
    };
    for (int a = 0; a < 3; ++a)
        for (int side = 0; side < 2; ++side) {
            int fe[4], nf = 0;
            for (int e = 0; e < 12; ++e)
                if (E[e].axis != a && corner_off(E[e].lo, a) == side && corner_off(E[e].hi, a) == side) fe[nf++] = e;
            if (nf != 4) return false;
            int ce[4], nc = 0;
            for (int k = 0; k < 4; ++k)
                if (cut[fe[k]]) ce[nc++] = fe[k];
            if (nc == 2) {
                link(ce[0], ce[1]);
            } else if (nc == 4) {
                for (int c = 0; c < 8; ++c) {  // each inside corner of the face: its two face edges
                    if (corner_off(c, a) != side || !in[c]) continue;
                    int at[2], na = 0;
                    for (int k = 0; k < 4; ++k)
                        if ((E[fe[k]].lo == c || E[fe[k]].hi == c) && na < 2) at[na++] = fe[k];
                    if (na != 2) return false;
                    link(at[0], at[1]);
                }
            } else if (nc != 0) {
                return false;
            }
        }
    for (int e = 0; e < 12; ++e)
        if (cut[e] != (nn[e] == 2) || nn[e] > 2) return false;
    bool seen[12] = {false};
    for (int s = 0; s < 12; ++s) {
        if (!cut[s] || seen[s]) continue;
        int loop[12], nl = 0;
        loop[nl++] = s;
        seen[s] = true;
        int cur = s, nxt = nb[s][0] < nb[s][1] ? nb[s][0] : nb[s][1];
        while (nxt != s) {
            if (nl >= 12) return false;
            loop[nl++] = nxt;
            seen[nxt] = true;
            const int after = nb[nxt][0] == cur ? nb[nxt][1] : nb[nxt][0];
            cur = nxt;
            nxt = after;
        }
        // Newell normal of the edge midpoints against inside -> outside
        double mid[12][3], n[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < nl; ++k)
            for (int a = 0; a < 3; ++a)
                mid[k][a] = 0.5 * (corner_off(E[loop[k]].lo, a) + corner_off(E[loop[k]].hi, a));
        for (int k = 0; k < nl; ++k) {
            const double *p = mid[k], *q = mid[(k + 1) % nl];
            n[0] += (p[1] - q[1]) * (p[2] + q[2]);
            n[1] += (p[2] - q[2]) * (p[0] + q[0]);
            n[2] += (p[0] - q[0]) * (p[1] + q[1]);
        }
        double score = 0.0;
        for (int k = 0; k < nl; ++k) {
            const CubeEdge &ed = E[loop[k]];
            const int ci = in[ed.lo] ? ed.lo : ed.hi, co = in[ed.lo] ? ed.hi : ed.lo;
            for (int a = 0; a < 3; ++a) score += (corner_off(co, a) - corner_off(ci, a)) * n[a];
        }
        if (score == 0.0) return false;
        if (score < 0.0)
            for (int x = 1, y = nl - 1; x < y; ++x, --y) std::swap(loop[x], loop[y]);
        for (int k = 1; k + 1 < nl; ++k) {
            tris.push_back(loop[0]);
            tris.push_back(loop[k]);
            tris.push_back(loop[k + 1]);
        }
    }
    return (int)tris.size() <= 3 * MC_MAXT;
}

// the table: tri[case][3 k + v] cube edges, n[case] triangles; false on a rule failure
static bool mc_table(int8_t (*tri)[3 * MC_MAXT], uint8_t *n)
{
    const std::vector<CubeEdge> E = cube_edges();
    std::vector<int> t;
    for (int cs = 0; cs < 256; ++cs) {
        if (!mc_case(cs, E, t)) return false;
        n[cs] = (uint8_t)(t.size() / 3);
        for (int k = 0; k < 3 * MC_MAXT; ++k) tri[cs][k] = k < (int)t.size() ? (int8_t)t[k] : (int8_t)-1;
    }
    return true;
}

int mesh_table_host(int8_t *tri, uint8_t *n, int max_tri)
{
    static int8_t T[256][3 * MC_MAXT];
    static uint8_t N[256];
    if (!mc_table(T, N)) return -1;
    for (int cs = 0; cs < 256; ++cs) {
        if (N[cs] > max_tri) return -1;
        n[cs] = N[cs];
        for (int k = 0; k < 3 * max_tri; ++k) tri[cs * 3 * max_tri + k] = k < 3 * MC_MAXT ? T[cs][k] : (int8_t)-1;
    }
    return 0;
}

int mesh_init()
{
    static int8_t T[256][3 * MC_MAXT];
    static uint8_t N[256];
    if (!mc_table(T, N)) return -1;
    int8_t ed[12][4];
    const std::vector<CubeEdge> E = cube_edges();
    for (int e = 0; e < 12; ++e) {
        ed[e][0] = (int8_t)E[e].axis;
        for (int a = 0; a < 3; ++a) ed[e][1 + a] = (int8_t)corner_off(E[e].lo, a);
    }
    if (cudaMemcpyToSymbol(c_mc_tri, T, sizeof(T)) != cudaSuccess) return -1;
    if (cudaMemcpyToSymbol(c_mc_n, N, sizeof(N)) != cudaSuccess) return -1;
    if (cudaMemcpyToSymbol(c_mc_edge, ed, sizeof(ed)) != cudaSuccess) return -1;
    return 0;
}

// ---------------------------------------------------------------------------
// kernels (one molecule: B.grid[0], tiles 0 .. n_tiles - 1)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tile_point(const int *t, int p, long long *g)
{
    g[0] = (long long)TILE * t[0] + (p >> 6);
    g[1] = (long long)TILE * t[1] + ((p >> 3) & 7);
    g[2] = (long long)TILE * t[2] + (p & 7);
}

// case of the cube whose lower corner is g (-1 when the cube leaves the grid)
__device__ __forceinline__ int cube_case(const int8_t *__restrict__ labels, const long long *d, const long long *g)
{
    if (g[0] + 1 >= d[0] || g[1] + 1 >= d[1] || g[2] + 1 >= d[2]) return -1;
    int cs = 0;
    for (int c = 0; c < 8; ++c) {
        const long long i = g[0] + ((c >> 2) & 1), j = g[1] + ((c >> 1) & 1), k = g[2] + (c & 1);
        if (labels[(i * d[1] + j) * d[2] + k]) cs |= 1 << c;
    }
    return cs;
}

__global__ void __launch_bounds__(MESH_WARPS * 32) k_mesh_masks(Batch B, const int8_t *__restrict__ labels,
                                                               uint32_t *__restrict__ mask)
{
    const int lane = threadIdx.x & 31;
    const Grid &G = B.grid[0];
    const long long d[3] = {G.dims[0], G.dims[1], G.dims[2]};
    const long long str[3] = {d[1] * d[2], d[2], 1};
    const long long nw = (long long)gridDim.x * MESH_WARPS;
    for (long long gt = (long long)blockIdx.x * MESH_WARPS + (threadIdx.x >> 5); gt < B.n_tiles; gt += nw) {
        int t[3];
        tile_coords(G, gt, t);
        for (int r = 0; r < TILE_PTS / 32; ++r) {
            long long g[3];
            tile_point(t, 32 * r + lane, g);
            const bool valid = g[0] < d[0] && g[1] < d[1] && g[2] < d[2];
            const long long idx = (g[0] * d[1] + g[1]) * d[2] + g[2];
            const int l0 = valid ? labels[idx] : 0;
            for (int a = 0; a < 3; ++a) {
                const bool c = valid && g[a] + 1 < d[a] && labels[idx + str[a]] != l0;
                const unsigned m = __ballot_sync(0xffffffffu, c);
                if (lane == 0) mask[(gt * 3 + a) * (TILE_PTS / 32) + r] = m;
            }
        }
    }
}

__global__ void __launch_bounds__(MESH_WARPS * 32) k_mesh_count(Batch B, const int8_t *__restrict__ labels,
                                                               int *__restrict__ tile_tri)
{
    const int lane = threadIdx.x & 31;
    const Grid &G = B.grid[0];
    const long long d[3] = {G.dims[0], G.dims[1], G.dims[2]};
    const long long nw = (long long)gridDim.x * MESH_WARPS;
    for (long long gt = (long long)blockIdx.x * MESH_WARPS + (threadIdx.x >> 5); gt < B.n_tiles; gt += nw) {
        int t[3];
        tile_coords(G, gt, t);
        int n = 0;
        for (int p = lane; p < TILE_PTS; p += 32) {
            long long g[3];
            tile_point(t, p, g);
            const int cs = cube_case(labels, d, g);
            if (cs >= 0) n += c_mc_n[cs];
        }
        n = __reduce_add_sync(0xffffffffu, n);
        if (lane == 0) tile_tri[gt] = n;
    }
}

__global__ void __launch_bounds__(MESH_WARPS * 32) k_mesh_emit(Batch B, const int8_t *__restrict__ labels,
                                                              const uint32_t *__restrict__ mask,
                                                              const int *__restrict__ edge_start, EdgeOut out,
                                                              const int *__restrict__ tile_off,
                                                              long long *__restrict__ keys, double *__restrict__ xyz,
                                                              int *__restrict__ err)
{
    const int lane = threadIdx.x & 31;
    const Grid &G = B.grid[0];
    const long long d[3] = {G.dims[0], G.dims[1], G.dims[2]};
    const long long nt = B.n_tiles;
    const long long nw = (long long)gridDim.x * MESH_WARPS;
    const double h = G.h;
    for (long long gt = (long long)blockIdx.x * MESH_WARPS + (threadIdx.x >> 5); gt < nt; gt += nw) {
        int t[3];
        tile_coords(G, gt, t);
        long long run = tile_off[gt];
        for (int r = 0; r < TILE_PTS / 32; ++r) {
            long long g[3];
            tile_point(t, 32 * r + lane, g);
            const int cs = cube_case(labels, d, g);
            const int cnt = cs >= 0 ? c_mc_n[cs] : 0;
            int inc = cnt;  // cubes in local order: inclusive warp scan
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += u;
            }
            const long long first = run + inc - cnt;
            run += __shfl_sync(0xffffffffu, inc, 31);
            for (int k = 0; k < cnt; ++k)
                for (int v = 0; v < 3; ++v) {
                    const int e = c_mc_tri[cs][3 * k + v];
                    const int a = c_mc_edge[e][0];
                    const long long gl[3] = {g[0] + c_mc_edge[e][1], g[1] + c_mc_edge[e][2], g[2] + c_mc_edge[e][3]};
                    // the edge's rank in its tile's run of axis a's output
                    const long long tl = ((gl[0] >> 3) * G.tiles[1] + (gl[1] >> 3)) * G.tiles[2] + (gl[2] >> 3);
                    const int lp = (int)(((gl[0] & 7) * TILE + (gl[1] & 7)) * TILE + (gl[2] & 7));
                    const uint32_t *mw = mask + (tl * 3 + a) * (TILE_PTS / 32);
                    const uint32_t w = mw[lp >> 5];
                    int rank = __popc(w & ((1u << (lp & 31)) - 1u));
                    for (int q = 0; q < (lp >> 5); ++q) rank += __popc(mw[q]);
                    const long long id = (long long)edge_start[a * nt + tl] - edge_start[a * nt] + rank;
                    const long long na = (long long)edge_start[(a + 1) * nt] - edge_start[a * nt];
                    double tau = 0.0;
                    if (((w >> (lp & 31)) & 1u) && id >= 0 && id < na) tau = out.tau[a][id];
                    else atomicOr(err, 1);  // the cube's cut edge is not in the run's output
                    const long long o = 3 * (first + k) + v;
                    keys[o] = 3 * ((gl[0] * d[1] + gl[1]) * d[2] + gl[2]) + a;
                    for (int b = 0; b < 3; ++b)
                        xyz[3 * o + b] = G.lo[b] + h * (double)gl[b] + (b == a ? tau * h : 0.0);
                }
        }
    }
}

static int warp_grid(long long n_tiles)
{
    const long long g = (n_tiles + MESH_WARPS - 1) / MESH_WARPS;
    return (int)(g < 1 ? 1 : (g > 1048576 ? 1048576 : g));
}

int launch_mesh_masks(const Batch &B, const int8_t *labels, uint32_t *mask, cudaStream_t st)
{
    k_mesh_masks<<<warp_grid(B.n_tiles), MESH_WARPS * 32, 0, st>>>(B, labels, mask);
    return 1;
}

int launch_mesh_count(const Batch &B, const int8_t *labels, int *tile_tri, cudaStream_t st)
{
    k_mesh_count<<<warp_grid(B.n_tiles), MESH_WARPS * 32, 0, st>>>(B, labels, tile_tri);
    return 1;
}

int launch_mesh_emit(const Batch &B, const int8_t *labels, const uint32_t *mask, const int *edge_start,
                     const EdgeOut &out, const int *tile_off, long long *keys, double *xyz, int *err, cudaStream_t st)
{
    k_mesh_emit<<<warp_grid(B.n_tiles), MESH_WARPS * 32, 0, st>>>(B, labels, mask, edge_start, out, tile_off, keys,
                                                                  xyz, err);
    return 1;
}

}  // namespace eses
