// eses_classify.cu -- grid-point classification kernels (the second ESES
// stage, Eq. 2), one CTA per 8x8x8 tile.
//
// k_classify<T, FILT>:
//   1. stages the tile's atoms, free-arc pairs and free triple points in
//      shared memory (tile frame) and lists, for every staged atom, the staged
//      pairs it belongs to;
//   2. splits the tile into 16 bricks of 2x4x4 points, one warp per brick:
//      the lanes test the staged atoms against the brick's box and ballots
//      give the set of atoms whose expanded ball reaches the brick.  A warp
//      with an empty set labels its 32 points outside at once; otherwise every
//      lane tests its point against the set: inside a van der Waals ball -> 1,
//      in no expanded ball -> 0, else a shell point;
//   3. shell points go to a per-tile queue; when there are any, the block
//      builds the staged atoms' neighbour sets (expanded spheres that meet)
//      and works through the queue: free triple points within r_p, convex
//      witnesses of the containing balls, saddle witnesses of the pairs of
//      the containing balls, each witness tested for freeness against the
//      neighbours of its atoms only.
//   T = double, FILT = false is the plain FP64 form; T = float, FILT = true
//   is the filtered form, whose undecided points get LABEL_BAND and are
//   counted per tile.
// k_band: re-labels the undecided points of the tiles that have any, in FP64:
//   one warp per point runs the witness search over every staged item.
#include "eses_kernels.h"
#include "eses_tile.cuh"

namespace eses {

constexpr int CLS_THREADS = 256;
constexpr int NBRICK = 16;     // 2x4x4-point bricks per tile

template <class CP>
struct ClsSmem {
    static constexpr int HS = slot_hash_size<CP>(), AWC = atom_words<CP>();
    int hkey[HS];                  // staged-atom lookup (pair_slots)
    short hval[HS];
    short2 pslot[CP::P];           // staged slots of each pair's atoms (-1: not staged)
    int inc_start[CP::A + 1];      // incident pairs per staged atom (CSR)
    int inc_fill[CP::A];
    short inc[2 * CP::P];
    unsigned bmask[NBRICK][AWC];   // per-brick sets of the atoms whose expanded ball reaches the brick
    unsigned nbm[CP::A * AWC];     // neighbour set of every staged atom (build_neighbour_sets)
    int bcount[NBRICK];
    short queue[TILE_PTS];         // shell points
    int nq, band, next;            // queue length, band points, next queue position to take
};

// a tile that overflowed the shared-memory staging goes to the list of the
// global-memory tier: ovf[0] counts such tiles over the run, ovf[1] is the
// stage's list length, ovf[2..] the global tiles
__device__ __forceinline__ void ovf_push(int *ovf, long long gt)
{
    atomicAdd(&ovf[0], 1);
    const int k = atomicAdd(&ovf[1], 1);
    ovf[2 + k] = (int)gt;
}

__device__ __forceinline__ void brick_point(int brick, int lane, int &li, int &lj, int &lk)
{
    int bi = brick >> 2, bj = (brick >> 1) & 1, bk = brick & 1;
    li = bi * 2 + (lane >> 4);
    lj = bj * 4 + ((lane >> 2) & 3);
    lk = bk * 4 + (lane & 3);
}

// tile-frame coordinate of local point k: FP32 table, or FP64 k * h
template <class T>
__device__ __forceinline__ T pt_coord(const Grid &G, int k)
{
    if constexpr (sizeof(T) == sizeof(float)) return G.hl[k];
    else return (double)k * G.h;
}

// per-atom incident pair lists (whole block)
template <class T, class CP>
__device__ void build_incidence(const TileS<T, CP> &S, ClsSmem<CP> &C)
{
    constexpr int A_CAP = CP::A;
    for (int a = threadIdx.x; a < A_CAP + 1; a += blockDim.x) C.inc_start[a] = 0;
    pair_slots<T>(S, C.hkey, C.hval, C.pslot);
    for (int p = threadIdx.x; p < S.np; p += blockDim.x) {
        const short2 sl = C.pslot[p];
        if (sl.x >= 0 && sl.y >= 0) {
            atomicAdd(&C.inc_start[sl.x + 1], 1);
            atomicAdd(&C.inc_start[sl.y + 1], 1);
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // inclusive scan of inc_start[1..A_CAP] by one warp
        const int lane = threadIdx.x;
        const int per = (A_CAP + 31) / 32;
        const int base = 1 + lane * per;
        int s = 0;
        for (int k = 0; k < per; ++k)
            if (base + k <= A_CAP) s += C.inc_start[base + k];
        int inc = s;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += t;
        }
        int run = inc - s;
        for (int k = 0; k < per; ++k)
            if (base + k <= A_CAP) {
                run += C.inc_start[base + k];
                C.inc_start[base + k] = run;
            }
    }
    __syncthreads();
    for (int a = threadIdx.x; a < A_CAP; a += blockDim.x) C.inc_fill[a] = C.inc_start[a];
    __syncthreads();
    for (int p = threadIdx.x; p < S.np; p += blockDim.x) {
        short2 sl = C.pslot[p];
        if (sl.x >= 0 && sl.y >= 0) {
            C.inc[atomicAdd(&C.inc_fill[sl.x], 1)] = (short)p;
            C.inc[atomicAdd(&C.inc_fill[sl.y], 1)] = (short)p;
        }
    }
    __syncthreads();
}

// Shell point: witnesses among free triple points, the containing balls and
// their pairs.  A group of G lanes (G a power of two) shares one point: the
// candidates (triple points; per containing ball its face, then its incident
// pairs) are numbered and lane r of the group tests those numbered r mod G.
// Returns this lane's part: 0 a free witness within r_p (certain), 2 one is
// undecided, 1 none; the group's label is 0 if any part is 0, else 2 if any
// part is 2, else 1 -- the label of one lane testing every candidate.  nt
// counts the atom tests of the witnesses' freeness.
template <bool FILT, class T, class CP>
__device__ int shell_part(const TileS<T, CP> &S, const ClsSmem<CP> &C, int brick, T x, T y, T z, T rp, T d0, int r,
                          int G, int &nt)
{
    SmemAcc<T, CP> A(S);
    constexpr int aw = ClsSmem<CP>::AWC;
    bool unsure = false;
    const T thr = rp, thr2 = rp * rp;
    for (int v = r; v < S.nv; v += G) {
        P4<T> q = S.vq[v];
        T dx = x - q.x, dy = y - q.y, dz = z - q.z;
        int t = lt_sq<FILT>(dx * dx + dy * dy + dz * dz, thr2, thr, d0);
        if (t == 1) return 0;
        if (t < 0) unsure = true;
    }
    const int nw = (S.na + 31) >> 5;
    int u = 0;  // candidate number
    for (int wd = 0; wd < nw; ++wd) {
      unsigned bits = C.bmask[brick][wd];
      while (bits) {
        const int a = (wd << 5) + __ffs(bits) - 1;
        bits &= bits - 1;
        P4<T> c = S.atom[a];
        T dx = x - c.x, dy = y - c.y, dz = z - c.z;
        T R = c.w + rp;
        if (lt_sq<FILT>(dx * dx + dy * dy + dz * dz, R * R, R, d0) == 0) continue;  // ball does not hold x
        if ((u & (G - 1)) == r) {
            int w = face_witness<FILT>(A, a, x, y, z, rp, thr, d0, C.nbm, aw, nt);
            if (w == 1) return 0;
            if (w < 0) unsure = true;
        }
        ++u;
        const int k0 = C.inc_start[a], k1 = C.inc_start[a + 1];
        for (int k = k0 + ((r - u) & (G - 1)); k < k1; k += G) {
            const int p = (int)C.inc[k];
            const short2 sl = C.pslot[p];
            // a pair whose other ball holds x too is tested once, under the
            // lower slot (the balls are taken in slot order; the same test
            // decides whether that ball is taken)
            const int b = sl.x == a ? sl.y : sl.x;
            if (b >= 0 && b < a && ((C.bmask[brick][b >> 5] >> (b & 31)) & 1u)) {
                const P4<T> cb = S.atom[b];
                const T ex = x - cb.x, ey = y - cb.y, ez = z - cb.z;
                const T Rb = cb.w + rp;
                if (lt_sq<FILT>(ex * ex + ey * ey + ez * ez, Rb * Rb, Rb, d0) != 0) continue;
            }
            int ws = saddle_witness<FILT>(A, p, x, y, z, rp, thr, d0, C.nbm, aw, (int)sl.x, (int)sl.y, nt);
            if (ws == 1) return 0;
            if (ws < 0) unsure = true;
        }
        u += k1 - k0;
      }
    }
    return unsure ? 2 : 1;
}

// bytes of a CTA's staging (TileS, then ClsSmem 16-byte aligned), rounded up to
// 256 so that consecutive slices of the global-memory tier stay aligned
template <class T, class CP>
__host__ __device__ constexpr size_t cls_bytes()
{
    return (((sizeof(TileS<T, CP>) + 15) & ~(size_t)15) + sizeof(ClsSmem<CP>) + 255) & ~(size_t)255;
}

// CP = CapMid: the staged lists in shared memory; a tile that overflows
// them goes to ovf.  CP = CapBig (BIG): the tiles listed in ovf, with the
// staged lists in this CTA's slice of the global scratch `big`; overflowing
// that too is a capacity error.
template <class T, bool FILT, class CP, bool BIG>
__global__ void __launch_bounds__(CLS_THREADS) k_classify(Model M, Batch B, TileSched Q, int8_t *__restrict__ labels_all,
                                                          int *__restrict__ tile_band, int *__restrict__ err,
                                                          int *__restrict__ ovf, unsigned char *__restrict__ big,
                                                          unsigned long long *__restrict__ n_tests)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *store = BIG ? big + (size_t)blockIdx.x * cls_bytes<T, CP>() : smem_raw;
    TileS<T, CP> &S = *reinterpret_cast<TileS<T, CP> *>(store);
    ClsSmem<CP> &C = *reinterpret_cast<ClsSmem<CP> *>(store + ((sizeof(TileS<T, CP>) + 15) & ~(size_t)15));
    __shared__ long long q_base;
    __shared__ Grid sG;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const T rp = (T)M.rp;
    long long iter = 0;
    int ntests = 0;  // this thread's atom tests (witness freeness)
    const long long npos = sched_count(Q, B.n_tiles);
    for (;;) {
      const long long base = next_tiles(Q, iter, &q_base);
      if (base >= npos) break;
      const long long bend = min(base + (long long)Q.per, npos);
      for (long long pos = base; pos < bend; ++pos) {
        const long long gt = sched_tile(Q, pos);
        const int mol = mol_of_tile(B, gt);
        load_grid(B, mol, sG);
        const Grid &G = sG;
        const long long tile = gt - G.tile0;
        int8_t *__restrict__ labels = labels_all + G.lab0;
        const T d0 = FILT ? (T)G.d0 : T(0);
        const T h = (T)G.h;
        double x0[3];
        stage_tile<T>(M, G, mol, tile, S, x0);
        if (!BIG && (S.flags & ERR_CAP_ANY)) {  // uniform: set before stage_tile's last barrier
            if (threadIdx.x == 0) ovf_push(ovf, gt);
            __syncthreads();
            continue;
        }
        // (the global-memory tier classifies even a tile that overflows it,
        // with its lists cut at capacity, so every label is written; the
        // error bit makes the run report ESES_ECAPACITY)
        if (threadIdx.x == 0) {
            C.nq = 0;
            C.band = 0;
            C.next = 0;
            if (S.flags) atomicOr(err, S.flags);
        }
        int t[3];
        tile_coords(G, tile, t);
        if (S.na == 0) {  // no atom within reach: every point is free
            for (int p = threadIdx.x; p < TILE_PTS; p += CLS_THREADS) {
                int li = p >> 6, lj = (p >> 3) & 7, lk = p & 7;
                long long gi = (long long)TILE * t[0] + li, gj = (long long)TILE * t[1] + lj,
                          gk = (long long)TILE * t[2] + lk;
                if (gi < G.dims[0] && gj < G.dims[1] && gk < G.dims[2])
                    labels[(gi * G.dims[1] + gj) * G.dims[2] + gk] = LABEL_OUT;
            }
            if (threadIdx.x == 0 && tile_band) tile_band[gt] = 0;
            __syncthreads();
            continue;
        }
        build_incidence<T, CP>(S, C);
        // phase 1: bricks
        for (int brick = warp; brick < NBRICK; brick += CLS_THREADS / 32) {
            int li, lj, lk;
            brick_point(brick, 0, li, lj, lk);
            const T b0x = (T)li * h, b0y = (T)lj * h, b0z = (T)lk * h;
            const T b1x = b0x + h, b1y = b0y + T(3) * h, b1z = b0z + T(3) * h;
            int cnt = 0;
            for (int base = 0; base < S.na; base += 32) {
                int a = base + lane;
                bool hit = false;
                if (a < S.na) {
                    P4<T> c = S.atom[a];
                    T ex = c.x < b0x ? b0x - c.x : (c.x > b1x ? c.x - b1x : T(0));
                    T ey = c.y < b0y ? b0y - c.y : (c.y > b1y ? c.y - b1y : T(0));
                    T ez = c.z < b0z ? b0z - c.z : (c.z > b1z ? c.z - b1z : T(0));
                    T reach = c.w + rp + T(1e-3);
                    hit = ex * ex + ey * ey + ez * ez < reach * reach;
                }
                unsigned m = __ballot_sync(0xffffffffu, hit);
                if (lane == 0) C.bmask[brick][base >> 5] = m;
                cnt += __popc(m);
            }
            if (lane == 0) C.bcount[brick] = cnt;
            __syncwarp();
            brick_point(brick, lane, li, lj, lk);
            long long gi = (long long)TILE * t[0] + li, gj = (long long)TILE * t[1] + lj,
                      gk = (long long)TILE * t[2] + lk;
            bool valid = gi < G.dims[0] && gj < G.dims[1] && gk < G.dims[2];
            int lab = LABEL_OUT;
            if (cnt > 0) {
                T x = pt_coord<T>(G, li), y = pt_coord<T>(G, lj), z = pt_coord<T>(G, lk);
                bool vdw = false, sas = false, sas_u = false;
                const int nw = (S.na + 31) >> 5;
                for (int wd = 0; wd < nw && !vdw; ++wd) {
                    unsigned bits = C.bmask[brick][wd];
                    while (bits) {
                        const int a = (wd << 5) + __ffs(bits) - 1;
                        bits &= bits - 1;
                        P4<T> c = S.atom[a];
                        T dx = x - c.x, dy = y - c.y, dz = z - c.z;
                        T d2 = dx * dx + dy * dy + dz * dz;
                        T r = c.w, R = c.w + rp;
                        if (lt_sq<FILT>(d2, r * r, r, d0) == 1) {
                            vdw = true;
                            break;
                        }
                        int s = lt_sq<FILT>(d2, R * R, R, d0);
                        if (s == 1) sas = true;
                        else if (s < 0) sas_u = true;
                    }
                }
                if (vdw) lab = LABEL_IN;
                else if (!sas) lab = sas_u ? LABEL_BAND : LABEL_OUT;
                else lab = -1;  // shell point
            }
            if (valid) {
                if (lab == -1) {
                    C.queue[atomicAdd(&C.nq, 1)] = (short)((li << 6) | (lj << 3) | lk | (brick << 9));
                } else {
                    labels[(gi * G.dims[1] + gj) * G.dims[2] + gk] = (int8_t)lab;
                    if (FILT && lab == LABEL_BAND) atomicAdd(&C.band, 1);
                }
            }
        }
        __syncthreads();
        const int nq = C.nq;
        if (nq > 0) {  // neighbour sets for the witnesses' freeness tests
            build_neighbour_sets<T, CP>(S, C.nbm, rp);
            __syncthreads();
        }
        // phase 2: shell points, the whole block; with few points, groups of
        // up to 32 lanes share one (so a tile's last point is not left to one
        // lane).  A thread (or group) takes the next point from a block counter
        // when it is done, so the slow points do not pile up on a few threads.
        int gs = 1;
        while (gs < 32 && nq * gs * 2 <= CLS_THREADS) gs <<= 1;
        const int r = lane & (gs - 1);
        const unsigned gmask = (gs == 32 ? 0xffffffffu : ((1u << gs) - 1u)) << (lane & ~(gs - 1));
        for (;;) {
            int k = 0;
            if (r == 0) k = atomicAdd(&C.next, 1);
            k = __shfl_sync(gmask, k, lane & ~(gs - 1));
            if (k >= nq) break;
            int code = C.queue[k];
            int brick = (code >> 9) & 15;
            int li = (code >> 6) & 7, lj = (code >> 3) & 7, lk = code & 7;
            T x = pt_coord<T>(G, li), y = pt_coord<T>(G, lj), z = pt_coord<T>(G, lk);
            int part = shell_part<FILT, T, CP>(S, C, brick, x, y, z, rp, d0, r, gs, ntests);
            // group label: 0 if any part found a witness, else 2 if any is undecided, else 1
            for (int o = 1; o < gs; o <<= 1) {
                const int q = __shfl_xor_sync(gmask, part, o);
                part = (part == 0 || q == 0) ? 0 : max(part, q);
            }
            if (r == 0) {
                long long gi = (long long)TILE * t[0] + li, gj = (long long)TILE * t[1] + lj,
                          gk = (long long)TILE * t[2] + lk;
                labels[(gi * G.dims[1] + gj) * G.dims[2] + gk] = (int8_t)part;
                if (FILT && part == LABEL_BAND) atomicAdd(&C.band, 1);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0 && tile_band) tile_band[gt] = C.band;
        __syncthreads();
      }
    }
    unsigned long long nw = (unsigned long long)ntests;
    for (int o = 16; o > 0; o >>= 1) nw += __shfl_down_sync(0xffffffffu, nw, o);
    if (lane == 0 && nw && n_tests) atomicAdd(n_tests, nw);
}

// The undecided points of global tile gt re-labelled in FP64 (whole block):
// one warp per point runs the witness search over every staged item.  A tile
// that overflows the staging goes to ovf (or, in the global-memory tier, is a
// capacity error).
template <class CP>
__device__ void band_tile(const Model &M, const Batch &B, long long gt, int8_t *__restrict__ labels_all,
                          TileS<double, CP> &S, Grid &sG, short *s_pts, int &s_np, int *err, int *ovf, bool big)
{
    const int mol = mol_of_tile(B, gt);
    load_grid(B, mol, sG);
    const Grid &G = sG;
    const long long tile = gt - G.tile0;
    int8_t *__restrict__ labels = labels_all + G.lab0;
    double x0[3];
    stage_tile<double>(M, G, mol, tile, S, x0);
    if (!big && (S.flags & ERR_CAP_ANY)) {  // the global-memory tier relabels even an overflowing tile
        if (threadIdx.x == 0) ovf_push(ovf, gt);
        __syncthreads();
        return;
    }
    if (threadIdx.x == 0 && S.flags) atomicOr(err, S.flags);
    int t[3];
    tile_coords(G, tile, t);
    SmemAcc<double, CP> A(S);
    // the tile's undecided points, then one warp per point: the FP64
    // witness search (a free probe centre closer than r_p: outside)
    if (threadIdx.x == 0) s_np = 0;
    __syncthreads();
    for (int p = threadIdx.x; p < TILE_PTS; p += CLS_THREADS) {
        int li = p >> 6, lj = (p >> 3) & 7, lk = p & 7;
        long long gi = (long long)TILE * t[0] + li, gj = (long long)TILE * t[1] + lj, gk = (long long)TILE * t[2] + lk;
        if (gi >= G.dims[0] || gj >= G.dims[1] || gk >= G.dims[2]) continue;
        if (labels[(gi * G.dims[1] + gj) * G.dims[2] + gk] == LABEL_BAND) s_pts[atomicAdd(&s_np, 1)] = (short)p;
    }
    __syncthreads();
    const int npts = s_np;
    for (int k = threadIdx.x >> 5; k < npts; k += CLS_THREADS / 32) {
        const int p = s_pts[k];
        const int li = p >> 6, lj = (p >> 3) & 7, lk = p & 7;
        unsigned um_p, um_v;
        const int r = warp_witness<false>(A, (double)li * G.h, (double)lj * G.h, (double)lk * G.h, M.rp, M.rp, 0.0, -1,
                                          -1, um_p, um_v);
        if ((threadIdx.x & 31) == 0) {
            const long long gi = (long long)TILE * t[0] + li, gj = (long long)TILE * t[1] + lj,
                            gk = (long long)TILE * t[2] + lk;
            labels[(gi * G.dims[1] + gj) * G.dims[2] + gk] = r == 1 ? LABEL_OUT : LABEL_IN;
        }
    }
    __syncthreads();
}

template <class CP>
__host__ __device__ constexpr size_t band_bytes()
{
    return (sizeof(TileS<double, CP>) + 255) & ~(size_t)255;
}

// CapSmall: chunks of CLS_THREADS tiles, the threads pick out the tiles with
// undecided points, then the block re-labels them one after the other.
// CapBig (BIG): the tiles listed in ovf, staged in global memory.
template <class CP, bool BIG>
__global__ void __launch_bounds__(CLS_THREADS) k_band(Model M, Batch B, int8_t *__restrict__ labels_all,
                                                      const int *__restrict__ tile_band, int *__restrict__ err,
                                                      int *__restrict__ ovf, unsigned char *__restrict__ big)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *store = BIG ? big + (size_t)blockIdx.x * band_bytes<CP>() : smem_raw;
    TileS<double, CP> &S = *reinterpret_cast<TileS<double, CP> *>(store);
    __shared__ Grid sG;
    __shared__ int s_list[CLS_THREADS];
    __shared__ short s_pts[TILE_PTS];
    __shared__ int s_n, s_np;
    if (BIG) {
        const int n = ovf[1];
        for (int k = blockIdx.x; k < n; k += gridDim.x) band_tile<CP>(M, B, ovf[2 + k], labels_all, S, sG, s_pts, s_np,
                                                                     err, ovf, true);
        return;
    }
    for (long long c0 = (long long)blockIdx.x * CLS_THREADS; c0 < B.n_tiles; c0 += (long long)gridDim.x * CLS_THREADS) {
        if (threadIdx.x == 0) s_n = 0;
        __syncthreads();
        if (c0 + threadIdx.x < B.n_tiles && tile_band[c0 + threadIdx.x] != 0) s_list[atomicAdd(&s_n, 1)] = threadIdx.x;
        __syncthreads();
        const int nband = s_n;
        for (int q = 0; q < nband; ++q)
            band_tile<CP>(M, B, c0 + s_list[q], labels_all, S, sG, s_pts, s_np, err, ovf, false);
    }
}

static long long g_band_grid = 1;  // resident k_band CTAs on the device
static int g_n_sm = 1;              // SMs: the grid of the global-memory tier

// dynamic shared memory limits and the band kernel's grid (once per device,
// before any launch or capture)
void classify_init()
{
    cudaFuncSetAttribute(k_classify<double, false, CapMid, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)cls_bytes<double, CapMid>());
    cudaFuncSetAttribute(k_classify<float, true, CapMid, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)cls_bytes<float, CapMid>());
    cudaFuncSetAttribute(k_band<CapSmall, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)band_bytes<CapSmall>());
    int dev = 0, n_sm = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_band<CapSmall, false>, CLS_THREADS,
                                                  band_bytes<CapSmall>());
    g_n_sm = n_sm > 0 ? n_sm : 1;
    g_band_grid = (long long)g_n_sm * (per_sm > 0 ? per_sm : 1);
}

// bytes of global scratch the global-memory tier of the classification and
// the band re-labelling need (one slice per CTA, one CTA per SM)
size_t classify_big_bytes()
{
    size_t per = cls_bytes<double, CapBig>();
    if (cls_bytes<float, CapBig>() > per) per = cls_bytes<float, CapBig>();
    if (band_bytes<CapBig>() > per) per = band_bytes<CapBig>();
    return per * (size_t)g_n_sm;
}

int classify_ctas_per_sm(int precision)
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    if (precision == 0)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_classify<double, false, CapMid, false>, CLS_THREADS,
                                                      cls_bytes<double, CapMid>());
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_classify<float, true, CapMid, false>, CLS_THREADS,
                                                      cls_bytes<float, CapMid>());
    return n > 0 ? n : 1;
}

// the shared-memory tier over the scheduled tiles, then the global-memory
// tier over the tiles that overflowed it (ovf: count, then tiles)
int launch_classify(const Model &M, const Batch &B, int precision, const TileSched &Q, int grid, int8_t *labels,
                    int *tile_band, int *err, int *ovf, unsigned char *big, unsigned long long *n_tests,
                    cudaStream_t st)
{
    if (grid < 1) grid = 1;
    cudaMemsetAsync(ovf + 1, 0, sizeof(int), st);
    TileSched QB{nullptr, 1, ovf + 2, ovf + 1};
    if (precision == 0) {
        k_classify<double, false, CapMid, false><<<grid, CLS_THREADS, cls_bytes<double, CapMid>(), st>>>(
            M, B, Q, labels, tile_band, err, ovf, nullptr, n_tests);
        k_classify<double, false, CapBig, true><<<g_n_sm, CLS_THREADS, 0, st>>>(M, B, QB, labels, tile_band, err, ovf,
                                                                               big, n_tests);
    } else {
        k_classify<float, true, CapMid, false><<<grid, CLS_THREADS, cls_bytes<float, CapMid>(), st>>>(
            M, B, Q, labels, tile_band, err, ovf, nullptr, n_tests);
        k_classify<float, true, CapBig, true><<<g_n_sm, CLS_THREADS, 0, st>>>(M, B, QB, labels, tile_band, err, ovf,
                                                                             big, n_tests);
    }
    return 2;
}

int launch_band(const Model &M, const Batch &B, int8_t *labels, const int *tile_band, int *err, int *ovf,
                unsigned char *big, cudaStream_t st)
{
    const long long chunks = (B.n_tiles + CLS_THREADS - 1) / CLS_THREADS;
    const long long grid = chunks < 1 ? 1 : (chunks < g_band_grid ? chunks : g_band_grid);
    cudaMemsetAsync(ovf + 1, 0, sizeof(int), st);
    k_band<CapSmall, false><<<(int)grid, CLS_THREADS, band_bytes<CapSmall>(), st>>>(M, B, labels, tile_band, err, ovf,
                                                                                 nullptr);
    k_band<CapBig, true><<<g_n_sm, CLS_THREADS, 0, st>>>(M, B, labels, tile_band, err, ovf, big);
    return 2;
}

}  // namespace eses
