// hk_device.cuh -- device-side data structures and the tile-local labelling
// shared by the tile pass (K1) and the flatten pass (K4).
//
// Tiles are 32 sites along x (one 32-bit occupancy word per tile row) by TY
// rows along y by TZ planes along z.  Inside a tile the Hoshen-Kopelman raster
// scan of Sec. 2 is replaced by union-find over x-runs: a run is a maximal
// stretch of occupied sites along x within one tile row, runs are numbered in
// row-major order, and runs of neighbouring rows (y-1, z-1) that overlap are
// joined.  Union is by minimum run id, so every piece's root is its first run
// in row-major order, i.e. the run holding the piece's smallest site index --
// the same "smallest possible number" that Sec. 2's relabelling produces.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hk {

constexpr int TX = 32;
constexpr uint16_t FACE_NONE = 0xFFFF;

// One lattice of a launch.  Every pass works on the concatenated tiles of all
// lattices; tile0/seg0 locate this lattice's slice of the global tile and
// segment index spaces.  A segment is one tile row: 32 consecutive x sites.
struct LatDev {
    const float *phi;
    int32_t *labels;
    int64_t *sizes;
    int64_t sizes_cap;
    int64_t *hist;
    int64_t *ncl;
    int nx, ny, nz;
    int per[3];
    int nbx, nby, nbz;
    int pad_;
    int64_t tile0;   // first global tile id
    int64_t seg0;    // first global segment id (row-major: ((z*ny + y)*nbx + bx))
};

// Workspace pointers shared by all passes of one launch.
struct Work {
    uint32_t *mask;     // [ntiles * R] occupancy words, tile-major (tile t, row r)
    uint32_t *cnt;      // [nseg] cluster roots per segment (row-major segment order)
    uint32_t *pre;      // [nseg + 1] exclusive prefix of cnt
    uint32_t *bsum;     // [nblocks] scan block sums
    uint16_t *face;     // [ntiles * face_stride] boundary-piece numbers of face sites
    int2 *tinfo;        // [ntiles] (piece base, piece count) of each tile
    int32_t *parent;    // [piece_cap] union-find parent over boundary pieces
    int32_t *key;       // [piece_cap] lattice-local site index of the piece's first site
    int32_t *psize;     // [piece_cap] piece size, then cluster size at cluster roots
    int32_t *npieces;   // [1] piece allocation counter
    int32_t *status;    // [1] device-side error flags (STATUS_*), owned by the context
    int64_t piece_cap;  // entries of parent/key/psize: bounds every union-find path
};

// A union-find path longer than the number of its nodes means corrupted
// parents; every loop below is capped by that count, and on reaching the cap
// it records one of these flags and stops instead of spinning.
constexpr int32_t STATUS_LOCAL_LOOP = 1;
constexpr int32_t STATUS_GLOBAL_LOOP = 2;

template <int TY, int TZ>
struct TileShape {
    static constexpr int R = TY * TZ;            // rows per tile
    static constexpr int MAXRUNS = 16 * R;       // at most 16 runs in a 32-site row
    static constexpr int NT = R;                 // one thread per row
    // face layout inside a tile's face block
    static constexpr int OFF_LX = 0;
    static constexpr int OFF_HX = R;
    static constexpr int OFF_LY = 2 * R;                 // [lz][x]
    static constexpr int OFF_HY = 2 * R + TX * TZ;
    static constexpr int OFF_LZ = 2 * R + 2 * TX * TZ;   // [ly][x]
    static constexpr int OFF_HZ = 2 * R + 2 * TX * TZ + TX * TY;
    static constexpr int FACE_STRIDE = 2 * R + 2 * TX * TZ + 2 * TX * TY;
    // Upper bound on boundary pieces of one tile: pieces touching one face are
    // pairwise non-adjacent on that face's 2D grid, so at most ceil(area/2) of
    // them touch it.
    static constexpr int MAX_BOUNDARY = (R + 1) / 2 * 2 + (TX * TZ + 1) / 2 * 2 + (TX * TY + 1) / 2 * 2;
};

template <int TY, int TZ>
struct TileSmem {
    using S = TileShape<TY, TZ>;
    uint32_t m[S::R];           // occupancy word of each row
    int rbase[S::R];            // first run id of each row
    int par[S::MAXRUNS];        // union-find over run ids (par[i] <= i)
    int aux[S::MAXRUNS];        // per root: piece size, later the final label
    int kmap[S::MAXRUNS];       // per boundary root: boundary number inside the tile
    uint32_t bflag[S::MAXRUNS / 32];   // boundary flag per run id (meaningful at roots)
    int warp_tmp[32];
    int nruns;
    int nbound;
    int base;
    int hist[32];
};

// Tile geometry of global tile t.
struct TileGeo {
    int lat;
    int bx, by, bz;
    int x0, y0, z0;
    int lastX, lastY, lastZ;    // last valid local coordinate (ragged edges)
    bool extXlo, extXhi, extYlo, extYhi, extZlo, extZhi;   // faces with a neighbour tile
    bool wrapX, wrapY, wrapZ;   // periodic edge inside this tile (axis spans one tile)
};

__device__ __forceinline__ int find_lattice(const LatDev *lats, int nlat, int64_t t) {
    int lo = 0, hi = nlat - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (lats[mid].tile0 <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <int TY, int TZ>
__device__ __forceinline__ TileGeo tile_geo(const LatDev &L, int lat, int64_t t) {
    TileGeo g;
    g.lat = lat;
    int64_t lt = t - L.tile0;
    g.bx = (int)(lt % L.nbx);
    int64_t q = lt / L.nbx;
    g.by = (int)(q % L.nby);
    g.bz = (int)(q / L.nby);
    g.x0 = g.bx * TX; g.y0 = g.by * TY; g.z0 = g.bz * TZ;
    g.lastX = min(TX, L.nx - g.x0) - 1;
    g.lastY = min(TY, L.ny - g.y0) - 1;
    g.lastZ = min(TZ, L.nz - g.z0) - 1;
    const bool px = L.per[0] && L.nbx >= 2, py = L.per[1] && L.nby >= 2, pz = L.per[2] && L.nbz >= 2;
    g.extXlo = g.bx > 0 || px; g.extXhi = g.bx < L.nbx - 1 || px;
    g.extYlo = g.by > 0 || py; g.extYhi = g.by < L.nby - 1 || py;
    g.extZlo = g.bz > 0 || pz; g.extZhi = g.bz < L.nbz - 1 || pz;
    g.wrapX = L.per[0] && L.nbx == 1 && L.nx >= 2;
    g.wrapY = L.per[1] && L.nby == 1 && L.ny >= 2;
    g.wrapZ = L.per[2] && L.nbz == 1 && L.nz >= 2;
    return g;
}

__device__ __forceinline__ uint32_t run_starts(uint32_t m) { return m & ~(m << 1); }
// bits 0..x set
__device__ __forceinline__ uint32_t le_mask(int x) { return (2u << x) - 1u; }
// run id (global within the tile) of occupied site x of a row with run starts rs
__device__ __forceinline__ int run_of(int rbase, uint32_t rs, int x) { return rbase + __popc(rs & le_mask(x)) - 1; }

// ---- shared-memory union-find over run ids (union by minimum id) ----------------------
// par[i] <= i always holds, so a path visits at most `cap` (= number of runs) ids.
__device__ __forceinline__ int s_find(int *par, int x, int cap, int32_t *status) {
    volatile int *vp = par;
    int p = vp[x];
    for (int it = 0; p != x; ++it) {
        if (it > cap) { atomicOr(status, STATUS_LOCAL_LOOP); return x; }
        int gp = vp[p];
        if (gp == p) return p;
        vp[x] = gp;          // path halving: gp is an ancestor of x
        x = gp;
        p = vp[x];
    }
    return x;
}

// Read-only find for the compression step: without halving stores, no thread
// can overwrite another thread's final par[i] = root with an older ancestor.
__device__ __forceinline__ int s_find_ro(const int *par, int x, int cap, int32_t *status) {
    const volatile int *vp = par;
    int p = vp[x];
    for (int it = 0; p != x; ++it) {
        if (it > cap) { atomicOr(status, STATUS_LOCAL_LOOP); return x; }
        x = p;
        p = vp[x];
    }
    return x;
}

// Each retry strictly lowers b, so at most `cap` rounds.
__device__ __forceinline__ void s_union(int *par, int a, int b, int cap, int32_t *status) {
    for (int it = 0; it <= cap; ++it) {
        a = s_find(par, a, cap, status);
        b = s_find(par, b, cap, status);
        if (a == b) return;
        if (a > b) { int t = a; a = b; b = t; }
        int old = atomicMin(&par[b], a);
        if (old == b) return;
        b = old;
    }
    atomicOr(status, STATUS_LOCAL_LOOP);
}

// join the runs of row r and row q that overlap along x
__device__ __forceinline__ void join_rows(int *par, uint32_t m, uint32_t rs, int rb, uint32_t mq, int rbq, int cap,
                                          int32_t *status) {
    uint32_t o = m & mq;
    if (!o) return;
    uint32_t os = run_starts(o);
    uint32_t rsq = run_starts(mq);
    while (os) {
        int x = __ffs(os) - 1;
        os &= os - 1;
        s_union(par, run_of(rb, rs, x), run_of(rbq, rsq, x), cap, status);
    }
}

// Block-wide exclusive scan of one int per thread (blockDim.x == NT, NT % 32 == 0).
template <int NT>
__device__ __forceinline__ int block_exscan(int v, int *warp_tmp, int &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int u = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += u;
    }
    if (lane == 31) warp_tmp[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int w = (lane < NT / 32) ? warp_tmp[lane] : 0;
        int wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int u = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += u;
        }
        if (lane < NT / 32) warp_tmp[lane] = wi - w;
        if (lane == NT / 32 - 1) warp_tmp[31] = wi;
    }
    __syncthreads();
    int r = warp_tmp[wid] + inc - v;
    total = warp_tmp[31];
    __syncthreads();
    return r;
}

// Tile-local labelling from the occupancy words in S.m (filled by the caller).
// On return: S.par[i] is the root run of run i, S.aux[root] the piece size,
// S.bflag marks boundary roots, S.kmap[root] numbers the boundary roots in run
// order, S.nbound their count.  Identical in K1 and K4, so both derive the same
// pieces and the same boundary numbering.
template <int TY, int TZ>
__device__ void tile_local_label(TileSmem<TY, TZ> &S, const TileGeo &g, int32_t *status) {
    using SH = TileShape<TY, TZ>;
    const int r = threadIdx.x;               // one row per thread
    const int ly = r % TY, lz = r / TY;
    const uint32_t m = S.m[r];
    const uint32_t rs = run_starts(m);

    // 1. run ids: exclusive scan of run counts over rows
    int total;
    const int rb = block_exscan<SH::NT>(__popc(rs), S.warp_tmp, total);
    S.rbase[r] = rb;
    if (r == 0) S.nruns = total;
    for (int i = r; i < total; i += SH::NT) { S.par[i] = i; S.aux[i] = 0; }
    for (int i = r; i < (total + 31) / 32; i += SH::NT) S.bflag[i] = 0u;
    __syncthreads();

    // 2. unions with the y-1 and z-1 rows, and periodic edges inside the tile
    if (m) {
        if (ly > 0) join_rows(S.par, m, rs, rb, S.m[r - 1], S.rbase[r - 1], total, status);
        if (lz > 0) join_rows(S.par, m, rs, rb, S.m[r - TY], S.rbase[r - TY], total, status);
        if (g.wrapY && ly == g.lastY && ly > 0)
            join_rows(S.par, m, rs, rb, S.m[r - ly], S.rbase[r - ly], total, status);
        if (g.wrapZ && lz == g.lastZ && lz > 0)
            join_rows(S.par, m, rs, rb, S.m[r - lz * TY], S.rbase[r - lz * TY], total, status);
        if (g.wrapX && g.lastX > 0 && (m & 1u) && ((m >> g.lastX) & 1u))
            s_union(S.par, rb, run_of(rb, rs, g.lastX), total, status);
    }
    __syncthreads();

    // 3. full compression
    for (int i = r; i < total; i += SH::NT) S.par[i] = s_find_ro(S.par, i, total, status);
    __syncthreads();

    // 4. piece sizes and boundary flags
    if (m) {
        const bool face_row = (ly == 0 && g.extYlo) || (ly == g.lastY && g.extYhi) ||
                              (lz == 0 && g.extZlo) || (lz == g.lastZ && g.extZhi);
        uint32_t w = rs;
        int id = rb;
        while (w) {
            const int x0 = __ffs(w) - 1;
            w &= w - 1;
            const uint32_t v = m >> x0;                       // bit 0 is site x0
            const int len = (v == 0xffffffffu) ? 32 : __ffs(~v) - 1;
            const int root = S.par[id];
            atomicAdd(&S.aux[root], len);
            const bool touch = face_row || (x0 == 0 && g.extXlo) ||
                               (g.extXhi && x0 <= g.lastX && x0 + len - 1 >= g.lastX);
            if (touch) atomicOr(&S.bflag[root >> 5], 1u << (root & 31));
            ++id;
        }
    }
    __syncthreads();

    // 5. number the boundary roots in run order
    constexpr int PER = SH::MAXRUNS / SH::NT;   // 16 run ids per thread
    const int i0 = r * PER;
    int cnt = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int i = i0 + j;
        if (i < total && S.par[i] == i && ((S.bflag[i >> 5] >> (i & 31)) & 1u)) ++cnt;
    }
    int nb;
    int k = block_exscan<SH::NT>(cnt, S.warp_tmp, nb);
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int i = i0 + j;
        if (i < total && S.par[i] == i && ((S.bflag[i >> 5] >> (i & 31)) & 1u)) S.kmap[i] = k++;
    }
    if (r == 0) S.nbound = nb;
    __syncthreads();
}

__device__ __forceinline__ bool is_boundary(const uint32_t *bflag, int i) { return (bflag[i >> 5] >> (i & 31)) & 1u; }

// ---- global union-find over boundary pieces --------------------------------------------
// Links go from a root to a root with a smaller key (the piece's first site), so
// keys strictly decrease along parent pointers and each cluster's root is the
// piece holding the cluster's smallest site index.
// A path visits distinct pieces, so `cap` (the piece-table size) bounds it.
__device__ __forceinline__ int g_find(int32_t *parent, int x, int64_t cap, int32_t *status) {
    int p = __ldcg(parent + x);
    for (int64_t it = 0; p != x; ++it) {
        if (it > cap) { atomicOr(status, STATUS_GLOBAL_LOOP); return x; }
        int gp = __ldcg(parent + p);
        if (gp == p) return p;
        __stcg(parent + x, gp);    // path halving
        x = gp;
        p = __ldcg(parent + x);
    }
    return x;
}

// Read-only find for the compression pass: no halving writes, so the one store
// each thread makes afterwards (parent[pid] = root) cannot be overwritten by
// another thread's halving store of an older, non-root ancestor.
__device__ __forceinline__ int g_find_ro(const int32_t *parent, int x, int64_t cap, int32_t *status) {
    int p = __ldcg(parent + x);
    for (int64_t it = 0; p != x; ++it) {
        if (it > cap) { atomicOr(status, STATUS_GLOBAL_LOOP); return x; }
        x = p;
        p = __ldcg(parent + x);
    }
    return x;
}

// A failed CAS means b was linked meanwhile, which lowers the key of b's root;
// keys are distinct, so at most `cap` retries.
__device__ __forceinline__ void g_union(int32_t *parent, const int32_t *key, int a, int b, int64_t cap,
                                        int32_t *status) {
    for (int64_t it = 0; it <= cap; ++it) {
        a = g_find(parent, a, cap, status);
        b = g_find(parent, b, cap, status);
        if (a == b) return;
        if (__ldg(key + b) < __ldg(key + a)) { int t = a; a = b; b = t; }
        if (atomicCAS(parent + b, b, a) == b) return;
    }
    atomicOr(status, STATUS_GLOBAL_LOOP);
}

}  // namespace hk
