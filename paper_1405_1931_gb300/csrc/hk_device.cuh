// hk_device.cuh -- device-side data structures, PTX helpers (TMA, mbarrier,
// cp.async) and the union-find primitives of the labelling passes.
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
#include <cuda.h>
#include <cuda_runtime.h>

namespace hk {

constexpr int TX = 32;
// Run codes (one uint16 per x-run, written by the tile pass, decoded by flatten):
//   CODE_BOUNDARY | k               a run of boundary piece k of the tile
//   CODE_BOUNDARY | CODE_ROOT | k   the first run of boundary piece k
//   CODE_ROOT | size                the first run of an interior piece (its size, <= 8192)
//   (row << 5) | x0  (< CODE_ROOT)  another run of the interior piece whose first run starts
//                                   at tile row `row`, column x0
constexpr uint16_t CODE_BOUNDARY = 0x8000;
constexpr uint16_t CODE_ROOT = 0x4000;
constexpr uint16_t CODE_LOW = 0x3fff;

// One lattice of a launch.  Every pass works on the concatenated tiles of all
// lattices; tile0/seg0/row0 locate this lattice's slice of the global tile,
// segment and row index spaces.  A segment is one tile row: 32 consecutive x
// sites; a row is one lattice row (all x at one y, z).
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
    int occ_mode;    // 0: occupied iff phi > 0; 1: iff phi < -0.5 (far sites of an index field)
    int8_t *inside;  // interior/exterior tag per cluster (index fields), or nullptr
    int64_t tile0;   // first global tile id
    int64_t seg0;    // first global segment id (row-major: ((z*ny + y)*nbx + bx))
    int64_t row0;    // first global row id (z*ny + y)
};

// The lattices of one launch (a kernel parameter).
template <int NL>
struct LatBatch {
    int n;
    int pad_;
    LatDev lat[NL];
};

// Workspace pointers shared by all passes of one launch.
struct Work {
    uint32_t *mask;     // [ntiles * R] occupancy words, tile-major (tile t, row r)
    uint16_t *codes;    // [ntiles * MAXRUNS] one code per run (CODE_* above)
    uint8_t *cnt;       // [nseg] cluster roots per segment (row-major segment order; <= 16)
    uint32_t *pre;      // [nrows + 1] exclusive prefix of the roots per lattice row
    uint32_t *bsum;     // [nblocks] scan block sums
    uint16_t *face;     // [ntiles * face_stride] per-face lists of boundary-piece numbers
    int4 *tinfo;        // [ntiles] (piece base, piece count, run count, 0) of each tile
    int32_t *parent;    // [piece_cap] union-find parent over boundary pieces; tile t owns
                        // the slice [t * MAX_BOUNDARY, t * MAX_BOUNDARY + piece count)
    int32_t *key;       // [piece_cap] lattice-local site index of the piece's first site;
                        // after piece_finalize: the label of the piece's cluster
    int32_t *psize;     // [piece_cap] piece size; after piece_finalize: the cluster size at
                        // the cluster's root piece, -1 elsewhere
    uint32_t *xcol;     // [ntiles * 2 * R/32] occupancy of each tile's first (x = 0) and last
                        // (x = lastX) column, one bit per tile row
    int32_t *status;    // [1] device-side error flags (STATUS_*), owned by the context
    uint32_t *rootbits; // [nseg] cluster-root run starts of each row segment (index fields only)
    uint32_t *segpre;   // [nseg] clusters ranked before each row segment (index fields only)
    int32_t *votes;     // [sizes_cap] sign votes per cluster (index fields only)
    int32_t *ovf;       // [ntiles] tiles with more runs than the fast tile pass holds
    int32_t *novf;      // [1] entries of ovf (reset by the occupancy pass of every call)
    int64_t piece_cap;  // bound of every global union-find loop: the entries of parent/key/psize
                        // (a path visits distinct pieces), or a lower test bound
    int32_t local_cap;  // bound of the shared-memory union retries: 0 = the tile's run count,
                        // > 0 a lower test bound
    // one slab of a lattice split along z (single-lattice launches only): added to every
    // label, the index of the slab's first site in the whole lattice (else 0); and, when
    // not null, the label of each cluster in rank order (sizes_cap entries, like sizes)
    int64_t site_off;
    int32_t *roots;
};

// Tensor maps of the single-lattice fast path (TMA tile loads of phi and TMA
// tile stores of labels).  Unused when `valid` is 0.
struct TmapPair {
    CUtensorMap phi;
    CUtensorMap labels;
    int valid;
};

// The tensor maps of every lattice of a launch (kernel parameters, so graphs keep them
// by value).
template <int NL>
struct TmapBatch {
    TmapPair tm[NL];
};

// A union-find path longer than the number of its nodes means corrupted
// parents, and a TMA wait that never completes means a lost copy; every loop
// below is capped, and on reaching the cap it records one of these flags and
// stops instead of spinning.
constexpr int32_t STATUS_LOCAL_LOOP = 1;
constexpr int32_t STATUS_GLOBAL_LOOP = 2;
constexpr int32_t STATUS_TMA_TIMEOUT = 4;

template <int TY, int TZ>
struct TileShape {
    static constexpr int R = TY * TZ;            // rows per tile
    static constexpr int SITES = TX * R;
    static constexpr int MAXRUNS = 16 * R;       // at most 16 runs in a 32-site row
    // Run (and union-pair) capacity of the fast tile pass: 9 runs a row on average,
    // above the 8 of the densest i.i.d. field (p = 1/2), and small enough that eight
    // CTAs of the pass share an SM.  Tiles beyond it go to a second pass sized for
    // MAXRUNS.
    static constexpr int MR_FAST = 9 * R;
    static constexpr int NT = R;                 // threads per CTA: one per row
    // Face lists inside a tile's face block: 8 counts (one per face, two unused),
    // then per face the boundary numbers of its emitted connected sites.  Emitted
    // sites are pairwise non-adjacent along x (y and z faces: at most 16 a row) or
    // along y (x faces: at most R / 2).
    static constexpr int OFF_CNT = 0;                     // [6] lo-x, hi-x, lo-y, hi-y, lo-z, hi-z
    static constexpr int OFF_LX = 8;
    static constexpr int OFF_HX = 8 + R / 2;
    static constexpr int OFF_LY = 8 + R;
    static constexpr int OFF_HY = 8 + R + 16 * TZ;
    static constexpr int OFF_LZ = 8 + R + 32 * TZ;
    static constexpr int OFF_HZ = 8 + R + 32 * TZ + 16 * TY;
    static constexpr int FACE_STRIDE = 8 + R + 32 * TZ + 32 * TY;
    // rows with ly = 0 inside a 32-row word (x-face lists)
    static constexpr uint32_t LY0 = TY == 8 ? 0x01010101u : TY == 16 ? 0x00010001u : 0x00000001u;
    static_assert(TY == 8 || TY == 16 || TY == 32, "tile rows along y");
    // Upper bound on boundary pieces of one tile: pieces touching one face are
    // pairwise non-adjacent on that face's 2D grid, so at most ceil(area/2) of
    // them touch it.
    static constexpr int MAX_BOUNDARY = (R + 1) / 2 * 2 + (TX * TZ + 1) / 2 * 2 + (TX * TY + 1) / 2 * 2;
};

// Tile geometry of global tile t.
struct TileGeo {
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

// the lattice holding global row q
__device__ __forceinline__ int find_lattice_row(const LatDev *lats, int nlat, int64_t q) {
    int lo = 0, hi = nlat - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (lats[mid].row0 <= q) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <int TY, int TZ>
__device__ __forceinline__ TileGeo tile_geo(const LatDev &L, int64_t t) {
    TileGeo g;
    // a lattice has fewer than 2^31 sites, so its tile index fits in 32 bits
    const uint32_t lt = (uint32_t)(t - L.tile0);
    const uint32_t q = lt / (uint32_t)L.nbx;
    g.bx = (int)(lt - q * (uint32_t)L.nbx);
    g.bz = (int)(q / (uint32_t)L.nby);
    g.by = (int)(q - (uint32_t)g.bz * (uint32_t)L.nby);
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

// Occupancy of a site: phi > 0 (Sec. 2); for an index field (Sec. 6, step 4) the
// sites far from every membrane, I < -0.5.  NaN is never occupied.
__device__ __forceinline__ bool occupied(float v, int mode) { return mode ? (v < -0.5f) : (v > 0.0f); }

__device__ __forceinline__ uint32_t run_starts(uint32_t m) { return m & ~(m << 1); }
// the last site of every run: bit x set when x is occupied and x + 1 is not (or x = 31)
__device__ __forceinline__ uint32_t run_ends(uint32_t m) { return m & ~(m >> 1); }
// bits 0..x set
__device__ __forceinline__ uint32_t le_mask(int x) { return (2u << x) - 1u; }
// run id (within the tile) of occupied site x of a row with run starts rs
__device__ __forceinline__ int run_of(int rbase, uint32_t rs, int x) { return rbase + __popc(rs & le_mask(x)) - 1; }
// length of the run starting at bit x0 of m: the first run end at or above x0, which
// __ffs counts from 1
__device__ __forceinline__ int run_len(uint32_t m, int x0) { return __ffs(run_ends(m) >> x0); }

// ---- PTX helpers ----------------------------------------------------------------------
// Programmatic dependent launch: the kernels of the labelling sequence are launched so
// that one may be set up while the previous one is still finishing.  Each waits here,
// before its first access to global memory, until the previous kernel of the stream has
// completed and its writes are visible (a kernel launched without that attribute
// returns at once).
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// TMA tile load of box (32, TY, TZ) at element coordinates (x, y, z); x*4 bytes is a multiple of 16.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned) from global to
// shared memory, completed on an mbarrier.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// TMA tile store; elements outside the tensor are not written.  Coordinates are never negative.
__device__ __forceinline__ void tma_store_3d(const CUtensorMap *map, const void *src, int x, int y, int z) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];"
                 ::"l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// 4-byte asynchronous global->shared copy; src_bytes == 0 writes a zero.
__device__ __forceinline__ void cp_async4(void *dst, const void *src, int src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Wait for phase `parity` of an mbarrier with an iteration cap; returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    for (uint32_t it = 0; it < (1u << 26); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// ---- shared-memory union-find over run ids (union by minimum id) ----------------------
// Every store to par[] lowers it to an ancestor (a root is linked to a smaller id
// of the other tree, halving stores a grandparent, compression stores the root),
// so par[i] <= i always holds and a find walks strictly decreasing ids: it ends
// within i steps by construction.  For the same reason the finds use plain loads: a
// value that another thread has since lowered is still an ancestor.  Linking goes
// through atomicMin, whose old value tells whether a root was still a root.  The
// union's retry loop is the one that depends on other threads, and it keeps an
// explicit bound.

// read-only find: used by compression, where finds run while others store final
// roots (a halving store there could overwrite a final root with an ancestor)
__device__ __forceinline__ int s_find_ro(const int *par, int x) {
    int p = par[x];
    while (p != x) {
        x = p;
        p = par[x];
    }
    return x;
}

// find with path splitting (during the unions): every node passed is pointed at its
// grandparent, an ancestor, so concurrent finds and links stay valid
__device__ __forceinline__ int s_find(int *par, int x) {
    int p = par[x];
    while (p != x) {
        const int gp = par[p];
        if (gp == p) return p;
        par[x] = gp;
        x = p;
        p = gp;
    }
    return x;
}

// Each retry strictly lowers max(a, b), so at most `cap` rounds.
__device__ __forceinline__ void s_union(int *par, int a, int b, int cap, int32_t *status) {
    for (int it = 0; it <= cap; ++it) {
        a = s_find(par, a);
        b = s_find(par, b);
        if (a == b) return;
        const int hi = a > b ? a : b, lo = a > b ? b : a;
        const int old = atomicMin(&par[hi], lo);
        if (old == hi) return;
        a = lo;
        b = old;
    }
    atomicOr(status, STATUS_LOCAL_LOOP);
}

// join the runs of row r and row q that overlap along x (used for the rare in-tile wraps)
__device__ __forceinline__ void join_rows(int *par, uint32_t m, int rb, uint32_t mq, int rbq, int cap,
                                          int32_t *status) {
    uint32_t o = m & mq;
    if (!o) return;
    const uint32_t rs = run_starts(m), rsq = run_starts(mq);
    uint32_t os = run_starts(o);
    while (os) {
        int x = __ffs(os) - 1;
        os &= os - 1;
        s_union(par, run_of(rb, rs, x), run_of(rbq, rsq, x), cap, status);
    }
}

// Sum of the first n (<= 8) bytes of w, each at most 16: the multiply adds every byte
// into the top one, which holds the sum (at most 128).
__device__ __forceinline__ uint32_t bytes8_sum(uint64_t w, int n) {
    const uint64_t keep = n >= 8 ? ~0ull : (n <= 0 ? 0ull : (1ull << (8 * n)) - 1ull);
    return (uint32_t)(((w & keep) * 0x0101010101010101ull) >> 56);
}

// Sum of the n bytes at base[start, start + n), each at most 16.  A range of at most 32
// bytes that starts 16-byte aligned (a lattice row of up to 32 segments) is read as two
// 16-byte loads issued together; any other range as the aligned 32-bit words that cover
// it (the bytes outside the range are masked off).  The array must extend to the end of
// the 16-byte block holding its last byte.
__device__ __forceinline__ uint32_t bytes_sum(const uint8_t *base, int64_t start, int64_t n) {
    if (n <= 32 && (start & 15) == 0) {
        if (n <= 0) return 0;
        const ulonglong2 a = *reinterpret_cast<const ulonglong2 *>(base + start);
        const ulonglong2 b = n > 16 ? *reinterpret_cast<const ulonglong2 *>(base + start + 16) : make_ulonglong2(0, 0);
        const int k = (int)n;
        return bytes8_sum(a.x, k) + bytes8_sum(a.y, k - 8) + bytes8_sum(b.x, k - 16) + bytes8_sum(b.y, k - 24);
    }
    uint32_t s = 0;
    const int64_t e = start + n;
    for (int64_t w = start & ~(int64_t)3; w < e; w += 4) {
        const uint32_t v = *reinterpret_cast<const uint32_t *>(base + w);
        const int lo = start > w ? (int)(start - w) : 0;    // keep bytes [lo, hi) of the word
        const int hi = e - w < 4 ? (int)(e - w) : 4;
        const uint32_t keep = (hi == 4 ? 0xffffffffu : ((1u << (8 * hi)) - 1u)) & ~((1u << (8 * lo)) - 1u);
        s = __dp4a(v & keep, 0x01010101u, s);
    }
    return s;
}

// Block-wide exclusive scan of one int per thread (blockDim.x == NT, NT % 32 == 0, NT <= 992).
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


// ---- global union-find over boundary pieces --------------------------------------------
// Links go from a root to a root with a smaller key (the piece's first site), so
// keys strictly decrease along parent pointers and each cluster's root is the
// piece holding the cluster's smallest site index.  The parent array is kept at
// 4 bytes a piece: finds hop across the whole table, so its footprint in L2 matters.
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

// The finds of a and b with path halving, walked in lockstep so that the loads of
// both chains are in flight together.
__device__ __forceinline__ void g_find_pair(int32_t *parent, int &a, int &b, int64_t cap, int32_t *status) {
    int pa = __ldcg(parent + a), pb = __ldcg(parent + b);
    for (int64_t it = 0; pa != a || pb != b; ++it) {
        if (it > cap) { atomicOr(status, STATUS_GLOBAL_LOOP); return; }
        const bool ma = pa != a, mb = pb != b;       // chains not yet at a root
        const int ga = ma ? __ldcg(parent + pa) : a;
        const int gb = mb ? __ldcg(parent + pb) : b;
        bool la = false, lb = false;                 // parent of the new a / b still to load
        if (ma) {
            if (ga == pa) {
                a = pa;                              // pa is a root
                pa = a;
            } else {
                __stcg(parent + a, ga);              // path halving: ga is an ancestor of a
                a = ga;
                la = true;
            }
        }
        if (mb) {
            if (gb == pb) {
                b = pb;
                pb = b;
            } else {
                __stcg(parent + b, gb);
                b = gb;
                lb = true;
            }
        }
        if (la) pa = __ldcg(parent + a);
        if (lb) pb = __ldcg(parent + b);
    }
}

// A failed CAS means b was linked meanwhile, which lowers the key of b's root;
// keys are distinct, so at most `cap` retries.
__device__ __forceinline__ void g_union(int32_t *parent, const int32_t *key, int a, int b, int64_t cap,
                                        int32_t *status) {
    for (int64_t it = 0; it <= cap; ++it) {
        g_find_pair(parent, a, b, cap, status);
        if (a == b) return;
        if (__ldg(key + b) < __ldg(key + a)) { int t = a; a = b; b = t; }
        if (atomicCAS(parent + b, b, a) == b) return;
    }
    atomicOr(status, STATUS_GLOBAL_LOOP);
}

}  // namespace hk
