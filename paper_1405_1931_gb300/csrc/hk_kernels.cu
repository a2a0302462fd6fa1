// hk_kernels.cu -- the labelling passes.
//
//   K0 occupancy      stream phi once (coalesced row loads) and write the
//                     occupancy mask phi > 0, one 32-bit word per tile row.
//   K1 tile_label     label each tile from its mask words (Sec. 2's rules
//                     become union-find over x-runs), register boundary
//                     pieces, and write one code per run, the face summaries
//                     and the per-row count of interior cluster roots.
//   K2 face_merge     join boundary pieces across tile faces and periodic
//                     edges: the intra-GPU counterpart of Sec. 3's halo
//                     equivalences, resolved directly on a global union-find
//                     instead of being gathered to a root process.
//   K3 piece_finalize compress the union-find, add piece sizes into cluster
//                     roots and count cluster roots per row segment.
//   S1-S3 scan        exclusive prefix of the root counts: the compactified
//                     cluster numbering 1..n of Sec. 2 in row-major order.
//   K4 flatten        persistent: decode the run codes, write the labels
//                     (staged in shared memory, TMA tensor stores), the sizes
//                     in label order and the histogram.
#include <cstring>
#include <mutex>
#include <type_traits>

#include "hk_device.cuh"
#include "hk_launch.h"

namespace hk {

// --------------------------------------------------------------------------------------
// K0: occupancy.  One warp per tile streams phi row by row (one coalesced 128-byte
// load per row, 16 rows in flight per warp) and keeps phi > 0 (Sec. 2) as one
// 32-bit word per tile row, written tile-major.  Sites outside the lattice count
// as medium.
// --------------------------------------------------------------------------------------
template <int TY, int TZ, int NL>
__global__ void __launch_bounds__(256, 4) k_occupancy(const __grid_constant__ LatBatch<NL> B, Work W, int64_t ntiles) {
    grid_dep_wait();
    using SH = TileShape<TY, TZ>;
    constexpr int R = SH::R, U = 16;
    const int lane = threadIdx.x & 31;
    const int64_t t = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (blockIdx.x == 0 && threadIdx.x == 0) *W.novf = 0;   // the tile pass appends after this pass
    if (t >= ntiles) return;
    const LatDev &L = B.lat[(NL == 1) ? 0 : find_lattice(B.lat, B.n, t)];
    const TileGeo g = tile_geo<TY, TZ>(L, t);
    const int64_t sxy = (int64_t)L.nx * L.ny;
    const float *base = L.phi + (int64_t)g.z0 * sxy + (int64_t)g.y0 * L.nx + g.x0 + lane;
    const bool xin = lane <= g.lastX;
    uint32_t *out = W.mask + t * R;
    // Whole 128-byte rows at 16-byte aligned addresses: lane l loads 4 sites (x = 4 (l % 8)
    // .. + 3) of row l / 8 of each group of 4 rows, and the 8 lanes of a row OR their
    // nibbles into the row's word.
    const bool vec = g.lastX == TX - 1 && (L.nx & 3) == 0 && (reinterpret_cast<uintptr_t>(L.phi) & 15) == 0;
    const int x4 = (lane & 7) * 4;
    const float *base4 = L.phi + (int64_t)g.z0 * sxy + (int64_t)g.y0 * L.nx + g.x0 + x4;
    for (int r0 = 0; r0 < R; r0 += 32) {        // lane j keeps the word of row r0 + j
        uint32_t mine = 0;
        if (vec) {
            float4 v[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int rr = r0 + 4 * q + (lane >> 3), ly = rr % TY, lz = rr / TY;
                v[q] = (ly <= g.lastY && lz <= g.lastZ)
                           ? __ldcs(reinterpret_cast<const float4 *>(base4 + (int64_t)lz * sxy + (int64_t)ly * L.nx))
                           : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                uint32_t w = ((uint32_t)occupied(v[q].x, L.occ_mode) | ((uint32_t)occupied(v[q].y, L.occ_mode) << 1) |
                              ((uint32_t)occupied(v[q].z, L.occ_mode) << 2) | ((uint32_t)occupied(v[q].w, L.occ_mode) << 3))
                             << x4;
                w |= __shfl_xor_sync(0xffffffffu, w, 1);
                w |= __shfl_xor_sync(0xffffffffu, w, 2);
                w |= __shfl_xor_sync(0xffffffffu, w, 4);
                const uint32_t wq = __shfl_sync(0xffffffffu, w, (lane & 3) * 8);   // row r0 + 4 q + (lane & 3)
                if ((lane >> 2) == q) mine = wq;
            }
        } else {
#pragma unroll
            for (int u0 = 0; u0 < 32; u0 += U) {
                float v[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int rr = r0 + u0 + u, ly = rr % TY, lz = rr / TY;
                    v[u] = (xin && ly <= g.lastY && lz <= g.lastZ)
                               ? __ldcs(base + (int64_t)lz * sxy + (int64_t)ly * L.nx) : 0.0f;
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const uint32_t w = __ballot_sync(0xffffffffu, occupied(v[u], L.occ_mode));
                    if (lane == u0 + u) mine = w;
                }
            }
        }
        out[r0 + lane] = mine;
        // first and last column of the tile, one bit per row (faces along x)
        const uint32_t c0 = __ballot_sync(0xffffffffu, mine & 1u);
        const uint32_t cl = __ballot_sync(0xffffffffu, (mine >> g.lastX) & 1u);
        if (lane == 0) {
            W.xcol[(t * 2) * (R / 32) + (r0 >> 5)] = c0;
            W.xcol[(t * 2 + 1) * (R / 32) + (r0 >> 5)] = cl;
        }
    }
}

// K0 with TMA (every lattice of the launch with 16-byte aligned rows): persistent, a
// ring of two tile buffers per CTA filled by cp.async.bulk.tensor loads completed on
// mbarriers; while one tile is converted the next is in flight.
template <int TY, int TZ>
struct OccSmem {
    using SH = TileShape<TY, TZ>;
    alignas(128) float buf[2][SH::SITES];
    uint64_t bar[2];
};

template <int TY, int TZ, int NL>
__global__ void __launch_bounds__(256) k_occupancy_tma(const __grid_constant__ TmapBatch<NL> TB,
                                                       const __grid_constant__ LatBatch<NL> B, Work W, int64_t ntiles) {
    grid_dep_wait();
    using SH = TileShape<TY, TZ>;
    constexpr int R = SH::R;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    OccSmem<TY, TZ> &S = *reinterpret_cast<OccSmem<TY, TZ> *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (blockIdx.x == 0 && tid == 0) *W.novf = 0;           // the tile pass appends after this pass
    if (tid == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int64_t t, int s) {
        const int lat = (NL == 1) ? 0 : find_lattice(B.lat, B.n, t);
        const TileGeo g = tile_geo<TY, TZ>(B.lat[lat], t);
        fence_proxy_async();
        mbar_arrive_expect_tx(&S.bar[s], SH::SITES * 4);
        tma_load_3d(S.buf[s], &TB.tm[lat].phi, &S.bar[s], g.x0, g.y0, g.z0);
    };
    const int64_t t0 = blockIdx.x, step = gridDim.x;
    if (tid == 0) {
        if (t0 < ntiles) issue(t0, 0);
        if (t0 + step < ntiles) issue(t0 + step, 1);
    }
    int k = 0;
    for (int64_t t = t0; t < ntiles; t += step, ++k) {
        const int s = k & 1;
        // the decision to give up is the CTA's, so that every thread leaves together
        if (__syncthreads_or(!mbar_wait_bounded(&S.bar[s], (uint32_t)((k >> 1) & 1)))) {
            if (tid == 0) atomicOr(W.status, STATUS_TMA_TIMEOUT);
            // a second bounded wait for the copies still in flight into this CTA's
            // buffers (this tile's and the next one's) before its shared memory goes
            mbar_wait_bounded(&S.bar[s], (uint32_t)((k >> 1) & 1));
            if (t + step < ntiles) mbar_wait_bounded(&S.bar[s ^ 1], (uint32_t)(((k + 1) >> 1) & 1));
            return;
        }
        const LatDev &L = B.lat[(NL == 1) ? 0 : find_lattice(B.lat, B.n, t)];
        const int lastX = tile_geo<TY, TZ>(L, t).lastX;
        // warp w converts rows [32 w', 32 w' + 32) in turns; lane j keeps row 32 w' + j
        for (int r0 = wid * 32; r0 < R; r0 += 32 * (256 / 32)) {
            uint32_t mine = 0;
#pragma unroll 8
            for (int j = 0; j < 32; ++j) {
                const uint32_t w = __ballot_sync(0xffffffffu, occupied(S.buf[s][(r0 + j) * 32 + lane], L.occ_mode));
                if (lane == j) mine = w;
            }
            W.mask[t * R + r0 + lane] = mine;
            const uint32_t c0 = __ballot_sync(0xffffffffu, mine & 1u);
            const uint32_t cl = __ballot_sync(0xffffffffu, (mine >> lastX) & 1u);
            if (lane == 0) {
                W.xcol[(t * 2) * (R / 32) + (r0 >> 5)] = c0;
                W.xcol[(t * 2 + 1) * (R / 32) + (r0 >> 5)] = cl;
            }
        }
        __syncthreads();                       // every warp is done with buffer s
        if (tid == 0 && t + 2 * step < ntiles) issue(t + 2 * step, s);
    }
}

// --------------------------------------------------------------------------------------
// K1: tile labelling from the occupancy words (one tile per CTA)
// --------------------------------------------------------------------------------------
template <int TY, int TZ, int CAP, int BL>
struct LabelSmem {
    using SH = TileShape<TY, TZ>;
    uint32_t m[SH::R];                     // occupancy word of each row
    uint16_t rbase[SH::R];                 // first run id of each row
    int par[CAP];                          // union-find over run ids; after compression: the root
    int aux[CAP];                          // union pair lists; then per root: size + AUX_FACE *
                                           // (runs touching a face); then -1 - k for boundary root k
    uint16_t desc[CAP];                    // per run: DESC_TOUCH | (tile row << 5) | first x
    uint16_t blist[BL];                    // run ids of the boundary roots, by boundary number
    uint32_t nylo[TZ], nyhi[TZ];           // neighbour rows across the y faces, per plane
    uint32_t nzlo[TY], nzhi[TY];           // neighbour rows across the z faces, per row
    uint32_t nxlo[SH::R / 32], nxhi[SH::R / 32];   // neighbour columns across the x faces
    uint32_t xo0[SH::R / 32], xol[SH::R / 32];     // this tile's first and last column
    static_assert(TZ <= 16 && TY <= 32 && SH::R / 32 <= 16 && SH::NT >= 64, "face loads use threads 0..63");
    static_assert(SH::R <= 256 && CAP <= 4096, "desc holds an 8-bit row and run ids fit in 16 bits");
    uint32_t chunkbal[CAP / 32];           // boundary-root ballot of each chunk of 32 run ids
    uint32_t chunkint[CAP / 32];           // interior-root ballot of each chunk
    int chunkpre[CAP / 32];                // boundary roots before each chunk
    int nbnd;                              // boundary roots of the tile
    int warp_tmp[32];
};

constexpr int AUX_FACE = 1 << 14;   // > any piece size (a tile has at most 8192 sites)
constexpr int DESC_TOUCH = 1 << 13;  // desc flag: the run has a site connected across a tile face

// Resident CTAs per SM of the fast tile pass (its shared memory and 32 registers a
// thread allow 2048 threads) and of the pass over the tiles it hands on.
template <int TY, int TZ, bool FAST>
struct LabelCfg {
    static constexpr int CAP = FAST ? TileShape<TY, TZ>::MR_FAST : TileShape<TY, TZ>::MAXRUNS;
    // boundary pieces the fast pass lists (more go to the second pass, which has room for all)
    static constexpr int BL = FAST && TileShape<TY, TZ>::MAX_BOUNDARY > 512 ? 512 : TileShape<TY, TZ>::MAX_BOUNDARY;
    static constexpr int BLOCKS = FAST ? (2048 / (TY * TZ) < 32 ? 2048 / (TY * TZ) : 32)
                                       : (1280 / (TY * TZ) < 32 ? 1280 / (TY * TZ) : 32);
};

// FAST: tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... below ntiles; a tile with
// more than MR_FAST runs or union pairs of one kind is appended to W.ovf instead.
// !FAST: the tiles listed in W.ovf, with room for every tile.
template <int TY, int TZ, int NL, bool FAST>
__global__ void __launch_bounds__(TY * TZ, (LabelCfg<TY, TZ, FAST>::BLOCKS))
k_tile_label(const __grid_constant__ LatBatch<NL> B, Work W, int64_t ntiles) {
    grid_dep_wait();
    using SH = TileShape<TY, TZ>;
    constexpr int R = SH::R, NT = SH::NT, MR = SH::MAXRUNS, CAP = LabelCfg<TY, TZ, FAST>::CAP;
    constexpr int BL = LabelCfg<TY, TZ, FAST>::BL;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    LabelSmem<TY, TZ, CAP, BL> &S = *reinterpret_cast<LabelSmem<TY, TZ, CAP, BL> *>(smem_raw);
    const int tid = threadIdx.x;
    const int64_t nwork = FAST ? ntiles : (int64_t)*reinterpret_cast<volatile int32_t *>(W.novf);

    for (int64_t it = blockIdx.x; it < nwork; it += gridDim.x) {
        const int64_t t = FAST ? it : (int64_t)W.ovf[it];
        const LatDev &L = B.lat[(NL == 1) ? 0 : find_lattice(B.lat, B.n, t)];
        const TileGeo g = tile_geo<TY, TZ>(L, t);

        const int r = tid, ly = r % TY, lz = r / TY;
        const uint32_t m = W.mask[t * R + r];
        S.m[r] = m;
        const uint32_t rs = run_starts(m);
        {
            const uint32_t c0 = __ballot_sync(0xffffffffu, m & 1u);
            const uint32_t cl = __ballot_sync(0xffffffffu, (m >> g.lastX) & 1u);
            if ((tid & 31) == 0) {
                S.xo0[tid >> 5] = c0;
                S.xol[tid >> 5] = cl;
            }
        }

        // Occupancy across the six faces, from the neighbour tiles' masks (the
        // occupancy pass has written all of them).  A face site is connected when
        // it and its neighbour across the face are both occupied; only pieces with a
        // connected site take part in the merge between tiles.
        {
            const int64_t plane = (int64_t)L.nbx * L.nby;
            const int lastY_lo = g.by > 0 ? TY - 1 : L.ny - 1 - (L.nby - 1) * TY;   // neighbour's last row
            const int lastZ_lo = g.bz > 0 ? TZ - 1 : L.nz - 1 - (L.nbz - 1) * TZ;
            constexpr int RW = R / 32;
            if (tid < TZ) {
                const int64_t tylo = g.by > 0 ? t - L.nbx : t + (int64_t)(L.nby - 1) * L.nbx;
                const int64_t tyhi = g.by < L.nby - 1 ? t + L.nbx : t - (int64_t)(L.nby - 1) * L.nbx;
                S.nylo[tid] = g.extYlo ? W.mask[tylo * R + tid * TY + lastY_lo] : 0u;
                S.nyhi[tid] = g.extYhi ? W.mask[tyhi * R + tid * TY] : 0u;
            } else if (tid >= 16 && tid < 16 + TY) {     // TZ <= 16, TY <= 32, R/32 <= 8, NT >= 64
                const int q = tid - 16;
                const int64_t tzlo = g.bz > 0 ? t - plane : t + (int64_t)(L.nbz - 1) * plane;
                const int64_t tzhi = g.bz < L.nbz - 1 ? t + plane : t - (int64_t)(L.nbz - 1) * plane;
                S.nzlo[q] = g.extZlo ? W.mask[tzlo * R + lastZ_lo * TY + q] : 0u;
                S.nzhi[q] = g.extZhi ? W.mask[tzhi * R + q] : 0u;
            } else if (tid >= 48 && tid < 48 + RW) {
                const int q = tid - 48;
                const int64_t txlo = g.bx > 0 ? t - 1 : t + (L.nbx - 1);
                const int64_t txhi = g.bx < L.nbx - 1 ? t + 1 : t - (L.nbx - 1);
                S.nxlo[q] = g.extXlo ? W.xcol[(txlo * 2 + 1) * RW + q] : 0u;   // its last column
                S.nxhi[q] = g.extXhi ? W.xcol[(txhi * 2) * RW + q] : 0u;       // its first column
            }
        }

        // a2: run ids (row-major), union lists, unions
        int total;
        const int rb = block_exscan<NT>(__popc(rs), S.warp_tmp, total);   // ends with a barrier
        if (FAST && total > CAP) {               // block-uniform; nothing read from S after the scan
            if (tid == 0) W.ovf[atomicAdd(W.novf, 1)] = (int32_t)t;
            continue;
        }
        S.rbase[r] = (uint16_t)rb;
        // Each run's own union-find node and its descriptor: position and whether one of
        // its sites is connected across a tile face with a neighbour tile (the site and
        // its neighbour there both occupied).
        if (m) {
            uint32_t conn = 0;
            if (ly == 0) conn |= S.nylo[lz];
            if (ly == g.lastY) conn |= S.nyhi[lz];
            if (lz == 0) conn |= S.nzlo[ly];
            if (lz == g.lastZ) conn |= S.nzhi[ly];
            if ((S.nxlo[r >> 5] >> (r & 31)) & 1u) conn |= 1u;
            if ((S.nxhi[r >> 5] >> (r & 31)) & 1u) conn |= 1u << g.lastX;
            conn &= m;
            // The run starts whose run holds a connected site, for the whole row at once:
            // conn is spread towards lower x inside each run by doubling (after the step
            // of shift s, bit i holds the OR of conn over [i, i + 2s - 1] when m is set
            // all the way from i; rr marks where m is set over [i, i + s]).
            uint32_t f = conn, rr = m & (m >> 1);
            f |= (f >> 1) & rr;
            rr &= rr >> 1;
            f |= (f >> 2) & rr;
            rr &= rr >> 2;
            f |= (f >> 4) & rr;
            rr &= rr >> 4;
            f |= (f >> 8) & rr;
            rr &= rr >> 8;
            f |= (f >> 16) & rr;
            const uint32_t touched = f & rs;
            uint32_t w = rs;
            int id = rb;
            while (w) {
                const int x0 = __ffs(w) - 1;
                w &= w - 1;
                S.par[id] = id;
                S.desc[id] = (uint16_t)((((touched >> x0) & 1u) ? DESC_TOUCH : 0) | (r << 5) | x0);
                ++id;
            }
        }
        const int ucap = (W.local_cap > 0 && W.local_cap < total) ? W.local_cap : total;   // union retry bound

        // y- and z-neighbours: one union per overlapping run pair of rows (y-1, y) and
        // (z-1, z).  Both pair lists come from one scan of packed counts (each total
        // is at most 16 * R < 2^16) and normally share one pass of unions, the z pairs
        // listed first (measured faster than y first).
        const uint32_t osy = ly > 0 ? run_starts(m & S.m[r - 1]) : 0u;
        const uint32_t osz = lz > 0 ? run_starts(m & S.m[r - TY]) : 0u;
        int tot_packed;
        const int packed = block_exscan<NT>(__popc(osy) | (__popc(osz) << 16), S.warp_tmp, tot_packed);
        const int ny_tot = tot_packed & 0xffff, nz_tot = tot_packed >> 16;
        if (FAST && (ny_tot > CAP || nz_tot > CAP)) {   // block-uniform, as above
            if (tid == 0) W.ovf[atomicAdd(W.novf, 1)] = (int32_t)t;
            continue;
        }
        auto write_pairs = [&](uint32_t os, int q, int j) {
            const uint32_t mq = S.m[q];
            const uint32_t rsq = run_starts(mq);
            const int rbq = S.rbase[q];
            while (os) {
                const int x = __ffs(os) - 1;
                os &= os - 1;
                S.aux[j++] = (run_of(rb, rs, x) << 16) | run_of(rbq, rsq, x);
            }
        };
        auto union_pairs = [&](int n) {
            for (int i = tid; i < n; i += NT) {
                const uint32_t p = (uint32_t)S.aux[i];
                s_union(S.par, (int)(p >> 16), (int)(p & 0xffffu), ucap, W.status);
            }
        };
        if (ny_tot + nz_tot <= CAP) {           // block-uniform
            if (osz) write_pairs(osz, r - TY, packed >> 16);
            if (osy) write_pairs(osy, r - 1, nz_tot + (packed & 0xffff));
            __syncthreads();
            union_pairs(ny_tot + nz_tot);
            __syncthreads();
        } else {
            if (osy) write_pairs(osy, r - 1, packed & 0xffff);
            __syncthreads();
            union_pairs(ny_tot);
            __syncthreads();
            if (osz) write_pairs(osz, r - TY, packed >> 16);
            __syncthreads();
            union_pairs(nz_tot);
            __syncthreads();
        }

        // periodic edges inside the tile (an axis that fits in one tile)
        if (g.wrapX || g.wrapY || g.wrapZ) {
            if (m) {
                if (g.wrapY && ly == g.lastY && ly > 0)
                    join_rows(S.par, m, rb, S.m[r - ly], S.rbase[r - ly], ucap, W.status);
                if (g.wrapZ && lz == g.lastZ && lz > 0)
                    join_rows(S.par, m, rb, S.m[r - lz * TY], S.rbase[r - lz * TY], ucap, W.status);
                if (g.wrapX && g.lastX > 0 && (m & 1u) && ((m >> g.lastX) & 1u))
                    s_union(S.par, rb, run_of(rb, rs, g.lastX), ucap, W.status);
            }
            __syncthreads();
        }

        // Sizes accumulate in aux, which held the pair lists until the unions above.
        for (int i = 4 * tid; i < total; i += 4 * NT)
            *reinterpret_cast<int4 *>(&S.aux[i]) = make_int4(0, 0, 0, 0);
        __syncthreads();

        // Compression and piece sizes, one run id per thread: par[i] = root (the piece's
        // first run), and the run's length -- plus AUX_FACE if it touches a face -- is
        // added to its root.  The finds are read-only, so storing final roots while
        // others still search is safe.  A piece is a boundary piece iff its sum reaches
        // AUX_FACE (sizes stay below it).
        for (int i = tid; i < total; i += NT) {
            const int root = s_find_ro(S.par, i);
            S.par[i] = root;
            const int d = S.desc[i];
            const int len = run_len(S.m[(d >> 5) & 0xff], d & 31);
            atomicAdd(&S.aux[root], len + ((d & DESC_TOUCH) ? AUX_FACE : 0));
        }
        __syncthreads();

        // Number the boundary roots in run order and write their records to the tile's
        // slice of the piece table.  Chunks of 32 run ids are counted by ballot, the chunk
        // counts scanned by one warp, and the boundary roots listed by number, so that only
        // they do the record writes.  Interior roots are kept as a ballot per chunk for the
        // per-row counts below.
        const int base = (int)(t * SH::MAX_BOUNDARY);   // fixed slice of the piece table
        {
            const int lane = tid & 31, wid = tid >> 5;
            constexpr int NW = NT / 32;
            const int nchunks = (total + 31) / 32;
            for (int c = wid; c < nchunks; c += NW) {
                const int i = c * 32 + lane;
                const bool root = i < total && S.par[i] == i;
                const bool bnd = root && S.aux[i] >= AUX_FACE;
                const uint32_t bb = __ballot_sync(0xffffffffu, bnd);
                const uint32_t bi = __ballot_sync(0xffffffffu, root && !bnd);
                if (lane == 0) {
                    S.chunkbal[c] = bb;
                    S.chunkint[c] = bi;
                }
            }
            __syncthreads();
            if (wid == 0) {   // at most CAP / 32 <= 128 chunks
                int carry = 0;
                for (int c0 = 0; c0 < nchunks; c0 += 32) {
                    const int c = c0 + lane;
                    const int v = c < nchunks ? __popc(S.chunkbal[c]) : 0;
                    int inc = v;
#pragma unroll
                    for (int d = 1; d < 32; d <<= 1) {
                        const int u = __shfl_up_sync(0xffffffffu, inc, d);
                        if (lane >= d) inc += u;
                    }
                    if (c < nchunks) S.chunkpre[c] = carry + inc - v;
                    carry += __shfl_sync(0xffffffffu, inc, 31);
                }
                if (lane == 0) S.nbnd = carry;
            }
            __syncthreads();
        }
        const int nb_ = S.nbnd;
        if (FAST && nb_ > BL) {                 // block-uniform; nothing global written yet
            if (tid == 0) W.ovf[atomicAdd(W.novf, 1)] = (int32_t)t;
            continue;
        }
        {
            const int lane = tid & 31, wid = tid >> 5;
            constexpr int NW = NT / 32;
            const int nchunks = (total + 31) / 32;
            for (int c = wid; c < nchunks; c += NW) {
                const uint32_t bal = S.chunkbal[c];
                if ((bal >> lane) & 1u)
                    S.blist[S.chunkpre[c] + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)(c * 32 + lane);
            }
        }
        __syncthreads();
        for (int k = tid; k < nb_; k += NT) {
            const int i = S.blist[k];
            const int d = S.desc[i];
            const int row = (d >> 5) & 0xff;
            const int pid = base + k;
            W.parent[pid] = pid;
            W.key[pid] = ((g.z0 + row / TY) * L.ny + (g.y0 + row % TY)) * L.nx + g.x0 + (d & 31);
            W.psize[pid] = S.aux[i] & (AUX_FACE - 1);
            S.aux[i] = -1 - k;                   // from here on: boundary root k
        }
        if (tid == 0) W.tinfo[t] = make_int4(base, nb_, total, 0);
        __syncthreads();

        // interior roots per row segment (a row's runs span at most two chunks)
        if (ly <= g.lastY && lz <= g.lastZ) {
            const int n = __popc(rs);
            int interior = 0;
            if (n) {
                const int a = rb, b = rb + n - 1;             // the row's run ids [a, b]
                const int ca = a >> 5, cb = b >> 5;
                const uint32_t lo = S.chunkint[ca] >> (a & 31);
                if (ca == cb) {
                    interior = __popc(lo & ((1u << n) - 1u));   // n <= 16
                } else {
                    const int nh = (b & 31) + 1;                 // ids of the row in chunk cb
                    interior = __popc(lo) + __popc(S.chunkint[cb] & ((1u << nh) - 1u));
                }
            }
            const int64_t seg = L.seg0 + ((int64_t)(g.z0 + lz) * L.ny + (g.y0 + ly)) * L.nbx + g.bx;
            W.cnt[seg] = (uint8_t)interior;
        }

        // one code per run (CODE_* encoding): aux of the run's root is -1 - k for boundary
        // piece k, else the interior piece's size
        uint16_t *C = W.codes + t * MR;
        for (int i = tid; i < total; i += NT) {
            const int v = S.par[i];
            const int a = S.aux[v];
            uint16_t c;
            if (v == i)
                c = a < 0 ? (uint16_t)(CODE_BOUNDARY | CODE_ROOT | (-1 - a)) : (uint16_t)(CODE_ROOT | a);
            else
                c = a < 0 ? (uint16_t)(CODE_BOUNDARY | (-1 - a)) : (uint16_t)(S.desc[v] & (DESC_TOUCH - 1));
            C[i] = c;
        }

        // Face lists.  A face site is connected when it and its neighbour across the
        // face are occupied.  Adjacent connected sites of a face lie in one piece on
        // either side, so one union per component of connected face sites suffices: a
        // connected site is emitted unless its face neighbour at lower x (y and z
        // faces) or at lower y or z (x faces) is connected too, which keeps the
        // lowest site of every component.  Both tiles of a face compute the same
        // connected sites, so their lists pair up entry by entry.  Warps take the faces
        // in turn (lo-x, hi-x, lo-y, hi-y, lo-z, hi-z); lane j owns one 32-bit word.
        {
            const int lane = tid & 31;
            for (int f = tid >> 5; f < 6; f += NT / 32) {
                const int hi = f & 1, axis = f >> 1;
                const bool ext = axis == 0 ? (hi ? g.extXhi : g.extXlo)
                               : axis == 1 ? (hi ? g.extYhi : g.extYlo) : (hi ? g.extZhi : g.extZlo);
                uint32_t c = 0;
                int row0 = 0;   // y and z faces: the row of this lane's word
                if (ext) {
                    if (axis == 0) {
                        if (lane < R / 32) c = hi ? (S.xol[lane] & S.nxhi[lane]) : (S.xo0[lane] & S.nxlo[lane]);
                    } else if (axis == 1) {
                        row0 = lane * TY + (hi ? g.lastY : 0);
                        if (lane < TZ) c = S.m[row0] & (hi ? S.nyhi[lane] : S.nylo[lane]);
                    } else {
                        row0 = (hi ? g.lastZ : 0) * TY + lane;
                        if (lane < TY) c = S.m[row0] & (hi ? S.nzhi[lane] : S.nzlo[lane]);
                    }
                }
                uint32_t prev = __shfl_up_sync(0xffffffffu, c, 1);
                if (lane == 0) prev = 0;
                uint32_t e;
                if (axis == 0) {
                    // bit i of word j is row 32 j + i; rows r - 1 (same plane) and r - TY
                    const uint32_t ym = ((c << 1) | (prev >> 31)) & ~SH::LY0;
                    const uint32_t zm = TY == 32 ? prev : ((c << (TY & 31)) | (prev >> ((32 - TY) & 31)));
                    e = c & ~ym & ~zm;
                } else {
                    e = c & ~(c << 1) & ~prev;
                }
                const int cnt = __popc(e);
                int inc = cnt;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const int u = __shfl_up_sync(0xffffffffu, inc, d);
                    if (lane >= d) inc += u;
                }
                const int n = __shfl_sync(0xffffffffu, inc, 31);
                uint16_t *F = W.face + t * SH::FACE_STRIDE;
                const int off = f == 0 ? SH::OFF_LX : f == 1 ? SH::OFF_HX : f == 2 ? SH::OFF_LY
                              : f == 3 ? SH::OFF_HY : f == 4 ? SH::OFF_LZ : SH::OFF_HZ;
                int j = off + inc - cnt;
                while (e) {
                    const int b = __ffs(e) - 1;
                    e &= e - 1;
                    const int row = axis == 0 ? lane * 32 + b : row0;
                    const int x = axis == 0 ? (hi ? g.lastX : 0) : b;
                    F[j++] = (uint16_t)(-1 - S.aux[S.par[run_of(S.rbase[row], run_starts(S.m[row]), x)]]);
                }
                if (lane == 0) F[SH::OFF_CNT + f] = (uint16_t)n;
            }
        }
        __syncthreads();
    }
}

// --------------------------------------------------------------------------------------
// K2: face merge.  One warp per tile: its low face lists along x, y and z are joined
// entry by entry with the high face lists of its lower neighbours (for tile 0 of a
// periodic axis: the last tile, the wrap).  Each lane takes U entries at a time (a
// merge-schedule parameter: 1, 2 or 4) and
// walks the finds of all their endpoints in lockstep, so their loads are in flight
// together; the roots are then linked by CAS, and a lost CAS falls back to g_union.
// CTAs of FM_WARPS warps: a CTA's resources return only when its slowest warp (longest
// parent chain) is done, so small CTAs keep more warps waiting on loads in flight
// (32 CTAs of 2 warps still fill an SM).
// --------------------------------------------------------------------------------------
constexpr int FM_WARPS = 2;
constexpr int PF_WARPS = 4;
template <int TY, int TZ, int NL, int U>
__global__ void __launch_bounds__(32 * FM_WARPS)
k_face_merge(const __grid_constant__ LatBatch<NL> B, Work W, int64_t ntiles) {
    grid_dep_wait();
    using SH = TileShape<TY, TZ>;
    constexpr int C = 2 * U;   // U unions, 2 U find chains per lane and step
    const int lane = threadIdx.x & 31;
    const int64_t t = (int64_t)blockIdx.x * FM_WARPS + (threadIdx.x >> 5);
    if (t >= ntiles) return;
    const LatDev &L = B.lat[(NL == 1) ? 0 : find_lattice(B.lat, B.n, t)];
    const TileGeo g = tile_geo<TY, TZ>(L, t);
    const int64_t plane = (int64_t)L.nbx * L.nby;
    const int64_t nbr[3] = {g.bx > 0 ? t - 1 : t + (L.nbx - 1),
                            g.by > 0 ? t - L.nbx : t + (int64_t)(L.nby - 1) * L.nbx,
                            g.bz > 0 ? t - plane : t + (int64_t)(L.nbz - 1) * plane};
    const uint16_t *F = W.face + t * SH::FACE_STRIDE;
    const int n0 = g.extXlo ? F[SH::OFF_CNT + 0] : 0;
    const int n1 = g.extYlo ? F[SH::OFF_CNT + 2] : 0;
    const int n2 = g.extZlo ? F[SH::OFF_CNT + 4] : 0;
    const int total = n0 + n1 + n2;
    const int64_t base = t * SH::MAX_BOUNDARY;   // each tile owns a fixed slice of the piece table
    for (int i0 = 0; i0 < total; i0 += 32 * U) {
        int x[C], p[C];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = i0 + u * 32 + lane;
            if (i < total) {
                const int axis = i < n0 ? 0 : (i < n0 + n1 ? 1 : 2);
                const int j = i - (axis == 0 ? 0 : (axis == 1 ? n0 : n0 + n1));
                const int lo = axis == 0 ? SH::OFF_LX : axis == 1 ? SH::OFF_LY : SH::OFF_LZ;
                const int hi = axis == 0 ? SH::OFF_HX : axis == 1 ? SH::OFF_HY : SH::OFF_HZ;
                const int64_t nb = nbr[axis];
                x[2 * u] = (int)(base + F[lo + j]);
                x[2 * u + 1] = (int)(nb * SH::MAX_BOUNDARY + W.face[nb * SH::FACE_STRIDE + hi + j]);
            } else {
                x[2 * u] = x[2 * u + 1] = -1;   // no entry
            }
        }
#pragma unroll
        for (int c = 0; c < C; ++c) p[c] = x[c] >= 0 ? __ldcg(W.parent + x[c]) : x[c];
        // finds with path halving, all chains one step per round
        for (int64_t it = 0;; ++it) {
            bool moving = false;
#pragma unroll
            for (int c = 0; c < C; ++c) moving |= p[c] != x[c];
            if (!moving) break;
            if (it > W.piece_cap) { atomicOr(W.status, STATUS_GLOBAL_LOOP); break; }
            int gp[C];
#pragma unroll
            for (int c = 0; c < C; ++c) gp[c] = p[c] != x[c] ? __ldcg(W.parent + p[c]) : x[c];
#pragma unroll
            for (int c = 0; c < C; ++c) {
                if (p[c] == x[c]) continue;
                if (gp[c] == p[c]) {
                    x[c] = p[c];                      // p is a root
                } else {
                    __stcg(W.parent + x[c], gp[c]);   // path halving: gp is an ancestor of x
                    x[c] = gp[c];
                    p[c] = -2;                        // to reload
                }
            }
#pragma unroll
            for (int c = 0; c < C; ++c) p[c] = p[c] == -2 ? __ldcg(W.parent + x[c]) : (p[c] == x[c] || x[c] < 0 ? x[c] : p[c]);
        }
        // link the roots: the root with the larger key under the one with the smaller key
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int a = x[2 * u], b = x[2 * u + 1];
            if (a < 0 || a == b) continue;
            if (__ldg(W.key + b) < __ldg(W.key + a)) { const int tmp = a; a = b; b = tmp; }
            if (atomicCAS(W.parent + b, b, a) != b) g_union(W.parent, W.key, a, b, W.piece_cap, W.status);
        }
    }
}

// --------------------------------------------------------------------------------------
// K3: piece finalize (one warp per tile, one piece per lane).  Size additions into
// the same cluster root are combined per group of lanes; with HOT (a merge-schedule
// parameter) the root that collects most of them -- the percolating cluster's -- is
// further combined per warp and per CTA of PF_WARPS warps, because it collects pieces
// from most tiles.
// --------------------------------------------------------------------------------------
template <int NL, bool HOT>
__global__ void __launch_bounds__(32 * PF_WARPS)
k_piece_finalize(const __grid_constant__ LatBatch<NL> B, Work W, int64_t ntiles) {
    grid_dep_wait();
    __shared__ int hot_target[PF_WARPS];   // per warp: the cluster root its pieces fed most, and the sum
    __shared__ int hot_sum[PF_WARPS];
    const int64_t t = (int64_t)blockIdx.x * PF_WARPS + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // The root that collects most sizes (the percolating cluster's, above all) is added
    // once per warp and then once per CTA; other roots once per group of lanes.
    int hot = -1, hot_acc = 0;
    const int4 ti = t < ntiles ? W.tinfo[t] : make_int4(0, 0, 0, 0);
    if (ti.y > 0) {
        const LatDev &L = B.lat[(NL == 1) ? 0 : find_lattice(B.lat, B.n, t)];
        for (int j0 = 0; j0 < ti.y; j0 += 32) {
            const int j = j0 + lane;
            const bool valid = j < ti.y;
            const int pid = ti.x + j;
            int root = -1, add = 0;
            if (valid) {
                root = g_find_ro(W.parent, pid, W.piece_cap, W.status);
                if (root != pid) {
                    __stcg(W.parent + pid, root);
                    add = W.psize[pid];
                    // from here on key[pid] is the cluster's label and psize[pid] < 0 marks a
                    // non-root; only roots' keys are read by other threads, and a root's key
                    // never changes
                    W.key[pid] = __ldcg(W.key + root);
                    W.psize[pid] = -1;
                } else {
                    const int k = W.key[pid];
                    const int q = k / L.nx, x = k - q * L.nx;          // q = z * ny + y
                    const int64_t seg = L.seg0 + (int64_t)q * L.nbx + (x >> 5);
                    // one byte per segment (at most 16 roots): add to it inside its aligned word
                    atomicAdd(reinterpret_cast<unsigned int *>(W.cnt + (seg & ~(int64_t)3)),
                              1u << (8 * (int)(seg & 3)));
                }
            }
            const int target = (valid && root != pid) ? root : -1;
            const unsigned peers = __match_any_sync(0xffffffffu, target);
            const int sum = (int)__reduce_add_sync(peers, (unsigned)add);
            const bool leader = target >= 0 && lane == __ffs(peers) - 1;
            if (HOT && hot < 0) {   // warp-uniform: the first chunk names the warp's hot root (its largest group)
                const unsigned key = leader ? ((unsigned)__popc(peers) << 5) | (unsigned)lane : 0u;
                const unsigned best = __reduce_max_sync(0xffffffffu, key);
                if (best) hot = __shfl_sync(0xffffffffu, target, (int)(best & 31u));
            }
            if (leader) {
                if (target == hot) hot_acc += sum;
                else atomicAdd(W.psize + target, sum);
            }
        }
    }
    if (!HOT) return;
    hot_acc = (int)__reduce_add_sync(0xffffffffu, (unsigned)hot_acc);
    if (lane == 0) {
        hot_target[wid] = hot;
        hot_sum[wid] = hot_acc;
    }
    __syncthreads();
    if (threadIdx.x < PF_WARPS) {   // one add per distinct hot root of the CTA
        const int h = hot_target[threadIdx.x];
        if (h >= 0) {
            bool first = true;
            int s = 0;
            for (int w = 0; w < PF_WARPS; ++w)
                if (hot_target[w] == h) {
                    if (w < (int)threadIdx.x) first = false;
                    s += hot_sum[w];
                }
            if (first) atomicAdd(W.psize + h, s);
        }
    }
}

// --------------------------------------------------------------------------------------
// S1-S3: exclusive scan of the cluster roots per lattice row (the sum of the row's
// segment counts); ranks inside a row are completed by flatten from the segment
// counts before its own.
// --------------------------------------------------------------------------------------
constexpr int SCAN_NT = 256;
constexpr int SCAN_PER = 16;
constexpr int SCAN_CH = SCAN_NT * SCAN_PER;

template <int NL>
__device__ __forceinline__ uint32_t row_roots(const LatBatch<NL> &B, const uint8_t *cnt, int64_t q) {
    const LatDev &L = B.lat[(NL == 1) ? 0 : find_lattice_row(B.lat, B.n, q)];
    return bytes_sum(cnt, L.seg0 + (q - L.row0) * L.nbx, L.nbx);
}

template <int NL>
__global__ void __launch_bounds__(SCAN_NT) k_scan_reduce(const __grid_constant__ LatBatch<NL> B,
                                                         const uint8_t *cnt, int64_t n, uint32_t *bsum) {
    grid_dep_wait();
    __shared__ uint32_t red[SCAN_NT / 32];
    const int64_t b0 = (int64_t)blockIdx.x * SCAN_CH;
    uint32_t s = 0;
    for (int j = 0; j < SCAN_PER; ++j) {
        const int64_t i = b0 + (int64_t)j * SCAN_NT + threadIdx.x;
        if (i < n) s += row_roots(B, cnt, i);
    }
    for (int d = 16; d; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t tot = 0;
        for (int w = 0; w < SCAN_NT / 32; ++w) tot += red[w];
        bsum[blockIdx.x] = tot;
    }
}

// single block: exclusive scan of the block sums in place
__global__ void __launch_bounds__(1024) k_scan_blocks(uint32_t *bsum, int64_t nb) {
    grid_dep_wait();
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < nb; c0 += 1024) {
        const int64_t i = c0 + threadIdx.x;
        const uint32_t v = i < nb ? bsum[i] : 0u;
        uint32_t inc = v;
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= d) inc += u;
        }
        if (lane == 31) wsum[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            uint32_t w = wsum[lane], wi = w;
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t u = __shfl_up_sync(0xffffffffu, wi, d);
                if (lane >= d) wi += u;
            }
            wsum[lane] = wi - w;
        }
        __syncthreads();
        const uint32_t ex = carry + wsum[wid] + inc - v;
        if (i < nb) bsum[i] = ex;
        __syncthreads();
        if (threadIdx.x == 1023) carry = ex + v;
        __syncthreads();
    }
}

template <int NL>
__global__ void __launch_bounds__(SCAN_NT) k_scan_apply(const __grid_constant__ LatBatch<NL> B, const uint8_t *cnt,
                                                        int64_t n, const uint32_t *bsum, uint32_t *pre) {
    grid_dep_wait();
    __shared__ uint32_t wsum[SCAN_NT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t b0 = (int64_t)blockIdx.x * SCAN_CH + (int64_t)threadIdx.x * SCAN_PER;
    uint32_t v[SCAN_PER];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_PER; ++j) {
        const int64_t i = b0 + j;
        v[j] = i < n ? row_roots(B, cnt, i) : 0u;
        s += v[j];
    }
    uint32_t inc = s;
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += u;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = lane < SCAN_NT / 32 ? wsum[lane] : 0u, wi = w;
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += u;
        }
        if (lane < SCAN_NT / 32) wsum[lane] = wi - w;
    }
    __syncthreads();
    uint32_t run = bsum[blockIdx.x] + wsum[wid] + inc - s;
#pragma unroll
    for (int j = 0; j < SCAN_PER; ++j) {
        const int64_t i = b0 + j;
        if (i <= n) pre[i] = run;   // pre[n] = total
        run += v[j];
    }
}

// per-lattice: cluster count from the prefix, clear the histogram
template <int NL>
__global__ void k_lattice_finish(const __grid_constant__ LatBatch<NL> B, Work W) {
    grid_dep_wait();
    const int l = blockIdx.x;
    if (l >= B.n) return;
    const LatDev &L = B.lat[l];
    if (threadIdx.x < 32 && L.hist) L.hist[threadIdx.x] = 0;
    if (threadIdx.x == 0 && L.ncl) {
        // uint32 difference: the prefix may wrap over a launch, a lattice's count does not
        L.ncl[0] = (int64_t)(uint32_t)(W.pre[L.row0 + (int64_t)L.nz * L.ny] - W.pre[L.row0]);
    }
}

// --------------------------------------------------------------------------------------
// K4: flatten (decode run codes; no union-find)
// --------------------------------------------------------------------------------------
// The staged tile uses the TMA 128-byte swizzle: in each tile row (128 bytes) the
// 16-byte chunk index is XORed with the row index mod 8, so that threads writing the
// same x of consecutive rows hit different banks.
__device__ __forceinline__ int stage_idx(int row, int x) { return row * 32 + (x ^ ((row & 7) << 2)); }

template <int TY, int TZ>
struct FlatSmem {
    using SH = TileShape<TY, TZ>;
    alignas(1024) int32_t stage[SH::SITES];   // labels [lz][ly][x], swizzled (TMA store source)
    static constexpr int GL = SH::MAX_BOUNDARY < 384 ? SH::MAX_BOUNDARY : 384;   // staged boundary pieces
    static_assert(GL % 4 == 0 && (SH::MAX_BOUNDARY * 4) % 16 == 0 && (SH::MAXRUNS * 2) % 16 == 0,
                  "bulk copies of whole 16-byte blocks from 16-byte aligned slices");
    alignas(16) uint16_t codes[SH::MAXRUNS];  // the tile's run codes (bulk copy)
    alignas(16) int gl[GL];                   // label of each boundary piece's cluster
    alignas(16) int gsize[GL];                // cluster size if the piece is the cluster root, else -1
    uint64_t bar;                             // completion of the tile's bulk copies
    int warp_tmp[32];
    int hist[32];
};

template <int TY, int TZ>
__device__ __forceinline__ int site_of(const TileGeo &g, const LatDev &L, int pos) {
    const int row = pos >> 5, x = pos & 31;
    return ((g.z0 + row / TY) * L.ny + (g.y0 + row % TY)) * L.nx + g.x0 + x;
}

// SLAB: one slab of a lattice split along z (W.site_off added to every label, each
// cluster's label written to W.roots); a separate instance, so that the common path
// carries neither.
template <int TY, int TZ, int NL, bool SLAB>
__global__ void __launch_bounds__(TY * TZ, 1280 / (TY * TZ))
k_flatten(const __grid_constant__ LatBatch<NL> B, const __grid_constant__ TmapBatch<NL> TB, Work W, int64_t ntiles) {
    grid_dep_wait();
    using SH = TileShape<TY, TZ>;
    constexpr int R = SH::R, NT = SH::NT, NW = NT / 32, MR = SH::MAXRUNS;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    FlatSmem<TY, TZ> &S = *reinterpret_cast<FlatSmem<TY, TZ> *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    // the swizzled TMA store needs a 1024-byte aligned source; otherwise plain stores
    const bool stage_ok = (smem_u32(S.stage) & 1023u) == 0;

    if (tid < 32) S.hist[tid] = 0;
    if (tid == 0) {
        mbar_init(&S.bar, 1);
        fence_mbar_init();
    }
    // The tile's run codes and its staged boundary-piece records arrive by bulk copies
    // issued at the start of the tile, so that the run loop reads shared memory.  If a
    // copy does not complete within its bound the CTA records STATUS_TMA_TIMEOUT and
    // reads global memory from then on (prefetch becomes false, uniformly).
    bool prefetch = true;
    int ktile = 0;
    int cur_lat = -1;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++ktile) {
        const int lat = (NL == 1) ? 0 : find_lattice(B.lat, B.n, t);
        const LatDev &L = B.lat[lat];
        const TileGeo g = tile_geo<TY, TZ>(L, t);
        const bool use_tma = TB.tm[lat].valid && stage_ok;
        const int4 ti = W.tinfo[t];
        const int base = ti.x, nb = ti.y;
        const int r = tid, ly = r % TY, lz = r / TY;
        const uint32_t m = W.mask[t * R + r];
        const uint32_t rs = run_starts(m);
        const bool valid_row = ly <= g.lastY && lz <= g.lastZ;
        // rank base of this row: issued early, used after the barriers below
        uint32_t pre_row = 0, pre_lat = 0;
        if (rs && valid_row) {
            // roots of the lattice's earlier rows, then of this row's earlier segments
            const int64_t q = (int64_t)(g.z0 + lz) * L.ny + (g.y0 + ly);
            pre_row = W.pre[L.row0 + q] + bytes_sum(W.cnt, L.seg0 + q * L.nbx, g.bx);
            pre_lat = W.pre[L.row0];
        }

        const uint16_t *C = W.codes + t * MR;
        constexpr int GL = FlatSmem<TY, TZ>::GL;
        if (tid == 0) bulk_wait_read0();               // a previous tile's store has read S.stage
        __syncthreads();                               // ... and every thread is done with S.codes, S.gl
        if (prefetch && tid == 0) {
            const int ncode = (ti.z + 7) & ~7;                       // whole 16-byte blocks
            const int ng = ((nb < GL ? nb : GL) + 3) & ~3;
            mbar_arrive_expect_tx(&S.bar, (uint32_t)(2 * ncode + 8 * ng));
            if (ncode) bulk_load(S.codes, C, 2u * ncode, &S.bar);
            if (ng) {
                bulk_load(S.gl, W.key + base, 4u * ng, &S.bar);
                bulk_load(S.gsize, W.psize + base, 4u * ng, &S.bar);
            }
        }
        if (lat != cur_lat) {                          // uniform: flush the histogram per lattice
            if (cur_lat >= 0 && tid < 32 && S.hist[tid] && B.lat[cur_lat].hist)
                atomicAdd(reinterpret_cast<unsigned long long *>(B.lat[cur_lat].hist) + tid,
                          (unsigned long long)S.hist[tid]);
            __syncthreads();
            if (tid < 32) S.hist[tid] = 0;
            cur_lat = lat;
        }

        for (int i = tid; i < SH::SITES / 4; i += NT)
            reinterpret_cast<int4 *>(S.stage)[i] = make_int4(-1, -1, -1, -1);
        int tot2;
        const int rb = block_exscan<NT>(__popc(rs), S.warp_tmp, tot2);   // ends with a barrier
        if (prefetch) {
            const bool done = mbar_wait_bounded(&S.bar, (uint32_t)(ktile & 1));
            if (__syncthreads_or(!done)) {             // uniform: give up the prefetch
                if (tid == 0) atomicOr(W.status, STATUS_TMA_TIMEOUT);
                mbar_wait_bounded(&S.bar, (uint32_t)(ktile & 1));   // the copies still in flight
                prefetch = false;
            }
        }
        if (!prefetch) {                               // staged by the threads instead
            for (int k = tid; k < nb && k < GL; k += NT) {
                S.gl[k] = __ldg(W.key + base + k);       // cluster label (written by piece_finalize)
                S.gsize[k] = __ldg(W.psize + base + k);  // cluster size at the root piece, else -1
            }
            __syncthreads();
        }

        // a4-a7: one pass over the runs of each row in x order: cluster roots get
        // their rank, size and histogram entry; every run writes its label.  The loop
        // is compiled for each case of two tile-uniform conditions, so that neither is
        // tested per run: PF, the codes and piece records arrived by bulk copy (else
        // they are read from global memory); BIG, the tile has boundary pieces beyond
        // the staged ones (read from global memory).
        int64_t rank = (int64_t)(uint32_t)(pre_row - pre_lat);
        const int site_row = ((g.z0 + lz) * L.ny + (g.y0 + ly)) * L.nx + g.x0;
        const int site_row0 = (g.z0 * L.ny + g.y0) * L.nx + g.x0, sxy_i = L.nx * L.ny;
        uint32_t rootbits = 0;                // first sites of cluster roots in this row
        const int soff = SLAB ? (int)W.site_off : 0;   // labels of a slab are sites of the whole lattice
        const uint32_t re = run_ends(m);
        auto run_loop = [&](auto PF, auto BIG) {
            constexpr bool pf = decltype(PF)::value, big = decltype(BIG)::value;
            uint32_t w = rs;
            int id = rb;
            while (w) {
                const int x0 = __ffs(w) - 1;
                w &= w - 1;
                const int c = pf ? (int)S.codes[id] : (int)__ldg(C + id);
                ++id;
                const int k = c & CODE_LOW;
                const bool isb = (c & CODE_BOUNDARY) != 0, isr = (c & CODE_ROOT) != 0;
                const int kk = k < FlatSmem<TY, TZ>::GL ? k : 0;
                int gl = S.gl[kk], gs = S.gsize[kk];
                if (big && isb && k >= FlatSmem<TY, TZ>::GL) {
                    gl = __ldg(W.key + base + k);
                    gs = __ldg(W.psize + base + k);
                }
                // all three labels are formed and one is selected (no divergent branches)
                const int ci = (isb || isr) ? 0 : c;   // an interior non-root run: its root's position
                const int crow = ci >> 5;
                const int own = site_row + x0;
                const int other = site_row0 + (crow / TY) * sxy_i + (crow % TY) * L.nx + (ci & 31);
                const int lab = SLAB ? (isb ? gl : (isr ? own : other)) + soff : (isb ? gl : (isr ? own : other));
                const int size = isr ? (isb ? gs : k) : -1;
                if (size > 0) {
                    if (rank < L.sizes_cap) {
                        L.sizes[rank] = size;
                        if (SLAB) W.roots[rank] = lab;
                    }
                    ++rank;
                    rootbits |= 1u << x0;
                    atomicAdd(&S.hist[31 - __clz(size)], 1);
                }
                const int xe = x0 + __ffs(re >> x0);   // one past the run's last site
                int *row = S.stage + r * 32;
                const int sw = (r & 7) << 2;
                row[x0 ^ sw] = lab;
#pragma unroll 1
                for (int x = x0 + 1; x < xe; ++x) row[x ^ sw] = lab;
            }
        };
        if (!prefetch) run_loop(std::false_type{}, std::true_type{});
        else if (nb > FlatSmem<TY, TZ>::GL) run_loop(std::true_type{}, std::true_type{});
        else run_loop(std::true_type{}, std::false_type{});
        if (L.inside && ly <= g.lastY && lz <= g.lastZ)   // index fields: ranks of any root, later
            W.rootbits[L.seg0 + ((int64_t)(g.z0 + lz) * L.ny + (g.y0 + ly)) * L.nbx + g.bx] = rootbits;
        if (use_tma) fence_proxy_async();
        __syncthreads();
        if (use_tma) {
            if (tid == 0) {
                tma_store_3d(&TB.tm[lat].labels, S.stage, g.x0, g.y0, g.z0);
                bulk_commit();
            }
        } else if (g.lastX == TX - 1 && (L.nx & 3) == 0 && (reinterpret_cast<uintptr_t>(L.labels) & 15) == 0) {
            // whole rows at 16-byte aligned addresses: lane l stores 4 labels (x = 4 (l % 8)
            // .. + 3) of row l / 8 of each group of 4 rows (the swizzle keeps them together)
            const int64_t sxy = (int64_t)L.nx * L.ny;
            const int x4 = (lane & 7) * 4;
            int32_t *out = L.labels + (int64_t)g.z0 * sxy + (int64_t)g.y0 * L.nx + g.x0 + x4;
            for (int r4 = wid * 4; r4 < R; r4 += NW * 4) {
                const int rr = r4 + (lane >> 3), yy = rr % TY, zz = rr / TY;
                if (yy <= g.lastY && zz <= g.lastZ)
                    __stcs(reinterpret_cast<int4 *>(out + (int64_t)zz * sxy + (int64_t)yy * L.nx),
                           *reinterpret_cast<const int4 *>(S.stage + rr * 32 + (x4 ^ ((rr & 7) << 2))));
            }
        } else {
            const int64_t sxy = (int64_t)L.nx * L.ny;
            int32_t *out = L.labels + (int64_t)g.z0 * sxy + (int64_t)g.y0 * L.nx + g.x0 + lane;
            if (lane <= g.lastX)
                for (int rr = wid; rr < R; rr += NW) {
                    const int yy = rr % TY, zz = rr / TY;
                    if (yy <= g.lastY && zz <= g.lastZ)
                        __stcs(out + (int64_t)zz * sxy + (int64_t)yy * L.nx, S.stage[stage_idx(rr, lane)]);
                }
        }
    }
    if (tid == 0) bulk_wait0();
    __syncthreads();
    if (cur_lat >= 0 && tid < 32 && S.hist[tid] && B.lat[cur_lat].hist)
        atomicAdd(reinterpret_cast<unsigned long long *>(B.lat[cur_lat].hist) + tid, (unsigned long long)S.hist[tid]);
}

// --------------------------------------------------------------------------------------
// Interior/exterior identification (Sec. 6, step 5) for an index field labelled with
// occ_mode 1: every face pair (cluster site, near site) votes with the sign of I at
// the near site; a cluster with more negative votes is interior.  One lattice.
// --------------------------------------------------------------------------------------
// Clusters ranked before each row segment of an index field: the roots of the
// lattice's earlier rows and of the row's earlier segments.  One thread per row.
__global__ void __launch_bounds__(256) k_segpre(const LatDev L, Work W) {
    const int64_t rows = (int64_t)L.ny * L.nz;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < rows; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t rowseg = L.seg0 + q * L.nbx;
        uint32_t acc = W.pre[L.row0 + q] - W.pre[L.row0];
        for (int b = 0; b < L.nbx; ++b) {
            W.segpre[rowseg + b] = acc;
            acc += W.cnt[rowseg + b];
        }
    }
}

// Rank (compacted id - 1) of the cluster whose first site is `lab`: the clusters
// ranked before its segment and the roots of its segment before it.
__device__ __forceinline__ int64_t rank_of_root(const LatDev &L, const Work &W, int lab) {
    const int q = lab / L.nx, x = lab - q * L.nx;
    const int64_t seg = L.seg0 + (int64_t)q * L.nbx + (x >> 5);
    return (int64_t)W.segpre[seg] + __popc(W.rootbits[seg] & ((1u << (x & 31)) - 1u));
}

__global__ void __launch_bounds__(256) k_votes_clear(const LatDev L, Work W) {
    const int64_t n = *L.ncl < L.sizes_cap ? *L.ncl : L.sizes_cap;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        W.votes[k] = 0;
}

// Votes into the first VOTE_SMEM ranks are summed per CTA in shared memory and
// added to the global counters once per CTA (a few clusters, such as the exterior
// fluid, collect most votes); higher ranks go straight to global memory.
constexpr int VOTE_SMEM = 1024;

// The votes of near site s (value v): one per face neighbour that is a cluster site.
__device__ __forceinline__ void vote_site(const LatDev &L, const Work &W, int64_t s, float v, int *sv) {
    if (!(v >= -0.5f)) return;                 // a cluster site (or NaN): not a near site
    const int sign = v < 0.0f ? -1 : (v > 0.0f ? 1 : 0);
    if (sign == 0) return;
    const int dims[3] = {L.nx, L.ny, L.nz};
    const int x = (int)(s % L.nx);
    const int64_t q = s / L.nx;
    const int y = (int)(q % L.ny), z = (int)(q / L.ny);
#pragma unroll
    for (int dir = 0; dir < 6; ++dir) {
        const int axis = dir >> 1;
        int c[3] = {x, y, z};
        c[axis] += (dir & 1) ? 1 : -1;
        if (c[axis] < 0 || c[axis] >= dims[axis]) {
            if (!L.per[axis]) continue;
            c[axis] = c[axis] < 0 ? dims[axis] - 1 : 0;
        }
        const int lab = L.labels[c[0] + (int64_t)L.nx * (c[1] + (int64_t)L.ny * c[2])];
        if (lab < 0) continue;
        const int64_t k = rank_of_root(L, W, lab);
        if (k >= L.sizes_cap) continue;
        if (k < VOTE_SMEM) atomicAdd(&sv[k], sign);
        else atomicAdd(W.votes + k, sign);
    }
}

__global__ void __launch_bounds__(256) k_votes(const LatDev L, Work W) {
    __shared__ int sv[VOTE_SMEM];
    for (int i = threadIdx.x; i < VOTE_SMEM; i += blockDim.x) sv[i] = 0;
    __syncthreads();
    const int64_t N = (int64_t)L.nx * L.ny * L.nz;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x)
        vote_site(L, W, s, L.phi[s], sv);
    __syncthreads();
    for (int i = threadIdx.x; i < VOTE_SMEM; i += blockDim.x)
        if (sv[i]) atomicAdd(W.votes + i, sv[i]);
}

__global__ void __launch_bounds__(256) k_inside(const LatDev L, Work W) {
    const int64_t n = *L.ncl < L.sizes_cap ? *L.ncl : L.sizes_cap;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int v = W.votes[k];
        L.inside[k] = (int8_t)(v < 0 ? 1 : (v > 0 ? 0 : -1));
    }
}

// Interior state of every site (Sec. 6: 1 far inside, 0 far outside): a far site
// (I < -0.5) takes its cluster's tag, a near site the side its value names (step 2:
// -d inside, +d outside), 1 for I < 0 and 0 otherwise.  Two passes: each cluster's
// first site (labels[s] == s) gets the tag of its rank, then every far site copies the
// tag from its label's site.  Near sites are never a cluster's first site, so the
// second pass only rewrites first sites with the value they hold.
__device__ __forceinline__ void state_root(const LatDev &L, const Work &W, int8_t *state, int64_t s, int lab) {
    if (lab != s) return;
    const int64_t k = rank_of_root(L, W, (int)s);
    state[s] = k < L.sizes_cap ? L.inside[k] : (int8_t)-1;
}

// vec: labels 16-byte aligned, 4 sites at a time
__global__ void __launch_bounds__(256) k_state_roots(const LatDev L, Work W, int8_t *state, bool vec) {
    const int64_t N = (int64_t)L.nx * L.ny * L.nz;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    int64_t done = 0;
    if (vec) {
        for (int64_t i = t0; i < N / 4; i += stride) {
            const int4 lb = __ldcs(reinterpret_cast<const int4 *>(L.labels) + i);
            state_root(L, W, state, 4 * i, lb.x);
            state_root(L, W, state, 4 * i + 1, lb.y);
            state_root(L, W, state, 4 * i + 2, lb.z);
            state_root(L, W, state, 4 * i + 3, lb.w);
        }
        done = N / 4 * 4;
    }
    for (int64_t s = done + t0; s < N; s += stride) state_root(L, W, state, s, L.labels[s]);
}

__device__ __forceinline__ uint32_t state_byte(const int8_t *state, float v, int lab) {
    if (v < -0.5f) return (uint32_t)(uint8_t)state[lab];
    return v < 0.0f ? 1u : 0u;
}

// vec: phi, labels and state 16-byte aligned, 16 sites at a time (one 16-byte store)
__global__ void __launch_bounds__(256) k_state(const LatDev L, int8_t *state, bool vec) {
    const int64_t N = (int64_t)L.nx * L.ny * L.nz;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    int64_t done = 0;
    if (vec) {
        for (int64_t i = t0; i < N / 16; i += stride) {
            uint32_t w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 v = __ldcs(reinterpret_cast<const float4 *>(L.phi) + 4 * i + q);
                const int4 lb = __ldcs(reinterpret_cast<const int4 *>(L.labels) + 4 * i + q);
                w[q] = state_byte(state, v.x, lb.x) | (state_byte(state, v.y, lb.y) << 8) |
                       (state_byte(state, v.z, lb.z) << 16) | (state_byte(state, v.w, lb.w) << 24);
            }
            reinterpret_cast<int4 *>(state)[i] = make_int4((int)w[0], (int)w[1], (int)w[2], (int)w[3]);
        }
        done = N / 16 * 16;
    }
    for (int64_t s = done + t0; s < N; s += stride) state[s] = (int8_t)state_byte(state, L.phi[s], L.labels[s]);
}

cudaError_t launch_interior(const LatDev &L, const Work &W, cudaStream_t st, int8_t *state) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t N = (int64_t)L.nx * L.ny * L.nz;
    int64_t gv = (N + 255) / 256;
    if (gv > (int64_t)nsm * 16) gv = (int64_t)nsm * 16;
    const unsigned gc = (unsigned)(nsm > 0 ? nsm * 4 : 1);
    k_votes_clear<<<gc, 256, 0, st>>>(L, W);
    auto a16 = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
    const int64_t rows = (int64_t)L.ny * L.nz;
    k_segpre<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(L, W);
    k_votes<<<(unsigned)(gv > 0 ? gv : 1), 256, 0, st>>>(L, W);
    k_inside<<<gc, 256, 0, st>>>(L, W);
    if (state) {
        k_state_roots<<<(unsigned)(gv > 0 ? gv : 1), 256, 0, st>>>(L, W, state, a16(L.labels));
        k_state<<<(unsigned)(gv > 0 ? gv : 1), 256, 0, st>>>(L, state, a16(L.phi) && a16(L.labels) && a16(state));
    }
    return cudaGetLastError();
}

// --------------------------------------------------------------------------------------
// Interior state of slowly moving membranes (Sec. 6, last paragraph): only the sites
// near a membrane now change, to the side their value names; every other site keeps
// its state.
// --------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t update_byte(uint32_t w, int b, float v) {
    const uint32_t side = v < 0.0f ? 1u : 0u;
    return (v < -0.5f) ? w : ((w & ~(0xffu << (8 * b))) | (side << (8 * b)));
}

// Dense form.  vec: all three arrays 16-byte aligned; then 16 sites per step, one
// 16-byte state load and store and four 16-byte index loads.
__global__ void __launch_bounds__(256) k_interior_update(const int8_t *prev, const float *index, int64_t n,
                                                          int8_t *out, bool vec) {
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    int64_t done = 0;
    if (vec) {
        const int64_t nv = n / 16;
        for (int64_t i = t0; i < nv; i += stride) {
            const int4 sp = __ldcs(reinterpret_cast<const int4 *>(prev) + i);
            uint32_t w[4] = {(uint32_t)sp.x, (uint32_t)sp.y, (uint32_t)sp.z, (uint32_t)sp.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 v = __ldcs(reinterpret_cast<const float4 *>(index) + 4 * i + q);
                w[q] = update_byte(w[q], 0, v.x);
                w[q] = update_byte(w[q], 1, v.y);
                w[q] = update_byte(w[q], 2, v.z);
                w[q] = update_byte(w[q], 3, v.w);
            }
            __stcs(reinterpret_cast<int4 *>(out) + i, make_int4((int)w[0], (int)w[1], (int)w[2], (int)w[3]));
        }
        done = nv * 16;
    }
    for (int64_t s = done + t0; s < n; s += stride) {
        const float v = index[s];
        out[s] = (v < -0.5f) ? prev[s] : (int8_t)(v < 0.0f ? 1 : 0);
    }
}

// Sparse form: the caller lists the near sites with their values.
__global__ void __launch_bounds__(256) k_interior_update_sites(int8_t *state, int64_t n, const int32_t *sites,
                                                                const float *values, int64_t m) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = sites[i];
        const float v = values[i];
        if (s >= 0 && s < n && !(v < -0.5f)) state[s] = (int8_t)(v < 0.0f ? 1 : 0);
    }
}

static unsigned stream_grid(int64_t units) {
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int64_t g = (units + 255) / 256;
    const int64_t cap = (int64_t)(nsm > 0 ? nsm : 1) * 8;
    if (g > cap) g = cap;
    return (unsigned)(g > 0 ? g : 1);
}

cudaError_t launch_interior_update(const int8_t *prev, const float *index, int64_t n, int8_t *out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const bool vec = ((reinterpret_cast<uintptr_t>(prev) | reinterpret_cast<uintptr_t>(index) |
                       reinterpret_cast<uintptr_t>(out)) & 15) == 0;
    k_interior_update<<<stream_grid(vec ? n / 16 + 1 : n), 256, 0, st>>>(prev, index, n, out, vec);
    return cudaGetLastError();
}

cudaError_t launch_interior_update_sites(int8_t *state, int64_t n, const int32_t *sites, const float *values,
                                         int64_t m, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    k_interior_update_sites<<<stream_grid(m), 256, 0, st>>>(state, n, sites, values, m);
    return cudaGetLastError();
}

// Copy sized on the device: the host does not know the cluster count when it enqueues
// the copy of the sizes, so a grid-stride kernel reads it and copies that many (dst
// may be page-locked host memory, written across the host link).
__global__ void __launch_bounds__(256) k_copy_counted(const int64_t *src, const int64_t *count, int64_t cap,
                                                       int64_t *dst) {
    const int64_t n = min(*count, cap);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __ldcs(src + i);
}

cudaError_t launch_copy_counted(const int64_t *src, const int64_t *count, int64_t cap, int64_t *dst,
                                cudaStream_t st) {
    if (cap <= 0) return cudaSuccess;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int64_t g = (cap + 255) / 256;
    if (g > (int64_t)nsm * 8) g = (int64_t)nsm * 8;
    k_copy_counted<<<(unsigned)(g > 0 ? g : 1), 256, 0, st>>>(src, count, cap, dst);
    return cudaGetLastError();
}

// --------------------------------------------------------------------------------------
// launch sequence
// --------------------------------------------------------------------------------------
// A kernel of the sequence, launched so that it may be set up while the previous kernel of
// the stream finishes (programmatic dependent launch; the kernel's grid_dep_wait()
// orders it after that kernel).  The first launch error of a sequence is kept in
// launch_error for launch_all to return.
static thread_local cudaError_t launch_error = cudaSuccess;
template <typename... KArgs, typename... Args>
static void launch_dep(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                       Args... args) {
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(block, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, args...);
    if (e != cudaSuccess && launch_error == cudaSuccess) launch_error = e;
}

template <typename K>
static int persistent_grid(K kernel, int threads, size_t smem, int64_t ntiles) {
    int dev = 0, nsm = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
    int64_t g = (int64_t)nsm * (per > 0 ? per : 1);
    if (g > ntiles) g = ntiles;
    return (int)(g > 0 ? g : 1);
}

template <int TY, int TZ, int NL>
static cudaError_t launch_all(const LatDev *lats, int n, const Plan &P, const Work &W, const TmapPair *tms,
                              cudaStream_t st, cudaEvent_t *ev, MergeSchedule ms) {
    using SH = TileShape<TY, TZ>;
    LatBatch<NL> B;
    B.n = n;
    B.pad_ = 0;
    for (int i = 0; i < n; ++i) B.lat[i] = lats[i];
    // tensor maps: the TMA occupancy pass needs every lattice's; flatten picks per tile
    TmapBatch<NL> TB;
    std::memset(&TB, 0, sizeof(TB));
    bool all_tma = n > 0 && tms != nullptr;
    for (int i = 0; i < n; ++i) {
        if (tms) TB.tm[i] = tms[i];
        all_tma = all_tma && TB.tm[i].valid;
    }
    constexpr int CAP1 = LabelCfg<TY, TZ, true>::CAP, CAP1B = LabelCfg<TY, TZ, false>::CAP;
    const size_t smem1 = sizeof(LabelSmem<TY, TZ, CAP1, LabelCfg<TY, TZ, true>::BL>);
    const size_t smem1b = sizeof(LabelSmem<TY, TZ, CAP1B, LabelCfg<TY, TZ, false>::BL>);
    const size_t smem4 = sizeof(FlatSmem<TY, TZ>);
    cudaError_t e;
    // Once per device a process uses: the shared-memory opt-ins (a device attribute of
    // each kernel) and the resident-CTA counts of the persistent passes.
    int dev = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    static std::mutex init_mu;
    static int grid_cache[MAX_DEVICES][3];          // tile pass over dense tiles, flatten, TMA occupancy
    const size_t smem0 = sizeof(OccSmem<TY, TZ>);
    int grid1b, grid4, grid0;
    {
        std::lock_guard<std::mutex> init_lock(init_mu);
        int *c = grid_cache[dev];
        if (!c[1]) {
            e = cudaFuncSetAttribute(k_tile_label<TY, TZ, NL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem1);
            if (e != cudaSuccess) return e;
            e = cudaFuncSetAttribute(k_tile_label<TY, TZ, NL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem1b);
            if (e != cudaSuccess) return e;
            e = cudaFuncSetAttribute(k_flatten<TY, TZ, NL, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem4);
            if (e != cudaSuccess) return e;
            if constexpr (NL == 1) {
                e = cudaFuncSetAttribute(k_flatten<TY, TZ, NL, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem4);
                if (e != cudaSuccess) return e;
            }
            e = cudaFuncSetAttribute(k_occupancy_tma<TY, TZ, NL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem0);
            if (e != cudaSuccess) return e;
            c[0] = persistent_grid(k_tile_label<TY, TZ, NL, false>, SH::NT, smem1b, INT32_MAX);
            c[2] = persistent_grid(k_occupancy_tma<TY, TZ, NL>, 256, smem0, INT32_MAX);
            c[1] = persistent_grid(k_flatten<TY, TZ, NL, false>, SH::NT, smem4, INT32_MAX);
        }
        grid1b = c[0];
        grid4 = c[1];
        grid0 = c[2];
    }
    const unsigned g4 = (unsigned)(P.ntiles < grid4 ? P.ntiles : grid4);
    auto mark = [&](int i) { if (ev) cudaEventRecord(ev[i], st); };
    launch_error = cudaSuccess;
    mark(0);
    if (all_tma) {
        const unsigned g0 = (unsigned)(P.ntiles < grid0 ? P.ntiles : grid0);
        launch_dep(k_occupancy_tma<TY, TZ, NL>, g0, 256, smem0, st, TB, B, W, P.ntiles);
    } else {
        launch_dep(k_occupancy<TY, TZ, NL>, (unsigned)((P.ntiles + 7) / 8), 256, 0, st, B, W, P.ntiles);
    }
    mark(1);
    launch_dep(k_tile_label<TY, TZ, NL, true>, (unsigned)P.ntiles, SH::NT, smem1, st, B, W, P.ntiles);
    // the tiles handed on (none for fields with at most MR_FAST / R runs a row on average)
    launch_dep(k_tile_label<TY, TZ, NL, false>, (unsigned)(P.ntiles < grid1b ? P.ntiles : grid1b), SH::NT, smem1b, st,
               B, W, P.ntiles);
    mark(2);
    const unsigned gfm = (unsigned)((P.ntiles + FM_WARPS - 1) / FM_WARPS);
    if (ms.unions == 1) launch_dep(k_face_merge<TY, TZ, NL, 1>, gfm, 32 * FM_WARPS, 0, st, B, W, P.ntiles);
    else if (ms.unions == 4) launch_dep(k_face_merge<TY, TZ, NL, 4>, gfm, 32 * FM_WARPS, 0, st, B, W, P.ntiles);
    else launch_dep(k_face_merge<TY, TZ, NL, 2>, gfm, 32 * FM_WARPS, 0, st, B, W, P.ntiles);
    mark(3);
    const unsigned gpf = (unsigned)((P.ntiles + PF_WARPS - 1) / PF_WARPS);
    if (ms.hot) launch_dep(k_piece_finalize<NL, true>, gpf, 32 * PF_WARPS, 0, st, B, W, P.ntiles);
    else launch_dep(k_piece_finalize<NL, false>, gpf, 32 * PF_WARPS, 0, st, B, W, P.ntiles);
    mark(4);
    const int64_t nb = (P.nrows + SCAN_CH) / SCAN_CH;   // covers index nrows (the total)
    launch_dep(k_scan_reduce<NL>, (unsigned)nb, SCAN_NT, 0, st, B, (const uint8_t *)W.cnt, P.nrows, W.bsum);
    launch_dep(k_scan_blocks, 1u, 1024u, 0, st, W.bsum, nb);
    launch_dep(k_scan_apply<NL>, (unsigned)nb, SCAN_NT, 0, st, B, (const uint8_t *)W.cnt, P.nrows,
               (const uint32_t *)W.bsum, W.pre);
    mark(5);
    launch_dep(k_lattice_finish<NL>, (unsigned)n, 32u, 0, st, B, W);
    mark(6);
    if constexpr (NL == 1) {
        if (W.roots || W.site_off) launch_dep(k_flatten<TY, TZ, NL, true>, g4, SH::NT, smem4, st, B, TB, W, P.ntiles);
        else launch_dep(k_flatten<TY, TZ, NL, false>, g4, SH::NT, smem4, st, B, TB, W, P.ntiles);
    } else {
        launch_dep(k_flatten<TY, TZ, NL, false>, g4, SH::NT, smem4, st, B, TB, W, P.ntiles);
    }
    mark(7);
    if (launch_error != cudaSuccess) return launch_error;
    return cudaGetLastError();
}

template <int TY, int TZ>
static cudaError_t launch_shape(const LatDev *lats, int n, const Plan &P, const Work &W, const TmapPair *tms,
                                cudaStream_t st, cudaEvent_t *ev, MergeSchedule ms) {
    if (n == 1) return launch_all<TY, TZ, 1>(lats, n, P, W, tms, st, ev, ms);
    return launch_all<TY, TZ, MAX_LAT_PER_LAUNCH>(lats, n, P, W, tms, st, ev, ms);
}

template <int TY, int TZ>
static void shape_info(TileInfo &ti) {
    using SH = TileShape<TY, TZ>;
    ti.ty = TY;
    ti.tz = TZ;
    ti.rows = SH::R;
    ti.maxruns = SH::MAXRUNS;
    ti.face_stride = SH::FACE_STRIDE;
    ti.max_boundary = SH::MAX_BOUNDARY;
}

bool tile_info(int ty, int tz, TileInfo &ti) {
    if (ty == 8 && tz == 8) { shape_info<8, 8>(ti); return true; }
    if (ty == 16 && tz == 8) { shape_info<16, 8>(ti); return true; }
    if (ty == 16 && tz == 16) { shape_info<16, 16>(ti); return true; }
    if (ty == 32 && tz == 8) { shape_info<32, 8>(ti); return true; }
    return false;
}

cudaError_t launch_label(int ty, int tz, const LatDev *lats, int n, const Plan &P, const Work &W, const TmapPair *tms,
                         cudaStream_t st, cudaEvent_t *ev, MergeSchedule ms) {
    if (ty == 8 && tz == 8) return launch_shape<8, 8>(lats, n, P, W, tms, st, ev, ms);
    if (ty == 16 && tz == 8) return launch_shape<16, 8>(lats, n, P, W, tms, st, ev, ms);
    if (ty == 16 && tz == 16) return launch_shape<16, 16>(lats, n, P, W, tms, st, ev, ms);
    if (ty == 32 && tz == 8) return launch_shape<32, 8>(lats, n, P, W, tms, st, ev, ms);
    return cudaErrorInvalidValue;
}

}  // namespace hk
