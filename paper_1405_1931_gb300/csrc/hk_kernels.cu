// hk_kernels.cu -- the labelling passes.
//
//   K1 tile_label     read phi once, write the occupancy mask, label each tile
//                     locally (Sec. 2's rules become union-find over x-runs),
//                     register boundary pieces, write face summaries and the
//                     per-row count of interior cluster roots.
//   K2 face_merge     join boundary pieces across tile faces and periodic
//                     edges: the intra-GPU counterpart of Sec. 3's halo
//                     equivalences, resolved directly on a global union-find
//                     instead of being gathered to a root process.
//   K3 piece_finalize compress the union-find, add piece sizes into cluster
//                     roots and count cluster roots per row segment.
//   S1-S3 scan        exclusive prefix of the root counts: the compactified
//                     cluster numbering 1..n of Sec. 2 in row-major order.
//   K4 flatten        rebuild each tile's local labelling from the mask, map
//                     pieces to their cluster's smallest site index, write the
//                     labels, the sizes in label order and the histogram.
#include "hk_device.cuh"
#include "hk_launch.h"

namespace hk {

template <int NL>
struct LatBatch {
    int n;
    int pad_;
    LatDev lat[NL];
};

// --------------------------------------------------------------------------------------
// K1: tile labelling
// --------------------------------------------------------------------------------------
template <int TY, int TZ, int NL>
__global__ void __launch_bounds__(TY * TZ)
k_tile_label(const __grid_constant__ LatBatch<NL> B, Work W) {
    using SH = TileShape<TY, TZ>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSmem<TY, TZ> &S = *reinterpret_cast<TileSmem<TY, TZ> *>(smem_raw);
    constexpr int R = SH::R, NT = SH::NT, NW = NT / 32;

    const int64_t t = blockIdx.x;
    const int lat = (NL == 1) ? 0 : find_lattice(B.lat, B.n, t);
    const LatDev &L = B.lat[lat];
    const TileGeo g = tile_geo<TY, TZ>(L, lat, t);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;

    // a1: coalesced 128-byte row loads of phi, occupancy by warp ballot
    {
        const int64_t sxy = (int64_t)L.nx * L.ny;
        const float *base = L.phi + (int64_t)g.z0 * sxy + (int64_t)g.y0 * L.nx + g.x0 + lane;
        const bool xin = lane <= g.lastX;
        constexpr int U = 8;
        for (int r0 = wid; r0 < R; r0 += NW * U) {
            float v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int r = r0 + u * NW;
                const int ly = r % TY, lz = r / TY;
                v[u] = 0.0f;
                if (r < R && xin && ly <= g.lastY && lz <= g.lastZ)
                    v[u] = __ldcs(base + (int64_t)lz * sxy + (int64_t)ly * L.nx);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int r = r0 + u * NW;
                const uint32_t word = __ballot_sync(0xffffffffu, v[u] > 0.0f);
                if (lane == 0 && r < R) S.m[r] = word;
            }
        }
    }
    __syncthreads();
    W.mask[t * R + threadIdx.x] = S.m[threadIdx.x];

    tile_local_label<TY, TZ>(S, g, W.status);

    const int r = threadIdx.x;
    if (r == 0) {
        const int base = atomicAdd(W.npieces, S.nbound);
        S.base = base;
        W.tinfo[t] = make_int2(base, S.nbound);
    }
    __syncthreads();
    const int base = S.base;

    // boundary pieces into the global table; interior roots counted per row segment
    const int ly = r % TY, lz = r / TY;
    if (ly <= g.lastY && lz <= g.lastZ) {
        const uint32_t m = S.m[r];
        uint32_t w = run_starts(m);
        int id = S.rbase[r];
        int interior = 0;
        const int site_row = ((g.z0 + lz) * L.ny + (g.y0 + ly)) * L.nx + g.x0;
        while (w) {
            const int x = __ffs(w) - 1;
            w &= w - 1;
            if (S.par[id] == id) {
                if (is_boundary(S.bflag, id)) {
                    const int pid = base + S.kmap[id];
                    W.parent[pid] = pid;
                    W.key[pid] = site_row + x;
                    W.psize[pid] = S.aux[id];
                } else {
                    ++interior;
                }
            }
            ++id;
        }
        const int64_t seg = L.seg0 + ((int64_t)(g.z0 + lz) * L.ny + (g.y0 + ly)) * L.nbx + g.bx;
        W.cnt[seg] = (uint32_t)interior;
    }

    // face summaries: boundary number of the piece holding each face site
    uint16_t *F = W.face + t * SH::FACE_STRIDE;
    auto site_k = [&](int row, int x) -> uint16_t {
        const uint32_t m = S.m[row];
        if (!((m >> x) & 1u)) return FACE_NONE;
        return (uint16_t)S.kmap[S.par[run_of(S.rbase[row], run_starts(m), x)]];
    };
    if (g.extXlo) F[SH::OFF_LX + r] = site_k(r, 0);
    if (g.extXhi) F[SH::OFF_HX + r] = site_k(r, g.lastX);
    for (int e = r; e < TX * TZ; e += NT) {
        const int fz = e / TX, x = e % TX;
        if (g.extYlo) F[SH::OFF_LY + e] = site_k(fz * TY, x);
        if (g.extYhi) F[SH::OFF_HY + e] = site_k(fz * TY + g.lastY, x);
    }
    for (int e = r; e < TX * TY; e += NT) {
        const int fy = e / TX, x = e % TX;
        if (g.extZlo) F[SH::OFF_LZ + e] = site_k(fy, x);
        if (g.extZhi) F[SH::OFF_HZ + e] = site_k(g.lastZ * TY + fy, x);
    }
}

// --------------------------------------------------------------------------------------
// K2: face merge.  Each tile joins its three low faces with the high faces of its
// lower neighbours (for tile 0 of a periodic axis: with the last tile, the wrap).
// --------------------------------------------------------------------------------------
__device__ __forceinline__ void merge_face_run(const uint16_t *Fa, const uint16_t *Fb, int n, int base_a,
                                               int base_b, Work &W) {
    // n is a multiple of 32; lanes cover consecutive x, so a run of equal pairs
    // along x is joined once
    const int lane = threadIdx.x & 31;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const uint16_t a = Fa[e], b = Fb[e];
        const uint32_t pair = ((uint32_t)a << 16) | b;
        const uint32_t prev = __shfl_up_sync(0xffffffffu, pair, 1);
        const bool valid = a != FACE_NONE && b != FACE_NONE;
        if (valid && (lane == 0 || prev != pair))
            g_union(W.parent, W.key, base_a + a, base_b + b, W.piece_cap, W.status);
    }
}

template <int TY, int TZ, int NL>
__global__ void __launch_bounds__(TY * TZ)
k_face_merge(const __grid_constant__ LatBatch<NL> B, Work W) {
    using SH = TileShape<TY, TZ>;
    const int64_t t = blockIdx.x;
    const int lat = (NL == 1) ? 0 : find_lattice(B.lat, B.n, t);
    const LatDev &L = B.lat[lat];
    const TileGeo g = tile_geo<TY, TZ>(L, lat, t);
    const int base = W.tinfo[t].x;
    const uint16_t *F = W.face + t * SH::FACE_STRIDE;

    if (g.extXlo) {
        const int64_t tp = g.bx > 0 ? t - 1 : t + (L.nbx - 1);
        const int bp = W.tinfo[tp].x;
        const uint16_t *Fp = W.face + tp * SH::FACE_STRIDE;
        for (int r = threadIdx.x; r < SH::R; r += blockDim.x) {
            const uint16_t a = F[SH::OFF_LX + r], b = Fp[SH::OFF_HX + r];
            if (a != FACE_NONE && b != FACE_NONE) g_union(W.parent, W.key, base + a, bp + b, W.piece_cap, W.status);
        }
    }
    if (g.extYlo) {
        const int64_t tp = g.by > 0 ? t - L.nbx : t + (int64_t)(L.nby - 1) * L.nbx;
        const uint16_t *Fp = W.face + tp * SH::FACE_STRIDE;
        merge_face_run(F + SH::OFF_LY, Fp + SH::OFF_HY, TX * TZ, base, W.tinfo[tp].x, W);
    }
    if (g.extZlo) {
        const int64_t plane = (int64_t)L.nbx * L.nby;
        const int64_t tp = g.bz > 0 ? t - plane : t + (int64_t)(L.nbz - 1) * plane;
        const uint16_t *Fp = W.face + tp * SH::FACE_STRIDE;
        merge_face_run(F + SH::OFF_LZ, Fp + SH::OFF_HZ, TX * TY, base, W.tinfo[tp].x, W);
    }
}

// --------------------------------------------------------------------------------------
// K3: piece finalize (one warp per tile)
// --------------------------------------------------------------------------------------
template <int NL>
__global__ void __launch_bounds__(256)
k_piece_finalize(const __grid_constant__ LatBatch<NL> B, Work W, int64_t ntiles) {
    const int64_t t = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (t >= ntiles) return;
    const int lane = threadIdx.x & 31;
    const int2 ti = W.tinfo[t];
    if (ti.y == 0) return;
    const int lat = (NL == 1) ? 0 : find_lattice(B.lat, B.n, t);
    const LatDev &L = B.lat[lat];
    for (int j = lane; j < ti.y; j += 32) {
        const int pid = ti.x + j;
        const int root = g_find_ro(W.parent, pid, W.piece_cap, W.status);
        if (root != pid) {
            __stcg(W.parent + pid, root);
            atomicAdd(W.psize + root, W.psize[pid]);
        } else {
            const int k = W.key[pid];
            const int y = (k / L.nx) % L.ny, z = (k / L.nx) / L.ny, x = k % L.nx;
            const int64_t seg = L.seg0 + ((int64_t)z * L.ny + y) * L.nbx + (x >> 5);
            atomicAdd(W.cnt + seg, 1u);
        }
    }
}

// --------------------------------------------------------------------------------------
// S1-S3: exclusive scan of the per-segment root counts
// --------------------------------------------------------------------------------------
constexpr int SCAN_NT = 256;
constexpr int SCAN_PER = 16;
constexpr int SCAN_CH = SCAN_NT * SCAN_PER;

__global__ void __launch_bounds__(SCAN_NT) k_scan_reduce(const uint32_t *cnt, int64_t n, uint32_t *bsum) {
    __shared__ uint32_t red[SCAN_NT / 32];
    const int64_t b0 = (int64_t)blockIdx.x * SCAN_CH;
    uint32_t s = 0;
    for (int j = 0; j < SCAN_PER; ++j) {
        const int64_t i = b0 + (int64_t)j * SCAN_NT + threadIdx.x;
        if (i < n) s += cnt[i];
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

__global__ void __launch_bounds__(SCAN_NT) k_scan_apply(const uint32_t *cnt, int64_t n, const uint32_t *bsum,
                                                        uint32_t *pre) {
    __shared__ uint32_t wsum[SCAN_NT / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t b0 = (int64_t)blockIdx.x * SCAN_CH + (int64_t)threadIdx.x * SCAN_PER;
    uint32_t v[SCAN_PER];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_PER; ++j) {
        const int64_t i = b0 + j;
        v[j] = i < n ? cnt[i] : 0u;
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
        if (i < n) pre[i] = run;
        if (i == n) pre[i] = run;   // total at pre[n]
        run += v[j];
    }
}

// per-lattice: cluster count from the prefix, clear the histogram
template <int NL>
__global__ void k_lattice_finish(const __grid_constant__ LatBatch<NL> B, Work W, int64_t nseg_total) {
    const int l = blockIdx.x;
    if (l >= B.n) return;
    const LatDev &L = B.lat[l];
    if (threadIdx.x < 32 && L.hist) L.hist[threadIdx.x] = 0;
    if (threadIdx.x == 0 && L.ncl) {
        const int64_t nseg = (int64_t)L.nz * L.ny * L.nbx;
        L.ncl[0] = (int64_t)W.pre[L.seg0 + nseg] - (int64_t)W.pre[L.seg0];
    }
}

// --------------------------------------------------------------------------------------
// K4: flatten
// --------------------------------------------------------------------------------------
template <int TY, int TZ, int NL>
__global__ void __launch_bounds__(TY * TZ)
k_flatten(const __grid_constant__ LatBatch<NL> B, Work W) {
    using SH = TileShape<TY, TZ>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSmem<TY, TZ> &S = *reinterpret_cast<TileSmem<TY, TZ> *>(smem_raw);
    constexpr int R = SH::R, NW = SH::NT / 32;

    const int64_t t = blockIdx.x;
    const int lat = (NL == 1) ? 0 : find_lattice(B.lat, B.n, t);
    const LatDev &L = B.lat[lat];
    const TileGeo g = tile_geo<TY, TZ>(L, lat, t);
    const int r = threadIdx.x;
    S.m[r] = W.mask[t * R + r];
    if (r < 32) S.hist[r] = 0;
    __syncthreads();

    tile_local_label<TY, TZ>(S, g, W.status);

    const int base = W.tinfo[t].x;
    const int ly = r % TY, lz = r / TY;
    if (ly <= g.lastY && lz <= g.lastZ) {
        const uint32_t m = S.m[r];
        uint32_t w = run_starts(m);
        if (w) {
            const int64_t seg = L.seg0 + ((int64_t)(g.z0 + lz) * L.ny + (g.y0 + ly)) * L.nbx + g.bx;
            int64_t rank = (int64_t)W.pre[seg] - (int64_t)W.pre[L.seg0];
            const int site_row = ((g.z0 + lz) * L.ny + (g.y0 + ly)) * L.nx + g.x0;
            int id = S.rbase[r];
            while (w) {
                const int x = __ffs(w) - 1;
                w &= w - 1;
                if (S.par[id] == id) {
                    int lab, size = 0;
                    bool root;
                    if (is_boundary(S.bflag, id)) {
                        const int pid = base + S.kmap[id];
                        const int gr = __ldg(W.parent + pid);
                        lab = __ldg(W.key + gr);
                        root = gr == pid;
                        if (root) size = __ldg(W.psize + pid);
                    } else {
                        lab = site_row + x;
                        root = true;
                        size = S.aux[id];
                    }
                    if (root) {
                        if (rank < L.sizes_cap) L.sizes[rank] = size;
                        atomicAdd(&S.hist[31 - __clz(size)], 1);
                        ++rank;
                    }
                    S.aux[id] = lab;
                }
                ++id;
            }
        }
    }
    __syncthreads();

    // a5: labels, one coalesced 128-byte row store per warp step
    {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        const int64_t sxy = (int64_t)L.nx * L.ny;
        int32_t *out = L.labels + (int64_t)g.z0 * sxy + (int64_t)g.y0 * L.nx + g.x0 + lane;
        const bool xin = lane <= g.lastX;
        for (int rr = wid; rr < R; rr += NW) {
            const int yy = rr % TY, zz = rr / TY;
            if (!xin || yy > g.lastY || zz > g.lastZ) continue;
            const uint32_t m = S.m[rr];
            int lab = -1;
            if ((m >> lane) & 1u) lab = S.aux[S.par[run_of(S.rbase[rr], run_starts(m), lane)]];
            __stcs(out + (int64_t)zz * sxy + (int64_t)yy * L.nx, lab);
        }
    }
    if (L.hist && r < 32 && S.hist[r])
        atomicAdd(reinterpret_cast<unsigned long long *>(L.hist) + r, (unsigned long long)S.hist[r]);
}

// --------------------------------------------------------------------------------------
// launch sequence
// --------------------------------------------------------------------------------------
template <int TY, int TZ>
static size_t tile_smem_bytes() { return sizeof(TileSmem<TY, TZ>); }

template <int TY, int TZ, int NL>
static cudaError_t launch_all(const LatDev *lats, int n, const Plan &P, const Work &W, cudaStream_t st,
                              cudaEvent_t *ev) {
    using SH = TileShape<TY, TZ>;
    LatBatch<NL> B;
    B.n = n;
    B.pad_ = 0;
    for (int i = 0; i < n; ++i) B.lat[i] = lats[i];
    const size_t smem = tile_smem_bytes<TY, TZ>();
    cudaError_t e;
    static bool attr_done = false;
    if (!attr_done) {
        e = cudaFuncSetAttribute(k_tile_label<TY, TZ, NL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_flatten<TY, TZ, NL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    e = cudaMemsetAsync(W.npieces, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)P.ntiles;
    auto mark = [&](int i) { if (ev) cudaEventRecord(ev[i], st); };
    mark(0);
    k_tile_label<TY, TZ, NL><<<grid, SH::NT, smem, st>>>(B, W);
    mark(1);
    k_face_merge<TY, TZ, NL><<<grid, SH::NT, 0, st>>>(B, W);
    mark(2);
    k_piece_finalize<NL><<<(unsigned)((P.ntiles + 7) / 8), 256, 0, st>>>(B, W, P.ntiles);
    mark(3);
    const int64_t nb = (P.nseg + SCAN_CH) / SCAN_CH;   // covers index nseg (the total)
    k_scan_reduce<<<(unsigned)nb, SCAN_NT, 0, st>>>(W.cnt, P.nseg, W.bsum);
    k_scan_blocks<<<1, 1024, 0, st>>>(W.bsum, nb);
    k_scan_apply<<<(unsigned)nb, SCAN_NT, 0, st>>>(W.cnt, P.nseg, W.bsum, W.pre);
    mark(4);
    k_lattice_finish<NL><<<(unsigned)n, 32, 0, st>>>(B, W, P.nseg);
    mark(5);
    k_flatten<TY, TZ, NL><<<grid, SH::NT, smem, st>>>(B, W);
    mark(6);
    return cudaGetLastError();
}

template <int TY, int TZ>
static cudaError_t launch_shape(const LatDev *lats, int n, const Plan &P, const Work &W, cudaStream_t st,
                                cudaEvent_t *ev) {
    if (n == 1) return launch_all<TY, TZ, 1>(lats, n, P, W, st, ev);
    return launch_all<TY, TZ, MAX_LAT_PER_LAUNCH>(lats, n, P, W, st, ev);
}

template <int TY, int TZ>
static void shape_info(TileInfo &ti) {
    using SH = TileShape<TY, TZ>;
    ti.ty = TY;
    ti.tz = TZ;
    ti.rows = SH::R;
    ti.face_stride = SH::FACE_STRIDE;
    ti.max_boundary = SH::MAX_BOUNDARY;
    ti.smem = sizeof(TileSmem<TY, TZ>);
}

bool tile_info(int ty, int tz, TileInfo &ti) {
    if (ty == 8 && tz == 8) { shape_info<8, 8>(ti); return true; }
    if (ty == 16 && tz == 8) { shape_info<16, 8>(ti); return true; }
    if (ty == 16 && tz == 16) { shape_info<16, 16>(ti); return true; }
    if (ty == 32 && tz == 8) { shape_info<32, 8>(ti); return true; }
    return false;
}

cudaError_t launch_label(int ty, int tz, const LatDev *lats, int n, const Plan &P, const Work &W, cudaStream_t st,
                         cudaEvent_t *ev) {
    if (ty == 8 && tz == 8) return launch_shape<8, 8>(lats, n, P, W, st, ev);
    if (ty == 16 && tz == 8) return launch_shape<16, 8>(lats, n, P, W, st, ev);
    if (ty == 16 && tz == 16) return launch_shape<16, 16>(lats, n, P, W, st, ev);
    if (ty == 32 && tz == 8) return launch_shape<32, 8>(lats, n, P, W, st, ev);
    return cudaErrorInvalidValue;
}

}  // namespace hk
