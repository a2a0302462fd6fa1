// hk_small.cu -- one launch for small lattices: one CTA labels a whole lattice of at
// most SMALL_MAX_SITES sites in shared memory (a batch of such lattices: one CTA each).
//
// The tiled passes of hk_kernels.cu need about ten launches per call, whose gaps are
// the whole cost of a 32^3 lattice.  Here every step runs in one kernel, separated by
// barriers instead of launches:
//   a1  occupancy phi > 0 (Sec. 2) as one 32-bit word per row segment (32 sites along x);
//   a2  x-runs numbered in row-major order, union-find over them in shared memory with
//       union by minimum run id (Sec. 2's rules 1-3 applied to runs);
//   a3  the unions along x between segments, along y and z, and across every periodic
//       edge (Sec. 3, halo paragraph and Fig. 2 caption);
//   a4  the clusters' ranks: a scan of the root flags in run order, which is label order
//       (Sec. 2, final paragraph);
//   a5  labels: the smallest site of the cluster, -1 for the medium;
//   a6  sizes in label order (Sec. 5), a7 the floor(log2 size) histogram.
// Runs are numbered in row-major order of their first sites, so each cluster's root
// (its smallest run id) holds its smallest site, and ranking roots by run id ranks the
// clusters by label.  No workspace is used: the results go straight to the outputs.
#include <cooperative_groups.h>

#include <cstddef>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "hk_device.cuh"
#include "hk_launch.h"

namespace hk {

namespace {

constexpr int SNT = 1024;   // threads of the one CTA per lattice

struct SmallSmem {
    uint32_t m[SMALL_MAX_SEG];         // occupancy word of each row segment (row-major)
    uint16_t sb[SMALL_MAX_SEG];        // first run id of each segment
    int par[SMALL_MAX_RUNS];           // union-find over run ids; after compression: the root
    int sz[SMALL_MAX_RUNS];            // piece size, summed at each root
    uint16_t desc[SMALL_MAX_RUNS];     // per run: (segment << 5) | first x
    int warp_tmp[32];
    int scan_total;
    int hist[32];
};
static_assert(SMALL_MAX_SEG <= 2048 && SMALL_MAX_RUNS <= 65535, "desc holds an 11-bit segment, sb a 16-bit run id");
static_assert(sizeof(SmallSmem) <= 227 * 1024, "one CTA's shared memory");

// Division by a lattice constant d >= 1 by one multiply: floor(x / d) =
// (x * ceil(2^32 / d)) >> 32, exact while x * d < 2^32 (here x < 2^16 and d <= 2^15).
struct FastDiv {
    uint64_t m;
    __device__ explicit FastDiv(uint32_t d) : m(((1ull << 32) + d - 1) / d) {}
    __device__ __forceinline__ uint32_t operator()(uint32_t x) const { return (uint32_t)((x * m) >> 32); }
};

// the run of segment s (first run id b, occupancy word w) holding bit x
__device__ __forceinline__ int srun(int b, uint32_t w, int x) { return b + __popc(run_starts(w) & le_mask(x)) - 1; }

// Exclusive scan of one int per thread over the CTA's NT threads (NT a multiple of 32,
// at most 1024); *total gets the sum.  Ends with a barrier, after which warp_tmp and
// scan_total may be reused.
template <int NT, class SM>
__device__ __forceinline__ int cta_exscan(int v, SM &S, int &total) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int u = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += u;
    }
    if (lane == 31) S.warp_tmp[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const int w = lane < NW ? S.warp_tmp[lane] : 0;
        int wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += u;
        }
        if (lane < NW) S.warp_tmp[lane] = wi - w;
        if (lane == 31) S.scan_total = wi;
    }
    __syncthreads();
    const int r = S.warp_tmp[wid] + inc - v;
    total = S.scan_total;
    __syncthreads();
    return r;
}

template <int NL>
__global__ void __launch_bounds__(SNT, 1) k_small_label(const __grid_constant__ LatBatch<NL> B, int32_t *status,
                                                         int32_t local_cap) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmallSmem &S = *reinterpret_cast<SmallSmem *>(smem_raw);
    const LatDev &L = B.lat[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    constexpr int NW = SNT / 32;
    const int nx = L.nx, ny = L.ny, nz = L.nz, nbx = L.nbx;
    const int nseg = nbx * ny * nz;
    const FastDiv div_nbx((uint32_t)nbx), div_ny((uint32_t)ny);
    if (tid < 32) S.hist[tid] = 0;

    // a1: occupancy words; each warp keeps up to 32 segments' loads in flight (a 32^3
    // lattice in one round trip)
    constexpr int INF = 32;
    for (int s0 = wid; s0 < nseg; s0 += NW * INF) {
        float v[INF];
#pragma unroll
        for (int j = 0; j < INF; ++j) {
            const int s = s0 + NW * j;
            const int q = (int)div_nbx((uint32_t)s), x = (s - q * nbx) * 32 + lane;
            v[j] = (s < nseg && x < nx) ? __ldg(L.phi + (int64_t)q * nx + x) : 0.0f;
        }
#pragma unroll
        for (int j = 0; j < INF; ++j) {
            const uint32_t w = __ballot_sync(0xffffffffu, occupied(v[j], L.occ_mode));
            if (lane == 0 && s0 + NW * j < nseg) S.m[s0 + NW * j] = w;
        }
    }
    __syncthreads();

    // a2: run ids: a scan of the run counts of segments 2t and 2t + 1
    const int s_a = 2 * tid, s_b = 2 * tid + 1;
    const int n_a = s_a < nseg ? __popc(run_starts(S.m[s_a])) : 0;
    const int n_b = s_b < nseg ? __popc(run_starts(S.m[s_b])) : 0;
    int total;
    const int base = cta_exscan<SNT>(n_a + n_b, S, total);
    if (s_a < nseg) S.sb[s_a] = (uint16_t)base;
    if (s_b < nseg) S.sb[s_b] = (uint16_t)(base + n_a);
    for (int h = 0; h < 2; ++h) {   // own node and descriptor of every run
        const int s = 2 * tid + h;
        if (s >= nseg) break;
        uint32_t w = run_starts(S.m[s]);
        int id = base + (h ? n_a : 0);
        while (w) {
            const int x0 = __ffs(w) - 1;
            w &= w - 1;
            S.par[id] = id;
            S.sz[id] = 0;
            S.desc[id] = (uint16_t)((s << 5) | x0);
            ++id;
        }
    }
    __syncthreads();

    // a3: unions with the lower neighbours along x (previous segment), y and z, and
    // across the periodic edges (the wrap of an axis of length 1 is a self-edge; one of
    // length 2 repeats an interior edge)
    const int cap = (local_cap > 0 && local_cap < total) ? local_cap : total;
    const int lastbit = (nx - 1) & 31;   // bit of x = nx - 1 in the last segment of a row
    for (int s = tid; s < nseg; s += SNT) {   // strided: every thread has a segment up to 1024 of them
        const uint32_t w = S.m[s];
        if (!w) continue;
        const int b = S.sb[s];
        const int q = (int)div_nbx((uint32_t)s), bx = s - q * nbx, z = (int)div_ny((uint32_t)q), y = q - z * ny;
        auto join = [&](int t) {   // every overlap of segment s with segment t
            const uint32_t wt = S.m[t];
            uint32_t os = run_starts(w & wt);
            const int bt = S.sb[t];
            while (os) {
                const int x = __ffs(os) - 1;
                os &= os - 1;
                s_union(S.par, srun(b, w, x), srun(bt, wt, x), cap, status);
            }
        };
        if (y > 0) join(s - nbx);
        else if (L.per[1] && ny >= 2) join(s + (ny - 1) * nbx);
        if (z > 0) join(s - nbx * ny);
        else if (L.per[2] && nz >= 2) join(s + (nz - 1) * nbx * ny);
        if ((w & 1u) && bx > 0 && (S.m[s - 1] >> 31))
            s_union(S.par, b, srun(S.sb[s - 1], S.m[s - 1], 31), cap, status);
        if ((w & 1u) && bx == 0 && L.per[0] && nx >= 2) {
            const int t = s + nbx - 1;
            if ((S.m[t] >> lastbit) & 1u) s_union(S.par, b, srun(S.sb[t], S.m[t], lastbit), cap, status);
        }
    }
    __syncthreads();

    // compression and piece sizes
    for (int i = tid; i < total; i += SNT) {
        const int root = s_find_ro(S.par, i);
        S.par[i] = root;
        const int d = S.desc[i];
        atomicAdd(&S.sz[root], run_len(S.m[d >> 5], d & 31));
    }
    __syncthreads();

    // a4, a6, a7: roots in run order get consecutive ranks; each thread takes a
    // contiguous block of run ids
    const int per = (total + SNT - 1) / SNT;
    const int i0 = tid * per, i1 = min(i0 + per, total);
    int nr = 0;
    for (int i = i0; i < i1; ++i) nr += S.par[i] == i;
    int nclus;
    int rank = cta_exscan<SNT>(nr, S, nclus);
    const int64_t capr = L.sizes_cap;
    for (int i = i0; i < i1; ++i) {
        if (S.par[i] != i) continue;
        const int size = S.sz[i];
        if (rank < capr) L.sizes[rank] = size;
        ++rank;
        atomicAdd(&S.hist[31 - __clz(size)], 1);
        const int d = S.desc[i], rs_ = d >> 5, rq = (int)div_nbx((uint32_t)rs_);
        S.sz[i] = rq * nx + (rs_ - rq * nbx) * 32 + (d & 31);   // from here on: the root's site (its label)
    }
    __syncthreads();

    // a5: labels, one warp per segment, one lane per site
    for (int s = wid; s < nseg; s += NW) {
        const int q = (int)div_nbx((uint32_t)s), x = (s - q * nbx) * 32 + lane;
        if (x >= nx) continue;
        const uint32_t w = S.m[s];
        const int lab = ((w >> lane) & 1u) ? S.sz[S.par[srun(S.sb[s], w, lane)]] : -1;
        L.labels[(int64_t)q * nx + x] = lab;
    }
    __syncthreads();
    if (tid < 32 && L.hist) L.hist[tid] = S.hist[tid];
    if (tid == 0 && L.ncl) L.ncl[0] = nclus;
}

// ---------------------------------------------------------------------------------------
// The same steps on a thread-block cluster: CS CTAs on CS SMs label one lattice, each
// holding the rows [c RP, (c + 1) RP) of the lattice (RP = ceil(ny nz / CS)) in its own
// shared memory, so that the loads, unions, ranks and label stores are spread over CS
// SMs.  A run of CTA c is numbered (c << CRUN_BITS) | its local id: numbers grow with
// the runs' first sites in row-major order, so union by minimum number still makes each
// cluster's root its first run.  Each CTA first joins the edges inside it on local ids;
// the edges to other CTAs are then joined between local roots, through distributed
// shared memory (the other CTAs' parents, occupancy words and run bases); every local
// root then learns its cluster root, so each run reaches its root in two steps, and
// each run's label is resolved once per run, not per site.  The phases that reach other
// CTAs are separated by cluster barriers.
// ---------------------------------------------------------------------------------------
// CTAs per lattice: 16 where the device co-schedules that many (a non-portable cluster
// size), else 8 (the portable size); a template parameter of the kernel (CSB = log2).
constexpr int CNT = 1024;          // threads per CTA
constexpr int CSEG = 1024;         // row segments per CTA
constexpr int CRUN_BITS = 14;
constexpr int CRUN = 1 << CRUN_BITS;   // runs per CTA: at most 16 per segment
constexpr int DESC_LROOT = 0x8000;     // desc flag: the run is the root of its CTA-local tree
static_assert(16 * CSEG <= CRUN && CSEG <= 2 * CNT, "run ids of a CTA; two segments per thread in the scan");

struct ClusterSmem {
    uint32_t m[CSEG];        // occupancy word of each of this CTA's row segments
    uint16_t sb[CSEG];       // first local run id of each segment
    int par[CRUN];           // union-find over cluster run numbers; after compression: the root
    int sz[CRUN];            // piece size, summed at each root; after ranking: the root's site
    uint16_t desc[CRUN];     // per run: (local segment << 5) | first x, and DESC_LROOT
    int roots;               // cluster roots among this CTA's runs
    uint64_t bar;            // completion of the bulk copy of this CTA's rows of phi
    int warp_tmp[32];
    int scan_total;
    int hist[32];
};
static_assert(sizeof(ClusterSmem) <= 227 * 1024, "one CTA's shared memory");
static_assert(offsetof(ClusterSmem, sz) == offsetof(ClusterSmem, par) + sizeof(int) * CRUN &&
                  sizeof(int) * 2 * CRUN >= sizeof(float) * TX * CSEG,
              "par and sz together hold a CTA's rows of phi");

namespace cg = cooperative_groups;

struct ClusterView {
    ClusterSmem &S;
    cg::cluster_group cl;
    int c;
    // parent of run number g, wherever it lives
    __device__ __forceinline__ int *par(int g) const {
        int *p = &S.par[g & (CRUN - 1)];
        const int o = g >> CRUN_BITS;
        return o == c ? p : cl.map_shared_rank(p, o);
    }
    __device__ __forceinline__ int *sz(int g) const {
        int *p = &S.sz[g & (CRUN - 1)];
        const int o = g >> CRUN_BITS;
        return o == c ? p : cl.map_shared_rank(p, o);
    }
    // find with path halving (every store lowers a parent to an ancestor)
    __device__ int find(int x) const {
        int p = *par(x);
        while (p != x) {
            const int gp = *par(p);
            if (gp == p) return p;
            *par(x) = gp;
            x = gp;
            p = *par(x);
        }
        return x;
    }
    __device__ int find_ro(int x) const {
        int p = *par(x);
        while (p != x) {
            x = p;
            p = *par(x);
        }
        return x;
    }
    // each retry strictly lowers max(a, b): at most `cap` rounds
    __device__ void unite(int a, int b, int cap, int32_t *status) const {
        for (int it = 0; it <= cap; ++it) {
            a = find(a);
            b = find(b);
            if (a == b) return;
            const int hi = a > b ? a : b, lo = a > b ? b : a;
            const int old = atomicMin(par(hi), lo);
            if (old == hi) return;
            a = lo;
            b = old;
        }
        atomicOr(status, STATUS_LOCAL_LOOP);
    }
};

template <int CSB, int NL>
__global__ void __cluster_dims__(1 << CSB, 1, 1) __launch_bounds__(CNT, 1)
    k_small_cluster(const __grid_constant__ LatBatch<NL> B, int32_t *status, int32_t local_cap) {
    constexpr int CS_BITS = CSB, CS = 1 << CSB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ClusterSmem &S = *reinterpret_cast<ClusterSmem *>(smem_raw);
    cg::cluster_group cl = cg::this_cluster();
    const int c = (int)cl.block_rank();
    const ClusterView V{S, cl, c};
    const LatDev &L = B.lat[blockIdx.x / CS];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    constexpr int NW = CNT / 32;
    const int nx = L.nx, ny = L.ny, nz = L.nz, nbx = L.nbx;
    const int nrows = ny * nz, rp = (nrows + CS - 1) / CS;       // rows per CTA
    const int q0 = min(c * rp, nrows), q1 = min(q0 + rp, nrows);
    const int seg0 = q0 * nbx, nseg = (q1 - q0) * nbx;           // this CTA's segments
    const FastDiv div_nbx((uint32_t)nbx), div_ny((uint32_t)ny), div_rp((uint32_t)rp);
    const int cbase = c << CRUN_BITS;
    if (tid < 32) S.hist[tid] = 0;

    // a1: occupancy words of this CTA's segments.  Its rows of phi are one contiguous
    // range: one bulk copy lands it in par and sz (not in use yet) when it is 16-byte
    // aligned, and each warp turns landed segments into words by ballots; otherwise (or
    // if the copy does not complete within its bound) 32 loads in flight per warp.
    bool landed = false;
    {
        const float *src = L.phi + (int64_t)q0 * nx;
        const int nfl = (q1 - q0) * nx;
        if (nfl > 0 && (nfl & 3) == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {   // uniform
            const float *land = reinterpret_cast<const float *>(S.par);
            if (tid == 0) {
                mbar_init(&S.bar, 1);
                fence_mbar_init();
            }
            __syncthreads();
            if (tid == 0) {
                mbar_arrive_expect_tx(&S.bar, (uint32_t)nfl * 4u);
                bulk_load(S.par, src, (uint32_t)nfl * 4u, &S.bar);
            }
            landed = mbar_wait_bounded(&S.bar, 0);
            if (__syncthreads_or(!landed)) {
                if (tid == 0) atomicOr(status, STATUS_TMA_TIMEOUT);
                mbar_wait_bounded(&S.bar, 0);   // the copy still in flight
                landed = false;
            } else {
                landed = true;
                for (int ls = wid; ls < nseg; ls += NW) {
                    const int r = (int)div_nbx((uint32_t)ls), x = (ls - r * nbx) * 32 + lane;
                    const float v = x < nx ? land[r * nx + x] : 0.0f;
                    const uint32_t w = __ballot_sync(0xffffffffu, occupied(v, L.occ_mode));
                    if (lane == 0) S.m[ls] = w;
                }
            }
        }
    }
    constexpr int INF = 32;
    for (int l0 = landed ? nseg : wid; l0 < nseg; l0 += NW * INF) {
        float v[INF];
#pragma unroll
        for (int j = 0; j < INF; ++j) {
            const int ls = l0 + NW * j, sg = seg0 + ls;
            const int q = (int)div_nbx((uint32_t)sg), x = (sg - q * nbx) * 32 + lane;
            v[j] = (ls < nseg && x < nx) ? __ldg(L.phi + (int64_t)q * nx + x) : 0.0f;
        }
#pragma unroll
        for (int j = 0; j < INF; ++j) {
            const uint32_t w = __ballot_sync(0xffffffffu, occupied(v[j], L.occ_mode));
            if (lane == 0 && l0 + NW * j < nseg) S.m[l0 + NW * j] = w;
        }
    }
    __syncthreads();

    // a2: local run ids (segments 2t and 2t + 1 of thread t), nodes and descriptors
    const int s_a = 2 * tid, s_b = 2 * tid + 1;
    const int n_a = s_a < nseg ? __popc(run_starts(S.m[s_a])) : 0;
    const int n_b = s_b < nseg ? __popc(run_starts(S.m[s_b])) : 0;
    int total;
    const int base = cta_exscan<CNT>(n_a + n_b, S, total);
    if (s_a < nseg) S.sb[s_a] = (uint16_t)base;
    if (s_b < nseg) S.sb[s_b] = (uint16_t)(base + n_a);
    for (int h = 0; h < 2; ++h) {
        const int ls = 2 * tid + h;
        if (ls >= nseg) break;
        uint32_t w = run_starts(S.m[ls]);
        int id = base + (h ? n_a : 0);
        while (w) {
            const int x0 = __ffs(w) - 1;
            w &= w - 1;
            S.par[id] = id;   // local ids until the edges inside this CTA are joined
            S.desc[id] = (uint16_t)((ls << 5) | x0);
            ++id;
        }
    }
    __syncthreads();

    // a3: unions with the lower neighbours along x, y and z and across the periodic
    // edges, in two rounds.  First the edges inside this CTA, on local run ids in its own
    // shared memory; then, once every CTA has compressed its runs onto their local roots,
    // the edges to runs of other CTAs, joined between local roots through distributed
    // shared memory.  Each round lists its run pairs first (a scan of per-segment counts;
    // sz serves as the list), so that the unions spread over all threads; a round whose
    // list would not fit joins each segment's pairs where they are found.
    const int lastbit = (nx - 1) & 31;
    auto neighbours = [&](int ls, auto &&edge) {   // edge(global segment t) for every lower neighbour
        const int sg = seg0 + ls;
        const int q = (int)div_nbx((uint32_t)sg), z = (int)div_ny((uint32_t)q), y = q - z * ny;
        if (y > 0) edge(sg - nbx);
        else if (L.per[1] && ny >= 2) edge(sg + (ny - 1) * nbx);
        if (z > 0) edge(sg - nbx * ny);
        else if (L.per[2] && nz >= 2) edge(sg + (nz - 1) * nbx * ny);
    };
    auto owner = [&](int t, int &lt) {   // the CTA holding global segment t, and its local index there
        const int tq = (int)div_nbx((uint32_t)t), o = (int)div_rp((uint32_t)tq);
        lt = t - o * rp * nbx;
        return o;
    };
    // every pair of runs joined by an edge of segment ls: pair(own local run, CTA, its run)
    auto pairs = [&](int ls, bool cross, auto &&pair) {
        const uint32_t w = S.m[ls];
        if (!w) return;
        const int b = S.sb[ls];
        neighbours(ls, [&](int t) {
            int lt;
            const int o = owner(t, lt);
            if ((o != c) != cross) return;
            const uint32_t wt = o == c ? S.m[lt] : *cl.map_shared_rank(&S.m[lt], o);
            uint32_t os = run_starts(w & wt);
            if (!os) return;
            const int bt = o == c ? S.sb[lt] : *cl.map_shared_rank(&S.sb[lt], o);
            while (os) {
                const int x = __ffs(os) - 1;
                os &= os - 1;
                pair(srun(b, w, x), o, srun(bt, wt, x));
            }
        });
        if (cross) return;
        const int bx = (seg0 + ls) - (int)div_nbx((uint32_t)(seg0 + ls)) * nbx;   // a row lives in one CTA
        if ((w & 1u) && bx > 0 && (S.m[ls - 1] >> 31)) pair(b, c, srun(S.sb[ls - 1], S.m[ls - 1], 31));
        if ((w & 1u) && bx == 0 && L.per[0] && nx >= 2) {
            const int t = ls + nbx - 1;
            if ((S.m[t] >> lastbit) & 1u) pair(b, c, srun(S.sb[t], S.m[t], lastbit));
        }
    };
    // one round: count, list and join the pairs of this thread's segments (2t, 2t + 1)
    auto round = [&](bool cross, auto &&join) {
        int np = 0;
        for (int h = 0; h < 2; ++h)
            if (2 * tid + h < nseg) pairs(2 * tid + h, cross, [&](int, int, int) { ++np; });
        int npairs;
        int j = cta_exscan<CNT>(np, S, npairs);
        if (npairs <= CRUN) {
            for (int h = 0; h < 2; ++h)
                if (2 * tid + h < nseg)
                    pairs(2 * tid + h, cross, [&](int a, int o, int bb) {
                        S.sz[j++] = (int)(((uint32_t)a << (CRUN_BITS + CS_BITS)) | ((uint32_t)o << CRUN_BITS) |
                                          (uint32_t)bb);
                    });
            __syncthreads();
            for (int k = tid; k < npairs; k += CNT) {
                const int v = S.sz[k];
                const uint32_t u = (uint32_t)v;
                join((int)(u >> (CRUN_BITS + CS_BITS)), (int)((u >> CRUN_BITS) & (CS - 1)), (int)(u & (CRUN - 1)));
            }
        } else {
            for (int h = 0; h < 2; ++h)
                if (2 * tid + h < nseg) pairs(2 * tid + h, cross, join);
        }
    };
    static_assert(2 * CRUN_BITS + CS_BITS <= 32 && CS <= 32, "a listed pair packs into 32 bits");
    {
        const int lcap = (local_cap > 0 && local_cap < total) ? local_cap : total;
        round(false, [&](int a, int, int bb) { s_union(S.par, a, bb, lcap, status); });
        __syncthreads();
        // local roots, then cluster numbers: every run points at its local root
        for (int i = tid; i < total; i += CNT) S.sz[i] = s_find_ro(S.par, i);
        __syncthreads();
        for (int i = tid; i < total; i += CNT) {
            const int r = S.sz[i];
            S.par[i] = cbase | r;
            if (r == i) S.desc[i] |= DESC_LROOT;
        }
    }
    cl.sync();
    {   // the edges to other CTAs, joined between the two runs' local roots
        const int cap = (local_cap > 0 && local_cap < CS * CRUN) ? local_cap : CS * CRUN;
        round(true, [&](int a, int o, int bb) {
            V.unite(S.par[a], *cl.map_shared_rank(&S.par[bb], o), cap, status);
        });
    }
    __syncthreads();                                  // the pair list is read
    for (int i = tid; i < total; i += CNT) S.sz[i] = 0;
    cl.sync();                                        // ... and every size slot cleared
    // every local root learns its cluster's root (the finds that cross CTAs walk only
    // local roots); the other runs still point at their local roots
    for (int i = tid; i < total; i += CNT)
        if (S.desc[i] & DESC_LROOT) S.par[i] = V.find_ro(cbase | i);
    __syncthreads();

    // piece sizes: every run's length goes to its local root, in this CTA's shared
    // memory; a local root that is not its cluster's root then passes its sum on to the
    // cluster root, once per group of lanes with the same cluster root
    for (int i = tid; i < total; i += CNT) {
        const int d = S.desc[i];
        const int lr = (d & DESC_LROOT) ? i : (S.par[i] & (CRUN - 1));
        atomicAdd(&S.sz[lr], run_len(S.m[(d & ~DESC_LROOT) >> 5], d & 31));
    }
    __syncthreads();
    for (int i0 = 0; i0 < total; i0 += CNT) {   // warp-uniform trips
        const int i = i0 + tid;
        int root = -1, sum = 0;
        if (i < total && (S.desc[i] & DESC_LROOT) && S.par[i] != (cbase | i)) {
            root = S.par[i];
            sum = S.sz[i];
        }
        const unsigned peers = __match_any_sync(0xffffffffu, root);
        const int tot = (int)__reduce_add_sync(peers, (unsigned)sum);
        if (root >= 0 && lane == __ffs(peers) - 1) atomicAdd(V.sz(root), tot);
    }
    __syncthreads();
    for (int i = tid; i < total; i += CNT)   // every run now points at its cluster root
        if (!(S.desc[i] & DESC_LROOT)) S.par[i] = S.par[S.par[i] & (CRUN - 1)];

    // a4, a6, a7: the roots in run order get consecutive ranks; the roots of the CTAs
    // before this one come first.  The cluster roots (local roots pointing at
    // themselves) are counted before the barrier that completes the sizes, which then
    // publishes the counts too.
    const int per = (total + CNT - 1) / CNT;
    const int i0 = tid * per, i1 = min(i0 + per, total);
    int nr = 0;
    for (int i = i0; i < i1; ++i) nr += S.par[i] == (cbase | i);
    int nroots;
    int rank = cta_exscan<CNT>(nr, S, nroots);
    if (tid == 0) S.roots = nroots;
    cl.sync();
    int all = 0;
    if (wid == 0) {
        const int r = lane < CS ? (lane == c ? nroots : *cl.map_shared_rank(&S.roots, lane)) : 0;
        const int before = (int)__reduce_add_sync(0xffffffffu, (unsigned)(lane < c ? r : 0));
        all = (int)__reduce_add_sync(0xffffffffu, (unsigned)r);
        if (lane == 0) S.scan_total = before;
    }
    __syncthreads();
    rank += S.scan_total;
    const int64_t capr = L.sizes_cap;
    for (int i = i0; i < i1; ++i) {
        if (S.par[i] != (cbase | i)) continue;
        const int size = S.sz[i];
        if (rank < capr) L.sizes[rank] = size;
        ++rank;
        atomicAdd(&S.hist[31 - __clz(size)], 1);
    }
    __syncthreads();   // this CTA's sizes are out: sz now takes each run's label

    // each run's label, the first site of its cluster's root run (the root's descriptor,
    // read once per group of lanes with the same root)
    for (int i0 = 0; i0 < total; i0 += CNT) {
        const int i = i0 + tid;
        const int root = i < total ? S.par[i] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, root);
        const int leader = __ffs(peers) - 1;
        int d = 0;
        if (root >= 0 && lane == leader) {
            const int o = root >> CRUN_BITS;
            const uint16_t *dp = &S.desc[root & (CRUN - 1)];
            d = o == c ? *dp : *cl.map_shared_rank(dp, o);
        }
        d = __shfl_sync(0xffffffffu, d, leader) & ~DESC_LROOT;
        if (i < total) {
            const int sg = (root >> CRUN_BITS) * rp * nbx + (d >> 5), rq = (int)div_nbx((uint32_t)sg);
            S.sz[i] = rq * nx + (sg - rq * nbx) * 32 + (d & 31);
        }
    }
    __syncthreads();

    // a5: labels, one warp per segment, one lane per site, four segments a step
    for (int l0 = wid; l0 < nseg; l0 += 4 * NW) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int ls = l0 + u * NW;
            if (ls >= nseg) break;
            const int sg = seg0 + ls;
            const int q = (int)div_nbx((uint32_t)sg), x = (sg - q * nbx) * 32 + lane;
            const uint32_t w = S.m[ls];
            const int lab = ((w >> lane) & 1u) ? S.sz[srun(S.sb[ls], w, lane)] : -1;
            if (x < nx) L.labels[(int64_t)q * nx + x] = lab;
        }
    }
    // the histogram of the whole lattice gathers in CTA 0
    if (c != 0 && tid < 32 && S.hist[tid]) atomicAdd(cl.map_shared_rank(&S.hist[tid], 0), S.hist[tid]);
    cl.sync();   // no CTA's shared memory is reached after this
    if (c == 0) {
        if (tid < 32 && L.hist) L.hist[tid] = S.hist[tid];
        if (tid == 0 && L.ncl) L.ncl[0] = all;
    }
}

}  // namespace

bool small_fits(int nx, int ny, int nz) {
    const int64_t N = (int64_t)nx * ny * nz;
    const int64_t nseg = (int64_t)((nx + TX - 1) / TX) * ny * nz;
    return N <= SMALL_MAX_SITES && nseg <= SMALL_MAX_SEG;
}

// log2 of the cluster size this device runs the cluster kernel with (4 or 3), or 0 if
// it cannot run it, and how many such clusters it holds at once; checked once per device
static int cluster_bits(int *slots_out = nullptr) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        return 0;
    }
    static int state[MAX_DEVICES];   // -1 unknown, else the cluster bits (0: none)
    static int slots[MAX_DEVICES];   // clusters resident at once
    static bool init = false;
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (!init) {
        for (int &v : state) v = -1;
        init = true;
    }
    if (state[dev] < 0) {
        // the kernels take the attributes, and a cluster fits the device
        auto fits = [](auto k1, auto kn, int cs, int &nclusters) {
            if (cs > 8 && (cudaFuncSetAttribute(k1, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess ||
                           cudaFuncSetAttribute(kn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess))
                return false;
            if (cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ClusterSmem)) !=
                    cudaSuccess ||
                cudaFuncSetAttribute(kn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ClusterSmem)) !=
                    cudaSuccess)
                return false;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(cs, 1, 1);
            cfg.blockDim = dim3(CNT, 1, 1);
            cfg.dynamicSmemBytes = sizeof(ClusterSmem);
            cudaLaunchAttribute attr;
            attr.id = cudaLaunchAttributeClusterDimension;
            attr.val.clusterDim.x = cs;
            attr.val.clusterDim.y = 1;
            attr.val.clusterDim.z = 1;
            cfg.attrs = &attr;
            cfg.numAttrs = 1;
            nclusters = 0;
            return cudaOccupancyMaxActiveClusters(&nclusters, k1, &cfg) == cudaSuccess && nclusters > 0;
        };
        int bits = 0, n = 0;
        if (fits(k_small_cluster<4, 1>, k_small_cluster<4, MAX_LAT_PER_LAUNCH>, 16, n)) bits = 4;
        else if (fits(k_small_cluster<3, 1>, k_small_cluster<3, MAX_LAT_PER_LAUNCH>, 8, n)) bits = 3;
        cudaGetLastError();
        state[dev] = bits;
        slots[dev] = bits ? n : 0;
    }
    if (slots_out) *slots_out = slots[dev];
    return state[dev];
}

int cluster_slots() {
    int n = 0;
    cluster_bits(&n);
    return n;
}

bool cluster_ok() { return cluster_bits() > 0; }

bool cluster_fits(int nx, int ny, int nz) {
    const int cs = 1 << cluster_bits();
    const int64_t nbx = (nx + TX - 1) / TX, rows = (int64_t)ny * nz;
    return cluster_bits() > 0 && nx >= 1 && ny >= 1 && nz >= 1 && ((rows + cs - 1) / cs) * nbx <= CSEG;
}

template <int CSB>
static void launch_cluster(const LatDev *lats, int n, int32_t *status, int32_t local_cap, cudaStream_t st) {
    constexpr int CS = 1 << CSB;
    if (n == 1) {
        LatBatch<1> B;
        std::memset(&B, 0, sizeof(B));
        B.n = 1;
        B.lat[0] = lats[0];
        k_small_cluster<CSB, 1><<<CS, CNT, sizeof(ClusterSmem), st>>>(B, status, local_cap);
    } else {
        LatBatch<MAX_LAT_PER_LAUNCH> B;
        std::memset(&B, 0, sizeof(B));
        B.n = n;
        for (int i = 0; i < n; ++i) B.lat[i] = lats[i];
        k_small_cluster<CSB, MAX_LAT_PER_LAUNCH><<<(unsigned)(CS * n), CNT, sizeof(ClusterSmem), st>>>(B, status,
                                                                                                    local_cap);
    }
}

cudaError_t launch_small(const LatDev *lats, int n, int32_t *status, int32_t local_cap, cudaStream_t st,
                         bool cluster) {
    if (n <= 0) return cudaSuccess;
    if (n > MAX_LAT_PER_LAUNCH) return cudaErrorInvalidValue;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    if (cluster) {   // cluster_bits() has set the kernels' attributes
        const int bits = cluster_bits();
        if (bits == 4) launch_cluster<4>(lats, n, status, local_cap, st);
        else if (bits == 3) launch_cluster<3>(lats, n, status, local_cap, st);
        else return cudaErrorNotSupported;
        return cudaGetLastError();
    }
    static bool attr_set[MAX_DEVICES][2];
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (n == 1) {
        if (!attr_set[dev][0]) {
            e = cudaFuncSetAttribute(k_small_label<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sizeof(SmallSmem));
            if (e != cudaSuccess) return e;
            attr_set[dev][0] = true;
        }
        LatBatch<1> B;
        std::memset(&B, 0, sizeof(B));
        B.n = 1;
        B.lat[0] = lats[0];
        k_small_label<1><<<1, SNT, sizeof(SmallSmem), st>>>(B, status, local_cap);
    } else {
        if (!attr_set[dev][1]) {
            e = cudaFuncSetAttribute(k_small_label<MAX_LAT_PER_LAUNCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)sizeof(SmallSmem));
            if (e != cudaSuccess) return e;
            attr_set[dev][1] = true;
        }
        LatBatch<MAX_LAT_PER_LAUNCH> B;
        std::memset(&B, 0, sizeof(B));
        B.n = n;
        for (int i = 0; i < n; ++i) B.lat[i] = lats[i];
        k_small_label<MAX_LAT_PER_LAUNCH><<<(unsigned)n, SNT, sizeof(SmallSmem), st>>>(B, status, local_cap);
    }
    return cudaGetLastError();
}

}  // namespace hk
