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

// Exclusive scan of one int per thread over the CTA's 1024 threads; *total gets the sum.
// Ends with a barrier, after which warp_tmp and scan_total may be reused.
__device__ __forceinline__ int cta_exscan(int v, SmallSmem &S, int &total) {
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
        const int w = S.warp_tmp[lane];
        int wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += u;
        }
        S.warp_tmp[lane] = wi - w;
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
    const int base = cta_exscan(n_a + n_b, S, total);
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
    int rank = cta_exscan(nr, S, nclus);
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

}  // namespace

bool small_fits(int nx, int ny, int nz) {
    const int64_t N = (int64_t)nx * ny * nz;
    const int64_t nseg = (int64_t)((nx + TX - 1) / TX) * ny * nz;
    return N <= SMALL_MAX_SITES && nseg <= SMALL_MAX_SEG;
}

cudaError_t launch_small(const LatDev *lats, int n, int32_t *status, int32_t local_cap, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
    static bool attr_set[MAX_DEVICES][2];
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (n == 1) {
        if (!attr_set[dev][0]) {
            e = cudaFuncSetAttribute(k_small_label<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SmallSmem));
            if (e != cudaSuccess) return e;
            attr_set[dev][0] = true;
        }
        LatBatch<1> B;
        std::memset(&B, 0, sizeof(B));
        B.n = 1;
        B.lat[0] = lats[0];
        k_small_label<1><<<1, SNT, sizeof(SmallSmem), st>>>(B, status, local_cap);
    } else {
        if (n > MAX_LAT_PER_LAUNCH) return cudaErrorInvalidValue;
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
