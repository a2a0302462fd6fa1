// hk_slab.cu -- the domain-decomposed scheme of Sec. 3 across ranks: a lattice split
// into slabs along z, one slab per rank (one GPU each), labelled locally and merged
// across the slab faces.
//
// The paper labels each process's domain with the serial algorithm, makes labels
// unique with an offset per process (Eq. 1), records the equivalences across each
// domain face from a halo plane, gathers them at a root process that resolves them,
// and scatters the result.  Here:
//   - each rank labels its slab with the tiled passes, every label being a site index of
//     the whole lattice (its offset is the slab's first site, so no Eq. 1 offset is
//     needed), and lists each local cluster's label in rank order (hk_label_slab);
//   - the clusters touching the slab's two z faces (the face clusters) are numbered
//     densely, each with its label and local size, and every face site gets its face
//     cluster's number (k_face_rank, k_face_number, k_face_ids);
//   - the ranks exchange these face data (the halo of Sec. 3, both faces at once), and
//     every rank resolves the equivalences across all slab interfaces -- the facing
//     sites of consecutive slabs, and of the last and first slab when z is periodic --
//     with a union-find over the face clusters of all ranks, linked by smallest label,
//     so each class's root is its cluster's smallest site (k_merge_*); there is no root
//     process, every rank computes the same classes;
//   - each rank rewrites its merged clusters: the first site of each merged-away face
//     cluster takes its class's label, then every site follows its label to that site
//     once (k_relabel); and it lists the sizes of the clusters whose smallest site lies
//     in its slab, in label order, a class's size summed over all its face clusters
//     (k_own_*).  A last exchange of these counts gives each rank its offset in the
//     global numbering.
#include <cstdint>
#include <cstring>

#include "hk_device.cuh"
#include "hk_launch.h"

namespace hk {

namespace {

constexpr int NTB = 256;

unsigned grid_for(int64_t n, int per_thread = 1) {
    int64_t g = (n + (int64_t)NTB * per_thread - 1) / ((int64_t)NTB * per_thread);
    if (g < 1) g = 1;
    if (g > (1 << 20)) g = 1 << 20;
    return (unsigned)g;
}

// Face site p of side s (0: the slab's first plane, 1: its last): its label, and the
// rank of its cluster (the position of the label in the ascending label list).
__global__ void k_face_rank(const int32_t *labels, int64_t P, int nzr, const int32_t *roots, const int64_t *ncl,
                            int32_t *face_k) {
    const int64_t n = *ncl;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 2 * P; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t site = i < P ? i : (int64_t)(nzr - 1) * P + (i - P);
        const int32_t l = labels[site];
        int32_t k = -1;
        if (l >= 0) {
            int64_t lo = 0, hi = n - 1;   // roots[0..n) ascending, l is one of them
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (roots[mid] < l) lo = mid + 1; else hi = mid;
            }
            k = (int32_t)lo;
        }
        face_k[i] = k;
    }
}

// Number each distinct face cluster once: the first face site of cluster k to claim it
// takes a number f, and records the cluster's label and local size under f.
__global__ void k_face_number(const int32_t *face_k, int64_t P, int32_t *fmap, const int32_t *roots,
                              const int64_t *sizes, int64_t *nf, int32_t *list_lab, int64_t *list_size) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 2 * P; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = face_k[i];
        if (k < 0) continue;
        if (atomicCAS(fmap + k, -1, -2) == -1) {
            const int32_t f = (int32_t)atomicAdd(reinterpret_cast<unsigned long long *>(nf), 1ull);
            list_lab[f] = roots[k];
            list_size[f] = sizes[k];
            fmap[k] = f;
        }
    }
}

__global__ void k_face_ids(int32_t *face, int64_t P, const int32_t *fmap) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 2 * P; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = face[i];
        face[i] = k < 0 ? -1 : fmap[k];
    }
}

// ---- the merge over the face clusters of all ranks ----------------------------------
// Node g = off[r] + f is face cluster f of rank r; lab[g] its label, distinct per node.

__global__ void k_merge_init(int32_t *parent, int32_t *lab, int64_t *size, int64_t *csize, const int32_t *list_lab,
                             const int64_t *list_size, const int64_t *off, const int64_t *cnt, int R, int64_t maxF) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)R * maxF;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / maxF);
        const int64_t f = i - (int64_t)r * maxF;
        if (f >= cnt[r]) continue;
        const int64_t g = off[r] + f;
        parent[g] = (int32_t)g;
        lab[g] = list_lab[i];
        size[g] = list_size[i];
        csize[g] = 0;
    }
}

__device__ __forceinline__ int32_t m_find(int32_t *parent, int32_t x, int64_t cap, int32_t *status) {
    int32_t p = __ldcg(parent + x);
    for (int64_t it = 0; p != x; ++it) {
        if (it > cap) { atomicOr(status, STATUS_GLOBAL_LOOP); return x; }
        const int32_t gp = __ldcg(parent + p);
        if (gp == p) return p;
        __stcg(parent + x, gp);   // path halving
        x = gp;
        p = __ldcg(parent + x);
    }
    return x;
}

// Interface i joins the last plane of slab i with the first plane of slab i + 1 (mod R
// for the periodic interface): facing sites of two face clusters join their classes.
// Links go from the root with the larger label to the one with the smaller, so labels
// decrease along every path and a class's root holds its smallest label.
__global__ void k_merge_union(int32_t *parent, const int32_t *lab, const int32_t *face_all, const int64_t *off,
                              int64_t P, int R, int ninterfaces, int64_t cap, int32_t *status) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < (int64_t)ninterfaces * P;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(i / P);
        const int64_t p = i - (int64_t)q * P;
        const int ra = q, rb = (q + 1) % R;
        const int32_t fa = face_all[(int64_t)ra * 2 * P + P + p];   // last plane of slab ra
        const int32_t fb = face_all[(int64_t)rb * 2 * P + p];       // first plane of slab rb
        if (fa < 0 || fb < 0) continue;
        int32_t a = (int32_t)(off[ra] + fa), b = (int32_t)(off[rb] + fb);
        for (int64_t it = 0;; ++it) {
            if (it > cap) { atomicOr(status, STATUS_GLOBAL_LOOP); break; }
            a = m_find(parent, a, cap, status);
            b = m_find(parent, b, cap, status);
            if (a == b) break;
            if (lab[b] < lab[a]) { const int32_t t = a; a = b; b = t; }
            if (atomicCAS(parent + b, b, a) == b) break;   // b was still a root: linked under a
        }
    }
}

// final roots (read-only finds, then one store each) and class sizes at the roots
__global__ void k_merge_compress(int32_t *parent, const int64_t *size, int64_t *csize, int64_t G, int64_t cap,
                                 int32_t *status) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < G; g += (int64_t)gridDim.x * blockDim.x) {
        int32_t x = (int32_t)g, p = __ldcg(parent + x);
        for (int64_t it = 0; p != x; ++it) {
            if (it > cap) { atomicOr(status, STATUS_GLOBAL_LOOP); break; }
            x = p;
            p = __ldcg(parent + x);
        }
        __stcg(parent + g, x);
        atomicAdd(reinterpret_cast<unsigned long long *>(csize + x), (unsigned long long)size[g]);
    }
}

// The first site of each of this rank's merged-away face clusters takes its class's label.
__global__ void k_merge_firstsites(const int32_t *parent, const int32_t *lab, int64_t g0, int64_t nf, int32_t *labels,
                                   int64_t site_off) {
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = g0 + f;
        const int32_t root = parent[g];
        if (root != (int32_t)g) labels[(int64_t)lab[g] - site_off] = lab[root];
    }
}

// Every site follows its label once: the label's site holds the class label (itself
// for a cluster that was not merged away).  Labels outside this slab are final already.
__global__ void k_relabel(int32_t *labels, int64_t n, int64_t site_off) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const int32_t l = labels[s];
        if (l < 0) continue;
        const int64_t j = (int64_t)l - site_off;
        if (j < 0 || j >= n) continue;
        const int32_t v = labels[j];
        if (v != l) labels[s] = v;
    }
}

// ---- this rank's own clusters: those whose smallest site lies in its slab ----------
// Cluster k of the slab is kept unless it is a face cluster merged into a class with a
// smaller label; a kept face cluster carries its class's size.  Kept clusters are
// compacted in rank order (label order) by a scan over blocks of OWN_CH clusters.
constexpr int OWN_PER = 16;
constexpr int OWN_CH = NTB * OWN_PER;

__device__ __forceinline__ bool own_keep(int64_t k, const int32_t *fmap, const int32_t *parent, int64_t g0,
                                         const int64_t *sizes, const int64_t *csize, int64_t &size) {
    const int32_t f = fmap[k];
    if (f < 0) {
        size = sizes[k];
        return true;
    }
    const int64_t g = g0 + f;
    if (parent[g] != (int32_t)g) return false;
    size = csize[g];
    return true;
}

__global__ void __launch_bounds__(NTB) k_own_count(const int64_t *ncl, const int32_t *fmap, const int32_t *parent,
                                                   int64_t g0, const int64_t *sizes, const int64_t *csize,
                                                   uint32_t *bsum) {
    __shared__ uint32_t red[NTB / 32];
    const int64_t n = *ncl;
    const int64_t k0 = (int64_t)blockIdx.x * OWN_CH + (int64_t)threadIdx.x * OWN_PER;
    uint32_t c = 0;
    for (int j = 0; j < OWN_PER; ++j) {
        int64_t size;
        if (k0 + j < n && own_keep(k0 + j, fmap, parent, g0, sizes, csize, size)) ++c;
    }
    for (int d = 16; d; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < NTB / 32; ++w) t += red[w];
        bsum[blockIdx.x] = t;
    }
}

// single block: exclusive scan of the block counts in place; the total goes to *total
__global__ void __launch_bounds__(1024) k_own_scan(uint32_t *bsum, int64_t nb, int64_t *total) {
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
            const uint32_t w = wsum[lane];
            uint32_t wi = w;
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
    if (threadIdx.x == 0) *total = (int64_t)carry;
}

__global__ void __launch_bounds__(NTB) k_own_write(const int64_t *ncl, const int32_t *fmap, const int32_t *parent,
                                                   int64_t g0, const int64_t *sizes, const int64_t *csize,
                                                   const uint32_t *bsum, int64_t *own_sizes, int64_t own_cap,
                                                   int64_t *hist) {
    __shared__ uint32_t wsum[NTB / 32];
    __shared__ int shist[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x < 32) shist[threadIdx.x] = 0;
    const int64_t n = *ncl;
    const int64_t k0 = (int64_t)blockIdx.x * OWN_CH + (int64_t)threadIdx.x * OWN_PER;
    uint32_t c = 0;
    for (int j = 0; j < OWN_PER; ++j) {
        int64_t size;
        if (k0 + j < n && own_keep(k0 + j, fmap, parent, g0, sizes, csize, size)) ++c;
    }
    uint32_t inc = c;
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc += u;
    }
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        const uint32_t w = lane < NTB / 32 ? wsum[lane] : 0u;
        uint32_t wi = w;
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += u;
        }
        if (lane < NTB / 32) wsum[lane] = wi - w;
    }
    __syncthreads();
    int64_t pos = (int64_t)bsum[blockIdx.x] + wsum[wid] + inc - c;
    for (int j = 0; j < OWN_PER; ++j) {
        int64_t size;
        if (k0 + j < n && own_keep(k0 + j, fmap, parent, g0, sizes, csize, size)) {
            if (pos < own_cap) own_sizes[pos] = size;
            ++pos;
            atomicAdd(&shist[63 - __clzll(size)], 1);
        }
    }
    __syncthreads();
    if (threadIdx.x < 32 && shist[threadIdx.x])
        atomicAdd(reinterpret_cast<unsigned long long *>(hist) + threadIdx.x, (unsigned long long)shist[threadIdx.x]);
}

}  // namespace

cudaError_t launch_slab_faces(const int32_t *labels, int nx, int ny, int nzr, const int32_t *roots, const int64_t *ncl,
                              const int64_t *sizes, int64_t ncl_cap, int32_t *fmap, int32_t *face_out,
                              int32_t *list_lab, int64_t *list_size, int64_t *nf, cudaStream_t st) {
    const int64_t P = (int64_t)nx * ny;
    cudaError_t e = cudaMemsetAsync(fmap, 0xff, (size_t)ncl_cap * sizeof(int32_t), st);   // -1
    if (e == cudaSuccess) e = cudaMemsetAsync(nf, 0, sizeof(int64_t), st);
    if (e != cudaSuccess) return e;
    k_face_rank<<<grid_for(2 * P), NTB, 0, st>>>(labels, P, nzr, roots, ncl, face_out);
    k_face_number<<<grid_for(2 * P), NTB, 0, st>>>(face_out, P, fmap, roots, sizes, nf, list_lab, list_size);
    k_face_ids<<<grid_for(2 * P), NTB, 0, st>>>(face_out, P, fmap);
    return cudaGetLastError();
}

cudaError_t launch_slab_merge(const SlabMerge &M, cudaStream_t st) {
    const int64_t G = M.G;
    k_merge_init<<<grid_for((int64_t)M.R * M.maxF), NTB, 0, st>>>(M.parent, M.lab, M.size, M.csize, M.list_lab_all,
                                                                   M.list_size_all, M.off, M.cnt, M.R, M.maxF);
    if (M.ninterfaces > 0)
        k_merge_union<<<grid_for((int64_t)M.ninterfaces * M.P), NTB, 0, st>>>(M.parent, M.lab, M.face_all, M.off, M.P,
                                                                              M.R, M.ninterfaces, G, M.status);
    k_merge_compress<<<grid_for(G), NTB, 0, st>>>(M.parent, M.size, M.csize, G, G, M.status);
    k_merge_firstsites<<<grid_for(M.nf_own), NTB, 0, st>>>(M.parent, M.lab, M.g0, M.nf_own, M.labels, M.site_off);
    k_relabel<<<grid_for(M.nsites, 4), NTB, 0, st>>>(M.labels, M.nsites, M.site_off);
    const int64_t nb = M.ncl_cap / OWN_CH + 1;
    cudaError_t e = cudaMemsetAsync(M.hist, 0, 32 * sizeof(int64_t), st);
    if (e != cudaSuccess) return e;
    k_own_count<<<(unsigned)nb, NTB, 0, st>>>(M.ncl, M.fmap, M.parent, M.g0, M.sizes, M.csize, M.bsum);
    k_own_scan<<<1, 1024, 0, st>>>(M.bsum, nb, M.own_ncl);
    k_own_write<<<(unsigned)nb, NTB, 0, st>>>(M.ncl, M.fmap, M.parent, M.g0, M.sizes, M.csize, M.bsum, M.own_sizes,
                                              M.own_cap, M.hist);
    return cudaGetLastError();
}

}  // namespace hk
