// hk_api.cu -- the C ABI declared in include/hk.h: contexts, workspace,
// argument checks and the pass sequence of hk_kernels.cu.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "../../include/hk.h"
#include "hk_device.cuh"
#include "hk_launch.h"

using hk::LatDev;
using hk::Plan;
using hk::TileInfo;
using hk::Work;

namespace hk {

Work bind_work(char *base, const Layout &Ly, int32_t *status, int64_t piece_cap, int64_t loop_cap) {
    Work W;
    W.mask = reinterpret_cast<uint32_t *>(base + Ly.mask);
    W.codes = reinterpret_cast<uint16_t *>(base + Ly.codes);
    W.cnt = reinterpret_cast<uint8_t *>(base + Ly.cnt);
    W.pre = reinterpret_cast<uint32_t *>(base + Ly.pre);
    W.bsum = reinterpret_cast<uint32_t *>(base + Ly.bsum);
    W.face = reinterpret_cast<uint16_t *>(base + Ly.face);
    W.tinfo = reinterpret_cast<int4 *>(base + Ly.tinfo);
    W.parent = reinterpret_cast<int32_t *>(base + Ly.parent);
    W.key = reinterpret_cast<int32_t *>(base + Ly.key);
    W.psize = reinterpret_cast<int32_t *>(base + Ly.psize);
    W.xcol = reinterpret_cast<uint32_t *>(base + Ly.xcol);
    W.status = status;
    W.ovf = reinterpret_cast<int32_t *>(base + Ly.ovf);
    W.rootbits = reinterpret_cast<uint32_t *>(base + Ly.rootbits);
    W.segpre = reinterpret_cast<uint32_t *>(base + Ly.segpre);
    W.votes = reinterpret_cast<int32_t *>(base + Ly.votes);
    W.novf = status + 1;
    W.piece_cap = (loop_cap > 0 && loop_cap < piece_cap) ? loop_cap : piece_cap;
    W.local_cap = (loop_cap > 0 && loop_cap < INT32_MAX) ? (int32_t)loop_cap : 0;
    W.site_off = 0;
    W.roots = nullptr;
    return W;
}

}  // namespace hk

struct hk_ctx {
    int device = 0;
    int ty = 16, tz = 16;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    void *io = nullptr;       // device buffers of hk_label_host
    size_t io_bytes = 0;
    void *sbuf = nullptr;     // device buffers of hk_interior_state
    size_t sbuf_bytes = 0;
    int last_cuda = 0;
    int32_t *dstatus = nullptr;   // device status word (STATUS_* flags), survives workspace growth
    int64_t loop_cap = 0;         // test bound of the capped union-find loops (0: natural bounds)
    int64_t *dcounts = nullptr;   // device cluster counts of the one-CTA path when the caller gives none
    int small_path = 1;           // one-launch kernels: 0 off, 1 the library picks, 2 one CTA only, 3 cluster only
    hk::MergeSchedule merge;      // unions per lane of the face merge, hot-root combining
    void *slab_fmap = nullptr;    // face-cluster number of each local cluster (hk_slab_faces -> hk_slab_merge)
    size_t slab_fmap_bytes = 0;
    void *slab_merge = nullptr;   // scratch of hk_slab_merge
    size_t slab_merge_bytes = 0;
    // per-pass timing: a ring of event sets, one per timed call
    static constexpr int RING = 64;
    bool timing = false;
    int64_t ncalls = 0;        // timed calls since timing was enabled
    int64_t nacc = 0;          // calls already folded into acc
    double acc[hk::NUM_PASSES] = {};
    cudaEvent_t ev[RING][hk::NUM_PASSES + 1] = {};
    // CUDA graphs of batched calls, keyed by the exact descriptors and tile shape
    struct GraphEntry {
        std::vector<hk_lattice> key;
        int ty, tz;
        cudaGraphExec_t exec;
    };   // graphs are dropped whenever the schedule changes
    static constexpr int MAX_GRAPHS = 8;
    bool graphs = false;
    std::vector<GraphEntry> gcache;
};

namespace {

constexpr int DEFAULT_TY = 16, DEFAULT_TZ = 16;
constexpr int64_t MAX_SITES = (int64_t)1 << 31;

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

void add_lattice(const TileInfo &ti, int nx, int ny, int nz, Plan &P) {
    const int64_t nbx = ceil_div(nx, hk::TX), nby = ceil_div(ny, ti.ty), nbz = ceil_div(nz, ti.tz);
    P.ntiles += nbx * nby * nbz;
    P.nseg += nbx * (int64_t)ny * nz;
    P.nrows += (int64_t)ny * nz;
}

int fail_cuda(hk_ctx *ctx, cudaError_t e) {
    ctx->last_cuda = (int)e;
    return HK_ERR_CUDA;
}

void drop_graphs(hk_ctx *ctx) {
    for (auto &g : ctx->gcache) cudaGraphExecDestroy(g.exec);
    ctx->gcache.clear();
}

int ensure_ws(hk_ctx *ctx, size_t bytes) {
    if (bytes <= ctx->ws_bytes) return HK_OK;
    drop_graphs(ctx);   // captured graphs point into the old workspace
    if (ctx->ws) {
        cudaDeviceSynchronize();
        cudaFree(ctx->ws);
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    }
    const size_t want = bytes + bytes / 8;   // headroom against frequent regrowth
    cudaError_t e = cudaMalloc(&ctx->ws, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        e = cudaMalloc(&ctx->ws, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            ctx->ws = nullptr;
            return HK_ERR_NOMEM;
        }
        ctx->ws_bytes = bytes;
        return HK_OK;
    }
    ctx->ws_bytes = want;
    return HK_OK;
}

int check_lattice(const hk_lattice &l) {
    if (!l.phi || !l.labels) return HK_ERR_ARG;
    if (l.nx < 1 || l.ny < 1 || l.nz < 1) return HK_ERR_ARG;
    if (l.sizes_cap < 0 || (l.sizes_cap > 0 && !l.sizes)) return HK_ERR_ARG;
    if ((int64_t)l.nx * l.ny * l.nz >= MAX_SITES) return HK_ERR_TOO_LARGE;
    return HK_OK;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link).
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// Tensor maps for TMA tile loads of phi and tile stores of labels: box (32, ty, tz),
// zero fill outside the lattice.  TMA needs 16-byte aligned base addresses and row
// pitches, so nx must be a multiple of 4; otherwise tm.valid stays 0 and the
// kernels use cp.async loads and plain stores.
void make_tmaps(const hk_lattice &l, int ty, int tz, hk::TmapPair &tm) {
    std::memset(&tm, 0, sizeof(tm));
    auto fn = encode_fn();
    if (!fn || (l.nx % 4) != 0 || (reinterpret_cast<uintptr_t>(l.phi) & 15) ||
        (reinterpret_cast<uintptr_t>(l.labels) & 15))
        return;
    const cuuint64_t dims[3] = {(cuuint64_t)l.nx, (cuuint64_t)l.ny, (cuuint64_t)l.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)l.nx * 4, (cuuint64_t)l.nx * l.ny * 4};
    const cuuint32_t box[3] = {(cuuint32_t)hk::TX, (cuuint32_t)ty, (cuuint32_t)tz};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (fn(&tm.phi, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(l.phi), dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return;
    // labels leave a staged tile laid out with the 128-byte swizzle (box rows are 128 bytes)
    if (fn(&tm.labels, CU_TENSOR_MAP_DATA_TYPE_INT32, 3, l.labels, dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return;
    tm.valid = 1;
}

// Add the pass durations of ring slot `slot` (a completed call) to the totals.
cudaError_t fold_slot(hk_ctx *ctx, int slot) {
    cudaError_t e = cudaEventSynchronize(ctx->ev[slot][hk::NUM_PASSES]);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < hk::NUM_PASSES; ++i) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, ctx->ev[slot][i], ctx->ev[slot][i + 1]);
        if (e != cudaSuccess) return e;
        ctx->acc[i] += ms;
    }
    ctx->nacc += 1;
    return cudaSuccess;
}

// Fold the oldest unfolded call, which occupies `slot`, before the slot is reused.
void fold_timing(hk_ctx *ctx, int slot) {
    if (fold_slot(ctx, slot) != cudaSuccess) ctx->timing = false;
}

int grow(void *&buf, size_t &have, size_t need) {
    if (need <= have) return HK_OK;
    if (buf) {
        cudaDeviceSynchronize();
        cudaFree(buf);
        buf = nullptr;
        have = 0;
    }
    if (cudaMalloc(&buf, need) != cudaSuccess) {
        cudaGetLastError();
        buf = nullptr;
        return HK_ERR_NOMEM;
    }
    have = need;
    return HK_OK;
}

int ensure_status(hk_ctx *ctx) {
    if (ctx->dstatus) return HK_OK;
    cudaError_t e = cudaMalloc(&ctx->dstatus, 256);
    if (e != cudaSuccess) { cudaGetLastError(); ctx->dstatus = nullptr; return HK_ERR_NOMEM; }
    e = cudaMemset(ctx->dstatus, 0, 256);
    return e == cudaSuccess ? HK_OK : fail_cuda(ctx, e);
}

// Lattices that all fit the one-CTA path (hk::small_fits), n <= MAX_LAT_PER_LAUNCH: one
// launch, no workspace.  Same capacity rule and outputs as the tiled path; with timing on,
// the whole launch counts as the first pass.
int run_small(hk_ctx *ctx, const hk_lattice *lats, int n, cudaStream_t st, bool check_capacity, bool cluster) {
    int rc = ensure_status(ctx);
    if (rc != HK_OK) return rc;
    if (!ctx->dcounts) {
        cudaError_t e = cudaMalloc(&ctx->dcounts, hk::MAX_LAT_PER_LAUNCH * sizeof(int64_t));
        if (e != cudaSuccess) { cudaGetLastError(); ctx->dcounts = nullptr; return HK_ERR_NOMEM; }
    }
    std::vector<LatDev> dev(n);
    bool check = false;
    for (int i = 0; i < n; ++i) {
        const hk_lattice &l = lats[i];
        LatDev &d = dev[i];
        std::memset(&d, 0, sizeof(d));
        d.phi = l.phi;
        d.labels = l.labels;
        d.sizes = l.sizes;
        d.sizes_cap = l.sizes ? l.sizes_cap : 0;
        d.hist = l.hist;
        d.ncl = l.n_clusters ? l.n_clusters : ctx->dcounts + i;
        d.nx = l.nx; d.ny = l.ny; d.nz = l.nz;
        for (int a = 0; a < 3; ++a) d.per[a] = l.periodic[a] ? 1 : 0;
        d.nbx = (int)ceil_div(l.nx, hk::TX);
        const int64_t N = (int64_t)l.nx * l.ny * l.nz;
        if (check_capacity && d.sizes_cap < (N + 1) / 2) check = true;
    }
    cudaEvent_t *ev = nullptr;
    if (ctx->timing) {
        const int slot = (int)(ctx->ncalls % hk_ctx::RING);
        if (ctx->ncalls - ctx->nacc >= hk_ctx::RING) fold_timing(ctx, slot);
        ev = ctx->ev[slot];
        ctx->ncalls += 1;
        cudaEventRecord(ev[0], st);
    }
    const int32_t lcap = (ctx->loop_cap > 0 && ctx->loop_cap < INT32_MAX) ? (int32_t)ctx->loop_cap : 0;
    cudaError_t e = hk::launch_small(dev.data(), n, ctx->dstatus, lcap, st, cluster);
    if (e != cudaSuccess) return fail_cuda(ctx, e);
    if (ev)
        for (int i = 1; i <= hk::NUM_PASSES; ++i) cudaEventRecord(ev[i], st);
    if (check) {
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail_cuda(ctx, e);
        for (int i = 0; i < n; ++i) {
            int64_t c = 0;
            e = cudaMemcpy(&c, dev[i].ncl, sizeof(c), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return fail_cuda(ctx, e);
            if (c > lats[i].sizes_cap) return HK_ERR_CAPACITY;
        }
    }
    return HK_OK;
}

// Label lats[0..n) with at most MAX_LAT_PER_LAUNCH lattices per pass sequence.
// index_field (one lattice only): the lattice is an index field; label its far sites
// (I < -0.5) and, when inside != nullptr, write the interior/exterior tags of its
// clusters to inside.
// check_capacity == false: never wait for the counts (the caller compares them).
// state != nullptr (index fields with inside): also the interior state of every site.
int run_lattices(hk_ctx *ctx, const hk_lattice *lats, int n, cudaStream_t st, bool index_field = false,
                 int8_t *inside = nullptr, bool check_capacity = true, int8_t *state = nullptr,
                 int64_t site_off = 0, int32_t *roots = nullptr) {
    TileInfo ti;
    if (!hk::tile_info(ctx->ty, ctx->tz, ti)) return HK_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        int rc = check_lattice(lats[i]);
        if (rc != HK_OK) return rc;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return fail_cuda(ctx, e);

    // Small lattices take one launch: a thread-block cluster per lattice for calls of a
    // few lattices (latency: the work of a lattice spread over the cluster's SMs), one
    // CTA per lattice for larger batches of lattices that fit it (throughput); up to
    // MAX_LAT_PER_LAUNCH lattices per launch.
    if (!index_field && ctx->small_path && !roots && site_off == 0) {
        bool all_one = ctx->small_path != 3, all_cluster = ctx->small_path != 2 && hk::cluster_ok();
        for (int i = 0; i < n && (all_one || all_cluster); ++i) {
            all_one = all_one && hk::small_fits(lats[i].nx, lats[i].ny, lats[i].nz);
            all_cluster = all_cluster && hk::cluster_fits(lats[i].nx, lats[i].ny, lats[i].nz);
        }
        if (all_one || all_cluster) {
            // clusters win while they fill about half of the device's cluster slots; past
            // that, lattices that fit one CTA each finish sooner that way (measured at 32^3
            // with 7 slots of 16 CTAs: 4 lattices 31 against 38 us, 8 lattices 48 against 39 us)
            const bool cluster = all_cluster && (!all_one || 2 * n <= hk::cluster_slots() + 1);
            int rc_cap = HK_OK;
            for (int c0 = 0; c0 < n; c0 += hk::MAX_LAT_PER_LAUNCH) {
                const int rc = run_small(ctx, lats + c0, std::min(n - c0, hk::MAX_LAT_PER_LAUNCH), st, check_capacity,
                                         cluster);
                if (rc == HK_ERR_CAPACITY) rc_cap = rc;
                else if (rc != HK_OK) return rc;
            }
            return rc_cap;
        }
    }

    // Launch chunks: at most MAX_LAT_PER_LAUNCH lattices, and few enough tiles that
    // every piece id (tile * max_boundary + k) and every root count fits in 31 bits.
    const int64_t max_tiles = ((int64_t)1 << 31) / ti.max_boundary - 1;
    std::vector<int> chunk_start;
    {
        int c0 = 0;
        while (c0 < n) {
            chunk_start.push_back(c0);
            Plan P{0, 0, 0, 0};
            int c1 = c0;
            while (c1 < n && c1 - c0 < hk::MAX_LAT_PER_LAUNCH) {
                Plan Q = P;
                add_lattice(ti, lats[c1].nx, lats[c1].ny, lats[c1].nz, Q);
                if (c1 > c0 && Q.ntiles > max_tiles) break;
                P = Q;
                ++c1;
            }
            c0 = c1;
        }
        chunk_start.push_back(n);
    }
    // size the workspace for the largest chunk
    size_t need = 0;
    for (size_t c = 0; c + 1 < chunk_start.size(); ++c) {
        Plan P{0, 0, 0, 0};
        for (int i = chunk_start[c]; i < chunk_start[c + 1]; ++i) add_lattice(ti, lats[i].nx, lats[i].ny, lats[i].nz, P);
        P.piece_cap = P.ntiles * ti.max_boundary;
        need = std::max(need, hk::make_layout(ti, P, inside ? lats[0].sizes_cap : 0).total);
    }
    int rc = ensure_ws(ctx, need);
    if (rc != HK_OK) return rc;
    rc = ensure_status(ctx);
    if (rc != HK_OK) return rc;

    bool any_check = false;
    std::vector<int64_t> counts(n, 0);
    for (size_t c = 0; c + 1 < chunk_start.size(); ++c) {
        const int c0 = chunk_start[c];
        const int cn = chunk_start[c + 1] - c0;
        Plan P{0, 0, 0, 0};
        std::vector<LatDev> dev(cn);
        for (int i = 0; i < cn; ++i) {
            const hk_lattice &l = lats[c0 + i];
            LatDev &d = dev[i];
            std::memset(&d, 0, sizeof(d));
            d.phi = l.phi;
            d.labels = l.labels;
            d.sizes = l.sizes;
            d.sizes_cap = l.sizes ? l.sizes_cap : 0;
            d.hist = l.hist;
            d.ncl = l.n_clusters;
            d.nx = l.nx; d.ny = l.ny; d.nz = l.nz;
            for (int a = 0; a < 3; ++a) d.per[a] = l.periodic[a] ? 1 : 0;
            d.nbx = (int)ceil_div(l.nx, hk::TX);
            d.nby = (int)ceil_div(l.ny, ti.ty);
            d.nbz = (int)ceil_div(l.nz, ti.tz);
            d.tile0 = P.ntiles;
            d.seg0 = P.nseg;
            d.row0 = P.nrows;
            d.occ_mode = index_field ? 1 : 0;
            d.inside = inside;
            add_lattice(ti, l.nx, l.ny, l.nz, P);
        }
        P.piece_cap = P.ntiles * ti.max_boundary;
        const hk::Layout Ly = hk::make_layout(ti, P, inside ? lats[0].sizes_cap : 0);
        char *base = static_cast<char *>(ctx->ws);
        Work W = hk::bind_work(base, Ly, ctx->dstatus, P.piece_cap, ctx->loop_cap);
        if (!inside) {
            W.rootbits = nullptr;
            W.segpre = nullptr;
            W.votes = nullptr;
        }
        W.site_off = site_off;   // slab calls: one lattice
        W.roots = roots;
        int64_t *slots = reinterpret_cast<int64_t *>(base + Ly.ncl);
        bool chunk_check = false;
        for (int i = 0; i < cn; ++i) {
            const hk_lattice &l = lats[c0 + i];
            const int64_t N = (int64_t)l.nx * l.ny * l.nz;
            if (!dev[i].ncl) dev[i].ncl = slots + i;
            if (check_capacity && dev[i].sizes_cap < (N + 1) / 2) chunk_check = true;
        }
        cudaEvent_t *ev = nullptr;
        if (ctx->timing) {
            const int slot = (int)(ctx->ncalls % hk_ctx::RING);
            if (ctx->ncalls - ctx->nacc >= hk_ctx::RING) fold_timing(ctx, slot);
            ev = ctx->ev[slot];
            ctx->ncalls += 1;
        }
        std::vector<hk::TmapPair> tms(cn);
        for (int i = 0; i < cn; ++i) make_tmaps(lats[c0 + i], ctx->ty, ctx->tz, tms[i]);
        e = hk::launch_label(ctx->ty, ctx->tz, dev.data(), cn, P, W, tms.data(), st, ev, ctx->merge);
        if (e != cudaSuccess) return fail_cuda(ctx, e);
        if (inside && dev[0].sizes_cap > 0) {
            e = hk::launch_interior(dev[0], W, st, state);
            if (e != cudaSuccess) return fail_cuda(ctx, e);
        }
        if (chunk_check) {
            // the capacity rule needs the counts: wait for this chunk
            any_check = true;
            e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) return fail_cuda(ctx, e);
            for (int i = 0; i < cn; ++i) {
                e = cudaMemcpy(&counts[c0 + i], dev[i].ncl, sizeof(int64_t), cudaMemcpyDeviceToHost);
                if (e != cudaSuccess) return fail_cuda(ctx, e);
            }
        }
    }
    if (any_check)
        for (int i = 0; i < n; ++i)
            if (counts[i] > lats[i].sizes_cap) return HK_ERR_CAPACITY;
    return HK_OK;
}

// Device copies of hk_label_host / hk_label_host_async in the context's io buffer
// (grown on demand): phi, labels, histogram, count and sizes.
struct HostIo {
    float *phi;
    int32_t *labels;
    int64_t *hist, *ncl, *sizes;
    hk_lattice lattice(int nx, int ny, int nz, const int periodic[3], int64_t sizes_cap) const {
        hk_lattice l;
        l.phi = phi;
        l.nx = nx; l.ny = ny; l.nz = nz;
        for (int a = 0; a < 3; ++a) l.periodic[a] = periodic[a];
        l.labels = labels;
        l.sizes = sizes;
        l.sizes_cap = sizes_cap;
        l.hist = hist;
        l.n_clusters = ncl;
        return l;
    }
};

int host_io(hk_ctx *ctx, int64_t N, int64_t sizes_cap, HostIo &io) {
    const size_t o_phi = 0, o_lab = align256(4 * N), o_hist = o_lab + align256(4 * N);
    const size_t o_ncl = o_hist + 256, o_sizes = o_ncl + 256;
    const size_t need = o_sizes + align256(8 * (size_t)std::max<int64_t>(sizes_cap, 1));
    if (need > ctx->io_bytes) {
        if (ctx->io) { cudaDeviceSynchronize(); cudaFree(ctx->io); ctx->io = nullptr; ctx->io_bytes = 0; }
        if (cudaMalloc(&ctx->io, need) != cudaSuccess) { cudaGetLastError(); return HK_ERR_NOMEM; }
        ctx->io_bytes = need;
    }
    char *b = static_cast<char *>(ctx->io);
    io.phi = reinterpret_cast<float *>(b + o_phi);
    io.labels = reinterpret_cast<int32_t *>(b + o_lab);
    io.hist = reinterpret_cast<int64_t *>(b + o_hist);
    io.ncl = reinterpret_cast<int64_t *>(b + o_ncl);
    io.sizes = reinterpret_cast<int64_t *>(b + o_sizes);
    return HK_OK;
}

// Label lats[0..n) as one call, replayed from a cached CUDA graph when graphs are on
// (non-default stream, timing off, every sizes_cap >= ceil(N/2), so no call waits on
// the host): the first call with given descriptors runs uncaptured (sizing the
// workspace and setting kernel attributes), then captures the same launches.
int run_graphed(hk_ctx *ctx, const hk_lattice *lats, int n, cudaStream_t st) {
    bool graphable = ctx->graphs && st != nullptr && !ctx->timing;
    for (int i = 0; i < n && graphable; ++i) {
        const int64_t N = (int64_t)lats[i].nx * lats[i].ny * lats[i].nz;
        if (check_lattice(lats[i]) != HK_OK || lats[i].sizes_cap < (N + 1) / 2) graphable = false;
    }
    if (!graphable) return run_lattices(ctx, lats, n, st);

    auto same = [&](const std::vector<hk_lattice> &key) {
        if ((int)key.size() != n) return false;
        for (int i = 0; i < n; ++i) {
            const hk_lattice &a = key[i], &b = lats[i];
            if (a.phi != b.phi || a.nx != b.nx || a.ny != b.ny || a.nz != b.nz || a.labels != b.labels ||
                a.sizes != b.sizes || a.sizes_cap != b.sizes_cap || a.hist != b.hist || a.n_clusters != b.n_clusters ||
                (a.periodic[0] != 0) != (b.periodic[0] != 0) || (a.periodic[1] != 0) != (b.periodic[1] != 0) ||
                (a.periodic[2] != 0) != (b.periodic[2] != 0))
                return false;
        }
        return true;
    };
    for (auto &g : ctx->gcache)
        if (g.ty == ctx->ty && g.tz == ctx->tz && same(g.key))
            return cudaGraphLaunch(g.exec, st) == cudaSuccess ? HK_OK : fail_cuda(ctx, cudaGetLastError());

    int rc = run_lattices(ctx, lats, n, st);
    if (rc != HK_OK) return rc;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return fail_cuda(ctx, e);
    rc = run_lattices(ctx, lats, n, st);
    e = cudaStreamEndCapture(st, &graph);
    if (rc != HK_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return rc != HK_OK ? rc : fail_cuda(ctx, e);
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail_cuda(ctx, e);
    if ((int)ctx->gcache.size() >= hk_ctx::MAX_GRAPHS) {
        cudaGraphExecDestroy(ctx->gcache.front().exec);
        ctx->gcache.erase(ctx->gcache.begin());
    }
    ctx->gcache.push_back({std::vector<hk_lattice>(lats, lats + n), ctx->ty, ctx->tz, exec});
    return HK_OK;   // this call's results came from the uncaptured run
}

}  // namespace

extern "C" {

int hk_create(hk_ctx **out, int device) {
    if (!out) return HK_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return HK_ERR_CUDA;
    }
    hk_ctx *c = new hk_ctx();
    c->device = device;
    c->ty = DEFAULT_TY;
    c->tz = DEFAULT_TZ;
    *out = c;
    return HK_OK;
}

void hk_destroy(hk_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->io) cudaFree(ctx->io);
    if (ctx->sbuf) cudaFree(ctx->sbuf);
    if (ctx->dstatus) cudaFree(ctx->dstatus);
    if (ctx->dcounts) cudaFree(ctx->dcounts);
    if (ctx->slab_fmap) cudaFree(ctx->slab_fmap);
    if (ctx->slab_merge) cudaFree(ctx->slab_merge);
    drop_graphs(ctx);
    for (auto &set : ctx->ev)
        for (auto &e : set)
            if (e) cudaEventDestroy(e);
    delete ctx;
}

size_t hk_workspace_bytes(int nx, int ny, int nz) {
    if (nx < 1 || ny < 1 || nz < 1 || (int64_t)nx * ny * nz >= MAX_SITES) return 0;
    TileInfo ti;
    hk::tile_info(DEFAULT_TY, DEFAULT_TZ, ti);
    Plan P{0, 0, 0, 0};
    add_lattice(ti, nx, ny, nz, P);
    P.piece_cap = P.ntiles * ti.max_boundary;
    return hk::make_layout(ti, P).total;
}

int hk_reserve(hk_ctx *ctx, size_t bytes) {
    if (!ctx) return HK_ERR_ARG;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail_cuda(ctx, cudaGetLastError());
    return ensure_ws(ctx, bytes);
}

int hk_label(hk_ctx *ctx, const float *phi, int nx, int ny, int nz, const int periodic[3],
             int32_t *labels_out, int64_t *sizes_out, int64_t sizes_cap, int64_t *hist_out,
             int64_t *n_clusters_out, void *stream) {
    if (!ctx || !periodic) return HK_ERR_ARG;
    hk_lattice l;
    l.phi = phi;
    l.nx = nx; l.ny = ny; l.nz = nz;
    for (int a = 0; a < 3; ++a) l.periodic[a] = periodic[a];
    l.labels = labels_out;
    l.sizes = sizes_out;
    l.sizes_cap = sizes_cap;
    l.hist = hist_out;
    l.n_clusters = n_clusters_out;
    return run_graphed(ctx, &l, 1, static_cast<cudaStream_t>(stream));
}

int hk_label_interior(hk_ctx *ctx, const float *index, int nx, int ny, int nz, const int periodic[3],
                      int32_t *labels_out, int64_t *sizes_out, int64_t sizes_cap, int64_t *hist_out,
                      int64_t *n_clusters_out, int8_t *inside_out, void *stream) {
    if (!ctx || !periodic) return HK_ERR_ARG;
    if (sizes_cap > 0 && !inside_out) return HK_ERR_ARG;
    hk_lattice l;
    l.phi = index;
    l.nx = nx; l.ny = ny; l.nz = nz;
    for (int a = 0; a < 3; ++a) l.periodic[a] = periodic[a];
    l.labels = labels_out;
    l.sizes = sizes_out;
    l.sizes_cap = sizes_cap;
    l.hist = hist_out;
    l.n_clusters = n_clusters_out;
    return run_lattices(ctx, &l, 1, static_cast<cudaStream_t>(stream), true, sizes_cap > 0 ? inside_out : nullptr);
}

int hk_interior_state(hk_ctx *ctx, const float *index, int nx, int ny, int nz, const int periodic[3],
                      int8_t *state_out, void *stream) {
    if (!ctx || !periodic || !index || !state_out) return HK_ERR_ARG;
    if (nx < 1 || ny < 1 || nz < 1) return HK_ERR_ARG;
    const int64_t N = (int64_t)nx * ny * nz;
    if (N >= MAX_SITES) return HK_ERR_TOO_LARGE;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return fail_cuda(ctx, e);
    // labels, sizes, histogram, count and tags of the far sites' clusters, in the
    // context; ceil(N / 2) clusters always fit
    const int64_t cap = (N + 1) / 2;
    const size_t o_lab = 0, o_sizes = align256(4 * N), o_hist = o_sizes + align256(8 * cap);
    const size_t o_ncl = o_hist + 256, o_inside = o_ncl + 256, need = o_inside + align256(cap);
    if (need > ctx->sbuf_bytes) {
        if (ctx->sbuf) { cudaDeviceSynchronize(); cudaFree(ctx->sbuf); ctx->sbuf = nullptr; ctx->sbuf_bytes = 0; }
        if (cudaMalloc(&ctx->sbuf, need) != cudaSuccess) { cudaGetLastError(); return HK_ERR_NOMEM; }
        ctx->sbuf_bytes = need;
    }
    char *b = static_cast<char *>(ctx->sbuf);
    hk_lattice l;
    l.phi = index;
    l.nx = nx; l.ny = ny; l.nz = nz;
    for (int a = 0; a < 3; ++a) l.periodic[a] = periodic[a];
    l.labels = reinterpret_cast<int32_t *>(b + o_lab);
    l.sizes = reinterpret_cast<int64_t *>(b + o_sizes);
    l.sizes_cap = cap;
    l.hist = reinterpret_cast<int64_t *>(b + o_hist);
    l.n_clusters = reinterpret_cast<int64_t *>(b + o_ncl);
    return run_lattices(ctx, &l, 1, static_cast<cudaStream_t>(stream), true, reinterpret_cast<int8_t *>(b + o_inside),
                        false, state_out);
}

int hk_interior_update(const int8_t *state_prev, const float *index, int64_t n_sites, int8_t *state_out,
                       void *stream) {
    if (n_sites < 0 || (n_sites > 0 && (!state_prev || !index || !state_out))) return HK_ERR_ARG;
    const cudaError_t e = hk::launch_interior_update(state_prev, index, n_sites, state_out,
                                                     static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? HK_OK : HK_ERR_CUDA;
}

int hk_interior_update_sites(int8_t *state, int64_t n_sites, const int32_t *sites, const float *values, int64_t m,
                             void *stream) {
    if (n_sites < 0 || m < 0 || (m > 0 && (!state || !sites || !values))) return HK_ERR_ARG;
    const cudaError_t e = hk::launch_interior_update_sites(state, n_sites, sites, values, m,
                                                           static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? HK_OK : HK_ERR_CUDA;
}

int hk_label_batched(hk_ctx *ctx, const hk_lattice *lats, int n, void *stream) {
    if (!ctx || n < 0 || (n > 0 && !lats)) return HK_ERR_ARG;
    if (n == 0) return HK_OK;
    return run_graphed(ctx, lats, n, static_cast<cudaStream_t>(stream));
}

int hk_label_slab(hk_ctx *ctx, const float *phi, int nx, int ny, int nz, int64_t z0, int periodic_x, int periodic_y,
                  int32_t *labels_out, int64_t *sizes_out, int64_t sizes_cap, int32_t *roots_out,
                  int64_t *n_clusters_out, void *stream) {
    if (!ctx || !phi || !labels_out || !sizes_out || !roots_out || !n_clusters_out) return HK_ERR_ARG;
    if (nx < 1 || ny < 1 || nz < 1 || z0 < 0) return HK_ERR_ARG;
    const int64_t N = (int64_t)nx * ny * nz;
    if ((z0 + nz) * (int64_t)nx * ny >= MAX_SITES) return HK_ERR_TOO_LARGE;
    if (sizes_cap < (N + 1) / 2) return HK_ERR_ARG;
    hk_lattice l;
    l.phi = phi;
    l.nx = nx; l.ny = ny; l.nz = nz;
    l.periodic[0] = periodic_x ? 1 : 0;
    l.periodic[1] = periodic_y ? 1 : 0;
    l.periodic[2] = 0;   // z joins across the slabs (hk_slab_merge)
    l.labels = labels_out;
    l.sizes = sizes_out;
    l.sizes_cap = sizes_cap;
    l.hist = nullptr;
    l.n_clusters = n_clusters_out;
    return run_lattices(ctx, &l, 1, static_cast<cudaStream_t>(stream), false, nullptr, false, nullptr,
                        z0 * (int64_t)nx * ny, roots_out);
}

int hk_slab_faces(hk_ctx *ctx, const int32_t *labels, int nx, int ny, int nz, const int32_t *roots,
                  const int64_t *sizes, const int64_t *n_clusters, int64_t sizes_cap, int32_t *face_out,
                  int32_t *list_lab_out, int64_t *list_size_out, int64_t *n_face_out, void *stream) {
    if (!ctx || !labels || !roots || !sizes || !n_clusters || !face_out || !list_lab_out || !list_size_out ||
        !n_face_out)
        return HK_ERR_ARG;
    if (nx < 1 || ny < 1 || nz < 1 || sizes_cap < 1) return HK_ERR_ARG;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return fail_cuda(ctx, e);
    int rc = grow(ctx->slab_fmap, ctx->slab_fmap_bytes, (size_t)sizes_cap * sizeof(int32_t));
    if (rc != HK_OK) return rc;
    e = hk::launch_slab_faces(labels, nx, ny, nz, roots, n_clusters, sizes, sizes_cap,
                              static_cast<int32_t *>(ctx->slab_fmap), face_out, list_lab_out, list_size_out,
                              n_face_out, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? HK_OK : fail_cuda(ctx, e);
}

int hk_slab_merge(hk_ctx *ctx, int nranks, int rank, int periodic_z, int nx, int ny, const int32_t *face_all,
                  const int64_t *n_face_all, const int32_t *list_lab_all, const int64_t *list_size_all,
                  int64_t max_face, int32_t *labels, int nz, int64_t z0, const int64_t *sizes,
                  const int64_t *n_clusters, int64_t sizes_cap, int64_t *own_sizes_out, int64_t own_cap,
                  int64_t *own_n_out, int64_t *hist_out, void *stream) {
    if (!ctx || nranks < 1 || rank < 0 || rank >= nranks || !face_all || !n_face_all || !labels || !sizes ||
        !n_clusters || !own_n_out || !hist_out || max_face < 0 || own_cap < 0 || (own_cap > 0 && !own_sizes_out))
        return HK_ERR_ARG;
    if (nx < 1 || ny < 1 || nz < 1 || z0 < 0 || sizes_cap < 1) return HK_ERR_ARG;
    if (max_face > 0 && (!list_lab_all || !list_size_all)) return HK_ERR_ARG;
    if (!ctx->slab_fmap || ctx->slab_fmap_bytes < (size_t)sizes_cap * sizeof(int32_t)) return HK_ERR_ARG;
    std::vector<int64_t> off(nranks), cnt(nranks);
    int64_t G = 0;
    for (int r = 0; r < nranks; ++r) {
        if (n_face_all[r] < 0 || n_face_all[r] > max_face) return HK_ERR_ARG;
        off[r] = G;
        cnt[r] = n_face_all[r];
        G += n_face_all[r];
    }
    if (G >= ((int64_t)1 << 31)) return HK_ERR_TOO_LARGE;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return fail_cuda(ctx, e);
    int rc = ensure_status(ctx);
    if (rc != HK_OK) return rc;
    // scratch: off, cnt (R each), parent, lab (G int32), size, csize (G int64), bsum
    const int64_t nb = sizes_cap / 4096 + 1;
    const size_t o_off = 0, o_cnt = align256(8 * (size_t)nranks), o_par = o_cnt + align256(8 * (size_t)nranks);
    const size_t o_lab = o_par + align256(4 * (size_t)G), o_size = o_lab + align256(4 * (size_t)G);
    const size_t o_csize = o_size + align256(8 * (size_t)G), o_bsum = o_csize + align256(8 * (size_t)G);
    const size_t need = o_bsum + align256(4 * (size_t)nb);
    rc = grow(ctx->slab_merge, ctx->slab_merge_bytes, need);
    if (rc != HK_OK) return rc;
    char *b = static_cast<char *>(ctx->slab_merge);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    e = cudaMemcpyAsync(b + o_off, off.data(), 8 * (size_t)nranks, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_cnt, cnt.data(), 8 * (size_t)nranks, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail_cuda(ctx, e);
    hk::SlabMerge M;
    M.R = nranks;
    M.ninterfaces = nranks - 1 + (periodic_z ? 1 : 0);
    M.P = (int64_t)nx * ny;
    M.maxF = max_face;
    M.G = G;
    M.g0 = off[rank];
    M.nf_own = cnt[rank];
    M.face_all = face_all;
    M.list_lab_all = list_lab_all;
    M.list_size_all = list_size_all;
    M.off = reinterpret_cast<int64_t *>(b + o_off);
    M.cnt = reinterpret_cast<int64_t *>(b + o_cnt);
    M.parent = reinterpret_cast<int32_t *>(b + o_par);
    M.lab = reinterpret_cast<int32_t *>(b + o_lab);
    M.size = reinterpret_cast<int64_t *>(b + o_size);
    M.csize = reinterpret_cast<int64_t *>(b + o_csize);
    M.labels = labels;
    M.nsites = (int64_t)nx * ny * nz;
    M.site_off = z0 * (int64_t)nx * ny;
    M.sizes = sizes;
    M.ncl = n_clusters;
    M.ncl_cap = sizes_cap;
    M.fmap = static_cast<const int32_t *>(ctx->slab_fmap);
    M.bsum = reinterpret_cast<uint32_t *>(b + o_bsum);
    M.own_sizes = own_sizes_out;
    M.own_cap = own_cap;
    M.own_ncl = own_n_out;
    M.hist = hist_out;
    M.status = ctx->dstatus;
    e = hk::launch_slab_merge(M, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // off and cnt are host arrays of this call
    return e == cudaSuccess ? HK_OK : fail_cuda(ctx, e);
}

int hk_set_graphs(hk_ctx *ctx, int enable) {
    if (!ctx) return HK_ERR_ARG;
    ctx->graphs = enable != 0;
    if (!ctx->graphs) drop_graphs(ctx);
    return HK_OK;
}

int hk_set_merge(hk_ctx *ctx, int unions_per_lane, int combine_hot) {
    if (!ctx) return HK_ERR_ARG;
    if (unions_per_lane == 0) unions_per_lane = 1;
    if (unions_per_lane != 1 && unions_per_lane != 2 && unions_per_lane != 4) return HK_ERR_ARG;
    if (combine_hot != 0 && combine_hot != 1) return HK_ERR_ARG;
    ctx->merge.unions = unions_per_lane;
    ctx->merge.hot = combine_hot;
    drop_graphs(ctx);
    return HK_OK;
}

int hk_set_small_path(hk_ctx *ctx, int enable) {
    if (!ctx || enable < 0 || enable > 3) return HK_ERR_ARG;
    ctx->small_path = enable;
    drop_graphs(ctx);
    return HK_OK;
}

int hk_set_loop_cap(hk_ctx *ctx, int64_t cap) {
    if (!ctx || cap < 0) return HK_ERR_ARG;
    ctx->loop_cap = cap;
    drop_graphs(ctx);   // captured launches carry the old bound
    return HK_OK;
}

int hk_label_host(hk_ctx *ctx, const float *phi_host, int nx, int ny, int nz, const int periodic[3],
                  int32_t *labels_host, int64_t *sizes_host, int64_t sizes_cap, int64_t *hist_host,
                  int64_t *n_clusters_host, void *stream) {
    if (!ctx || !periodic || !phi_host || !labels_host) return HK_ERR_ARG;
    if (nx < 1 || ny < 1 || nz < 1 || sizes_cap < 0 || (sizes_cap > 0 && !sizes_host)) return HK_ERR_ARG;
    const int64_t N = (int64_t)nx * ny * nz;
    if (N >= MAX_SITES) return HK_ERR_TOO_LARGE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return fail_cuda(ctx, e);
    HostIo io;
    int rc = host_io(ctx, N, sizes_cap, io);
    if (rc != HK_OK) return rc;
    e = cudaMemcpyAsync(io.phi, phi_host, 4 * N, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail_cuda(ctx, e);
    hk_lattice l = io.lattice(nx, ny, nz, periodic, sizes_cap);
    rc = run_lattices(ctx, &l, 1, st);
    if (rc != HK_OK && rc != HK_ERR_CAPACITY) return rc;
    int64_t ncl = 0;
    e = cudaMemcpyAsync(&ncl, io.ncl, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(labels_host, io.labels, 4 * N, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && hist_host) e = cudaMemcpyAsync(hist_host, io.hist, 256, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail_cuda(ctx, e);
    const int64_t ns = std::min(ncl, sizes_cap);
    if (ns > 0) {
        e = cudaMemcpyAsync(sizes_host, io.sizes, 8 * ns, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail_cuda(ctx, e);
    }
    if (n_clusters_host) *n_clusters_host = ncl;
    return ncl > sizes_cap ? HK_ERR_CAPACITY : HK_OK;
}

int hk_label_host_async(hk_ctx *ctx, const float *phi_host, int nx, int ny, int nz, const int periodic[3],
                        int32_t *labels_host, int64_t *sizes_host, int64_t sizes_cap, int64_t *hist_host,
                        int64_t *n_clusters_host, void *stream) {
    if (!ctx || !periodic || !phi_host || !labels_host) return HK_ERR_ARG;
    if (nx < 1 || ny < 1 || nz < 1 || sizes_cap < 0 || (sizes_cap > 0 && !sizes_host)) return HK_ERR_ARG;
    const int64_t N = (int64_t)nx * ny * nz;
    if (N >= MAX_SITES) return HK_ERR_TOO_LARGE;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return fail_cuda(ctx, e);
    // every host buffer page-locked; the sizes are written by a kernel, through the
    // buffer's device address
    int64_t *sizes_dst = nullptr;
    {
        const void *bufs[5] = {phi_host, labels_host, sizes_cap > 0 ? sizes_host : nullptr, hist_host,
                               n_clusters_host};
        for (int i = 0; i < 5; ++i) {
            if (!bufs[i]) continue;
            cudaPointerAttributes a;
            if (cudaPointerGetAttributes(&a, bufs[i]) != cudaSuccess) { cudaGetLastError(); return HK_ERR_ARG; }
            if (a.type != cudaMemoryTypeHost || !a.devicePointer) return HK_ERR_ARG;
            if (i == 2) sizes_dst = static_cast<int64_t *>(a.devicePointer);
        }
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    HostIo io;
    int rc = host_io(ctx, N, sizes_cap, io);
    if (rc != HK_OK) return rc;
    e = cudaMemcpyAsync(io.phi, phi_host, 4 * N, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail_cuda(ctx, e);
    hk_lattice l = io.lattice(nx, ny, nz, periodic, sizes_cap);
    rc = run_lattices(ctx, &l, 1, st, false, nullptr, false);
    if (rc != HK_OK) return rc;
    if (n_clusters_host) e = cudaMemcpyAsync(n_clusters_host, io.ncl, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(labels_host, io.labels, 4 * N, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && hist_host) e = cudaMemcpyAsync(hist_host, io.hist, 256, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && sizes_dst) e = hk::launch_copy_counted(io.sizes, io.ncl, sizes_cap, sizes_dst, st);
    if (e != cudaSuccess) return fail_cuda(ctx, e);
    return HK_OK;
}

int hk_set_tile(hk_ctx *ctx, int ty, int tz) {
    if (!ctx) return HK_ERR_ARG;
    if (ty == 0 && tz == 0) { ctx->ty = DEFAULT_TY; ctx->tz = DEFAULT_TZ; return HK_OK; }
    TileInfo ti;
    if (!hk::tile_info(ty, tz, ti)) return HK_ERR_ARG;
    ctx->ty = ty;
    ctx->tz = tz;
    return HK_OK;
}

int hk_set_timing(hk_ctx *ctx, int enable) {
    if (!ctx) return HK_ERR_ARG;
    if (enable && !ctx->ev[0][0]) {
        if (cudaSetDevice(ctx->device) != cudaSuccess) return fail_cuda(ctx, cudaGetLastError());
        for (auto &set : ctx->ev)
            for (auto &e : set) {
                const cudaError_t ce = cudaEventCreate(&e);
                if (ce != cudaSuccess) return fail_cuda(ctx, ce);
            }
    }
    ctx->timing = enable != 0;
    ctx->ncalls = 0;
    ctx->nacc = 0;
    for (auto &a : ctx->acc) a = 0.0;
    return HK_OK;
}

int hk_get_timing(hk_ctx *ctx, float *ms_out, int max_n, int *n_out) {
    if (!ctx || !ms_out || ctx->ncalls == 0) return HK_ERR_ARG;
    while (ctx->nacc < ctx->ncalls) {
        const cudaError_t e = fold_slot(ctx, (int)(ctx->nacc % hk_ctx::RING));
        if (e != cudaSuccess) return fail_cuda(ctx, e);
    }
    const int n = std::min(max_n, hk::NUM_PASSES);
    for (int i = 0; i < n; ++i) ms_out[i] = (float)(ctx->acc[i] / (double)ctx->nacc);
    if (n_out) *n_out = hk::NUM_PASSES;
    return HK_OK;
}

int hk_sync_status(hk_ctx *ctx, void *stream) {
    if (!ctx) return HK_ERR_ARG;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return fail_cuda(ctx, e);
    if (!ctx->dstatus) return HK_OK;
    int32_t s = 0;
    e = cudaMemcpy(&s, ctx->dstatus, sizeof(s), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && s) {   // cleared on the caller's stream, ahead of its later calls
        e = cudaMemsetAsync(ctx->dstatus, 0, sizeof(s), static_cast<cudaStream_t>(stream));
        if (e == cudaSuccess) e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    }
    if (e != cudaSuccess) return fail_cuda(ctx, e);
    return s ? HK_ERR_TIMEOUT : HK_OK;
}

int hk_last_cuda_error(const hk_ctx *ctx) { return ctx ? ctx->last_cuda : 0; }

const char *hk_strerror(int status) {
    switch (status) {
        case HK_OK: return "ok";
        case HK_ERR_ARG: return "invalid argument";
        case HK_ERR_TOO_LARGE: return "lattice too large (nx*ny*nz >= 2^31, or beyond the allocation-free scratch)";
        case HK_ERR_CAPACITY: return "more clusters than sizes_cap";
        case HK_ERR_CUDA: return "CUDA runtime error";
        case HK_ERR_TIMEOUT: return "device-side wait timed out";
        case HK_ERR_NOMEM: return "workspace allocation failed";
        default: return "unknown status";
    }
}

}  // extern "C"
