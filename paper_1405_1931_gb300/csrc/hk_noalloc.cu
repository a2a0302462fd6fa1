// hk_noalloc.cu -- hk_label_noalloc: labelling without any device allocation.
//
// Some callers cannot allocate device memory: a simulation that has already
// handed all free device memory to its own allocator, or a code path where a
// cudaMalloc/cudaFree would synchronise the device and stall the caller's
// other streams.  This entry point runs the same passes as hk_label, but its
// scratch (occupancy mask, run codes, face summaries, piece table, root counts
// and prefix, status word) lives in one file-scope __device__ array of fixed
// size instead of a context workspace.  The caller still passes phi and the
// output buffers.
#include <cstdint>
#include <cstring>

#include <cuda_runtime.h>

#include "../../include/hk.h"
#include "hk_device.cuh"
#include "hk_launch.h"

namespace {

constexpr size_t SCRATCH_BYTES = (size_t)HK_NOALLOC_SCRATCH_BYTES;
constexpr int TY = 16, TZ = 16;
using hk::MAX_DEVICES;

// Every GPU that loads the library holds this array until the process exits.
__device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

// Device address of g_scratch on each device.  In host code the name g_scratch
// is only a host-side stand-in for the symbol, never a device pointer.
void *g_scratch_addr[MAX_DEVICES];

size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }

struct Carve {
    size_t mask, codes, cnt, pre, bsum, face, tinfo, parent, key, psize, xcol, ovf, status, ncl, total;
};

Carve carve(const hk::TileInfo &ti, const hk::Plan &P) {
    Carve c{};
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += a256(bytes); return o; };
    const int64_t nb = (P.nrows + 4096) / 4096;
    c.mask = take((size_t)P.ntiles * ti.rows * 4);
    c.codes = take((size_t)P.ntiles * ti.maxruns * 2);
    c.cnt = take((size_t)P.nseg);
    c.pre = take((size_t)(P.nrows + 1) * 4);
    c.bsum = take((size_t)nb * 4);
    c.face = take((size_t)P.ntiles * ti.face_stride * 2);
    c.tinfo = take((size_t)P.ntiles * 16);
    c.parent = take((size_t)P.piece_cap * 4);
    c.key = take((size_t)P.piece_cap * 4);
    c.psize = take((size_t)P.piece_cap * 4);
    c.xcol = take((size_t)P.ntiles * (ti.rows / 32) * 2 * 4);
    c.ovf = take((size_t)P.ntiles * 4);
    c.status = take(8);   // status word, then the count of ovf
    c.ncl = take(8);
    c.total = off;
    return c;
}

}  // namespace

extern "C" int hk_label_noalloc(const float *phi, int nx, int ny, int nz, const int periodic[3],
                                int32_t *labels_out, int64_t *sizes_out, int64_t sizes_cap,
                                int64_t *hist_out, int64_t *n_clusters_out, void *stream) {
    if (!phi || !periodic || !labels_out || nx < 1 || ny < 1 || nz < 1) return HK_ERR_ARG;
    if (sizes_cap < 0 || (sizes_cap > 0 && !sizes_out)) return HK_ERR_ARG;
    const int64_t N = (int64_t)nx * ny * nz;
    if (N >= ((int64_t)1 << 31)) return HK_ERR_TOO_LARGE;

    hk::TileInfo ti;
    hk::tile_info(TY, TZ, ti);
    hk::Plan P{0, 0, 0, 0};
    const int64_t nbx = (nx + hk::TX - 1) / hk::TX, nby = (ny + TY - 1) / TY, nbz = (nz + TZ - 1) / TZ;
    P.ntiles = nbx * nby * nbz;
    P.nseg = nbx * (int64_t)ny * nz;
    P.nrows = (int64_t)ny * nz;
    P.piece_cap = P.ntiles * ti.max_boundary;
    const Carve c = carve(ti, P);
    if (c.total > SCRATCH_BYTES) return HK_ERR_TOO_LARGE;   // rejected before touching the GPU

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return HK_ERR_CUDA;
    if (!g_scratch_addr[dev]) {
        // one-time set-up on this device (the current one)
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return HK_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    char *base = static_cast<char *>(g_scratch_addr[dev]);
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    hk::Work W;
    W.mask = reinterpret_cast<uint32_t *>(base + c.mask);
    W.codes = reinterpret_cast<uint16_t *>(base + c.codes);
    W.cnt = reinterpret_cast<uint8_t *>(base + c.cnt);
    W.pre = reinterpret_cast<uint32_t *>(base + c.pre);
    W.bsum = reinterpret_cast<uint32_t *>(base + c.bsum);
    W.face = reinterpret_cast<uint16_t *>(base + c.face);
    W.tinfo = reinterpret_cast<int4 *>(base + c.tinfo);
    W.parent = reinterpret_cast<int32_t *>(base + c.parent);
    W.key = reinterpret_cast<int32_t *>(base + c.key);
    W.psize = reinterpret_cast<int32_t *>(base + c.psize);
    W.xcol = reinterpret_cast<uint32_t *>(base + c.xcol);
    W.status = reinterpret_cast<int32_t *>(base + c.status);
    W.ovf = reinterpret_cast<int32_t *>(base + c.ovf);
    W.rootbits = nullptr;   // no interior/exterior identification here
    W.segpre = nullptr;
    W.votes = nullptr;
    W.novf = W.status + 1;
    W.piece_cap = P.piece_cap;

    // The array keeps the previous call's contents.  Everything the passes read is
    // written earlier in the same call, except the status word, which is cleared.
    e = cudaMemsetAsync(W.status, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return HK_ERR_CUDA;

    hk::LatDev d;
    std::memset(&d, 0, sizeof(d));
    d.phi = phi;
    d.labels = labels_out;
    d.sizes = sizes_out;
    d.sizes_cap = sizes_out ? sizes_cap : 0;
    d.hist = hist_out;
    d.ncl = n_clusters_out ? n_clusters_out : reinterpret_cast<int64_t *>(base + c.ncl);
    d.nx = nx; d.ny = ny; d.nz = nz;
    for (int a = 0; a < 3; ++a) d.per[a] = periodic[a] ? 1 : 0;
    d.nbx = (int)nbx; d.nby = (int)nby; d.nbz = (int)nbz;
    d.tile0 = 0;
    d.seg0 = 0;
    d.row0 = 0;

    hk::TmapPair tm;
    std::memset(&tm, 0, sizeof(tm));   // plain-load path: no tensor maps
    e = hk::launch_label(TY, TZ, &d, 1, P, W, &tm, st, nullptr);
    if (e != cudaSuccess) return HK_ERR_CUDA;

    if (d.sizes_cap < (N + 1) / 2) {
        int64_t n = 0;
        e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) e = cudaMemcpy(&n, d.ncl, sizeof(n), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return HK_ERR_CUDA;
        if (n > d.sizes_cap) return HK_ERR_CAPACITY;
    }
    return HK_OK;
}
