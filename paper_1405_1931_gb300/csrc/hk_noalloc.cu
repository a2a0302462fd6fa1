// hk_noalloc.cu -- hk_label_noalloc: labelling without any device allocation.
//
// Some callers cannot allocate device memory: a simulation that has already
// handed all free device memory to its own allocator, or a code path where a
// cudaMalloc/cudaFree would synchronise the device and stall the caller's
// other streams.  This entry point runs the same passes as hk_label, but its
// scratch (a status header, then the workspace of a context's layout: occupancy
// mask, run codes, face summaries, piece table, root counts and prefix) lives in
// one file-scope __device__ array of fixed size instead of a context workspace.
// The caller still passes phi and the output buffers.
#include <cstdint>
#include <cstring>

#include <cuda_runtime.h>

#include "../../include/hk.h"
#include "hk_device.cuh"
#include "hk_launch.h"

namespace {

constexpr size_t SCRATCH_BYTES = (size_t)HK_NOALLOC_SCRATCH_BYTES;
constexpr size_t HEADER_BYTES = 256;   // the status word and the dense-tile count, then the workspace
constexpr int TY = 16, TZ = 16;
using hk::MAX_DEVICES;

// Every GPU that loads the library holds this array until the process exits.
__device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

// Device address of g_scratch on each device.  In host code the name g_scratch
// is only a host-side stand-in for the symbol, never a device pointer.
void *g_scratch_addr[MAX_DEVICES];

// The array's device address on the current device, looked up the first time a
// device is used (the status header is then cleared on `st`, ahead of that call's
// passes); nullptr on a CUDA error.
char *scratch_base(int dev, cudaStream_t st) {
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return nullptr;
        e = cudaMemsetAsync(p, 0, HEADER_BYTES, st);   // the status word starts clear
        if (e != cudaSuccess) return nullptr;
        g_scratch_addr[dev] = p;
    }
    return static_cast<char *>(g_scratch_addr[dev]);
}

int current_device(int &dev) {
    return (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < MAX_DEVICES) ? HK_OK : HK_ERR_CUDA;
}

// Read and clear the status word once `st` has been synchronised.
int take_status(char *base, cudaStream_t st) {
    int32_t s = 0;
    cudaError_t e = cudaMemcpy(&s, base, sizeof(s), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && s) {
        e = cudaMemsetAsync(base, 0, sizeof(s), st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) return HK_ERR_CUDA;
    return s ? HK_ERR_TIMEOUT : HK_OK;
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
    const hk::Layout Ly = hk::make_layout(ti, P);   // the same workspace layout as a context's
    if (HEADER_BYTES + Ly.total > SCRATCH_BYTES) return HK_ERR_TOO_LARGE;   // rejected before touching the GPU

    int dev = 0;
    if (current_device(dev) != HK_OK) return HK_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    char *base = scratch_base(dev, st);
    if (!base) return HK_ERR_CUDA;

    // The array keeps the previous call's contents.  Everything the passes read is
    // written earlier in the same call; the status word is cleared only when it is
    // read (here on the capacity path, or by hk_noalloc_sync_status), so a give-up is
    // reported even when several calls run before the check.
    hk::Work W = hk::bind_work(base + HEADER_BYTES, Ly, reinterpret_cast<int32_t *>(base), P.piece_cap, 0);
    W.rootbits = nullptr;   // no interior/exterior identification here
    W.segpre = nullptr;
    W.votes = nullptr;

    hk::LatDev d;
    std::memset(&d, 0, sizeof(d));
    d.phi = phi;
    d.labels = labels_out;
    d.sizes = sizes_out;
    d.sizes_cap = sizes_out ? sizes_cap : 0;
    d.hist = hist_out;
    d.ncl = n_clusters_out ? n_clusters_out : reinterpret_cast<int64_t *>(base + HEADER_BYTES + Ly.ncl);
    d.nx = nx; d.ny = ny; d.nz = nz;
    for (int a = 0; a < 3; ++a) d.per[a] = periodic[a] ? 1 : 0;
    d.nbx = (int)nbx; d.nby = (int)nby; d.nbz = (int)nbz;
    d.tile0 = 0;
    d.seg0 = 0;
    d.row0 = 0;

    hk::TmapPair tm;
    std::memset(&tm, 0, sizeof(tm));   // plain-load path: no tensor maps
    cudaError_t e = hk::launch_label(TY, TZ, &d, 1, P, W, &tm, st, nullptr);
    if (e != cudaSuccess) return HK_ERR_CUDA;

    if (d.sizes_cap < (N + 1) / 2) {
        // the capacity rule needs the count: wait, and report the status word with it
        int64_t n = 0;
        e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) e = cudaMemcpy(&n, d.ncl, sizeof(n), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return HK_ERR_CUDA;
        const int rc = take_status(base, st);
        if (rc != HK_OK) return rc;
        if (n > d.sizes_cap) return HK_ERR_CAPACITY;
    }
    return HK_OK;
}

extern "C" int hk_noalloc_sync_status(void *stream) {
    int dev = 0;
    if (current_device(dev) != HK_OK) return HK_ERR_CUDA;
    if (!g_scratch_addr[dev]) return HK_OK;   // no call on this device yet
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(st) != cudaSuccess) return HK_ERR_CUDA;
    return take_status(static_cast<char *>(g_scratch_addr[dev]), st);
}
