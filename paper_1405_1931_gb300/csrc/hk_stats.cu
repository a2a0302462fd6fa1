// hk_stats.cu -- droplet-size statistics from the cluster sizes (Fig. 5).
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/hk.h"

namespace {

constexpr int MAX_EDGES = 64;
// 4 pi / 3, folded at compile time in double precision
constexpr double FOUR_THIRDS_PI = 4.0 * 3.14159265358979323846 / 3.0;

struct Thresholds {
    double t[MAX_EDGES];   // t_b = (e_b^3) (4 pi / 3): R_c >= e_b  <=>  V >= t_b
    int m;
};

// One pass over the sizes: a histogram per CTA in shared memory, the sum of R_c per
// CTA by warp shuffles, both added to the outputs once per CTA.
__global__ void __launch_bounds__(256) k_rc_hist(const int64_t *sizes, const int64_t *n_dev, int64_t cap,
                                                 const __grid_constant__ Thresholds T, int64_t *hist,
                                                 double *rc_sum) {
    __shared__ unsigned long long sh[MAX_EDGES + 1];
    __shared__ double wsum[8];
    for (int b = threadIdx.x; b <= T.m; b += blockDim.x) sh[b] = 0ull;
    __syncthreads();
    const int64_t n = *n_dev < cap ? *n_dev : cap;
    double acc = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const double V = (double)sizes[k];
        int bin = 0;
        for (int b = 0; b < T.m; ++b)
            if (V >= T.t[b]) bin = b + 1;
        atomicAdd(&sh[bin], 1ull);
        acc += cbrt(V / FOUR_THIRDS_PI);
    }
    for (int d = 16; d; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0 && rc_sum) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += wsum[w];
        if (s != 0.0) atomicAdd(rc_sum, s);
    }
    for (int b = threadIdx.x; b <= T.m; b += blockDim.x)
        if (sh[b]) atomicAdd(reinterpret_cast<unsigned long long *>(hist) + b, sh[b]);
}

}  // namespace

extern "C" int hk_rc_histogram(const int64_t *sizes, const int64_t *n_clusters, int64_t sizes_cap,
                               const double *edges, int n_edges, int64_t *hist_out, double *rc_sum_out,
                               int accumulate, void *stream) {
    if (!n_clusters || !edges || !hist_out || sizes_cap < 0 || (sizes_cap > 0 && !sizes)) return HK_ERR_ARG;
    if (n_edges < 1 || n_edges > MAX_EDGES) return HK_ERR_ARG;
    Thresholds T;
    T.m = n_edges;
    for (int b = 0; b < n_edges; ++b) {
        if (b > 0 && !(edges[b - 1] < edges[b])) return HK_ERR_ARG;
        const double e = edges[b];
        T.t[b] = ((e * e) * e) * FOUR_THIRDS_PI;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!accumulate) {
        if (cudaMemsetAsync(hist_out, 0, sizeof(int64_t) * (size_t)(n_edges + 1), st) != cudaSuccess) return HK_ERR_CUDA;
        if (rc_sum_out && cudaMemsetAsync(rc_sum_out, 0, sizeof(double), st) != cudaSuccess) return HK_ERR_CUDA;
    }
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HK_ERR_CUDA;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int64_t grid = (sizes_cap + 255) / 256;
    if (grid > (int64_t)nsm * 4) grid = (int64_t)nsm * 4;
    if (grid < 1) grid = 1;
    k_rc_hist<<<(unsigned)grid, 256, 0, st>>>(sizes, n_clusters, sizes_cap, T, hist_out, rc_sum_out);
    return cudaGetLastError() == cudaSuccess ? HK_OK : HK_ERR_CUDA;
}
