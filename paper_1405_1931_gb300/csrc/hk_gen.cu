// hk_gen.cu -- device generators of synthetic phi fields (inputs, not the method).
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/hk_gen.h"

namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_gen_iid(float *phi, int64_t n, uint64_t seed, float c) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * 4;
    for (int64_t s0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; s0 < n; s0 += stride) {
        float v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint64_t h = splitmix64((seed << 40) + (uint64_t)(s0 + j));
            const float u = (float)(uint32_t)(h >> 40) * 5.9604644775390625e-8f;   // 2^-24
            v[j] = __fsub_rn(u, c);
        }
        if (s0 + 3 < n && ((reinterpret_cast<uintptr_t>(phi + s0) & 15) == 0)) {
            *reinterpret_cast<float4 *>(phi + s0) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
            for (int j = 0; j < 4 && s0 + j < n; ++j) phi[s0 + j] = v[j];
        }
    }
}

__global__ void k_fill(float *phi, int64_t n, float v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        phi[i] = v;
}

__device__ __forceinline__ void atomic_max_float(float *addr, float value) {
    if (value >= 0.0f) atomicMax(reinterpret_cast<int *>(addr), __float_as_int(value));
    else atomicMin(reinterpret_cast<unsigned int *>(addr), __float_as_uint(value));
}

struct Sphere { float cx, cy, cz, r; };

// one block per sphere: visit the periodic bounding box of radius r + reach
__global__ void k_gen_spheres(float *phi, int nx, int ny, int nz, const Sphere *sp, float reach) {
    const Sphere s = sp[blockIdx.x];
    const float ext = s.r + reach;
    const int bx0 = (int)floorf(s.cx - ext), by0 = (int)floorf(s.cy - ext), bz0 = (int)floorf(s.cz - ext);
    const int wx = min((int)ceilf(s.cx + ext) - bx0 + 1, nx);
    const int wy = min((int)ceilf(s.cy + ext) - by0 + 1, ny);
    const int wz = min((int)ceilf(s.cz + ext) - bz0 + 1, nz);
    const int64_t total = (int64_t)wx * wy * wz;
    for (int64_t i = threadIdx.x; i < total; i += blockDim.x) {
        const int ix = (int)(i % wx), iy = (int)((i / wx) % wy), iz = (int)(i / ((int64_t)wx * wy));
        const int x = ((bx0 + ix) % nx + nx) % nx, y = ((by0 + iy) % ny + ny) % ny, z = ((bz0 + iz) % nz + nz) % nz;
        float dx = fabsf((float)x - s.cx), dy = fabsf((float)y - s.cy), dz = fabsf((float)z - s.cz);
        dx = fminf(dx, (float)nx - dx);
        dy = fminf(dy, (float)ny - dy);
        dz = fminf(dz, (float)nz - dz);
        const float d = sqrtf(dx * dx + dy * dy + dz * dz);
        if (d <= ext) atomic_max_float(phi + ((int64_t)z * ny + y) * nx + x, tanhf((s.r - d) * 0.5f));
    }
}

__device__ __forceinline__ double capsule_F(double gx, double gy, double gz, double ax, double ay, double az) {
    const double fx = __dmul_rn(__ddiv_rn(gx, ax), __ddiv_rn(gx, ax));
    const double fy = __dmul_rn(__ddiv_rn(gy, ay), __ddiv_rn(gy, ay));
    const double fz = __dmul_rn(__ddiv_rn(gz, az), __ddiv_rn(gz, az));
    return __dadd_rn(__dadd_rn(fz, fy), fx);
}

__global__ void k_gen_capsule(float *phi, int L, double ax, double ay, double az) {
    const int64_t n = (int64_t)L * L * L;
    const double h = 0.5 * L;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % L), y = (int)((i / L) % L), z = (int)(i / ((int64_t)L * L));
        const double gx = x - h, gy = y - h, gz = z - h;
        bool shell = false;
        if (capsule_F(gx, gy, gz, ax, ay, az) <= 1.0) {
            shell = capsule_F(gx - 1, gy, gz, ax, ay, az) > 1.0 || capsule_F(gx + 1, gy, gz, ax, ay, az) > 1.0 ||
                    capsule_F(gx, gy - 1, gz, ax, ay, az) > 1.0 || capsule_F(gx, gy + 1, gz, ax, ay, az) > 1.0 ||
                    capsule_F(gx, gy, gz - 1, ax, ay, az) > 1.0 || capsule_F(gx, gy, gz + 1, ax, ay, az) > 1.0;
        }
        phi[i] = shell ? -1.0f : 1.0f;
    }
}

int grid_for(int64_t n, int per_thread) {
    int64_t b = (n / per_thread + 255) / 256;
    if (b < 1) b = 1;
    if (b > 152 * 64) b = 152 * 64;
    return (int)b;
}

}  // namespace

extern "C" {

int hk_gen_iid(float *phi, int nx, int ny, int nz, uint64_t seed, double occupancy, void *stream) {
    if (!phi || nx < 1 || ny < 1 || nz < 1) return 1;
    const int64_t n = (int64_t)nx * ny * nz;
    const float c = (float)(1.0 - occupancy);
    k_gen_iid<<<grid_for(n, 4), 256, 0, static_cast<cudaStream_t>(stream)>>>(phi, n, seed, c);
    return cudaGetLastError() == cudaSuccess ? 0 : 4;
}

int hk_gen_spheres(float *phi, int nx, int ny, int nz, const double *centres_xyz, const double *radii,
                   int n_spheres, double reach, void *stream) {
    if (!phi || nx < 1 || ny < 1 || nz < 1 || n_spheres < 0 || (n_spheres > 0 && (!centres_xyz || !radii)))
        return 1;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t n = (int64_t)nx * ny * nz;
    k_fill<<<grid_for(n, 1), 256, 0, st>>>(phi, n, -1.0f);
    if (n_spheres == 0) return cudaGetLastError() == cudaSuccess ? 0 : 4;
    std::vector<Sphere> h(n_spheres);
    for (int i = 0; i < n_spheres; ++i)
        h[i] = Sphere{(float)centres_xyz[3 * i], (float)centres_xyz[3 * i + 1], (float)centres_xyz[3 * i + 2],
                      (float)radii[i]};
    Sphere *d = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void **>(&d), sizeof(Sphere) * n_spheres, st) != cudaSuccess) return 4;
    if (cudaMemcpyAsync(d, h.data(), sizeof(Sphere) * n_spheres, cudaMemcpyHostToDevice, st) != cudaSuccess) return 4;
    k_gen_spheres<<<n_spheres, 256, 0, st>>>(phi, nx, ny, nz, d, (float)reach);
    cudaFreeAsync(d, st);
    // a copy from pageable memory is staged before cudaMemcpyAsync returns, so the
    // host vector may go out of scope here
    return cudaGetLastError() == cudaSuccess ? 0 : 4;
}

int hk_gen_spheres_dev(float *phi, int nx, int ny, int nz, const float *spheres, int n_spheres, double reach,
                       void *stream) {
    if (!phi || nx < 1 || ny < 1 || nz < 1 || n_spheres < 0 || (n_spheres > 0 && !spheres)) return 1;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t n = (int64_t)nx * ny * nz;
    k_fill<<<grid_for(n, 1), 256, 0, st>>>(phi, n, -1.0f);
    if (n_spheres > 0)
        k_gen_spheres<<<n_spheres, 256, 0, st>>>(phi, nx, ny, nz, reinterpret_cast<const Sphere *>(spheres),
                                                  (float)reach);
    return cudaGetLastError() == cudaSuccess ? 0 : 4;
}

int hk_gen_capsule(float *phi, int L, double ax, double ay, double az, void *stream) {
    if (!phi || L < 1 || ax <= 0 || ay <= 0 || az <= 0) return 1;
    const int64_t n = (int64_t)L * L * L;
    k_gen_capsule<<<grid_for(n, 1), 256, 0, static_cast<cudaStream_t>(stream)>>>(phi, L, ax, ay, az);
    return cudaGetLastError() == cudaSuccess ? 0 : 4;
}

}  // extern "C"
