/*
 * hk_gen.h -- synthetic order-parameter fields generated on the device.
 *
 * These stand in for the lattice-Boltzmann fields of the paper's applications
 * (emulsion droplets, Sec. 5; capsule index fields, Sec. 6), which are not
 * available here.  They are inputs only, not part of the labelling method.
 * All pointers are device memory owned by the caller; calls are asynchronous
 * on `stream` (cudaStream_t as void*).  Layout: float32 phi[nz][ny][nx].
 * Return: 0 on success, 1 on a bad argument, 4 on a CUDA error.
 *
 * Random stream: u(seed, k) = (splitmix64((seed << 40) + k) >> 40) * 2^-24,
 * with splitmix64 the finaliser of Steele, Lea and Flood (OOPSLA 2014).  The
 * host generator (paper_1405_1931_gb300/fields.py) implements the same
 * definition, and hk_gen_iid produces bit-identical fields to it.
 */
#ifndef HK_GEN_H
#define HK_GEN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* phi[s] = u(seed, s) - c in float32, with c = (float)(1 - occupancy). */
int hk_gen_iid(float *phi, int nx, int ny, int nz, uint64_t seed, double occupancy, void *stream);

/* Droplets: phi = -1, then for each sphere i (centre cx,cy,cz, radius r; host
 * arrays of n_spheres entries, copied during the call) and every site within
 * the periodic minimum-image distance d <= r + reach:
 * phi = max(phi, tanh((r - d) / 2)), evaluated in float32. */
int hk_gen_spheres(float *phi, int nx, int ny, int nz, const double *centres_xyz, const double *radii,
                   int n_spheres, double reach, void *stream);

/* As hk_gen_spheres, with the spheres already on the device: `spheres` is a
 * device array of n_spheres x 4 floats (cx, cy, cz, r).  Launches only; the
 * host does not wait. */
int hk_gen_spheres_dev(float *phi, int nx, int ny, int nz, const float *spheres, int n_spheres, double reach,
                       void *stream);

/* Closed ellipsoidal shell in an L^3 box: phi = -1 where F <= 1 and some
 * 6-neighbour has F > 1, else +1; F = sum_i ((x_i - L/2) / a_i)^2 evaluated in
 * float64 without contraction, identical to the host generator. */
int hk_gen_capsule(float *phi, int L, double ax, double ay, double az, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* HK_GEN_H */
