// hk_launch.h -- internal interface between the C ABI (hk_api.cu) and the
// kernels (hk_kernels.cu).  Not installed; the public interface is include/hk.h.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace hk {

struct LatDev;
struct Work;
struct TmapPair;

// lattices per launch: the descriptors and tensor maps of a launch travel as kernel
// parameters (under the 32 KB parameter limit)
constexpr int MAX_LAT_PER_LAUNCH = 64;
// devices one process may use (per-device launch state is kept for this many)
constexpr int MAX_DEVICES = 64;

struct TileInfo {
    int ty, tz;
    int rows;            // tile rows (ty * tz), one 32-bit occupancy word each
    int maxruns;         // run-code entries per tile
    int face_stride;     // uint16 face entries per tile
    int max_boundary;    // bound on boundary pieces per tile
};

struct Plan {
    int64_t ntiles;      // tiles of all lattices in the launch
    int64_t nseg;        // row segments of all lattices
    int64_t nrows;       // lattice rows (y, z) of all lattices
    int64_t piece_cap;   // ntiles * max_boundary
};

constexpr int NUM_PASSES = 7;   // occupancy, tile_label, face_merge, piece_finalize, scan, lattice_finish, flatten

bool tile_info(int ty, int tz, TileInfo &ti);

// ev: NUM_PASSES + 1 events recorded around the passes, or nullptr.  tms: the tensor
// maps of each of the n lattices (valid == 0: that lattice takes the plain-load and
// plain-store paths), or nullptr for none.
cudaError_t launch_label(int ty, int tz, const LatDev *lats, int n, const Plan &P, const Work &W,
                         const TmapPair *tms, cudaStream_t st, cudaEvent_t *ev);

// Interior/exterior tags of a lattice labelled with occ_mode 1 (after launch_label on
// the same stream; needs W.rootbits and W.votes).
// state != nullptr: also the interior state of every site
cudaError_t launch_interior(const LatDev &L, const Work &W, cudaStream_t st, int8_t *state = nullptr);
// out[s] = the side index[s] names where the site is near a membrane (index >= -0.5 or
// NaN), else prev[s]; out may be prev
cudaError_t launch_interior_update(const int8_t *prev, const float *index, int64_t n, int8_t *out, cudaStream_t st);
// state[sites[i]] = the side values[i] names, for near values and sites in [0, n)
cudaError_t launch_interior_update_sites(int8_t *state, int64_t n, const int32_t *sites, const float *values,
                                         int64_t m, cudaStream_t st);
// dst[i] = src[i] for i < min(*count, cap): a copy sized on the device (dst may be
// device-accessible host memory)
cudaError_t launch_copy_counted(const int64_t *src, const int64_t *count, int64_t cap, int64_t *dst,
                                cudaStream_t st);

}  // namespace hk
