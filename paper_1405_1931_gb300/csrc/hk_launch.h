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

// Byte offsets of the workspace buffers of one launch (every offset 256-byte aligned).
struct Layout {
    size_t mask, codes, cnt, pre, bsum, face, tinfo, parent, key, psize, xcol, ovf, rootbits, segpre, votes, ncl, total;
};

// The workspace of one launch.  votes_cap > 0: also the root bits, the segment prefix
// and the per-cluster votes of the interior/exterior identification (index fields).
inline Layout make_layout(const TileInfo &ti, const Plan &P, int64_t votes_cap = 0) {
    Layout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    const int64_t nb = (P.nrows + 4096) / 4096;   // scan blocks (4096 rows each) covering index nrows
    L.mask = take((size_t)P.ntiles * ti.rows * 4);
    L.codes = take((size_t)P.ntiles * ti.maxruns * 2);
    L.cnt = take((size_t)P.nseg);
    L.pre = take((size_t)(P.nrows + 1) * 4);
    L.bsum = take((size_t)nb * 4);
    L.face = take((size_t)P.ntiles * ti.face_stride * 2);
    L.tinfo = take((size_t)P.ntiles * 16);
    L.parent = take((size_t)P.piece_cap * 4);
    L.key = take((size_t)P.piece_cap * 4);
    L.psize = take((size_t)P.piece_cap * 4);
    L.xcol = take((size_t)P.ntiles * (ti.rows / 32) * 2 * 4);
    L.ovf = take((size_t)P.ntiles * 4);
    L.rootbits = take(votes_cap > 0 ? (size_t)P.nseg * 4 : 0);
    L.segpre = take(votes_cap > 0 ? (size_t)P.nseg * 4 : 0);
    L.votes = take((size_t)votes_cap * 4);
    L.ncl = take((size_t)MAX_LAT_PER_LAUNCH * 8);
    L.total = off;
    return L;
}

// The Work pointers of a workspace laid out by `Ly` at device address `base`.  status:
// two device int32 words (the STATUS_* flags, then the count of tiles handed to the
// dense tile pass).  loop_cap > 0 lowers the bound of every capped union-find loop
// (0: the natural bounds, the run count and the piece-table size).
Work bind_work(char *base, const Layout &Ly, int32_t *status, int64_t piece_cap, int64_t loop_cap);

bool tile_info(int ty, int tz, TileInfo &ti);

// One-CTA path for small lattices (hk_small.cu): a lattice of at most SMALL_MAX_SITES
// sites and SMALL_MAX_SEG row segments is labelled by one kernel in shared memory, with
// no workspace.  Runs never exceed N/2 + nseg/2 <= SMALL_MAX_RUNS.
constexpr int SMALL_MAX_SITES = 32768;
constexpr int SMALL_MAX_SEG = 2048;
constexpr int SMALL_MAX_RUNS = 16384 + 2048;
bool small_fits(int nx, int ny, int nz);
// The cluster form (hk_small.cu): a cluster of CS CTAs on CS SMs labels one lattice
// whose rows, split into CS equal blocks, come to at most 1024 row segments a block.
// CS is 16 where the device co-schedules a cluster that large, else 8 (64^3 fits
// either way); cluster_fits applies this device's CS.
bool cluster_fits(int nx, int ny, int nz);
// whether this device can run the cluster form, and how many of its clusters the device
// holds at once (checked once per device)
bool cluster_ok();
int cluster_slots();
// n lattices that all fit the chosen form (n <= MAX_LAT_PER_LAUNCH): one CTA each, or with
// cluster (after cluster_ok()) one cluster of CS CTAs each; every lat[i].ncl must be a
// device int64.  status: the device status word; local_cap as in Work.
cudaError_t launch_small(const LatDev *lats, int n, int32_t *status, int32_t local_cap, cudaStream_t st,
                         bool cluster);

// The merge schedule: unions per lane and step of the face merge (1, 2 or 4), and
// whether the piece finalize combines the size additions of the cluster root that
// collects most of them per warp and per CTA (hot) or adds each group's directly.
struct MergeSchedule {
    int unions = 1;
    int hot = 1;
};

// ev: NUM_PASSES + 1 events recorded around the passes, or nullptr.  tms: the tensor
// maps of each of the n lattices (valid == 0: that lattice takes the plain-load and
// plain-store paths), or nullptr for none.
cudaError_t launch_label(int ty, int tz, const LatDev *lats, int n, const Plan &P, const Work &W,
                         const TmapPair *tms, cudaStream_t st, cudaEvent_t *ev, MergeSchedule ms = MergeSchedule());

// The slab merge (hk_slab.cu): the face data of all R ranks and this rank's slab.
struct SlabMerge {
    int R;                          // ranks (slabs)
    int ninterfaces;                // R - 1, plus one when z is periodic (slab R - 1 to slab 0)
    int64_t P;                      // sites of a z plane, nx * ny
    int64_t maxF;                   // row length of the gathered face-cluster lists
    int64_t G;                      // face clusters of all ranks
    int64_t g0, nf_own;             // this rank's first node and its face-cluster count
    const int32_t *face_all;        // [R][2][P] face-cluster number of each face site, or -1
    const int32_t *list_lab_all;    // [R][maxF] labels of the face clusters
    const int64_t *list_size_all;   // [R][maxF] local sizes of the face clusters
    const int64_t *off, *cnt;       // [R] device: first node and face-cluster count of each rank
    int32_t *parent, *lab;          // [G] scratch
    int64_t *size, *csize;          // [G] scratch
    int32_t *labels;                // this slab's labels, rewritten in place
    int64_t nsites, site_off;       // sites of the slab and the index of its first site
    const int64_t *sizes, *ncl;     // this slab's local cluster sizes and count (device)
    int64_t ncl_cap;                // entries of sizes / fmap
    const int32_t *fmap;            // [ncl_cap] face-cluster number of each local cluster, or -1
    uint32_t *bsum;                 // [ncl_cap / 4096 + 1] scratch
    int64_t *own_sizes, own_cap, *own_ncl, *hist;   // outputs
    int32_t *status;
};
cudaError_t launch_slab_faces(const int32_t *labels, int nx, int ny, int nzr, const int32_t *roots, const int64_t *ncl,
                              const int64_t *sizes, int64_t ncl_cap, int32_t *fmap, int32_t *face_out,
                              int32_t *list_lab, int64_t *list_size, int64_t *nf, cudaStream_t st);
cudaError_t launch_slab_merge(const SlabMerge &M, cudaStream_t st);

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
