/*
 * hk.h -- C ABI of the GB300 Hoshen-Kopelman cluster-labelling library (libhk).
 *
 * Method: Frijters, Krueger, Harting, "Parallelised Hoshen-Kopelman algorithm
 * for lattice-Boltzmann simulations", Comput. Phys. Commun. (2014).
 *
 * What a call computes, for a 3D lattice of nx*ny*nz sites holding a float32
 * order parameter phi:
 *   - occupancy: site x belongs to a cluster iff phi(x) > 0 (Sec. 2, opening
 *     paragraph); phi <= 0, -0 and NaN are the medium;
 *   - clusters: the connected components of the occupied sites under
 *     nearest-neighbour (face, 6-)connectivity, diagonals excluded (Sec. 2,
 *     remark after the three rules), with per-axis periodic edges
 *     (n_a - 1) <-> 0 (Sec. 3, Fig. 2 caption and the halo paragraph);
 *   - labels: each cluster is labelled by its smallest row-major site index
 *     s = x + nx*(y + ny*z) (x fastest, phi laid out as C array
 *     phi[nz][ny][nx]); the medium gets -1.  This is the "smallest possible
 *     number" relabelling of Sec. 2 (final paragraph) expressed as a site
 *     index rather than a compacted id;
 *   - sizes: sizes_out[k] = number of sites of the cluster with the (k+1)-th
 *     smallest label, i.e. clusters in the compactified order 1..n of Sec. 2
 *     (final paragraph); the site counts are those of Sec. 5 ("counting the
 *     number of sites with a particular label");
 *   - histogram: hist_out[b] = number of clusters whose size has
 *     floor(log2(size)) == b, 0 <= b < 32 (the droplet-size histogram of
 *     Fig. 5, binned by integer size; any radius binning R_c ~ size^(1/3) is a
 *     monotone re-binning done by the caller);
 *   - n_clusters_out = n.
 * The result is unique, so it is bit-identical to the serial algorithm.
 *
 * Conventions shared by every entry point:
 *   - Device pointers are caller-owned CUDA device memory on the context's
 *     device; the library never frees them.  Host pointers are read during the
 *     call only.
 *   - Calls are asynchronous on the given stream (a cudaStream_t passed as
 *     void*, NULL = legacy default stream) unless stated otherwise; results are
 *     valid once that stream has reached the end of the call.
 *   - A context owns a workspace that it grows on demand (cudaMalloc) and
 *     reuses.  Calls that share a context must be issued on one stream (or be
 *     otherwise ordered); use one context per concurrent stream.
 *   - Return codes: HK_OK, or one of the HK_ERR_* codes below.  Argument
 *     errors are detected on the host before anything is enqueued.
 *   - N = nx*ny*nz must be < 2^31 (labels are int32 site indices).
 */
#ifndef HK_H
#define HK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HK_OK            0
#define HK_ERR_ARG       1  /* null pointer, dimension < 1, negative capacity, bad count */
#define HK_ERR_TOO_LARGE 2  /* nx*ny*nz >= 2^31 (hk_label_noalloc: scratch too small) */
#define HK_ERR_CAPACITY  3  /* more clusters than sizes_cap (labels, hist, count still valid) */
#define HK_ERR_CUDA      4  /* a CUDA runtime call failed (see hk_last_cuda_error) */
#define HK_ERR_TIMEOUT   5  /* a bounded device-side wait gave up */
#define HK_ERR_NOMEM     6  /* workspace allocation failed */

typedef struct hk_ctx hk_ctx;

/* Create a context bound to CUDA device `device`.  *out receives the handle.
 * Errors: HK_ERR_ARG (out == NULL), HK_ERR_CUDA (bad device). */
int hk_create(hk_ctx **out, int device);

/* Release a context and its workspace.  The caller must make sure no call on
 * it is still running on the GPU.  NULL is ignored. */
void hk_destroy(hk_ctx *ctx);

/* Device workspace in bytes that one hk_label call on an nx*ny*nz lattice
 * needs (an upper bound, independent of phi).  Used for admission control.
 * Returns 0 for invalid dimensions. */
size_t hk_workspace_bytes(int nx, int ny, int nz);

/* Grow the context's workspace to at least `bytes` now, so later calls do not
 * allocate.  Errors: HK_ERR_ARG, HK_ERR_NOMEM. */
int hk_reserve(hk_ctx *ctx, size_t bytes);

/* Label one lattice (Sec. 2 rules with Sec. 3's periodic merging; see above).
 *   phi            device, float32[nz][ny][nx], read only.
 *   periodic       host, int[3]: nonzero = periodic along x, y, z.
 *   labels_out     device, int32[nz][ny][nx]: min site index of the cluster, -1 medium.
 *   sizes_out      device, int64[sizes_cap]: cluster sizes in label order (may be
 *                  NULL when sizes_cap == 0).  ceil(N/2) entries always suffice
 *                  (clusters are pairwise non-adjacent: at most V/2 of them, Sec. 3).
 *   hist_out       device, int64[32] (may be NULL).
 *   n_clusters_out device, int64[1] (may be NULL).
 *   stream         cudaStream_t as void*.
 * When sizes_cap < ceil(N/2) the call synchronises the stream at its end to
 * check the count and returns HK_ERR_CAPACITY if n > sizes_cap (then only the
 * first sizes_cap sizes are written; everything else is complete); otherwise it
 * is fully asynchronous.
 * Errors: HK_ERR_ARG, HK_ERR_TOO_LARGE, HK_ERR_NOMEM, HK_ERR_CUDA, HK_ERR_CAPACITY. */
int hk_label(hk_ctx *ctx, const float *phi, int nx, int ny, int nz, const int periodic[3],
             int32_t *labels_out, int64_t *sizes_out, int64_t sizes_cap,
             int64_t *hist_out, int64_t *n_clusters_out, void *stream);

/* Interior and exterior of closed membranes (Sec. 6, steps 3-5).
 *   index          device, float32[nz][ny][nx]: the index field I of Sec. 6, step 2:
 *                  I < -0.5 far from every membrane (the initial I_0), -0.5 <= I <= 0.5
 *                  near one, negative on its inner side and positive on its outer side.
 *   inside_out     device, int8[sizes_cap] (may be NULL when sizes_cap == 0):
 *                  inside_out[k] = 1 if the cluster with the (k+1)-th smallest label is
 *                  interior, 0 if exterior, -1 if undetermined.
 *   The other arguments are those of hk_label.
 * The clusters are those of the far sites, I < -0.5 (step 4, with the labels,
 * sizes, histogram and count of hk_label for that occupancy).  Step 5 decides
 * a cluster by the signs of I around it: every face-neighbour pair (cluster
 * site, near site), along the six directions with the same periodic wraps,
 * votes with the sign of I at the near site (I == 0 and NaN do not vote); more
 * negative votes -> interior, more positive -> exterior, a tie -> -1.
 * Same stream and capacity rules as hk_label; the tags of clusters beyond
 * sizes_cap are not written.  The workspace grows by N/4 bytes (a word of root
 * sites and a rank prefix per 32-site row segment) and 4 B per sizes_cap entry
 * for the votes.
 * Errors: HK_ERR_ARG, HK_ERR_TOO_LARGE, HK_ERR_NOMEM, HK_ERR_CUDA, HK_ERR_CAPACITY. */
int hk_label_interior(hk_ctx *ctx, const float *index, int nx, int ny, int nz, const int periodic[3],
                      int32_t *labels_out, int64_t *sizes_out, int64_t sizes_cap,
                      int64_t *hist_out, int64_t *n_clusters_out, int8_t *inside_out, void *stream);

/* One lattice of a batch: the arguments of hk_label bundled (device pointers,
 * same meaning and layout). */
typedef struct hk_lattice {
    const float *phi;
    int nx, ny, nz;
    int periodic[3];
    int32_t *labels;
    int64_t *sizes;
    int64_t sizes_cap;
    int64_t *hist;
    int64_t *n_clusters;
} hk_lattice;

/* Label n independent lattices of arbitrary, uneven shapes in one pass
 * sequence: every kernel runs once over the tiles of all lattices together
 * (one launch per pass for the whole batch, replayed from a cached CUDA graph
 * keyed by the batch's shapes).  Results are bit-identical to n separate
 * hk_label calls.  `lats` is a host array of n descriptors, read during the
 * call.  The capacity rule of hk_label applies per lattice.
 * Errors: HK_ERR_ARG (n < 0, bad descriptor), HK_ERR_TOO_LARGE, HK_ERR_NOMEM,
 * HK_ERR_CUDA, HK_ERR_CAPACITY (some lattice overflowed its sizes_cap). */
int hk_label_batched(hk_ctx *ctx, const hk_lattice *lats, int n, void *stream);

/* ---- A lattice split into slabs along z across ranks (Sec. 3) -------------------
 * The domain decomposition of Sec. 3: each rank (one GPU, one context) holds planes
 * [z0, z0 + nz) of an nx * ny * NZ lattice, labels them, and the ranks merge the
 * clusters that cross the slab faces.  Every label is a site index of the whole
 * lattice, so labels are unique without Eq. 1's per-process offsets.  The caller moves
 * the face data between ranks (paper_1405_1931_gb300/distributed.py does it with
 * torch.distributed); every rank then resolves all equivalences itself, which replaces
 * the gather at a root process and the scatter.  Per rank, on one stream:
 *   1. hk_label_slab: labels of the slab's clusters (the x and y periodic edges apply
 *      inside the slab; z joins across slabs in step 3), their sizes, and each
 *      cluster's label (smallest site) in the same rank order;
 *   2. hk_slab_faces: the face clusters (clusters with a site on the slab's first or
 *      last plane), numbered 0 .. n_face - 1 in no particular order, with their labels
 *      and sizes, and for each site of the two face planes its face cluster or -1;
 *   3. the caller gathers every rank's face arrays, counts and lists, then
 *      hk_slab_merge: joins facing sites of consecutive slabs (and of the last and
 *      first slab when z is periodic) into classes, rewrites this slab's labels to the
 *      class label (the smallest site of the whole cluster), and writes the sizes of
 *      the clusters whose smallest site is in this slab, in label order, with their
 *      floor(log2 size) histogram;
 *   4. the caller adds the own counts of the earlier ranks to place this rank's sizes
 *      in the global order, and sums the histograms.
 * The results equal hk_label on the whole lattice: the concatenated slabs' labels, the
 * ranks' size lists in rank order, the summed histograms and counts.  Not tested on
 * several GPUs: the tests run two ranks on one GPU, exchanging through the host. */

/* Step 1.  phi: device float32[nz][ny][nx], the slab's planes z0 .. z0 + nz - 1 of a
 * lattice with (z0 + nz) * nx * ny < 2^31 sites up to the slab.  labels_out: device
 * int32[nz][ny][nx], labels as site indices of the whole lattice (-1 medium).
 * sizes_out (int64) and roots_out (int32): device, sizes_cap >= ceil(nx*ny*nz / 2)
 * entries; cluster k's size and label, k in label order.  n_clusters_out: device int64.
 * Asynchronous.  Errors: HK_ERR_ARG (null pointers, bad dimensions, smaller sizes_cap),
 * HK_ERR_TOO_LARGE, HK_ERR_NOMEM, HK_ERR_CUDA. */
int hk_label_slab(hk_ctx *ctx, const float *phi, int nx, int ny, int nz, int64_t z0, int periodic_x, int periodic_y,
                  int32_t *labels_out, int64_t *sizes_out, int64_t sizes_cap, int32_t *roots_out,
                  int64_t *n_clusters_out, void *stream);

/* Step 2, after step 1 on the same context and stream (the arguments are step 1's
 * outputs).  face_out: device int32[2][ny][nx], the face-cluster number of each site of
 * plane 0 and plane nz - 1 of the slab, or -1 for the medium.  list_lab_out (int32) and
 * list_size_out (int64): device, 2 * nx * ny entries; the label and size of face cluster
 * f.  n_face_out: device int64, the number of face clusters.  The context keeps each
 * local cluster's face-cluster number for step 3.  Asynchronous.
 * Errors: HK_ERR_ARG, HK_ERR_NOMEM, HK_ERR_CUDA. */
int hk_slab_faces(hk_ctx *ctx, const int32_t *labels, int nx, int ny, int nz, const int32_t *roots,
                  const int64_t *sizes, const int64_t *n_clusters, int64_t sizes_cap, int32_t *face_out,
                  int32_t *list_lab_out, int64_t *list_size_out, int64_t *n_face_out, void *stream);

/* Step 3, after step 2 on the same context, with the face data of all nranks ranks in
 * rank order (rank r holds planes after those of rank r - 1):
 *   face_all       device int32[nranks][2][ny][nx]: every rank's face_out;
 *   n_face_all     host int64[nranks]: every rank's n_face;
 *   list_lab_all   device int32[nranks][max_face], list_size_all device int64[nranks][max_face]:
 *                  every rank's lists, each padded to max_face >= every n_face;
 *   labels         this rank's labels (step 1), rewritten in place; nz, z0 its slab;
 *   sizes, n_clusters, sizes_cap: this rank's step-1 sizes and count;
 *   own_sizes_out  device int64[own_cap]: the sizes of the clusters whose smallest site
 *                  lies in this slab, in label order (a cluster that crosses slabs is
 *                  listed once, by the slab of its smallest site, with its whole size);
 *   own_n_out      device int64: their number (own_cap >= n_clusters always suffices);
 *   hist_out       device int64[32]: their floor(log2 size) histogram.
 * Synchronises the stream at its end.  Errors: HK_ERR_ARG (bad counts, step 2 missing),
 * HK_ERR_TOO_LARGE (2^31 face clusters or more), HK_ERR_NOMEM, HK_ERR_CUDA. */
int hk_slab_merge(hk_ctx *ctx, int nranks, int rank, int periodic_z, int nx, int ny, const int32_t *face_all,
                  const int64_t *n_face_all, const int32_t *list_lab_all, const int64_t *list_size_all,
                  int64_t max_face, int32_t *labels, int nz, int64_t z0, const int64_t *sizes,
                  const int64_t *n_clusters, int64_t sizes_cap, int64_t *own_sizes_out, int64_t own_cap,
                  int64_t *own_n_out, int64_t *hist_out, void *stream);

/* Replay calls from CUDA graphs.  When enabled, hk_label and hk_label_batched on a
 * non-default stream, with timing off and every sizes_cap >= ceil(N/2), keep
 * an instantiated CUDA graph of their launch sequence keyed by the exact
 * descriptors (pointers, shapes, periodic flags, capacities) and the tile
 * shape; a later call with the same descriptors (a simulation labelling its
 * field in place, step after step) replays it: one graph launch instead of one
 * launch per pass.  The first call with new descriptors runs normally and then
 * captures.  Graphs are dropped when the workspace grows,
 * when graphs are disabled and by hk_destroy; at most 8 are kept.  Buffers
 * named by a kept graph must stay allocated while it may be replayed.
 * Errors: HK_ERR_ARG. */
int hk_set_graphs(hk_ctx *ctx, int enable);

/* hk_label on HOST buffers: copies phi host->device, labels on the device and
 * copies labels, sizes, hist and the count back; synchronous.  Host buffers
 * may be pageable or pinned (pinned is faster).  Same argument meaning as
 * hk_label with every pointer in host memory.  The device copies live in the
 * context's workspace. */
int hk_label_host(hk_ctx *ctx, const float *phi_host, int nx, int ny, int nz, const int periodic[3],
                  int32_t *labels_host, int64_t *sizes_host, int64_t sizes_cap,
                  int64_t *hist_host, int64_t *n_clusters_host, void *stream);

/* hk_label_host without the wait, so that consecutive fields stream through
 * the host link: a simulation hands over snapshot i+1 while the labels of
 * snapshot i are still coming back.  Enqueues on `stream`, in order, the copy
 * of phi host->device, the labelling, the copies of the count, the labels and
 * the histogram back, and a kernel that writes the first min(count, sizes_cap)
 * sizes straight into sizes_host; then returns.  The paper has no counterpart
 * (its fields stay in the simulation's memory); this is a property of the
 * library.
 *
 * Arguments as hk_label_host, except:
 *   - every host buffer must be page-locked and device-accessible
 *     (cudaHostAlloc, cudaMallocHost or cudaHostRegister): a pageable one is
 *     rejected with HK_ERR_ARG before anything is enqueued;
 *   - host buffers are read and written after the call returns: phi_host must
 *     stay unchanged and the outputs unread until the stream has reached the
 *     end of the call (cudaStreamSynchronize, or an event recorded after it);
 *   - there is no capacity error: after completion, *n_clusters_host >
 *     sizes_cap means sizes_host holds only the first sizes_cap sizes
 *     (labels, histogram and count are complete either way);
 *   - n_clusters_host may be NULL.
 * Calls on one context are ordered by its stream rule (above): one context per
 * stream.  Two contexts on two streams, used for alternate fields, overlap one
 * field's phi copy with the other's label copy.
 * Errors: HK_ERR_ARG, HK_ERR_TOO_LARGE, HK_ERR_NOMEM, HK_ERR_CUDA. */
int hk_label_host_async(hk_ctx *ctx, const float *phi_host, int nx, int ny, int nz, const int periodic[3],
                        int32_t *labels_host, int64_t *sizes_host, int64_t sizes_cap,
                        int64_t *hist_host, int64_t *n_clusters_host, void *stream);

/* hk_label without any device allocation, for callers that cannot allocate
 * device memory (for example a simulation that has handed all free device
 * memory to its own allocator, or a loop in which a cudaMalloc/cudaFree would
 * synchronise the device and stall the caller's other streams).  The paper has
 * no counterpart; this is a property of the library, not of the method.
 *
 * Arguments, layout, results and the capacity rule are those of hk_label, on
 * the current CUDA device, with no context.  Instead of a context workspace
 * the call uses one file-scope __device__ scratch array of
 * HK_NOALLOC_SCRATCH_BYTES (64 MiB), which every GPU that loads the library
 * holds until the process exits; that is enough for lattices up to about 16
 * million sites (256^3).  A lattice whose scratch would not fit is rejected
 * with HK_ERR_TOO_LARGE before anything is enqueued.  The call never calls
 * cudaMalloc, cudaFree or any allocating library routine.
 *
 * The first call on a device looks up the array's device address on that
 * device (cudaGetSymbolAddress); make that first call before any stream
 * capture.  Every call shares the one array and it keeps the last call's
 * contents (each call rewrites what it reads), so calls that overlap on the
 * GPU -- on different streams, or from different host threads -- race and
 * must be serialised by the caller.  It uses the plain-load path (no TMA).
 *
 * The bounded device loops of these calls (see hk_sync_status) report to a
 * status word at the head of the array.  It is cleared only when it is read:
 * by this call when it synchronises for the capacity rule (it then returns
 * HK_ERR_TIMEOUT if a loop gave up), and by hk_noalloc_sync_status.
 * Errors: HK_ERR_ARG, HK_ERR_TOO_LARGE, HK_ERR_CUDA, HK_ERR_CAPACITY,
 * HK_ERR_TIMEOUT (capacity path only). */
#define HK_NOALLOC_SCRATCH_BYTES (64u << 20)
int hk_label_noalloc(const float *phi, int nx, int ny, int nz, const int periodic[3],
                     int32_t *labels_out, int64_t *sizes_out, int64_t sizes_cap,
                     int64_t *hist_out, int64_t *n_clusters_out, void *stream);

/* The status check of hk_label_noalloc, which has no context to ask
 * hk_sync_status: synchronises `stream` (the stream of the calls to check),
 * then reads and clears the status word of the current device's scratch
 * array.  HK_OK if no bounded device loop gave up since the last check (or no
 * call has run on this device), HK_ERR_TIMEOUT if one did; HK_ERR_CUDA on a
 * CUDA error.  Allocates nothing. */
int hk_noalloc_sync_status(void *stream);

/* Droplet-size histogram by R_c, the radius of a sphere with the cluster's
 * volume (Fig. 5 caption: (4 pi / 3) R_c^3 = V), over caller-given bin edges.
 *   sizes       device, int64[sizes_cap]: cluster sizes (e.g. hk_label's sizes_out).
 *   n_clusters  device, int64[1]: the count; min(*n_clusters, sizes_cap) sizes are read.
 *   edges       host, double[n_edges], strictly ascending, 1 <= n_edges <= 64; copied.
 *   hist_out    device, int64[n_edges + 1]: [0] counts R_c < edges[0], [b] counts
 *               edges[b-1] <= R_c < edges[b], [n_edges] counts R_c >= edges[n_edges-1].
 *   rc_sum_out  device, double[1] or NULL: the sum of R_c (mean droplet radius =
 *               rc_sum / count).
 *   accumulate  0: the outputs are cleared first; nonzero: added to (the stacked
 *               histograms of several realisations, Fig. 5).
 * R_c >= e is decided as V >= ((e*e)*e)*(4 pi/3) in double precision (thresholds
 * computed on the host), so no cube root decides a bin; rc_sum uses cbrt and is
 * summed in an unspecified order.  Asynchronous on `stream`.
 * Errors: HK_ERR_ARG (bad pointers, edges not ascending, n_edges out of range),
 * HK_ERR_CUDA. */
int hk_rc_histogram(const int64_t *sizes, const int64_t *n_clusters, int64_t sizes_cap,
                    const double *edges, int n_edges, int64_t *hist_out, double *rc_sum_out,
                    int accumulate, void *stream);

/* Interior state of every site of an index field (Sec. 6): the field the
 * simulation keeps up to date, 1 inside a closed membrane and 0 outside.
 *   index      device, float[nz][ny][nx]: I < -0.5 far from every membrane, near
 *              one the signed proximity value (step 2: -d inside, +d outside).
 *   state_out  device, int8[nz][ny][nx]: a far site (I < -0.5) takes the tag of
 *              its cluster (steps 3-5, as hk_label_interior: 1 interior, 0
 *              exterior, -1 undetermined); a near site (any other value, NaN
 *              included) the side its value names, 1 for I < 0 and 0 otherwise.
 * This is the full identification the paper uses to initialise the field and to
 * refresh it from time to time.  The clusters' labels, sizes and tags live in
 * the context (about 8.5 bytes a site, grown on demand).  Asynchronous on `stream`.
 * Errors: HK_ERR_ARG, HK_ERR_TOO_LARGE, HK_ERR_NOMEM, HK_ERR_CUDA. */
int hk_interior_state(hk_ctx *ctx, const float *index, int nx, int ny, int nz, const int periodic[3],
                      int8_t *state_out, void *stream);

/* The step between refreshes (Sec. 6, last paragraph): for membranes that move
 * much less than a lattice constant per step, only the sites near a membrane
 * now change.
 *   state_prev  device, int8[n_sites]: the previous state (hk_interior_state or
 *               an earlier update).
 *   index       device, float[n_sites]: the current index field.
 *   state_out   device, int8[n_sites]; may be state_prev (in place).
 * state_out[s] = 1 if I[s] is near and negative, 0 if near and not negative (near:
 * not I < -0.5), state_prev[s] if far.  A far site keeps its state because a
 * membrane that moves that slowly cannot carry it across without it being near
 * now; the tests check the result against hk_interior_state on capsules moving
 * under half a lattice constant per step.  No context; asynchronous on `stream`.
 * Errors: HK_ERR_ARG (n_sites < 0, null pointers), HK_ERR_CUDA. */
int hk_interior_update(const int8_t *state_prev, const float *index, int64_t n_sites, int8_t *state_out,
                       void *stream);

/* The same step from a list of near sites, as a simulation that walks its
 * membrane mesh (step 2) produces it: state[sites[i]] = 1 if values[i] < 0, else
 * 0, for each i < m with values[i] not below -0.5 and 0 <= sites[i] < n_sites
 * (other entries are skipped); unlisted sites keep their state.  A site listed
 * twice with values of different sides gets either.  sites (int32) and values
 * (float) are device arrays of m entries; state is device int8[n_sites],
 * updated in place.  No context; asynchronous on `stream`.
 * Errors: HK_ERR_ARG (negative counts, null pointers), HK_ERR_CUDA. */
int hk_interior_update_sites(int8_t *state, int64_t n_sites, const int32_t *sites, const float *values, int64_t m,
                             void *stream);

/* Select the tile shape (rows per tile along y and z; x tiles are always 32
 * sites wide).  Supported: (ty, tz) in {(8,8), (16,8), (16,16), (32,8)}; 0,0 =
 * the library default.  Applies to later calls on this context.
 * Errors: HK_ERR_ARG for an unsupported shape. */
int hk_set_tile(hk_ctx *ctx, int ty, int tz);

/* Select the merge schedule of the tiled passes (results are identical for every
 * schedule; only the time differs):
 *   unions_per_lane  face merge: unions each lane takes per step, their find chains
 *                    walked in lockstep so their loads overlap: 1, 2 or 4 (0 = the
 *                    default, 1);
 *   combine_hot      piece finalize: 1 (default) combines the size additions of the
 *                    cluster root that collects most of them -- the percolating
 *                    cluster's -- per warp and per CTA before the global add; 0 adds
 *                    each group of lanes' sum directly.
 * The tile shape (hk_set_tile) and this schedule are what autotune.py searches.
 * Applies to later calls on this context; drops its graphs.
 * Errors: HK_ERR_ARG for other values. */
int hk_set_merge(hk_ctx *ctx, int unions_per_lane, int combine_hot);

/* The one-launch path for small lattices: every step of hk_label (occupancy, x-runs,
 * their union-find with the periodic edges, ranks, sizes, histogram, labels) in one
 * kernel, in shared memory, with no workspace.  Two kernels:
 *   - one CTA holds a lattice of at most 32768 sites and 2048 row segments of 32
 *     sites along x (nx rounded up to a multiple of 32, times ny * nz);
 *   - a thread-block cluster of CS CTAs on CS SMs holds a lattice whose ny * nz
 *     rows, cut into CS equal blocks, come to at most 1024 row segments a block;
 *     CS is 16 where the device co-schedules clusters that large, else 8 (64^3
 *     fits either way); the CTAs reach each other's runs through distributed
 *     shared memory.
 * hk_label, hk_label_host(_async) and hk_label_batched take this path when every
 * lattice of the call fits: the cluster kernel when they all fit it and their clusters
 * take about half of the clusters the device holds at once, or fewer
 * (cudaOccupancyMaxActiveClusters), else one CTA per lattice where they all fit that,
 * else the cluster kernel; 64 lattices per launch.  Results are identical to the tiled passes.  With timing on, such a call
 * reports all its time as the first pass.  enable: 1 (default) as described; 0 this
 * context uses the tiled passes for every lattice; 2 the one-CTA kernel only; 3 the
 * cluster kernel only (for tests and comparisons; lattices the chosen kernel cannot
 * take go to the tiled passes).  Drops the context's graphs.
 * Errors: HK_ERR_ARG for ctx == NULL or enable outside 0 .. 3. */
int hk_set_small_path(hk_ctx *ctx, int enable);

/* Per-pass timing.  hk_set_timing(ctx, 1) resets the totals and makes every
 * later call record CUDA events on its own stream between its passes (a ring
 * of 64 event sets; the host waits for a call 64 calls old before reusing its
 * set).  hk_get_timing synchronises on the timed calls still in flight and
 * writes up to max_n per-pass AVERAGE durations in milliseconds over all timed
 * calls since timing was enabled to ms_out (host), in pass order: occupancy,
 * tile_label, face_merge, piece_finalize, scan (three kernels), lattice_finish,
 * flatten;
 * *n_out gets the number of passes.  For a batch split into several launch
 * chunks each chunk counts as one call.  Timing adds event records only;
 * results are unchanged.  Errors: HK_ERR_ARG (no timed call yet, NULL ctx or
 * ms_out), HK_ERR_CUDA. */
#define HK_NUM_PASSES 7
int hk_set_timing(hk_ctx *ctx, int enable);
int hk_get_timing(hk_ctx *ctx, float *ms_out, int max_n, int *n_out);

/* Synchronise `stream` and report whether any bounded device-side loop of the
 * context's calls since the previous check gave up (a corrupted union-find
 * would otherwise never terminate).  Clears the flag.  Returns HK_OK,
 * HK_ERR_TIMEOUT or HK_ERR_CUDA. */
int hk_sync_status(hk_ctx *ctx, void *stream);

/* Test control of the failure detection above: lower the bound of every
 * capped union-find loop of later calls on this context to `cap` iterations
 * (the shared-memory union retries and the global finds, unions and
 * compression of the piece merge), so that a test can make a loop give up on
 * an ordinary input and see HK_ERR_TIMEOUT from hk_sync_status.  A loop that
 * gives up leaves every index it holds in range (a find stops at a valid piece
 * or run id; a union stops without linking), so the labels of such a call are
 * wrong but every access stays inside the workspace and the outputs.  The
 * waits on TMA copies keep their bound.  cap == 0 restores the natural bounds
 * (the tile's run count and the piece-table size).  Drops the context's
 * graphs.  Errors: HK_ERR_ARG (NULL ctx, cap < 0). */
int hk_set_loop_cap(hk_ctx *ctx, int64_t cap);

/* The last CUDA error code seen by the context (cudaError_t as int). */
int hk_last_cuda_error(const hk_ctx *ctx);

/* Human-readable name of a status code (static string). */
const char *hk_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* HK_H */
