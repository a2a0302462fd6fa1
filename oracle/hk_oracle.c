/*
 * hk_oracle.c -- serial Hoshen-Kopelman oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * CPU definition that the CUDA path is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or helper with the CUDA library: it declares
 * its own entry points below and includes only the C standard library.
 *
 * What it computes (Frijters, Krueger, Harting, "Parallelised Hoshen-Kopelman
 * algorithm for lattice-Boltzmann simulations", CPC 2014):
 *
 *   - Occupancy (Sec. 2, opening paragraph; Fig. 1 caption): a site x is part
 *     of a cluster iff phi(x) > 0; phi <= 0 (and NaN) is the medium.
 *   - Initialisation (Sec. 2; Fig. 1b): l(x) = 0 on the medium and l(x) = -1
 *     ("to be labelled") on occupied sites.
 *   - Raster scan (Sec. 2, Fig. 1c and the remark after the three rules): the
 *     lattice is visited row by row (x fastest, then y, then z) and each site
 *     looks only "backwards" at its face neighbours x-1, y-1, z-1; diagonal
 *     sites are not neighbours.
 *   - Rules 1-3 (Sec. 2, enumerated rules): no labelled neighbour -> a new
 *     label l_max + 1; exactly one -> copy it; more than one -> take the
 *     minimum of the neighbours' labels and store the equivalences between
 *     them.
 *   - Equivalence store (Sec. 3, tuning paragraph): a singly linked list of
 *     label ids ("label of labels"), where following the list from any id ends
 *     at the lowest id of its class; a new equivalence walks both lists to
 *     their ends and re-points the end with the larger value at the smaller.
 *   - Periodic boundaries (Sec. 3, Fig. 2 caption and the halo paragraph): the
 *     paper merges across periodic edges through halo equivalences; serially
 *     that is one extra equivalence for every occupied pair (n_a - 1, 0) along
 *     each periodic axis a.  An axis of length 1 only has a self-edge.
 *   - Relabelling and compactification (Sec. 2, final paragraph; Fig. 1g/h):
 *     every id is reduced to the lowest id of its class, and the classes are
 *     numbered 1..n in increasing order of that lowest id.
 *   - Cluster sizes (Sec. 5, counting the sites with a given label) and the
 *     droplet-size histogram (Fig. 5 caption), here binned by
 *     floor(log2(size)).
 *
 * Output conventions (the readings listed in the design notes):
 *   labels_out[s]  = the smallest row-major site index s = x + nx*(y + ny*z)
 *                    of the cluster containing s, or -1 on the medium.  The
 *                    lowest label id of a class is the one created at the
 *                    class's first raster site, so this is the site at which
 *                    that id was created.
 *   sizes_out[k]   = number of sites of the cluster with compacted id k+1
 *                    (clusters ordered by their smallest site index).
 *   hist_out[b]    = number of clusters with floor(log2(size)) == b, b < 32.
 *   n_clusters_out = number of clusters.
 *
 * hk_oracle_interior follows the interior/exterior identification of Sec. 6
 * (steps 3-5) on an index field I: sites far from every membrane keep
 * I = I_0 < -0.5, sites within half a lattice constant of a membrane have
 * -0.5 <= I <= 0.5, negative on the inner side and positive on the outer side
 * (step 2).  Readings used:
 *   - step 4: the clusters are those of the far sites, taken as I < -0.5,
 *     labelled exactly as above (same labels, sizes, histogram, count);
 *   - step 5 ("an interior cluster is surrounded by sites with negative I
 *     while an exterior cluster borders on sites with positive I"): every
 *     face-neighbour pair (cluster site, near site) votes with the sign of I at
 *     the near site (I == 0 or NaN: no vote), along the six directions with
 *     the same periodic wraps as the labelling; a cluster with more negative
 *     votes is interior (1), with more positive votes exterior (0), otherwise
 *     undetermined (-1).  inside_out[k] is the tag of the cluster with
 *     compacted id k+1.
 *
 * hk_oracle_interior_state gives every site its interior state (Sec. 6: 0 far
 * outside, 1 far inside): a far site (I < -0.5) takes its cluster's tag from
 * hk_oracle_interior (1 interior, 0 exterior, -1 undetermined); a near site
 * takes the side its proximity value names (step 2: -d inside, +d outside),
 * 1 for I < 0 and 0 otherwise.
 *
 * hk_oracle_interior_update is the cheaper step of the last paragraph of Sec. 6
 * for membranes that move much less than a lattice constant per step: only the
 * sites near a membrane now are updated, to the side their value names now;
 * every other site keeps its previous state.  The paper's premise is that a
 * membrane moves much less than a lattice constant per step, so a site that is
 * far from every membrane now has not changed sides since the last step.  Under
 * that premise the result equals hk_oracle_interior_state of the current field;
 * a test checks this on capsules moving by under half a lattice constant per
 * step, and shows that it fails for a jump of several lattice constants.
 *
 * hk_oracle_mt_label is the paper's parallel scheme (Sec. 3) on host threads, one
 * thread for each process of a decomposition into slabs along z:
 *   1. every domain is labelled by the serial algorithm above on its own sites,
 *      its x and y periodic edges included;
 *   2. n_max, the largest local label count, is shared, and local label k of
 *      domain w becomes the global id w * n_max + k (Eq. 1);
 *   3. halo: each domain reads the labels of the first plane of the next domain
 *      along z (the last domain the first's, when z is periodic) and records an
 *      equivalence of global ids for every pair of occupied sites across that face;
 *   4. the equivalences are gathered at the root, which resolves them, gives every
 *      class the smallest site index of its members and scatters that back;
 *   5. every domain relabels its sites.
 * The root computes the sizes, the compactified order and the histogram.  The
 * result is the same as hk_oracle_label's (the output is unique); a test checks it.
 *
 * hk_oracle_rc_histogram bins cluster sizes V by R_c, the radius of a sphere of
 * volume V (Fig. 5 caption: (4 pi / 3) R_c^3 = V), with caller-given ascending
 * edges e_0 < ... < e_{m-1}.  R_c >= e is decided as V >= t(e) with
 * t(e) = ((e * e) * e) * (4 pi / 3) in double precision, so no cube root decides
 * a bin.  hist[0] counts R_c < e_0, hist[b] (1 <= b < m) counts
 * e_{b-1} <= R_c < e_b and hist[m] counts R_c >= e_{m-1}.  rc_sum = sum of
 * cbrt(3 V / (4 pi)) over the clusters (for the mean droplet radius).
 */
#define _POSIX_C_SOURCE 200809L   /* pthread barriers */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define HKO_OK 0
#define HKO_ERR_ARG 1
#define HKO_ERR_TOO_LARGE 2
#define HKO_ERR_CAPACITY 3
#define HKO_ERR_NOMEM 6

int hk_oracle_label(const float *phi, int nx, int ny, int nz, const int periodic[3],
                    int32_t *labels_out, int64_t *sizes_out, int64_t sizes_cap,
                    int64_t *hist_out, int64_t *n_clusters_out);
int hk_oracle_version(void);
int hk_oracle_interior(const float *index, int nx, int ny, int nz, const int periodic[3],
                       int32_t *labels_out, int64_t *sizes_out, int64_t sizes_cap,
                       int64_t *hist_out, int64_t *n_clusters_out, int8_t *inside_out);
int hk_oracle_rc_histogram(const int64_t *sizes, int64_t n, const double *edges, int n_edges,
                           int64_t *hist_out, double *rc_sum_out);
int hk_oracle_interior_state(const float *index, int nx, int ny, int nz, const int periodic[3],
                             int8_t *state_out);
int hk_oracle_interior_update(const int8_t *state_prev, const float *index, int64_t n, int8_t *state_out);
int hk_oracle_mt_label(const float *phi, int nx, int ny, int nz, const int periodic[3], int threads,
                       int32_t *labels_out, int64_t *sizes_out, int64_t sizes_cap,
                       int64_t *hist_out, int64_t *n_clusters_out);

int hk_oracle_version(void) { return 1; }

/* Growable per-label arrays: lol[k] (next id in k's equivalence list) and
 * first[k] (the site at which id k was created).  Index 0 is unused, so that
 * id k lives at index k and 0 keeps meaning "medium" as in the paper. */
typedef struct {
    int32_t *lol;
    int64_t *first;
    int64_t cap;
} label_table;

static int table_push(label_table *t, int32_t id, int64_t site) {
    if (id >= t->cap) {
        int64_t nc = t->cap ? 2 * t->cap : 1024;
        while (nc <= id) nc *= 2;
        int32_t *nl = (int32_t *)realloc(t->lol, (size_t)nc * sizeof(int32_t));
        if (!nl) return HKO_ERR_NOMEM;
        t->lol = nl;
        int64_t *nf = (int64_t *)realloc(t->first, (size_t)nc * sizeof(int64_t));
        if (!nf) return HKO_ERR_NOMEM;
        t->first = nf;
        t->cap = nc;
    }
    t->lol[id] = id; /* a new id is the end of its own list */
    t->first[id] = site;
    return HKO_OK;
}

/* Follow the linked list from id k to its end: the lowest id of k's class. */
static int32_t list_end(const int32_t *lol, int32_t k) {
    while (lol[k] != k) k = lol[k];
    return k;
}

/* Record a == b: walk both lists to their ends and re-point the end with the
 * larger value at the smaller one (Sec. 3, tuning paragraph). */
static void store_equivalence(int32_t *lol, int32_t a, int32_t b) {
    int32_t ea = list_end(lol, a);
    int32_t eb = list_end(lol, b);
    if (ea < eb) lol[eb] = ea;
    else if (eb < ea) lol[ea] = eb;
}

int hk_oracle_label(const float *phi, int nx, int ny, int nz, const int periodic[3],
                    int32_t *labels_out, int64_t *sizes_out, int64_t sizes_cap,
                    int64_t *hist_out, int64_t *n_clusters_out) {
    if (!phi || !periodic || !labels_out || !hist_out || !n_clusters_out) return HKO_ERR_ARG;
    if (nx < 1 || ny < 1 || nz < 1 || sizes_cap < 0) return HKO_ERR_ARG;
    if (sizes_cap > 0 && !sizes_out) return HKO_ERR_ARG;
    const int64_t sx = 1, sy = nx, sz = (int64_t)nx * ny;
    const int64_t N = (int64_t)nx * ny * nz;
    if (N >= ((int64_t)1 << 31)) return HKO_ERR_TOO_LARGE;

    /* The label field l(x) lives in labels_out until the final relabelling. */
    int32_t *l = labels_out;

    /* Initialisation: 0 on the medium, -1 on sites still to be labelled. */
    for (int64_t s = 0; s < N; ++s) l[s] = (phi[s] > 0.0f) ? -1 : 0;

    label_table t = {0, 0, 0};
    int32_t l_max = 0;
    int rc = HKO_OK;

    /* Raster scan with rules 1-3, looking only at x-1, y-1 and z-1. */
    for (int z = 0; z < nz && rc == HKO_OK; ++z) {
        for (int y = 0; y < ny && rc == HKO_OK; ++y) {
            for (int x = 0; x < nx; ++x) {
                const int64_t s = x * sx + y * sy + z * sz;
                if (l[s] != -1) continue;
                int32_t nb[3];
                int n_nb = 0;
                if (x > 0 && l[s - sx] > 0) nb[n_nb++] = l[s - sx];
                if (y > 0 && l[s - sy] > 0) nb[n_nb++] = l[s - sy];
                if (z > 0 && l[s - sz] > 0) nb[n_nb++] = l[s - sz];
                if (n_nb == 0) {                /* rule 1 */
                    l_max += 1;
                    rc = table_push(&t, l_max, s);
                    if (rc != HKO_OK) break;
                    l[s] = l_max;
                } else if (n_nb == 1) {         /* rule 2 */
                    l[s] = nb[0];
                } else {                        /* rule 3 */
                    int32_t m = nb[0];
                    for (int i = 1; i < n_nb; ++i) if (nb[i] < m) m = nb[i];
                    l[s] = m;
                    for (int i = 0; i < n_nb; ++i)
                        for (int j = i + 1; j < n_nb; ++j)
                            store_equivalence(t.lol, nb[i], nb[j]);
                }
            }
        }
    }
    if (rc != HKO_OK) { free(t.lol); free(t.first); return rc; }

    /* Periodic edges: the pair (n_a - 1, 0) along every periodic axis. */
    if (periodic[0] && nx >= 2)
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y) {
                int64_t a = (nx - 1) * sx + y * sy + z * sz, b = y * sy + z * sz;
                if (l[a] > 0 && l[b] > 0) store_equivalence(t.lol, l[a], l[b]);
            }
    if (periodic[1] && ny >= 2)
        for (int z = 0; z < nz; ++z)
            for (int x = 0; x < nx; ++x) {
                int64_t a = x * sx + (ny - 1) * sy + z * sz, b = x * sx + z * sz;
                if (l[a] > 0 && l[b] > 0) store_equivalence(t.lol, l[a], l[b]);
            }
    if (periodic[2] && nz >= 2)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int64_t a = x * sx + y * sy + (nz - 1) * sz, b = x * sx + y * sy;
                if (l[a] > 0 && l[b] > 0) store_equivalence(t.lol, l[a], l[b]);
            }

    /* Reduce every id to the lowest id of its class, then compactify: the
     * classes get 1..n in increasing order of that lowest id. */
    int32_t *compact = (int32_t *)malloc((size_t)(l_max + 1) * sizeof(int32_t));
    int64_t *count = (int64_t *)calloc((size_t)l_max + 1, sizeof(int64_t));
    if (!compact || !count) { free(compact); free(count); free(t.lol); free(t.first); return HKO_ERR_NOMEM; }
    for (int32_t k = 1; k <= l_max; ++k) t.lol[k] = list_end(t.lol, k);
    int32_t n = 0;
    for (int32_t k = 1; k <= l_max; ++k) compact[k] = (t.lol[k] == k) ? ++n : compact[t.lol[k]];

    /* Final pass over the lattice: apply the equivalences and count sites. */
    for (int64_t s = 0; s < N; ++s) {
        if (l[s] > 0) {
            int32_t root = t.lol[l[s]];
            count[compact[root]] += 1;
            l[s] = (int32_t)t.first[root];
        } else {
            l[s] = -1;
        }
    }

    memset(hist_out, 0, 32 * sizeof(int64_t));
    for (int32_t c = 1; c <= n; ++c) {
        int64_t size = count[c];
        int b = 0;
        while (((int64_t)2 << b) <= size) ++b;   /* floor(log2(size)) */
        hist_out[b] += 1;
        if (c - 1 < sizes_cap) sizes_out[c - 1] = size;
    }
    *n_clusters_out = n;

    free(compact); free(count); free(t.lol); free(t.first);
    return (n > sizes_cap) ? HKO_ERR_CAPACITY : HKO_OK;
}

int hk_oracle_interior(const float *index, int nx, int ny, int nz, const int periodic[3],
                       int32_t *labels_out, int64_t *sizes_out, int64_t sizes_cap,
                       int64_t *hist_out, int64_t *n_clusters_out, int8_t *inside_out) {
    if (!index || !periodic || !labels_out || !hist_out || !n_clusters_out) return HKO_ERR_ARG;
    if (nx < 1 || ny < 1 || nz < 1 || sizes_cap < 0) return HKO_ERR_ARG;
    if (sizes_cap > 0 && (!sizes_out || !inside_out)) return HKO_ERR_ARG;
    const int64_t N = (int64_t)nx * ny * nz;
    if (N >= ((int64_t)1 << 31)) return HKO_ERR_TOO_LARGE;

    /* Step 4: the far sites (I < -0.5) are the occupied sites of the labelling. */
    float *far = (float *)malloc((size_t)N * sizeof(float));
    if (!far) return HKO_ERR_NOMEM;
    for (int64_t s = 0; s < N; ++s) far[s] = (index[s] < -0.5f) ? 1.0f : -1.0f;
    int rc = hk_oracle_label(far, nx, ny, nz, periodic, labels_out, sizes_out, sizes_cap, hist_out,
                             n_clusters_out);
    free(far);
    if (rc != HKO_OK && rc != HKO_ERR_CAPACITY) return rc;
    const int64_t n = *n_clusters_out;

    /* Compacted id of every cluster, from its label (the cluster's first site):
     * labels are ordered like the compacted ids. */
    int32_t *rank = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    int64_t *votes = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    if (!rank || !votes) { free(rank); free(votes); return HKO_ERR_NOMEM; }
    int32_t next = 0;
    for (int64_t s = 0; s < N; ++s) if (labels_out[s] == s) rank[s] = next++;

    /* Step 5: each (cluster site, near site) face pair votes with the sign of I
     * at the near site. */
    const int dims[3] = {nx, ny, nz};
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const int64_t s = x + (int64_t)nx * (y + (int64_t)ny * z);
                if (labels_out[s] >= 0) continue;          /* a cluster site, not a near site */
                const float v = index[s];
                const int sign = (v < 0.0f) ? -1 : (v > 0.0f) ? 1 : 0;
                if (sign == 0) continue;
                for (int axis = 0; axis < 3; ++axis)
                    for (int d = -1; d <= 1; d += 2) {
                        int c[3] = {x, y, z};
                        c[axis] += d;
                        if (c[axis] < 0 || c[axis] >= dims[axis]) {
                            if (!periodic[axis]) continue;
                            c[axis] = (c[axis] + dims[axis]) % dims[axis];
                        }
                        const int64_t m = c[0] + (int64_t)nx * (c[1] + (int64_t)ny * c[2]);
                        if (labels_out[m] >= 0) votes[rank[labels_out[m]]] += sign;
                    }
            }
    for (int64_t k = 0; k < n && k < sizes_cap; ++k)
        inside_out[k] = (int8_t)(votes[k] < 0 ? 1 : votes[k] > 0 ? 0 : -1);
    free(rank);
    free(votes);
    return rc;
}

int hk_oracle_rc_histogram(const int64_t *sizes, int64_t n, const double *edges, int n_edges,
                           int64_t *hist_out, double *rc_sum_out) {
    if ((n > 0 && !sizes) || !edges || n_edges < 1 || !hist_out || n < 0) return HKO_ERR_ARG;
    for (int b = 1; b < n_edges; ++b) if (!(edges[b - 1] < edges[b])) return HKO_ERR_ARG;
    const double four_thirds_pi = 4.0 * 3.14159265358979323846 / 3.0;
    for (int b = 0; b <= n_edges; ++b) hist_out[b] = 0;
    double rc_sum = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        const double V = (double)sizes[k];
        int bin = 0;                                   /* number of edges with R_c >= e */
        for (int b = 0; b < n_edges; ++b) {
            const double e = edges[b];
            if (V >= ((e * e) * e) * four_thirds_pi) bin = b + 1;
        }
        hist_out[bin] += 1;
        rc_sum += cbrt(V / four_thirds_pi);
    }
    if (rc_sum_out) *rc_sum_out = rc_sum;
    return HKO_OK;
}

/* Side of a near site named by its proximity value (Sec. 6, step 2). */
static int8_t near_side(float v) { return (int8_t)(v < 0.0f ? 1 : 0); }

int hk_oracle_interior_state(const float *index, int nx, int ny, int nz, const int periodic[3],
                             int8_t *state_out) {
    if (!index || !periodic || !state_out) return HKO_ERR_ARG;
    if (nx < 1 || ny < 1 || nz < 1) return HKO_ERR_ARG;
    const int64_t N = (int64_t)nx * ny * nz;
    if (N >= ((int64_t)1 << 31)) return HKO_ERR_TOO_LARGE;
    const int64_t cap = (N + 1) / 2;                 /* always enough clusters */
    int32_t *labels = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    int64_t *sizes = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
    int8_t *inside = (int8_t *)malloc((size_t)cap);
    int32_t *rank = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    int64_t hist[32], n = 0;
    int rc = HKO_ERR_NOMEM;
    if (labels && sizes && inside && rank) {
        rc = hk_oracle_interior(index, nx, ny, nz, periodic, labels, sizes, cap, hist, &n, inside);
        if (rc == HKO_OK) {
            int32_t next = 0;
            for (int64_t s = 0; s < N; ++s) if (labels[s] == s) rank[s] = next++;
            for (int64_t s = 0; s < N; ++s)
                state_out[s] = (index[s] < -0.5f) ? inside[rank[labels[s]]] : near_side(index[s]);
        }
    }
    free(labels); free(sizes); free(inside); free(rank);
    return rc;
}

int hk_oracle_interior_update(const int8_t *state_prev, const float *index, int64_t n, int8_t *state_out) {
    if (n < 0 || (n > 0 && (!state_prev || !index || !state_out))) return HKO_ERR_ARG;
    for (int64_t s = 0; s < n; ++s)
        state_out[s] = (index[s] < -0.5f) ? state_prev[s] : near_side(index[s]);
    return HKO_OK;
}

/* ---------------------------------------------------------------------------
 * The parallel scheme of Sec. 3 on host threads (see the header).
 * ------------------------------------------------------------------------- */
typedef struct {
    int z0, z1;              /* the domain's planes */
    label_table t;           /* its label-of-labels list and first sites (global indices) */
    int32_t l_max;
    int64_t *size;           /* [l_max + 1] sites of each local root */
    int64_t *pairs;          /* equivalences across the face to the next domain, 2 global ids each */
    int64_t npairs, cap;
    int32_t *out;            /* [l_max + 1] final label of each local root (from the root) */
    int rc;
} mt_domain;

typedef struct {
    const float *phi;
    int nx, ny, nz, P;
    const int *periodic;
    int32_t *l;
    mt_domain *d;
    pthread_barrier_t bar;
    pthread_mutex_t gate_mu;   /* workers start once every thread exists (go), or leave (!ok) */
    pthread_cond_t gate_cv;
    int go, ok;
    int64_t *sizes_out, sizes_cap, *hist_out, n;
    int rc;
} mt_job;

typedef struct {
    mt_job *job;
    int w;
} mt_arg;

static int mt_push_pair(mt_domain *D, int64_t a, int64_t b) {
    if (D->npairs == D->cap) {
        int64_t nc = D->cap ? 2 * D->cap : 1024;
        int64_t *np = (int64_t *)realloc(D->pairs, (size_t)nc * 2 * sizeof(int64_t));
        if (!np) return HKO_ERR_NOMEM;
        D->pairs = np;
        D->cap = nc;
    }
    D->pairs[2 * D->npairs] = a;
    D->pairs[2 * D->npairs + 1] = b;
    D->npairs += 1;
    return HKO_OK;
}

/* Step 1: the serial algorithm on the planes z0 .. z1 - 1; afterwards every
 * occupied site holds its local root id and size[] counts the sites of each. */
static int mt_local(mt_job *J, mt_domain *D) {
    const int nx = J->nx, ny = J->ny;
    const int64_t sx = 1, sy = nx, sz = (int64_t)nx * ny;
    int32_t *l = J->l;
    for (int64_t s = D->z0 * sz; s < D->z1 * sz; ++s) l[s] = (J->phi[s] > 0.0f) ? -1 : 0;
    for (int z = D->z0; z < D->z1; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const int64_t s = x * sx + y * sy + z * sz;
                if (l[s] != -1) continue;
                int32_t nb[3];
                int n_nb = 0;
                if (x > 0 && l[s - sx] > 0) nb[n_nb++] = l[s - sx];
                if (y > 0 && l[s - sy] > 0) nb[n_nb++] = l[s - sy];
                if (z > D->z0 && l[s - sz] > 0) nb[n_nb++] = l[s - sz];   /* not across the domain face */
                if (n_nb == 0) {
                    D->l_max += 1;
                    if (table_push(&D->t, D->l_max, s) != HKO_OK) return HKO_ERR_NOMEM;
                    l[s] = D->l_max;
                } else {
                    int32_t m = nb[0];
                    for (int i = 1; i < n_nb; ++i) if (nb[i] < m) m = nb[i];
                    l[s] = m;
                    for (int i = 0; i < n_nb; ++i)
                        for (int j = i + 1; j < n_nb; ++j) store_equivalence(D->t.lol, nb[i], nb[j]);
                }
            }
    /* the periodic edges inside the domain: x and y always, z when one domain holds all planes */
    for (int z = D->z0; z < D->z1; ++z) {
        if (J->periodic[0] && nx >= 2)
            for (int y = 0; y < ny; ++y) {
                const int64_t a = (nx - 1) * sx + y * sy + z * sz, b = y * sy + z * sz;
                if (l[a] > 0 && l[b] > 0) store_equivalence(D->t.lol, l[a], l[b]);
            }
        if (J->periodic[1] && ny >= 2)
            for (int x = 0; x < nx; ++x) {
                const int64_t a = x * sx + (ny - 1) * sy + z * sz, b = x * sx + z * sz;
                if (l[a] > 0 && l[b] > 0) store_equivalence(D->t.lol, l[a], l[b]);
            }
    }
    if (J->P == 1 && J->periodic[2] && J->nz >= 2)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const int64_t a = x * sx + y * sy + (J->nz - 1) * sz, b = x * sx + y * sy;
                if (l[a] > 0 && l[b] > 0) store_equivalence(D->t.lol, l[a], l[b]);
            }
    D->size = (int64_t *)calloc((size_t)D->l_max + 1, sizeof(int64_t));
    if (!D->size) return HKO_ERR_NOMEM;
    for (int32_t k = 1; k <= D->l_max; ++k) D->t.lol[k] = list_end(D->t.lol, k);
    for (int64_t s = D->z0 * sz; s < D->z1 * sz; ++s)
        if (l[s] > 0) {
            l[s] = D->t.lol[l[s]];
            D->size[l[s]] += 1;
        }
    return HKO_OK;
}

static int64_t mt_find(int64_t *parent, int64_t x) {
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];
        x = parent[x];
    }
    return x;
}

/* Step 4 at the root: resolve the gathered equivalences over all local roots. */
static int mt_resolve(mt_job *J, int64_t n_max) {
    const int P = J->P;
    int64_t *off = (int64_t *)malloc((size_t)(P + 1) * sizeof(int64_t));
    if (!off) return HKO_ERR_NOMEM;
    off[0] = 0;
    for (int w = 0; w < P; ++w) off[w + 1] = off[w] + J->d[w].l_max;
    const int64_t T = off[P];
    int64_t *parent = (int64_t *)malloc((size_t)(T > 0 ? T : 1) * sizeof(int64_t));
    int64_t *minsite = (int64_t *)malloc((size_t)(T > 0 ? T : 1) * sizeof(int64_t));
    int64_t *csize = (int64_t *)calloc((size_t)(T > 0 ? T : 1), sizeof(int64_t));
    int rc = (parent && minsite && csize) ? HKO_OK : HKO_ERR_NOMEM;
    if (rc == HKO_OK) {
        for (int64_t i = 0; i < T; ++i) { parent[i] = i; minsite[i] = INT64_MAX; }
        /* a global id g = w * n_max + k (Eq. 1) is local root k of domain w */
        for (int w = 0; w < P; ++w)
            for (int64_t e = 0; e < J->d[w].npairs; ++e) {
                const int64_t ga = J->d[w].pairs[2 * e], gb = J->d[w].pairs[2 * e + 1];
                const int64_t wa = (ga - 1) / n_max, wb = (gb - 1) / n_max;
                const int64_t a = mt_find(parent, off[wa] + (ga - wa * n_max) - 1);
                const int64_t b = mt_find(parent, off[wb] + (gb - wb * n_max) - 1);
                if (a < b) parent[b] = a;
                else if (b < a) parent[a] = b;
            }
        for (int w = 0; w < P; ++w)
            for (int32_t k = 1; k <= J->d[w].l_max; ++k) {
                if (J->d[w].size[k] == 0) continue;                 /* not a local root */
                const int64_t r = mt_find(parent, off[w] + k - 1);
                if (J->d[w].t.first[k] < minsite[r]) minsite[r] = J->d[w].t.first[k];
                csize[r] += J->d[w].size[k];
            }
        /* compactified order: domains in z order and each domain's local roots in
         * creation (raster) order visit first sites in increasing order; a class is
         * counted at the local root that holds its smallest site */
        int64_t n = 0;
        for (int b = 0; b < 32; ++b) J->hist_out[b] = 0;
        for (int w = 0; w < P; ++w)
            for (int32_t k = 1; k <= J->d[w].l_max; ++k) {
                if (J->d[w].size[k] == 0) continue;
                const int64_t r = mt_find(parent, off[w] + k - 1);
                if (minsite[r] != J->d[w].t.first[k]) continue;
                int b = 0;
                while (((int64_t)2 << b) <= csize[r]) ++b;
                J->hist_out[b] += 1;
                if (n < J->sizes_cap) J->sizes_out[n] = csize[r];
                ++n;
            }
        J->n = n;
        /* scatter: the final label of every local root */
        for (int w = 0; w < P && rc == HKO_OK; ++w) {
            mt_domain *D = &J->d[w];
            D->out = (int32_t *)malloc((size_t)(D->l_max + 1) * sizeof(int32_t));
            if (!D->out) { rc = HKO_ERR_NOMEM; break; }
            for (int32_t k = 1; k <= D->l_max; ++k)
                D->out[k] = D->size[k] ? (int32_t)minsite[mt_find(parent, off[w] + k - 1)] : -1;
        }
    }
    free(off); free(parent); free(minsite); free(csize);
    return rc;
}

static void *mt_worker(void *p) {
    mt_arg *a = (mt_arg *)p;
    mt_job *J = a->job;
    const int w = a->w;
    mt_domain *D = &J->d[w];
    const int64_t sy = J->nx, sz = (int64_t)J->nx * J->ny;
    pthread_mutex_lock(&J->gate_mu);
    while (!J->go) pthread_cond_wait(&J->gate_cv, &J->gate_mu);
    const int ok = J->ok;
    pthread_mutex_unlock(&J->gate_mu);
    if (!ok) return NULL;
    D->rc = mt_local(J, D);
    pthread_barrier_wait(&J->bar);
    /* steps 2-3: Eq. 1's offsets and the equivalences across the face to the next domain */
    int64_t n_max = 1;
    for (int v = 0; v < J->P; ++v) if (J->d[v].l_max > n_max) n_max = J->d[v].l_max;
    const int next = (w + 1 < J->P) ? w + 1 : ((J->periodic[2] && J->nz >= 2 && J->P >= 2) ? 0 : -1);
    if (D->rc == HKO_OK && next >= 0) {
        const int zt = D->z1 - 1, zb = J->d[next].z0;
        for (int y = 0; y < J->ny && D->rc == HKO_OK; ++y)
            for (int x = 0; x < J->nx; ++x) {
                const int32_t la = J->l[x + y * sy + zt * sz], lb = J->l[x + y * sy + zb * sz];
                if (la > 0 && lb > 0) {
                    D->rc = mt_push_pair(D, w * n_max + la, next * n_max + lb);
                    if (D->rc != HKO_OK) break;
                }
            }
    }
    pthread_barrier_wait(&J->bar);
    if (w == 0) {                                          /* step 4: gather at the root */
        J->rc = HKO_OK;
        for (int v = 0; v < J->P; ++v) if (J->d[v].rc != HKO_OK) J->rc = J->d[v].rc;
        if (J->rc == HKO_OK) J->rc = mt_resolve(J, n_max);
    }
    pthread_barrier_wait(&J->bar);
    if (J->rc == HKO_OK)                                   /* step 5: relabel */
        for (int64_t s = D->z0 * sz; s < D->z1 * sz; ++s) J->l[s] = J->l[s] > 0 ? D->out[J->l[s]] : -1;
    return NULL;
}

int hk_oracle_mt_label(const float *phi, int nx, int ny, int nz, const int periodic[3], int threads,
                       int32_t *labels_out, int64_t *sizes_out, int64_t sizes_cap,
                       int64_t *hist_out, int64_t *n_clusters_out) {
    if (!phi || !periodic || !labels_out || !hist_out || !n_clusters_out || threads < 1) return HKO_ERR_ARG;
    if (nx < 1 || ny < 1 || nz < 1 || sizes_cap < 0) return HKO_ERR_ARG;
    if (sizes_cap > 0 && !sizes_out) return HKO_ERR_ARG;
    if ((int64_t)nx * ny * nz >= ((int64_t)1 << 31)) return HKO_ERR_TOO_LARGE;
    const int P = threads < nz ? threads : nz;
    mt_job J;
    memset(&J, 0, sizeof(J));
    J.phi = phi; J.nx = nx; J.ny = ny; J.nz = nz; J.P = P; J.periodic = periodic; J.l = labels_out;
    J.sizes_out = sizes_out; J.sizes_cap = sizes_cap; J.hist_out = hist_out;
    J.d = (mt_domain *)calloc((size_t)P, sizeof(mt_domain));
    pthread_t *th = (pthread_t *)malloc((size_t)P * sizeof(pthread_t));
    mt_arg *args = (mt_arg *)malloc((size_t)P * sizeof(mt_arg));
    if (!J.d || !th || !args || pthread_barrier_init(&J.bar, NULL, (unsigned)P) != 0) {
        free(J.d); free(th); free(args);
        return HKO_ERR_NOMEM;
    }
    pthread_mutex_init(&J.gate_mu, NULL);
    pthread_cond_init(&J.gate_cv, NULL);
    for (int w = 0; w < P; ++w) {
        J.d[w].z0 = (int)((int64_t)w * nz / P);
        J.d[w].z1 = (int)((int64_t)(w + 1) * nz / P);
        args[w].job = &J;
        args[w].w = w;
    }
    int started = 1;
    while (started < P && pthread_create(&th[started], NULL, mt_worker, &args[started]) == 0) ++started;
    /* open the gate: with every thread running they all take part; otherwise the ones
     * that started leave before any barrier */
    pthread_mutex_lock(&J.gate_mu);
    J.go = 1;
    J.ok = started == P;
    pthread_cond_broadcast(&J.gate_cv);
    pthread_mutex_unlock(&J.gate_mu);
    int rc = HKO_ERR_NOMEM;
    if (J.ok) {
        mt_worker(&args[0]);
        rc = J.rc;
    }
    for (int w = 1; w < started; ++w) pthread_join(th[w], NULL);
    pthread_cond_destroy(&J.gate_cv);
    pthread_mutex_destroy(&J.gate_mu);
    if (rc == HKO_OK) *n_clusters_out = J.n;
    pthread_barrier_destroy(&J.bar);
    for (int w = 0; w < P; ++w) {
        free(J.d[w].t.lol); free(J.d[w].t.first); free(J.d[w].size); free(J.d[w].pairs); free(J.d[w].out);
    }
    free(J.d); free(th); free(args);
    if (rc != HKO_OK) return rc;
    return J.n > sizes_cap ? HKO_ERR_CAPACITY : HKO_OK;
}
