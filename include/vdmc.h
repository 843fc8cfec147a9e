/*
 * vdmc.h -- C ABI of the B300 (sm_103a) per-vertex directed motif counter.
 *
 * The operation (VDMC, arXiv 2201.11655):
 *   For a directed, unweighted, simple graph G = (V, E) (Definitions) and
 *   k in {3, 4}, X_{k,m}(i) is the number of vertex sets S with |S| = k and
 *   i in S such that S is connected in the underlying undirected graph G_U
 *   and the directed sub-graph induced by S is of motif class m (the
 *   definition of X_{k,m}(i) in "Comparison to theory in G(n,p)"; the motif
 *   index of Fig. 1: the k x k adjacency matrix read row-major with the
 *   diagonal removed, most significant bit first; a class is named by the
 *   minimum index over its isomorphs, per the isomorph-merge paragraph of
 *   "The Algorithm").
 *
 *   Output columns are the connected classes in ascending order of their
 *   minimum index: C_3 = 13 columns, C_4 = 199 columns
 *   (vdmc_class_masks() returns that list).
 *
 * Conventions for every call:
 *   - Vertex ids are int32 in [0, n).  Self-loops are ignored and repeated
 *     arcs collapsed (the paper assumes a simple graph); both are counted in
 *     vdmc_graph_info_t.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous on it unless documented otherwise.
 *   - Errors detected on the host are returned at once.  Errors detected in a
 *     kernel are written to the graph's device status word; read it with
 *     vdmc_get_device_status() after synchronising the stream.
 *   - The library never calls exit(), never traps on the device and never
 *     spins on a device flag.
 *   - A graph's device memory comes from the device's default stream-ordered
 *     memory pool (cudaMallocAsync); on the first graph built on a device
 *     the library lets that pool keep up to 16 GiB of freed memory for reuse
 *     (its release threshold), so repeated builds do not map memory afresh.
 *   - All counts are exact uint64; no floating point is used anywhere.
 */
#ifndef VDMC_H
#define VDMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VDMC_OK = 0,
    VDMC_ERR_INVALID_ARG = 1,          /* bad k, NULL pointer, negative size, n >= 2^30 */
    VDMC_ERR_OUT_OF_RANGE_VERTEX = 2,  /* an arc endpoint outside [0, n) */
    VDMC_ERR_OOM = 3,                  /* device allocation failed */
    VDMC_ERR_CUDA = 4,                 /* a CUDA runtime call failed */
    VDMC_ERR_DEVICE_LIMIT = 5,         /* a kernel hit an internal limit (status word) */
    VDMC_ERR_BUSY = 6                  /* a resource is in use by another call */
} vdmc_status;

/* Opaque graph: owns its device CSR (degree-ordered ids, 2-bit arc flags
 * per undirected edge), id maps, task list and work-queue cursor. */
typedef struct vdmc_graph vdmc_graph;

typedef struct {
    int32_t n;                 /* vertices */
    int32_t max_degree;        /* max undirected degree in G_U */
    int64_t arcs_in;           /* arcs passed to vdmc_graph_create */
    int64_t self_loops;        /* dropped */
    int64_t duplicate_arcs;    /* repeated (u,v) collapsed */
    int64_t arcs_kept;         /* distinct directed arcs */
    int64_t edges_u;           /* edges of G_U (a reciprocal pair is one edge) */
    int64_t reciprocal_pairs;  /* edges of G_U carrying arcs both ways */
    int64_t num_tasks;         /* (root, depth-1 slice) work items of the warp kernel */
    int64_t num_hub_roots;     /* roots handled by the root-per-CTA kernel */
    int64_t num_graphs;        /* graphs in the union (vdmc_graph_create_batch), else 1 */
    int64_t device_bytes;      /* bytes held on the device by this graph */
} vdmc_graph_info_t;

/* Launch schedule of the counting kernels.  Results never depend on it. */
typedef struct {
    int32_t a_chunk;            /* warp-per-task kernel: depth-1 neighbours of one
                                   root per task (>= 1); a root with L such
                                   neighbours is split into ceil(L / a_chunk)
                                   interleaved tasks */
    int32_t warps_per_block;    /* warp-per-task kernel: 1..8 */
    int32_t blocks_per_sm;      /* warp-per-task kernel: 0 = as many as fit */
    int32_t hub_min_l;          /* roots with at least this many higher-rank
                                   neighbours go to the root-per-CTA kernel;
                                   0 = every root to the warp-per-task kernel */
    int32_t hub_blocks_per_sm;  /* root-per-CTA kernel: CTAs per SM (>= 1); each
                                   owns a scratch slot of about 4n + 52 tcap bytes */
    int32_t hub_split;          /* root-per-CTA kernel: the largest roots are
                                   each counted by this many CTAs (0..16; 0 or 1 =
                                   no split); every part builds the root's lists and
                                   takes a share of its members and second-hop
                                   vertices */
    int32_t hub_split_roots;    /* how many of the largest roots are split (>= 0) */
    int32_t hub_warps;          /* root-per-CTA kernel: warps per CTA, 16 or 32;
                                   0 (the default) = 32 when the graph's largest
                                   hub root has at least 640 higher-rank
                                   neighbours, else 16 */
    int32_t d3_bits;            /* root-per-CTA kernel, k = 4: width of the depth-3
                                   credit counters; 0 = 32 bits when a per-graph
                                   bound shows that no vertex can reach 2^32 of
                                   them in one count, else 64; 64 = always 64 */
} vdmc_schedule_t;

/*
 * Build a graph from a directed arc list (Definitions; CSR paragraph of
 * "The Algorithm"; degree order of "Vertex ordering and splitting over the
 * GPU").
 *   n                 number of vertices, 0 <= n < 2^30
 *   m                 number of arcs, >= 0
 *   src, dst          int32[m]: arc e is src[e] -> dst[e].  Host pointers
 *                     when ptrs_on_device == 0 (copied before the call
 *                     returns), device pointers otherwise (read on `stream`).
 *                     The caller keeps ownership.
 *   stream            cudaStream_t for the build.
 *   out               receives the new graph.
 * Synchronises `stream` (it reads sizes back to size its buffers).
 * Returns VDMC_ERR_OUT_OF_RANGE_VERTEX if an endpoint is outside [0, n).
 */
vdmc_status vdmc_graph_create(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                              int ptrs_on_device, void *stream, vdmc_graph **out);

/* Options of vdmc_graph_create_ex. */
#define VDMC_GRAPH_UNDIRECTED 1u  /* count the undirected motifs of G_U (arc directions ignored) */

/*
 * vdmc_graph_create with options.  VDMC_GRAPH_UNDIRECTED: the undirected
 * variant (the undirected motifs the paper reports beside the directed ones,
 * Tables 1-2 and Fig. 5): every edge of G_U is taken with arcs both ways, so
 * each connected k-set is classified by its induced undirected graph; counts
 * of such a graph have vdmc_num_classes_undirected(k) columns (2 for k = 3,
 * 6 for k = 4), the connected undirected classes in ascending order of the
 * minimum index of their symmetric adjacency matrix
 * (vdmc_undirected_class_masks).  Unknown option bits return
 * VDMC_ERR_INVALID_ARG.  Otherwise as vdmc_graph_create.
 */
vdmc_status vdmc_graph_create_ex(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                                 int ptrs_on_device, uint32_t options, void *stream, vdmc_graph **out);

/*
 * Build ONE graph from many independent graphs (a batch; no paper
 * counterpart): the disjoint union of graphs 0..num-1.
 *   num        number of graphs, >= 1
 *   ns, ms     host int32[num] vertex counts and int64[num] arc counts
 *   src, dst   the graphs' arc lists concatenated in graph order (arcs of
 *              graph i first, then graph i+1, ...), each in that graph's
 *              LOCAL ids 0..ns[i]-1; host or device pointers as for
 *              vdmc_graph_create
 * Vertex x of graph i becomes vertex voff[i] + x of the union, with
 * voff[i] = ns[0] + ... + ns[i-1]; the union's total vertex count must be
 * < 2^30.  The union's vertex order keeps each graph's vertices in one
 * contiguous block, in that graph's own degree order, so the roots counted
 * at the same time belong to the same graph and their credits stay local.  No k-set of the union spans two graphs (they are not connected),
 * so one vdmc_count on the union counts all graphs in one launch and graph
 * i's counts are rows voff[i] .. voff[i+1]-1 of the output.  A local id
 * outside [0, ns[i]) returns VDMC_ERR_OUT_OF_RANGE_VERTEX.  Synchronises
 * `stream`.
 */
vdmc_status vdmc_graph_create_batch(int32_t num, const int32_t *ns, const int64_t *ms, const int32_t *src,
                                    const int32_t *dst, int ptrs_on_device, void *stream, vdmc_graph **out);

/* Free the graph's device memory.  Stream-ordered: the frees are queued
 * behind the graph's last build or count (on whatever stream it ran), so
 * the call does not wait for the device or for other graphs' work; the
 * caller must not use the graph, or read an output of a count still in
 * flight through it, after this call only via the graph handle (outputs
 * belong to the caller and stay valid).  A graph that led a
 * vdmc_count_batch plan synchronises the device instead. */
vdmc_status vdmc_graph_destroy(vdmc_graph *g);

/* Sizes and drop counters of a built graph (host struct, filled in). */
vdmc_status vdmc_graph_info(const vdmc_graph *g, vdmc_graph_info_t *info);

/*
 * Copy the CSR to host buffers (a test and inspection hook).  Rows are in
 * degree order (rank); entry = (neighbour rank << 2) | flags with flag bit 0
 * = arc row -> neighbour and bit 1 = arc neighbour -> row; rows sorted by
 * neighbour rank.  rowptr: int64[n+1], col: uint32[2*edges_u],
 * new2old: int32[n] (original id of each rank).  Any pointer may be NULL.
 * Synchronous.
 */
vdmc_status vdmc_graph_export_csr(const vdmc_graph *g, int64_t *rowptr, uint32_t *col,
                                  int32_t *new2old);

/* Number of output columns for k: 13 for k = 3, 199 for k = 4, -1 otherwise. */
int vdmc_num_classes(int k);

/* Columns of an undirected graph's counts: 2 for k = 3, 6 for k = 4, -1 otherwise. */
int vdmc_num_classes_undirected(int k);

/* Minimum (symmetric) motif index of each undirected column, ascending
 * (uint16[vdmc_num_classes_undirected(k)]).  Host-side table. */
vdmc_status vdmc_undirected_class_masks(int k, uint16_t *canon_out);

/* Columns of g's counts for k: vdmc_num_classes(k), or
 * vdmc_num_classes_undirected(k) for a graph built with
 * VDMC_GRAPH_UNDIRECTED; -1 for a bad k or graph. */
int vdmc_graph_num_classes(const vdmc_graph *g, int k);

/* Minimum motif index of each output column, ascending (uint16[C_k]).
 * Host-side table; needs no device. */
vdmc_status vdmc_class_masks(int k, uint16_t *canon_out);

/* Output column of every motif index: lut_out[idx] for idx in
 * [0, 2^(k(k-1))), 255 where the indexed graph is not weakly connected
 * (the isomorph merge of "The Algorithm").  Host-side table; needs no
 * device. */
vdmc_status vdmc_class_lut(int k, uint8_t *lut_out);

/*
 * Per-vertex counts (the VDMC algorithm of "The Algorithm"; proper k-BFS of
 * Lemma 1; BFS structures of Lemma 2; ordering rules of Lemma 3; the
 * direct-adjacency test of the comment after Lemma 4).
 *   g        graph from vdmc_graph_create (or _ex / _batch)
 *   k        3 or 4
 *   out_dev  device uint64[n * C], C = vdmc_graph_num_classes(g, k) (C_k, or
 *            the undirected columns for a VDMC_GRAPH_UNDIRECTED graph),
 *            row-major by ORIGINAL vertex id; overwritten (not accumulated).
 *            Caller owns it.
 *   stream   cudaStream_t
 * Asynchronous (the first k = 4 count of a graph with hub roots synchronises
 * `stream` once, to size its depth-3 counters).  Calls on one graph must not
 * overlap (they share the graph's work-queue cursor); a call waits, on the
 * device, for the graph's previous call on any stream.
 */
vdmc_status vdmc_count(vdmc_graph *g, int k, uint64_t *out_dev, void *stream);

/*
 * Like vdmc_count, but only the sets whose lowest-rank member has rank in
 * [rank_lo, rank_hi) (Lemma 1: every set has one proper root).  Disjoint
 * ranges covering [0, n) sum to vdmc_count.  This is the unit of the
 * root-chunk distribution of the Discussion.  Overwrites out_dev.
 */
vdmc_status vdmc_count_roots(vdmc_graph *g, int k, int32_t rank_lo, int32_t rank_hi,
                             uint64_t *out_dev, void *stream);

/*
 * Per-edge counts (the edge variant of the Discussion: a motif credits the
 * edges it contains instead of its vertices).  For every edge {u, v} of G_U
 * and class m: the number of connected k-sets containing u and v whose
 * induced motif is of class m (the edges of a set are the edges of G_U with
 * both ends in it).  Rows are the edges {u, v}, u < v in ORIGINAL ids, in
 * ascending (u, v) order -- the order vdmc_graph_edges lists them;
 * columns as for vdmc_count on this graph (vdmc_graph_num_classes).
 *   out_dev  device uint64[edges_u * columns], overwritten.  Caller owns it.
 * Every root is enumerated set by set with the warp-per-task kernel (the
 * root-per-CTA kernel has no per-edge form), so this costs the number of
 * sets, not the neighbourhood volume, on graphs with hubs.  The first call
 * builds an edge index owned by the graph (about 17 bytes per edge).
 * Asynchronous; calls on one graph must not overlap (as vdmc_count).
 */
vdmc_status vdmc_count_edges(vdmc_graph *g, int k, uint64_t *out_dev, void *stream);

/*
 * The rows of vdmc_count_edges: edge i is {u[i], v[i]}, u[i] < v[i] original
 * ids, ascending; flags[i] bit 0 = arc u -> v present, bit 1 = arc v -> u
 * (always 3 for a graph built with VDMC_GRAPH_UNDIRECTED).  Host arrays of
 * edges_u entries; any may be NULL.  Synchronous.
 */
vdmc_status vdmc_graph_edges(vdmc_graph *g, int32_t *u, int32_t *v, uint8_t *flags);

/*
 * Count `num` independent graphs, built one by one, in ONE launch (a batch
 * of uneven small graphs; no paper counterpart).  outs[i] is a device
 * uint64[n_i * C_k] for graphs[i], overwritten.  `graphs` and `outs` are
 * host arrays.  Results equal num separate vdmc_count calls bit for bit.
 * The first call for a given (graphs, outs, k, schedule) concatenates the
 * graphs' CSRs into a plan cached on graphs[0] (allocates; synchronises
 * `stream`), counts and scatters the rows to outs; the second call captures
 * the count and scatter into a CUDA graph and later calls replay it.  Any
 * change of graphs, outs, k or schedule rebuilds the plan.  Plans die with
 * graphs[0]; destroying another member graph makes the plan stale, so build
 * a new list after destroying graphs.  Calls on one plan must not overlap.
 * Directed graphs only (an undirected member returns VDMC_ERR_INVALID_ARG).
 * Destroying graphs[0] synchronises the device (its plan may have been
 * replayed on any stream).
 */
vdmc_status vdmc_count_batch(vdmc_graph *const *graphs, int num, int k, uint64_t *const *outs,
                             void *stream);

/*
 * Allocation-free count (the paper has no counterpart; an integration aid).
 *
 * Some callers cannot allocate device memory at the point where they count:
 * real-time or serving loops that reserved a fixed device-memory budget at
 * start-up (where a cudaMalloc could fail, fragment the pool or stall the
 * device while it synchronises), and host applications whose own allocator
 * owns all device memory, so that a library allocating behind their back
 * would break their accounting.  This entry point calls no cudaMalloc,
 * cudaFree or allocating library routine.  It counts with the warp-per-task
 * kernel of vdmc_count (one task per root, no root-per-CTA kernel) and keeps
 * its scratch -- task list, work-queue cursor, class tables -- in one fixed
 * array of about 4.2 MB that every GPU holds for as long as the library is
 * loaded.
 *
 * Inputs are a degree-ordered CSR in the layout vdmc_graph_export_csr
 * returns, in device memory owned by the caller:
 *   n          vertices, 0 <= n <= 262144 (2^18)
 *   nnz        entries of col (2 * edges), >= 0
 *   rowptr     int64[n+1]; col uint32[nnz] = (neighbour rank << 2) | flags,
 *              rows sorted by neighbour rank
 *   pbeg       int64[n]: first entry of row r whose neighbour rank is > r
 *   new2old    int32[n]: original id of each rank
 *   k          3 or 4
 *   out_dev    uint64[n * C_k], overwritten, rows by original id
 *   status_dev int32 on the device, required: receives the kernel's status
 *              word (0 = ok, VDMC_ERR_DEVICE_LIMIT = an index check failed);
 *              read it after synchronising `stream`
 *   stream     cudaStream_t
 * n above 2^18, k not in {3, 4}, or a NULL pointer (status_dev included)
 * returns VDMC_ERR_INVALID_ARG before any device work.
 *
 * The first call on a device sets the scratch up (looks up its device
 * address and copies the class tables into it, synchronously); make that
 * first call before any stream capture.  That set-up is done once per device
 * for the life of the process: after cudaDeviceReset (or any other teardown
 * of the device's primary context) this entry point must not be called again
 * in the same process.  Every call on a device shares the one scratch array,
 * which keeps the previous call's contents; each call clears its cursor and
 * the status word it is given before counting.  Calls whose work overlaps on
 * the GPU (different streams, or concurrent host threads) race on the array
 * and must be serialised by the caller.  Asynchronous otherwise.
 */
vdmc_status vdmc_count_csr_noalloc(int32_t n, int64_t nnz, const int64_t *rowptr, const uint32_t *col,
                                   const int64_t *pbeg, const int32_t *new2old, int k, uint64_t *out_dev,
                                   int *status_dev, void *stream);

/* After synchronising the last stream used with g: the device status word
 * (VDMC_OK or VDMC_ERR_DEVICE_LIMIT); reading it resets it to VDMC_OK. */
vdmc_status vdmc_get_device_status(vdmc_graph *g);

/*
 * Measurement hook: the algorithmic byte model of one vdmc_count(g, k) (the
 * cost model of the section on efficacy on simulated graphs: work
 * proportional to the neighbourhoods visited).  Per root r with
 * P = N+(r), the adjacency rows the method must stream, 4 bytes per entry:
 * N(r), N(a) for every a in P and, for k = 4, N(b) for every DISTINCT
 * depth-2 vertex b (rank > r, not adjacent to r, adjacent to some a in P);
 * plus the 8 * n * C_k bytes of the output and 4 * n bytes of the id map.
 * `bytes_per_use` counts N(b) once per (a, b) adjacency instead (what an
 * enumeration without reuse of N(b) streams).  Synchronous; runs on the
 * legacy default stream.
 */
typedef struct {
    uint64_t bytes;                   /* the model above (roofline numerator) */
    uint64_t bytes_per_use;           /* N(b) counted once per (a, b) */
    uint64_t entries_root;            /* sum over roots of |N(r)| */
    uint64_t entries_depth1;          /* sum over roots of sum_{a in P} |N(a)| */
    uint64_t entries_depth2;          /* k = 4: sum over roots of sum over distinct b of |N(b)| */
    uint64_t entries_depth2_per_use;  /* k = 4: the same per (a, b) adjacency */
    uint64_t output_bytes;            /* 8 n C_k + 4 n */
} vdmc_work_model_t;

vdmc_status vdmc_work_model(const vdmc_graph *g, int k, vdmc_work_model_t *model);

/* vdmc_work_model(g, k).bytes */
vdmc_status vdmc_work_bytes(const vdmc_graph *g, int k, uint64_t *bytes);

/*
 * Counters of the last count on g (vdmc_count / vdmc_count_roots; read after
 * synchronising its stream).  Every connected k-set is found either one by
 * one (the paper's enumeration, and the rare exceptions the root-per-CTA
 * kernel enumerates) or, for sets rooted at the root-per-CTA kernel's roots,
 * in bulk through a signature formula; the two are reported apart.
 * Synchronous.
 */
typedef struct {
    uint64_t sets_plain;           /* sets the warp-per-task kernel enumerated */
    uint64_t sets_hub;             /* sets rooted at roots of the root-per-CTA kernel */
    uint64_t sets_hub_enumerated;  /* of those, sets visited one at a time */
    uint64_t sets_by_signature;    /* sets_hub - sets_hub_enumerated */
    uint64_t sets_enumerated;      /* sets_plain + sets_hub_enumerated */
} vdmc_count_stats_t;

vdmc_status vdmc_count_stats(const vdmc_graph *g, vdmc_count_stats_t *stats);

/*
 * Estimated work of every root (the unit of the root-chunk distribution of
 * the Discussion: contiguous rank ranges of roots go to different devices,
 * and by Lemma 1 the ranges' counts sum to the full count).  cost_dev is a
 * device uint64[n] indexed by RANK: the adjacency entries the root's count
 * streams (N(r), N(a) for a in N+(r), and for k = 4 N(b) per (a, b) with b at
 * depth 2), plus C(L, k-1) for roots the warp-per-task kernel enumerates
 * under the current schedule.  An estimate for balancing, not a count.
 * Asynchronous on `stream`.
 */
vdmc_status vdmc_root_costs(const vdmc_graph *g, int k, uint64_t *cost_dev, void *stream);

/* Global launch schedule (the autotuner's knobs).  Affects later calls. */
vdmc_status vdmc_set_schedule(const vdmc_schedule_t *s);
vdmc_status vdmc_get_schedule(vdmc_schedule_t *s);

/* Static description of a status code. */
const char *vdmc_status_string(vdmc_status s);

#ifdef __cplusplus
}
#endif

#endif /* VDMC_H */
