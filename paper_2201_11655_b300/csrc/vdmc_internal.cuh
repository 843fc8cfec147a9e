// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>

#include "vdmc.h"

#define VDMC_MAX_CLASSES 199

// One unit of enumeration work: root rank r, and the slice of its depth-1
// neighbours it owns: positions j, j + stride, j + 2*stride, ... of N+(r).
// (The paper computes each (vertex, neighbour) pair separately on the GPU,
// "Vertex ordering and splitting over the GPU"; a slice groups such pairs.)
struct Task {
    int32_t r;
    int32_t j;
    int32_t stride;
    int32_t g;       // graph index inside a batch launch
};

// Read-only view of one graph's device CSR plus the output it writes.
struct GraphDesc {
    const int64_t *rowptr;   // [n+1]
    const uint32_t *col;     // [2E_U]  (rank << 2) | flags
    const int64_t *pbeg;     // [n]  first entry of row r with rank > r
    const int32_t *new2old;  // [n]
    uint64_t *out;           // [n * C_k], original-id rows
    int32_t n;
    int32_t pad;
    int64_t nnz;             // entries of col
};

struct vdmc_graph {
    int device;
    int32_t n;
    int64_t nnz;             // 2 * E_U
    int64_t *rowptr;
    uint32_t *col;
    int64_t *pbeg;
    int32_t *new2old;
    int32_t *old2new;
    Task *tasks;
    int64_t ntasks;
    int32_t tasks_a_chunk;
    unsigned long long *qhead;   // work-queue cursor
    int *status;                 // device status word
    vdmc_graph_info_t info;
    // root-per-CTA kernel (hub.cu)
    int32_t *hubs;               // ranks of the roots it handles, heavy first
    int32_t nhubs;
    int32_t hub_min_l;
    int64_t hub_lmax, hub_hcap, hub_tcap, hub_npcap;
    int hub_slots;
    void *hub_scratch;
    size_t hub_scratch_bytes;
    unsigned long long *hub_qhead;
    void *hub_split_buf;         // split roots: nsplit * (C_k partial sums + a ticket)
    int32_t hub_split_cap;
    cudaStream_t side;           // second stream: the two kernels overlap; also frees the graph
    cudaEvent_t ev_fork, ev_join;
    cudaEvent_t ev_done;         // recorded after the graph's last build or count step
    uint64_t serial;             // creation number (identifies the graph in cached batch plans)
    int32_t num_graphs;          // > 1 for a graph built by vdmc_graph_create_batch
    void *batch_plan;            // cached plan of vdmc_count_batch calls led by this graph
    uint64_t *racc;              // rank-space credit accumulator, n * VDMC_MAX_CLASSES
    uint64_t *d3acc;             // k = 4 depth-3 credits of the root-per-CTA kernel, n * VDMC_D3_COLS (rank space)
    uint64_t *d3w;               // k = 4 per-vertex type counts spread to the neighbours' depth-3 credits, n * 9
    int d3_mode;                 // 0 unknown, 1: 32-bit depth-3 credits suffice (d3_bound), 2: 64-bit
    unsigned long long *stats;   // VDMC_NSTATS counters of the last count (vdmc_count_stats)
    int undirected;              // VDMC_GRAPH_UNDIRECTED: every edge carries flags 3, output in undirected classes
    // per-edge counts (vdmc_count_edges), built on first use
    int64_t *ebase;              // n + 1: the edges of rank r's upper row have ids ebase[r] .. ebase[r+1]-1
    int64_t *erow;               // edge id -> output row (edges in (min, max) original-id order)
    uint64_t *ekeys;             // output row -> (min original id << 30) | max original id
    uint8_t *eflags;             // output row -> bit 0: arc min -> max, bit 1: arc max -> min
    Task *etasks;                // every root, for the per-edge kernel
    int64_t netasks;
    int32_t etasks_a_chunk;
};

// Counters of one count, reset at its start (vdmc_count_stats_t):
//   [0] sets the warp-per-task kernel enumerated one by one
//   [1] sets rooted at roots of the root-per-CTA kernel (all of its sets)
//   [2] of those, sets that kernel visited one at a time (the rest are
//       accounted for by signature formulas)
constexpr int VDMC_NSTATS = 4;

// Depth-3 credit columns per vertex (k = 4, root-per-CTA kernel): the paths
// r - x - b - c credited to c are typed by (colour of x, h(x, b), h(b, c)),
// 27 types in 15 classes (a path and its reverse are isomorphic); one column
// per class, 16 columns = one 128-byte line per vertex.
constexpr int VDMC_D3_COLS = 16;
// hub_warps = 0: 32-warp root-per-CTA CTAs when the largest hub root has at
// least this many higher-rank neighbours (measured: 32 warps faster from ~830,
// slower at ~500 and below)
constexpr int64_t VDMC_HUB_WARPS32_MIN_L = 640;

// ---- device memory ----
// Graph-owned device memory is stream-ordered (cudaMallocAsync on the stream
// of the call that needs it, cudaFreeAsync when the graph is destroyed), so
// creating, counting or destroying one graph never waits for the work of
// other graphs on other streams.
inline cudaError_t vdmc_malloc(void **p, size_t bytes, cudaStream_t s) {
    return cudaMallocAsync(p, bytes ? bytes : 1, s);
}
template <typename T>
inline cudaError_t vdmc_malloc(T **p, size_t bytes, cudaStream_t s) {
    return vdmc_malloc(reinterpret_cast<void **>(p), bytes, s);
}
inline void vdmc_free(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

// ---- status helpers ----
#define VDMC_CUDA_TRY(expr)                                         \
    do {                                                            \
        cudaError_t _e = (expr);                                    \
        if (_e != cudaSuccess) {                                    \
            return (_e == cudaErrorMemoryAllocation) ? VDMC_ERR_OOM \
                                                     : VDMC_ERR_CUDA; \
        }                                                           \
    } while (0)

// ---- primitives (sort_scan.cu) ----
// Exclusive prefix sum in place-or-not: out[i] = sum_{j<i} in[i]; out[count] = total
// when `out` has count+1 slots (total_slot != 0).  Temporary storage comes
// from the stream-ordered allocator.
cudaError_t vdmc_exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t count, cudaStream_t s);
cudaError_t vdmc_exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t count, cudaStream_t s);
// LSD radix sort of 64-bit keys on bits [begin_bit, end_bit); the other bits
// ride along.  Stable.  On return *result points at whichever of keys / tmp
// holds the sorted keys.
cudaError_t vdmc_radix_sort_u64(uint64_t *keys, uint64_t *tmp, int64_t count, int begin_bit,
                                int end_bit, cudaStream_t s, uint64_t **result);

// ---- classes (classes.cpp) ----
// lut[mask] = output column of the motif with index `mask`, 255 if the
// induced graph is not weakly connected.  Built once per k, host memory.
const uint8_t *vdmc_host_lut(int k);
const uint16_t *vdmc_host_canon(int k, int *num_classes);
// undirected variant: column of each directed class among the symmetric ones
// (255 = not symmetric), and their number (2 for k = 3, 6 for k = 4)
const uint8_t *vdmc_host_ucol(int k, int *num_undirected);
// column of each class in the counting kernels' accumulator, and the class of
// each accumulator column (classes.cpp: accumulator_order)
const uint8_t *vdmc_host_acc_col(int k);
const uint8_t *vdmc_host_acc_class(int k);

// ---- counting (count.cu) ----
vdmc_status vdmc_count_internal(vdmc_graph *g, int k, int32_t lo, int32_t hi, uint64_t *out, cudaStream_t s);
// device copies (per device, built once): lut maps a motif index to its
// ACCUMULATOR column (255 = not weakly connected); colmap maps an
// accumulator column to an output column (directed classes, or undirected
// columns with 255 where a class is not symmetric)
cudaError_t vdmc_device_lut(int k, const uint8_t **out);
cudaError_t vdmc_device_colmap(int k, bool undirected, const uint8_t **out);

// ---- per-edge counts (edges.cu) ----
// builds g->ebase, g->erow, g->ekeys, g->eflags on first use (on stream s)
vdmc_status vdmc_edge_index(vdmc_graph *g, cudaStream_t s);

// ---- graph build (graph_build.cu) ----
vdmc_status vdmc_graph_create_grouped(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                                      int ptrs_on_device, void *stream, vdmc_graph **out, const int64_t *goff,
                                      int32_t ngroups, uint32_t options);

// ---- batch plans (batch.cu) ----
void vdmc_batch_plan_free(vdmc_graph *g);
uint64_t vdmc_next_serial();
vdmc_status vdmc_graph_init_streams(vdmc_graph *g);

// ---- schedule / tasks (count.cu) ----
vdmc_status vdmc_build_tasks(vdmc_graph *g, int32_t a_chunk, int32_t hub_min_l, cudaStream_t s);
void vdmc_current_schedule(vdmc_schedule_t *s);

// ---- root-per-CTA kernel (hub.cu) ----
vdmc_status vdmc_build_hubs(vdmc_graph *g, int32_t min_l, cudaStream_t s);
vdmc_status vdmc_hub_launch(vdmc_graph *g, int k, uint64_t *out, uint64_t *d3, int d3_narrow, uint64_t *d3w,
                            const uint8_t *lut,
                            int32_t lo, int32_t hi, int blocks_per_sm, int split, int split_roots, int warps,
                            cudaStream_t s);
void vdmc_hub_free(vdmc_graph *g, cudaStream_t s);
