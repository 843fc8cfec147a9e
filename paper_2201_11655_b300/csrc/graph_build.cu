// Device graph build: arc list -> degree-ordered undirected CSR with 2-bit
// arc flags per edge.
//
// Paper: G_U is the undirected graph underlying G (Definitions); a
// reciprocal pair is one undirected edge (CSR example of "The Algorithm":
// 0<->2 appears once per endpoint); vertices are indexed by decreasing
// undirected degree, ties arbitrary ("Vertex ordering and splitting over
// the GPU"; here: ties by original id); each row lists its neighbours in
// increasing index order so the neighbours of higher index -- the only ones
// a proper k-BFS may visit (Lemma 1) -- form a suffix of the row.
//
// Steps (all on the device, one stream):
//   1. key per arc = min*n + max with the arc's direction in bits 62..63;
//      self-loops become a sentinel key n*n; endpoints are range-checked.
//   2. radix sort on the low bits; runs of equal keys merge their flags
//      (duplicate arcs collapse, u->v and v->u become one edge with flags 3).
//   3. undirected degree, then ranks: stable radix sort of ids by
//      (max_degree - degree).
//   4. both orientations of every edge in rank space, radix sorted by
//      (row, neighbour) -> rowptr / col; pbeg[r] = first entry above r.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>

#include "vdmc_internal.cuh"

namespace {

constexpr uint64_t LOW_MASK = (1ull << 62) - 1ull;

int bits_for(uint64_t v) {  // bits needed to represent values 0..v
    int b = 0;
    while (b < 64 && (v >> b) != 0) b++;
    return b;
}

__global__ void arc_keys(const int32_t *__restrict__ src, const int32_t *__restrict__ dst, int64_t m,
                         int32_t n, uint64_t *__restrict__ keys, unsigned long long *counters, int *bad) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t self_loop = 0;
    if (e < m) {
        int32_t u = src[e], v = dst[e];
        uint64_t key;
        if (u < 0 || v < 0 || u >= n || v >= n) {
            atomicExch(bad, 1);
            key = (uint64_t)n * (uint64_t)n;
        } else if (u == v) {
            self_loop = 1;
            key = (uint64_t)n * (uint64_t)n;
        } else {
            uint32_t lo = u < v ? u : v, hi = u < v ? v : u;
            uint64_t flag = (u == (int32_t)lo) ? 1ull : 2ull;  // bit0: lo->hi, bit1: hi->lo
            key = ((uint64_t)lo * (uint64_t)n + hi) | (flag << 62);
        }
        keys[e] = key;
    }
    uint32_t b = __ballot_sync(0xffffffffu, self_loop);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(&counters[0], (unsigned long long)__popc(b));
}

// head[i] = 1 if keys[i] starts a run of equal low bits and is not a sentinel
__global__ void run_heads(const uint64_t *__restrict__ keys, int64_t m, uint64_t sentinel, uint32_t *head) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    uint64_t lo = keys[i] & LOW_MASK;
    head[i] = (lo != sentinel && (i == 0 || (keys[i - 1] & LOW_MASK) != lo)) ? 1u : 0u;
}

// For every run head: merge flags of the run, write the unique edge.
// counters[1] = distinct directed arcs, counters[2] = reciprocal pairs.
__global__ void merge_runs(const uint64_t *__restrict__ keys, int64_t m, const uint32_t *__restrict__ pos,
                           const uint32_t *__restrict__ head, uint64_t *__restrict__ uedges,
                           unsigned long long *counters) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t arcs = 0, recip = 0;
    if (i < m && head[i]) {
        uint64_t lo = keys[i] & LOW_MASK;
        uint64_t f = 0;
        for (int64_t j = i; j < m && (keys[j] & LOW_MASK) == lo; j++) f |= keys[j] >> 62;
        uedges[pos[i]] = lo | (f << 62);
        arcs = (f == 3) ? 2 : 1;
        recip = (f == 3);
    }
    // warp-aggregate the two counters
    for (int o = 16; o > 0; o >>= 1) {
        arcs += __shfl_down_sync(0xffffffffu, arcs, o);
        recip += __shfl_down_sync(0xffffffffu, recip, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (arcs) atomicAdd(&counters[1], (unsigned long long)arcs);
        if (recip) atomicAdd(&counters[2], (unsigned long long)recip);
    }
}

__global__ void edge_degrees(const uint64_t *__restrict__ uedges, int64_t eu, int32_t n, int32_t *deg) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= eu) return;
    uint64_t lo = uedges[i] & LOW_MASK;
    atomicAdd(&deg[lo / (uint64_t)n], 1);
    atomicAdd(&deg[lo % (uint64_t)n], 1);
}

__global__ void max_degree(const int32_t *deg, int32_t n, int *out) {
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    int v = i < n ? deg[i] : 0;
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_down_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, v);
}

// Sort key of vertex v: (group, max_degree - degree, id).  Without groups
// (a single graph) the order is the paper's degree order; with groups (a
// batch of graphs) each graph's vertices form one contiguous block of ranks,
// in that graph's own degree order, so roots counted at the same time come
// from the same graph and their credits stay in a small region.
__global__ void rank_keys(const int32_t *deg, int32_t n, const int *dmax, const int64_t *goff, int32_t ngroups,
                          int dbits, uint64_t *keys) {
    int32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    uint64_t grp = 0;
    if (goff) {
        int lo = 0, hi = ngroups;
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (goff[mid] <= v) lo = mid;
            else hi = mid;
        }
        grp = (uint64_t)lo;
    }
    keys[v] = (grp << (32 + dbits)) | ((uint64_t)(uint32_t)(*dmax - deg[v]) << 32) | (uint32_t)v;
}

__global__ void rank_maps(const uint64_t *sorted, int32_t n, const int32_t *deg, int32_t *new2old,
                          int32_t *old2new, int64_t *deg_rank) {
    int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int32_t v = (int32_t)(uint32_t)sorted[r];
    new2old[r] = v;
    old2new[v] = r;
    deg_rank[r] = deg[v];
}

__global__ void oriented_entries(const uint64_t *__restrict__ uedges, int64_t eu, int32_t n,
                                 const int32_t *__restrict__ old2new, uint64_t *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= eu) return;
    uint64_t e = uedges[i];
    uint64_t lo = e & LOW_MASK, f = e >> 62;  // f bit0: x->y, bit1: y->x with x < y (original ids)
    uint32_t x = (uint32_t)(lo / (uint64_t)n), y = (uint32_t)(lo % (uint64_t)n);
    uint64_t rx = (uint32_t)old2new[x], ry = (uint32_t)old2new[y];
    uint64_t fswap = ((f & 1) << 1) | (f >> 1);
    out[2 * i] = (rx * (uint64_t)n + ry) | (f << 62);
    out[2 * i + 1] = (ry * (uint64_t)n + rx) | (fswap << 62);
}

// or_flags = 3 for an undirected graph: every edge is taken as arcs both ways
__global__ void fill_col(const uint64_t *__restrict__ sorted, int64_t nnz, int32_t n, const int64_t *rowptr,
                         uint32_t *__restrict__ col, int64_t *__restrict__ pbeg, uint32_t or_flags) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nnz) return;
    uint64_t k = sorted[i];
    uint64_t lo = k & LOW_MASK;
    uint32_t row = (uint32_t)(lo / (uint64_t)n), c = (uint32_t)(lo % (uint64_t)n);
    col[i] = (c << 2) | (uint32_t)(k >> 62) | or_flags;
    if (c > row) {
        bool first = (i == rowptr[row]);
        if (!first) {
            uint32_t prev = (uint32_t)((sorted[i - 1] & LOW_MASK) % (uint64_t)n);
            first = prev < row;
        }
        if (first) pbeg[row] = i;
    }
}

__global__ void init_pbeg(const int64_t *rowptr, int32_t n, int64_t *pbeg) {
    int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) pbeg[r] = rowptr[r + 1];
}

unsigned blocks_for(int64_t count, int tpb) { return (unsigned)((count + tpb - 1) / tpb); }

struct Tmp {
    cudaStream_t s;
    void *p[12];
    int np = 0;
    explicit Tmp(cudaStream_t st) : s(st) {}
    template <typename T>
    cudaError_t get(T **out, size_t count) {
        *out = nullptr;
        cudaError_t e = cudaMallocAsync((void **)out, sizeof(T) * (count ? count : 1), s);
        if (e == cudaSuccess) p[np++] = *out;
        return e;
    }
    void release(void *q) {
        for (int i = 0; i < np; i++)
            if (p[i] == q) {
                cudaFreeAsync(q, s);
                p[i] = p[--np];
                return;
            }
    }
    ~Tmp() {
        for (int i = 0; i < np; i++) cudaFreeAsync(p[i], s);
    }
};

// Stream-ordered release: the frees are queued on the graph's side stream
// behind its last build or count step (ev_done), so destroying a graph waits
// for nothing else on the device.
void free_graph_buffers(vdmc_graph *g) {
    cudaStream_t fs = g->side;
    if (fs && g->ev_done) cudaStreamWaitEvent(fs, g->ev_done, 0);
    vdmc_free(g->rowptr, fs);
    vdmc_free(g->col, fs);
    vdmc_free(g->pbeg, fs);
    vdmc_free(g->new2old, fs);
    vdmc_free(g->old2new, fs);
    vdmc_free(g->tasks, fs);
    vdmc_free(g->qhead, fs);
    vdmc_free(g->status, fs);
    vdmc_hub_free(g, fs);
    vdmc_batch_plan_free(g);
    vdmc_free(g->racc, fs);
    vdmc_free(g->d3acc, fs);
    vdmc_free(g->d3w, fs);
    vdmc_free(g->stats, fs);
    vdmc_free(g->ebase, fs);
    vdmc_free(g->erow, fs);
    vdmc_free(g->ekeys, fs);
    vdmc_free(g->eflags, fs);
    vdmc_free(g->etasks, fs);
    if (g->side) cudaStreamDestroy(g->side);  // released once its queued frees have run
    if (g->ev_fork) cudaEventDestroy(g->ev_fork);
    if (g->ev_join) cudaEventDestroy(g->ev_join);
    if (g->ev_done) cudaEventDestroy(g->ev_done);
}

// Graph memory comes from the device's default stream-ordered pool.  By
// default the pool returns freed memory to the driver at every
// synchronisation, so each new graph would map its gigabytes afresh; the
// library lets the pool keep up to VDMC_POOL_KEEP_BYTES of freed memory for
// reuse (set once per device, on the first graph built there).
constexpr uint64_t VDMC_POOL_KEEP_BYTES = 16ull << 30;
std::once_flag g_pool_once[64];

void keep_pool_memory(int dev) {
    if (dev < 0 || dev >= 64) return;
    std::call_once(g_pool_once[dev], [dev] {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
        uint64_t keep = VDMC_POOL_KEEP_BYTES, cur = 0;
        if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &cur) == cudaSuccess && cur < keep)
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    });
}

vdmc_status create_impl(int32_t n, int64_t m, const int32_t *src, const int32_t *dst, int on_device,
                        cudaStream_t s, vdmc_graph *g, const int64_t *goff, int32_t ngroups, uint32_t options) {
    g->n = n;
    g->undirected = (options & VDMC_GRAPH_UNDIRECTED) ? 1 : 0;
    g->info.n = n;
    g->info.arcs_in = m;
    VDMC_CUDA_TRY(cudaGetDevice(&g->device));
    keep_pool_memory(g->device);
    VDMC_CUDA_TRY(vdmc_malloc(&g->qhead, sizeof(unsigned long long), s));
    VDMC_CUDA_TRY(vdmc_malloc(&g->status, sizeof(int), s));
    VDMC_CUDA_TRY(vdmc_malloc(&g->stats, sizeof(unsigned long long) * VDMC_NSTATS, s));
    VDMC_CUDA_TRY(cudaMemsetAsync(g->stats, 0, sizeof(unsigned long long) * VDMC_NSTATS, s));
    {
        vdmc_status st0 = vdmc_graph_init_streams(g);
        if (st0 != VDMC_OK) return st0;
    }
    g->serial = vdmc_next_serial();
    g->num_graphs = 1;
    VDMC_CUDA_TRY(cudaMemsetAsync(g->status, 0, sizeof(int), s));

    Tmp tmp(s);
    const int32_t *dsrc = src, *ddst = dst;
    if (!on_device && m > 0) {
        int32_t *a, *b;
        VDMC_CUDA_TRY(tmp.get(&a, (size_t)m));
        VDMC_CUDA_TRY(tmp.get(&b, (size_t)m));
        VDMC_CUDA_TRY(cudaMemcpyAsync(a, src, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, s));
        VDMC_CUDA_TRY(cudaMemcpyAsync(b, dst, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, s));
        dsrc = a;
        ddst = b;
    }
    unsigned long long *counters;  // [0] self loops, [1] distinct arcs, [2] reciprocal, [3] spare
    int *bad, *dmax;
    VDMC_CUDA_TRY(tmp.get(&counters, 4));
    VDMC_CUDA_TRY(tmp.get(&bad, 2));
    dmax = bad + 1;
    VDMC_CUDA_TRY(cudaMemsetAsync(counters, 0, sizeof(unsigned long long) * 4, s));
    VDMC_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int) * 2, s));

    // 1-2: arc keys, sort, merge runs into unique undirected edges
    const uint64_t sentinel = (uint64_t)n * (uint64_t)n;
    int64_t eu = 0;
    uint64_t *uedges = nullptr;
    {
        uint64_t *keys, *keys2;
        VDMC_CUDA_TRY(tmp.get(&keys, (size_t)m));
        VDMC_CUDA_TRY(tmp.get(&keys2, (size_t)m));
        if (m > 0) {
            arc_keys<<<blocks_for(m, 256), 256, 0, s>>>(dsrc, ddst, m, n, keys, counters, bad);
            VDMC_CUDA_TRY(cudaGetLastError());
        }
        uint64_t *sorted;
        VDMC_CUDA_TRY(vdmc_radix_sort_u64(keys, keys2, m, 0, bits_for(sentinel), s, &sorted));
        uint32_t *head, *pos;
        VDMC_CUDA_TRY(tmp.get(&head, (size_t)m));
        VDMC_CUDA_TRY(tmp.get(&pos, (size_t)m + 1));
        if (m > 0) {
            run_heads<<<blocks_for(m, 256), 256, 0, s>>>(sorted, m, sentinel, head);
            VDMC_CUDA_TRY(cudaGetLastError());
        }
        VDMC_CUDA_TRY(vdmc_exclusive_scan_u32(head, pos, m, s));
        uint32_t eu32 = 0;
        int hbad = 0;
        VDMC_CUDA_TRY(cudaMemcpyAsync(&eu32, pos + m, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        VDMC_CUDA_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        VDMC_CUDA_TRY(cudaStreamSynchronize(s));
        if (hbad) return VDMC_ERR_OUT_OF_RANGE_VERTEX;
        eu = eu32;
        VDMC_CUDA_TRY(tmp.get(&uedges, (size_t)eu));
        if (m > 0) {
            merge_runs<<<blocks_for(m, 256), 256, 0, s>>>(sorted, m, pos, head, uedges, counters);
            VDMC_CUDA_TRY(cudaGetLastError());
        }
        tmp.release(keys);
        tmp.release(keys2);
        tmp.release(head);
        tmp.release(pos);
        if (!on_device && m > 0) {
            tmp.release((void *)dsrc);
            tmp.release((void *)ddst);
        }
    }

    // 3: degrees and ranks
    const int64_t nnz = 2 * eu;
    g->nnz = nnz;
    VDMC_CUDA_TRY(vdmc_malloc(&g->rowptr, sizeof(int64_t) * ((size_t)n + 1), s));
    VDMC_CUDA_TRY(vdmc_malloc(&g->col, sizeof(uint32_t) * (size_t)nnz, s));
    VDMC_CUDA_TRY(vdmc_malloc(&g->pbeg, sizeof(int64_t) * (size_t)n, s));
    VDMC_CUDA_TRY(vdmc_malloc(&g->new2old, sizeof(int32_t) * (size_t)n, s));
    VDMC_CUDA_TRY(vdmc_malloc(&g->old2new, sizeof(int32_t) * (size_t)n, s));
    int32_t *deg;
    int64_t *deg_rank;
    uint64_t *rk, *rk2, *rsorted;
    VDMC_CUDA_TRY(tmp.get(&deg, (size_t)n));
    VDMC_CUDA_TRY(tmp.get(&deg_rank, (size_t)n));
    VDMC_CUDA_TRY(tmp.get(&rk, (size_t)n));
    VDMC_CUDA_TRY(tmp.get(&rk2, (size_t)n));
    VDMC_CUDA_TRY(cudaMemsetAsync(deg, 0, sizeof(int32_t) * (size_t)(n ? n : 1), s));
    if (eu > 0) {
        edge_degrees<<<blocks_for(eu, 256), 256, 0, s>>>(uedges, eu, n, deg);
        VDMC_CUDA_TRY(cudaGetLastError());
    }
    if (n > 0) {
        max_degree<<<blocks_for(n, 256), 256, 0, s>>>(deg, n, dmax);
        VDMC_CUDA_TRY(cudaGetLastError());
    }
    int hdmax = 0;
    VDMC_CUDA_TRY(cudaMemcpyAsync(&hdmax, dmax, sizeof(int), cudaMemcpyDeviceToHost, s));
    VDMC_CUDA_TRY(cudaStreamSynchronize(s));
    const int dbits = bits_for((uint64_t)hdmax);
    const int gbits = goff ? bits_for((uint64_t)(ngroups > 0 ? ngroups - 1 : 0)) : 0;
    if (32 + dbits + gbits > 64) return VDMC_ERR_INVALID_ARG;
    if (n > 0) {
        rank_keys<<<blocks_for(n, 256), 256, 0, s>>>(deg, n, dmax, goff, ngroups, dbits, rk);
        VDMC_CUDA_TRY(cudaGetLastError());
    }
    VDMC_CUDA_TRY(vdmc_radix_sort_u64(rk, rk2, n, 32, 32 + dbits + gbits, s, &rsorted));
    if (n > 0) {
        rank_maps<<<blocks_for(n, 256), 256, 0, s>>>(rsorted, n, deg, g->new2old, g->old2new, deg_rank);
        VDMC_CUDA_TRY(cudaGetLastError());
    }
    VDMC_CUDA_TRY(vdmc_exclusive_scan_i64(deg_rank, g->rowptr, n, s));

    // 4: rank-space CSR
    {
        uint64_t *ck, *ck2, *csorted;
        VDMC_CUDA_TRY(tmp.get(&ck, (size_t)nnz));
        VDMC_CUDA_TRY(tmp.get(&ck2, (size_t)nnz));
        if (eu > 0) {
            oriented_entries<<<blocks_for(eu, 256), 256, 0, s>>>(uedges, eu, n, g->old2new, ck);
            VDMC_CUDA_TRY(cudaGetLastError());
        }
        uint64_t maxkey = n > 0 ? (uint64_t)n * (uint64_t)n - 1 : 0;
        VDMC_CUDA_TRY(vdmc_radix_sort_u64(ck, ck2, nnz, 0, bits_for(maxkey), s, &csorted));
        if (n > 0) {
            init_pbeg<<<blocks_for(n, 256), 256, 0, s>>>(g->rowptr, n, g->pbeg);
            VDMC_CUDA_TRY(cudaGetLastError());
        }
        if (nnz > 0) {
            fill_col<<<blocks_for(nnz, 256), 256, 0, s>>>(csorted, nnz, n, g->rowptr, g->col, g->pbeg,
                                                          g->undirected ? 3u : 0u);
            VDMC_CUDA_TRY(cudaGetLastError());
        }
    }
    unsigned long long hc[4];
    VDMC_CUDA_TRY(cudaMemcpyAsync(hc, counters, sizeof hc, cudaMemcpyDeviceToHost, s));
    VDMC_CUDA_TRY(cudaStreamSynchronize(s));
    g->info.self_loops = (int64_t)hc[0];
    g->info.arcs_kept = (int64_t)hc[1];
    g->info.reciprocal_pairs = (int64_t)hc[2];
    g->info.duplicate_arcs = m - (int64_t)hc[0] - (int64_t)hc[1];
    g->info.edges_u = eu;
    g->info.max_degree = hdmax;

    vdmc_schedule_t sch;
    vdmc_current_schedule(&sch);
    vdmc_status st = vdmc_build_tasks(g, sch.a_chunk, sch.hub_min_l, s);
    if (st != VDMC_OK) return st;
    VDMC_CUDA_TRY(cudaEventRecord(g->ev_done, s));
    VDMC_CUDA_TRY(cudaStreamSynchronize(s));
    return VDMC_OK;
}

}  // namespace

extern "C" vdmc_status vdmc_graph_create(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                                         int ptrs_on_device, void *stream, vdmc_graph **out) {
    return vdmc_graph_create_grouped(n, m, src, dst, ptrs_on_device, stream, out, nullptr, 0, 0u);
}

extern "C" vdmc_status vdmc_graph_create_ex(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                                            int ptrs_on_device, uint32_t options, void *stream, vdmc_graph **out) {
    if (options & ~(uint32_t)VDMC_GRAPH_UNDIRECTED) {
        if (out) *out = nullptr;
        return VDMC_ERR_INVALID_ARG;
    }
    return vdmc_graph_create_grouped(n, m, src, dst, ptrs_on_device, stream, out, nullptr, 0, options);
}

// goff: device int64[ngroups + 1] vertex offsets of the graphs of a batch,
// or nullptr for a single graph
vdmc_status vdmc_graph_create_grouped(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                                      int ptrs_on_device, void *stream, vdmc_graph **out, const int64_t *goff,
                                      int32_t ngroups, uint32_t options) {
    if (!out) return VDMC_ERR_INVALID_ARG;
    *out = nullptr;
    if (n < 0 || n >= (1 << 30) || m < 0 || m > 0xffffffffll) return VDMC_ERR_INVALID_ARG;
    if (m > 0 && (!src || !dst)) return VDMC_ERR_INVALID_ARG;
    vdmc_graph *g = new (std::nothrow) vdmc_graph;
    if (!g) return VDMC_ERR_OOM;
    std::memset(g, 0, sizeof *g);
    cudaStream_t s = (cudaStream_t)stream;
    vdmc_status st = create_impl(n, m, src, dst, ptrs_on_device, s, g, goff, ngroups, options);
    if (st != VDMC_OK) {
        cudaStreamSynchronize(s);
        cudaGetLastError();
        free_graph_buffers(g);
        delete g;
        return st;
    }
    g->info.device_bytes = (int64_t)(sizeof(int64_t) * ((size_t)n + 1) + sizeof(uint32_t) * (size_t)g->nnz +
                                     sizeof(int64_t) * (size_t)n + 2 * sizeof(int32_t) * (size_t)n +
                                     sizeof(Task) * (size_t)g->ntasks + 16);
    *out = g;
    return VDMC_OK;
}

extern "C" vdmc_status vdmc_graph_destroy(vdmc_graph *g) {
    if (!g) return VDMC_ERR_INVALID_ARG;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(g->device);
    free_graph_buffers(g);
    cudaSetDevice(cur);
    delete g;
    return VDMC_OK;
}

extern "C" vdmc_status vdmc_graph_info(const vdmc_graph *g, vdmc_graph_info_t *info) {
    if (!g || !info) return VDMC_ERR_INVALID_ARG;
    *info = g->info;
    info->num_graphs = g->num_graphs;
    info->num_tasks = g->ntasks;
    info->num_hub_roots = g->nhubs;
    info->device_bytes += (int64_t)g->hub_scratch_bytes;
    if (g->racc) info->device_bytes += (int64_t)(sizeof(uint64_t) * (size_t)g->n * VDMC_MAX_CLASSES);
    if (g->d3acc) info->device_bytes += (int64_t)(sizeof(uint64_t) * (size_t)g->n * VDMC_D3_COLS);
    if (g->d3w) info->device_bytes += (int64_t)(sizeof(uint64_t) * (size_t)g->n * 9);
    return VDMC_OK;
}

extern "C" vdmc_status vdmc_graph_export_csr(const vdmc_graph *g, int64_t *rowptr, uint32_t *col,
                                             int32_t *new2old) {
    if (!g) return VDMC_ERR_INVALID_ARG;
    VDMC_CUDA_TRY(cudaDeviceSynchronize());
    if (rowptr)
        VDMC_CUDA_TRY(cudaMemcpy(rowptr, g->rowptr, sizeof(int64_t) * ((size_t)g->n + 1), cudaMemcpyDeviceToHost));
    if (col && g->nnz)
        VDMC_CUDA_TRY(cudaMemcpy(col, g->col, sizeof(uint32_t) * (size_t)g->nnz, cudaMemcpyDeviceToHost));
    if (new2old && g->n)
        VDMC_CUDA_TRY(cudaMemcpy(new2old, g->new2old, sizeof(int32_t) * (size_t)g->n, cudaMemcpyDeviceToHost));
    return VDMC_OK;
}

extern "C" vdmc_status vdmc_get_device_status(vdmc_graph *g) {
    if (!g) return VDMC_ERR_INVALID_ARG;
    int h = 0;
    VDMC_CUDA_TRY(cudaMemcpy(&h, g->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) VDMC_CUDA_TRY(cudaMemset(g->status, 0, sizeof(int)));
    return (vdmc_status)h;
}

extern "C" const char *vdmc_status_string(vdmc_status s) {
    switch (s) {
        case VDMC_OK: return "ok";
        case VDMC_ERR_INVALID_ARG: return "invalid argument";
        case VDMC_ERR_OUT_OF_RANGE_VERTEX: return "arc endpoint outside [0, n)";
        case VDMC_ERR_OOM: return "device out of memory";
        case VDMC_ERR_CUDA: return "CUDA runtime error";
        case VDMC_ERR_DEVICE_LIMIT: return "kernel hit an internal limit";
        case VDMC_ERR_BUSY: return "resource busy";
    }
    return "unknown status";
}
