// Edge index of a graph, for per-edge motif counts (the edge variant of the
// Discussion: each motif credits its edges instead of its vertices).
//
// Edge ids live in rank space: the edge {u, v}, u < v in rank, is entry v of
// u's upper row, with id ebase[u] + its position there (ebase = exclusive sum
// of the upper-row lengths).  Output rows are the edges in ascending order of
// (min original id, max original id); erow maps an id to its row.  The order
// is found by sorting the keys (min << 30) | max (ids < 2^30) and searching
// each edge's key in the sorted list.
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "vdmc_internal.cuh"

namespace {

__global__ void upper_lengths(const int64_t *rowptr, const int64_t *pbeg, int32_t n, int64_t *len) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) len[r] = rowptr[r + 1] - pbeg[r];
}

// key of every edge id and its arcs oriented from the smaller original id
// (bit 0: min -> max, bit 1: max -> min); one warp per row
__global__ void edge_keys(const int64_t *__restrict__ rowptr, const int64_t *__restrict__ pbeg,
                          const uint32_t *__restrict__ col, const int32_t *__restrict__ new2old,
                          const int64_t *__restrict__ ebase, int32_t n, uint64_t *__restrict__ key,
                          uint8_t *__restrict__ oflag) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n) return;
    const int32_t r = (int32_t)w;
    const int64_t b = pbeg[r], e = rowptr[r + 1], base = ebase[r];
    const uint64_t o_r = (uint64_t)new2old[r];
    for (int64_t p = b + lane; p < e; p += 32) {
        const uint32_t ent = col[p];
        const uint64_t o_v = (uint64_t)new2old[ent >> 2];
        const uint32_t f = ent & 3u;  // bit 0: r -> v, bit 1: v -> r
        const bool r_first = o_r < o_v;
        key[base + (p - b)] = r_first ? ((o_r << 30) | o_v) : ((o_v << 30) | o_r);
        oflag[base + (p - b)] = (uint8_t)(r_first ? f : (((f & 1u) << 1) | (f >> 1)));
    }
}

// erow[id] = position of key[id] in the sorted keys; flags to that position
__global__ void edge_rows(const uint64_t *__restrict__ key, const uint8_t *__restrict__ oflag,
                          const uint64_t *__restrict__ sorted, int64_t ne, int64_t *__restrict__ erow,
                          uint8_t *__restrict__ eflags) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    const uint64_t k = key[i];
    int64_t lo = 0, hi = ne;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (sorted[mid] < k) lo = mid + 1;
        else hi = mid;
    }
    erow[i] = lo;
    eflags[lo] = oflag[i];
}

unsigned blocks_for(int64_t count, int tpb) { return (unsigned)((count + tpb - 1) / tpb); }

}  // namespace

vdmc_status vdmc_edge_index(vdmc_graph *g, cudaStream_t s) {
    if (g->erow || g->n == 0) return VDMC_OK;
    const int32_t n = g->n;
    const int64_t ne = g->nnz / 2;
    VDMC_CUDA_TRY(vdmc_malloc(&g->ebase, sizeof(int64_t) * ((size_t)n + 1), s));
    int64_t *len = nullptr;
    uint64_t *key = nullptr, *tmp = nullptr, *sorted = nullptr;
    uint8_t *oflag = nullptr;
    cudaError_t e = vdmc_malloc(&len, sizeof(int64_t) * ((size_t)n + 1), s);
    if (e == cudaSuccess) {
        upper_lengths<<<blocks_for(n, 256), 256, 0, s>>>(g->rowptr, g->pbeg, n, len);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = vdmc_exclusive_scan_i64(len, g->ebase, n, s);
    if (e == cudaSuccess) e = vdmc_malloc(&key, sizeof(uint64_t) * (size_t)ne, s);
    if (e == cudaSuccess) e = vdmc_malloc(&tmp, sizeof(uint64_t) * (size_t)ne, s);
    if (e == cudaSuccess) e = vdmc_malloc(&oflag, (size_t)ne, s);
    if (e == cudaSuccess) e = vdmc_malloc(&g->erow, sizeof(int64_t) * (size_t)ne, s);
    if (e == cudaSuccess) e = vdmc_malloc(&g->ekeys, sizeof(uint64_t) * (size_t)ne, s);
    if (e == cudaSuccess) e = vdmc_malloc(&g->eflags, (size_t)ne, s);
    if (e == cudaSuccess && ne > 0) {
        edge_keys<<<blocks_for((int64_t)n * 32, 256), 256, 0, s>>>(g->rowptr, g->pbeg, g->col, g->new2old, g->ebase, n,
                                                                    key, oflag);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->ekeys, key, sizeof(uint64_t) * (size_t)ne, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && ne > 0) e = vdmc_radix_sort_u64(g->ekeys, tmp, ne, 0, 60, s, &sorted);
    if (e == cudaSuccess && ne > 0 && sorted != g->ekeys)
        e = cudaMemcpyAsync(g->ekeys, sorted, sizeof(uint64_t) * (size_t)ne, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && ne > 0) {
        edge_rows<<<blocks_for(ne, 256), 256, 0, s>>>(key, oflag, g->ekeys, ne, g->erow, g->eflags);
        e = cudaGetLastError();
    }
    vdmc_free(len, s);
    vdmc_free(key, s);
    vdmc_free(tmp, s);
    vdmc_free(oflag, s);
    if (e != cudaSuccess) {
        vdmc_free(g->erow, s);
        g->erow = nullptr;
        return e == cudaErrorMemoryAllocation ? VDMC_ERR_OOM : VDMC_ERR_CUDA;
    }
    return VDMC_OK;
}

extern "C" vdmc_status vdmc_graph_edges(vdmc_graph *g, int32_t *u, int32_t *v, uint8_t *flags) {
    if (!g) return VDMC_ERR_INVALID_ARG;
    const int64_t ne = g->nnz / 2;
    if (ne == 0) return VDMC_OK;
    cudaStream_t s = g->side;
    VDMC_CUDA_TRY(cudaStreamWaitEvent(s, g->ev_done, 0));
    vdmc_status st = vdmc_edge_index(g, s);
    if (st != VDMC_OK) return st;
    std::vector<uint64_t> k((size_t)ne);
    VDMC_CUDA_TRY(cudaMemcpyAsync(k.data(), g->ekeys, sizeof(uint64_t) * (size_t)ne, cudaMemcpyDeviceToHost, s));
    if (flags) VDMC_CUDA_TRY(cudaMemcpyAsync(flags, g->eflags, (size_t)ne, cudaMemcpyDeviceToHost, s));
    VDMC_CUDA_TRY(cudaEventRecord(g->ev_done, s));
    VDMC_CUDA_TRY(cudaStreamSynchronize(s));
    for (int64_t i = 0; i < ne; i++) {
        if (u) u[i] = (int32_t)(k[(size_t)i] >> 30);
        if (v) v[i] = (int32_t)(k[(size_t)i] & ((1u << 30) - 1u));
    }
    return VDMC_OK;
}
