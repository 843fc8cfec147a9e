// Batched counting of many independent graphs in one launch.
//
// Two routes, both over one concatenated CSR (the disjoint union of the
// graphs; a set of k vertices from two graphs is never connected, so the
// union's counts are the graphs' counts stacked row by row):
//
//   vdmc_graph_create_batch  builds the union directly from the graphs' arc
//                            lists; one vdmc_count on it counts them all.
//   vdmc_count_batch         takes graphs built one by one; on its first call
//                            for a given list of graphs and outputs it
//                            concatenates their CSRs on the device into a
//                            cached plan (ranks of graph i shifted by the
//                            vertices before it), counts, and scatters the
//                            union's rows to the callers' outputs.  The
//                            second call captures that sequence into a CUDA
//                            graph, later calls replay it.
//
// The paper has no batched mode; within the union every root keeps its
// proper k-BFS (Lemma 1) because the union's order restricted to each graph
// is that graph's own degree order.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "vdmc_internal.cuh"

namespace {

std::atomic<uint64_t> g_serial{1};

struct PartDesc {
    const int64_t *rowptr;
    const uint32_t *col;
    const int64_t *pbeg;
    const int32_t *new2old;
};

// index i with off[i] <= x < off[i+1]
__device__ __forceinline__ int part_of(const int64_t *off, int num, int64_t x) {
    int lo = 0, hi = num;  // off[0] = 0 <= x < off[num]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (off[mid] <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void concat_rows(const PartDesc *parts, int num, const int64_t *roff, const int64_t *eoff, int64_t N,
                            int64_t NNZ, int64_t *rowptr, int64_t *pbeg, int32_t *new2old) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v == N) rowptr[N] = NNZ;
    if (v >= N) return;
    const int i = part_of(roff, num, v);
    const int64_t lv = v - roff[i];
    rowptr[v] = parts[i].rowptr[lv] + eoff[i];
    pbeg[v] = parts[i].pbeg[lv] + eoff[i];
    new2old[v] = parts[i].new2old[lv] + (int32_t)roff[i];
}

__global__ void concat_cols(const PartDesc *parts, int num, const int64_t *roff, const int64_t *eoff, int64_t NNZ,
                            uint32_t *col) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NNZ) return;
    const int i = part_of(eoff, num, e);
    const uint32_t x = parts[i].col[e - eoff[i]];
    col[e] = (((x >> 2) + (uint32_t)roff[i]) << 2) | (x & 3u);
}

__global__ void scatter_rows(const uint64_t *uout, int C, int64_t N, const int64_t *roff, int num,
                             uint64_t *const *outs) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * C) return;
    const int64_t v = idx / C;
    const int i = part_of(roff, num, v);
    outs[i][(v - roff[i]) * C + (idx - v * C)] = uout[idx];
}

// arcs of graph i (local ids, arc range [aoff[i], aoff[i+1])) -> union ids
__global__ void offset_arcs(int32_t *src, int32_t *dst, int64_t m, const int64_t *aoff, const int64_t *voff,
                            int num, int *bad) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    const int i = part_of(aoff, num, e);
    const int64_t ni = voff[i + 1] - voff[i];
    const int32_t u = src[e], v = dst[e];
    if (u < 0 || v < 0 || u >= ni || v >= ni) {
        atomicExch(bad, 1);
        src[e] = dst[e] = (int32_t)voff[i];  // harmless self-loop, dropped by the build
        return;
    }
    src[e] = u + (int32_t)voff[i];
    dst[e] = v + (int32_t)voff[i];
}

struct Plan {
    std::vector<uint64_t> serials;
    std::vector<uint64_t *> outs;
    int k = 0;
    vdmc_schedule_t sch{};
    vdmc_graph U;                   // the concatenated graph (owns its arrays)
    uint64_t *uout = nullptr;       // union output
    int64_t *roff_d = nullptr;      // num + 1
    uint64_t **outs_d = nullptr;    // num
    int num = 0;
    int calls = 0;
    cudaStream_t cap = nullptr;     // private stream the count is captured on
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

// the plan's union graph; called with the device idle (plan_free)
void free_union(vdmc_graph *U, cudaStream_t fs) {
    vdmc_free(U->rowptr, fs);
    vdmc_free(U->col, fs);
    vdmc_free(U->pbeg, fs);
    vdmc_free(U->new2old, fs);
    vdmc_free(U->old2new, fs);
    vdmc_free(U->tasks, fs);
    vdmc_free(U->qhead, fs);
    vdmc_free(U->status, fs);
    vdmc_free(U->racc, fs);
    vdmc_free(U->d3acc, fs);
    vdmc_free(U->d3w, fs);
    vdmc_free(U->stats, fs);
    vdmc_hub_free(U, fs);
    if (U->side) cudaStreamDestroy(U->side);
    if (U->ev_fork) cudaEventDestroy(U->ev_fork);
    if (U->ev_join) cudaEventDestroy(U->ev_join);
    if (U->ev_done) cudaEventDestroy(U->ev_done);
}

// A plan may have been replayed on any stream, so it is released with the
// device idle (this is the one release path that synchronises the device).
void plan_free(Plan *p) {
    if (!p) return;
    cudaDeviceSynchronize();
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->cap) cudaStreamDestroy(p->cap);
    vdmc_free(p->uout, 0);
    vdmc_free(p->roff_d, 0);
    vdmc_free(p->outs_d, 0);
    free_union(&p->U, 0);
    cudaDeviceSynchronize();
    delete p;
}

bool same_schedule(const vdmc_schedule_t &a, const vdmc_schedule_t &b) {
    return a.a_chunk == b.a_chunk && a.warps_per_block == b.warps_per_block && a.blocks_per_sm == b.blocks_per_sm &&
           a.hub_min_l == b.hub_min_l && a.hub_blocks_per_sm == b.hub_blocks_per_sm && a.hub_split == b.hub_split &&
           a.hub_split_roots == b.hub_split_roots && a.hub_warps == b.hub_warps && a.d3_bits == b.d3_bits;
}

vdmc_status build_plan(vdmc_graph *const *gs, int num, int k, uint64_t *const *outs, cudaStream_t s, Plan *p) {
    p->num = num;
    p->k = k;
    vdmc_current_schedule(&p->sch);
    std::vector<int64_t> roff(num + 1, 0), eoff(num + 1, 0);
    std::vector<PartDesc> parts(num);
    for (int i = 0; i < num; i++) {
        roff[i + 1] = roff[i] + gs[i]->n;
        eoff[i + 1] = eoff[i] + gs[i]->nnz;
        parts[i] = PartDesc{gs[i]->rowptr, gs[i]->col, gs[i]->pbeg, gs[i]->new2old};
        p->serials.push_back(gs[i]->serial);
        p->outs.push_back(outs[i]);
    }
    const int64_t N = roff[num], NNZ = eoff[num];
    if (N >= (int64_t(1) << 30)) return VDMC_ERR_INVALID_ARG;
    const int C = k == 3 ? 13 : 199;
    vdmc_graph &U = p->U;
    std::memset(&U, 0, sizeof U);
    U.n = (int32_t)N;
    U.nnz = NNZ;
    U.info.n = (int32_t)N;
    U.serial = vdmc_next_serial();
    VDMC_CUDA_TRY(cudaGetDevice(&U.device));
    VDMC_CUDA_TRY(vdmc_malloc(&U.rowptr, sizeof(int64_t) * (size_t)(N + 1), s));
    VDMC_CUDA_TRY(vdmc_malloc(&U.col, sizeof(uint32_t) * (size_t)NNZ, s));
    VDMC_CUDA_TRY(vdmc_malloc(&U.pbeg, sizeof(int64_t) * (size_t)N, s));
    VDMC_CUDA_TRY(vdmc_malloc(&U.new2old, sizeof(int32_t) * (size_t)N, s));
    VDMC_CUDA_TRY(vdmc_malloc(&U.qhead, sizeof(unsigned long long), s));
    VDMC_CUDA_TRY(vdmc_malloc(&U.status, sizeof(int), s));
    VDMC_CUDA_TRY(cudaMemsetAsync(U.status, 0, sizeof(int), s));
    VDMC_CUDA_TRY(vdmc_malloc(&U.stats, sizeof(unsigned long long) * VDMC_NSTATS, s));
    vdmc_status st = vdmc_graph_init_streams(&U);
    if (st != VDMC_OK) return st;
    VDMC_CUDA_TRY(vdmc_malloc(&p->uout, sizeof(uint64_t) * (size_t)(N * C), s));
    VDMC_CUDA_TRY(vdmc_malloc(&p->roff_d, sizeof(int64_t) * (size_t)(num + 1), s));
    VDMC_CUDA_TRY(vdmc_malloc(&p->outs_d, sizeof(uint64_t *) * (size_t)num, s));
    int64_t *eoff_d = nullptr;
    PartDesc *parts_d = nullptr;
    VDMC_CUDA_TRY(vdmc_malloc(&eoff_d, sizeof(int64_t) * (size_t)(num + 1), s));
    cudaError_t e = vdmc_malloc(&parts_d, sizeof(PartDesc) * (size_t)num, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->roff_d, roff.data(), sizeof(int64_t) * (num + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(eoff_d, eoff.data(), sizeof(int64_t) * (num + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(parts_d, parts.data(), sizeof(PartDesc) * num, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p->outs_d, outs, sizeof(uint64_t *) * num, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        concat_rows<<<(unsigned)((N + 1 + 255) / 256), 256, 0, s>>>(parts_d, num, p->roff_d, eoff_d, N, NNZ,
                                                                     U.rowptr, U.pbeg, U.new2old);
        if (NNZ > 0)
            concat_cols<<<(unsigned)((NNZ + 255) / 256), 256, 0, s>>>(parts_d, num, p->roff_d, eoff_d, NNZ, U.col);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host vectors copied above die with this call
    vdmc_free(eoff_d, s);
    vdmc_free(parts_d, s);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? VDMC_ERR_OOM : VDMC_ERR_CUDA;
    return vdmc_build_tasks(&U, p->sch.a_chunk, p->sch.hub_min_l, s);
}

vdmc_status run_plan(Plan *p, cudaStream_t s) {
    const int C = p->k == 3 ? 13 : 199;
    const int64_t N = p->U.n;
    vdmc_status st = vdmc_count_internal(&p->U, p->k, 0, p->U.n, p->uout, s);
    if (st != VDMC_OK) return st;
    if (N > 0) {
        scatter_rows<<<(unsigned)((N * C + 255) / 256), 256, 0, s>>>(p->uout, C, N, p->roff_d, p->num, p->outs_d);
        VDMC_CUDA_TRY(cudaGetLastError());
    }
    return VDMC_OK;
}

}  // namespace

uint64_t vdmc_next_serial() { return g_serial.fetch_add(1); }

vdmc_status vdmc_graph_init_streams(vdmc_graph *g) {
    VDMC_CUDA_TRY(cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking));
    VDMC_CUDA_TRY(cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming));
    VDMC_CUDA_TRY(cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming));
    VDMC_CUDA_TRY(cudaEventCreateWithFlags(&g->ev_done, cudaEventDisableTiming));
    return VDMC_OK;
}

void vdmc_batch_plan_free(vdmc_graph *g) {
    plan_free((Plan *)g->batch_plan);
    g->batch_plan = nullptr;
}

extern "C" vdmc_status vdmc_count_batch(vdmc_graph *const *graphs, int num, int k, uint64_t *const *outs,
                                        void *stream) {
    if (num < 0 || (num > 0 && (!graphs || !outs)) || (k != 3 && k != 4)) return VDMC_ERR_INVALID_ARG;
    if (num == 0) return VDMC_OK;
    for (int i = 0; i < num; i++)
        if (!graphs[i] || (!outs[i] && graphs[i]->n > 0) || graphs[i]->undirected) return VDMC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    vdmc_graph *lead = graphs[0];
    Plan *p = (Plan *)lead->batch_plan;
    vdmc_schedule_t sch;
    vdmc_current_schedule(&sch);
    bool reuse = p && p->k == k && p->num == num && same_schedule(p->sch, sch);
    for (int i = 0; reuse && i < num; i++)
        reuse = p->serials[i] == graphs[i]->serial && p->outs[i] == outs[i];
    if (!reuse) {
        VDMC_CUDA_TRY(cudaStreamSynchronize(s));
        vdmc_batch_plan_free(lead);
        p = new (std::nothrow) Plan;
        if (!p) return VDMC_ERR_OOM;
        vdmc_status st = build_plan(graphs, num, k, outs, s, p);
        if (st != VDMC_OK) {
            cudaStreamSynchronize(s);
            plan_free(p);
            return st;
        }
        lead->batch_plan = p;
    }
    p->calls++;
    if (p->calls == 1) return run_plan(p, s);  // direct; allocates the count's lazily created scratch
    if (!p->exec) {
        // capture the count + scatter once on the plan's own stream (the
        // caller's stream may be the legacy default stream, which cannot be
        // captured); every later call replays it on the caller's stream
        VDMC_CUDA_TRY(cudaStreamSynchronize(s));
        if (!p->cap) VDMC_CUDA_TRY(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking));
        VDMC_CUDA_TRY(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeRelaxed));
        vdmc_status st = run_plan(p, p->cap);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(p->cap, &graph);
        if (st != VDMC_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (e != cudaSuccess) return VDMC_ERR_CUDA;
        p->graph = graph;
        VDMC_CUDA_TRY(cudaGraphInstantiate(&p->exec, graph, 0));
    }
    VDMC_CUDA_TRY(cudaGraphLaunch(p->exec, s));
    return VDMC_OK;
}

extern "C" vdmc_status vdmc_graph_create_batch(int32_t num, const int32_t *ns, const int64_t *ms, const int32_t *src,
                                               const int32_t *dst, int ptrs_on_device, void *stream,
                                               vdmc_graph **out) {
    if (!out) return VDMC_ERR_INVALID_ARG;
    *out = nullptr;
    if (num < 1 || !ns || !ms) return VDMC_ERR_INVALID_ARG;
    std::vector<int64_t> voff(num + 1, 0), aoff(num + 1, 0);
    for (int i = 0; i < num; i++) {
        if (ns[i] < 0 || ms[i] < 0) return VDMC_ERR_INVALID_ARG;
        voff[i + 1] = voff[i] + ns[i];
        aoff[i + 1] = aoff[i] + ms[i];
    }
    const int64_t N = voff[num], M = aoff[num];
    if (N >= (int64_t(1) << 30) || M > 0xffffffffll) return VDMC_ERR_INVALID_ARG;
    if (M > 0 && (!src || !dst)) return VDMC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t *a = nullptr, *b = nullptr;
    int64_t *voff_d = nullptr, *aoff_d = nullptr;
    int *bad = nullptr;
    cudaError_t e = vdmc_malloc(&a, sizeof(int32_t) * (size_t)M, s);
    if (e == cudaSuccess) e = vdmc_malloc(&b, sizeof(int32_t) * (size_t)M, s);
    if (e == cudaSuccess) e = vdmc_malloc(&voff_d, sizeof(int64_t) * (size_t)(num + 1), s);
    if (e == cudaSuccess) e = vdmc_malloc(&aoff_d, sizeof(int64_t) * (size_t)(num + 1), s);
    if (e == cudaSuccess) e = vdmc_malloc(&bad, sizeof(int), s);
    const cudaMemcpyKind kind = ptrs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (e == cudaSuccess && M > 0) e = cudaMemcpyAsync(a, src, sizeof(int32_t) * (size_t)M, kind, s);
    if (e == cudaSuccess && M > 0) e = cudaMemcpyAsync(b, dst, sizeof(int32_t) * (size_t)M, kind, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(voff_d, voff.data(), sizeof(int64_t) * (num + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(aoff_d, aoff.data(), sizeof(int64_t) * (num + 1), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int), s);
    if (e == cudaSuccess && M > 0) {
        offset_arcs<<<(unsigned)((M + 255) / 256), 256, 0, s>>>(a, b, M, aoff_d, voff_d, num, bad);
        e = cudaGetLastError();
    }
    int hbad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    vdmc_status st = VDMC_OK;
    if (e != cudaSuccess) st = e == cudaErrorMemoryAllocation ? VDMC_ERR_OOM : VDMC_ERR_CUDA;
    else if (hbad) st = VDMC_ERR_OUT_OF_RANGE_VERTEX;
    else st = vdmc_graph_create_grouped((int32_t)N, M, a, b, 1, stream, out, voff_d, num, 0u);
    vdmc_free(a, s);
    vdmc_free(b, s);
    vdmc_free(voff_d, s);
    vdmc_free(aoff_d, s);
    vdmc_free(bad, s);
    if (st == VDMC_OK) {
        (*out)->num_graphs = num;
        (*out)->info.arcs_in = M;
    }
    return st;
}
