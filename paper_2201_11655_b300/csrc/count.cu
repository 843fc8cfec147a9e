// Per-vertex directed 3/4-motif enumeration (VDMC, "The Algorithm").
//
// Every connected k-set S is enumerated exactly once, from its lowest-rank
// vertex r (a proper k-BFS, Lemma 1), in exactly one BFS structure (Lemma 2)
// taken in one member order (Lemma 3).  Depths are set-internal BFS depths
// from r; the last vertex of a depth-3 chain is tested for direct adjacency
// to r and to the depth-1 vertex (the fix after Lemma 4), which needs no
// global depth marks.
//
// With P = N+(r) (neighbours of rank > r, sorted), the structures are
//   k = 3  star  (depth 2/3): a < b in P
//          path  (depth 1)  : a in P, b in N(a) \ N(r), b > r
//   k = 4  (1,1,1) depth 0.75: a < b < c in P
//          (1,1,2) depth 1   : a < b in P, c not in N(r), c > r, and
//                              c in N(a), or c in N(b) \ N(a)
//          (1,2,2) depth 1.25: a in P, b < c both in N(a) \ N(r), > r
//          (1,2,3) depth 1.5 : a in P, b in N(a) \ N(r), b > r,
//                              c in N(b) \ (N(r) u N(a)), c > r
// Each set's adjacency-matrix index (Fig. 1 bit order, members r,a,b,c) is
// mapped through the class table to an output column and every member gets
// +1 there ("increase the counter for each vertex in the k-BFS").
//
// Work decomposition: one warp per task; a task is a root and an
// interleaved slice of its depth-1 neighbours a (the paper's
// (vertex, neighbour) pairs).  Persistent warps take tasks from a device
// cursor with one atomicAdd; tasks are in rank order, so the heavy
// (high-degree, low-rank) roots go first.  Credits to r, a and b, which are
// fixed across inner loops, accumulate in per-warp shared-memory histograms
// and are flushed with one global atomicAdd per touched column; credits to
// the innermost member go straight to global memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "vdmc_internal.cuh"
#include "device_common.cuh"

namespace {

vdmc_schedule_t g_sched = {16, 8, 0, 64, 1, 1, 0, 16};
std::mutex g_sched_mu;

struct DevLut {
    uint8_t *lut[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
};
DevLut g_lut[64];  // per device
std::mutex g_lut_mu;

}  // namespace

cudaError_t vdmc_device_lut(int k, const uint8_t **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_lut_mu);
    if (!g_lut[dev].lut[k]) {
        size_t bytes = (size_t)1 << (k * (k - 1));
        uint8_t *p = nullptr;
        e = cudaMalloc((void **)&p, bytes);
        if (e != cudaSuccess) return e;
        e = cudaMemcpy(p, vdmc_host_lut(k), bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(p);
            return e;
        }
        g_lut[dev].lut[k] = p;
    }
    *out = g_lut[dev].lut[k];
    return cudaSuccess;
}

namespace {
cudaError_t device_lut(int k, const uint8_t **out) { return vdmc_device_lut(k, out); }

// ------------------------------------------------------------ tasks -----

// roots with L >= hub_min_l (> 0) belong to the root-per-CTA kernel
__global__ void task_counts(const int64_t *rowptr, const int64_t *pbeg, int32_t n, int32_t a_chunk,
                            int32_t hub_min_l, int64_t *cnt) {
    int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int64_t L = rowptr[r + 1] - pbeg[r];
    const bool hub = hub_min_l > 0 && L >= hub_min_l;
    cnt[r] = (L > 0 && !hub) ? (L + a_chunk - 1) / a_chunk : 0;
}

__global__ void task_fill(const int64_t *rowptr, const int64_t *pbeg, const int64_t *off, int32_t n,
                          int32_t a_chunk, int32_t hub_min_l, Task *tasks) {
    int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int64_t L = rowptr[r + 1] - pbeg[r];
    if (L <= 0 || (hub_min_l > 0 && L >= hub_min_l)) return;
    int32_t t = (int32_t)((L + a_chunk - 1) / a_chunk);
    int64_t o = off[r];
    for (int32_t j = 0; j < t; j++) tasks[o + j] = Task{r, j, t, 0};
}

template <int K>
__global__ void __launch_bounds__(256) count_kernel(GraphDesc single, const GraphDesc *__restrict__ multi,
                                                   const Task *__restrict__ tasks, int64_t ntasks,
                                                   unsigned long long *qhead, const uint8_t *__restrict__ lut_g,
                                                   int32_t rank_lo, int32_t rank_hi, int *status) {
    constexpr int C = (K == 3) ? 13 : 199;
    constexpr int NIDX = 1 << (K * (K - 1));
    constexpr int NH = (K == 3) ? 2 : 3;  // histograms per warp: r, a (, b)
    extern __shared__ unsigned long long smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    uint8_t *lut = (uint8_t *)(smem + (size_t)nwarps * NH * C);
    const Hist64 hist_r = hist64(smem + (size_t)warp * NH * C, C);
    const Hist64 hist_a = hist64(smem + (size_t)warp * NH * C + C, C);
    const Hist64 hist_b = hist64(smem + (size_t)warp * NH * C + 2 * C, C);  // K == 4 only
    // A disconnected index never reaches the table by construction; should
    // one appear, it is counted in no column and flags the status word.
    for (int i = threadIdx.x; i < NIDX; i += blockDim.x) {
        uint8_t v = lut_g[i];
        lut[i] = v;
    }
    for (int i = threadIdx.x; i < nwarps * NH * C; i += blockDim.x) smem[i] = 0ull;
    __syncthreads();

    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(qhead, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= (unsigned long long)ntasks) break;
        const Task task = tasks[t];
        const GraphDesc G = multi ? multi[task.g] : single;
        const int32_t r = task.r;
        if (r < rank_lo || r >= rank_hi) continue;
        Csr g{G.rowptr, G.col, G.pbeg, G.n, G.nnz, status};
        uint64_t *out = G.out;
        if (!in_bounds(g, r >= 0 && r < G.n && task.stride >= 1 && task.j >= 0)) continue;
        const int64_t pb = __ldg(g.pbeg + r), pe = __ldg(g.rowptr + r + 1);
        if (!in_bounds(g, pb >= 0 && pb <= pe && pe <= G.nnz)) continue;
        const int32_t L = (int32_t)(pe - pb);

        for (int32_t ia = task.j; ia < L; ia += task.stride) {
            const uint32_t ea = __ldg(g.col + pb + ia);
            const uint32_t a = ea >> 2, fra = ea & 3u;
            if (!in_bounds(g, a < G.n)) break;
            const int64_t a_beg = __ldg(g.rowptr + a), a_end = __ldg(g.rowptr + a + 1);
            if (!in_bounds(g, a_beg >= 0 && a_beg <= a_end && a_end <= G.nnz)) break;
            const int64_t a_up = upper_row(g.col, a_beg, a_end, (uint32_t)r);  // N(a) with rank > r
            if (K == 3) {
                // star: b in P after a
                for (int32_t ib = ia + 1 + lane; ib < L; ib += 32) {
                    const uint32_t eb = __ldg(g.col + pb + ib);
                    const uint32_t b = eb >> 2, frb = eb & 3u;
                    const uint32_t cls = lut[mask3(fra, frb, pair_flags(g, a, b))];
                    if (!in_bounds(g, cls < (uint32_t)C)) continue;
                    hinc(hist_r, cls);
                    hinc(hist_a, cls);
                    credit(g, out, G.new2old, b, C, cls);
                }
                // path: b in N(a) \ N(r), b > r
                for (int64_t x = a_up + lane; x < a_end; x += 32) {
                    const uint32_t eb = __ldg(g.col + x);
                    const uint32_t b = eb >> 2;
                    if (search_row(g.col, pb, pe, b)) continue;
                    const uint32_t cls = lut[mask3(fra, 0u, eb & 3u)];
                    if (!in_bounds(g, cls < (uint32_t)C)) continue;
                    hinc(hist_r, cls);
                    hinc(hist_a, cls);
                    credit(g, out, G.new2old, b, C, cls);
                }
            } else {
                // (A1) b in P after a
                for (int32_t ib = ia + 1; ib < L; ib++) {
                    const uint32_t eb = __ldg(g.col + pb + ib);
                    const uint32_t b = eb >> 2, frb = eb & 3u;
                    if (!in_bounds(g, b < G.n)) break;
                    const uint32_t fab = pair_flags(g, a, b);
                    const int64_t b_beg = __ldg(g.rowptr + b), b_end = __ldg(g.rowptr + b + 1);
                    if (!in_bounds(g, b_beg >= 0 && b_beg <= b_end && b_end <= G.nnz)) break;
                    // (1,1,1): c in P after b
                    for (int32_t ic = ib + 1 + lane; ic < L; ic += 32) {
                        const uint32_t ec = __ldg(g.col + pb + ic);
                        const uint32_t c = ec >> 2, frc = ec & 3u;
                        const uint32_t cls = lut[mask4(fra, frb, frc, fab, pair_flags(g, a, c), pair_flags(g, b, c))];
                        if (!in_bounds(g, cls < (uint32_t)C)) continue;
                        hinc(hist_r, cls);
                        hinc(hist_a, cls);
                        hinc(hist_b, cls);
                        credit(g, out, G.new2old, c, C, cls);
                    }
                    // (1,1,2) with c in N(a) \ N(r), c > r
                    for (int64_t x = a_up + lane; x < a_end; x += 32) {
                        const uint32_t ec = __ldg(g.col + x);
                        const uint32_t c = ec >> 2;
                        if (search_row(g.col, pb, pe, c)) continue;
                        const uint32_t cls = lut[mask4(fra, frb, 0u, fab, ec & 3u, pair_flags(g, b, c))];
                        if (!in_bounds(g, cls < (uint32_t)C)) continue;
                        hinc(hist_r, cls);
                        hinc(hist_a, cls);
                        hinc(hist_b, cls);
                        credit(g, out, G.new2old, c, C, cls);
                    }
                    // (1,1,2) with c in N(b) \ N(a) \ N(r), c > r
                    const int64_t b_up = upper_row(g.col, b_beg, b_end, (uint32_t)r);
                    for (int64_t x = b_up + lane; x < b_end; x += 32) {
                        const uint32_t ec = __ldg(g.col + x);
                        const uint32_t c = ec >> 2;
                        if (search_row(g.col, pb, pe, c)) continue;
                        if (pair_flags(g, a, c)) continue;
                        const uint32_t cls = lut[mask4(fra, frb, 0u, fab, 0u, ec & 3u)];
                        if (!in_bounds(g, cls < (uint32_t)C)) continue;
                        hinc(hist_r, cls);
                        hinc(hist_a, cls);
                        hinc(hist_b, cls);
                        credit(g, out, G.new2old, c, C, cls);
                    }
                    flush_hist(g, hist_b, C, out, row_of(G.new2old, b), lane);
                }
                // (A2) b in N(a) \ N(r), b > r
                for (int64_t xb = a_up; xb < a_end; xb++) {
                    const uint32_t eb = __ldg(g.col + xb);
                    const uint32_t b = eb >> 2, fab = eb & 3u;
                    if (!in_bounds(g, b < G.n)) break;
                    if (search_row(g.col, pb, pe, b)) continue;  // warp-uniform
                    const int64_t b_beg = __ldg(g.rowptr + b), b_end = __ldg(g.rowptr + b + 1);
                    if (!in_bounds(g, b_beg >= 0 && b_beg <= b_end && b_end <= G.nnz)) break;
                    // (1,2,2): c in N(a) after b, c not in N(r)
                    for (int64_t x = xb + 1 + lane; x < a_end; x += 32) {
                        const uint32_t ec = __ldg(g.col + x);
                        const uint32_t c = ec >> 2;
                        if (search_row(g.col, pb, pe, c)) continue;
                        const uint32_t cls = lut[mask4(fra, 0u, 0u, fab, ec & 3u, pair_flags(g, b, c))];
                        if (!in_bounds(g, cls < (uint32_t)C)) continue;
                        hinc(hist_r, cls);
                        hinc(hist_a, cls);
                        hinc(hist_b, cls);
                        credit(g, out, G.new2old, c, C, cls);
                    }
                    // (1,2,3): c in N(b), c > r, not in N(r), not adjacent to a
                    const int64_t b_up = upper_row(g.col, b_beg, b_end, (uint32_t)r);
                    for (int64_t x = b_up + lane; x < b_end; x += 32) {
                        const uint32_t ec = __ldg(g.col + x);
                        const uint32_t c = ec >> 2;
                        if (search_row(g.col, pb, pe, c)) continue;
                        if (pair_flags(g, a, c)) continue;
                        const uint32_t cls = lut[mask4(fra, 0u, 0u, fab, 0u, ec & 3u)];
                        if (!in_bounds(g, cls < (uint32_t)C)) continue;
                        hinc(hist_r, cls);
                        hinc(hist_a, cls);
                        hinc(hist_b, cls);
                        credit(g, out, G.new2old, c, C, cls);
                    }
                    flush_hist(g, hist_b, C, out, row_of(G.new2old, b), lane);
                }
            }
            flush_hist(g, hist_a, C, out, row_of(G.new2old, a), lane);
        }
        flush_hist(g, hist_r, C, out, row_of(G.new2old, r), lane);
    }
}

// out[new2old[r]] = acc[r] (+ the depth-3 credits d3[r], k = 4), one warp
// per row (coalesced row copies).  Column d of d3 holds the sets r' - x - b - c
// credited to c whose class is the d-th smallest of the depth-3 path classes
// (d3_column); unused columns stay zero.
__global__ void unrelabel_rows(const uint64_t *__restrict__ acc, const uint64_t *__restrict__ d3,
                               const uint8_t *__restrict__ lut, const int32_t *__restrict__ new2old, int32_t n,
                               int C, uint64_t *__restrict__ out) {
    __shared__ int d3cls[VDMC_D3_COLS];
    if (threadIdx.x < VDMC_D3_COLS) d3cls[threadIdx.x] = -1;
    __syncthreads();
    if (d3 && threadIdx.x < 27) {
        int cls = 0;
        const int col = d3_column(lut, threadIdx.x, &cls);
        if (col < VDMC_D3_COLS) d3cls[col] = cls;  // equal types write the same class
    }
    __syncthreads();
    const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (r >= n) return;
    const int32_t o = __ldg(new2old + r);
    if (o < 0 || o >= n) return;
    for (int c = lane; c < C; c += 32) {
        uint64_t v = acc[r * C + c];
        if (d3) {
            for (int j = 0; j < VDMC_D3_COLS; j++)
                if (d3cls[j] == c) v += d3[r * VDMC_D3_COLS + j];
        }
        out[(int64_t)o * C + c] = v;
    }
}

// Algorithmic bytes of one count: the adjacency rows each method must read
// at least once per use, 4 bytes per entry.
//  - roots of the warp-per-task kernel (plain enumeration): N(r), N(a) for
//    every depth-1 vertex a and, for k = 4, N(b) for every depth-2 vertex b;
//  - roots of the root-per-CTA kernel (L >= hub_min_l): N(r), N(x) for every
//    x in N+(r) and, for k = 4, N(b) for every Q-neighbour b of each such x
//    (counted once per adjacency x-b).
__global__ void work_bytes_kernel(Csr g, int32_t n, int k, int32_t hub_min_l, unsigned long long *total) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long acc = 0;
    for (int64_t r = wid; r < n; r += nw) {
        const int64_t rb = __ldg(g.rowptr + r), pb = __ldg(g.pbeg + r), pe = __ldg(g.rowptr + r + 1);
        const bool hub = hub_min_l > 0 && pe - pb >= hub_min_l;
        if (lane == 0) acc += (unsigned long long)(pe - rb);
        for (int64_t x = pb + lane; x < pe; x += 32) {
            const uint32_t a = __ldg(g.col + x) >> 2;
            const int64_t ab = __ldg(g.rowptr + a), ae = __ldg(g.rowptr + a + 1);
            acc += (unsigned long long)(ae - ab);
            if (k == 4) {
                for (int64_t y = upper_row(g.col, ab, ae, (uint32_t)r); y < ae; y++) {
                    const uint32_t b = __ldg(g.col + y) >> 2;
                    if (search_row(g.col, pb, pe, b)) continue;
                    acc += (unsigned long long)(__ldg(g.rowptr + b + 1) - __ldg(g.rowptr + b));
                }
            } else if (hub) {
                // k = 3 signature counting reads N(b) of each Q-neighbour once
                for (int64_t y = upper_row(g.col, ab, ae, (uint32_t)r); y < ae; y++) {
                    const uint32_t b = __ldg(g.col + y) >> 2;
                    if (search_row(g.col, pb, pe, b)) continue;
                    acc += (unsigned long long)(__ldg(g.rowptr + b + 1) - __ldg(g.rowptr + b));
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0 && acc) atomicAdd(total, acc * 4ull);
}

size_t smem_bytes(int k, int warps) {
    int C = k == 3 ? 13 : 199, NH = k == 3 ? 2 : 3;
    return (size_t)warps * NH * C * sizeof(unsigned long long) + ((size_t)1 << (k * (k - 1)));
}

vdmc_status launch_count(int k, const GraphDesc &single, const GraphDesc *multi, const Task *tasks,
                         int64_t ntasks, unsigned long long *qhead, int32_t lo, int32_t hi, int *status,
                         cudaStream_t s) {
    const uint8_t *lut = nullptr;
    VDMC_CUDA_TRY(device_lut(k, &lut));
    vdmc_schedule_t sch;
    vdmc_current_schedule(&sch);
    int warps = std::max(1, std::min(8, sch.warps_per_block));
    int threads = warps * 32;
    size_t smem = smem_bytes(k, warps);
    int dev = 0, sms = 0;
    VDMC_CUDA_TRY(cudaGetDevice(&dev));
    VDMC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    auto kern = (k == 3) ? count_kernel<3> : count_kernel<4>;
    VDMC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    VDMC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) per_sm = 1;
    if (sch.blocks_per_sm > 0) per_sm = std::min(per_sm, sch.blocks_per_sm);
    int64_t grid = (int64_t)sms * per_sm;
    int64_t need = (ntasks + warps - 1) / warps;
    if (grid > need) grid = std::max<int64_t>(1, need);
    VDMC_CUDA_TRY(cudaMemsetAsync(qhead, 0, sizeof(unsigned long long), s));
    if (ntasks > 0) {
        kern<<<(unsigned)grid, threads, smem, s>>>(single, multi, tasks, ntasks, qhead, lut, lo, hi, status);
        VDMC_CUDA_TRY(cudaGetLastError());
    }
    return VDMC_OK;
}

}  // namespace

void vdmc_current_schedule(vdmc_schedule_t *s) {
    std::lock_guard<std::mutex> lk(g_sched_mu);
    *s = g_sched;
}

vdmc_status vdmc_build_tasks(vdmc_graph *g, int32_t a_chunk, int32_t hub_min_l, cudaStream_t s) {
    if (a_chunk < 1 || hub_min_l < 0) return VDMC_ERR_INVALID_ARG;
    cudaFree(g->tasks);
    g->tasks = nullptr;
    g->ntasks = 0;
    const int32_t n = g->n;
    int64_t *cnt = nullptr;
    VDMC_CUDA_TRY(cudaMallocAsync((void **)&cnt, sizeof(int64_t) * ((size_t)n + 1), s));
    if (n > 0) {
        task_counts<<<(n + 255) / 256, 256, 0, s>>>(g->rowptr, g->pbeg, n, a_chunk, hub_min_l, cnt);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = vdmc_exclusive_scan_i64(cnt, cnt, n, s);
    int64_t total = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total, cnt + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMalloc((void **)&g->tasks, sizeof(Task) * (size_t)(total ? total : 1));
    if (e == cudaSuccess && n > 0) {
        task_fill<<<(n + 255) / 256, 256, 0, s>>>(g->rowptr, g->pbeg, cnt, n, a_chunk, hub_min_l, g->tasks);
        e = cudaGetLastError();
    }
    cudaFreeAsync(cnt, s);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? VDMC_ERR_OOM : VDMC_ERR_CUDA;
    g->ntasks = total;
    g->tasks_a_chunk = a_chunk;
    return vdmc_build_hubs(g, hub_min_l, s);
}

vdmc_status vdmc_count_internal(vdmc_graph *g, int k, int32_t lo, int32_t hi, uint64_t *out, cudaStream_t s) {
    if (!g || (k != 3 && k != 4)) return VDMC_ERR_INVALID_ARG;
    if (!out && g->n > 0) return VDMC_ERR_INVALID_ARG;
    const int C = k == 3 ? 13 : 199;
    vdmc_schedule_t sch;
    vdmc_current_schedule(&sch);
    if (g->tasks_a_chunk != sch.a_chunk || g->hub_min_l != sch.hub_min_l) {
        vdmc_status st = vdmc_build_tasks(g, sch.a_chunk, sch.hub_min_l, s);
        if (st != VDMC_OK) return st;
    }
    // Credits accumulate in a rank-space array owned by the graph (no id-map
    // load in front of each atomic); one coalesced pass then writes every row
    // to its original id in `out`.
    if (!g->racc && g->n > 0) {
        VDMC_CUDA_TRY(cudaStreamSynchronize(s));
        VDMC_CUDA_TRY(cudaMalloc((void **)&g->racc, sizeof(uint64_t) * (size_t)g->n * VDMC_MAX_CLASSES));
    }
    uint64_t *acc = g->racc;
    if (g->n > 0) VDMC_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(uint64_t) * (size_t)g->n * C, s));
    // depth-3 credits of the root-per-CTA kernel (k = 4): one column per path
    // class (16 per vertex) instead of 199, so that more reductions stay in L2
    uint64_t *d3 = nullptr;
    if (k == 4 && g->nhubs > 0 && g->n > 0) {
        if (!g->d3acc) {
            VDMC_CUDA_TRY(cudaStreamSynchronize(s));
            VDMC_CUDA_TRY(cudaMalloc((void **)&g->d3acc, sizeof(uint64_t) * (size_t)g->n * VDMC_D3_COLS));
        }
        d3 = g->d3acc;
        VDMC_CUDA_TRY(cudaMemsetAsync(d3, 0, sizeof(uint64_t) * (size_t)g->n * VDMC_D3_COLS, s));
    }
    const uint8_t *lut = nullptr;
    VDMC_CUDA_TRY(device_lut(k, &lut));
    GraphDesc d{g->rowptr, g->col, g->pbeg, nullptr, acc, g->n, 0, g->nnz};
    if (g->nhubs > 0) {
        // the root-per-CTA kernel runs on the graph's side stream, overlapped
        // with the warp kernel; the caller's stream waits for both
        VDMC_CUDA_TRY(cudaEventRecord(g->ev_fork, s));
        VDMC_CUDA_TRY(cudaStreamWaitEvent(g->side, g->ev_fork, 0));
        vdmc_status st = vdmc_hub_launch(g, k, acc, d3, lut, lo, hi, sch.hub_blocks_per_sm, sch.hub_split,
                                          sch.hub_split_roots, sch.hub_warps, g->side);
        if (st != VDMC_OK) return st;
        VDMC_CUDA_TRY(cudaEventRecord(g->ev_join, g->side));
    }
    vdmc_status st = launch_count(k, d, nullptr, g->tasks, g->ntasks, g->qhead, lo, hi, g->status, s);
    if (g->nhubs > 0) VDMC_CUDA_TRY(cudaStreamWaitEvent(s, g->ev_join, 0));
    if (st != VDMC_OK) return st;
    if (g->n > 0) {
        unrelabel_rows<<<(unsigned)((g->n + 7) / 8), 256, 0, s>>>(acc, d3, lut, g->new2old, g->n, C, out);
        VDMC_CUDA_TRY(cudaGetLastError());
    }
    return VDMC_OK;
}

extern "C" vdmc_status vdmc_count(vdmc_graph *g, int k, uint64_t *out_dev, void *stream) {
    return vdmc_count_internal(g, k, 0, g ? g->n : 0, out_dev, (cudaStream_t)stream);
}

extern "C" vdmc_status vdmc_count_roots(vdmc_graph *g, int k, int32_t rank_lo, int32_t rank_hi, uint64_t *out_dev,
                                        void *stream) {
    if (!g || rank_lo < 0 || rank_hi < rank_lo) return VDMC_ERR_INVALID_ARG;
    return vdmc_count_internal(g, k, rank_lo, std::min(rank_hi, g->n), out_dev, (cudaStream_t)stream);
}

extern "C" vdmc_status vdmc_work_bytes(const vdmc_graph *g, int k, uint64_t *bytes) {
    if (!g || !bytes || (k != 3 && k != 4)) return VDMC_ERR_INVALID_ARG;
    unsigned long long *d = nullptr;
    VDMC_CUDA_TRY(cudaMalloc((void **)&d, sizeof(unsigned long long)));
    cudaError_t e = cudaMemset(d, 0, sizeof(unsigned long long));
    if (e == cudaSuccess && g->n > 0) {
        Csr c{g->rowptr, g->col, g->pbeg, g->n, g->nnz, g->status};
        vdmc_schedule_t sch;
        vdmc_current_schedule(&sch);
        work_bytes_kernel<<<1184, 256>>>(c, g->n, k, sch.hub_min_l, d);
        e = cudaGetLastError();
    }
    unsigned long long h = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof h, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return VDMC_ERR_CUDA;
    const int C = k == 3 ? 13 : 199;
    *bytes = (uint64_t)h + 8ull * (uint64_t)g->n * (uint64_t)C + 4ull * (uint64_t)g->n;
    return VDMC_OK;
}

extern "C" vdmc_status vdmc_set_schedule(const vdmc_schedule_t *s) {
    if (!s || s->a_chunk < 1 || s->warps_per_block < 1 || s->warps_per_block > 8 || s->blocks_per_sm < 0 ||
        s->hub_min_l < 0 || s->hub_blocks_per_sm < 1 || s->hub_blocks_per_sm > 8 || s->hub_split < 0 ||
        s->hub_split > 16 || s->hub_split_roots < 0 || (s->hub_warps != 0 && s->hub_warps != 16 && s->hub_warps != 32))
        return VDMC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_sched_mu);
    g_sched = *s;
    return VDMC_OK;
}

extern "C" vdmc_status vdmc_get_schedule(vdmc_schedule_t *s) {
    if (!s) return VDMC_ERR_INVALID_ARG;
    vdmc_current_schedule(s);
    return VDMC_OK;
}

// ------------------------------------------------- allocation-free variant --
//
// vdmc_count_csr_noalloc: the warp-per-task count for callers that must not
// allocate device memory.  Its scratch (task list, work-queue cursor,
// status word, class tables) is the file-scope array below, which exists
// once per device for as long as the library is loaded.

namespace {

constexpr int64_t NOALLOC_MAX_N = int64_t(1) << 18;       // vertices
constexpr int64_t NOALLOC_MAX_TASKS = NOALLOC_MAX_N;      // one per root with L >= 1 at most
constexpr size_t NOALLOC_HDR = 256;                        // cursor (8 B) + status (4 B), padded
constexpr size_t NOALLOC_LUT = 4096 + 64;                  // k = 4 table, then k = 3 table
constexpr size_t NOALLOC_BYTES = NOALLOC_HDR + NOALLOC_LUT + sizeof(Task) * (size_t)NOALLOC_MAX_TASKS;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

struct NoallocDevice {
    bool ready = false;
    unsigned char *base = nullptr;  // device address of g_noalloc_scratch
};
NoallocDevice g_noalloc_dev[64];
std::mutex g_noalloc_mu;

// One CTA: one task per root with at least one higher-rank neighbour (the
// whole slice of depth-1 neighbours, stride 1), in rank order; the unused
// tail of the task array is marked empty (r = -1, skipped by the kernel).
// Also zeroes the cursor and the status word.
__global__ void __launch_bounds__(1024) noalloc_tasks(const int64_t *rowptr, const int64_t *pbeg, int32_t n,
                                                      Task *tasks, int64_t max_tasks, unsigned long long *cursor,
                                                      int *status) {
    __shared__ int32_t warp_tot[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t chunk = (n + 1023) / 1024;
    const int32_t beg = min(n, tid * chunk), end = min(n, beg + chunk);
    int32_t s = 0;
    for (int32_t r = beg; r < end; r++) s += (rowptr[r + 1] - pbeg[r]) > 0;
    int32_t inc = s;
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int32_t w = warp_tot[lane];
        int32_t wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        warp_tot[lane] = wi - w;
    }
    __syncthreads();
    int32_t o = warp_tot[warp] + inc - s;
    for (int32_t r = beg; r < end; r++)
        if ((rowptr[r + 1] - pbeg[r]) > 0 && o < max_tasks) tasks[o++] = Task{r, 0, 1, 0};
    // total = exclusive prefix of the last thread + its own count
    __syncthreads();
    if (tid == 1023) warp_tot[0] = o;
    __syncthreads();
    for (int64_t t = warp_tot[0] + tid; t < max_tasks; t += 1024) tasks[t] = Task{-1, 0, 1, 0};
    if (tid == 0) {
        *cursor = 0ull;
        *status = 0;
    }
}

}  // namespace

extern "C" vdmc_status vdmc_count_csr_noalloc(int32_t n, int64_t nnz, const int64_t *rowptr, const uint32_t *col,
                                              const int64_t *pbeg, const int32_t *new2old, int k, uint64_t *out_dev,
                                              int *status_dev, void *stream) {
    if (k != 3 && k != 4) return VDMC_ERR_INVALID_ARG;
    if (n < 0 || nnz < 0 || n > NOALLOC_MAX_N) return VDMC_ERR_INVALID_ARG;
    if (n > 0 && (!rowptr || !pbeg || !new2old || !out_dev || (nnz > 0 && !col))) return VDMC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    VDMC_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return VDMC_ERR_INVALID_ARG;
    unsigned char *base = nullptr;
    {
        // once per device: the device address of the scratch array and the
        // class tables copied into it (plain copies, no allocation)
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        NoallocDevice &D = g_noalloc_dev[dev];
        if (!D.ready) {
            void *p = nullptr;
            VDMC_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
            unsigned char *b = (unsigned char *)p;
            VDMC_CUDA_TRY(cudaMemcpy(b + NOALLOC_HDR, vdmc_host_lut(4), 4096, cudaMemcpyHostToDevice));
            VDMC_CUDA_TRY(cudaMemcpy(b + NOALLOC_HDR + 4096, vdmc_host_lut(3), 64, cudaMemcpyHostToDevice));
            D.base = b;
            D.ready = true;
        }
        base = D.base;
    }
    const int C = k == 3 ? 13 : 199;
    unsigned long long *cursor = (unsigned long long *)base;
    int *status = status_dev ? status_dev : (int *)(base + 8);
    const uint8_t *lut = base + NOALLOC_HDR + (k == 4 ? 0 : 4096);
    Task *tasks = (Task *)(base + NOALLOC_HDR + NOALLOC_LUT);
    if (n == 0) return VDMC_OK;
    VDMC_CUDA_TRY(cudaMemsetAsync(out_dev, 0, sizeof(uint64_t) * (size_t)n * C, s));
    noalloc_tasks<<<1, 1024, 0, s>>>(rowptr, pbeg, n, tasks, NOALLOC_MAX_TASKS, cursor, status);
    VDMC_CUDA_TRY(cudaGetLastError());
    vdmc_schedule_t sch;
    vdmc_current_schedule(&sch);
    const int warps = std::max(1, std::min(8, sch.warps_per_block));
    const size_t smem = smem_bytes(k, warps);
    int sms = 0, per_sm = 0;
    VDMC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    auto kern = (k == 3) ? count_kernel<3> : count_kernel<4>;
    VDMC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    VDMC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem));
    const int64_t grid = (int64_t)sms * std::max(1, per_sm);
    GraphDesc d{rowptr, col, pbeg, new2old, out_dev, n, 0, nnz};
    kern<<<(unsigned)grid, warps * 32, smem, s>>>(d, nullptr, tasks, NOALLOC_MAX_TASKS, cursor, lut, 0, n, status);
    VDMC_CUDA_TRY(cudaGetLastError());
    return VDMC_OK;
}
