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

vdmc_schedule_t g_sched = {16, 8, 0, 64, 1, 1, 0, 0, 0};
std::mutex g_sched_mu;

struct DevLut {
    uint8_t *lut[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    uint8_t *colmap[5][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr},
                             {nullptr, nullptr}};
};
DevLut g_lut[64];  // per device
std::mutex g_lut_mu;

// a device copy of a small host table, made once per device (kept for the
// life of the process)
cudaError_t device_table(uint8_t **slot, const std::vector<uint8_t> &host) {
    if (*slot) return cudaSuccess;
    uint8_t *p = nullptr;
    cudaError_t e = cudaMalloc((void **)&p, host.size());
    if (e != cudaSuccess) return e;
    e = cudaMemcpy(p, host.data(), host.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(p);
        return e;
    }
    *slot = p;
    return cudaSuccess;
}

}  // namespace

// motif index -> accumulator column (the kernels' class ids)
cudaError_t vdmc_device_lut(int k, const uint8_t **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || (k != 3 && k != 4)) return cudaErrorInvalidValue;
    std::lock_guard<std::mutex> lk(g_lut_mu);
    if (!g_lut[dev].lut[k]) {
        const size_t nidx = (size_t)1 << (k * (k - 1));
        const uint8_t *lut = vdmc_host_lut(k), *acc_col = vdmc_host_acc_col(k);
        std::vector<uint8_t> h(nidx);
        for (size_t i = 0; i < nidx; i++) h[i] = lut[i] == 255 ? 255 : acc_col[lut[i]];
        e = device_table(&g_lut[dev].lut[k], h);
        if (e != cudaSuccess) return e;
    }
    *out = g_lut[dev].lut[k];
    return cudaSuccess;
}

// accumulator column -> output column: the class itself (directed), or its
// undirected column (255 where the class is not symmetric)
cudaError_t vdmc_device_colmap(int k, bool undirected, const uint8_t **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || (k != 3 && k != 4)) return cudaErrorInvalidValue;
    std::lock_guard<std::mutex> lk(g_lut_mu);
    uint8_t **slot = &g_lut[dev].colmap[k][undirected ? 1 : 0];
    if (!*slot) {
        const int C = k == 3 ? 13 : 199;
        const uint8_t *acc_class = vdmc_host_acc_class(k);
        const uint8_t *ucol = vdmc_host_ucol(k, nullptr);
        std::vector<uint8_t> h(C);
        for (int j = 0; j < C; j++) h[j] = undirected ? ucol[acc_class[j]] : acc_class[j];
        e = device_table(slot, h);
        if (e != cudaSuccess) return e;
    }
    *out = *slot;
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

// +n for vertex (rank) v in column cls of its output row
__device__ __forceinline__ void credit_n(const Csr &g, uint64_t *out, const int32_t *new2old, uint32_t v, int C,
                                         uint32_t cls, uint32_t n) {
    if (!in_bounds(g, v < g.n)) return;
    const int32_t o = row_of(new2old, v);
    if (!in_bounds(g, o >= 0 && o < g.n)) return;
    atomicAdd((unsigned long long *)&out[(int64_t)o * C + cls], (unsigned long long)n);
}

// Per-edge mode (the edge variant of the Discussion): each set credits the
// edges of G_U inside it instead of its vertices.  Edge ids: the entries of
// the upper rows in rank order (the edge {u, v}, u < v in rank, is entry
// v of u's upper row, id ebase[u] + its position there); erow maps an id to
// its output row.  ucol maps the kernel's class id (accumulator column) to
// the output column (vdmc_device_colmap).
struct EdgeDesc {
    const int64_t *ebase;
    const int64_t *erow;
    const uint8_t *ucol;
    int32_t cout;
};

// id of the edge {u, v} (rank space); -1 (and the status word) if absent
__device__ __forceinline__ int64_t edge_id(const Csr &g, const int64_t *ebase, uint32_t u, uint32_t v) {
    if (u > v) {
        const uint32_t t = u;
        u = v;
        v = t;
    }
    if (!in_bounds(g, v < g.n)) return -1;
    const int64_t lo = __ldg(g.pbeg + u), hi = __ldg(g.rowptr + u + 1);
    const int64_t p = upper_row(g.col, lo, hi, v - 1);  // first entry with rank >= v
    if (!in_bounds(g, p < hi && (__ldg(g.col + p) >> 2) == v)) return -1;
    return __ldg(ebase + u) + (p - lo);
}

__device__ __forceinline__ void edge_credit(const Csr &g, const EdgeDesc &E, uint64_t *out, int64_t eid,
                                            uint32_t cls) {
    if (eid < 0) return;
    const uint32_t c = (uint32_t)__ldg(E.ucol + cls);
    if (!in_bounds(g, c < (uint32_t)E.cout && eid < g.nnz / 2)) return;
    const int64_t row = __ldg(E.erow + eid);
    atomicAdd((unsigned long long *)&out[row * E.cout + c], 1ull);
}

// credits of one set {r, a, b (, c)} to its edges: r-a always (a at position
// ia of N+(r)); r-b and r-c when b, c are in N+(r) (positions ib, ic >= 0);
// the other pairs when their flags say they are adjacent
template <int K>
__device__ __forceinline__ void edge_set(const Csr &g, const EdgeDesc &E, uint64_t *out, uint32_t r, uint32_t a,
                                         uint32_t b, uint32_t c, int32_t ia, int32_t ib, int32_t ic, uint32_t fab,
                                         uint32_t fac, uint32_t fbc, uint32_t cls) {
    const int64_t eb = __ldg(E.ebase + r);
    edge_credit(g, E, out, eb + ia, cls);
    if (ib >= 0) edge_credit(g, E, out, eb + ib, cls);
    if (fab) edge_credit(g, E, out, edge_id(g, E.ebase, a, b), cls);
    if (K == 4) {
        if (ic >= 0) edge_credit(g, E, out, eb + ic, cls);
        if (fac) edge_credit(g, E, out, edge_id(g, E.ebase, a, c), cls);
        if (fbc) edge_credit(g, E, out, edge_id(g, E.ebase, b, c), cls);
    }
}

// Every adjacency test of a set asks about two members of rank > r, so it
// searches the part of a member's row above the root.  N+(r), which every
// candidate is tested against, is staged per warp in shared memory when it
// fits; so is N(a) above r on the flattened k = 4 walk, where all lanes use
// it for every b.  The rows of b are searched in global memory (staging each
// b's row as well measured slower on the power-law workload: they are short
// and the copies cost more than they save).
constexpr int STAGE_P = 64, STAGE_A = 128;
constexpr int STAGE_WORDS = STAGE_P + STAGE_A;  // per warp
static_assert(STAGE_A >= 32 * 4, "the k = 3 walk keeps 4 words of star flags per a-item in the N(a) area");

struct View {
    const uint32_t *s;  // staged entries (shared memory), or nullptr
    int64_t beg, end;   // the row segment in col
};

// warp-wide: copy col[beg, end) to dst when it fits in cap entries
__device__ __forceinline__ View stage(const Csr &g, uint32_t *dst, int64_t beg, int64_t end, int cap, int lane) {
    __syncwarp();
    if (end - beg > cap) return View{nullptr, beg, end};
    for (int64_t x = beg + lane; x < end; x += 32) dst[x - beg] = __ldg(g.col + x);
    __syncwarp();
    return View{dst, beg, end};
}

__device__ __forceinline__ uint32_t view_entry(const Csr &g, const View &v, int64_t x) {
    return v.s ? v.s[x - v.beg] : __ldg(g.col + x);
}

// position of u in a staged view, -1 if absent
__device__ __forceinline__ int32_t view_pos(const View &v, uint32_t u) {
    int32_t lo = 0, len = (int32_t)(v.end - v.beg);
    while (len > 0) {
        const int32_t half = len >> 1;
        if ((v.s[lo + half] >> 2) < u) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return lo < (int32_t)(v.end - v.beg) && (v.s[lo] >> 2) == u ? lo : -1;
}

// flags of neighbour u in the view (0 if absent)
__device__ __forceinline__ uint32_t view_find(const Csr &g, const View &v, uint32_t u) {
    if (!v.s) return search_row(g.col, v.beg, v.end, u);
    int32_t lo = 0, len = (int32_t)(v.end - v.beg);
    while (len > 0) {
        const int32_t half = len >> 1;
        if ((v.s[lo + half] >> 2) < u) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    if (lo < (int32_t)(v.end - v.beg) && (v.s[lo] >> 2) == u) return v.s[lo] & 3u;
    return 0u;
}

// flush h to row orig and add its counts to the warp's histogram into
// (each lane owns its columns of both, so plain adds)
__device__ __forceinline__ void flush_hist_into(const Csr &g, const Hist64 &h, const Hist64 &into, int C,
                                                uint64_t *out, int32_t orig, int lane) {
    __syncwarp();
    const bool ok = in_bounds(g, orig >= 0 && orig < g.n);
    for (int c = lane; c < C; c += 32) {
        const unsigned long long v = hget(h, c);
        if (v) {
            if (ok) atomicAdd((unsigned long long *)&out[(int64_t)orig * C + c], v);
            const unsigned long long t = hget(into, c) + v;
            into.lo[c] = (uint32_t)t;
            into.hi[c] = (uint32_t)(t >> 32);
            h.lo[c] = 0u;
            h.hi[c] = 0u;
        }
    }
    __syncwarp();
}

// Per-warp open-addressing table of the k = 4 flattened walk (linear
// probing, 256 slots, at most 64 + 128 keys, so a probe always ends at an
// empty slot): word = (vertex << 4) | bits, vertex ids below 2^28.
constexpr int HT_SLOTS = 256;
constexpr uint32_t HT_EMPTY = 0xffffffffu;
constexpr int32_t HT_MAX_N = 1 << 28;

__device__ __forceinline__ uint32_t ht_slot(uint32_t v) { return (v * 0x9E3779B1u) >> 24; }

// add `bits` to v's word, inserting v if absent (keys of one call are
// distinct across the lanes, so no two lanes insert the same vertex)
__device__ __forceinline__ void ht_insert(uint32_t *ht, uint32_t v, uint32_t bits) {
    uint32_t h = ht_slot(v);
    for (int i = 0; i < HT_SLOTS; i++, h = (h + 1u) & (HT_SLOTS - 1)) {
        const uint32_t cur = ht[h];
        if (cur == HT_EMPTY) {
            const uint32_t prev = atomicCAS(ht + h, HT_EMPTY, (v << 4) | bits);
            if (prev == HT_EMPTY) return;
            if ((prev >> 4) == v) {
                atomicOr(ht + h, bits);
                return;
            }
        } else if ((cur >> 4) == v) {
            atomicOr(ht + h, bits);
            return;
        }
    }
}

// v's bits (0 if absent) and, when present, its slot
__device__ __forceinline__ uint32_t ht_find_slot(const uint32_t *ht, uint32_t v, uint32_t &slot) {
    uint32_t h = ht_slot(v);
    for (int i = 0; i < HT_SLOTS; i++, h = (h + 1u) & (HT_SLOTS - 1)) {
        const uint32_t cur = ht[h];
        if (cur == HT_EMPTY) return 0u;
        if ((cur >> 4) == v) {
            slot = h;
            return cur & 15u;
        }
    }
    return 0u;
}

// v's bits, 0 if absent
__device__ __forceinline__ uint32_t ht_find(const uint32_t *ht, uint32_t v) {
    uint32_t h = ht_slot(v);
    for (int i = 0; i < HT_SLOTS; i++, h = (h + 1u) & (HT_SLOTS - 1)) {
        const uint32_t cur = ht[h];
        if (cur == HT_EMPTY) return 0u;
        if ((cur >> 4) == v) return cur & 15u;
    }
    return 0u;
}

template <int K, bool EDGE>
__global__ void __launch_bounds__(256, 4) count_kernel(GraphDesc single, const GraphDesc *__restrict__ multi,
                                                   const Task *__restrict__ tasks, int64_t ntasks,
                                                   unsigned long long *qhead, const uint8_t *__restrict__ lut_g,
                                                   int32_t rank_lo, int32_t rank_hi, int *status,
                                                   unsigned long long *stats, EdgeDesc E) {
    constexpr int C = (K == 3) ? 13 : 199;
    constexpr int NIDX = 1 << (K * (K - 1));
    constexpr int NH = (K == 3) ? 2 : 3;  // histograms per warp: r, a (, b)
    extern __shared__ unsigned long long smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    uint32_t *lists = (uint32_t *)(smem + (size_t)nwarps * NH * C) + (size_t)warp * STAGE_WORDS;
    uint8_t *lut = (uint8_t *)((uint32_t *)(smem + (size_t)nwarps * NH * C) + (size_t)nwarps * STAGE_WORDS);
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
    // sets this lane credited (each set is credited by exactly one lane);
    // summed into stats[0] when the warp runs out of tasks
    unsigned long long nsets = 0ull;

    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(qhead, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= (unsigned long long)ntasks) {
            if (stats) {
                for (int o = 16; o > 0; o >>= 1) nsets += __shfl_xor_sync(0xffffffffu, nsets, o);
                if (lane == 0 && nsets) atomicAdd(stats, nsets);
            }
            break;
        }
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
        const View VP = stage(g, lists, pb, pe, STAGE_P, lane);  // N+(r)
        // one set: credit its members (r, a, b through the warp's histograms,
        // the innermost member directly) or, per edge, its edges
        auto set3 = [&](uint32_t a, uint32_t b, int32_t ia, int32_t ib, uint32_t fab, uint32_t cls) {
            if constexpr (EDGE) {
                edge_set<3>(g, E, out, (uint32_t)r, a, b, 0u, ia, ib, -1, fab, 0u, 0u, cls);
            } else {
                hinc(hist_a, cls);  // r gets a's totals when a is flushed
                credit(g, out, G.new2old, b, C, cls);
            }
            nsets++;
        };
        auto set4 = [&](uint32_t a, uint32_t b, uint32_t c, int32_t ia, int32_t ib, int32_t ic, uint32_t fab,
                        uint32_t fac, uint32_t fbc, uint32_t cls) {
            if constexpr (EDGE) {
                edge_set<4>(g, E, out, (uint32_t)r, a, b, c, ia, ib, ic, fab, fac, fbc, cls);
            } else {
                hinc(hist_a, cls);  // r gets a's totals when a is flushed
                hinc(hist_b, cls);
                credit(g, out, G.new2old, c, C, cls);
            }
            nsets++;
        };

        if (K == 3 && VP.s != nullptr) {
            // k = 3 flattened over the task's depth-1 vertices a: a-items (32
            // at a time, one per lane), each with the candidates b in P after
            // a (star) and b in N(a) above r, not in P (path); lanes take
            // consecutive (a, b) items.  Credits to a are combined over the
            // lanes holding the same (a, class).
            const int32_t na = task.j < L ? (L - 1 - task.j) / task.stride + 1 : 0;
            // per a-item of a pass: h(a, x) for every member x of P (2 bits per
            // position, at most 64 positions: 4 words), in the warp's N(a) staging
            // area, which this walk does not use -- set by a's own-row items, which
            // come first, and read by the star items, which then search no row
            uint32_t *fmask = lists + STAGE_P;  // [32][4]
            for (int32_t it0 = 0; it0 < na; it0 += 32) {
                const int32_t it = it0 + lane;
                uint32_t a = 0u, fra = 0u;
                int32_t ia = 0, cnt0 = 0, cnt1 = 0;  // items from a's row / star items
                int64_t a_up = 0, a_end = 0;
                if (it < na) {
                    ia = task.j + it * task.stride;
                    const uint32_t ea = VP.s[ia];
                    a = ea >> 2;
                    fra = ea & 3u;
                    if (in_bounds(g, a < G.n)) {
                        const int64_t ab = __ldg(g.rowptr + a);
                        a_end = __ldg(g.rowptr + a + 1);
                        if (in_bounds(g, ab >= 0 && ab <= a_end && a_end <= G.nnz)) {
                            a_up = upper_row(g.col, ab, a_end, (uint32_t)r);
                            cnt0 = (int32_t)(a_end - a_up);
                            cnt1 = L - 1 - ia;
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; q++) fmask[lane * 4 + q] = 0u;
                __syncwarp();
                for (int grp = 0; grp < 2; grp++) {
                    const int32_t cnt = grp == 0 ? cnt0 : cnt1;
                    int32_t incl = cnt;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += y;
                    }
                    const int32_t total = __shfl_sync(0xffffffffu, incl, 31);
                    for (int32_t j0 = 0; j0 < total; j0 += 32) {
                        const int32_t j = j0 + lane;
                        int32_t w = 0;
#pragma unroll
                        for (int sh = 16; sh >= 1; sh >>= 1)
                            if (__shfl_sync(0xffffffffu, incl, w + sh - 1) <= j) w += sh;
                        const uint32_t ao = __shfl_sync(0xffffffffu, a, w);
                        const uint32_t frao = __shfl_sync(0xffffffffu, fra, w);
                        const int32_t iao = __shfl_sync(0xffffffffu, ia, w);
                        const int32_t start = __shfl_sync(0xffffffffu, incl, w) - __shfl_sync(0xffffffffu, cnt, w);
                        const int64_t aupo = __shfl_sync(0xffffffffu, a_up, w);
                        uint32_t b = 0u, cls = 255u, fab = 0u;
                        int32_t ib = -1;  // position of b in N+(r) (star), else -1
                        if (j < total) {
                            const int32_t off = j - start;
                            if (grp == 0) {  // path: b in N(a) above r, not in P
                                const uint32_t eb = __ldg(g.col + aupo + off);
                                b = eb >> 2;
                                fab = eb & 3u;
                                const int32_t px = view_pos(VP, b);
                                if (px >= 0) {
                                    // b in P and adjacent to a: a star's flag, not a path
                                    atomicOr(fmask + w * 4 + (px >> 4), fab << ((px & 15) * 2));
                                } else {
                                    cls = lut[mask3(frao, 0u, fab)];
                                }
                            } else {  // star: b in P after a
                                ib = iao + 1 + off;
                                const uint32_t eb = VP.s[ib];
                                b = eb >> 2;
                                fab = (fmask[w * 4 + (ib >> 4)] >> ((ib & 15) * 2)) & 3u;
                                cls = lut[mask3(frao, eb & 3u, fab)];
                            }
                            if (cls != 255u && !in_bounds(g, cls < (uint32_t)C)) cls = 255u;
                        }
                        const bool hit = cls != 255u;
                        if (hit) {
                            if constexpr (EDGE) {
                                edge_set<3>(g, E, out, (uint32_t)r, ao, b, 0u, iao, ib, -1, fab, 0u, 0u, cls);
                            } else {
                                credit(g, out, G.new2old, b, C, cls);
                            }
                            nsets++;
                        }
                        if constexpr (!EDGE) {
                            // a's and r's credits once per group of lanes holding the same (a, class)
                            const unsigned long long key = hit ? (((unsigned long long)ao << 8) | cls) : (~0ull - lane);
                            const uint32_t grpm = __match_any_sync(0xffffffffu, key);
                            if (hit && lane == __ffs(grpm) - 1) {
                                credit_n(g, out, G.new2old, ao, C, cls, __popc(grpm));
                                hadd(hist_r, cls, (unsigned long long)__popc(grpm));
                            }
                        }
                    }
                    __syncwarp();  // a's flags complete before the star items
                }
            }
        } else
        for (int32_t ia = task.j; ia < L; ia += task.stride) {
            const uint32_t ea = view_entry(g, VP, pb + ia);
            const uint32_t a = ea >> 2, fra = ea & 3u;
            if (!in_bounds(g, a < G.n)) break;
            const int64_t a_beg = __ldg(g.rowptr + a), a_end = __ldg(g.rowptr + a + 1);
            if (!in_bounds(g, a_beg >= 0 && a_beg <= a_end && a_end <= G.nnz)) break;
            const int64_t a_up = upper_row(g.col, a_beg, a_end, (uint32_t)r);  // N(a) with rank > r
            const View VA{nullptr, a_up, a_end};
            if (K == 3) {
                // star: b in P after a
                for (int32_t ib = ia + 1 + lane; ib < L; ib += 32) {
                    const uint32_t eb = view_entry(g, VP, pb + ib);
                    const uint32_t b = eb >> 2, frb = eb & 3u;
                    const uint32_t fab = view_find(g, VA, b);
                    const uint32_t cls = lut[mask3(fra, frb, fab)];
                    if (!in_bounds(g, cls < (uint32_t)C)) continue;
                    set3(a, b, ia, ib, fab, cls);
                }
                // path: b in N(a) \ N(r), b > r
                for (int64_t x = a_up + lane; x < a_end; x += 32) {
                    const uint32_t eb = view_entry(g, VA, x);
                    const uint32_t b = eb >> 2;
                    if (view_find(g, VP, b)) continue;
                    const uint32_t cls = lut[mask3(fra, 0u, eb & 3u)];
                    if (!in_bounds(g, cls < (uint32_t)C)) continue;
                    set3(a, b, ia, -1, eb & 3u, cls);
                }
            } else if (VP.s != nullptr && a_end - a_up <= STAGE_A && G.n <= HT_MAX_N) {
                // Flattened walk of every set with this a, lanes on consecutive
                // (b, c) work items (short candidate lists would leave most
                // lanes idle).  b-items: the members of P after a, then the
                // entries of N(a) above r that are not in P.  Candidates c of a
                // b in P: the members of P after b (1,1,1), N(a) \ P (1,1,2),
                // N(b) \ N(a) \ P (1,1,2); of a b at depth 2: N(a) \ P after b
                // (1,2,2), N(b) \ (N(a) u P) (1,2,3) -- the same sets, shapes and
                // member order as the nested loops below.  32 b-items at a time,
                // one per lane; the owner of work item j is found by a binary
                // search over the lanes' inclusive sums.  Credits to b are
                // combined over the lanes holding the same (b, class).
                const View NA = stage(g, lists + STAGE_P, a_up, a_end, STAGE_A, lane);  // N(a) above r
                const int32_t la = (int32_t)(a_end - a_up);
                const int32_t n1 = L - 1 - ia;
                const int32_t nitems = n1 + la;
                // Membership in N+(r) and in N(a) above r, with the flags from r
                // and from a, in one open-addressing table: word = (vertex << 4) |
                // (h(a, v) << 2) | h(r, v), empty = ~0.  It lives in the warp's
                // b-histogram area (zero between b's, unused on this walk; 256 of
                // its 2C words for at most 64 + 128 keys) and is zeroed again after.
                static_assert(K == 3 || 2 * C >= HT_SLOTS + 128, "the table and signatures must fit the b-histogram area");
                uint32_t *ht = hist_b.lo;
                for (int i = lane; i < HT_SLOTS; i += 32) ht[i] = HT_EMPTY;
                __syncwarp();
                for (int32_t p = lane; p < L; p += 32) ht_insert(ht, VP.s[p] >> 2, VP.s[p] & 3u);
                __syncwarp();
                for (int32_t x = lane; x < la; x += 32) ht_insert(ht, NA.s[x] >> 2, (NA.s[x] & 3u) << 2);
                __syncwarp();
                // per b-item of a pass: a 128-bit signature of which table slots
                // (mod 128) hold a neighbour of b -- set by b's own-row items, which
                // come first, read by the staged-list items, which search b's row only
                // where their slot's bit is set
                uint32_t *sig = ht + HT_SLOTS;  // [32][4]
                for (int32_t it0 = 0; it0 < nitems; it0 += 32) {
                    const int32_t it = it0 + lane;
                    uint32_t b = 0u, frb = 0u, fab = 0u;
                    int32_t cnt0 = 0, cnt1 = 0, pos = 0;  // items from b's row / from the staged lists
                    int64_t b_up = 0, b_end = 0;
                    if (it < nitems) {
                        const bool inp = it < n1;
                        pos = inp ? ia + 1 + it : it - n1;
                        const uint32_t eb = inp ? VP.s[pos] : NA.s[pos];
                        b = eb >> 2;
                        bool ok = in_bounds(g, b < G.n);
                        const uint32_t hb = ht_find(ht, b);
                        if (inp) {
                            frb = eb & 3u;
                            fab = hb >> 2;
                        } else {
                            fab = eb & 3u;
                            ok = ok && (hb & 3u) == 0u;  // a member of P is not at depth 2
                        }
                        if (ok) {
                            const int64_t bb = __ldg(g.rowptr + b);
                            b_end = __ldg(g.rowptr + b + 1);
                            if (in_bounds(g, bb >= 0 && bb <= b_end && b_end <= G.nnz)) {
                                b_up = upper_row(g.col, bb, b_end, (uint32_t)r);
                                cnt0 = (int32_t)(b_end - b_up);
                                cnt1 = inp ? (L - 1 - pos) + la : (la - pos - 1);
                            }
                        }
                    }
#pragma unroll
                    for (int q = 0; q < 4; q++) sig[lane * 4 + q] = 0u;
                    __syncwarp();
                    for (int grp = 0; grp < 2; grp++) {
                        const int32_t cnt = grp == 0 ? cnt0 : cnt1;
                        int32_t incl = cnt;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                            if (lane >= o) incl += y;
                        }
                        const int32_t total = __shfl_sync(0xffffffffu, incl, 31);
                        for (int32_t j0 = 0; j0 < total; j0 += 32) {
                            const int32_t j = j0 + lane;
                            int32_t w = 0;
#pragma unroll
                            for (int sh = 16; sh >= 1; sh >>= 1)
                                if (__shfl_sync(0xffffffffu, incl, w + sh - 1) <= j) w += sh;
                            const uint32_t bo = __shfl_sync(0xffffffffu, b, w);
                            const uint32_t frbo = __shfl_sync(0xffffffffu, frb, w);
                            const uint32_t fabo = __shfl_sync(0xffffffffu, fab, w);
                            const int32_t poso = __shfl_sync(0xffffffffu, pos, w);
                            const int32_t start = __shfl_sync(0xffffffffu, incl, w) - __shfl_sync(0xffffffffu, cnt, w);
                            const int64_t bupo = __shfl_sync(0xffffffffu, b_up, w);
                            const int64_t bendo = __shfl_sync(0xffffffffu, b_end, w);
                            const bool inpo = it0 + w < n1;
                            uint32_t c = 0u, cls = 255u, fac_s = 0u, fbc_s = 0u;
                            int32_t ic = -1;  // position of c in N+(r), else -1 (per-edge credits)
                            if (j < total) {
                                // one path for every shape: the candidate's source and which
                                // memberships rule it out
                                //   b's row:      N(b) \ N(a) \ P (1,1,2) | N(b) \ (N(a) u P) (1,2,3)
                                //   staged lists: b in P: P after b (1,1,1) | N(a) \ P (1,1,2);
                                //                 b deeper: N(a) \ P after b (1,2,2)
                                const int32_t off = j - start;
                                int32_t sidx = 0;
                                bool not_p = true;
                                if (grp == 1) {
                                    if (inpo) {
                                        const int32_t n111 = L - 1 - poso;
                                        if (off < n111) {
                                            sidx = poso + 1 + off;
                                            not_p = false;
                                        } else {
                                            sidx = STAGE_P + (off - n111);
                                        }
                                    } else {
                                        sidx = STAGE_P + poso + 1 + off;
                                    }
                                }
                                const uint32_t ec = grp == 0 ? __ldg(g.col + bupo + off) : lists[sidx];
                                c = ec >> 2;
                                uint32_t slot = 0u;
                                const uint32_t hc = ht_find_slot(ht, c, slot);
                                const uint32_t frc = hc & 3u, fac = hc >> 2;
                                if (grp == 0) {
                                    if (hc != 0u) {
                                        // c in P or N(a) and adjacent to b: not a set here, but
                                        // b's signature learns of it
                                        atomicOr(sig + w * 4 + ((slot >> 5) & 3u), 1u << (slot & 31u));
                                    } else {
                                        fbc_s = ec & 3u;
                                        cls = lut[mask4(fra, inpo ? frbo : 0u, 0u, fabo, 0u, fbc_s)];
                                    }
                                } else if (!(not_p && frc != 0u)) {
                                    // a candidate from N(a) must not be in P
                                    const uint32_t sb = sig[w * 4 + ((slot >> 5) & 3u)];
                                    const uint32_t fbc = ((sb >> (slot & 31u)) & 1u) ? search_row(g.col, bupo, bendo, c) : 0u;
                                    cls = lut[mask4(fra, inpo ? frbo : 0u, frc, fabo, fac, fbc)];
                                    fac_s = fac;
                                    fbc_s = fbc;
                                    ic = not_p ? -1 : sidx;
                                }
                                if (cls != 255u && !in_bounds(g, cls < (uint32_t)C)) cls = 255u;
                            }
                            const bool hit = cls != 255u;
                            if (hit) {
                                if constexpr (EDGE) {
                                    edge_set<4>(g, E, out, (uint32_t)r, a, bo, c, ia, inpo ? poso : -1, ic, fabo, fac_s,
                                                fbc_s, cls);
                                } else {
                                    credit(g, out, G.new2old, c, C, cls);
                                }
                                nsets++;
                            }
                            if constexpr (!EDGE) {
                                // b's and a's credits once per group of lanes holding the same
                                // (b, class); r gets a's totals when a is flushed
                                const unsigned long long key = hit ? (((unsigned long long)bo << 8) | cls) : (~0ull - lane);
                                const uint32_t grpm = __match_any_sync(0xffffffffu, key);
                                if (hit && lane == __ffs(grpm) - 1) {
                                    credit_n(g, out, G.new2old, bo, C, cls, __popc(grpm));
                                    hadd(hist_a, cls, (unsigned long long)__popc(grpm));
                                }
                            }
                        }
                        __syncwarp();  // b's signatures complete before the staged-list items
                    }
                }
                __syncwarp();
                for (int i = lane; i < HT_SLOTS + 128; i += 32) ht[i] = 0u;  // the b-histogram again
                __syncwarp();
            } else {
                // (A1) b in P after a
                for (int32_t ib = ia + 1; ib < L; ib++) {
                    const uint32_t eb = view_entry(g, VP, pb + ib);
                    const uint32_t b = eb >> 2, frb = eb & 3u;
                    if (!in_bounds(g, b < G.n)) break;
                    const uint32_t fab = view_find(g, VA, b);
                    const int64_t b_beg = __ldg(g.rowptr + b), b_end = __ldg(g.rowptr + b + 1);
                    if (!in_bounds(g, b_beg >= 0 && b_beg <= b_end && b_end <= G.nnz)) break;
                    const int64_t b_up = upper_row(g.col, b_beg, b_end, (uint32_t)r);
                    const View VB{nullptr, b_up, b_end};
                    // (1,1,1): c in P after b
                    for (int32_t ic = ib + 1 + lane; ic < L; ic += 32) {
                        const uint32_t ec = view_entry(g, VP, pb + ic);
                        const uint32_t c = ec >> 2, frc = ec & 3u;
                        const uint32_t fac = view_find(g, VA, c), fbc = view_find(g, VB, c);
                        const uint32_t cls = lut[mask4(fra, frb, frc, fab, fac, fbc)];
                        if (!in_bounds(g, cls < (uint32_t)C)) continue;
                        set4(a, b, c, ia, ib, ic, fab, fac, fbc, cls);
                    }
                    // (1,1,2) with c in N(a) \ N(r), c > r
                    for (int64_t x = a_up + lane; x < a_end; x += 32) {
                        const uint32_t ec = view_entry(g, VA, x);
                        const uint32_t c = ec >> 2;
                        if (view_find(g, VP, c)) continue;
                        const uint32_t fbc = view_find(g, VB, c);
                        const uint32_t cls = lut[mask4(fra, frb, 0u, fab, ec & 3u, fbc)];
                        if (!in_bounds(g, cls < (uint32_t)C)) continue;
                        set4(a, b, c, ia, ib, -1, fab, ec & 3u, fbc, cls);
                    }
                    // (1,1,2) with c in N(b) \ N(a) \ N(r), c > r
                    for (int64_t x = b_up + lane; x < b_end; x += 32) {
                        const uint32_t ec = view_entry(g, VB, x);
                        const uint32_t c = ec >> 2;
                        if (view_find(g, VP, c)) continue;
                        if (view_find(g, VA, c)) continue;
                        const uint32_t cls = lut[mask4(fra, frb, 0u, fab, 0u, ec & 3u)];
                        if (!in_bounds(g, cls < (uint32_t)C)) continue;
                        set4(a, b, c, ia, ib, -1, fab, 0u, ec & 3u, cls);
                    }
                    if (!EDGE) flush_hist(g, hist_b, C, out, row_of(G.new2old, b), lane);
                }
                // (A2) b in N(a) \ N(r), b > r
                for (int64_t xb = a_up; xb < a_end; xb++) {
                    const uint32_t eb = view_entry(g, VA, xb);
                    const uint32_t b = eb >> 2, fab = eb & 3u;
                    if (!in_bounds(g, b < G.n)) break;
                    if (view_find(g, VP, b)) continue;  // warp-uniform
                    const int64_t b_beg = __ldg(g.rowptr + b), b_end = __ldg(g.rowptr + b + 1);
                    if (!in_bounds(g, b_beg >= 0 && b_beg <= b_end && b_end <= G.nnz)) break;
                    const int64_t b_up = upper_row(g.col, b_beg, b_end, (uint32_t)r);
                    const View VB{nullptr, b_up, b_end};
                    // (1,2,2): c in N(a) after b, c not in N(r)
                    for (int64_t x = xb + 1 + lane; x < a_end; x += 32) {
                        const uint32_t ec = view_entry(g, VA, x);
                        const uint32_t c = ec >> 2;
                        if (view_find(g, VP, c)) continue;
                        const uint32_t fbc = view_find(g, VB, c);
                        const uint32_t cls = lut[mask4(fra, 0u, 0u, fab, ec & 3u, fbc)];
                        if (!in_bounds(g, cls < (uint32_t)C)) continue;
                        set4(a, b, c, ia, -1, -1, fab, ec & 3u, fbc, cls);
                    }
                    // (1,2,3): c in N(b), c > r, not in N(r), not adjacent to a
                    for (int64_t x = b_up + lane; x < b_end; x += 32) {
                        const uint32_t ec = view_entry(g, VB, x);
                        const uint32_t c = ec >> 2;
                        if (view_find(g, VP, c)) continue;
                        if (view_find(g, VA, c)) continue;
                        const uint32_t cls = lut[mask4(fra, 0u, 0u, fab, 0u, ec & 3u)];
                        if (!in_bounds(g, cls < (uint32_t)C)) continue;
                        set4(a, b, c, ia, -1, -1, fab, 0u, ec & 3u, cls);
                    }
                    if (!EDGE) flush_hist(g, hist_b, C, out, row_of(G.new2old, b), lane);
                }
            }
            if (!EDGE) flush_hist_into(g, hist_a, hist_r, C, out, row_of(G.new2old, a), lane);
        }
        if (!EDGE) flush_hist(g, hist_r, C, out, row_of(G.new2old, r), lane);
    }
}

// out[new2old[r]] = acc[r] (+ the depth-3 credits d3[r], k = 4), one warp
// per row (coalesced row copies).  Column d of d3 holds the sets r' - x - b - c
// credited to c whose class is the d-th smallest of the depth-3 path classes
// (d3_column); unused columns stay zero.
// Accumulator column c goes to output column colmap[c] of Cout (its class,
// or its undirected column), and nowhere when that is 255.
__global__ void unrelabel_rows(const uint64_t *__restrict__ acc, const uint64_t *__restrict__ d3, int d3_narrow,
                               const uint8_t *__restrict__ lut, const int32_t *__restrict__ new2old, int32_t n,
                               int C, const uint8_t *__restrict__ colmap, int Cout, uint64_t *__restrict__ out) {
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
                if (d3cls[j] == c)
                    v += d3_narrow ? (uint64_t)__ldg(reinterpret_cast<const uint32_t *>(d3) + r * VDMC_D3_COLS + j)
                                   : __ldg(d3 + r * VDMC_D3_COLS + j);
        }
        const int oc = (int)__ldg(colmap + c);
        if (oc < Cout) out[(int64_t)o * Cout + oc] = v;
    }
}

// Algorithmic bytes of one count (the cost model of the section on efficacy
// on simulated graphs: work proportional to the neighbourhoods visited).
// Per root r with P = N+(r): the adjacency rows the method must stream,
// 4 bytes per entry -- N(r), N(a) for every a in P and, for k = 4, N(b) for
// every distinct depth-2 vertex b (rank > r, not adjacent to r, adjacent to
// some a in P).  One CTA per root; the depth-2 vertices already seen for this
// root are a bitmap over ranks (shared memory when it fits, else a slice of
// `gbits` per CTA), cleared again before the next root.  Also counts N(b) once
// per (a, b) adjacency, the volume an enumeration without reuse streams.
// tot: [0] entries of N(r), [1] of N(a), [2] of N(b) per distinct b, [3] of
// N(b) per (a, b).
__global__ void __launch_bounds__(256) work_model_kernel(Csr g, int32_t n, int k, uint32_t *gbits, int32_t words,
                                                         int in_smem, unsigned long long *tot) {
    extern __shared__ uint32_t sbits[];
    uint32_t *bits = in_smem ? sbits : gbits + (size_t)blockIdx.x * (size_t)words;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = 8;
    for (int i = tid; i < words; i += 256) bits[i] = 0u;
    __syncthreads();
    unsigned long long cr = 0, ca = 0, cbd = 0, cbu = 0;
    for (int64_t r = blockIdx.x; r < n; r += gridDim.x) {
        const int64_t rb = __ldg(g.rowptr + r), pb = __ldg(g.pbeg + r), pe = __ldg(g.rowptr + r + 1);
        if (tid == 0) cr += (unsigned long long)(pe - rb);
        if (pe == pb) continue;
        for (int64_t x = pb + tid; x < pe; x += 256) {
            const uint32_t a = __ldg(g.col + x) >> 2;
            ca += (unsigned long long)(__ldg(g.rowptr + a + 1) - __ldg(g.rowptr + a));
        }
        if (k != 4) continue;
        for (int pass = 0; pass < 2; pass++) {  // 0: mark and count, 1: clear
            for (int64_t x = pb + warp; x < pe; x += NW) {
                const uint32_t a = __ldg(g.col + x) >> 2;
                const int64_t ab = __ldg(g.rowptr + a), ae = __ldg(g.rowptr + a + 1);
                for (int64_t y = upper_row(g.col, ab, ae, (uint32_t)r) + lane; y < ae; y += 32) {
                    const uint32_t b = __ldg(g.col + y) >> 2;
                    if (search_row(g.col, pb, pe, b)) continue;  // b in P: depth 1
                    if (pass == 1) {
                        bits[b >> 5] = 0u;
                        continue;
                    }
                    const unsigned long long db = (unsigned long long)(__ldg(g.rowptr + b + 1) - __ldg(g.rowptr + b));
                    cbu += db;
                    const uint32_t m = 1u << (b & 31u);
                    if (!(atomicOr(bits + (b >> 5), m) & m)) cbd += db;
                }
            }
            __syncthreads();
        }
    }
    unsigned long long v[4] = {cr, ca, cbd, cbu};
    for (int i = 0; i < 4; i++) {
        for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
        if (lane == 0 && v[i]) atomicAdd(tot + i, v[i]);
    }
}

// Estimated work of each root, for splitting the roots into ranges of
// equal work (the root-chunk distribution of the Discussion): the adjacency
// entries its count streams -- N(r), N(a) for a in P and, for k = 4, N(b) for
// every (a, b) with b a depth-2 vertex -- plus, for a root of the
// warp-per-task kernel (L < hub_min_l, or hub_min_l = 0), the C(L, k-1)
// star-shaped sets it enumerates one by one.  One warp per root.
__global__ void root_cost_kernel(Csr g, int32_t n, int k, int32_t hub_min_l, unsigned long long *cost) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = wid; r < n; r += nw) {
        const int64_t rb = __ldg(g.rowptr + r), pb = __ldg(g.pbeg + r), pe = __ldg(g.rowptr + r + 1);
        unsigned long long acc = 0;
        for (int64_t x = pb + lane; x < pe; x += 32) {
            const uint32_t a = __ldg(g.col + x) >> 2;
            const int64_t ab = __ldg(g.rowptr + a), ae = __ldg(g.rowptr + a + 1);
            acc += (unsigned long long)(ae - ab);
            if (k == 4)
                for (int64_t y = upper_row(g.col, ab, ae, (uint32_t)r); y < ae; y++) {
                    const uint32_t b = __ldg(g.col + y) >> 2;
                    if (!search_row(g.col, pb, pe, b))
                        acc += (unsigned long long)(__ldg(g.rowptr + b + 1) - __ldg(g.rowptr + b));
                }
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            const unsigned long long L = (unsigned long long)(pe - pb);
            const bool plain = hub_min_l == 0 || (int64_t)L < hub_min_l;
            unsigned long long sets = 0;
            if (plain && L >= (unsigned long long)(k - 1))
                sets = k == 3 ? L * (L - 1) / 2 : L * (L - 1) / 2 * (L - 2) / 3;
            cost[r] = acc + (unsigned long long)(pe - rb) + sets;
        }
    }
}

// Bound on the depth-3 credits of one vertex c in one count: every such set
// is a path r - x - b - c, so their number is at most
// B(c) = sum over b in N(c) of sum over x in N(b) of d(x).  When every B(c) is
// below 2^32 the credits fit 32-bit counters (half the array, so more of it
// stays in L2).  s1[v] = sum over x in N(v) of d(x); then max over c of B(c).
__global__ void d3_bound_s1(const int64_t *__restrict__ rowptr, const uint32_t *__restrict__ col, int32_t n,
                            unsigned long long *__restrict__ s1) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n) return;
    unsigned long long acc = 0;
    for (int64_t e = rowptr[w] + lane; e < rowptr[w + 1]; e += 32) {
        const uint32_t x = col[e] >> 2;
        acc += (unsigned long long)(rowptr[x + 1] - rowptr[x]);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) s1[w] = acc;
}

__global__ void d3_bound_max(const int64_t *__restrict__ rowptr, const uint32_t *__restrict__ col, int32_t n,
                             const unsigned long long *__restrict__ s1, unsigned long long *__restrict__ mx) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n) return;
    unsigned long long acc = 0;
    for (int64_t e = rowptr[w] + lane; e < rowptr[w + 1]; e += 32) acc += s1[col[e] >> 2];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) atomicMax(mx, acc);
}

size_t smem_bytes(int k, int warps) {
    int C = k == 3 ? 13 : 199, NH = k == 3 ? 2 : 3;
    return (size_t)warps * NH * C * sizeof(unsigned long long) + (size_t)warps * STAGE_WORDS * sizeof(uint32_t) +
           ((size_t)1 << (k * (k - 1)));
}

vdmc_status launch_count(int k, const GraphDesc &single, const GraphDesc *multi, const Task *tasks,
                         int64_t ntasks, unsigned long long *qhead, int32_t lo, int32_t hi, int *status,
                         unsigned long long *stats, cudaStream_t s, bool edge = false, EdgeDesc E = EdgeDesc{}) {
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
    auto kern = edge ? ((k == 3) ? count_kernel<3, true> : count_kernel<4, true>)
                     : ((k == 3) ? count_kernel<3, false> : count_kernel<4, false>);
    // per-kernel attribute: the largest size any schedule uses, so that host
    // threads with different schedules never lower it under each other
    VDMC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(k, 8)));
    int per_sm = 0;
    VDMC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) per_sm = 1;
    if (sch.blocks_per_sm > 0) per_sm = std::min(per_sm, sch.blocks_per_sm);
    int64_t grid = (int64_t)sms * per_sm;
    int64_t need = (ntasks + warps - 1) / warps;
    if (grid > need) grid = std::max<int64_t>(1, need);
    VDMC_CUDA_TRY(cudaMemsetAsync(qhead, 0, sizeof(unsigned long long), s));
    if (ntasks > 0) {
        kern<<<(unsigned)grid, threads, smem, s>>>(single, multi, tasks, ntasks, qhead, lut, lo, hi, status, stats,
                                                   E);
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
    vdmc_free(g->tasks, s);  // stream-ordered behind the last count on s
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
    if (e == cudaSuccess) e = vdmc_malloc(&g->tasks, sizeof(Task) * (size_t)total, s);
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
    cudaStreamCaptureStatus cs0 = cudaStreamCaptureStatusNone;
    VDMC_CUDA_TRY(cudaStreamIsCapturing(s, &cs0));
    // the previous build or count of this graph (on any stream) comes first:
    // its buffers may be freed or reused below
    if (cs0 == cudaStreamCaptureStatusNone) VDMC_CUDA_TRY(cudaStreamWaitEvent(s, g->ev_done, 0));
    vdmc_schedule_t sch;
    vdmc_current_schedule(&sch);
    if (g->tasks_a_chunk != sch.a_chunk || g->hub_min_l != sch.hub_min_l) {
        vdmc_status st = vdmc_build_tasks(g, sch.a_chunk, sch.hub_min_l, s);
        if (st != VDMC_OK) return st;
    }
    // Credits accumulate in a rank-space array owned by the graph (no id-map
    // load in front of each atomic); one coalesced pass then writes every row
    // to its original id in `out`.
    if (!g->racc && g->n > 0)
        VDMC_CUDA_TRY(vdmc_malloc(&g->racc, sizeof(uint64_t) * (size_t)g->n * VDMC_MAX_CLASSES, s));
    uint64_t *acc = g->racc;
    if (g->n > 0) VDMC_CUDA_TRY(cudaMemsetAsync(acc, 0, sizeof(uint64_t) * (size_t)g->n * C, s));
    if (g->stats) VDMC_CUDA_TRY(cudaMemsetAsync(g->stats, 0, sizeof(unsigned long long) * VDMC_NSTATS, s));
    // depth-3 credits of the root-per-CTA kernel (k = 4): one column per path
    // class (16 per vertex) instead of 199, so that more reductions stay in L2
    uint64_t *d3 = nullptr;
    bool narrow = false;
    if (k == 4 && g->nhubs > 0 && g->n > 0) {
        if (g->d3_mode == 0) {
            // once per graph: can a depth-3 counter reach 2^32 in one count?
            unsigned long long *s1 = nullptr, *mx = nullptr, hmx = 0;
            VDMC_CUDA_TRY(vdmc_malloc(&s1, sizeof(unsigned long long) * (size_t)g->n, s));
            cudaError_t e = vdmc_malloc(&mx, sizeof(unsigned long long), s);
            const unsigned blocks = (unsigned)(((int64_t)g->n * 32 + 255) / 256);
            if (e == cudaSuccess) e = cudaMemsetAsync(mx, 0, sizeof(unsigned long long), s);
            if (e == cudaSuccess) {
                d3_bound_s1<<<blocks, 256, 0, s>>>(g->rowptr, g->col, g->n, s1);
                d3_bound_max<<<blocks, 256, 0, s>>>(g->rowptr, g->col, g->n, s1, mx);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaMemcpyAsync(&hmx, mx, sizeof hmx, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            vdmc_free(s1, s);
            vdmc_free(mx, s);
            if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? VDMC_ERR_OOM : VDMC_ERR_CUDA;
            g->d3_mode = hmx < (1ull << 32) ? 1 : 2;
        }
        if (!g->d3acc) VDMC_CUDA_TRY(vdmc_malloc(&g->d3acc, sizeof(uint64_t) * (size_t)g->n * VDMC_D3_COLS, s));
        if (!g->d3w) VDMC_CUDA_TRY(vdmc_malloc(&g->d3w, sizeof(uint64_t) * (size_t)g->n * 9, s));
        d3 = g->d3acc;
        narrow = g->d3_mode == 1 && sch.d3_bits != 64;
        const size_t width = narrow ? sizeof(uint32_t) : sizeof(uint64_t);
        VDMC_CUDA_TRY(cudaMemsetAsync(d3, 0, width * (size_t)g->n * VDMC_D3_COLS, s));
        VDMC_CUDA_TRY(cudaMemsetAsync(g->d3w, 0, width * (size_t)g->n * 9, s));
    }
    const uint8_t *lut = nullptr;
    VDMC_CUDA_TRY(device_lut(k, &lut));
    GraphDesc d{g->rowptr, g->col, g->pbeg, nullptr, acc, g->n, 0, g->nnz};
    if (g->nhubs > 0) {
        // the root-per-CTA kernel runs on the graph's side stream, overlapped
        // with the warp kernel; the caller's stream waits for both
        VDMC_CUDA_TRY(cudaEventRecord(g->ev_fork, s));
        VDMC_CUDA_TRY(cudaStreamWaitEvent(g->side, g->ev_fork, 0));
        vdmc_status st = vdmc_hub_launch(g, k, acc, d3, narrow ? 1 : 0, d3 ? g->d3w : nullptr, lut, lo, hi,
                                          sch.hub_blocks_per_sm,
                                          sch.hub_split, sch.hub_split_roots, sch.hub_warps, g->side);
        if (st != VDMC_OK) return st;
        VDMC_CUDA_TRY(cudaEventRecord(g->ev_join, g->side));
    }
    vdmc_status st = launch_count(k, d, nullptr, g->tasks, g->ntasks, g->qhead, lo, hi, g->status, g->stats, s);
    if (g->nhubs > 0) VDMC_CUDA_TRY(cudaStreamWaitEvent(s, g->ev_join, 0));
    if (st != VDMC_OK) return st;
    if (g->n > 0) {
        const uint8_t *colmap = nullptr;
        VDMC_CUDA_TRY(vdmc_device_colmap(k, g->undirected != 0, &colmap));
        const int Cout = g->undirected ? vdmc_num_classes_undirected(k) : C;
        unrelabel_rows<<<(unsigned)((g->n + 7) / 8), 256, 0, s>>>(acc, d3, narrow ? 1 : 0, lut, g->new2old, g->n,
                                                                   C, colmap, Cout, out);
        VDMC_CUDA_TRY(cudaGetLastError());
    }
    // the graph's memory is released behind this point (vdmc_graph_destroy);
    // a captured count (batch plans) is ordered by its replays instead
    if (cs0 == cudaStreamCaptureStatusNone) VDMC_CUDA_TRY(cudaEventRecord(g->ev_done, s));
    return VDMC_OK;
}

extern "C" int vdmc_graph_num_classes(const vdmc_graph *g, int k) {
    if (!g || (k != 3 && k != 4)) return -1;
    return g->undirected ? vdmc_num_classes_undirected(k) : vdmc_num_classes(k);
}

// Per-edge counts (edges.cu builds the edge index): the warp-per-task kernel
// over every root, crediting edges; out has one row per edge of G_U in
// (min, max) original-id order.
vdmc_status vdmc_count_edges_internal(vdmc_graph *g, int k, uint64_t *out, cudaStream_t s) {
    if (!g || (k != 3 && k != 4)) return VDMC_ERR_INVALID_ARG;
    const int64_t ne = g->nnz / 2;
    if (!out && ne > 0) return VDMC_ERR_INVALID_ARG;
    VDMC_CUDA_TRY(cudaStreamWaitEvent(s, g->ev_done, 0));
    vdmc_status st = vdmc_edge_index(g, s);
    if (st != VDMC_OK) return st;
    vdmc_schedule_t sch;
    vdmc_current_schedule(&sch);
    if (!g->etasks || g->etasks_a_chunk != sch.a_chunk) {
        // every root with a higher-rank neighbour (the root-per-CTA kernel
        // has no per-edge form)
        vdmc_free(g->etasks, s);
        g->etasks = nullptr;
        g->netasks = 0;
        const int32_t n = g->n;
        int64_t *cnt = nullptr;
        VDMC_CUDA_TRY(vdmc_malloc(&cnt, sizeof(int64_t) * ((size_t)n + 1), s));
        if (n > 0) task_counts<<<(n + 255) / 256, 256, 0, s>>>(g->rowptr, g->pbeg, n, sch.a_chunk, 0, cnt);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = vdmc_exclusive_scan_i64(cnt, cnt, n, s);
        int64_t total = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&total, cnt + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = vdmc_malloc(&g->etasks, sizeof(Task) * (size_t)total, s);
        if (e == cudaSuccess && n > 0) {
            task_fill<<<(n + 255) / 256, 256, 0, s>>>(g->rowptr, g->pbeg, cnt, n, sch.a_chunk, 0, g->etasks);
            e = cudaGetLastError();
        }
        vdmc_free(cnt, s);
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? VDMC_ERR_OOM : VDMC_ERR_CUDA;
        g->netasks = total;
        g->etasks_a_chunk = sch.a_chunk;
    }
    const int Cout = g->undirected ? vdmc_num_classes_undirected(k) : (k == 3 ? 13 : 199);
    const uint8_t *colmap = nullptr;
    VDMC_CUDA_TRY(vdmc_device_colmap(k, g->undirected != 0, &colmap));
    if (ne > 0) VDMC_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(uint64_t) * (size_t)ne * Cout, s));
    if (g->stats) VDMC_CUDA_TRY(cudaMemsetAsync(g->stats, 0, sizeof(unsigned long long) * VDMC_NSTATS, s));
    GraphDesc d{g->rowptr, g->col, g->pbeg, nullptr, out, g->n, 0, g->nnz};
    st = launch_count(k, d, nullptr, g->etasks, g->netasks, g->qhead, 0, g->n, g->status, g->stats, s, true,
                      EdgeDesc{g->ebase, g->erow, colmap, Cout});
    if (st != VDMC_OK) return st;
    VDMC_CUDA_TRY(cudaEventRecord(g->ev_done, s));
    return VDMC_OK;
}

extern "C" vdmc_status vdmc_count_edges(vdmc_graph *g, int k, uint64_t *out_dev, void *stream) {
    return vdmc_count_edges_internal(g, k, out_dev, (cudaStream_t)stream);
}

extern "C" vdmc_status vdmc_count(vdmc_graph *g, int k, uint64_t *out_dev, void *stream) {
    return vdmc_count_internal(g, k, 0, g ? g->n : 0, out_dev, (cudaStream_t)stream);
}

extern "C" vdmc_status vdmc_count_roots(vdmc_graph *g, int k, int32_t rank_lo, int32_t rank_hi, uint64_t *out_dev,
                                        void *stream) {
    if (!g || rank_lo < 0 || rank_hi < rank_lo) return VDMC_ERR_INVALID_ARG;
    return vdmc_count_internal(g, k, rank_lo, std::min(rank_hi, g->n), out_dev, (cudaStream_t)stream);
}

extern "C" vdmc_status vdmc_work_model(const vdmc_graph *g, int k, vdmc_work_model_t *m) {
    if (!g || !m || (k != 3 && k != 4)) return VDMC_ERR_INVALID_ARG;
    std::memset(m, 0, sizeof *m);
    const int C = k == 3 ? 13 : 199;
    unsigned long long h[4] = {0, 0, 0, 0};
    if (g->n > 0) {
        int dev = 0, sms = 0;
        VDMC_CUDA_TRY(cudaGetDevice(&dev));
        VDMC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int32_t words = (int32_t)(((int64_t)g->n + 31) / 32);
        const bool in_smem = words <= 46000;  // 184 KB of shared memory
        const int grid = std::max(1, std::min(g->n, sms * (in_smem ? 1 : 2)));
        unsigned long long *d = nullptr;
        uint32_t *gbits = nullptr;
        VDMC_CUDA_TRY(cudaMalloc((void **)&d, sizeof h));
        cudaError_t e = cudaMemset(d, 0, sizeof h);
        if (e == cudaSuccess && !in_smem) e = cudaMalloc((void **)&gbits, sizeof(uint32_t) * (size_t)words * grid);
        const size_t dsm = in_smem ? sizeof(uint32_t) * (size_t)words : 0;
        // per-kernel attribute: set to the largest bitmap, never lowered (see launch_hub)
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(work_model_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(46000 * sizeof(uint32_t)));
        if (e == cudaSuccess) {
            Csr c{g->rowptr, g->col, g->pbeg, g->n, g->nnz, g->status};
            work_model_kernel<<<grid, 256, dsm>>>(c, g->n, k, gbits, words, in_smem ? 1 : 0, d);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
        cudaFree(d);
        cudaFree(gbits);
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? VDMC_ERR_OOM : VDMC_ERR_CUDA;
    }
    m->entries_root = h[0];
    m->entries_depth1 = h[1];
    m->entries_depth2 = k == 4 ? h[2] : 0;
    m->entries_depth2_per_use = k == 4 ? h[3] : 0;
    m->output_bytes = 8ull * (uint64_t)g->n * (uint64_t)C + 4ull * (uint64_t)g->n;
    m->bytes = 4ull * (m->entries_root + m->entries_depth1 + m->entries_depth2) + m->output_bytes;
    m->bytes_per_use = 4ull * (m->entries_root + m->entries_depth1 + m->entries_depth2_per_use) + m->output_bytes;
    return VDMC_OK;
}

extern "C" vdmc_status vdmc_work_bytes(const vdmc_graph *g, int k, uint64_t *bytes) {
    if (!bytes) return VDMC_ERR_INVALID_ARG;
    vdmc_work_model_t m;
    const vdmc_status st = vdmc_work_model(g, k, &m);
    if (st == VDMC_OK) *bytes = m.bytes;
    return st;
}

extern "C" vdmc_status vdmc_count_stats(const vdmc_graph *g, vdmc_count_stats_t *out) {
    if (!g || !out) return VDMC_ERR_INVALID_ARG;
    unsigned long long h[VDMC_NSTATS] = {0, 0, 0, 0};
    if (g->stats) VDMC_CUDA_TRY(cudaMemcpy(h, g->stats, sizeof h, cudaMemcpyDeviceToHost));
    out->sets_plain = h[0];
    out->sets_hub = h[1];
    out->sets_hub_enumerated = h[2];
    out->sets_by_signature = h[1] >= h[2] ? h[1] - h[2] : 0;
    out->sets_enumerated = h[0] + h[2];
    return VDMC_OK;
}

extern "C" vdmc_status vdmc_root_costs(const vdmc_graph *g, int k, uint64_t *cost_dev, void *stream) {
    if (!g || (k != 3 && k != 4) || (g->n > 0 && !cost_dev)) return VDMC_ERR_INVALID_ARG;
    if (g->n == 0) return VDMC_OK;
    vdmc_schedule_t sch;
    vdmc_current_schedule(&sch);
    Csr c{g->rowptr, g->col, g->pbeg, g->n, g->nnz, g->status};
    const int64_t blocks = std::min<int64_t>(((int64_t)g->n * 32 + 255) / 256, 148 * 16);
    root_cost_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(c, g->n, k, sch.hub_min_l,
                                                                         (unsigned long long *)cost_dev);
    VDMC_CUDA_TRY(cudaGetLastError());
    return VDMC_OK;
}

extern "C" vdmc_status vdmc_set_schedule(const vdmc_schedule_t *s) {
    if (!s || s->a_chunk < 1 || s->warps_per_block < 1 || s->warps_per_block > 8 || s->blocks_per_sm < 0 ||
        s->hub_min_l < 0 || s->hub_blocks_per_sm < 1 || s->hub_blocks_per_sm > 8 || s->hub_split < 0 ||
        s->hub_split > 16 || s->hub_split_roots < 0 || (s->hub_warps != 0 && s->hub_warps != 16 && s->hub_warps != 32) ||
        (s->d3_bits != 0 && s->d3_bits != 64))
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
// allocate device memory (a fixed device-memory budget reserved up front, or
// a host allocator that owns the device).  Its scratch (task list,
// work-queue cursor, class tables) is the file-scope array below, which
// exists once per device for as long as the library is loaded.  Its device
// address is looked up once per device, with that device current; a reset of
// the device's primary context is not supported afterwards.

namespace {

constexpr int64_t NOALLOC_MAX_N = int64_t(1) << 18;       // vertices
constexpr int64_t NOALLOC_MAX_TASKS = NOALLOC_MAX_N;      // one per root with L >= 1 at most
constexpr size_t NOALLOC_HDR = 256;                        // cursor (8 B), padded
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
    if (!status_dev) return VDMC_ERR_INVALID_ARG;  // a lost status word would hide a failed index check
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
    int *status = status_dev;
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
    auto kern = (k == 3) ? count_kernel<3, false> : count_kernel<4, false>;
    VDMC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes(k, 8)));
    VDMC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem));
    const int64_t grid = (int64_t)sms * std::max(1, per_sm);
    GraphDesc d{rowptr, col, pbeg, new2old, out_dev, n, 0, nnz};
    kern<<<(unsigned)grid, warps * 32, smem, s>>>(d, nullptr, tasks, NOALLOC_MAX_TASKS, cursor, lut, 0, n, status,
                                                  nullptr, EdgeDesc{});
    VDMC_CUDA_TRY(cudaGetLastError());
    return VDMC_OK;
}
