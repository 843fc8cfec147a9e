// Root-per-CTA counting of high-degree roots (exact, no per-set loop for
// star-like sets).
//
// For a root r with many higher-rank neighbours P = N+(r) (L = |P|), almost
// all proper k-BFS(r) of the paper's enumeration ("The Algorithm"; Lemma 2
// structures) are stars: sets whose non-root members are pairwise
// non-adjacent.  The class of such a set (the isomorph-merged index of
// Fig. 1) depends only on the 2-bit arc flags between the root and each
// member -- the member's "colour".  So instead of visiting the O(L^3) stars
// one at a time, this kernel counts them by colour and flag signatures, and
// enumerates one by one only the sets that carry an edge between non-root
// members (rare: the sub-graph H induced on P is sparse).  Every set of the
// plain enumeration is accounted for exactly once and credited to each of
// its members in the same class; results are bit-identical to the plain
// kernel (count.cu), which handles the low-degree roots.
//
// Notation (root r fixed):
//   P     positions 0..L-1 of N+(r) in rank order; colour(x) = flags(r, x)
//   H     undirected graph induced on P; NH(x) its neighbours, h(u,v) the
//         2-bit flags of the pair (bit 0: u -> v, bit 1: v -> u)
//   Q     vertices of rank > r not adjacent to r; NQ(x) = N(x) n Q;
//         NP(c) = N(c) n P for c in Q
// k = 4 shapes with their counting rule:
//   S1 (1,1,1) {x,y,z} c P: sets with 0 or 1 H-edge are counted per member
//      by inclusion-exclusion over its H-neighbourhood; sets with 2 or 3
//      H-edges (wedges, triangles of H) are enumerated.
//   S2 (1,1,2) {x,y} c P, c in Q: c adjacent to exactly one of them is
//      counted per (x, c) by signature; c adjacent to both is enumerated.
//   S3 (1,2,2) x in P, {b,c} c NQ(x): counted per x by flag signature;
//      b ~ c (triangle) is enumerated.
//   S4 (1,2,3) x in P, b in NQ(x), c in NQ(b) \ N(x): counted per (x, b)
//      and per (b, c) by signature; triangles x-b-c correct the counts.
// k = 3: star {a,b} c P counted per member by colour; path a in P, b in
// NQ(a) counted per (a) and per b by signature.
//
// Work per root is O(sum of the degrees of P and of its Q-neighbours +
// enumerated exceptions) instead of O(number of sets).  Each CTA owns a
// slot of scratch: a rank-indexed position map (-1 = not yet seen), compact
// per-Q-vertex counters, the adjacency lists of H.  The rows of the Q
// vertices are walked by warps taking chunks of Q vertices, lanes on
// consecutive entries of the chunk's concatenated rows.  The largest roots
// can be split across several CTAs (members of P and Q vertices shared out
// by position / id; the three-member partials summed and divided by a
// finishing kernel).  Waits: none; the only cross-thread protocols are
// claim-by-atomicCAS followed by a barrier and work claims by atomicAdd.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "vdmc_internal.cuh"
#include "device_common.cuh"

namespace {

// CTA size of the root-per-CTA kernel: 16 or 32 warps (template parameter W;
// 32 warps hide more latency on large roots, 16 keep more registers and
// suit many small roots)
constexpr int32_t CLAIMED = -2;  // posmap: claimed, index being written
// largest P bitmap kept in shared memory next to the static shared memory
// (~39 KB with 16 warps, ~70 KB with 32): 46,000 words = 184 KB (graphs of up
// to 1,472,000 vertices) or 38,000 words = 152 KB (1,216,000 vertices)
constexpr int64_t hub_smem_bits_max_words(int warps) { return warps == 32 ? 38000 : 46000; }

struct HubArgs {
    Csr g;
    const int32_t *new2old;
    uint64_t *out;
    unsigned long long *d3;     // k = 4: n * VDMC_D3_COLS depth-3 credits (rank space)
    int d3_narrow;              // 1: the credits are 32-bit words (no vertex can reach 2^32 of them)
    unsigned long long *d3w;    // k = 4: n * 9 type counts per vertex, spread to its neighbours after the kernel
    unsigned long long *stats;  // [1] sets of hub roots, [2] of those visited one by one (or nullptr)
    const uint8_t *lut_g;
    const int32_t *hubs;
    int32_t nhubs;
    // the first nsplit hub roots are split into `split` parts (queue entries
    // e * split + part); the parts sum their three-member partials in
    // split_acc[e], which split_finish divides and credits after the kernel
    int32_t nsplit, split;
    unsigned long long *split_acc;  // nsplit * C
    int32_t rank_lo, rank_hi;
    unsigned long long *qhead;
    // per-slot scratch
    int32_t *posmap;   // n per slot, all -1 between roots
    uint32_t *qcnt;    // tcap * 9 per slot: P-neighbours of a Q vertex by (colour, flag)
    uint32_t *wq;      // tcap * 3 per slot: Q-neighbours of a Q vertex by flag
    int32_t *touched;  // tcap per slot
    int32_t *hptr;     // lmax + 1 per slot
    uint32_t *hlist;   // hcap per slot: (position << 2) | h(x, y)
    uint32_t *hcx;     // lmax * 3 per slot: |NH(x)| by colour
    uint32_t *wx;      // lmax * 3 per slot: |NQ(x)| by flag
    uint32_t *htx;     // lmax * 9 per slot: |NH(x)| by (colour, flag)
    uint32_t *tbits;   // (n + 31) / 32 words per slot: bit set = Q vertex already claimed
    int32_t pbits_words;  // > 0: membership of P as a bitmap in shared memory
    int32_t *npoff;    // tcap + 1 per slot: offsets of the NP lists
    uint32_t *nplist;  // npcap per slot: (position << 2) | h(x, b)
    longlong2 *qrow;   // k = 4, tcap per slot: row end of each Q vertex, (entries below r << 32) | entries above r
    int64_t tcap, hcap, lmax, npcap;
};

__device__ __forceinline__ uint32_t swapf(uint32_t f) { return ((f & 1u) << 1) | (f >> 1); }

// add (or subtract) v to word i of a depth-3 array, in the counters' width;
// sums are exact modulo that width, so a subtraction ahead of the addition it
// cancels is harmless.  The result is not used: a reduction, not a wait.
__device__ __forceinline__ void d3_add(unsigned long long *a, int narrow, int64_t i, uint32_t v, bool neg) {
    if (narrow)
        atomicAdd(reinterpret_cast<unsigned int *>(a) + i, neg ? 0u - v : v);
    else
        atomicAdd(a + i, neg ? 0ull - (unsigned long long)v : (unsigned long long)v);
}

// canonical index of an H-edge (y,z): colours cy, cz (1..3), flag f = h(y,z)
__device__ __forceinline__ int etype(uint32_t cy, uint32_t cz, uint32_t f) {
    if (cy > cz || (cy == cz && f == 2u)) {
        uint32_t t = cy;
        cy = cz;
        cz = t;
        f = swapf(f);
    }
    return (int)((cy - 1) * 9 + (cz - 1) * 3 + (f - 1));
}

// flags h(x, pos) if pos is in the sorted H-list hl[lo, hi) of x, else 0
__device__ __forceinline__ uint32_t hlist_find(const uint32_t *hl, int32_t lo, int32_t hi, uint32_t pos) {
    int32_t a = lo, b = hi;
    while (a < b) {
        int32_t mid = (a + b) >> 1;
        uint32_t e = hl[mid];
        if ((e >> 2) < pos) a = mid + 1;
        else b = mid;
    }
    if (a < hi) {
        uint32_t e = hl[a];
        if ((e >> 2) == pos) return e & 3u;
    }
    return 0u;
}

// Where credits go: the output rows (original ids) and the checked view.
struct Sink {
    Csr g;
    const int32_t *new2old;
    uint64_t *out;
};

__device__ __forceinline__ void gadd(const Sink &A, uint32_t v, uint32_t cls, unsigned long long cnt, int C) {
    if (cnt == 0ull) return;
    if (!in_bounds(A.g, v < A.g.n && cls < (uint32_t)C)) return;
    const int32_t o = row_of(A.new2old, v);
    if (!in_bounds(A.g, o >= 0 && o < A.g.n)) return;
    atomicAdd((unsigned long long *)&A.out[(int64_t)o * C + cls], cnt);
}

__device__ __forceinline__ void sadd(const Hist64 &h, uint32_t cls, unsigned long long cnt) {
    if (cnt) hadd(h, cls, cnt);
}

// exclusive scan of hptr[0, L) in place (hptr[L] = total), whole CTA
template <int HUB_WARPS>
__device__ void cta_scan(int32_t *hptr, int32_t L, int32_t *warp_sums, int32_t *total_out) {
    constexpr int HUB_THREADS = HUB_WARPS * 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int32_t chunk = (L + HUB_THREADS - 1) / HUB_THREADS;
    const int32_t beg = min(L, tid * chunk), end = min(L, beg + chunk);
    int32_t s = 0;
    for (int32_t p = beg; p < end; p++) s += hptr[p];
    int32_t inc = s;
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_sums[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int32_t w = lane < HUB_WARPS ? warp_sums[lane] : 0, wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < HUB_WARPS) warp_sums[lane] = wi - w;
        if (lane == HUB_WARPS - 1) *total_out = wi;
    }
    __syncthreads();
    int32_t run = warp_sums[warp] + inc - s;
    for (int32_t p = beg; p < end; p++) {
        int32_t d = hptr[p];
        hptr[p] = run;
        run += d;
    }
    __syncthreads();
    if (tid == 0) hptr[L] = *total_out;
    __syncthreads();
}

// return the slot to its resting state (posmap -1, counters and bits 0)
template <int HUB_THREADS>
__device__ void reset_slot(int32_t *posmap, uint32_t *qcnt, const int32_t *touched, const uint32_t *P, int32_t L,
                           int32_t tcount, uint32_t *pbits, bool sbits, uint32_t *tbits) {
    for (int32_t p = threadIdx.x; p < L; p += HUB_THREADS) {
        const uint32_t u = __ldg(P + p) >> 2;
        posmap[u] = -1;
        if (sbits) pbits[u >> 5] = 0u;
    }
    for (int32_t t = threadIdx.x; t < tcount; t += HUB_THREADS) {
        const int32_t u = touched[t];
        posmap[u] = -1;
        tbits[u >> 5] = 0u;
        for (int k = 0; k < 9; k++) qcnt[(int64_t)t * 9 + k] = 0u;
    }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int K, int W>
__global__ void __launch_bounds__(W * 32, 1) hub_kernel(const HubArgs args) {
    constexpr int HUB_WARPS = W, HUB_THREADS = W * 32;
    constexpr int C = (K == 3) ? 13 : 199;
    constexpr int NIDX = 1 << (K * (K - 1));
    __shared__ uint8_t lut[NIDX];
    __shared__ unsigned long long rootP[C], rootD[C];
    __shared__ unsigned long long whist[HUB_WARPS][C];
    __shared__ uint32_t esub[HUB_WARPS][27], eins[HUB_WARPS][27];
    __shared__ uint32_t vq[HUB_WARPS][32];  // queued Q entries of a P member's row
    // per-member counters of phases 2 and 3 (k = 4 keeps them in the warp's
    // histogram, which is too small for them at k = 3)
    static_assert(K == 3 || 2 * C >= 32 * 10, "member counters must fit the warp histogram");
    __shared__ uint32_t mscr[HUB_WARPS][K == 3 ? 32 * 10 : 1];
    __shared__ unsigned long long Etype[27];
    __shared__ unsigned long long Wtot[9];
    __shared__ uint32_t ncol[3];
    __shared__ int32_t s_root, s_part, s_esplit, s_tcount, s_total, s_skip, s_chunk, s_chunk2, s_chunk3, s_chunk4, s_vnext;
    __shared__ int32_t warp_sums[32];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const int64_t slot = blockIdx.x;
    const HubArgs A = args;  // local copy; no references into the parameter block
    const Csr g = A.g;
    const Sink S{g, A.new2old, A.out};
    int32_t *posmap = A.posmap + slot * g.n;
    uint32_t *qcnt = A.qcnt + slot * A.tcap * 9;
    uint32_t *wq = A.wq + slot * A.tcap * 3;
    int32_t *touched = A.touched + slot * A.tcap;
    int32_t *hptr = A.hptr + slot * (A.lmax + 1);
    uint32_t *hlist = A.hlist + slot * A.hcap;
    uint32_t *hcx = A.hcx + slot * A.lmax * 3;
    uint32_t *wx = A.wx + slot * A.lmax * 3;
    uint32_t *htx = A.htx + slot * A.lmax * 9;
    int32_t *npoff = A.npoff + slot * (A.tcap + 1);
    uint32_t *tbits = A.tbits + slot * (int64_t)((g.n + 31) / 32);
    // P membership: a bit per vertex in shared memory (when n fits), else
    // the position map; "claimed Q vertex": a bit per vertex per slot (small
    // enough to stay in L2, unlike the position map)
    extern __shared__ uint32_t pbits[];
    const bool sbits = A.pbits_words > 0;
    auto in_P = [&](uint32_t u) -> bool {
        return sbits ? ((pbits[u >> 5] >> (u & 31u)) & 1u) != 0u : __ldcg(posmap + u) >= 0;
    };
    auto claimed = [&](uint32_t u) -> bool { return ((__ldcg(tbits + (u >> 5)) >> (u & 31u)) & 1u) != 0u; };
    uint32_t *nplist = A.nplist + slot * A.npcap;
    longlong2 *qrow = A.qrow + slot * A.tcap;
    unsigned long long *hv = whist[warp];
    const Hist64 hvh = hist64(hv, C), hP = hist64(rootP, C), hD = hist64(rootD, C);
    const Hist64 hE = hist64(Etype, 27), hW = hist64(Wtot, 9);

    for (int i = tid; i < NIDX; i += HUB_THREADS) lut[i] = A.lut_g[i];
    __shared__ uint8_t d3col[27];  // depth-3 credit type -> column (k = 4)
    __syncthreads();
    if (K == 4 && tid < 27) {
        int cls = 0;
        d3col[tid] = (uint8_t)min(d3_column(lut, tid, &cls), VDMC_D3_COLS - 1);
    }
    for (int i = tid; i < A.pbits_words; i += HUB_THREADS) pbits[i] = 0u;
    for (int i = tid; i < HUB_WARPS * C; i += HUB_THREADS) (&whist[0][0])[i] = 0ull;
    // sets this thread visited one at a time (the enumerated exceptions of
    // the signature counting); summed into stats[2] when the queue is empty
    unsigned long long nenum = 0ull;

    for (;;) {
        __syncthreads();
        if (tid == 0) {
            const unsigned long long q = atomicAdd(A.qhead, 1ull);
            const unsigned long long qs = (unsigned long long)A.nsplit * A.split;
            if (q < qs) {
                s_root = A.hubs[q / A.split];
                s_part = (int32_t)(q % A.split);
                s_esplit = (int32_t)(q / A.split);
            } else {
                const unsigned long long h = q - qs + A.nsplit;
                s_root = h < (unsigned long long)A.nhubs ? A.hubs[h] : -1;
                s_part = -1;
                s_esplit = -1;
            }
            s_vnext = 0;
            s_chunk2 = 0;
            s_chunk3 = 0;
            s_tcount = 0;
            s_skip = 0;
            s_chunk = 0;
            s_chunk4 = 0;
        }
        for (int i = tid; i < C; i += HUB_THREADS) {
            rootP[i] = 0ull;
            rootD[i] = 0ull;
        }
        if (tid < 27) Etype[tid] = 0ull;
        if (tid < 9) Wtot[tid] = 0ull;
        if (tid < 3) ncol[tid] = 0u;
        __syncthreads();
        const int32_t r = s_root;
        if (r < 0) {
            if (A.stats) {
                nenum = warp_sum(nenum);
                if (lane == 0 && nenum) atomicAdd(A.stats + 2, nenum);
            }
            break;
        }
        // part `part` of `nparts` of a split root: P members i with
        // i % nparts == part and Q vertices b with b % nparts == part
        const int32_t part = s_part >= 0 ? s_part : 0, nparts = s_part >= 0 ? A.split : 1;
        if (r < A.rank_lo || r >= A.rank_hi || r >= g.n) continue;
        const int64_t pb = __ldg(g.pbeg + r), pe = __ldg(g.rowptr + r + 1);
        if (!in_bounds(g, pb >= 0 && pb <= pe && pe <= g.nnz && pe - pb <= A.lmax)) continue;
        const int32_t L = (int32_t)(pe - pb);
        const uint32_t *P = g.col + pb;  // entries (rank << 2) | colour

        // ---- phase 1: position map of P, colour counts
        for (int32_t p = tid; p < L; p += HUB_THREADS) {
            const uint32_t e = __ldg(P + p);
            posmap[e >> 2] = p;
            if (sbits) atomicOr(&pbits[(e >> 2) >> 5], 1u << ((e >> 2) & 31u));
            atomicAdd(&ncol[(e & 3u) - 1u], 1u);
        }
        __syncthreads();

        // ---- phase 2: per x in P: |NH(x)|, colours of NH(x), |NQ(x)| by flag;
        // claim the Q vertices (compact index per Q vertex).  A warp takes a
        // chunk of members (32, fewer when P is small) and walks their
        // concatenated upper rows, lanes on consecutive entries.
        const int32_t psz = max(1, min(32, L / (HUB_WARPS * 4)));
        {
            // [7][32] per member of the chunk: |NH(x)|, NH(x) by colour, NQ(x) by
            // flag -- in the warp's histogram (k = 4) or a small array (k = 3)
            uint32_t *cnt = K == 4 ? reinterpret_cast<uint32_t *>(hv) : mscr[warp];
            for (;;) {
                int32_t c0 = 0;
                if (lane == 0) c0 = atomicAdd(&s_chunk2, psz);
                c0 = __shfl_sync(0xffffffffu, c0, 0);
                if (c0 >= L) break;
                const int32_t i = lane < psz ? c0 + lane : L;
                int64_t xe = 0;
                int32_t len = 0;
                if (i < L) {
                    const uint32_t x = __ldg(P + i) >> 2;
                    const int64_t xb = __ldg(g.rowptr + x);
                    xe = __ldg(g.rowptr + x + 1);
                    len = (int32_t)(xe - upper_row(g.col, xb, xe, (uint32_t)r));
                }
#pragma unroll
                for (int m = 0; m < 7; m++) cnt[m * 32 + lane] = 0u;
                int32_t incl = len;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                const int32_t total = __shfl_sync(0xffffffffu, incl, 31);
                __syncwarp();
                for (int32_t base = 0; base < total; base += 32) {
                    const int32_t jj = base + lane;
                    int32_t w = 0;
#pragma unroll
                    for (int sh = 16; sh >= 1; sh >>= 1)
                        if (__shfl_sync(0xffffffffu, incl, w + sh - 1) <= jj) w += sh;
                    const int64_t xeo = __shfl_sync(0xffffffffu, xe, w);
                    const int32_t io = __shfl_sync(0xffffffffu, incl, w);
                    if (jj >= total) continue;
                    const uint32_t ent = __ldg(g.col + (xeo - (int64_t)(io - jj)));  // x's upper row ends at xe
                    const uint32_t u = ent >> 2, f = ent & 3u;
                    if (in_P(u)) {
                        const int32_t p = __ldcg(posmap + u);
                        if (!in_bounds(g, p >= 0 && p < L)) continue;
                        const uint32_t cu = __ldg(P + p) & 3u;
                        atomicAdd(&cnt[w], 1u);
                        atomicAdd(&cnt[cu * 32 + w], 1u);
                    } else {
                        if (in_bounds(g, f != 0u)) atomicAdd(&cnt[(3 + f) * 32 + w], 1u);
                        if (!claimed(u) && atomicCAS(posmap + u, -1, CLAIMED) == -1) {
                            const int32_t t = atomicAdd(&s_tcount, 1);
                            if (in_bounds(g, t < A.tcap)) {
                                touched[t] = (int32_t)u;
                                posmap[u] = -3 - t;
                            }
                            atomicOr(tbits + (u >> 5), 1u << (u & 31u));
                        }
                    }
                }
                __syncwarp();
                if (i < L) {
                    hptr[i] = (int32_t)cnt[lane];
                    hcx[i * 3 + 0] = cnt[1 * 32 + lane]; hcx[i * 3 + 1] = cnt[2 * 32 + lane]; hcx[i * 3 + 2] = cnt[3 * 32 + lane];
                    wx[i * 3 + 0] = cnt[4 * 32 + lane]; wx[i * 3 + 1] = cnt[5 * 32 + lane]; wx[i * 3 + 2] = cnt[6 * 32 + lane];
                }
                __syncwarp();
            }
            for (int c = lane; c < C; c += 32) hv[c] = 0ull;
        }
        __syncthreads();
        const int32_t tcount = s_tcount;
        // Q vertices per warp chunk in phases 4 and 6: 32, fewer when Q is small
        // so that every warp gets several chunks
        const int32_t csz = max(1, min(32, tcount / (HUB_WARPS * 4)));
        if (tcount > A.tcap) {
            if (tid == 0) s_skip = 1;
        }
        cta_scan<HUB_WARPS>(hptr, L, warp_sums, &s_total);
        if (!in_bounds(g, s_total <= A.hcap && s_skip == 0)) {
            // leave the slot clean before giving up on this root
            reset_slot<HUB_THREADS>(posmap, qcnt, touched, P, L, min(tcount, (int32_t)A.tcap), pbits, sbits, tbits);
            continue;
        }

        // ---- phase 3: H adjacency lists, H-edge types, per-Q-vertex P counts
        // (chunks of members as in phase 2; H-lists in row = position order)
        {
            // [32] entries of NH(x) written so far, [9][32] NH(x) by (colour, flag)
            uint32_t *srun = K == 4 ? reinterpret_cast<uint32_t *>(hv) : mscr[warp];
            uint32_t *t9 = srun + 32;
            for (;;) {
                int32_t c0 = 0;
                if (lane == 0) c0 = atomicAdd(&s_chunk3, psz);
                c0 = __shfl_sync(0xffffffffu, c0, 0);
                if (c0 >= L) break;
                const int32_t i = lane < psz ? c0 + lane : L;
                int64_t xe = 0;
                int32_t len = 0, hb = 0;
                uint32_t fx = 0u;
                if (i < L) {
                    const uint32_t ex = __ldg(P + i);
                    const uint32_t x = ex >> 2;
                    fx = ex & 3u;
                    const int64_t xb = __ldg(g.rowptr + x);
                    xe = __ldg(g.rowptr + x + 1);
                    len = (int32_t)(xe - upper_row(g.col, xb, xe, (uint32_t)r));
                    hb = hptr[i];
                }
                srun[lane] = 0u;
#pragma unroll
                for (int m = 0; m < 9; m++) t9[m * 32 + lane] = 0u;
                int32_t incl = len;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                const int32_t total = __shfl_sync(0xffffffffu, incl, 31);
                __syncwarp();
                for (int32_t base = 0; base < total; base += 32) {
                    const int32_t jj = base + lane;
                    int32_t w = 0;
#pragma unroll
                    for (int sh = 16; sh >= 1; sh >>= 1)
                        if (__shfl_sync(0xffffffffu, incl, w + sh - 1) <= jj) w += sh;
                    const int64_t xeo = __shfl_sync(0xffffffffu, xe, w);
                    const int32_t io = __shfl_sync(0xffffffffu, incl, w);
                    const int32_t hbo = __shfl_sync(0xffffffffu, hb, w);
                    const uint32_t fxo = __shfl_sync(0xffffffffu, fx, w);
                    const int32_t iown = __shfl_sync(0xffffffffu, i, w);
                    const bool valid = jj < total;
                    const uint32_t ent = valid ? __ldg(g.col + (xeo - (int64_t)(io - jj))) : 0u;
                    const uint32_t u = ent >> 2, f = ent & 3u;
                    const int32_t p = valid ? __ldcg(posmap + u) : -1;
                    const bool isH = valid && p >= 0;
                    // lanes of the same member in this window (idle lanes apart)
                    const uint32_t grp = __match_any_sync(0xffffffffu, valid ? w : 32 + lane);
                    const uint32_t bal = __ballot_sync(0xffffffffu, isH) & grp;
                    const uint32_t before = srun[w];
                    if (isH && in_bounds(g, p < L && f != 0u)) {
                        const int64_t idx = (int64_t)hbo + before + __popc(bal & lt);
                        if (in_bounds(g, idx < A.hcap)) hlist[idx] = ((uint32_t)p << 2) | f;
                        const uint32_t cu = __ldg(P + p) & 3u;
                        atomicAdd(&t9[((cu - 1) * 3 + (f - 1)) * 32 + w], 1u);
                        if (iown < p) hinc(hE, (uint32_t)etype(fxo, cu, f));
                    } else if (valid && p <= -3 && in_bounds(g, (-3 - (int64_t)p) < tcount && f != 0u)) {
                        const int64_t t = -3 - (int64_t)p;
                        atomicAdd(qcnt + t * 9 + (fxo - 1) * 3 + (f - 1), 1u);
                    }
                    __syncwarp();
                    if (valid && lane == __ffs(grp) - 1) srun[w] = before + __popc(bal);
                    __syncwarp();
                }
                if (i < L) {
                    in_bounds(g, (int32_t)srun[lane] == hptr[i + 1] - hb);
                    uint32_t *h9 = htx + (int64_t)i * 9;
#pragma unroll
                    for (int m = 0; m < 9; m++) h9[m] = t9[m * 32 + lane];
                    for (int f = 0; f < 3; f++) {
                        const uint32_t wv = wx[i * 3 + f];
                        if (wv) hadd(hW, (uint32_t)((fx - 1) * 3 + f), (unsigned long long)wv);
                    }
                }
                __syncwarp();
            }
            for (int c = lane; c < C; c += 32) hv[c] = 0ull;
        }
        __syncthreads();

        // ---- phase 4: NP(b) lists (P-neighbours of each Q vertex b, in
        // position order, read from b's own row) and |NQ(b)| by flag
        if constexpr (K == 4) {  // k = 3 needs neither NP lists nor |NQ(b)|
            for (int32_t t = tid; t < tcount; t += HUB_THREADS) {
                uint32_t s9 = 0;
                for (int k = 0; k < 9; k++) s9 += __ldcg(qcnt + (int64_t)t * 9 + k);
                npoff[t] = (int32_t)s9;
            }
            __syncthreads();
            cta_scan<HUB_WARPS>(npoff, tcount, warp_sums, &s_total);
            if (!in_bounds(g, s_total <= A.npcap)) {
                reset_slot<HUB_THREADS>(posmap, qcnt, touched, P, L, tcount, pbits, sbits, tbits);
                continue;
            }
            // a warp takes a chunk of 32 Q vertices and walks their concatenated
            // upper rows, lanes on consecutive entries; P-neighbours go to NP(b) in
            // row (= position) order, the others are counted by flag
            {
                // per lane of the chunk: entries of NP(b) written so far, |NQ(b)| by
                // flag (in the warp's histogram, zero again before phase 5)
                static_assert(2 * C >= 32 * 4, "chunk counters must fit the warp histogram");
                uint32_t *srun = reinterpret_cast<uint32_t *>(hv);
                uint32_t *swq = srun + 32;
                for (;;) {
                    int32_t c0 = 0;
                    if (lane == 0) c0 = atomicAdd(&s_chunk4, csz);
                    c0 = __shfl_sync(0xffffffffu, c0, 0);
                    if (c0 >= tcount) break;
                    const int32_t t = lane < csz ? c0 + lane : tcount;
                    int64_t be = 0;
                    int32_t len = 0, nb0 = 0;
                    if (t < tcount) {
                        const uint32_t b = (uint32_t)touched[t];
                        const int64_t bb = __ldg(g.rowptr + b);
                        be = __ldg(g.rowptr + b + 1);
                        len = (int32_t)(be - upper_row(g.col, bb, be, (uint32_t)r));
                        nb0 = npoff[t];
                        // b's row end and the lengths of its parts above and below r,
                        // for phase 6 (spares it the row pointers and the search)
                        qrow[t] = make_longlong2(be, (long long)((uint64_t)(be - len - bb) << 32 | (uint32_t)len));
                    }
                    srun[lane] = 0u;
                    swq[lane * 3 + 0] = swq[lane * 3 + 1] = swq[lane * 3 + 2] = 0u;
                    int32_t incl = len;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += y;
                    }
                    const int32_t total = __shfl_sync(0xffffffffu, incl, 31);
                    __syncwarp();
                    // owner lane of entry j: the first lane whose inclusive sum exceeds j
                    auto owner = [&](int32_t j) {
                        int32_t w = 0;
#pragma unroll
                        for (int sh = 16; sh >= 1; sh >>= 1)
                            if (__shfl_sync(0xffffffffu, incl, w + sh - 1) <= j) w += sh;
                        return w;
                    };
                    auto entry = [&](int32_t j, int32_t w) {
                        const int64_t beo = __shfl_sync(0xffffffffu, be, w);
                        const int32_t io = __shfl_sync(0xffffffffu, incl, w);
                        return j < total ? __ldg(g.col + (beo - (int64_t)(io - j))) : 0u;
                    };
                    // the next window's entry is loaded before this one is processed
                    int32_t wn = owner(lane);
                    uint32_t entn = entry(lane, wn);
                    for (int32_t base = 0; base < total; base += 32) {
                        const int32_t j = base + lane;
                        const int32_t w = wn;
                        const uint32_t ent = entn;
                        wn = owner(j + 32);
                        entn = entry(j + 32, wn);
                        const int32_t nbo = __shfl_sync(0xffffffffu, nb0, w);
                        const bool valid = j < total;
                        const bool isP = valid && in_P(ent >> 2);
                        // lanes of the same Q vertex in this window (idle lanes apart)
                        const uint32_t grp = __match_any_sync(0xffffffffu, valid ? w : 32 + lane);
                        const uint32_t bal = __ballot_sync(0xffffffffu, isP) & grp;
                        const uint32_t before = srun[w];
                        if (isP) {
                            const int32_t p = __ldcg(posmap + (ent >> 2));
                            const int64_t idx = (int64_t)nbo + before + __popc(bal & lt);
                            if (in_bounds(g, idx < A.npcap)) nplist[idx] = ((uint32_t)p << 2) | swapf(ent & 3u);  // h(x, b)
                        } else if (valid && in_bounds(g, (ent & 3u) != 0u)) {
                            atomicAdd(&swq[w * 3 + (ent & 3u) - 1u], 1u);
                        }
                        __syncwarp();
                        if (valid && lane == __ffs(grp) - 1) srun[w] = before + __popc(bal);
                        __syncwarp();
                    }
                    if (t < tcount) {
                        in_bounds(g, (int32_t)srun[lane] == npoff[t + 1] - nb0);
#pragma unroll
                        for (int f = 0; f < 3; f++) wq[(int64_t)t * 3 + f] = swq[lane * 3 + f];
                    }
                    __syncwarp();
                }
                for (int c = lane; c < C; c += 32) hv[c] = 0ull;
            }
            __syncthreads();
        }

        // ---- phase 5: per member v of P
        for (;;) {
            int32_t ii = 0;
            if (lane == 0) ii = atomicAdd(&s_vnext, 1);
            ii = __shfl_sync(0xffffffffu, ii, 0);
            const int32_t i = part + nparts * ii;  // members in position order, largest first
            if (i >= L) break;
            const uint32_t ev = __ldg(P + i);
            const uint32_t v = ev >> 2, al = ev & 3u;
            const int32_t h0 = hptr[i], h1 = hptr[i + 1];
            const int32_t dH = h1 - h0;
            uint32_t hcv[3], Wv[3];
            for (int k = 0; k < 3; k++) {
                hcv[k] = hcx[i * 3 + k];
                Wv[k] = wx[i * 3 + k];
            }
            const int64_t vb = __ldg(g.rowptr + v), ve = __ldg(g.rowptr + v + 1);
            const int64_t vu = upper_row(g.col, vb, ve, (uint32_t)r);

            if (K == 3) {
                // star, partner not adjacent: by colour
                if (lane < 3) {
                    const uint32_t be = lane + 1;
                    const long long cnt = (long long)ncol[lane] - (al == be) - hcv[lane];
                    const uint32_t cls = lut[mask3(al, be, 0u)];
                    sadd(hvh, cls, (unsigned long long)cnt);
                    sadd(hP, cls, (unsigned long long)cnt);
                    // path with v as the depth-1 vertex: by flag
                    const uint32_t cls2 = lut[mask3(al, 0u, be)];
                    sadd(hvh, cls2, Wv[lane]);
                    sadd(hD, cls2, Wv[lane]);
                }
                for (int32_t j = lane; j < dH; j += 32) {
                    const uint32_t eu = hlist[h0 + j];
                    const uint32_t cu = __ldg(P + (eu >> 2)) & 3u;
                    const uint32_t cls = lut[mask3(al, cu, eu & 3u)];
                    sadd(hvh, cls, 1ull);
                    sadd(hP, cls, 1ull);
                    nenum += (uint32_t)i < (eu >> 2) ? 1ull : 0ull;  // visited from both members
                }
            } else {
                // -- S1 per-member counts: H-edges inside R_v = P \ N_H[v] by type,
                // and H-neighbours w shared by v and u in NH(v) (S1 with the one
                // H-edge (v,u), third member w adjacent to both: corrected per w).
                // Lanes walk the concatenated H-lists of N_H[v] = {v} + NH(v) in
                // chunks of 32 owners (owner j = -1 is v itself).
                for (int k = lane; k < 27; k += 32) {
                    esub[warp][k] = 0u;
                    eins[warp][k] = 0u;
                }
                __syncwarp();
                for (int32_t j0 = -1; j0 < dH; j0 += 32) {
                    const int32_t j = j0 + lane;
                    uint32_t up = 0u, fvu = 0u, cu = 0u;
                    int32_t u0 = 0, len = 0;
                    if (j < dH) {
                        const uint32_t eu = j < 0 ? ((uint32_t)i << 2) : hlist[h0 + j];
                        up = eu >> 2;
                        fvu = j < 0 ? 0u : (eu & 3u);
                        cu = __ldg(P + up) & 3u;
                        u0 = hptr[up];
                        len = hptr[up + 1] - u0;
                        if (j >= 0) {
                            // S1 one H-edge (v,u), third member isolated from both, by its
                            // colour (the shared H-neighbours are added back per w below)
#pragma unroll
                            for (uint32_t ga = 1; ga <= 3; ga++) {
                                const long long cnt = (long long)ncol[ga - 1] - hcv[ga - 1] - hcx[up * 3 + ga - 1];
                                const uint32_t cls = lut[mask4(al, cu, ga, fvu, 0u, 0u)];
                                sadd(hvh, cls, (unsigned long long)cnt);
                                sadd(hP, cls, (unsigned long long)cnt);
                            }
                        }
                    }
                    int32_t incl = len;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += y;
                    }
                    const int32_t total = __shfl_sync(0xffffffffu, incl, 31);
                    for (int32_t base = 0; base < total; base += 32) {
                        const int32_t jj = base + lane;
                        int32_t w = 0;
#pragma unroll
                        for (int sh = 16; sh >= 1; sh >>= 1)
                            if (__shfl_sync(0xffffffffu, incl, w + sh - 1) <= jj) w += sh;
                        const uint32_t upo = __shfl_sync(0xffffffffu, up, w);
                        const uint32_t cuo = __shfl_sync(0xffffffffu, cu, w);
                        const uint32_t fvo = __shfl_sync(0xffffffffu, fvu, w);
                        const int32_t u0o = __shfl_sync(0xffffffffu, u0, w);
                        const int32_t io = __shfl_sync(0xffffffffu, incl, w);
                        const int32_t leno = __shfl_sync(0xffffffffu, len, w);
                        if (jj >= total) continue;
                        const uint32_t ew = hlist[u0o + (jj - (io - leno))];
                        const uint32_t wp = ew >> 2;
                        const uint32_t cw = __ldg(P + wp) & 3u;
                        const int t = etype(cuo, cw, ew & 3u);
                        atomicAdd(&esub[warp][t], 1u);
                        const bool vside = upo == (uint32_t)i || wp == (uint32_t)i;
                        const bool inh = !vside && hlist_find(hlist, h0, h1, wp) != 0u;  // w in NH(v)
                        if (upo < wp && (vside || inh)) atomicAdd(&eins[warp][t], 1u);
                        if (inh) {
                            const uint32_t cls = lut[mask4(al, cuo, cw, fvo, 0u, 0u)];
                            sadd(hvh, cls, 1ull);
                            sadd(hP, cls, 1ull);
                        }
                    }
                }
                __syncwarp();
                // e_tau(R_v) = E_tau - (edges touching N_H[v])
                for (int k = lane; k < 27; k += 32) {
                    const long long e = (long long)hget(hE, k) - esub[warp][k] + eins[warp][k];
                    esub[warp][k] = (uint32_t)e;
                    const uint32_t be = k / 9 + 1, ga = (k / 3) % 3 + 1, f = k % 3 + 1;
                    if (e > 0) {
                        // S1 one H-edge (y,z) of type k, v isolated from both
                        const uint32_t cls = lut[mask4(be, ga, al, f, 0u, 0u)];
                        sadd(hvh, cls, (unsigned long long)e);
                        sadd(hP, cls, (unsigned long long)e);
                    }
                }
                __syncwarp();
                if (lane < 6) {
                    // S1 no H-edge: pairs {y,z} c R_v by colour pair minus H-edges
                    const uint32_t be = lane < 3 ? 1u : (lane < 5 ? 2u : 3u);
                    const uint32_t ga = lane < 3 ? (uint32_t)lane + 1 : (lane < 5 ? (uint32_t)lane - 1 : 3u);
                    const long long ab = (long long)ncol[be - 1] - (al == be) - hcv[be - 1];
                    const long long ag = (long long)ncol[ga - 1] - (al == ga) - hcv[ga - 1];
                    long long pairs = be < ga ? ab * ag : ab * (ab - 1) / 2;
                    for (uint32_t f = 1; f <= 3; f++) pairs -= (long long)esub[warp][(be - 1) * 9 + (ga - 1) * 3 + (f - 1)];
                    const uint32_t cls = lut[mask4(al, be, ga, 0u, 0u, 0u)];
                    sadd(hvh, cls, (unsigned long long)pairs);
                    sadd(hP, cls, (unsigned long long)pairs);
                }
                // -- S2 across each H-edge (v,u), handled once by the endpoint of
                // larger degree: common Q-neighbours c of v and u.  Lanes walk the
                // concatenated upper rows of the u handled from v, 32 u per chunk.
                const int64_t dv = ve - vb;
                const bool vshort = ve - vu <= 256;
                for (int32_t j0 = 0; j0 < dH; j0 += 32) {
                    const int32_t j = j0 + lane;
                    uint32_t u = 0u, cu = 0u, fvu = 0u;
                    int64_t ue = 0;
                    int32_t len = 0;
                    if (j < dH) {
                        const uint32_t eu = hlist[h0 + j];
                        const uint32_t up = eu >> 2;
                        fvu = eu & 3u;
                        const uint32_t pu = __ldg(P + up);
                        u = pu >> 2;
                        cu = pu & 3u;
                        const int64_t ub = __ldg(g.rowptr + u);
                        ue = __ldg(g.rowptr + u + 1);
                        const int64_t du = ue - ub;
                        if (dv > du || (dv == du && (uint32_t)i < up)) {
                            len = (int32_t)(ue - upper_row(g.col, ub, ue, (uint32_t)r));
                            // S2 credit of u for c in NQ(v) and of v for c in NQ(u), as if no
                            // c were adjacent to both (taken back per common c below)
                            const uint32_t fuv = swapf(fvu);
#pragma unroll
                            for (uint32_t f = 1; f <= 3; f++) {
                                gadd(S, u, lut[mask4(al, cu, 0u, fvu, f, 0u)], (unsigned long long)Wv[f - 1], C);
                                sadd(hvh, lut[mask4(cu, al, 0u, fuv, f, 0u)], (unsigned long long)wx[up * 3 + f - 1]);
                            }
                        }
                    }
                    int32_t incl = len;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += y;
                    }
                    const int32_t total = __shfl_sync(0xffffffffu, incl, 31);
                    for (int32_t base = 0; base < total; base += 32) {
                        const int32_t jj = base + lane;
                        int32_t w = 0;
#pragma unroll
                        for (int sh = 16; sh >= 1; sh >>= 1)
                            if (__shfl_sync(0xffffffffu, incl, w + sh - 1) <= jj) w += sh;
                        const uint32_t uo = __shfl_sync(0xffffffffu, u, w);
                        const uint32_t cuo = __shfl_sync(0xffffffffu, cu, w);
                        const uint32_t fvo = __shfl_sync(0xffffffffu, fvu, w);
                        const int64_t ueo = __shfl_sync(0xffffffffu, ue, w);
                        const int32_t io = __shfl_sync(0xffffffffu, incl, w);
                        if (jj >= total) continue;
                        const uint32_t ec = __ldg(g.col + (ueo - (int64_t)(io - jj)));  // u's upper row ends at ue
                        const uint32_t c = ec >> 2;
                        if (in_P(c)) continue;
                        // h(v, c): a search of v's upper row when it is short (it stays
                        // in L1), else the position of v in NP(c)
                        uint32_t fvc;
                        if (vshort) {
                            fvc = search_row(g.col, vu, ve, c);
                        } else {
                            const int32_t pc = __ldcg(posmap + c);
                            if (!in_bounds(g, pc <= -3 && (-3 - (int64_t)pc) < tcount)) continue;
                            const int64_t tc = -3 - (int64_t)pc;
                            fvc = hlist_find(nplist, npoff[tc], npoff[tc + 1], (uint32_t)i);
                        }
                        if (!fvc) continue;
                        const uint32_t fuc = ec & 3u;
                        // both adjacent to c and to each other: enumerate, and take the
                        // pair out of the bulk counts
                        const uint32_t cle = lut[mask4(al, cuo, 0u, fvo, fvc, fuc)];
                        const uint32_t clb = lut[mask4(al, cuo, 0u, 0u, fvc, fuc)];
                        nenum++;
                        sadd(hvh, cle, 1ull);
                        gadd(S, uo, cle, 1ull, C);
                        gadd(S, c, cle, 1ull, C);
                        sadd(hD, cle, 1ull);
                        sadd(hvh, clb, ~0ull);
                        gadd(S, uo, clb, ~0ull, C);
                        gadd(S, c, clb, ~0ull, C);
                        sadd(hD, clb, ~0ull);
                        gadd(S, uo, lut[mask4(al, cuo, 0u, fvo, fvc, 0u)], ~0ull, C);
                        sadd(hvh, lut[mask4(cuo, al, 0u, swapf(fvo), fuc, 0u)], ~0ull);
                    }
                }
                // -- S1 sets with two or three H-edges, v the centre: lanes over the
                // pairs (j1 < j2) of NH(v) in row order, lane l on pairs l, l+32, ...
                {
                    int32_t j1 = 0, j2 = 1 + lane;
                    while (j1 < dH - 1 && j2 >= dH) {  // carry into the next row
                        j1++;
                        j2 = j2 - dH + j1 + 1;
                    }
                    for (; j1 < dH - 1;) {
                        const uint32_t e1 = hlist[h0 + j1];
                        const uint32_t yp = e1 >> 2, fvy = e1 & 3u;
                        const uint32_t cy = __ldg(P + yp) & 3u;
                        const int32_t y0 = hptr[yp], y1 = hptr[yp + 1];
                        const uint32_t e2 = hlist[h0 + j2];
                        const uint32_t zp = e2 >> 2, fvz = e2 & 3u;
                        const uint32_t cz = __ldg(P + zp) & 3u;
                        const uint32_t fyz = hlist_find(hlist, y0, y1, zp);
                        if (fyz == 0u || (uint32_t)i < yp) {
                            const uint32_t cls = lut[mask4(al, cy, cz, fvy, fvz, fyz)];
                            sadd(hvh, cls, 1ull);
                            gadd(S, __ldg(P + yp) >> 2, cls, 1ull, C);
                            gadd(S, __ldg(P + zp) >> 2, cls, 1ull, C);
                            sadd(hP, cls, 3ull);
                            nenum++;
                        }
                        j2 += 32;
                        while (j1 < dH - 1 && j2 >= dH) {
                            j1++;
                            j2 = j2 - dH + j1 + 1;
                        }
                    }
                }

                // -- Q side: lanes over c in NQ(v)
                uint32_t hx9[9];
#pragma unroll
                for (int k = 0; k < 9; k++) hx9[k] = htx[(int64_t)i * 9 + k];
                long long Z[9];
#pragma unroll
                for (int k = 0; k < 9; k++) Z[k] = 0;
                // Q entries of v's row wait in a queue and are processed 32 at a
                // time, one per lane
                uint32_t *qv = vq[warp];
                auto qside = [&](const uint32_t ec) {
                        const uint32_t c = ec >> 2, f = ec & 3u;
                        const int32_t pc = __ldcg(posmap + c);
                        if (!in_bounds(g, pc <= -3 && (-3 - (int64_t)pc) < tcount)) return;
                        const int64_t tc = -3 - (int64_t)pc;
                        uint32_t q[9], np[3] = {0u, 0u, 0u};
#pragma unroll
                        for (int k = 0; k < 9; k++) {
                            q[k] = __ldcg(qcnt + tc * 9 + k);
                            np[k / 3] += q[k];
                        }
                        const int32_t o0 = npoff[tc], o1 = npoff[tc + 1];
                        // NH(v) n NP(c) by (colour, h(v,y)) and by (colour, h(y,c))
                        uint32_t comT[9], comC[9];
#pragma unroll
                        for (int k = 0; k < 9; k++) comT[k] = comC[k] = 0u;
                        if (dH > 0) {
                            if (o1 - o0 <= dH) {
                                for (int32_t x = o0; x < o1; x++) {
                                    const uint32_t ey = nplist[x];
                                    const uint32_t py = ey >> 2;
                                    if (py == (uint32_t)i) continue;
                                    const uint32_t fvy = hlist_find(hlist, h0, h1, py);
                                    if (!fvy) continue;
                                    const uint32_t cy = __ldg(P + py) & 3u;
                                    const uint32_t kt = (cy - 1) * 3 + fvy - 1, kc = (cy - 1) * 3 + (ey & 3u) - 1;
#pragma unroll
                                    for (int k = 0; k < 9; k++) {
                                        comT[k] += (uint32_t)k == kt ? 1u : 0u;
                                        comC[k] += (uint32_t)k == kc ? 1u : 0u;
                                    }
                                }
                            } else {
                                for (int32_t j = 0; j < dH; j++) {
                                    const uint32_t eyv = hlist[h0 + j];
                                    const uint32_t yp = eyv >> 2;
                                    const uint32_t fyc = hlist_find(nplist, o0, o1, yp);
                                    if (!fyc) continue;
                                    const uint32_t cy = __ldg(P + yp) & 3u;
                                    const uint32_t kt = (cy - 1) * 3 + (eyv & 3u) - 1, kc = (cy - 1) * 3 + fyc - 1;
#pragma unroll
                                    for (int k = 0; k < 9; k++) {
                                        comT[k] += (uint32_t)k == kt ? 1u : 0u;
                                        comC[k] += (uint32_t)k == kc ? 1u : 0u;
                                    }
                                }
                            }
                        }
                        // S2 (x = v, c adjacent to v only): partner y by (colour, h(v,y))
#pragma unroll
                        for (uint32_t be = 1; be <= 3; be++) {
                            uint32_t combe = 0u;
#pragma unroll
                            for (uint32_t fy = 1; fy <= 3; fy++) {
                                const uint32_t k = (be - 1) * 3 + fy - 1;
                                combe += comT[k];
                                const long long cnt = (long long)hx9[k] - comT[k];
                                const uint32_t cls = lut[mask4(al, be, 0u, fy, f, 0u)];
                                sadd(hvh, cls, (unsigned long long)cnt);
                                gadd(S, c, cls, (unsigned long long)cnt, C);
                                sadd(hD, cls, (unsigned long long)cnt);
                            }
                            const long long cnt = (long long)ncol[be - 1] - hcv[be - 1] - np[be - 1] + combe;
                            const uint32_t cls = lut[mask4(al, be, 0u, 0u, f, 0u)];
                            sadd(hvh, cls, (unsigned long long)cnt);
                            gadd(S, c, cls, (unsigned long long)cnt, C);
                            sadd(hD, cls, (unsigned long long)cnt);
                        }
                        // S2 with c adjacent to v and to another P member y: credit of
                        // v, partners y in NP(c) by (colour, h(y,c)), counted as if v, y
                        // were not adjacent (H-adjacent pairs are corrected per H-edge)
                        const uint32_t kself = (al - 1) * 3 + f - 1;
#pragma unroll
                        for (int k = 0; k < 9; k++) {
                            const uint32_t cnt = q[k] - ((uint32_t)k == kself ? 1u : 0u);
                            sadd(hvh, lut[mask4(al, (uint32_t)(k / 3 + 1), 0u, 0u, f, (uint32_t)(k % 3 + 1))], cnt);
                        }
                        // S2 credit of v as the P member not adjacent to c (collected in Z)
#pragma unroll
                        for (int k = 0; k < 9; k++) Z[k] += (long long)q[k] - comC[k] - ((uint32_t)k == kself ? 1 : 0);
#pragma unroll
                        for (uint32_t f2 = 1; f2 <= 3; f2++) {
                            // S3 credit of c: every other c2 in NQ(v) as partner
                            // (adjacent partners are corrected per triangle)
                            const long long cnt3 = (long long)Wv[f2 - 1] - (f == f2);
                            gadd(S, c, lut[mask4(al, 0u, 0u, f, f2, 0u)], (unsigned long long)cnt3, C);
                            // S4 with (x, b) = (v, c): every Q-neighbour of c as the
                            // depth-3 vertex (those adjacent to v corrected per triangle)
                            const unsigned long long cnt4 = wq[tc * 3 + f2 - 1];
                            const uint32_t cls = lut[mask4(al, 0u, 0u, f, 0u, f2)];
                            sadd(hvh, cls, cnt4);
                            sadd(hD, cls, cnt4);
                        }
                };
                int32_t qn = 0;
                for (int64_t e0 = vu; e0 < ve; e0 += 32) {
                    const int64_t e = e0 + lane;
                    const uint32_t ent = e < ve ? __ldg(g.col + e) : 0u;
                    const bool isQ = e < ve && !in_P(ent >> 2);
                    const uint32_t bal = __ballot_sync(0xffffffffu, isQ);
                    const int32_t nc = __popc(bal);
                    if (qn + nc > 32) {
                        if (lane < qn) qside(qv[lane]);
                        __syncwarp();
                        qn = 0;
                    }
                    if (isQ) qv[qn + __popc(bal & lt)] = ent;
                    qn += nc;
                    __syncwarp();
                }
                if (lane < qn) qside(qv[lane]);
                __syncwarp();
                long long zl = 0;  // Z[lane] for lanes 0..8
#pragma unroll
                for (int k = 0; k < 9; k++) {
                    const long long zk = warp_sum(Z[k]);
                    if (k == lane) zl = zk;
                }
                // S2 credit of v as the non-adjacent P member (x not in N_H[v])
                if (lane < 9) {
                    long long wsum = 0;
                    for (int32_t j = -1; j < dH; j++) {
                        const uint32_t xp = j < 0 ? (uint32_t)i : (hlist[h0 + j] >> 2);
                        if ((__ldg(P + xp) & 3u) == (uint32_t)(lane / 3 + 1)) wsum += wx[xp * 3 + lane % 3];
                    }
                    const long long base = (long long)hget(hW, lane) - wsum - zl;
                    const uint32_t cls = lut[mask4((uint32_t)(lane / 3 + 1), al, 0u, 0u, (uint32_t)(lane % 3 + 1), 0u)];
                    sadd(hvh, cls, (unsigned long long)base);
                }
                // S3 credit of v and r: pairs {b, c} c NQ(v) by flags (adjacent
                // pairs corrected per triangle)
                if (lane < 6) {
                    const uint32_t f1 = lane < 3 ? 1u : (lane < 5 ? 2u : 3u);
                    const uint32_t f2 = lane < 3 ? (uint32_t)lane + 1 : (lane < 5 ? (uint32_t)lane - 1 : 3u);
                    const long long pairs = f1 < f2 ? (long long)Wv[f1 - 1] * Wv[f2 - 1]
                                                    : (long long)Wv[f1 - 1] * ((long long)Wv[f1 - 1] - 1) / 2;
                    const uint32_t cls = lut[mask4(al, 0u, 0u, f1, f2, 0u)];
                    sadd(hvh, cls, (unsigned long long)pairs);
                    sadd(hD, cls, (unsigned long long)pairs);
                }
            }
            __syncwarp();
            flush_hist(g, hvh, C, A.out, row_of(A.new2old, v), lane);
        }
        __syncthreads();

        // ---- phase 6: per Q vertex b.  A warp takes a chunk of 32 Q
        // vertices (claimed dynamically); each lane first credits its own b,
        // then the warp walks the concatenated upper rows of the chunk with
        // its lanes on consecutive entries, so long and short rows alike keep
        // the lanes busy.
        {
            // [32][9] P-neighbour counts of the chunk's Q vertices and a queue of
            // 32 triangle candidates, in the warp's histogram (k = 4 only; k = 3
            // credits b directly)
            static_assert(K == 3 || 2 * C >= 32 * 9 + 64, "chunk counts and candidate queue must fit the warp histogram");
            uint32_t *sq = reinterpret_cast<uint32_t *>(hv);
            for (;;) {
                int32_t c0 = 0;
                if (lane == 0) c0 = atomicAdd(&s_chunk, csz);
                c0 = __shfl_sync(0xffffffffu, c0, 0);
                if (c0 >= tcount) break;
                const int32_t t = lane < csz ? c0 + lane : tcount;
                uint32_t b = 0u, nzm = 0u, nzd = 0u;  // nzd: types whose depth-3 credits the walk issues
                int64_t be = 0;
                int32_t len = 0, o0 = 0, o1 = 0;
                if (t < tcount) b = (uint32_t)touched[t];
                if (t < tcount && (int32_t)(b % (uint32_t)nparts) == part) {
                    int64_t bb;
                    if constexpr (K == 4) {
                        // row end and part lengths saved by phase 4
                        const longlong2 qr = __ldcg(qrow + t);
                        be = qr.x;
                        len = (int32_t)(uint32_t)qr.y;
                        bb = be - len - (int64_t)((uint64_t)qr.y >> 32);
                    } else {
                        bb = __ldg(g.rowptr + b);
                        be = __ldg(g.rowptr + b + 1);
                        len = (int32_t)(be - upper_row(g.col, bb, be, (uint32_t)r));
                    }
                    o0 = npoff[t];
                    o1 = npoff[t + 1];
#pragma unroll
                    for (int k = 0; k < 9; k++) {
                        const uint32_t qk = __ldcg(qcnt + (int64_t)t * 9 + k);
                        if (K == 3) {
                            // path with b at depth 2: by (colour, flag) of its P neighbours
                            gadd(S, b, lut[mask3((uint32_t)(k / 3 + 1), 0u, (uint32_t)(k % 3 + 1))], qk, C);
                        } else {
                            sq[lane * 9 + k] = qk;
                            nzm |= (qk != 0u ? 1u : 0u) << k;
                        }
                    }
                    if (K == 4) {
                        uint32_t w3[3];
#pragma unroll
                        for (int f = 0; f < 3; f++) w3[f] = wq[(int64_t)t * 3 + f];
                        for (uint32_t m1 = nzm; m1; m1 &= m1 - 1u) {
                            const int t1 = __ffs(m1) - 1;
                            const unsigned long long q1 = sq[lane * 9 + t1];
                            const uint32_t c1 = (uint32_t)(t1 / 3 + 1), h1 = (uint32_t)(t1 % 3 + 1);
                            // S4 credit of b: P neighbours x by (colour, h(x,b)), Q
                            // neighbours by flag
#pragma unroll
                            for (int f = 0; f < 3; f++)
                                gadd(S, b, lut[mask4(c1, 0u, 0u, h1, 0u, (uint32_t)f + 1)], q1 * w3[f], C);
                            // S2 with b adjacent to two members x, y of P, counted as
                            // if x, y were not adjacent (H-adjacent pairs are
                            // corrected per H-edge): pairs of NP(b) by type
                            {
                                const unsigned long long cnt = q1 * (q1 - 1ull) / 2ull;
                                const uint32_t cls = lut[mask4(c1, c1, 0u, 0u, h1, h1)];
                                gadd(S, b, cls, cnt, C);
                                sadd(hD, cls, cnt);
                            }
                            for (uint32_t m2 = m1 & (m1 - 1u); m2; m2 &= m2 - 1u) {
                                const int t2 = __ffs(m2) - 1;
                                const unsigned long long cnt = q1 * sq[lane * 9 + t2];
                                const uint32_t cls = lut[mask4(c1, (uint32_t)(t2 / 3 + 1), 0u, 0u, h1, (uint32_t)(t2 % 3 + 1))];
                                gadd(S, b, cls, cnt, C);
                                sadd(hD, cls, cnt);
                            }
                        }
                        // S4 credits of the depth-3 vertices c: the neighbours of b in
                        // its upper row outside P, each by (type of x, h(b, c)).  Either
                        // the walk below adds b's type counts at every such c, or -- when
                        // the rest of b's row (ranks below r, members of P) is the
                        // shorter part -- they go once to d3w[b], d3_spread adds d3w[b]
                        // at every neighbour of b after the kernel, and the neighbours
                        // that must not have them are subtracted here.
                        nzd = nzm;
                        const int64_t ub = be - len;
                        const int32_t lower = (int32_t)(ub - bb), npn = o1 - o0;
                        if (nzm && 1 + npn + lower < len - npn) {
                            nzd = 0u;
                            for (uint32_t m1 = nzm; m1; m1 &= m1 - 1u) {
                                const int t1 = __ffs(m1) - 1;
                                d3_add(A.d3w, A.d3_narrow, (int64_t)b * 9 + t1, sq[lane * 9 + t1], false);
                            }
                            for (int32_t x = o0; x < o1; x++) {
                                const uint32_t ex = nplist[x];
                                const uint32_t xv = __ldg(P + (ex >> 2)) >> 2, hbx = swapf(ex & 3u);  // h(b, x)
                                if (!in_bounds(g, xv < (uint32_t)g.n && hbx != 0u)) continue;
                                for (uint32_t m1 = nzm; m1; m1 &= m1 - 1u) {
                                    const int t1 = __ffs(m1) - 1;
                                    d3_add(A.d3, A.d3_narrow, (int64_t)xv * VDMC_D3_COLS + d3col[t1 * 3 + hbx - 1],
                                           sq[lane * 9 + t1], true);
                                }
                            }
                            for (int64_t j = bb; j < ub; j++) {
                                const uint32_t ent = __ldg(g.col + j);
                                const uint32_t cv = ent >> 2, gg = ent & 3u;
                                if (!in_bounds(g, cv < (uint32_t)g.n && gg != 0u)) continue;
                                for (uint32_t m1 = nzm; m1; m1 &= m1 - 1u) {
                                    const int t1 = __ffs(m1) - 1;
                                    d3_add(A.d3, A.d3_narrow, (int64_t)cv * VDMC_D3_COLS + d3col[t1 * 3 + gg - 1],
                                           sq[lane * 9 + t1], true);
                                }
                            }
                        }
                        // without depth-3 credits to issue, the walk only looks for
                        // triangle candidates c > b: the part of the row above b
                        if (nzd == 0u) len = (int32_t)(be - max(ub, __ldg(g.pbeg + b)));
                    }
                }
                if (K == 3) continue;
                __syncwarp();
                int32_t incl = len;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                const int32_t total = __shfl_sync(0xffffffffu, incl, 31);
                // owner lane of entry j: the first lane whose inclusive sum exceeds j
                auto owner = [&](int32_t j) {
                    int32_t w = 0;
#pragma unroll
                    for (int sh = 16; sh >= 1; sh >>= 1)
                        if (__shfl_sync(0xffffffffu, incl, w + sh - 1) <= j) w += sh;
                    return w;
                };
                // entry j of the chunk (b's upper row ends at be); 0 past the end
                auto entry = [&](int32_t j, int32_t w) {
                    const int64_t beo = __shfl_sync(0xffffffffu, be, w);
                    const int32_t io = __shfl_sync(0xffffffffu, incl, w);
                    return j < total ? __ldg(g.col + (beo - (int64_t)(io - j))) : 0u;
                };
                // triangle candidates (c in NQ(b), b < c, c claimed) wait in a
                // queue and are resolved 32 at a time, one per lane
                uint32_t *qc = sq + 32 * 9, *qm = qc + 32;
                int32_t qn = 0;
                auto drain = [&](int32_t cnt) {
                    const bool act = lane < cnt;
                    const uint32_t c = act ? qc[lane] : 0u, m = act ? qm[lane] : 0u;
                    const int32_t wv = (int32_t)(m & 31u);
                    const uint32_t gg = m >> 5;
                    const uint32_t bo = __shfl_sync(0xffffffffu, b, wv);
                    const int32_t oo0 = __shfl_sync(0xffffffffu, o0, wv), oo1 = __shfl_sync(0xffffffffu, o1, wv);
                    __syncwarp();
                    if (!act) return;
                    // triangles v - b - c: enumerate the S3 set and correct the bulk counts
                    const int32_t pc = __ldcg(posmap + c);
                    if (!in_bounds(g, pc <= -3 && (-3 - (int64_t)pc) < tcount)) return;
                    const int64_t t2 = -3 - (int64_t)pc;
                    const int32_t p0 = npoff[t2], p1 = npoff[t2 + 1];
                    const bool short_b = (oo1 - oo0) <= (p1 - p0);
                    const int32_t s0 = short_b ? oo0 : p0, s1 = short_b ? oo1 : p1;
                    for (int32_t x = s0; x < s1; x++) {
                        const uint32_t ex = nplist[x];
                        const uint32_t vp = ex >> 2;
                        const uint32_t fo = short_b ? hlist_find(nplist, p0, p1, vp) : hlist_find(nplist, oo0, oo1, vp);
                        if (!fo) continue;
                        const uint32_t fvb = short_b ? (ex & 3u) : fo;    // h(v, b)
                        const uint32_t fvc = short_b ? fo : (ex & 3u);    // h(v, c)
                        const uint32_t pv = __ldg(P + vp);
                        const uint32_t cv = pv & 3u, vv = pv >> 2;
                        const uint32_t clE = lut[mask4(cv, 0u, 0u, fvb, fvc, gg)];
                        const uint32_t clF = lut[mask4(cv, 0u, 0u, fvb, fvc, 0u)];
                        const uint32_t clA = lut[mask4(cv, 0u, 0u, fvb, 0u, gg)];
                        const uint32_t clB = lut[mask4(cv, 0u, 0u, fvc, 0u, swapf(gg))];
                        const uint32_t who[3] = {vv, bo, c};
                        nenum++;
#pragma unroll
                        for (int m3 = 0; m3 < 3; m3++) {
                            gadd(S, who[m3], clE, 1ull, C);
                            gadd(S, who[m3], clF, ~0ull, C);
                            gadd(S, who[m3], clA, ~0ull, C);
                            gadd(S, who[m3], clB, ~0ull, C);
                        }
                        sadd(hD, clE, 1ull);
                        sadd(hD, clF, ~0ull);
                        sadd(hD, clA, ~0ull);
                        sadd(hD, clB, ~0ull);
                    }
                };
                // the next window's entry is loaded before this one is processed
                int32_t wn = owner(lane);
                uint32_t entn = entry(lane, wn);
                for (int32_t base = 0; base < total; base += 32) {
                    const int32_t j = base + lane;
                    const int32_t w = wn;
                    const uint32_t ent = entn;
                    wn = owner(j + 32);
                    entn = entry(j + 32, wn);
                    const uint32_t bo = __shfl_sync(0xffffffffu, b, w);
                    const uint32_t nzo = __shfl_sync(0xffffffffu, nzd, w);
                    const uint32_t c = ent >> 2, gg = ent & 3u;
                    bool cand = false;
                    if (j < total && !in_P(c)) {
                        // S4 credit of c (b at depth 2, c at depth 3), in c's
                        // depth-3 column of the class of (type of x, h(b, c))
                        if (nzo && in_bounds(g, c < (uint32_t)g.n && gg != 0u)) {
#pragma unroll
                            for (int k = 0; k < 9; k++)
                                if ((nzo >> k) & 1u) {
                                    // a reduction: its result is not needed, so the warp
                                    // does not wait for it (a 32-bit add with a carry
                                    // check would make it wait on every entry)
                                    d3_add(A.d3, A.d3_narrow, (int64_t)c * VDMC_D3_COLS + d3col[k * 3 + gg - 1],
                                           sq[w * 9 + k], false);
                                }
                        }
                        cand = c > bo && claimed(c);  // else counted from c, or no P neighbour
                    }
                    const uint32_t bal = __ballot_sync(0xffffffffu, cand);
                    const int32_t nc = __popc(bal);
                    if (qn + nc > 32) {
                        drain(qn);
                        __syncwarp();
                        qn = 0;
                    }
                    if (cand) {
                        const int32_t pos = qn + __popc(bal & lt);
                        qc[pos] = c;
                        qm[pos] = (uint32_t)w | (gg << 5);
                    }
                    qn += nc;
                    __syncwarp();
                }
                if (qn > 0) drain(qn);
                __syncwarp();
            }
            __syncwarp();
            for (int c = lane; c < C; c += 32) hv[c] = 0ull;  // the chunk area is the warp's histogram
        }
        __syncthreads();

        // ---- phase 7: root credit, reset the slot
        {
            const int32_t orig = row_of(A.new2old, (uint32_t)r);
            const bool ok = in_bounds(g, orig >= 0 && orig < g.n);
            unsigned long long *out_r = (unsigned long long *)&A.out[(int64_t)orig * C];
            // S1 sets are counted once per member of P: a split root's parts
            // sum their partials, divided after the kernel (split_finish)
            unsigned long long *acc = nparts > 1 ? A.split_acc + (int64_t)s_esplit * C : nullptr;
            unsigned long long tot = 0ull;  // sets of this root credited here
            for (int c = tid; c < C; c += HUB_THREADS) {
                const unsigned long long p1 = hget(hP, c), d1 = hget(hD, c);
                const unsigned long long v = (nparts == 1 ? p1 / (K == 3 ? 2ull : 3ull) : 0ull) + d1;
                if (nparts > 1 && p1) atomicAdd(acc + c, p1);
                if (v && ok) atomicAdd(out_r + c, v);
                tot += v;
            }
            if (A.stats) {
                tot = warp_sum(tot);
                if (lane == 0 && tot) atomicAdd(A.stats + 1, tot);
            }
        }
        reset_slot<HUB_THREADS>(posmap, qcnt, touched, P, L, tcount, pbits, sbits, tbits);
    }
}

// After the root-per-CTA kernel (k = 4): every vertex c adds the type counts
// d3w[b] of each neighbour b to its depth-3 columns, by (type, h(b, c)) -- the
// second half of the per-vertex route of phase 6 (the kernel has already
// subtracted the neighbours of b that are not at depth 3).  One warp per vertex,
// lanes over its row; plain adds, since nothing else writes d3 meanwhile.
__global__ void d3_spread(const int64_t *__restrict__ rowptr, const uint32_t *__restrict__ col, int32_t n,
                          const unsigned long long *__restrict__ d3w, int narrow, const uint8_t *__restrict__ lut,
                          unsigned long long *__restrict__ d3) {
    __shared__ uint8_t d3c[27];
    if (threadIdx.x < 27) {
        int cls = 0;
        d3c[threadIdx.x] = (uint8_t)min(d3_column(lut, threadIdx.x, &cls), VDMC_D3_COLS - 1);
    }
    __syncthreads();
    const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= n) return;
    const uint32_t *w32 = reinterpret_cast<const uint32_t *>(d3w);
    unsigned long long acc[VDMC_D3_COLS];
#pragma unroll
    for (int q = 0; q < VDMC_D3_COLS; q++) acc[q] = 0ull;
    bool any = false;
    for (int64_t p = __ldg(rowptr + c) + lane; p < __ldg(rowptr + c + 1); p += 32) {
        const uint32_t ent = __ldg(col + p);
        const uint32_t b = ent >> 2, hbc = swapf(ent & 3u);  // c's row holds h(c, b)
        if (b >= (uint32_t)n || hbc == 0u) continue;
        for (int k = 0; k < 9; k++) {
            const unsigned long long v = narrow ? (unsigned long long)__ldg(w32 + (int64_t)b * 9 + k)
                                                : __ldg(d3w + (int64_t)b * 9 + k);
            if (!v) continue;
            any = true;
            const uint32_t q0 = d3c[k * 3 + hbc - 1];
#pragma unroll
            for (int q = 0; q < VDMC_D3_COLS; q++) acc[q] += q == (int)q0 ? v : 0ull;
        }
    }
    if (!__any_sync(0xffffffffu, any)) return;
    unsigned long long mine = 0ull;
#pragma unroll
    for (int q = 0; q < VDMC_D3_COLS; q++) {
        unsigned long long v = acc[q];
        for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == q) mine = v;
    }
    if (lane < VDMC_D3_COLS && mine) {
        if (narrow) {
            uint32_t *d = reinterpret_cast<uint32_t *>(d3) + c * VDMC_D3_COLS + lane;
            *d += (uint32_t)mine;
        } else {
            d3[c * VDMC_D3_COLS + lane] += mine;
        }
    }
}

// root credit of the three-member sets of split roots: the parts' summed
// partials / |P-members per set| (2 for k = 3, 3 for k = 4); one block per root
__global__ void split_finish(const unsigned long long *__restrict__ acc, const int32_t *__restrict__ hubs,
                             int32_t nsplit, int C, unsigned long long times, int64_t n, uint64_t *out,
                             unsigned long long *stats) {
    const int32_t e = blockIdx.x;
    if (e >= nsplit) return;
    const int32_t r = hubs[e];
    if (r < 0 || r >= n) return;
    unsigned long long tot = 0ull;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        const unsigned long long v = acc[(int64_t)e * C + c] / times;
        if (v) atomicAdd((unsigned long long *)&out[(int64_t)r * C + c], v);
        tot += v;
    }
    if (stats && tot) atomicAdd(stats + 1, tot);
}

__global__ void fill_i32(int32_t *p, int64_t n, int32_t v) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

}  // namespace

// ------------------------------------------------------------------ host --

namespace {

__global__ void hub_flags(const int64_t *rowptr, const int64_t *pbeg, int32_t n, int32_t min_l, uint32_t *flag) {
    int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t L = rowptr[r + 1] - pbeg[r];
    flag[r] = (min_l > 0 && L >= min_l) ? 1u : 0u;
}

__global__ void hub_compact(const uint32_t *flag, const uint32_t *pos, int32_t n, int32_t *hubs) {
    int32_t r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n && flag[r]) hubs[pos[r]] = r;
}

// per hub root: L, sum over P of min(d(x), L) (bound on its H lists) and of
// d(x) (bound on its Q vertices)
__global__ void hub_sizes(const int64_t *rowptr, const uint32_t *col, const int64_t *pbeg, const int32_t *hubs,
                          int32_t nhubs, unsigned long long *mx) {
    const int lane = threadIdx.x & 31;
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= nhubs) return;
    const int32_t r = hubs[w];
    const int64_t pb = pbeg[r], pe = rowptr[r + 1];
    const int64_t L = pe - pb;
    unsigned long long s1 = 0, s2 = 0;
    for (int64_t e = pb + lane; e < pe; e += 32) {
        const uint32_t x = col[e] >> 2;
        const int64_t d = rowptr[x + 1] - rowptr[x];
        s1 += (unsigned long long)(d < L ? d : L);
        s2 += (unsigned long long)d;
    }
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    if (lane == 0) {
        atomicMax(&mx[0], (unsigned long long)L);
        atomicMax(&mx[1], s1);
        atomicMax(&mx[2], s2);
    }
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

void vdmc_hub_free(vdmc_graph *g, cudaStream_t s) {
    vdmc_free(g->hubs, s);
    vdmc_free(g->hub_scratch, s);
    vdmc_free(g->hub_qhead, s);
    vdmc_free(g->hub_split_buf, s);
    g->hub_split_buf = nullptr;
    g->hub_split_cap = 0;
    g->hubs = nullptr;
    g->hub_scratch = nullptr;
    g->hub_qhead = nullptr;
    g->nhubs = 0;
    g->hub_slots = 0;
    g->hub_scratch_bytes = 0;
}

vdmc_status vdmc_build_hubs(vdmc_graph *g, int32_t min_l, cudaStream_t s) {
    vdmc_hub_free(g, s);
    g->hub_min_l = min_l;
    const int32_t n = g->n;
    if (min_l <= 0 || n == 0) return VDMC_OK;
    uint32_t *flag = nullptr, *pos = nullptr;
    VDMC_CUDA_TRY(cudaMallocAsync((void **)&flag, sizeof(uint32_t) * (size_t)n, s));
    cudaError_t e = cudaMallocAsync((void **)&pos, sizeof(uint32_t) * ((size_t)n + 1), s);
    unsigned long long *mx = nullptr;
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&mx, sizeof(unsigned long long) * 3, s);
    if (e == cudaSuccess) {
        hub_flags<<<(n + 255) / 256, 256, 0, s>>>(g->rowptr, g->pbeg, n, min_l, flag);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = vdmc_exclusive_scan_u32(flag, pos, n, s);
    uint32_t nh = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nh, pos + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && nh > 0) {
        e = vdmc_malloc(&g->hubs, sizeof(int32_t) * nh, s);
        if (e == cudaSuccess) {
            hub_compact<<<(n + 255) / 256, 256, 0, s>>>(flag, pos, n, g->hubs);
            e = cudaMemsetAsync(mx, 0, sizeof(unsigned long long) * 3, s);
        }
        if (e == cudaSuccess) {
            hub_sizes<<<(unsigned)((nh * 32 + 255) / 256), 256, 0, s>>>(g->rowptr, g->col, g->pbeg, g->hubs, (int32_t)nh, mx);
            e = cudaGetLastError();
        }
        unsigned long long h[3] = {0, 0, 0};
        if (e == cudaSuccess) e = cudaMemcpyAsync(h, mx, sizeof h, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        g->hub_lmax = (int64_t)h[0];
        g->hub_hcap = std::max<int64_t>(1, (int64_t)h[1]);
        g->hub_tcap = std::max<int64_t>(1, std::min<int64_t>((int64_t)n, (int64_t)h[2]));
        g->hub_npcap = std::max<int64_t>(1, std::min<int64_t>((int64_t)0x7fffffff, (int64_t)h[2]));
        g->nhubs = (int32_t)nh;
    }
    cudaFreeAsync(flag, s);
    cudaFreeAsync(pos, s);
    cudaFreeAsync(mx, s);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? VDMC_ERR_OOM : VDMC_ERR_CUDA;
    return VDMC_OK;
}

namespace {

struct HubLayout {
    size_t posmap, qcnt, wq, touched, hptr, hlist, hcx, wx, htx, npoff, nplist, qrow, tbits, total;
};

HubLayout hub_layout(const vdmc_graph *g, int slots) {
    HubLayout L{};
    size_t o = 0;
    const size_t S = (size_t)slots, n = (size_t)g->n, t = (size_t)g->hub_tcap, lm = (size_t)g->hub_lmax;
    L.posmap = o; o += align256(S * n * 4);
    L.qcnt = o; o += align256(S * t * 9 * 4);
    L.wq = o; o += align256(S * t * 3 * 4);
    L.touched = o; o += align256(S * t * 4);
    L.hptr = o; o += align256(S * (lm + 1) * 4);
    L.hlist = o; o += align256(S * (size_t)g->hub_hcap * 4);
    L.hcx = o; o += align256(S * lm * 3 * 4);
    L.wx = o; o += align256(S * lm * 3 * 4);
    L.htx = o; o += align256(S * lm * 9 * 4);
    L.npoff = o; o += align256(S * (t + 1) * 4);
    L.nplist = o; o += align256(S * (size_t)g->hub_npcap * 4);
    L.qrow = o; o += align256(S * t * 16);
    L.tbits = o; o += align256(S * ((n + 31) / 32) * 4);
    L.total = o;
    return L;
}

}  // namespace

int vdmc_hub_count(const vdmc_graph *g) { return g->nhubs; }

template <int K, int W>
cudaError_t launch_hub(int slots, size_t dsmem, const HubArgs &A, cudaStream_t s) {
    // The attribute is per kernel, not per launch: host threads launching for
    // graphs of different sizes must not lower it under each other, so it is
    // always set to the largest P bitmap this CTA size may use.
    const int dmax = (int)(hub_smem_bits_max_words(W) * 4);
    if ((int)dsmem > dmax) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(hub_kernel<K, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, dmax);
    if (e != cudaSuccess) return e;
    hub_kernel<K, W><<<(unsigned)slots, W * 32, dsmem, s>>>(A);
    return cudaGetLastError();
}

vdmc_status vdmc_hub_launch(vdmc_graph *g, int k, uint64_t *out, uint64_t *d3, int d3_narrow, uint64_t *d3w,
                            const uint8_t *lut,
                            int32_t lo,
                            int32_t hi, int blocks_per_sm, int split, int split_roots, int warps, cudaStream_t s) {
    // 0: by the largest root -- 32 warps hide more of a long root's load
    // latency, 16 cost less per launch for graphs of small roots
    if (warps == 0) warps = g->hub_lmax >= VDMC_HUB_WARPS32_MIN_L ? 32 : 16;
    warps = warps == 32 ? 32 : 16;
    if (g->nhubs <= 0) return VDMC_OK;
    int dev = 0, sms = 0;
    VDMC_CUDA_TRY(cudaGetDevice(&dev));
    VDMC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // the largest roots (first in the hub list) are split into `split` parts
    const int C = k == 3 ? 13 : 199;
    const int32_t nsplit = split > 1 ? std::min(split_roots, g->nhubs) : 0;
    const int64_t queue = (int64_t)g->nhubs + (int64_t)nsplit * (split - 1);
    const size_t split_bytes = (size_t)nsplit * sizeof(unsigned long long) * C;
    if (nsplit > g->hub_split_cap) {
        vdmc_free(g->hub_split_buf, s);
        g->hub_split_buf = nullptr;
        g->hub_split_cap = 0;
        VDMC_CUDA_TRY(vdmc_malloc(&g->hub_split_buf, (size_t)nsplit * sizeof(unsigned long long) * 199, s));
        g->hub_split_cap = nsplit;
    }
    if (nsplit > 0) VDMC_CUDA_TRY(cudaMemsetAsync(g->hub_split_buf, 0, split_bytes, s));
    int slots = std::max(1, sms * std::max(1, blocks_per_sm));
    slots = (int)std::min<int64_t>(slots, queue);
    if (slots > g->hub_slots) {
        // (re)allocate the per-slot scratch; posmap starts at -1, counters at 0
        vdmc_free(g->hub_scratch, s);
        g->hub_scratch = nullptr;
        g->hub_slots = 0;
        HubLayout L = hub_layout(g, slots);
        VDMC_CUDA_TRY(vdmc_malloc(&g->hub_scratch, L.total, s));
        if (!g->hub_qhead) VDMC_CUDA_TRY(vdmc_malloc(&g->hub_qhead, sizeof(unsigned long long), s));
        char *base = (char *)g->hub_scratch;
        VDMC_CUDA_TRY(cudaMemsetAsync(base + L.qcnt, 0, L.wq - L.qcnt, s));
        VDMC_CUDA_TRY(cudaMemsetAsync(base + L.tbits, 0, L.total - L.tbits, s));
        const int64_t np = (int64_t)slots * g->n;
        if (np > 0) {
            fill_i32<<<(unsigned)((np + 255) / 256), 256, 0, s>>>((int32_t *)(base + L.posmap), np, -1);
            VDMC_CUDA_TRY(cudaGetLastError());
        }
        g->hub_slots = slots;
        g->hub_scratch_bytes = L.total;
    }
    HubLayout L = hub_layout(g, g->hub_slots);
    char *base = (char *)g->hub_scratch;
    HubArgs A;
    A.g = Csr{g->rowptr, g->col, g->pbeg, g->n, g->nnz, g->status};
    A.new2old = nullptr;  // credits in rank space (see vdmc_count_internal)
    A.out = out;
    A.d3 = (unsigned long long *)d3;
    A.d3_narrow = d3_narrow;
    A.d3w = (unsigned long long *)d3w;
    A.stats = g->stats;
    A.lut_g = lut;
    A.hubs = g->hubs;
    A.nhubs = g->nhubs;
    A.nsplit = nsplit;
    A.split = nsplit > 0 ? split : 1;
    A.split_acc = (unsigned long long *)g->hub_split_buf;
    A.rank_lo = lo;
    A.rank_hi = hi;
    A.qhead = g->hub_qhead;
    A.posmap = (int32_t *)(base + L.posmap);
    A.qcnt = (uint32_t *)(base + L.qcnt);
    A.wq = (uint32_t *)(base + L.wq);
    A.touched = (int32_t *)(base + L.touched);
    A.hptr = (int32_t *)(base + L.hptr);
    A.hlist = (uint32_t *)(base + L.hlist);
    A.hcx = (uint32_t *)(base + L.hcx);
    A.wx = (uint32_t *)(base + L.wx);
    A.htx = (uint32_t *)(base + L.htx);
    A.npoff = (int32_t *)(base + L.npoff);
    A.nplist = (uint32_t *)(base + L.nplist);
    A.npcap = g->hub_npcap;
    A.qrow = (longlong2 *)(base + L.qrow);
    A.tbits = (uint32_t *)(base + L.tbits);
    const int64_t words = ((int64_t)g->n + 31) / 32;
    A.pbits_words = words <= hub_smem_bits_max_words(warps) ? (int32_t)words : 0;
    const size_t dsmem = (size_t)A.pbits_words * 4;
    A.tcap = g->hub_tcap;
    A.hcap = g->hub_hcap;
    A.lmax = g->hub_lmax;
    VDMC_CUDA_TRY(cudaMemsetAsync(g->hub_qhead, 0, sizeof(unsigned long long), s));
    cudaError_t le;
    if (k == 3) le = warps == 32 ? launch_hub<3, 32>(slots, dsmem, A, s) : launch_hub<3, 16>(slots, dsmem, A, s);
    else le = warps == 32 ? launch_hub<4, 32>(slots, dsmem, A, s) : launch_hub<4, 16>(slots, dsmem, A, s);
    VDMC_CUDA_TRY(le);
    if (nsplit > 0) {
        split_finish<<<(unsigned)nsplit, 256, 0, s>>>(A.split_acc, g->hubs, nsplit, C, k == 3 ? 2ull : 3ull, g->n, out,
                                                      g->stats);
        VDMC_CUDA_TRY(cudaGetLastError());
    }
    if (k == 4 && d3 && d3w) {
        d3_spread<<<(unsigned)(((int64_t)g->n * 32 + 255) / 256), 256, 0, s>>>(g->rowptr, g->col, g->n, A.d3w, d3_narrow,
                                                                             lut, A.d3);
        VDMC_CUDA_TRY(cudaGetLastError());
    }
    return VDMC_OK;
}
