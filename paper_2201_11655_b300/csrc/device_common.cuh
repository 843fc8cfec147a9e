// Device helpers shared by the enumeration kernels: CSR view, checked
// accessors, adjacency search, motif index and credit.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "vdmc_internal.cuh"

namespace {

// ------------------------------------------------------- enumeration -----

struct Csr {
    const int64_t *__restrict__ rowptr;
    const uint32_t *__restrict__ col;
    const int64_t *__restrict__ pbeg;
    int64_t n;
    int64_t nnz;
    int *status;  // device status word; also receives bounds violations
};

// Every data-dependent index is checked before use.  A violation (which a
// correct CSR never produces) sets the status word and the access is
// skipped, so a corrupted input cannot make the kernel fault.
__device__ __forceinline__ bool in_bounds(const Csr &g, bool ok) {
    if (!ok) atomicExch(g.status, (int)VDMC_ERR_DEVICE_LIMIT);
    return ok;
}

// flags of neighbour v in the sorted entries col[lo, hi); 0 if absent.
// A stored edge always has non-zero flags.
__device__ __forceinline__ uint32_t search_row(const uint32_t *__restrict__ col, int64_t lo, int64_t hi,
                                               uint32_t v) {
    const uint32_t *p = col + lo;
    int32_t len = (int32_t)(hi - lo);
    while (len > 0) {
        int32_t half = len >> 1;
        uint32_t e = __ldg(p + half);
        if ((e >> 2) < v) {
            p += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    if (p < col + hi) {
        uint32_t e = __ldg(p);
        if ((e >> 2) == v) return e & 3u;
    }
    return 0u;
}

// first position in col[lo, hi) with neighbour rank > v
__device__ __forceinline__ int64_t upper_row(const uint32_t *__restrict__ col, int64_t lo, int64_t hi,
                                             uint32_t v) {
    int32_t len = (int32_t)(hi - lo);
    int64_t base = lo;
    while (len > 0) {
        int32_t half = len >> 1;
        if ((__ldg(col + base + half) >> 2) <= v) {
            base += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return base;
}

// flags of the pair (u, v): bit0 = arc u->v, bit1 = arc v->u; 0 = no edge.
__device__ __forceinline__ uint32_t pair_flags(const Csr &g, uint32_t u, uint32_t v) {
    if (!in_bounds(g, u < g.n && v < g.n)) return 0u;
    int64_t ub = __ldg(g.rowptr + u), ue = __ldg(g.rowptr + u + 1);
    int64_t vb = __ldg(g.rowptr + v), ve = __ldg(g.rowptr + v + 1);
    if (!in_bounds(g, ub >= 0 && ub <= ue && ue <= g.nnz && vb >= 0 && vb <= ve && ve <= g.nnz)) return 0u;
    if (ue - ub <= ve - vb) return search_row(g.col, ub, ue, v);
    uint32_t f = search_row(g.col, vb, ve, u);
    return ((f & 1u) << 1) | (f >> 1);
}

// Motif index of the ordered tuple (r, a, b) from the three pair flags.
// Bit order (Fig. 1): (0,1) (0,2) (1,0) (1,2) (2,0) (2,1), MSB first.
__device__ __forceinline__ uint32_t mask3(uint32_t fra, uint32_t frb, uint32_t fab) {
    return ((fra & 1u) << 5) | ((frb & 1u) << 4) | ((fra >> 1) << 3) | ((fab & 1u) << 2) | ((frb >> 1) << 1) |
           (fab >> 1);
}

// Motif index of (r, a, b, c): (0,1) (0,2) (0,3) (1,0) (1,2) (1,3) (2,0)
// (2,1) (2,3) (3,0) (3,1) (3,2), MSB first.
__device__ __forceinline__ uint32_t mask4(uint32_t fra, uint32_t frb, uint32_t frc, uint32_t fab, uint32_t fac,
                                          uint32_t fbc) {
    return ((fra & 1u) << 11) | ((frb & 1u) << 10) | ((frc & 1u) << 9) | ((fra >> 1) << 8) | ((fab & 1u) << 7) |
           ((fac & 1u) << 6) | ((frb >> 1) << 5) | ((fab >> 1) << 4) | ((fbc & 1u) << 3) | ((frc >> 1) << 2) |
           ((fac >> 1) << 1) | (fbc >> 1);
}

// Column of the depth-3 credit type j = 3 * type + flag - 1 (type = 3 *
// (colour - 1) + h(x, b) - 1, flag = h(b, c)): the rank of its class among the
// distinct classes of the 27 types.  *cls_out gets the class itself.
__device__ __forceinline__ int d3_column(const uint8_t *lut, int j, int *cls_out) {
    auto cls_of = [&](int t) {
        const uint32_t k = (uint32_t)t / 3;
        return (int)lut[mask4(k / 3 + 1, 0u, 0u, k % 3 + 1, 0u, (uint32_t)t % 3 + 1)];
    };
    const int c = cls_of(j);
    int rank = 0;
    for (int i = 0; i < 27; i++) {
        const int ci = cls_of(i);
        bool first = ci < c;
        for (int m = 0; m < i && first; m++) first = cls_of(m) != ci;
        rank += first ? 1 : 0;
    }
    *cls_out = c;
    return rank;
}

// Output row of vertex (rank) v: its original id through the id map, or v
// itself when the kernel accumulates in rank space (map == nullptr; the
// rows are permuted to original ids afterwards).
__device__ __forceinline__ int32_t row_of(const int32_t *map, uint32_t v) {
    return map ? __ldg(map + v) : (int32_t)v;
}

// +1 for vertex (rank) v in column cls of its output row
__device__ __forceinline__ void credit(const Csr &g, uint64_t *out, const int32_t *new2old, uint32_t v, int C,
                                       uint32_t cls) {
    if (!in_bounds(g, v < g.n)) return;
    const int32_t o = row_of(new2old, v);
    if (!in_bounds(g, o >= 0 && o < g.n)) return;
    atomicAdd((unsigned long long *)&out[(int64_t)o * C + cls], 1ull);
}

// A uint64 histogram in shared memory kept as 32-bit halves (lo[C], hi[C])
// in the same C * 8 bytes.  An add is one native 32-bit shared atomic on the
// low half, plus one on the high half only for the carry of a wrap (or the
// upper word of a large or negative add); 64-bit shared-memory atomics are
// compare-and-swap loops that collapse when many lanes hit one counter.
// Exact modulo 2^64 once all adds have completed.
struct Hist64 {
    uint32_t *lo, *hi;
};

__device__ __forceinline__ Hist64 hist64(unsigned long long *h, int C) {
    return Hist64{reinterpret_cast<uint32_t *>(h), reinterpret_cast<uint32_t *>(h) + C};
}

__device__ __forceinline__ void hadd(const Hist64 &h, uint32_t i, unsigned long long v) {
    const uint32_t vl = (uint32_t)v, vh = (uint32_t)(v >> 32);
    uint32_t carry = 0u;
    if (vl) {
        const uint32_t old = atomicAdd(h.lo + i, vl);
        carry = (uint32_t)(old + vl) < old ? 1u : 0u;
    }
    if (vh + carry) atomicAdd(h.hi + i, vh + carry);
}

__device__ __forceinline__ void hinc(const Hist64 &h, uint32_t i) {
    if (atomicAdd(h.lo + i, 1u) == 0xffffffffu) atomicAdd(h.hi + i, 1u);
}

__device__ __forceinline__ unsigned long long hget(const Hist64 &h, uint32_t i) {
    return ((unsigned long long)h.hi[i] << 32) | h.lo[i];
}

// add a warp's histogram to output row orig (one global atomic per non-zero
// column) and leave it zero
__device__ __forceinline__ void flush_hist(const Csr &g, const Hist64 &h, int C, uint64_t *out, int32_t orig,
                                           int lane) {
    __syncwarp();
    const bool ok = in_bounds(g, orig >= 0 && orig < g.n);
    for (int c = lane; c < C; c += 32) {
        const unsigned long long v = hget(h, c);
        if (v) {
            if (ok) atomicAdd((unsigned long long *)&out[(int64_t)orig * C + c], v);
            h.lo[c] = 0u;
            h.hi[c] = 0u;
        }
    }
    __syncwarp();
}


}  // namespace
