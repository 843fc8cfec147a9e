// Device-wide exclusive scan and LSD radix sort used by the graph build.
//
// Scan: tiles of 4096 elements (512 threads x 8); per-tile sums are scanned
// recursively and added back.  Radix sort: 8-bit digits; per pass a tile
// histogram kernel, a scan of the digit-major histogram, and a scatter
// kernel that ranks keys stably inside each tile (warp match on the digit,
// per-warp running counts in shared memory).
#include <cuda_runtime.h>

#include <cstdint>

#include "vdmc_internal.cuh"

namespace {

constexpr int SCAN_TPB = 512;
constexpr int SCAN_IPT = 8;
constexpr int SCAN_TILE = SCAN_TPB * SCAN_IPT;

template <typename T>
__device__ T block_exclusive_scan(T x, T *total) {
    __shared__ T warp_tot[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        T w = lane < nw ? warp_tot[lane] : T(0);
        T wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < nw) warp_tot[lane] = wi - w;  // exclusive prefix of warps
        if (lane == nw - 1) warp_tot[31] = wi;   // block total (nw <= 31 here)
    }
    __syncthreads();
    T res = warp_tot[warp] + inc - x;
    *total = warp_tot[31];
    __syncthreads();
    return res;
}

template <typename T>
__global__ void __launch_bounds__(SCAN_TPB) scan_tiles(const T *in, T *out, T *tile_sums, int64_t count) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_IPT;
    T v[SCAN_IPT];
    T sum = 0;
#pragma unroll
    for (int i = 0; i < SCAN_IPT; i++) {
        int64_t idx = base + i;
        v[i] = idx < count ? in[idx] : T(0);
        sum += v[i];
    }
    T total;
    T run = block_exclusive_scan<T>(sum, &total);
#pragma unroll
    for (int i = 0; i < SCAN_IPT; i++) {
        int64_t idx = base + i;
        if (idx < count) out[idx] = run;
        run += v[i];
    }
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

template <typename T>
__global__ void add_tile_offsets(T *out, const T *offs, int64_t count) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < count) out[idx] += offs[idx / SCAN_TILE];
}

template <typename T>
__global__ void copy_one(T *dst, const T *src) { *dst = *src; }

// out has count+1 slots; out[count] receives the total.  in may equal out.
template <typename T>
cudaError_t exclusive_scan(const T *in, T *out, int64_t count, cudaStream_t s) {
    if (count <= 0) return cudaMemsetAsync(out, 0, sizeof(T), s);
    const int64_t nb = (count + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 1) {
        scan_tiles<T><<<1, SCAN_TPB, 0, s>>>(in, out, out + count, count);
        return cudaGetLastError();
    }
    T *sums = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&sums, sizeof(T) * (size_t)(nb + 1), s);
    if (e != cudaSuccess) return e;
    scan_tiles<T><<<(unsigned)nb, SCAN_TPB, 0, s>>>(in, out, sums, count);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = exclusive_scan<T>(sums, sums, nb, s);
    if (e == cudaSuccess) {
        add_tile_offsets<T><<<(unsigned)((count + 255) / 256), 256, 0, s>>>(out, sums, count);
        copy_one<T><<<1, 1, 0, s>>>(out + count, sums + nb);
        e = cudaGetLastError();
    }
    cudaFreeAsync(sums, s);
    return e;
}

constexpr int RS_TPB = 256;
constexpr int RS_WARPS = RS_TPB / 32;
constexpr int RS_IPW = 16;                        // rounds of 32 keys per warp
constexpr int RS_TILE = RS_TPB * RS_IPW;          // 4096 keys per block

__global__ void __launch_bounds__(RS_TPB) rs_hist(const uint64_t *keys, int64_t count, int shift,
                                                  uint32_t dmask, uint32_t *hist, int64_t ntiles) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int i = 0; i < RS_IPW; i++) {
        int64_t idx = base + (int64_t)i * RS_TPB + threadIdx.x;
        if (idx < count) atomicAdd(&h[(uint32_t)(keys[idx] >> shift) & dmask], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RS_TPB) rs_scatter(const uint64_t *keys, uint64_t *out, int64_t count,
                                                     int shift, uint32_t dmask, const uint32_t *offs,
                                                     int64_t ntiles) {
    __shared__ uint32_t wc[RS_WARPS][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_TPB) (&wc[0][0])[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)w * (32 * RS_IPW);
    const uint32_t lt = (1u << lane) - 1u;
    uint64_t k[RS_IPW];
    uint32_t pos[RS_IPW];
#pragma unroll
    for (int i = 0; i < RS_IPW; i++) {
        int64_t idx = base + i * 32 + lane;
        bool valid = idx < count;
        k[i] = valid ? keys[idx] : 0ull;
        uint32_t d = valid ? ((uint32_t)(k[i] >> shift) & dmask) : 256u;
        uint32_t peers = __match_any_sync(0xffffffffu, d);
        uint32_t before = valid ? wc[w][d] : 0u;
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) wc[w][d] = before + __popc(peers);
        __syncwarp();
        pos[i] = before + __popc(peers & lt);
    }
    __syncthreads();
    {
        const int d = threadIdx.x;  // RS_TPB == 256 digits
        uint32_t run = offs[(int64_t)d * ntiles + blockIdx.x];
#pragma unroll
        for (int ww = 0; ww < RS_WARPS; ww++) {
            uint32_t t = wc[ww][d];
            wc[ww][d] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RS_IPW; i++) {
        int64_t idx = base + i * 32 + lane;
        if (idx < count) {
            uint32_t d = (uint32_t)(k[i] >> shift) & dmask;
            out[wc[w][d] + pos[i]] = k[i];
        }
    }
}

}  // namespace

cudaError_t vdmc_exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t count, cudaStream_t s) {
    return exclusive_scan<uint32_t>(in, out, count, s);
}

cudaError_t vdmc_exclusive_scan_i64(const int64_t *in, int64_t *out, int64_t count, cudaStream_t s) {
    return exclusive_scan<int64_t>(in, out, count, s);
}

cudaError_t vdmc_radix_sort_u64(uint64_t *keys, uint64_t *tmp, int64_t count, int begin_bit, int end_bit,
                                cudaStream_t s, uint64_t **result) {
    *result = keys;
    if (count <= 1 || begin_bit >= end_bit) return cudaSuccess;
    if (count > 0xffffffffll) return cudaErrorInvalidValue;
    const int64_t ntiles = (count + RS_TILE - 1) / RS_TILE;
    uint32_t *hist = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&hist, sizeof(uint32_t) * (size_t)(256 * ntiles + 1), s);
    if (e != cudaSuccess) return e;
    uint64_t *src = keys, *dst = tmp;
    for (int shift = begin_bit; shift < end_bit && e == cudaSuccess; shift += 8) {
        int nb = end_bit - shift < 8 ? end_bit - shift : 8;
        uint32_t dmask = (1u << nb) - 1u;
        rs_hist<<<(unsigned)ntiles, RS_TPB, 0, s>>>(src, count, shift, dmask, hist, ntiles);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = exclusive_scan<uint32_t>(hist, hist, 256 * ntiles, s);
        if (e == cudaSuccess) {
            rs_scatter<<<(unsigned)ntiles, RS_TPB, 0, s>>>(src, dst, count, shift, dmask, hist, ntiles);
            e = cudaGetLastError();
        }
        uint64_t *t = src;
        src = dst;
        dst = t;
    }
    cudaFreeAsync(hist, s);
    *result = src;
    return e;
}
