// Exclusive prefix sum of unsigned counts, in place, in two launches: per-chunk
// totals, then per-chunk scans, each chunk's offset summed by its own block
// from the totals before it (no separate pass over the totals).
// Used by the radix sort (digit histograms) and by the vertex adjacency
// (degree counts).
#include "ag_internal.cuh"

namespace ag {
namespace {

constexpr int SB = 256;            // threads per block
constexpr int SI = 8;              // items per thread
constexpr int SCHUNK = SB * SI;    // items per block

__device__ __forceinline__ unsigned warp_incl(unsigned v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// exclusive scan of one value per thread over the block; returns the block total
__device__ __forceinline__ unsigned block_excl(unsigned v, unsigned *excl) {
    __shared__ unsigned wsum[SB / 32];
    __shared__ unsigned s_total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned inc = warp_incl(v);
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        unsigned w = lane < SB / 32 ? wsum[lane] : 0u;
        unsigned wi = warp_incl(w);
        if (lane < SB / 32) wsum[lane] = wi - w;
        if (lane == SB / 32 - 1) s_total = wi;
    }
    __syncthreads();
    *excl = inc - v + wsum[warp];
    unsigned total = s_total;
    __syncthreads();
    return total;
}

__global__ void __launch_bounds__(SB) k_scan_reduce(const unsigned *__restrict__ d, int64_t n, unsigned *__restrict__ bsum) {
    int64_t base = (int64_t)blockIdx.x * SCHUNK;
    unsigned s = 0;
    for (int i = threadIdx.x; i < SCHUNK; i += SB) {
        int64_t j = base + i;
        if (j < n) s += d[j];
    }
    unsigned ex;
    unsigned tot = block_excl(s, &ex);
    if (threadIdx.x == SB - 1) bsum[blockIdx.x] = tot;
    (void)ex;
}

// the chunk's offset: the sum of the chunk totals before it (the last chunk
// also writes the grand total)
__global__ void __launch_bounds__(SB) k_scan_apply(unsigned *__restrict__ d, int64_t n, const unsigned *__restrict__ bsum,
                                                   unsigned *__restrict__ total) {
    __shared__ unsigned tile[SCHUNK];
    unsigned before = 0;
    for (unsigned j = threadIdx.x; j < blockIdx.x; j += SB) before += __ldg(&bsum[j]);
    unsigned ex0;
    const unsigned chunk_off = block_excl(before, &ex0);   // block total = sum of the totals before this chunk
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total = chunk_off + bsum[blockIdx.x];
    int64_t base = (int64_t)blockIdx.x * SCHUNK;
    for (int i = threadIdx.x; i < SCHUNK; i += SB) {
        int64_t j = base + i;
        tile[i] = j < n ? d[j] : 0u;
    }
    __syncthreads();
    unsigned loc[SI], s = 0;
#pragma unroll
    for (int k = 0; k < SI; ++k) {
        loc[k] = s;
        s += tile[threadIdx.x * SI + k];
    }
    unsigned ex;
    block_excl(s, &ex);
    unsigned off = chunk_off + ex;
#pragma unroll
    for (int k = 0; k < SI; ++k) tile[threadIdx.x * SI + k] = off + loc[k];
    __syncthreads();
    for (int i = threadIdx.x; i < SCHUNK; i += SB) {
        int64_t j = base + i;
        if (j < n) d[j] = tile[i];
    }
}

// one block, the chunks in order with a running carry (short inputs: one
// launch instead of three)
__global__ void __launch_bounds__(SB) k_scan_small(unsigned *__restrict__ d, int64_t n, unsigned *__restrict__ total) {
    __shared__ unsigned tile[SCHUNK];
    __shared__ unsigned carry;
    if (threadIdx.x == 0) carry = 0;
    for (int64_t base = 0; base < n; base += SCHUNK) {
        __syncthreads();
        for (int i = threadIdx.x; i < SCHUNK; i += SB) {
            const int64_t j = base + i;
            tile[i] = j < n ? d[j] : 0u;
        }
        __syncthreads();
        unsigned loc[SI], s = 0;
#pragma unroll
        for (int k = 0; k < SI; ++k) {
            loc[k] = s;
            s += tile[threadIdx.x * SI + k];
        }
        unsigned ex;
        const unsigned tot = block_excl(s, &ex);
        const unsigned off = carry + ex;
#pragma unroll
        for (int k = 0; k < SI; ++k) tile[threadIdx.x * SI + k] = off + loc[k];
        __syncthreads();
        for (int i = threadIdx.x; i < SCHUNK; i += SB) {
            const int64_t j = base + i;
            if (j < n) d[j] = tile[i];
        }
        if (threadIdx.x == 0) carry += tot;
    }
    __syncthreads();
    if (threadIdx.x == 0 && total) *total = carry;
}

constexpr int64_t SMALL_CHUNKS = 4;   // inputs of up to this many chunks take k_scan_small

}  // namespace

size_t scan_scratch_bytes(int64_t n) {
    int64_t nb = (n + SCHUNK - 1) / SCHUNK;
    return sizeof(unsigned) * (size_t)(nb + 1);
}

cudaError_t launch_scan_exclusive(unsigned *d, int64_t n, unsigned *total, void *scratch, cudaStream_t s) {
    int64_t nb = (n + SCHUNK - 1) / SCHUNK;
    if (nb < 1) nb = 1;
    if (nb <= SMALL_CHUNKS) {
        k_scan_small<<<1, SB, 0, s>>>(d, n, total);
        return cudaGetLastError();
    }
    unsigned *bsum = static_cast<unsigned *>(scratch);
    k_scan_reduce<<<(unsigned)nb, SB, 0, s>>>(d, n, bsum);
    k_scan_apply<<<(unsigned)nb, SB, 0, s>>>(d, n, bsum, total);
    return cudaGetLastError();
}

}  // namespace ag
