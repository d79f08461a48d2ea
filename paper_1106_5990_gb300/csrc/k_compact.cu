// k_compact.cu -- the strength graph M^1 (§4.2) as CSR from the per-slot
// flags and per-row counts written by the edge pass.
//
// Three launches, no device-wide waits:
//   1. tile sums: every block sums the strong counts of kTileRows rows
//   2. one block turns the tile sums into exclusive tile offsets
//   3. every block writes s_row_ptr for its rows (block scan of the counts
//      plus the tile offset) and compacts the flagged slots of its rows'
//      contiguous slot range into s_col (16 flag bytes per thread, counted
//      with popc, one block scan per 4096 slots), keeping A's row and slot
//      order.
#include "amgd_internal.cuh"

namespace amgd {
namespace {

constexpr int kSumThreads = 256;
constexpr int kCompactThreads = 256;
constexpr int kRowsPerThread = kTileRows / kCompactThreads;     // 4
constexpr int kSlotsPerThread = 16;                             // one 16-byte flag load

// exclusive block scan of one int per thread; returns the block total
template <int NT>
__device__ __forceinline__ int block_exclusive_scan(int v, int &total, int *smem_warp)
{
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) smem_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        int w = lane < NT / 32 ? smem_warp[lane] : 0;
        int winc = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, winc, o);
            if (lane >= o) winc += t;
        }
        if (lane < NT / 32) smem_warp[lane] = winc - w;   // exclusive warp offsets
        if (lane == NT / 32 - 1) smem_warp[32] = winc;     // block total
    }
    __syncthreads();
    const int out = smem_warp[warp] + inc - v;
    total = smem_warp[32];
    __syncthreads();
    return out;
}

__global__ void __launch_bounds__(kSumThreads)
k_tile_sums(const int32_t *__restrict__ count, int32_t n, int32_t *__restrict__ tile_sum)
{
    __shared__ int sm[33];
    const int64_t r = (int64_t)blockIdx.x * kTileRows + threadIdx.x * 4;
    int s = 0;
    if (r + 3 < n) {
        const int4 c = __ldg(reinterpret_cast<const int4 *>(count + r));
        s = c.x + c.y + c.z + c.w;
    } else {
        for (int k = 0; k < 4; ++k) s += (r + k < n) ? count[r + k] : 0;
    }
    int total;
    block_exclusive_scan<kSumThreads>(s, total, sm);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

// in-place exclusive scan of ntiles tile sums by one block
__global__ void __launch_bounds__(1024) k_tile_scan(int32_t *__restrict__ tile_sum, int32_t ntiles)
{
    __shared__ int sm[33];
    int carry = 0;
    for (int base = 0; base < ntiles; base += 1024) {
        const int k = base + threadIdx.x;
        const int v = k < ntiles ? tile_sum[k] : 0;
        int total;
        const int ex = block_exclusive_scan<1024>(v, total, sm);
        if (k < ntiles) tile_sum[k] = carry + ex;
        carry += total;
    }
}

__global__ void __launch_bounds__(kCompactThreads)
k_compact(const int32_t *__restrict__ count, const int32_t *__restrict__ rp,
          const int32_t *__restrict__ col, const uint8_t *__restrict__ flag, int32_t n,
          const int32_t *__restrict__ tile_off, int64_t *__restrict__ s_row_ptr,
          int32_t *__restrict__ s_col)
{
    __shared__ int sm[33];
    const int64_t row0 = (int64_t)blockIdx.x * kTileRows;
    const int64_t row_end = min((int64_t)n, row0 + kTileRows);
    const int64_t off = tile_off[blockIdx.x];

    // row pointers: four consecutive rows per thread, block scan of the sums
    int c[kRowsPerThread];
    int mine = 0;
    const int64_t rbase = row0 + (int64_t)threadIdx.x * kRowsPerThread;
#pragma unroll
    for (int k = 0; k < kRowsPerThread; ++k) {
        c[k] = (rbase + k < row_end) ? count[rbase + k] : 0;
        mine += c[k];
    }
    int total;
    int run = block_exclusive_scan<kCompactThreads>(mine, total, sm);
#pragma unroll
    for (int k = 0; k < kRowsPerThread; ++k) {
        if (rbase + k < row_end) s_row_ptr[rbase + k] = off + run;
        run += c[k];
    }
    if (row_end == n && threadIdx.x == 0) s_row_ptr[n] = off + total;

    // kept slots of the tile's slot range [s0, s1), in slot order: every
    // thread takes 16 consecutive flag bytes (one 16-byte load from a
    // 16-byte-aligned base; the flag array is padded by 16 bytes) and, if any
    // is set, their 16 column indices (four 16-byte loads; the column array is
    // padded by 64 bytes).  The kept columns of a chunk are collected in
    // shared memory and written out with coalesced stores.
    __shared__ int32_t kept[kCompactThreads * kSlotsPerThread];
    const int64_t s0 = rp[row0], s1 = rp[row_end];
    int64_t out = off;
    for (int64_t base = s0 & ~(int64_t)15; base < s1;
         base += (int64_t)kCompactThreads * kSlotsPerThread) {
        const int64_t first = base + (int64_t)threadIdx.x * kSlotsPerThread;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (first < s1) v = __ldg(reinterpret_cast<const uint4 *>(flag + first));
        uint32_t w[4] = {v.x, v.y, v.z, v.w};
        // clear the bytes outside [s0, s1)
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int64_t slot = first + k;
            if (slot < s0 || slot >= s1) w[k / 4] &= ~(0xffu << (8 * (k % 4)));
        }
        const int cnt = __popc(w[0]) + __popc(w[1]) + __popc(w[2]) + __popc(w[3]);
        int chunk;
        int pos = block_exclusive_scan<kCompactThreads>(cnt, chunk, sm);
        if (cnt) {
            int c16[16];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int4 c4 = __ldg(reinterpret_cast<const int4 *>(col + first) + q);
                c16[4 * q] = c4.x; c16[4 * q + 1] = c4.y; c16[4 * q + 2] = c4.z; c16[4 * q + 3] = c4.w;
            }
#pragma unroll
            for (int k = 0; k < 16; ++k)
                if ((w[k / 4] >> (8 * (k % 4))) & 1u) kept[pos++] = c16[k];
        }
        __syncthreads();
        for (int q = threadIdx.x; q < chunk; q += kCompactThreads) s_col[out + q] = kept[q];
        __syncthreads();
        out += chunk;
    }
}

// row pointers only (first half of k_compact)
__global__ void __launch_bounds__(kCompactThreads)
k_row_ptr(const int32_t *__restrict__ count, int32_t n, const int32_t *__restrict__ tile_off,
          int64_t *__restrict__ row_ptr)
{
    __shared__ int sm[33];
    const int64_t row0 = (int64_t)blockIdx.x * kTileRows;
    const int64_t row_end = min((int64_t)n, row0 + kTileRows);
    const int64_t off = tile_off[blockIdx.x];
    int c[kRowsPerThread];
    int mine = 0;
    const int64_t rbase = row0 + (int64_t)threadIdx.x * kRowsPerThread;
#pragma unroll
    for (int k = 0; k < kRowsPerThread; ++k) {
        c[k] = (rbase + k < row_end) ? count[rbase + k] : 0;
        mine += c[k];
    }
    int total;
    int run = block_exclusive_scan<kCompactThreads>(mine, total, sm);
#pragma unroll
    for (int k = 0; k < kRowsPerThread; ++k) {
        if (rbase + k < row_end) row_ptr[rbase + k] = off + run;
        run += c[k];
    }
    if (row_end == n && threadIdx.x == 0) row_ptr[n] = off + total;
}

}  // namespace

cudaError_t launch_row_ptr(const int32_t *count, int32_t n, int32_t *tile_sum, int64_t *row_ptr,
                           cudaStream_t s)
{
    if (n == 0) {
        cudaError_t e = cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), s);
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    const int ntiles = (int)(((int64_t)n + kTileRows - 1) / kTileRows);
    k_tile_sums<<<ntiles, kSumThreads, 0, s>>>(count, n, tile_sum);
    k_tile_scan<<<1, 1024, 0, s>>>(tile_sum, ntiles);
    k_row_ptr<<<ntiles, kCompactThreads, 0, s>>>(count, n, tile_sum, row_ptr);
    return cudaGetLastError();
}

cudaError_t launch_strength(const int32_t *count, const int32_t *rp_orig, const int32_t *col_orig,
                            const uint8_t *flag, int32_t n, int32_t *tile_sum,
                            int64_t *s_row_ptr, int32_t *s_col, cudaStream_t s)
{
    if (n == 0) {
        cudaError_t e = cudaMemsetAsync(s_row_ptr, 0, sizeof(int64_t), s);
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    const int ntiles = (int)(((int64_t)n + kTileRows - 1) / kTileRows);
    k_tile_sums<<<ntiles, kSumThreads, 0, s>>>(count, n, tile_sum);
    k_tile_scan<<<1, 1024, 0, s>>>(tile_sum, ntiles);
    k_compact<<<ntiles, kCompactThreads, 0, s>>>(count, rp_orig, col_orig, flag, n, tile_sum,
                                                s_row_ptr, s_col);
    return cudaGetLastError();
}

}  // namespace amgd
