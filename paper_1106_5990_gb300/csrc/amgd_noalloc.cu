// amgd_noalloc.cu -- amgd_strength_noalloc: the row-relative threshold and
// the strength CSR computed from caller-supplied distances without allocating
// any memory.
//
// Why it exists: some callers cannot call cudaMalloc -- code running inside a
// memory pool or arena that owns every device allocation of the process, an
// allocator-free real-time loop, or a host thread that must never take the
// CUDA driver's allocation lock.  Every handle-based entry point allocates device
// memory (the handle owns its buffers), so such callers get this one entry
// point instead: the caller passes every input and output buffer, and the only
// working memory is the file-scope array below.
//
// The scratch array holds one int64 per tile of kNaTileRows rows (the
// exclusive offsets of the tiles' strong-edge counts; 64-bit, so a strength
// graph with 2^31 or more edges is counted exactly).  It lives in the
// library's device image, so every GPU that loads the library holds its
// 512 KiB until the process exits.  All calls share it: each call overwrites
// the entries of its own tiles before reading them (nothing has to start at
// zero), and two calls whose work overlaps on the GPU (different streams, or
// different host threads on the same device) race on it.
#include "../../include/amgd.h"

#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "amgd_internal.cuh"

namespace {

constexpr int kNaTileRows = 4096;
constexpr int kNaMaxTiles = 65536;            // 512 KiB of scratch
constexpr int64_t kNaMaxRows = (int64_t)kNaTileRows * kNaMaxTiles;
constexpr int kNaThreads = 512;
constexpr int kNaWarps = kNaThreads / 32;
constexpr int kNaMaxDevices = 64;

static __device__ __align__(256) int64_t g_na_tile_scratch[kNaMaxTiles];

// min_k LS_ik over the off-diagonal slots of row i, and the number of strong
// slots (LS = 0 or theta LS < min), evaluated by one warp
__device__ __forceinline__ void na_row(const int64_t *rp, const int32_t *col, const double *ls,
                                       int64_t i, double theta, double &m, int &cnt)
{
    const int lane = threadIdx.x % 32;
    const int64_t p0 = rp[i], p1 = rp[i + 1];
    m = INFINITY;
    for (int64_t p = p0 + lane; p < p1; p += 32)
        if (col[p] != i) m = fmin(m, ls[p]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    cnt = 0;
    for (int64_t base = p0; base < p1; base += 32) {
        const int64_t p = base + lane;
        bool s = false;
        if (p < p1 && col[p] != i) s = (ls[p] == 0.0) || (theta * ls[p] < m);
        cnt += __popc(__ballot_sync(0xffffffffu, s));
    }
}

// pass 1: strong count of every tile into the scratch array
__global__ void __launch_bounds__(kNaThreads)
k_na_tile_counts(const int64_t *rp, const int32_t *col, const double *ls, int64_t n,
                 double theta, int64_t *tile)
{
    __shared__ long long warp_tot[kNaWarps];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t r0 = (int64_t)blockIdx.x * kNaTileRows;
    const int64_t r1 = min(n, r0 + kNaTileRows);
    long long tot = 0;
    for (int64_t i = r0 + warp; i < r1; i += kNaWarps) {
        double m;
        int c;
        na_row(rp, col, ls, i, theta, m, c);
        tot += c;
    }
    if (lane == 0) warp_tot[warp] = tot;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long s = 0;
        for (int w = 0; w < kNaWarps; ++w) s += warp_tot[w];
        tile[blockIdx.x] = s;
    }
}

// pass 2: exclusive scan of the tile counts, one block (64-bit sums and carry)
__global__ void __launch_bounds__(1024) k_na_tile_scan(int64_t *tile, int ntiles)
{
    __shared__ long long part[1024];
    long long carry = 0;
    for (int base = 0; base < ntiles; base += 1024) {
        const int k = base + threadIdx.x;
        const long long v = k < ntiles ? tile[k] : 0;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const long long t = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
            __syncthreads();
            part[threadIdx.x] += t;
            __syncthreads();
        }
        if (k < ntiles) tile[k] = carry + part[threadIdx.x] - v;
        const long long total = part[1023];
        __syncthreads();
        carry += total;
    }
}

// pass 3: row pointers and kept columns of every tile
__global__ void __launch_bounds__(kNaThreads)
k_na_compact(const int64_t *rp, const int32_t *col, const double *ls, int64_t n, double theta,
             const int64_t *tile, int64_t *s_rp, int32_t *s_col, int64_t cap)
{
    __shared__ long long warp_tot[kNaWarps];
    __shared__ long long warp_off[kNaWarps];
    __shared__ long long blk_tot;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int64_t r0 = (int64_t)blockIdx.x * kNaTileRows;
    const int64_t r1 = min(n, r0 + kNaTileRows);
    // each warp owns a contiguous run of rows of the tile
    const int64_t rows_per_warp = (kNaTileRows + kNaWarps - 1) / kNaWarps;
    const int64_t w0 = min(r1, r0 + warp * rows_per_warp);
    const int64_t w1 = min(r1, w0 + rows_per_warp);
    long long tot = 0;
    for (int64_t i = w0; i < w1; ++i) {
        double m;
        int c;
        na_row(rp, col, ls, i, theta, m, c);
        tot += c;
    }
    if (lane == 0) warp_tot[warp] = tot;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long s = 0;
        for (int w = 0; w < kNaWarps; ++w) { warp_off[w] = s; s += warp_tot[w]; }
        blk_tot = s;
    }
    __syncthreads();
    int64_t out = (int64_t)tile[blockIdx.x] + warp_off[warp];
    for (int64_t i = w0; i < w1; ++i) {
        double m;
        int c;
        na_row(rp, col, ls, i, theta, m, c);
        if (lane == 0) s_rp[i] = out;
        const int64_t p0 = rp[i], p1 = rp[i + 1];
        for (int64_t base = p0; base < p1; base += 32) {
            const int64_t p = base + lane;
            bool s = false;
            if (p < p1 && col[p] != i) s = (ls[p] == 0.0) || (theta * ls[p] < m);
            const unsigned b = __ballot_sync(0xffffffffu, s);
            const int64_t pos = out + __popc(b & ((1u << lane) - 1u));
            if (s && pos < cap) s_col[pos] = col[p];
            out += __popc(b);
        }
    }
    if (r1 == n && threadIdx.x == 0) s_rp[n] = (int64_t)tile[blockIdx.x] + blk_tot;
}

std::mutex g_na_mu;
int64_t *g_na_ptr[kNaMaxDevices] = {};

}  // namespace

extern "C" int amgd_strength_noalloc(const int64_t *row_ptr, const int32_t *col, const double *ls,
                                     int64_t n, double theta, int64_t *s_row_ptr, int32_t *s_col,
                                     int64_t cap, void *stream)
{
    if (n < 0) {
        amgd::set_thread_error("amgd_strength_noalloc: n = " + std::to_string(n) + " < 0");
        return AMGD_ERR_ARG;
    }
    if (n > kNaMaxRows) {
        amgd::set_thread_error("amgd_strength_noalloc: n = " + std::to_string(n) +
                               " is above " + std::to_string(kNaMaxRows) +
                               " (the static scratch holds " + std::to_string(kNaMaxTiles) +
                               " tiles of " + std::to_string(kNaTileRows) + " rows)");
        return AMGD_ERR_UNSUPPORTED;
    }
    if (!(theta >= 0.0) || theta > 1e300 || cap < 0 || !row_ptr || !s_row_ptr ||
        (n > 0 && (!col || !ls)) || (cap > 0 && !s_col)) {
        amgd::set_thread_error("amgd_strength_noalloc: bad argument");
        return AMGD_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) {
        amgd::set_thread_error("amgd_strength_noalloc: no usable current device");
        return AMGD_ERR_CUDA;
    }
    int64_t *tile = nullptr;
    {
        // once per device, with that device current: the device address of
        // the scratch array (its host-side name is not a device address)
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na_ptr[dev]) {
            e = cudaGetSymbolAddress((void **)&g_na_ptr[dev], g_na_tile_scratch);
            if (e != cudaSuccess) {
                g_na_ptr[dev] = nullptr;
                amgd::set_thread_error(std::string("amgd_strength_noalloc: cudaGetSymbolAddress: ") +
                                       cudaGetErrorString(e));
                return AMGD_ERR_CUDA;
            }
        }
        tile = g_na_ptr[dev];
    }
    if (n == 0) {
        e = cudaMemsetAsync(s_row_ptr, 0, sizeof(int64_t), s);
    } else {
        const int ntiles = (int)((n + kNaTileRows - 1) / kNaTileRows);
        k_na_tile_counts<<<ntiles, kNaThreads, 0, s>>>(row_ptr, col, ls, n, theta, tile);
        k_na_tile_scan<<<1, 1024, 0, s>>>(tile, ntiles);
        k_na_compact<<<ntiles, kNaThreads, 0, s>>>(row_ptr, col, ls, n, theta, tile, s_row_ptr,
                                                   s_col, cap);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        amgd::set_thread_error(std::string("amgd_strength_noalloc: ") + cudaGetErrorString(e));
        return AMGD_ERR_CUDA;
    }
    return AMGD_OK;
}
