// amgd_internal.cuh -- types shared by the kernels and the host API of the
// GB300 algebraic-distance library (not part of the public ABI).
//
// Device data layout (all in HBM, owned by the handle):
//   * permuted CSR of A: rows reordered by color when a coloring is set
//     (identity otherwise), slot order inside a row unchanged; int32 row_ptr
//     and col, values as FP64 and (for the mixed paths) FP32.
//   * original CSR row_ptr / col: the numbering of every per-slot output.
//   * test vectors X: two n x Kp row-major buffers (ping-pong) in the
//     storage type; Kp = G * V pads K to a whole number of 16-byte vectors
//     per lane (V elements per 16 bytes, G lanes per row), padding is zero.
//   * per-slot outputs a, LS (FP64 or FP32), strength flag (u8); per-row
//     strong counts (int32, caller's row order).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <atomic>
#include <string>

namespace amgd {

enum Storage { ST_FP64 = 0, ST_FP32 = 1, ST_BF16 = 2 };

// ---------------------------------------------------------------------------
// storage traits: TS = stored element, C = arithmetic type, V = elements per
// 16-byte vector, A = stored matrix value type used by the sweeps.
// ---------------------------------------------------------------------------
template <class TS> struct Store;

template <> struct Store<double> {
    using C = double;
    using A = double;
    static constexpr int V = 2;
    __device__ __forceinline__ static void unpack(const uint4 &v, C (&x)[V]) {
        x[0] = __hiloint2double((int)v.y, (int)v.x);
        x[1] = __hiloint2double((int)v.w, (int)v.z);
    }
    __device__ __forceinline__ static void load(const double *p, C (&x)[V]) {
        double2 v = __ldg(reinterpret_cast<const double2 *>(p));
        x[0] = v.x;
        x[1] = v.y;
    }
    __device__ __forceinline__ static void store(double *p, const C (&x)[V]) {
        *reinterpret_cast<double2 *>(p) = make_double2(x[0], x[1]);
    }
    __device__ __forceinline__ static uint4 pack(const C (&x)[V]) {
        return make_uint4((uint32_t)__double2loint(x[0]), (uint32_t)__double2hiint(x[0]),
                          (uint32_t)__double2loint(x[1]), (uint32_t)__double2hiint(x[1]));
    }
};

template <> struct Store<float> {
    using C = float;
    using A = float;
    static constexpr int V = 4;
    __device__ __forceinline__ static void unpack(const uint4 &v, C (&x)[V]) {
        x[0] = __uint_as_float(v.x);
        x[1] = __uint_as_float(v.y);
        x[2] = __uint_as_float(v.z);
        x[3] = __uint_as_float(v.w);
    }
    __device__ __forceinline__ static void load(const float *p, C (&x)[V]) {
        float4 v = __ldg(reinterpret_cast<const float4 *>(p));
        x[0] = v.x;
        x[1] = v.y;
        x[2] = v.z;
        x[3] = v.w;
    }
    __device__ __forceinline__ static void store(float *p, const C (&x)[V]) {
        *reinterpret_cast<float4 *>(p) = make_float4(x[0], x[1], x[2], x[3]);
    }
    __device__ __forceinline__ static uint4 pack(const C (&x)[V]) {
        return make_uint4(__float_as_uint(x[0]), __float_as_uint(x[1]), __float_as_uint(x[2]),
                          __float_as_uint(x[3]));
    }
};

template <> struct Store<__nv_bfloat16> {
    using C = float;
    using A = float;
    static constexpr int V = 8;
    // bf16 -> fp32 is exact: the bf16 bits are the high half of the fp32 bits
    __device__ __forceinline__ static void unpack(const uint4 &v, C (&x)[V]) {
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            x[2 * k] = __uint_as_float(w[k] << 16);
            x[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
        }
    }
    __device__ __forceinline__ static void load(const __nv_bfloat16 *p, C (&x)[V]) {
        uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            x[2 * k] = __uint_as_float(w[k] << 16);
            x[2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
        }
    }
    __device__ __forceinline__ static void store(__nv_bfloat16 *p, const C (&x)[V]) {
        *reinterpret_cast<uint4 *>(p) = pack(x);
    }
    __device__ __forceinline__ static uint4 pack(const C (&x)[V]) {
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * k], x[2 * k + 1]);
            w[k] = (uint32_t)__bfloat16_as_ushort(h.x) | ((uint32_t)__bfloat16_as_ushort(h.y) << 16);
        }
        return make_uint4(w[0], w[1], w[2], w[3]);
    }
};

// 16-byte read-only load of a vector chunk
__device__ __forceinline__ uint4 ldg16(const void *p)
{
    return __ldg(reinterpret_cast<const uint4 *>(p));
}

// 32-byte read-only load of two adjacent chunks (sm_100 and later; the address
// is 32-byte aligned)
__device__ __forceinline__ void ldg32(const void *p, uint4 &a, uint4 &b)
{
    asm volatile("ld.global.nc.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
                 : "l"(p));
}

// a lane that owns a whole row (G = 1) of an even number of chunks reads them
// in pairs; the rows must then start on 32-byte boundaries, which the
// handle's buffers do (a row is P chunks, P even).  Launchers refuse other
// pointers instead of faulting.
inline bool rows_aligned32(const void *x, int Kp, size_t elem)
{
    return ((uintptr_t)x & 31) == 0 && (Kp * elem) % 32 == 0;
}

// Kernel shape of one storage type: G lanes per row, NV 16-byte vectors per
// lane (so a row holds P = G * NV vectors, Kp = P * V elements), U nonzeros
// gathered per batch.  P is fixed by (storage, K); G, NV and U are free.
struct Shape {
    int G, NV, U;
    int stage = 0;   // relaxation: 0 direct, 1 TMA-staged CSR, 2 cp.async pipelined,
                     // 3 chunked (one block per SM, L2 prefetch of the CSR ahead of use);
                     // edge pass: 0 row kernel, 1 tile kernel, 2 row kernel on the
                     // sweeps' row order in place
};

// per-device record of a one-time host setting of a kernel (a shared-memory
// opt-in, a resident-grid size): value 0 means "not yet known".  Host threads
// that race on an entry compute and store the same value.
constexpr int kMaxDevices = 64;
struct PerDevice {
    std::atomic<int> v[kMaxDevices] = {};
    int get(int dev) const { return dev >= 0 ? v[dev].load(std::memory_order_relaxed) : 0; }
    void set(int dev, int x) { if (dev >= 0) v[dev].store(x, std::memory_order_relaxed); }
};
// the current device, or -1 if it cannot be used with a PerDevice table
inline int current_device_index()
{
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= kMaxDevices) return -1;
    return d;
}

// device status bits: a bounded wait that gave up; an index that failed its
// bounds test (checked build)
constexpr uint32_t kStatusStagingTimeout = 1u;
constexpr uint32_t kStatusIndexRange = 2u;

// Checked build (compiled with -DAMGD_CHECKS=1 into libamgd_checked.so): the
// row index of every gather the sweep and distance kernels make -- a column
// index of the matrix, a renumbered column or a row map -- is tested against
// the vector block before the load.  An index outside [0, rows) sets
// kStatusIndexRange in the handle's device status word and is replaced by row
// 0, so the load stays in bounds; the results are then invalid and the next
// synchronising call returns AMGD_ERR_CHECK.  The normal build compiles the
// test away.
#ifndef AMGD_CHECKS
#define AMGD_CHECKS 0
#endif
__device__ __forceinline__ int64_t checked_row(int64_t j, int64_t rows, uint32_t *status)
{
#if AMGD_CHECKS
    if (j < 0 || j >= rows) {
        if (status) atomicOr(status, kStatusIndexRange);
        return 0;
    }
#endif
    return j;
}

// ---------------------------------------------------------------------------
// launch arguments
// ---------------------------------------------------------------------------
struct RelaxArgs {
    uint32_t *status = nullptr;     // device status word (bounded-wait time-outs)
    long long wait_limit = 0;       // cycles a staged wait may take
    uint32_t extra_tx = 0;          // test hook: bytes declared but never sent
    const int32_t *rp;    // permuted row_ptr
    const int32_t *col;   // permuted col
    const void *val;      // permuted values (double or float)
    const void *diag;     // permuted diagonal a_ii, same type as val
    const void *xold;     // iterate at the start of the sweep
    void *xnew;           // rows [r0, r1) written; rows < split read from here
    int32_t r0, r1;       // rows of this color phase
    int32_t split;        // rows < split take new values (earlier colors)
    int32_t Kp;           // padded row stride (elements)
    double omega;
    float avg_nnz = 0.f;  // stored entries per row of the whole matrix
    int32_t nrows = 0;    // rows of the vector block (the range of a gather index)
};

struct EdgeArgs {                // everything in the caller's numbering
    const int32_t *rp, *col;     // CSR pattern of A (targets)
    const int32_t *prp, *pcol;   // pattern of the fits: G_d (= rp, col for d = 1); every
                                 // per-slot output and the tiles follow this pattern
    const void *val;             // values, arithmetic type
    const void *diag;            // diagonal a_ii, arithmetic type
    const double *val64;         // values in FP64 (mixed-path fallback)
    const void *x;               // final test vectors, caller row order
    const void *w;               // LS weights, Kp long (zero padded), arithmetic type
    const double *w64;           // LS weights in FP64
    void *a_out, *ls_out;        // per slot, arithmetic type
    uint8_t *flag_out;           // per slot
    int32_t *count_out;          // per row
    uint32_t *defer_count;       // rows appended to defer_list (mixed paths)
    int32_t *defer_list;         // rows to redo in FP64 (capacity n)
    const int32_t *tiles;        // ntiles + 1 first rows of the row tiles
    int32_t ntiles;
    int32_t n, Kp, target;       // target: 0 residual, 1 plain
    double theta;
    // edge stage 2 (search depth 1): x is the vector block in the sweeps' row
    // order; xrow[i] is the vector row of caller row i (NULL: i) and xcol[p]
    // the vector row of the column of caller slot p
    const int32_t *xrow = nullptr, *xcol = nullptr;
    bool compensated = false;    // mixed paths of stage 2: compensated FP32 LS sums
    uint32_t *status = nullptr;  // device status word (checked build: index range)
};

// row tiles of the edge pass: consecutive rows, at most kEdgeTileRows rows and
// kEdgeTileSlots stored entries per tile (a row with more entries is a tile
// of its own)
constexpr int kEdgeTileRows = 256;
constexpr int kEdgeTileSlots = 4096;

struct InitArgs {
    void *x;                   // n x Kp, permuted rows
    const int32_t *perm;       // permuted row -> caller row (NULL = identity)
    const int64_t *mat_off;    // nmat+1 caller-row offsets of the batch
    const int64_t *mat_id;     // Philox key word 1 of each matrix (NULL: its index)
    int32_t nmat, n, K, Kp;
    uint64_t seed;
};

// ---------------------------------------------------------------------------
// launchers (defined in the .cu files; return cudaGetLastError())
// ---------------------------------------------------------------------------
cudaError_t launch_relax(int storage, Shape sh, const RelaxArgs &a, cudaStream_t s);
// false for a staged shape whose shared memory exceeds the per-block limit
bool relax_shape_available(int storage, Shape sh);
cudaError_t launch_edge(int storage, Shape sh, bool unit_w, const EdgeArgs &a, cudaStream_t s);
cudaError_t launch_init(int storage, const InitArgs &a, cudaStream_t s);

// scatter caller-order n x K doubles into permuted, padded storage and back
cudaError_t launch_import(int storage, const double *src, void *x, const int32_t *perm,
                          int32_t n, int32_t K, int32_t Kp, cudaStream_t s);
cudaError_t launch_export(int storage, const void *x, double *dst, const int32_t *perm,
                          int32_t n, int32_t K, int32_t Kp, cudaStream_t s);
// convert vectors between storage types (same permutation and padding)
cudaError_t launch_convert(int from, const void *src, int to, void *dst, int64_t count,
                           cudaStream_t s);
// per-slot outputs (arithmetic type of `storage`) -> doubles; NULL dst skipped
cudaError_t launch_export_slots(int storage, const void *a_in, const void *ls_in,
                                double *a, double *dist, double *ls, int64_t nnz,
                                cudaStream_t s);
// x_caller[perm[r]] = x[r] (rows of Kp storage elements)
cudaError_t launch_unpermute(int storage, const void *x, void *x_caller, const int32_t *perm,
                             int32_t n, int32_t Kp, cudaStream_t s);
// diagonal of every permuted row (double and float copies)
cudaError_t launch_diagonal(const int32_t *rp_perm, const int32_t *col_perm, const double *vp64,
                            double *d64, float *d32, int32_t n, cudaStream_t s);
// permuted values: vp[q] = v[slot of q in caller order] (double and float copies)
cudaError_t launch_permute_values(const double *v, const int32_t *rp_orig,
                                  const int32_t *perm, const int32_t *rp_perm, double *vp64,
                                  float *vp32, int32_t n, cudaStream_t s);

// one coalesced pass over caller-order values src[nnz] into the caller FP64 /
// FP32 copies and the row-permuted FP64 / FP32 copies (NULL targets skipped;
// slot_perm NULL = identity); err (NULL: none) |= 1 for a non-finite value
cudaError_t launch_scatter_values(const double *src, int64_t nnz, const int32_t *slot_perm,
                                  double *val_o, float *val32_o, double *vp64, float *vp32,
                                  cudaStream_t s, uint32_t *err = nullptr);
// diagonals (diag_slot = caller slot of each row's diagonal) in caller order
// and in permuted order (NULL targets skipped); err (NULL: none) |= 2 for a
// zero diagonal
cudaError_t launch_diag_values(const double *v, const int32_t *diag_slot, const int32_t *perm,
                               int32_t n, double *d64_o, float *d32_o, double *d64_p, float *d32_p,
                               cudaStream_t s, uint32_t *err = nullptr);

// value check of a staged val[nnz]: err |= 1 for a non-finite value, |= 2 for
// a zero diagonal (diag_slot[n] = slot of each row's diagonal)
cudaError_t launch_check_values(const double *v, int64_t nnz, const int32_t *diag_slot,
                                int32_t n, uint32_t *err, cudaStream_t s);

// strength CSR: tile sums of counts, scan of the tile sums, compaction
constexpr int kTileRows = 1024;   // rows per compaction tile (multiple of 4)
cudaError_t launch_strength(const int32_t *count, const int32_t *rp_orig, const int32_t *col_orig,
                            const uint8_t *flag, int32_t n, int32_t *tile_sum,
                            int64_t *s_row_ptr, int32_t *s_col, cudaStream_t s);

// ---------------------------------------------------------------------------
// reverse pass (Jacobi sweeps); every array in the caller's numbering, vector
// blocks n x Kp row-major; "C" = FP64 (the reverse pass computes in FP64 for
// every storage of the test vectors)
// ---------------------------------------------------------------------------
struct AdjArgs {
    const int32_t *rp, *col;          // CSR pattern of A
    const void *val, *diag;           // values and diagonal, C
    const int32_t *at_rp;             // transpose: column j owns entries [at_rp[j], at_rp[j+1])
    const int32_t *at_row, *at_slot;  // row i and slot p of each entry (rows ascending)
    const void *at_b;                 // b_q = a(i,j) / a_ii per entry, C
    const void *bm;                   // symmetric pattern: per slot (j, i) a_ij / a_ii, C (else NULL)
    const void *x;                    // storage type: X_nu (edge stages) or X_k (sweeps)
    const void *w;                    // LS weights, Kp, C
    const void *a;                    // fit coefficients per slot (FP64, from k_refit)
    void *a_fit;                      // k_refit's output: a per slot (FP64)
    double *ls64;                     // k_refit's output: LS per slot (FP64)
    const double *lsb;                // dL/dLS per slot (0 where no gradient flows)
    void *y, *ybar;                   // target Y and its adjoint, C
    const void *xbar_in;              // C
    void *xbar_out;                   // C
    void *gs, *gt;                    // per-slot sums <Xbar_{k+1,i}, X_k,j> (sweeps) and
                                      // <Ybar_i, X_nu,j> (target), C
    int32_t n, Kp, target, first;
    double omega;
    bool unit_w = false;              // every LS weight is 1 (the weight products are skipped)
};

// dL/dLS per slot from an upstream gradient (ls_bar) or the built-in loss
// sum r^2 = LS^-2 over kept slots with LS > 0; per-block loss partials
cudaError_t launch_adj_upstream(int storage, const int32_t *rp, const int32_t *col,
                                const void *ls, const uint8_t *flag, const double *ls_bar,
                                double *lsb, double *partial, int32_t nblocks, int32_t n,
                                int32_t target, cudaStream_t s);
// b_q = val[at_slot[q]] / a_ii, i = at_row[q], for every transposed entry (C)
cudaError_t launch_adj_bvals(int storage, const double *val64, const double *diag64,
                             const int32_t *at_row, const int32_t *at_slot, void *at_b,
                             int64_t nnz, cudaStream_t s);
// a and LS of every slot refitted in FP64 from the stored X_nu
cudaError_t launch_adj_refit(int storage, const AdjArgs &a, cudaStream_t s);
// Y, Ybar and (residual target) gt from the fits
cudaError_t launch_adj_edge(int storage, const AdjArgs &a, cudaStream_t s);
// Xbar_nu = direct part of the fits + the target's adjoint, per column
cudaError_t launch_adj_xbar_nu(int storage, const AdjArgs &a, cudaStream_t s);
// gs (+)= <Xbar_{k+1,i}, X_k,col_p>
cudaError_t launch_adj_gram(int storage, const AdjArgs &a, cudaStream_t s);
// Xbar_k = Xbar_{k+1} - omega (D^{-1} A)^T Xbar_{k+1}
cudaError_t launch_adj_spmm_t(int storage, const AdjArgs &a, cudaStream_t s);
// both of the above in one pass over the rows (structurally symmetric patterns)
cudaError_t launch_adj_sweep_sym(int storage, const AdjArgs &a, cudaStream_t s);
// dL/dval (FP64, caller slots) from gs, gt; per-block partials of dL/domega
cudaError_t launch_adj_finish(int storage, const AdjArgs &a, bool have_gs, const double *val64,
                              const double *diag64, const int32_t *diag_slot, double *val_bar,
                              double *partial, int32_t nblocks, cudaStream_t s);
// out[c] = sum of partial[c * nblocks .. (c+1) * nblocks) in a fixed order, c < nsums
cudaError_t launch_adj_reduce(const double *partial, int32_t nblocks, int32_t nsums, double *out,
                              cudaStream_t s);
constexpr int kAdjReduceBlocks = 608;   // 4 per SM

// row_ptr[n+1] (int64) = exclusive scan of count[n] (int32, 16-byte aligned,
// padded to a multiple of 4); tile_sum holds n / kTileRows + 2 entries
cudaError_t launch_row_ptr(const int32_t *count, int32_t n, int32_t *tile_sum, int64_t *row_ptr,
                           cudaStream_t s);

// least-squares interpolation (k_interp.cu)
constexpr int kInterpMaxCaliber = 4;
constexpr int kInterpMaxCand = 32;
struct InterpArgs {
    const int32_t *rp, *col;        // A (targets), caller order
    const double *val64;            // A's values (FP64)
    const int32_t *prp, *pcol;      // neighbourhood pattern (candidates: its coarse entries)
    const uint8_t *coarse;          // n, 1 = coarse
    const void *x;                  // vectors, caller order, storage type, row stride Kp
    const double *w64;              // weights (FP64, Kp)
    int32_t *sel_col;               // n x kInterpMaxCaliber chosen columns
    double *sel_val;                // n x kInterpMaxCaliber weights
    int32_t *cnt;                   // n chosen sizes (coarse rows: 1)
    double *ls;                     // n chosen LS
    uint32_t *err;                  // bit 1: a row had more than kInterpMaxCand candidates
    int32_t *pos;                   // n: position of a fine row inside its bucket
    uint8_t *bkt;                   // n: bucket of a fine row (candidate count, capped)
    int32_t *list;                  // n: fine rows grouped by bucket
    int32_t *bcnt;                  // kInterpBuckets bucket sizes (zeroed by the launcher)
    int32_t n, K, Kp, target, caliber;
    double gamma;
    bool unit_w;                    // all weights are 1 (the products by w are exact)
};
// fine rows with at most kInterpRowCand candidates take the thread-per-row
// kernel; bucket kInterpRowCand + 1 holds the rest (warp-per-row kernel)
constexpr int kInterpRowCand = 8;
constexpr int kInterpBuckets = kInterpRowCand + 2;
cudaError_t launch_ls_interp(int storage, const InterpArgs &a, cudaStream_t s);
// P as CSR from the fixed-stride selections and row_ptr
cudaError_t launch_interp_fill(const int64_t *row_ptr, const int32_t *sel_col,
                               const double *sel_val, int32_t n, int32_t *p_col, double *p_val,
                               cudaStream_t s);

// compatible-relaxation coarsening (k_cr.cu; priorities in k_init.cu)
struct CrArgs {
    const int32_t *rp, *col;        // A with rows in color order (the sweeps' layout)
    const double *val;              // its values (FP64)
    const double *diag;             // its diagonal
    double *cdiag;                  // omega / diagonal (color order), formed once per call
    const int32_t *perm;            // caller row of each color-ordered row (NULL: identity)
    uint8_t *coarse_p;              // coarse mask in color order
    const int32_t *prp, *pcol;      // pattern of the strength graph (G_d), caller order
    const double *ls;               // LS per pattern slot (FP64)
    uint8_t *coarse;                // n, 1 = coarse
    uint8_t *state;                 // n: 0 out, 1 undecided candidate, 2 selected
    uint8_t *ismax;                 // n
    uint8_t *strong;                // pattern slots
    int32_t *lam;                   // n
    const uint64_t *key;            // n
    unsigned long long *scal;       // [0] max |u| bits, [1] |F|, [2] undecided count
    int32_t n;
    double omega, theta;
};
// coarse_p from coarse, u = 1 on F and 0 on C (color order)
cudaError_t launch_cr_start(const CrArgs &a, double *u, cudaStream_t s);
// cdiag = omega / diag, the weight of every sweep of the call
cudaError_t launch_cr_cdiag(const CrArgs &a, cudaStream_t s);
// one F-relaxation sweep u -> un over color-ordered rows: Jacobi (one range
// [0, n)) or multicolor Gauss-Seidel (one launch per color range)
cudaError_t launch_cr_sweep(const CrArgs &a, bool mcgs, const int64_t *color_start,
                            int32_t ncolors, const double *u, double *un, cudaStream_t s);
cudaError_t launch_cr_norm(const double *u, const uint8_t *coarse_p, int32_t n,
                           unsigned long long *scal, cudaStream_t s);
// candidates, strength graph on F and the priorities' lambda
cudaError_t launch_cr_candidates(const CrArgs &a, const double *u, double tol, cudaStream_t s);
// `rounds` rounds of local maxima, then scal[2] = undecided points left
cudaError_t launch_cr_mis_rounds(const CrArgs &a, int32_t rounds, cudaStream_t s);
cudaError_t launch_cr_add(const CrArgs &a, cudaStream_t s);
// key[i] = word 0 of Philox4x64-10, counter (i, stage, 1, 0), key (seed, 0)
cudaError_t launch_cr_keys(int32_t n, int32_t stage, uint64_t seed, uint64_t *key, cudaStream_t s);

// message returned by amgd_last_error(NULL) on the calling host thread
void set_thread_error(const std::string &msg);

}  // namespace amgd
