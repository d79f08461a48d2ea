// k_interp.cu -- least-squares interpolation of a given caliber (§4.3): for
// every fine row i, among all sets W of at most c coarse points of its
// neighbourhood, the set whose one-row least-squares fit of the target
//   LS_W(p) = sum_k w_k (y_ik - sum_{j in W} p_j x_jk)^2
// is smallest, with the size penalty of §4.3 (a larger set replaces a smaller
// one only if its LS, normalised by S_yy = sum_k w_k y_ik^2, is below the
// smaller set's normalised LS raised to gamma times the size difference).
//
// All arithmetic is FP64 (the vectors are widened exactly), in the operation
// order of the definition:
//   * target y_i from row i of A, the same fused multiply-adds as the sweeps;
//   * Gram entries G_ab = sum_k (w_k x_ak) x_bk and b_a = sum_k (w_k y_k) x_ak,
//     one product and one addition per term in component order (explicit
//     roundings, no fused operations);
//   * every subset of each size, in lexicographic order, solved by Gaussian
//     elimination with partial pivoting and scored by its residual sum of
//     squares; the first set in lexicographic order with the smallest LS is
//     kept for each size.
// Every rounding follows that order, so the selected sets and weights are
// reproducible bit for bit, whichever kernel evaluates a row.
//
// FP64 issue rate is the bound (a GB300 SM retires two FP64 operations per
// clock), so lanes must not idle: fine rows are first grouped by their
// candidate count m; rows with m <= kInterpRowCand are evaluated one thread
// per row (its arrays in shared memory, interleaved across the block's
// threads), the rest one warp per row (lanes over Gram entries and subsets).
#include <math.h>

#include <atomic>
#include <type_traits>

#include "amgd_internal.cuh"

namespace amgd {
namespace {

constexpr int kWarps = 4;                    // warps per block
constexpr int kMaxK = 64;                    // components per vector
// shared memory of one warp, in doubles (the candidate list takes 16 doubles)

// exact widening to double.  Normal BF16/FP32 numbers are re-biased by bit
// manipulation on the integer pipe (exponent + 1023 - 127, mantissa shifted
// to the top of the 52-bit field); zeros, subnormals, infinities and NaNs
// take the conversion instruction.
__device__ __forceinline__ double widen_f32_bits(uint32_t u)
{
    const uint32_t e = (u >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)__uint_as_float(u);
    const uint64_t bits = ((uint64_t)(u >> 31) << 63) | ((uint64_t)(e + 896u) << 52) |
                          ((uint64_t)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)bits);
}

// the product of two BF16 numbers as a double: their 8-bit significands
// multiply exactly in FP32 whenever the result is a normal FP32 number, and
// that number widens exactly; otherwise the FP64 product (also exact)
__device__ __forceinline__ double bf16_product(uint16_t a, uint16_t b)
{
    const float p = __fmul_rn(__uint_as_float((uint32_t)a << 16), __uint_as_float((uint32_t)b << 16));
    const uint32_t u = __float_as_uint(p);
    const uint32_t e = (u >> 23) & 0xffu;
    if (e != 0u && e != 0xffu) return widen_f32_bits(u);
    return __dmul_rn(widen_f32_bits((uint32_t)a << 16), widen_f32_bits((uint32_t)b << 16));
}

template <class TS> __device__ __forceinline__ double widen(const TS *p, int k);
template <> __device__ __forceinline__ double widen<double>(const double *p, int k) { return p[k]; }
template <> __device__ __forceinline__ double widen<float>(const float *p, int k)
{
    return widen_f32_bits(__float_as_uint(p[k]));
}
template <> __device__ __forceinline__ double widen<__nv_bfloat16>(const __nv_bfloat16 *p, int k)
{
    return widen_f32_bits((uint32_t)__bfloat16_as_ushort(p[k]) << 16);
}

// The size penalty's decision r < pow(c, e) (r, c normalised LS values, e =
// gamma times the size difference), with CUDA's FP64 pow.  Most decisions are
// far from the boundary: log2 of both sides in FP32 decides them when they
// differ by more than a margin that covers the FP32 errors many times over;
// the rest call pow.  The decision is therefore always the one pow gives.
__device__ __forceinline__ bool penalty_less(double r, double c, double e)
{
    const float rf = (float)r, cf = (float)c;
    if (e > 0.0 && rf >= 1.17549435e-38f && cf >= 1.17549435e-38f && rf <= 3.0e38f && cf <= 3.0e38f) {
        const float lr = log2f(rf), lp = (float)e * log2f(cf);
        const float margin = 1e-3f * (1.0f + fabsf(lr) + fabsf(lp));
        if (lr < lp - margin) return true;
        if (lr > lp + margin) return false;
    }
    return r < pow(c, e);
}

// C(nn, kk) for nn <= 32, kk <= 4
__device__ __forceinline__ int64_t binom(int nn, int kk)
{
    if (kk < 0 || kk > nn) return 0;
    int64_t r = 1;
    for (int q = 1; q <= kk; ++q) r = r * (nn - kk + q) / q;
    return r;
}

// subset of size s with lexicographic rank t among the subsets of {0..m-1}
__device__ __forceinline__ void unrank(int m, int s, int64_t t, int *idx)
{
    int v = 0;
    for (int a = 0; a < s; ++a) {
        for (;; ++v) {
            const int64_t cnt = binom(m - v - 1, s - a - 1);
            if (t < cnt) break;
            t -= cnt;
        }
        idx[a] = v++;
    }
}

// Gs p = bs (s x s, row-major, copies of the subset's entries) by Gaussian
// elimination with partial pivoting; -1 when a pivot is below 1e-13 of the
// largest diagonal entry (singular set)
__device__ __forceinline__ int solve_small(int s, double *Gs, double *bs, double *p)
{
    double dmax = 0.0;
    for (int a = 0; a < s; ++a) dmax = fmax(dmax, fabs(Gs[a * s + a]));
    for (int k = 0; k < s; ++k) {
        int piv = k;
        for (int a = k + 1; a < s; ++a)
            if (fabs(Gs[a * s + k]) > fabs(Gs[piv * s + k])) piv = a;
        if (!(fabs(Gs[piv * s + k]) > __dmul_rn(1e-13, dmax))) return -1;
        if (piv != k) {
            for (int c = 0; c < s; ++c) {
                const double t = Gs[k * s + c];
                Gs[k * s + c] = Gs[piv * s + c];
                Gs[piv * s + c] = t;
            }
            const double t = bs[k];
            bs[k] = bs[piv];
            bs[piv] = t;
        }
        for (int a = k + 1; a < s; ++a) {
            const double f = __ddiv_rn(Gs[a * s + k], Gs[k * s + k]);
            for (int c = k; c < s; ++c) Gs[a * s + c] = __dsub_rn(Gs[a * s + c], __dmul_rn(f, Gs[k * s + c]));
            bs[a] = __dsub_rn(bs[a], __dmul_rn(f, bs[k]));
        }
    }
    for (int k = s - 1; k >= 0; --k) {
        double t = bs[k];
        for (int c = k + 1; c < s; ++c) t = __dsub_rn(t, __dmul_rn(Gs[k * s + c], p[c]));
        p[k] = __ddiv_rn(t, Gs[k * s + k]);
    }
    return 0;
}


// shared memory of one warp of k_ls_interp for K components: the Gram matrix
// (kInterpMaxCand^2), b and sqrt(G_aa) (kInterpMaxCand each), y and w (K
// each), in doubles; then the candidate rows in the storage type; then the
// candidate columns
template <class TS>
__host__ __device__ constexpr int warp_interp_bytes(int K)
{
    return (kInterpMaxCand * kInterpMaxCand + 2 * kInterpMaxCand + 2 * K) * 8 +
           ((kInterpMaxCand * K * (int)sizeof(TS) + 15) & ~15) + kInterpMaxCand * 4;
}

template <class TS> __device__ __forceinline__ double widen_val(TS v);
template <> __device__ __forceinline__ double widen_val<double>(double v) { return v; }
template <> __device__ __forceinline__ double widen_val<float>(float v)
{
    return widen_f32_bits(__float_as_uint(v));
}
template <> __device__ __forceinline__ double widen_val<__nv_bfloat16>(__nv_bfloat16 v)
{
    return widen_f32_bits((uint32_t)__bfloat16_as_ushort(v) << 16);
}

// (w_k x_ak) x_ck with the definition's rounding; with unit weights and BF16
// storage the product is formed exactly in FP32 (bf16_product)
template <class TS, bool UNIT_W>
__device__ __forceinline__ double gram_term(TS xa, TS xc, double wk)
{
    if constexpr (UNIT_W && std::is_same<TS, __nv_bfloat16>::value) {
        return bf16_product(__bfloat16_as_ushort(xa), __bfloat16_as_ushort(xc));
    } else {
        const double a = widen_val<TS>(xa);
        return __dmul_rn(UNIT_W ? a : __dmul_rn(wk, a), widen_val<TS>(xc));
    }
}

// One warp per fine row with more than kInterpRowCand candidates: lanes over
// Gram entries (one triangle under unit weights, where G_ac = G_ca bit for
// bit) and over subsets; each lane prunes its subsets against its own best
// explicit LS with the rounding-error bound of the thread kernel.
template <class TS, bool UNIT_W>
__global__ void __launch_bounds__(kWarps * 32) k_ls_interp(InterpArgs A)
{
    extern __shared__ __align__(16) unsigned char ism[];
    const int wib = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int K = A.K, Kp = A.Kp, C = A.caliber;
    unsigned char *base = ism + (size_t)wib * warp_interp_bytes<TS>(K);
    double *G = reinterpret_cast<double *>(base);                   // Gram matrix, stride m
    double *b = G + kInterpMaxCand * kInterpMaxCand;                // right-hand side
    double *sg = b + kInterpMaxCand;                                // sqrt(G_aa)
    double *y = sg + kInterpMaxCand;                                // target
    double *w = y + K;                                              // weights
    TS *xs = reinterpret_cast<TS *>(w + K);                         // candidate rows, stride K
    int32_t *cand = reinterpret_cast<int32_t *>(reinterpret_cast<unsigned char *>(xs) +
                                                ((kInterpMaxCand * K * (int)sizeof(TS) + 15) & ~15));
    const TS *X = (const TS *)A.x;
    for (int k = lane; k < K; k += 32) w[k] = A.w64[k];
    __syncwarp();

    // the rows of the last bucket (more than kInterpRowCand candidates)
    int32_t lo = 0;
    for (int q = 0; q <= kInterpRowCand; ++q) lo += A.bcnt[q];
    const int32_t hi = lo + A.bcnt[kInterpRowCand + 1];
    const int64_t warps = (int64_t)gridDim.x * kWarps;
    for (int64_t e = lo + (int64_t)blockIdx.x * kWarps + wib; e < hi; e += warps) {
        const int64_t i = A.list[e];
        // target y_i (the sweeps' rounding: one FMA per entry, x - (1/a_ii) s)
        const int p0 = A.rp[i], p1 = A.rp[i + 1];
        for (int k = lane; k < K; k += 32) {
            double s = 0.0, d = 1.0;
            for (int p = p0; p < p1; ++p) {
                const int j = A.col[p];
                if (j == i) d = A.val64[p];
                s = fma(A.val64[p], widen<TS>(X + (int64_t)j * Kp, k), s);
            }
            const double xi = widen<TS>(X + i * Kp, k);
            y[k] = A.target == 0 ? fma(-(1.0 / d), s, xi) : xi;
        }
        // candidates: the coarse entries of the neighbourhood, ascending
        const int q0 = A.prp[i], q1 = A.prp[i + 1];
        int m = 0;
        for (int qb = q0; qb < q1; qb += 32) {
            const int q = qb + lane;
            const int j = q < q1 ? A.pcol[q] : -1;
            const bool c = j >= 0 && A.coarse[j];
            const unsigned ball = __ballot_sync(0xffffffffu, c);
            const int pos = m + __popc(ball & ((1u << lane) - 1u));
            if (c && pos < kInterpMaxCand) cand[pos] = j;
            m += __popc(ball);
        }
        if (m > kInterpMaxCand) {
            if (lane == 0) {
                atomicOr(A.err, 1u);
                A.cnt[i] = 0;
                A.ls[i] = NAN;
            }
            continue;
        }
        __syncwarp();
        for (int t = lane; t < m * K; t += 32) {
            const int a = t / K, k = t % K;
            xs[a * K + k] = X[(int64_t)cand[a] * Kp + k];
        }
        __syncwarp();
        // Gram matrix (G_ac = sum_k (w_k x_ak) x_ck in component order) and b
        const int ntri = UNIT_W ? m * (m + 1) / 2 : m * m;
        for (int t = lane; t < ntri; t += 32) {
            int a, c;
            if (UNIT_W) {
                a = 0;
                int rowbase = 0;
                while (t >= rowbase + (m - a)) { rowbase += m - a; ++a; }
                c = a + (t - rowbase);
            } else {
                a = t / m;
                c = t % m;
            }
            double g = 0.0;
            for (int k = 0; k < K; ++k) g = __dadd_rn(g, gram_term<TS, UNIT_W>(xs[a * K + k], xs[c * K + k], w[k]));
            G[a * m + c] = g;
            if (UNIT_W) G[c * m + a] = g;
        }
        for (int a = lane; a < m; a += 32) {
            double g = 0.0;
            for (int k = 0; k < K; ++k) {
                const double wy = UNIT_W ? y[k] : __dmul_rn(w[k], y[k]);
                g = __dadd_rn(g, __dmul_rn(wy, widen_val<TS>(xs[a * K + k])));
            }
            b[a] = g;
        }
        double syy = 0.0;
        for (int k = 0; k < K; ++k) {
            const double wy = UNIT_W ? y[k] : __dmul_rn(w[k], y[k]);
            syy = __dadd_rn(syy, __dmul_rn(wy, y[k]));
        }
        __syncwarp();
        for (int a = lane; a < m; a += 32) sg[a] = sqrt(G[a * m + a]);
        const double sy = sqrt(syy);
        __syncwarp();

        // best set of every size: lane-local best (pruned against itself), then
        // a warp reduction (smallest LS, then smallest rank)
        double best_ls[kInterpMaxCaliber + 1];
        int best_idx[kInterpMaxCaliber + 1][kInterpMaxCaliber];
        double best_p[kInterpMaxCaliber + 1][kInterpMaxCaliber];
        bool have[kInterpMaxCaliber + 1];
        have[0] = true;
        best_ls[0] = syy;
        for (int s = 1; s <= kInterpMaxCaliber; ++s) {
            have[s] = false;
            if (s > C || s > m) continue;
            const int64_t total = binom(m, s);
            double mine = INFINITY;
            int64_t mine_rank = INT64_MAX;
            for (int64_t t = lane; t < total; t += 32) {
                int idx[kInterpMaxCaliber];
                double Gs[kInterpMaxCaliber * kInterpMaxCaliber], bs[kInterpMaxCaliber];
                double p[kInterpMaxCaliber];
                unrank(m, s, t, idx);
                for (int a = 0; a < s; ++a) {
                    bs[a] = b[idx[a]];
                    for (int c = 0; c < s; ++c) Gs[a * s + c] = G[idx[a] * m + idx[c]];
                }
                if (solve_small(s, Gs, bs, p) != 0) continue;
                if (mine_rank != INT64_MAX) {
                    // the bound of the thread kernel (see k_ls_interp_rows)
                    double q = syy, mm = sy;
                    for (int a = 0; a < s; ++a) {
                        q = __dsub_rn(q, __dmul_rn(__dmul_rn(2.0, p[a]), b[idx[a]]));
                        mm = __dadd_rn(mm, __dmul_rn(fabs(p[a]), sg[idx[a]]));
                    }
                    for (int a = 0; a < s; ++a)
                        for (int c = 0; c < s; ++c)
                            q = __dadd_rn(q, __dmul_rn(__dmul_rn(p[a], G[idx[a] * m + idx[c]]), p[c]));
                    const double bound = (double)(4 * (s * s + 6 * s + 2 * K + 8)) * 0x1p-53 * mm * mm;
                    if (__dsub_rn(q, bound) >= mine) continue;
                }
                double r = 0.0;
                for (int k = 0; k < K; ++k) {
                    double ek = y[k];
                    for (int a = 0; a < s; ++a) ek = __dsub_rn(ek, __dmul_rn(p[a], widen_val<TS>(xs[idx[a] * K + k])));
                    const double we = UNIT_W ? ek : __dmul_rn(w[k], ek);
                    r = __dadd_rn(r, __dmul_rn(we, ek));
                }
                if (r < mine) {
                    mine = r;
                    mine_rank = t;
                }
            }
            double bl = mine;
            int64_t br = mine_rank;
            for (int o = 16; o > 0; o >>= 1) {
                const double ol = __shfl_xor_sync(0xffffffffu, bl, o);
                const int64_t orr = __shfl_xor_sync(0xffffffffu, br, o);
                if (ol < bl || (ol == bl && orr < br)) { bl = ol; br = orr; }
            }
            if (br != INT64_MAX) {
                have[s] = true;
                best_ls[s] = bl;
                unrank(m, s, br, best_idx[s]);
                // the winning set's weights, solved again (the same elimination)
                double Gs[kInterpMaxCaliber * kInterpMaxCaliber], bs[kInterpMaxCaliber];
                for (int a = 0; a < s; ++a) {
                    bs[a] = b[best_idx[s][a]];
                    for (int c = 0; c < s; ++c) Gs[a * s + c] = G[best_idx[s][a] * m + best_idx[s][c]];
                }
                solve_small(s, Gs, bs, best_p[s]);
            }
        }
        if (lane == 0) {
            int chosen = 0;
            if (syy > 0.0) {
                for (int s = 1; s <= kInterpMaxCaliber; ++s) {
                    if (!have[s]) continue;
                    const double cur = best_ls[chosen] / syy;
                    if (penalty_less(best_ls[s] / syy, cur, A.gamma * (double)(s - chosen))) chosen = s;
                }
            }
            A.cnt[i] = chosen;
            A.ls[i] = best_ls[chosen];
            for (int a = 0; a < chosen; ++a) {
                A.sel_col[i * kInterpMaxCaliber + a] = cand[best_idx[chosen][a]];
                A.sel_val[i * kInterpMaxCaliber + a] = best_p[chosen][a];
            }
        }
        __syncwarp();
    }
}

// coarse rows interpolate themselves; fine rows get their candidate count
// (bucket min(m, kInterpRowCand + 1)) and a position inside the bucket
__global__ void k_interp_classify(InterpArgs A)
{
    // one row per thread; bucket positions come from block-local counters,
    // one global atomic per bucket and block
    __shared__ int32_t cnt_s[kInterpBuckets], base_s[kInterpBuckets];
    if (threadIdx.x < kInterpBuckets) cnt_s[threadIdx.x] = 0;
    __syncthreads();
    const int32_t i = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    int b = -1, local = 0;
    if (i < A.n) {
        if (A.coarse[i]) {
            A.cnt[i] = 1;
            A.sel_col[(int64_t)i * kInterpMaxCaliber] = i;
            A.sel_val[(int64_t)i * kInterpMaxCaliber] = 1.0;
            A.ls[i] = 0.0;
        } else {
            int m = 0;
            const int q1 = A.prp[i + 1];
            for (int q = A.prp[i]; q < q1; ++q) m += A.coarse[A.pcol[q]] != 0;
            if (m > kInterpMaxCand) {
                atomicOr(A.err, 1u);
                A.cnt[i] = 0;
                A.ls[i] = __longlong_as_double(0x7ff8000000000000ll);   // NaN
                A.bkt[i] = 0xff;
            } else {
                b = m <= kInterpRowCand ? m : kInterpRowCand + 1;
                A.bkt[i] = (uint8_t)b;
                local = atomicAdd(&cnt_s[b], 1);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < kInterpBuckets && cnt_s[threadIdx.x] > 0)
        base_s[threadIdx.x] = atomicAdd(&A.bcnt[threadIdx.x], cnt_s[threadIdx.x]);
    __syncthreads();
    if (b >= 0) A.pos[i] = base_s[b] + local;
}

// list = buckets kInterpRowCand, ..., 1, 0 (largest candidate count first, so
// that a warp's rows carry equal work), then bucket kInterpRowCand + 1
__global__ void k_interp_list(InterpArgs A)
{
    int32_t off[kInterpBuckets];
    int32_t acc = 0;
    for (int b = kInterpRowCand; b >= 0; --b) {
        off[b] = acc;
        acc += A.bcnt[b];
    }
    off[kInterpRowCand + 1] = acc;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < A.n; i += gridDim.x * blockDim.x) {
        if (A.coarse[i]) continue;
        const uint8_t b = A.bkt[i];
        if (b == 0xff) continue;
        A.list[off[b] + A.pos[i]] = i;
    }
}

// one thread per fine row with m <= kInterpRowCand candidates.  Per-thread
// arrays live in shared memory, element e of thread t at [e * T + t] (T the
// block size), so that a warp's accesses fall in distinct banks.
template <class TS, bool UNIT_W>
__global__ void __launch_bounds__(128) k_ls_interp_rows(InterpArgs A)
{
    extern __shared__ __align__(16) double rsm[];
    const int T = blockDim.x, t = threadIdx.x;
    const int K = A.K, Kp = A.Kp, C = A.caliber;
    constexpr int MT = kInterpRowCand;
    double *yv = rsm + t;                        // y_k        at yv[k * T]
    double *Gm = yv + (size_t)K * T;              // G_ab       at Gm[(a * MT + b) * T]
    double *bv = Gm + (size_t)MT * MT * T;        // b_a        at bv[a * T]
    double *sg = bv + (size_t)MT * T;             // sqrt(G_aa) at sg[a * T]
    int32_t *cd = reinterpret_cast<int32_t *>(rsm + (size_t)(K + MT * MT + 2 * MT) * T) + t;
    const TS *X = (const TS *)A.x;
    int32_t nrows = 0;
    for (int q = 0; q <= MT; ++q) nrows += A.bcnt[q];
    for (int32_t e = blockIdx.x * T + t; e < nrows; e += gridDim.x * T) {
        const int32_t i = A.list[e];
        // target: y_k = x_ik - (1/a_ii) sum_p a_ip x_{col_p,k}, one FMA per
        // entry in CSR order (row sums accumulated in place, entry by entry)
        const int p0 = A.rp[i], p1 = A.rp[i + 1];
        for (int k = 0; k < K; ++k) yv[k * T] = 0.0;
        double d = 1.0;
        for (int p = p0; p < p1; ++p) {
            const int j = A.col[p];
            const double v = A.val64[p];
            if (j == i) d = v;
            const TS *xr = X + (int64_t)j * Kp;
            for (int k = 0; k < K; ++k) yv[k * T] = fma(v, widen<TS>(xr, k), yv[k * T]);
        }
        {
            const TS *xi = X + (int64_t)i * Kp;
            const double c = -(1.0 / d);
            for (int k = 0; k < K; ++k) {
                const double xik = widen<TS>(xi, k);
                yv[k * T] = A.target == 0 ? fma(c, yv[k * T], xik) : xik;
            }
        }
        // candidates, ascending
        int m = 0;
        {
            const int q1 = A.prp[i + 1];
            for (int q = A.prp[i]; q < q1; ++q) {
                const int j = A.pcol[q];
                if (A.coarse[j]) cd[(m++) * T] = j;
            }
        }
        // Gram matrix row by row (row a kept in registers), right-hand side, S_yy.
        // With unit weights G_ab = sum_k x_ak x_bk = G_ba bit for bit (the same
        // products, summed in the same order), so only c >= a is computed.
        for (int a = 0; a < m; ++a) {
            double g[MT];
#pragma unroll
            for (int c = 0; c < MT; ++c) g[c] = 0.0;
            double ba = 0.0;
            const TS *xa = X + (int64_t)cd[a * T] * Kp;
            for (int k = 0; k < K; ++k) {
                const double xak = widen<TS>(xa, k);
                const double wk = UNIT_W ? 1.0 : A.w64[k];
                const double wxa = UNIT_W ? xak : __dmul_rn(wk, xak);
                const double yk = yv[k * T];
                const double wy = UNIT_W ? yk : __dmul_rn(wk, yk);
                ba = __dadd_rn(ba, __dmul_rn(wy, xak));
                if constexpr (UNIT_W && std::is_same<TS, __nv_bfloat16>::value) {
                    // x_ak x_ck of two BF16 numbers: exact FP32 product (bit-equal
                    // to the FP64 product), one FP64 addition per term
                    const uint16_t ab = __bfloat16_as_ushort(xa[k]);
#pragma unroll
                    for (int c = 0; c < MT; ++c)
                        if (c < m && c >= a)
                            g[c] = __dadd_rn(g[c], bf16_product(ab, __bfloat16_as_ushort(
                                                                        X[(int64_t)cd[c * T] * Kp + k])));
                } else {
#pragma unroll
                    for (int c = 0; c < MT; ++c)
                        if (c < m && (!UNIT_W || c >= a))
                            g[c] = __dadd_rn(g[c], __dmul_rn(wxa, widen<TS>(X + (int64_t)cd[c * T] * Kp, k)));
                }
            }
#pragma unroll
            for (int c = 0; c < MT; ++c) {
                if (c >= m) continue;
                if (!UNIT_W) {
                    Gm[(a * MT + c) * T] = g[c];
                } else if (c >= a) {
                    Gm[(a * MT + c) * T] = g[c];
                    Gm[(c * MT + a) * T] = g[c];
                }
            }
            bv[a * T] = ba;
            sg[a * T] = sqrt(Gm[(a * MT + a) * T]);
        }
        double syy = 0.0;
        for (int k = 0; k < K; ++k) {
            const double yk = yv[k * T];
            const double wy = UNIT_W ? yk : __dmul_rn(A.w64[k], yk);
            syy = __dadd_rn(syy, __dmul_rn(wy, yk));
        }
        const double sy = sqrt(syy);
        // every subset of each size in lexicographic order; first smallest LS
        double best_ls[kInterpMaxCaliber + 1];
        int best_idx[kInterpMaxCaliber + 1][kInterpMaxCaliber];
        double best_p[kInterpMaxCaliber + 1][kInterpMaxCaliber];
        bool have[kInterpMaxCaliber + 1];
        have[0] = true;
        best_ls[0] = syy;
#pragma unroll
        for (int s = 1; s <= kInterpMaxCaliber; ++s) {
            have[s] = false;
            if (s > C || s > m) continue;
            int idx[kInterpMaxCaliber];
            for (int a = 0; a < s; ++a) idx[a] = a;
            for (;;) {
                double Gs[kInterpMaxCaliber * kInterpMaxCaliber], bs[kInterpMaxCaliber];
                double p[kInterpMaxCaliber];
                for (int a = 0; a < s; ++a) {
                    bs[a] = bv[idx[a] * T];
                    for (int c = 0; c < s; ++c) Gs[a * s + c] = Gm[(idx[a] * MT + idx[c]) * T];
                }
                bool exact = false;
                if (solve_small(s, Gs, bs, p) == 0) {
                    exact = !have[s];
                    if (!exact) {
                        // Pruning.  With S, b, G the stored sums, the value
                        //   q = S - 2 p.b + p.G.p
                        // and the explicit residual sum both approximate
                        // sum_k w_k (y_k - p.x_k)^2; their rounding errors are
                        // at most (s^2 + 5s + 2K + 6) u M^2 together, with
                        // M = ||y||_w + sum_a |p_a| ||x_a||_w (Cauchy-Schwarz,
                        // Minkowski).  If q minus four times that bound is not
                        // below the best explicit value of this size, the
                        // subset can neither beat nor tie it (a tie goes to
                        // the earlier subset), and its explicit sum is skipped.
                        double q = syy, mm = sy;
                        for (int a = 0; a < s; ++a) {
                            q = __dsub_rn(q, __dmul_rn(__dmul_rn(2.0, p[a]), bv[idx[a] * T]));
                            mm = __dadd_rn(mm, __dmul_rn(fabs(p[a]), sg[idx[a] * T]));
                        }
                        for (int a = 0; a < s; ++a)
                            for (int c = 0; c < s; ++c)
                                q = __dadd_rn(q, __dmul_rn(__dmul_rn(p[a], Gm[(idx[a] * MT + idx[c]) * T]), p[c]));
                        const double bound = (double)(4 * (s * s + 6 * s + 2 * K + 8)) * 0x1p-53 * mm * mm;
                        exact = !(__dsub_rn(q, bound) >= best_ls[s]);
                    }
                }
                if (exact) {
                    double r = 0.0;
                    for (int k = 0; k < K; ++k) {
                        double ek = yv[k * T];
                        for (int a = 0; a < s; ++a)
                            ek = __dsub_rn(ek, __dmul_rn(p[a], widen<TS>(X + (int64_t)cd[idx[a] * T] * Kp, k)));
                        const double we = UNIT_W ? ek : __dmul_rn(A.w64[k], ek);
                        r = __dadd_rn(r, __dmul_rn(we, ek));
                    }
                    if (!have[s] || r < best_ls[s]) {
                        have[s] = true;
                        best_ls[s] = r;
                        for (int a = 0; a < s; ++a) {
                            best_idx[s][a] = idx[a];
                            best_p[s][a] = p[a];
                        }
                    }
                }
                // next subset in lexicographic order
                int a = s - 1;
                while (a >= 0 && idx[a] == m - s + a) --a;
                if (a < 0) break;
                ++idx[a];
                for (int c = a + 1; c < s; ++c) idx[c] = idx[c - 1] + 1;
            }
        }
        int chosen = 0;
        if (syy > 0.0) {
#pragma unroll
            for (int s = 1; s <= kInterpMaxCaliber; ++s) {
                if (!have[s]) continue;
                const double cur = best_ls[chosen] / syy;
                if (penalty_less(best_ls[s] / syy, cur, A.gamma * (double)(s - chosen))) chosen = s;
            }
        }
        A.cnt[i] = chosen;
        A.ls[i] = best_ls[chosen];
#pragma unroll
        for (int s = 1; s <= kInterpMaxCaliber; ++s) {
            if (s != chosen) continue;
            for (int a = 0; a < s; ++a) {
                A.sel_col[(int64_t)i * kInterpMaxCaliber + a] = cd[best_idx[s][a] * T];
                A.sel_val[(int64_t)i * kInterpMaxCaliber + a] = best_p[s][a];
            }
        }
    }
}

__global__ void k_interp_fill(const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ sel_col,
                              const double *__restrict__ sel_val, int32_t n,
                              int32_t *__restrict__ p_col, double *__restrict__ p_val)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t o = row_ptr[i], len = row_ptr[i + 1] - o;
    for (int a = 0; a < len; ++a) {
        p_col[o + a] = sel_col[i * kInterpMaxCaliber + a];
        p_val[o + a] = sel_val[i * kInterpMaxCaliber + a];
    }
}

// A dynamic shared-memory opt-in is an attribute of a kernel in one
// device's context, so it is made once per device (a second GPU driven by the
// same process gets its own).  Two host threads making the first call at once
// both set the same value, which is harmless.
constexpr int kOptDevices = 64;

template <class F>
cudaError_t opt_in_smem(F *kernel, std::atomic<bool> (&done)[kOptDevices], int bytes)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const bool tracked = dev >= 0 && dev < kOptDevices;
    if (tracked && done[dev].load(std::memory_order_acquire)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess && tracked) done[dev].store(true, std::memory_order_release);
    return e;
}

template <class TS, bool UNIT_W>
cudaError_t launch_rows_kernel(const InterpArgs &a, cudaStream_t s)
{
    constexpr int T = 128;
    constexpr int MT = kInterpRowCand;
    const size_t smem = (size_t)T * (8 * (a.K + MT * MT + 2 * MT) + 4 * MT);
    constexpr size_t smem_max = (size_t)T * (8 * (kMaxK + MT * MT + 2 * MT) + 4 * MT);
    static std::atomic<bool> opted[kOptDevices] = {};
    const cudaError_t e = opt_in_smem(k_ls_interp_rows<TS, UNIT_W>, opted, (int)smem_max);
    if (e != cudaSuccess) return e;
    const int64_t want = ((int64_t)a.n + T - 1) / T;
    const unsigned grid = (unsigned)(want < 152 * 4 ? want : 152 * 4);
    k_ls_interp_rows<TS, UNIT_W><<<grid, T, smem, s>>>(a);
    return cudaGetLastError();
}

template <class TS, bool UNIT_W>
cudaError_t launch_warp_kernel(const InterpArgs &a, cudaStream_t s)
{
    static std::atomic<bool> opted[kOptDevices] = {};
    const cudaError_t e = opt_in_smem(k_ls_interp<TS, UNIT_W>, opted,
                                      kWarps * warp_interp_bytes<TS>(kMaxK));
    if (e != cudaSuccess) return e;
    const int64_t want = ((int64_t)a.n + kWarps - 1) / kWarps;
    const unsigned grid = (unsigned)(want < 152 * 8 ? want : 152 * 8);
    k_ls_interp<TS, UNIT_W><<<grid, kWarps * 32, kWarps * warp_interp_bytes<TS>(a.K), s>>>(a);
    return cudaGetLastError();
}

template <class TS>
cudaError_t launch_interp_typed(const InterpArgs &a, cudaStream_t s)
{
    cudaError_t e = a.unit_w ? launch_rows_kernel<TS, true>(a, s) : launch_rows_kernel<TS, false>(a, s);
    if (e != cudaSuccess) return e;
    return a.unit_w ? launch_warp_kernel<TS, true>(a, s) : launch_warp_kernel<TS, false>(a, s);
}

}  // namespace

cudaError_t launch_ls_interp(int storage, const InterpArgs &a, cudaStream_t s)
{
    if (a.n == 0) return cudaSuccess;
    if (a.K > kMaxK || a.caliber < 1 || a.caliber > kInterpMaxCaliber) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(a.bcnt, 0, kInterpBuckets * sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    const int64_t nb = ((int64_t)a.n + 255) / 256;
    const unsigned g = (unsigned)(nb < 152 * 16 ? nb : 152 * 16);
    k_interp_classify<<<(unsigned)nb, 256, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_interp_list<<<g, 256, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    switch (storage) {
    case ST_FP64: return launch_interp_typed<double>(a, s);
    case ST_FP32: return launch_interp_typed<float>(a, s);
    case ST_BF16: return launch_interp_typed<__nv_bfloat16>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_interp_fill(const int64_t *row_ptr, const int32_t *sel_col,
                               const double *sel_val, int32_t n, int32_t *p_col, double *p_val,
                               cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_interp_fill<<<(unsigned)(((int64_t)n + 255) / 256), 256, 0, s>>>(row_ptr, sel_col, sel_val, n,
                                                                        p_col, p_val);
    return cudaGetLastError();
}

}  // namespace amgd
