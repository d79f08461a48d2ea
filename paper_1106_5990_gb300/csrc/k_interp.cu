// k_interp.cu -- least-squares interpolation of a given caliber (§4.3): for
// every fine row i, among all sets W of at most c coarse points of its
// neighbourhood, the set whose one-row least-squares fit of the target
//   LS_W(p) = sum_k w_k (y_ik - sum_{j in W} p_j x_jk)^2
// is smallest, with the size penalty of §4.3 (a larger set replaces a smaller
// one only if its LS, normalised by S_yy = sum_k w_k y_ik^2, is below the
// smaller set's normalised LS raised to gamma times the size difference).
//
// One warp per fine row, all in FP64 (the vectors are widened exactly):
//   * target y_i from row i of A, the same fused multiply-adds as the sweeps;
//   * candidate vectors x_j (the coarse entries of the neighbourhood, at most
//     32) into shared memory; Gram entries G_ab = sum_k (w_k x_ak) x_bk and
//     b_a = sum_k (w_k y_k) x_ak, one product and one addition per term in
//     component order (explicit roundings, no fused operations);
//   * every subset of each size (combinatorial unranking, lexicographic
//     order) is solved by Gaussian elimination with partial pivoting and
//     scored by its residual sum of squares, with the same operation order;
//     a warp reduction keeps the smallest LS per size, the first set in
//     lexicographic order on ties.
// Every rounding follows the documented order of the definition, so the
// selected sets and weights are reproducible bit for bit.
#include <math.h>

#include "amgd_internal.cuh"

namespace amgd {
namespace {

constexpr int kWarps = 4;                    // warps per block
constexpr int kMaxK = 64;                    // components per vector
// shared memory of one warp, in doubles (the candidate list takes 16 doubles)
constexpr int kWarpDoubles = kInterpMaxCand * kMaxK + kInterpMaxCand * kInterpMaxCand +
                             kInterpMaxCand + 2 * kMaxK + kInterpMaxCand / 2;
constexpr int kInterpSmem = kWarps * kWarpDoubles * (int)sizeof(double);

template <class TS> __device__ __forceinline__ double widen(const TS *p, int k);
template <> __device__ __forceinline__ double widen<double>(const double *p, int k) { return p[k]; }
template <> __device__ __forceinline__ double widen<float>(const float *p, int k) { return (double)p[k]; }
template <> __device__ __forceinline__ double widen<__nv_bfloat16>(const __nv_bfloat16 *p, int k)
{
    return (double)__bfloat162float(p[k]);
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

// the subset's fit: 0 and p, res, or -1 when the normal equations are singular
__device__ int fit_subset(int s, const int *idx, const double *G, const double *b, int m,
                          const double *xs, const double *y, const double *w, int K, double *p,
                          double &res)
{
    double Gs[kInterpMaxCaliber * kInterpMaxCaliber], bs[kInterpMaxCaliber];
    for (int a = 0; a < s; ++a) {
        bs[a] = b[idx[a]];
        for (int c = 0; c < s; ++c) Gs[a * s + c] = G[idx[a] * m + idx[c]];
    }
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
    double r = 0.0;
    for (int k = 0; k < K; ++k) {
        double e = y[k];
        for (int a = 0; a < s; ++a) e = __dsub_rn(e, __dmul_rn(p[a], xs[idx[a] * kMaxK + k]));
        r = __dadd_rn(r, __dmul_rn(__dmul_rn(w[k], e), e));
    }
    res = r;
    return 0;
}

template <class TS>
__global__ void __launch_bounds__(kWarps * 32) k_ls_interp(InterpArgs A)
{
    extern __shared__ __align__(16) double ism[];
    const int wib = threadIdx.x / 32, lane = threadIdx.x % 32;
    double *xs = ism + (size_t)wib * kWarpDoubles;                 // candidate vectors
    double *G = xs + kInterpMaxCand * kMaxK;                       // Gram matrix
    double *b = G + kInterpMaxCand * kInterpMaxCand;               // right-hand side
    double *y = b + kInterpMaxCand;                                // target
    double *w = y + kMaxK;                                         // weights
    int32_t *cand = reinterpret_cast<int32_t *>(w + kMaxK);        // candidate columns
    const TS *X = (const TS *)A.x;
    const int K = A.K, Kp = A.Kp, C = A.caliber;
    for (int k = lane; k < K; k += 32) w[k] = A.w64[k];
    __syncwarp();

    const int64_t warps = (int64_t)gridDim.x * kWarps;
    for (int64_t i = (int64_t)blockIdx.x * kWarps + wib; i < A.n; i += warps) {
        if (A.coarse[i]) {
            if (lane == 0) {
                A.cnt[i] = 1;
                A.sel_col[i * kInterpMaxCaliber] = (int32_t)i;
                A.sel_val[i * kInterpMaxCaliber] = 1.0;
                A.ls[i] = 0.0;
            }
            continue;
        }
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
            xs[a * kMaxK + k] = widen<TS>(X + (int64_t)cand[a] * Kp, k);
        }
        __syncwarp();
        // Gram matrix and right-hand side: sum_k (w_k u_k) v_k in component order
        for (int t = lane; t < m * m; t += 32) {
            const int a = t / m, c = t % m;
            double g = 0.0;
            for (int k = 0; k < K; ++k) g = __dadd_rn(g, __dmul_rn(__dmul_rn(w[k], xs[a * kMaxK + k]), xs[c * kMaxK + k]));
            G[t] = g;
        }
        for (int a = lane; a < m; a += 32) {
            double g = 0.0;
            for (int k = 0; k < K; ++k) g = __dadd_rn(g, __dmul_rn(__dmul_rn(w[k], y[k]), xs[a * kMaxK + k]));
            b[a] = g;
        }
        double syy = 0.0;
        for (int k = 0; k < K; ++k) syy = __dadd_rn(syy, __dmul_rn(__dmul_rn(w[k], y[k]), y[k]));
        __syncwarp();

        // best set of every size: lane-local best, then a warp reduction
        // (smallest LS, then smallest rank)
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
                double p[kInterpMaxCaliber], res;
                unrank(m, s, t, idx);
                if (fit_subset(s, idx, G, b, m, xs, y, w, K, p, res) == 0 && res < mine) {
                    mine = res;
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
                double res;
                fit_subset(s, best_idx[s], G, b, m, xs, y, w, K, best_p[s], res);
            }
        }
        if (lane == 0) {
            int chosen = 0;
            if (syy > 0.0) {
                for (int s = 1; s <= kInterpMaxCaliber; ++s) {
                    if (!have[s]) continue;
                    const double cur = best_ls[chosen] / syy;
                    if (best_ls[s] / syy < pow(cur, A.gamma * (double)(s - chosen))) chosen = s;
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

}  // namespace

cudaError_t launch_ls_interp(int storage, const InterpArgs &a, cudaStream_t s)
{
    if (a.n == 0) return cudaSuccess;
    if (a.K > kMaxK || a.caliber < 1 || a.caliber > kInterpMaxCaliber) return cudaErrorInvalidValue;
    const int64_t want = ((int64_t)a.n + kWarps - 1) / kWarps;
    const unsigned grid = (unsigned)(want < 152 * 16 ? want : 152 * 16);
    static bool opted[3] = {false, false, false};
    cudaError_t e = cudaSuccess;
    switch (storage) {
    case ST_FP64:
        if (!opted[0]) e = cudaFuncSetAttribute(k_ls_interp<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kInterpSmem);
        if (e != cudaSuccess) return e;
        opted[0] = true;
        k_ls_interp<double><<<grid, kWarps * 32, kInterpSmem, s>>>(a);
        break;
    case ST_FP32:
        if (!opted[1]) e = cudaFuncSetAttribute(k_ls_interp<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kInterpSmem);
        if (e != cudaSuccess) return e;
        opted[1] = true;
        k_ls_interp<float><<<grid, kWarps * 32, kInterpSmem, s>>>(a);
        break;
    case ST_BF16:
        if (!opted[2]) e = cudaFuncSetAttribute(k_ls_interp<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, kInterpSmem);
        if (e != cudaSuccess) return e;
        opted[2] = true;
        k_ls_interp<__nv_bfloat16><<<grid, kWarps * 32, kInterpSmem, s>>>(a);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
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
