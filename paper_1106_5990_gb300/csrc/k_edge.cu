// k_edge.cu -- fused per-row pass: LS target, one-point least-squares fit
// for every stored off-diagonal, row-relative threshold and strength flags.
//
// For row i (G lanes, V components per lane, as in k_relax.cu):
//   1. y_i = x_i - (1/a_ii) sum_p a(i,col_p) x(col_p)     (Eqs. (3.2), (4.1):
//      the residual-corrected target, one local Jacobi step; same rounding
//      as the relaxation sweep with omega = 1), or y_i = x_i (Eq. (3.1)).
//   2. for every off-diagonal slot p = (i,j) (§4.1, Eq. (4.3)):
//        S_xx = sum_k w_k x_jk^2, S_yx = sum_k w_k y_ik x_jk   (lane partial
//        sums, then an xor-shuffle reduction inside the G lanes)
//        a_ij = S_yx / S_xx (0 if S_xx = 0)
//        LS_ij = sum_k w_k (y_ik - a_ij x_jk)^2   (second pass, x_j still in
//        registers, so no cancellation of S_yy - a S_yx)
//      A residual-target row with one off-diagonal has y_i proportional to
//      x_j exactly: a = -a_ij/a_ii, LS = 0.
//      Mixed precisions (FP32 arithmetic on FP32/BF16 vectors): an edge with
//      LS < 1e-4 S_yy is recomputed in FP64, with y_i rebuilt from the FP64
//      values of A, so cancellation never decides a distance.
//   3. m_i = min_p LS_ip; slot p is strong iff LS_p = 0 or theta LS_p < m_i
//      (§4.2, Eq. (4.4), r = 1/LS); per-row strong count.
// Outputs go to the caller's slot numbering (row i of the permuted matrix is
// row perm[i] of the caller, slot order unchanged).
#include <type_traits>

#include "amgd_internal.cuh"

namespace amgd {
namespace {

constexpr int kEdgeThreads = 256;

template <int G, class T>
__device__ __forceinline__ T group_sum(T v, unsigned mask)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, G);
    return v;
}

// Mixed-path fallback, part 1: y_i rebuilt in FP64 from the FP64 values of
// A and the stored (exactly widened) vectors, same rounding as the FP64 path.
template <class TS>
__device__ __noinline__ void build_y64(const EdgeArgs &A, int64_t r, int p0, int p1, int lane,
                                       double (&y64)[Store<TS>::V])
{
    using S = Store<TS>;
    using C = typename S::C;
    constexpr int V = S::V;
    const TS *X = (const TS *)A.x;
    double acc64[V], xi64[V];
    double diag64 = 1.0;
#pragma unroll
    for (int e = 0; e < V; ++e) { acc64[e] = 0.0; xi64[e] = 0.0; }
    for (int q = p0; q < p1; ++q) {
        const int jj = __ldg(A.col + q);
        const double v64 = __ldg(A.val64 + q);
        C xq[V];
        S::load(X + (int64_t)jj * A.Kp + lane * V, xq);
        if (jj == r) {
            diag64 = v64;
#pragma unroll
            for (int e = 0; e < V; ++e) xi64[e] = (double)xq[e];
        }
#pragma unroll
        for (int e = 0; e < V; ++e) acc64[e] = fma(v64, (double)xq[e], acc64[e]);
    }
    const double d64 = 1.0 / diag64;
#pragma unroll
    for (int e = 0; e < V; ++e) y64[e] = (A.target == 0) ? fma(-d64, acc64[e], xi64[e]) : xi64[e];
}

// Mixed-path fallback, part 2: the one-point fit of one edge in FP64.
template <class TS, int G>
__device__ __forceinline__ void edge_fp64(const EdgeArgs &A, const typename Store<TS>::C (&xj)[Store<TS>::V],
                                          const double (&y64)[Store<TS>::V], int lane,
                                          unsigned gmask, double &a64, double &ls64)
{
    constexpr int V = Store<TS>::V;
    double sxx = 0.0, syx = 0.0;
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const double wx = A.w64[lane * V + e] * (double)xj[e];
        sxx = fma(wx, (double)xj[e], sxx);
        syx = fma(wx, y64[e], syx);
    }
    sxx = group_sum<G>(sxx, gmask);
    syx = group_sum<G>(syx, gmask);
    a64 = (sxx == 0.0) ? 0.0 : syx / sxx;
    double res = 0.0;
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const double d = fma(-a64, (double)xj[e], y64[e]);
        res = fma(A.w64[lane * V + e] * d, d, res);
    }
    ls64 = group_sum<G>(res, gmask);
}

template <class TS, int G>
__global__ void __launch_bounds__(kEdgeThreads) k_edge(EdgeArgs A)
{
    using S = Store<TS>;
    using C = typename S::C;
    using AV = typename S::A;
    constexpr int V = S::V;
    constexpr bool kMixed = !std::is_same<C, double>::value;

    const int lane = threadIdx.x % G;
    const int grp_in_warp = (threadIdx.x % 32) / G;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (grp_in_warp * G));
    const int64_t r = (int64_t)blockIdx.x * (kEdgeThreads / G) + threadIdx.x / G;
    if (r >= A.n) return;

    const int32_t *__restrict__ rp = A.rp;
    const int32_t *__restrict__ col = A.col;
    const AV *__restrict__ val = (const AV *)A.val;
    const TS *__restrict__ X = (const TS *)A.x;
    const int Kp = A.Kp;

    C w[V];
#pragma unroll
    for (int e = 0; e < V; ++e) w[e] = ((const C *)A.w)[lane * V + e];

    const int p0 = __ldg(rp + r), p1 = __ldg(rp + r + 1);

    // ---- 1. target ------------------------------------------------------
    C acc[V], xi[V], y[V];
#pragma unroll
    for (int e = 0; e < V; ++e) { acc[e] = C(0); xi[e] = C(0); }
    C diag = C(1);
    for (int p = p0; p < p1; ++p) {
        const int j = __ldg(col + p);
        const C v = (C)__ldg(val + p);
        C xj[V];
        S::load(X + (int64_t)j * Kp + lane * V, xj);
        if (j == r) {
            diag = v;
#pragma unroll
            for (int e = 0; e < V; ++e) xi[e] = xj[e];
        }
#pragma unroll
        for (int e = 0; e < V; ++e) acc[e] = fma(v, xj[e], acc[e]);
    }
    if (A.target == 0) {
        const C d = C(1) / diag;
#pragma unroll
        for (int e = 0; e < V; ++e) y[e] = fma(-d, acc[e], xi[e]);
    } else {
#pragma unroll
        for (int e = 0; e < V; ++e) y[e] = xi[e];
    }
    C syy = C(0);
    if (kMixed) {
#pragma unroll
        for (int e = 0; e < V; ++e) syy = fma(w[e] * y[e], y[e], syy);
        syy = group_sum<G>(syy, gmask);
    }

    const int off = p1 - p0 - 1;
    const int32_t orow = A.perm ? __ldg(A.perm + r) : (int32_t)r;
    const int64_t obase = __ldg(A.rp_orig + orow);
    C *a_out = (C *)A.a_out;
    C *ls_out = (C *)A.ls_out;

    // FP64 rebuild of y_i for the mixed-path fallback (built on first use)
    double y64[V];
    bool have_y64 = false;

    // ---- 2. one-point LS per off-diagonal ---------------------------------
    C m = C(INFINITY);
    for (int p = p0; p < p1; ++p) {
        const int j = __ldg(col + p);
        C a_, ls_;
        if (j == r) {
            a_ = C(0);
            ls_ = C(NAN);
        } else if (A.target == 0 && off == 1) {
            a_ = -(C)__ldg(val + p) / diag;
            ls_ = C(0);
        } else {
            C xj[V];
            S::load(X + (int64_t)j * Kp + lane * V, xj);
            C sxx = C(0), syx = C(0);
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const C wx = w[e] * xj[e];
                sxx = fma(wx, xj[e], sxx);
                syx = fma(wx, y[e], syx);
            }
            sxx = group_sum<G>(sxx, gmask);
            syx = group_sum<G>(syx, gmask);
            a_ = (sxx == C(0)) ? C(0) : syx / sxx;
            C res = C(0);
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const C d = fma(-a_, xj[e], y[e]);
                res = fma(w[e] * d, d, res);
            }
            ls_ = group_sum<G>(res, gmask);
            if constexpr (kMixed) {
                if (ls_ < C(1e-4) * syy) {
                    // cancellation: redo this edge in FP64 from the stored vectors
                    if (!have_y64) {
                        build_y64<TS>(A, r, p0, p1, lane, y64);
                        have_y64 = true;
                    }
                    double a64, ls64;
                    edge_fp64<TS, G>(A, xj, y64, lane, gmask, a64, ls64);
                    a_ = (C)a64;
                    ls_ = (C)ls64;
                }
            }
        }
        if (lane == 0) {
            const int64_t slot = obase + (p - p0);
            a_out[slot] = a_;
            ls_out[slot] = ls_;
        }
        if (j != r) m = fmin(m, ls_);
    }

    // ---- 3. strength flags -------------------------------------------------
    __syncwarp(gmask);
    const C theta = (C)A.theta;
    int cnt = 0;
    for (int p = p0 + lane; p < p1; p += G) {
        const int64_t slot = obase + (p - p0);
        const int j = __ldg(col + p);
        const C l = ls_out[slot];
        const int strong = (j != r) && (l == C(0) || theta * l < m);
        A.flag_out[slot] = (uint8_t)strong;
        cnt += strong;
    }
    cnt = group_sum<G>(cnt, gmask);
    if (lane == 0) A.count_out[orow] = cnt;
}

template <class TS, int G>
cudaError_t go(const EdgeArgs &a, cudaStream_t s)
{
    if (a.n <= 0) return cudaSuccess;
    const int rows_per_block = kEdgeThreads / G;
    const unsigned grid = (unsigned)(((int64_t)a.n + rows_per_block - 1) / rows_per_block);
    k_edge<TS, G><<<grid, kEdgeThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <class TS>
cudaError_t dispatch_g(int G, const EdgeArgs &a, cudaStream_t s)
{
    constexpr int V = Store<TS>::V;
    switch (G) {
    case 1: return go<TS, 1>(a, s);
    case 2: return go<TS, 2>(a, s);
    case 4: return go<TS, 4>(a, s);
    case 8: return go<TS, 8>(a, s);
    case 16: if constexpr (16 * V <= 64) return go<TS, 16>(a, s); break;
    case 32: if constexpr (32 * V <= 64) return go<TS, 32>(a, s); break;
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_edge(int storage, int G, const EdgeArgs &a, cudaStream_t s)
{
    switch (storage) {
    case ST_FP64: return dispatch_g<double>(G, a, s);
    case ST_FP32: return dispatch_g<float>(G, a, s);
    case ST_BF16: return dispatch_g<__nv_bfloat16>(G, a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace amgd
