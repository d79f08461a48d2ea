// k_edge.cuh -- fused per-row pass: LS target, one-point least-squares fit
// for every stored off-diagonal, row-relative threshold and strength flags.
//
// For row i (G lanes, NV vectors of V components per lane, as in k_relax.cu):
//   1. y_i = x_i - (1/a_ii) sum_p a(i,col_p) x(col_p)     (Eqs. (3.2), (4.1):
//      the residual-corrected target, one local Jacobi step; same rounding
//      as the relaxation sweep with omega = 1), or y_i = x_i (Eq. (3.1)).
//   2. for every off-diagonal slot p = (i,j) (§4.1, Eq. (4.3)):
//        S_xx = sum_k w_k x_jk^2, S_yx = sum_k w_k y_ik x_jk   (lane partial
//        sums, then an xor-shuffle reduction inside the G lanes)
//        a_ij = S_yx / S_xx (0 if S_xx = 0)
//        LS_ij = sum_k w_k (y_ik - a_ij x_jk)^2   (second pass over the K
//        components, each residual one fused multiply-add: no cancellation
//        of S_yy - a S_yx; an error in a_ij enters LS only to second order)
//      A residual-target row with one off-diagonal has y_i proportional to
//      x_j exactly: a = -a_ij/a_ii, LS = 0.
//      Mixed precisions (FP32 arithmetic on FP32/BF16 vectors): an edge with
//      LS < 1e-4 S_yy is recomputed in FP64, with y_i rebuilt from the FP64
//      values of A, so cancellation never decides a distance.
//   3. m_i = min_p LS_ip; slot p is strong iff LS_p = 0 or theta LS_p < m_i
//      (§4.2, Eq. (4.4), r = 1/LS); per-row strong count.
// Outputs go to the caller's slot numbering (row i of the permuted matrix is
// row perm[i] of the caller, slot order unchanged).  Neighbour rows are
// gathered U at a time with all loads in flight, as in k_relax.cu.
#pragma once
#include <type_traits>

#include "amgd_internal.cuh"

namespace amgd {
namespace edge_impl {

constexpr int kEdgeThreads = 256;

template <int G, class T>
__device__ __forceinline__ T group_sum(T v, unsigned mask)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, G);
    return v;
}

// Mixed-path fallback: the one-point fit of slot (r, j) in FP64 from the
// stored vectors (widened exactly) and the FP64 values of A, y_i rebuilt
// with the FP64 path's rounding.  Called by all G lanes of the row's group.
// It runs only for edges whose FP32 functional cancelled, so it trades work
// for registers: every component is rebuilt from scalar loads, twice.
template <class TS>
__device__ __forceinline__ double load_elem(const TS *p)
{
    if constexpr (std::is_same<TS, __nv_bfloat16>::value)
        return (double)__bfloat162float(*p);
    else
        return (double)*p;
}

template <class TS>
__device__ __forceinline__ double y64_elem(const EdgeArgs &A, int64_t r, int p0, int p1, int k)
{
    const TS *X = (const TS *)A.x;
    double acc = 0.0, xi = 0.0, diag = 1.0;
    for (int q = p0; q < p1; ++q) {
        const int jj = __ldg(A.col + q);
        const double v = __ldg(A.val64 + q);
        const double x = load_elem<TS>(X + (int64_t)jj * A.Kp + k);
        if (jj == r) { xi = x; diag = v; }
        acc = fma(v, x, acc);
    }
    return (A.target == 0) ? fma(-(1.0 / diag), acc, xi) : xi;
}

template <class TS, int G, int NV>
__device__ __forceinline__ void edge_fp64(const EdgeArgs &A, int64_t r, int p0, int p1, int j,
                                       int lane, unsigned gmask, double &a64, double &ls64)
{
    constexpr int V = Store<TS>::V;
    const TS *xj = (const TS *)A.x + (int64_t)j * A.Kp;
    double sxx = 0.0, syx = 0.0;
#pragma unroll 1
    for (int c = 0; c < NV * V; ++c) {
        const int k = ((c / V) * G + lane) * V + c % V;
        const double x = load_elem<TS>(xj + k), wx = A.w64[k] * x;
        sxx = fma(wx, x, sxx);
        syx = fma(wx, y64_elem<TS>(A, r, p0, p1, k), syx);
    }
    sxx = group_sum<G>(sxx, gmask);
    syx = group_sum<G>(syx, gmask);
    a64 = (sxx == 0.0) ? 0.0 : syx / sxx;
    double res = 0.0;
#pragma unroll 1
    for (int c = 0; c < NV * V; ++c) {
        const int k = ((c / V) * G + lane) * V + c % V;
        const double d = fma(-a64, load_elem<TS>(xj + k), y64_elem<TS>(A, r, p0, p1, k));
        res = fma(A.w64[k] * d, d, res);
    }
    ls64 = group_sum<G>(res, gmask);
}

template <class C> __device__ __forceinline__ C divide(C a, C b) { return a / b; }
// the mixed path's coefficient only needs FP32 relative accuracy (its error
// enters LS at second order): the fast division is enough
template <> __device__ __forceinline__ float divide<float>(float a, float b)
{
    return __fdividef(a, b);
}

template <class TS, int G, int NV, int U, bool UW>
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

    const int32_t *__restrict__ col = A.col;
    const AV *__restrict__ val = (const AV *)A.val;
    const TS *__restrict__ X = (const TS *)A.x;
    const int Kp = A.Kp;

    C w[NV][V];
    if constexpr (!UW) {
#pragma unroll
        for (int t = 0; t < NV; ++t)
#pragma unroll
            for (int e = 0; e < V; ++e) w[t][e] = ((const C *)A.w)[(t * G + lane) * V + e];
    }

    const int p0 = __ldg(A.rp + r), p1 = __ldg(A.rp + r + 1);

    // ---- 1. target ------------------------------------------------------
    C acc[NV][V], y[NV][V];
#pragma unroll
    for (int t = 0; t < NV; ++t)
#pragma unroll
        for (int e = 0; e < V; ++e) { acc[t][e] = C(0); y[t][e] = C(0); }
    C diag = C(1);
    for (int pb = p0; pb < p1; pb += U) {
        int jj[U];
        C vv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool ok = pb + u < p1;
            jj[u] = ok ? __ldg(col + pb + u) : -1;
            vv[u] = ok ? (C)__ldg(val + pb + u) : C(0);
        }
        uint4 raw[U][NV];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (jj[u] >= 0)
#pragma unroll
                for (int t = 0; t < NV; ++t)
                    raw[u][t] = ldg16(X + (int64_t)jj[u] * Kp + (t * G + lane) * V);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (jj[u] < 0) break;
#pragma unroll
            for (int t = 0; t < NV; ++t) {
                C x[V];
                S::unpack(raw[u][t], x);
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    if (jj[u] == r) y[t][e] = x[e];     // x_i for now
                    acc[t][e] = fma(vv[u], x[e], acc[t][e]);
                }
            }
            if (jj[u] == r) diag = vv[u];
        }
    }
    if (A.target == 0) {
        const C d = C(1) / diag;
#pragma unroll
        for (int t = 0; t < NV; ++t)
#pragma unroll
            for (int e = 0; e < V; ++e) y[t][e] = fma(-d, acc[t][e], y[t][e]);
    }
    C syy = C(0);
    if constexpr (kMixed) {
#pragma unroll
        for (int t = 0; t < NV; ++t)
#pragma unroll
            for (int e = 0; e < V; ++e)
                syy = fma(UW ? y[t][e] : w[t][e] * y[t][e], y[t][e], syy);
        syy = group_sum<G>(syy, gmask);
    }

    const int off = p1 - p0 - 1;
    const int32_t orow = A.perm ? __ldg(A.perm + r) : (int32_t)r;
    const int64_t obase = __ldg(A.rp_orig + orow);
    C *a_out = (C *)A.a_out;
    C *ls_out = (C *)A.ls_out;

    // ---- 2. one-point LS per off-diagonal ---------------------------------
    C m = C(INFINITY);
    for (int pb = p0; pb < p1; pb += U) {
        int jj[U];
#pragma unroll
        for (int u = 0; u < U; ++u) jj[u] = (pb + u < p1) ? __ldg(col + pb + u) : -1;
        uint4 raw[U][NV];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (jj[u] >= 0 && jj[u] != r)
#pragma unroll
                for (int t = 0; t < NV; ++t)
                    raw[u][t] = ldg16(X + (int64_t)jj[u] * Kp + (t * G + lane) * V);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (jj[u] < 0) break;
            const int p = pb + u;
            C a_, ls_;
            if (jj[u] == r) {
                a_ = C(0);
                ls_ = C(NAN);
            } else if (A.target == 0 && off == 1) {
                a_ = -(C)__ldg(val + p) / diag;
                ls_ = C(0);
            } else {
                C xj[NV][V];
                C sxx = C(0), syx = C(0);
#pragma unroll
                for (int t = 0; t < NV; ++t) {
                    S::unpack(raw[u][t], xj[t]);
#pragma unroll
                    for (int e = 0; e < V; ++e) {
                        const C wx = UW ? xj[t][e] : w[t][e] * xj[t][e];
                        sxx = fma(wx, xj[t][e], sxx);
                        syx = fma(wx, y[t][e], syx);
                    }
                }
                sxx = group_sum<G>(sxx, gmask);
                syx = group_sum<G>(syx, gmask);
                a_ = (sxx == C(0)) ? C(0) : divide(syx, sxx);
                C res = C(0);
#pragma unroll
                for (int t = 0; t < NV; ++t)
#pragma unroll
                    for (int e = 0; e < V; ++e) {
                        const C d = fma(-a_, xj[t][e], y[t][e]);
                        res = fma(UW ? d : w[t][e] * d, d, res);
                    }
                ls_ = group_sum<G>(res, gmask);
                if constexpr (kMixed) {
                    if (ls_ < C(1e-4) * syy) {
                        double a64, ls64;
                        edge_fp64<TS, G, NV>(A, r, p0, p1, jj[u], lane, gmask, a64, ls64);
                        a_ = (C)a64;
                        ls_ = (C)ls64;
                    }
                }
            }
            if (jj[u] != r) m = fmin(m, ls_);
            if (lane == 0) {
                const int64_t slot = obase + (p - p0);
                a_out[slot] = a_;
                ls_out[slot] = ls_;
            }
        }
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

template <class TS, int G, int NV, int U, bool UW>
cudaError_t go(const EdgeArgs &a, cudaStream_t s)
{
    if (a.n <= 0) return cudaSuccess;
    const int rows_per_block = kEdgeThreads / G;
    const unsigned grid = (unsigned)(((int64_t)a.n + rows_per_block - 1) / rows_per_block);
    k_edge<TS, G, NV, U, UW><<<grid, kEdgeThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <class TS, int G, int NV, bool UW>
cudaError_t dispatch_u(int U, const EdgeArgs &a, cudaStream_t s)
{
    switch (U) {
    case 4: return go<TS, G, NV, 4, UW>(a, s);
    case 8: return go<TS, G, NV, 8, UW>(a, s);
    }
    return cudaErrorInvalidValue;
}

template <class TS, int G, int NV>
cudaError_t dispatch_w(int U, bool unit_w, const EdgeArgs &a, cudaStream_t s)
{
    return unit_w ? dispatch_u<TS, G, NV, true>(U, a, s) : dispatch_u<TS, G, NV, false>(U, a, s);
}

template <class TS, int G>
cudaError_t dispatch_nv(int NV, int U, bool unit_w, const EdgeArgs &a, cudaStream_t s)
{
    constexpr int V = Store<TS>::V;
    switch (NV) {
    case 1: return dispatch_w<TS, G, 1>(U, unit_w, a, s);
    case 2: if constexpr (G * 2 * V <= 64) return dispatch_w<TS, G, 2>(U, unit_w, a, s); break;
    case 4: if constexpr (G * 4 * V <= 64) return dispatch_w<TS, G, 4>(U, unit_w, a, s); break;
    }
    return cudaErrorInvalidValue;
}

template <class TS>
cudaError_t dispatch_g(Shape sh, bool unit_w, const EdgeArgs &a, cudaStream_t s)
{
    constexpr int V = Store<TS>::V;
    switch (sh.G) {
    case 1: return dispatch_nv<TS, 1>(sh.NV, sh.U, unit_w, a, s);
    case 2: return dispatch_nv<TS, 2>(sh.NV, sh.U, unit_w, a, s);
    case 4: return dispatch_nv<TS, 4>(sh.NV, sh.U, unit_w, a, s);
    case 8: if constexpr (8 * V <= 64) return dispatch_nv<TS, 8>(sh.NV, sh.U, unit_w, a, s); break;
    case 16: if constexpr (16 * V <= 64) return dispatch_nv<TS, 16>(sh.NV, sh.U, unit_w, a, s); break;
    case 32: if constexpr (32 * V <= 64) return dispatch_nv<TS, 32>(sh.NV, sh.U, unit_w, a, s); break;
    }
    return cudaErrorInvalidValue;
}

}  // namespace edge_impl
}  // namespace amgd
