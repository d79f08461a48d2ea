// rowops.cuh -- per-row building blocks shared by the relaxation and edge
// kernels: gathering a row's neighbours in batches and accumulating the
// row sum  s = sum_p a(i, col_p) x(col_p)  component by component.
//
// Every component's sum is a chain of fused multiply-adds in CSR order, so
// the result does not depend on how lanes split the K components.  On the
// mixed paths (FP32 arithmetic) two components share one packed FP32 fused
// multiply-add (__ffma2_rn: two independent, correctly rounded FMAs), which
// halves the FMA instructions without changing a bit.
#pragma once

#include "amgd_internal.cuh"

namespace amgd {

// The piece of a row that lane `lane` of a row's G lanes holds as its t-th
// piece: with an even number of pieces per lane the lane holds them side by
// side (two move in one 32-byte access), otherwise they interleave over the
// G lanes.  Every component keeps its own FMA chain, so the layout never
// changes a row sum.
template <int G, int NV>
__device__ __forceinline__ int piece_of(int lane, int t)
{
    return (NV % 2 == 0) ? lane * NV + t : t * G + lane;
}

// read-only load of a CSR entry
template <class T>
__device__ __forceinline__ T ld_csr(const T *p)
{
    return __ldg(p);
}

// accumulator of the V components of one 16-byte piece
template <class C, int V> struct Acc;

template <int V> struct Acc<double, V> {
    double a[V];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int e = 0; e < V; ++e) a[e] = 0.0;
    }
    __device__ __forceinline__ void fma_piece(double v, const double (&x)[V]) {
#pragma unroll
        for (int e = 0; e < V; ++e) a[e] = fma(v, x[e], a[e]);
    }
    __device__ __forceinline__ double get(int e) const { return a[e]; }
};

template <int V> struct Acc<float, V> {
    static_assert(V % 2 == 0, "packed FP32 accumulation needs pairs");
    float2 a[V / 2];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int e = 0; e < V / 2; ++e) a[e] = make_float2(0.f, 0.f);
    }
    __device__ __forceinline__ void fma_piece(float v, const float (&x)[V]) {
        const float2 vv = make_float2(v, v);
#pragma unroll
        for (int e = 0; e < V / 2; ++e) a[e] = __ffma2_rn(vv, make_float2(x[2 * e], x[2 * e + 1]), a[e]);
    }
    __device__ __forceinline__ float get(int e) const { return (e & 1) ? a[e / 2].y : a[e / 2].x; }
};

// s[tt][e] = sum_{p in [p0,p1)} val[p] * X[col[p]] (lane's pieces), in CSR
// order.  SPLIT: rows j < split are read from xnew, the others from xold.
// rows, status: the gather range and status word of the checked build.
// Nonzeros are taken U at a time: U column indices and values, then all U
// gathers in flight before any is consumed.  A lane that holds an even number
// of pieces reads them in 32-byte pairs (piece_of): the rows are 32-byte
// aligned.
template <class TS, int G, int NV, int U, bool SPLIT>
__device__ __forceinline__ void row_sum(const int32_t *__restrict__ col,
                                        const typename Store<TS>::A *__restrict__ val,
                                        const TS *__restrict__ xold, const TS *__restrict__ xnew,
                                        int split, int Kp, int lane, int p0, int p1,
                                        Acc<typename Store<TS>::C, Store<TS>::V> (&acc)[NV],
                                        int64_t rows, uint32_t *status)
{
    using S = Store<TS>;
    using C = typename S::C;
    constexpr int V = S::V;
#pragma unroll
    for (int tt = 0; tt < NV; ++tt) acc[tt].zero();
    for (int pb = p0; pb < p1; pb += U) {
        int jj[U];
        C vv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool ok = pb + u < p1;
            jj[u] = ok ? ld_csr(col + pb + u) : -1;
            vv[u] = ok ? (C)ld_csr(val + pb + u) : C(0);
        }
        uint4 raw[U][NV];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (jj[u] >= 0) {
                const TS *src = (SPLIT && jj[u] < split ? xnew : xold) + checked_row(jj[u], rows, status) * Kp;
                if constexpr (NV % 2 == 0) {
#pragma unroll
                    for (int tt = 0; tt < NV; tt += 2)
                        ldg32(src + piece_of<G, NV>(lane, tt) * V, raw[u][tt], raw[u][tt + 1]);
                } else {
#pragma unroll
                    for (int tt = 0; tt < NV; ++tt) raw[u][tt] = ldg16(src + piece_of<G, NV>(lane, tt) * V);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (jj[u] < 0) break;
#pragma unroll
            for (int tt = 0; tt < NV; ++tt) {
                C x[V];
                S::unpack(raw[u][tt], x);
                acc[tt].fma_piece(vv[u], x);
            }
        }
    }
}

}  // namespace amgd
