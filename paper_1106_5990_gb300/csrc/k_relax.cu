// k_relax.cu -- relaxation of A x = 0 on an n x K block of test vectors
// (§3: the test vectors are produced by relaxing the homogeneous system from
// random starts; §2 and §5.2 use Gauss-Seidel).
//
// One launch processes the rows [r0, r1) of one color phase of the
// row-permuted matrix (all rows for Jacobi):
//     x_new(i) = x(i) - c_i * sum_p a(i, col_p) xhat(col_p),   c_i = omega / a_ii
// where xhat(j) is the new value for rows j < split (earlier colors of this
// sweep) and the value from the start of the sweep otherwise.  Jacobi is the
// case split = 0.  The row sum runs in CSR order with one fused multiply-add
// per term and the update is one fused multiply-add, so the FP64 path
// rounds exactly like a sequential row-by-row evaluation.
//
// Thread mapping: G lanes own one row; lane l holds the V consecutive
// components [l*V, l*V+V) of every K-vector it touches, loaded as one
// 16-byte vector.  A warp covers 32/G rows; every neighbour row x_j is one
// fully used 16*G-byte segment.  This is a CSR SpMM with K right-hand sides
// and is bound by HBM bandwidth (CSR once, x read and written once per
// phase); no tensor cores, nothing here is a dense contraction.
#include "amgd_internal.cuh"

namespace amgd {
namespace {

constexpr int kRelaxThreads = 256;

template <class TS, int G>
__global__ void __launch_bounds__(kRelaxThreads)
k_relax(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
        const typename Store<TS>::A *__restrict__ val, const TS *__restrict__ xold,
        TS *__restrict__ xnew, int32_t r0, int32_t r1, int32_t split, int32_t Kp,
        typename Store<TS>::C omega)
{
    using S = Store<TS>;
    using C = typename S::C;
    constexpr int V = S::V;
    const int lane = threadIdx.x % G;
    const int64_t r = (int64_t)r0 + (int64_t)blockIdx.x * (kRelaxThreads / G) + threadIdx.x / G;
    if (r >= r1) return;

    const int p0 = __ldg(rp + r), p1 = __ldg(rp + r + 1);
    C acc[V], xi[V];
#pragma unroll
    for (int e = 0; e < V; ++e) { acc[e] = C(0); xi[e] = C(0); }
    C diag = C(1);
    for (int p = p0; p < p1; ++p) {
        const int j = __ldg(col + p);
        const C v = (C)__ldg(val + p);
        const TS *src = (j < split ? (const TS *)xnew : xold) + (int64_t)j * Kp + lane * V;
        C xj[V];
        S::load(src, xj);
        if (j == r) {
            diag = v;
#pragma unroll
            for (int e = 0; e < V; ++e) xi[e] = xj[e];
        }
#pragma unroll
        for (int e = 0; e < V; ++e) acc[e] = fma(v, xj[e], acc[e]);
    }
    const C c = omega / diag;
    C out[V];
#pragma unroll
    for (int e = 0; e < V; ++e) out[e] = fma(-c, acc[e], xi[e]);
    S::store(xnew + r * Kp + lane * V, out);
}

template <class TS, int G>
cudaError_t go(const RelaxArgs &a, cudaStream_t s)
{
    using S = Store<TS>;
    const int64_t rows = (int64_t)a.r1 - a.r0;
    if (rows <= 0) return cudaSuccess;
    const int rows_per_block = kRelaxThreads / G;
    const unsigned grid = (unsigned)((rows + rows_per_block - 1) / rows_per_block);
    k_relax<TS, G><<<grid, kRelaxThreads, 0, s>>>(
        a.rp, a.col, (const typename S::A *)a.val, (const TS *)a.xold, (TS *)a.xnew, a.r0, a.r1,
        a.split, a.Kp, (typename S::C)a.omega);
    return cudaGetLastError();
}

template <class TS>
cudaError_t dispatch_g(int G, const RelaxArgs &a, cudaStream_t s)
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

cudaError_t launch_relax(int storage, int G, const RelaxArgs &a, cudaStream_t s)
{
    switch (storage) {
    case ST_FP64: return dispatch_g<double>(G, a, s);
    case ST_FP32: return dispatch_g<float>(G, a, s);
    case ST_BF16: return dispatch_g<__nv_bfloat16>(G, a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace amgd
