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
// Thread mapping (Shape): G lanes own one row; lane l holds the 16-byte
// vectors l, l+G, ..., l+(NV-1)G of every K-vector row it touches, so each
// neighbour row is read as G*NV fully used 16-byte pieces.  Nonzeros are
// taken U at a time: U column indices and values are loaded, then all U*NV
// vector pieces are requested before any is consumed, which keeps U*NV loads
// per lane in flight (the kernel is bound by HBM latency and bandwidth: CSR
// once, vectors read and written once per phase).  The sums still run in CSR
// order.  This is a CSR SpMM with K right-hand sides; no tensor cores.
#include "amgd_internal.cuh"

namespace amgd {
namespace {

constexpr int kRelaxThreads = 256;

template <class TS, int G, int NV, int U>
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
    C acc[NV][V], xi[NV][V];
#pragma unroll
    for (int t = 0; t < NV; ++t)
#pragma unroll
        for (int e = 0; e < V; ++e) { acc[t][e] = C(0); xi[t][e] = C(0); }
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
        for (int u = 0; u < U; ++u) {
            if (jj[u] >= 0) {
                const TS *src = (jj[u] < split ? (const TS *)xnew : xold) + (int64_t)jj[u] * Kp;
#pragma unroll
                for (int t = 0; t < NV; ++t) raw[u][t] = ldg16(src + (t * G + lane) * V);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (jj[u] < 0) break;
#pragma unroll
            for (int t = 0; t < NV; ++t) {
                C x[V];
                S::unpack(raw[u][t], x);
                if (jj[u] == r) {
#pragma unroll
                    for (int e = 0; e < V; ++e) xi[t][e] = x[e];
                }
#pragma unroll
                for (int e = 0; e < V; ++e) acc[t][e] = fma(vv[u], x[e], acc[t][e]);
            }
            if (jj[u] == r) diag = vv[u];
        }
    }
    const C c = omega / diag;
#pragma unroll
    for (int t = 0; t < NV; ++t) {
        C out[V];
#pragma unroll
        for (int e = 0; e < V; ++e) out[e] = fma(-c, acc[t][e], xi[t][e]);
        S::store(xnew + r * Kp + (t * G + lane) * V, out);
    }
}

template <class TS, int G, int NV, int U>
cudaError_t go(const RelaxArgs &a, cudaStream_t s)
{
    using S = Store<TS>;
    const int64_t rows = (int64_t)a.r1 - a.r0;
    if (rows <= 0) return cudaSuccess;
    const int rows_per_block = kRelaxThreads / G;
    const unsigned grid = (unsigned)((rows + rows_per_block - 1) / rows_per_block);
    k_relax<TS, G, NV, U><<<grid, kRelaxThreads, 0, s>>>(
        a.rp, a.col, (const typename S::A *)a.val, (const TS *)a.xold, (TS *)a.xnew, a.r0, a.r1,
        a.split, a.Kp, (typename S::C)a.omega);
    return cudaGetLastError();
}

template <class TS, int G, int NV>
cudaError_t dispatch_u(int U, const RelaxArgs &a, cudaStream_t s)
{
    switch (U) {
    case 4: return go<TS, G, NV, 4>(a, s);
    case 8: return go<TS, G, NV, 8>(a, s);
    }
    return cudaErrorInvalidValue;
}

template <class TS, int G>
cudaError_t dispatch_nv(int NV, int U, const RelaxArgs &a, cudaStream_t s)
{
    constexpr int V = Store<TS>::V;
    switch (NV) {
    case 1: return dispatch_u<TS, G, 1>(U, a, s);
    case 2: if constexpr (G * 2 * V <= 64) return dispatch_u<TS, G, 2>(U, a, s); break;
    case 4: if constexpr (G * 4 * V <= 64) return dispatch_u<TS, G, 4>(U, a, s); break;
    }
    return cudaErrorInvalidValue;
}

template <class TS>
cudaError_t dispatch_g(Shape sh, const RelaxArgs &a, cudaStream_t s)
{
    constexpr int V = Store<TS>::V;
    switch (sh.G) {
    case 1: return dispatch_nv<TS, 1>(sh.NV, sh.U, a, s);
    case 2: return dispatch_nv<TS, 2>(sh.NV, sh.U, a, s);
    case 4: return dispatch_nv<TS, 4>(sh.NV, sh.U, a, s);
    case 8: if constexpr (8 * V <= 64) return dispatch_nv<TS, 8>(sh.NV, sh.U, a, s); break;
    case 16: if constexpr (16 * V <= 64) return dispatch_nv<TS, 16>(sh.NV, sh.U, a, s); break;
    case 32: if constexpr (32 * V <= 64) return dispatch_nv<TS, 32>(sh.NV, sh.U, a, s); break;
    }
    return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_relax(int storage, Shape sh, const RelaxArgs &a, cudaStream_t s)
{
    switch (storage) {
    case ST_FP64: return dispatch_g<double>(sh, a, s);
    case ST_FP32: return dispatch_g<float>(sh, a, s);
    case ST_BF16: return dispatch_g<__nv_bfloat16>(sh, a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace amgd
