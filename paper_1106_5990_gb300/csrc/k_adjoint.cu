// k_adjoint.cu -- reverse pass of the strength build for weighted-Jacobi
// sweeps: the gradient of a loss on the LS values with respect to A's values
// and omega.  The paper differentiates nothing; this is the chain rule
// through its steps (§3 relaxation, Eqs. (3.2), (4.1) target, §4.1 Eq. (4.3)
// one-point fits), in the caller's numbering:
//
//   fits      dLS_p/dy_i = 2 w (y_i - a_p x_j),  dLS_p/dx_j = -2 w a_p (y_i - a_p x_j)
//             (a_p minimises LS_p, so the dependence through a_p drops out)
//   target    Y = X - D^{-1} A X:  Xbar += Ybar - (D^{-1}A)^T Ybar,
//             dL/da_ik -= <Ybar_i, X_k>/a_ii,  dL/da_ii += <Ybar_i, (AX)_i>/a_ii^2
//   sweep k   X_{k+1} = X_k - omega D^{-1} A X_k:
//             Xbar_k = Xbar_{k+1} - omega (D^{-1}A)^T Xbar_{k+1}
//             dL/da_ik -= omega <Xbar_{k+1,i}, X_k,k'>/a_ii, diagonal and
//             omega terms from <Xbar_{k+1,i}, (A X_k)_i> = sum_p a_p <., X_k,col_p>
//
// The per-slot inner products are summed over the sweeps (gs) and kept
// apart for the target (gt); one final pass turns them into dL/dval and
// dL/domega.  Products with (D^{-1}A)^T run row by row over a transposed
// pattern whose entries are in ascending row order, so every sum has a fixed
// order and the result is deterministic (no atomics anywhere).
//
// Arithmetic.  The target, the fits (a_ij and LS_ij refitted in FP64 from the
// stored X_nu, k_refit), Y, Ybar, the last sweep's Xbar_nu and every per-slot
// sum (gs, gt) are FP64 whatever the storage: the loss weights each fit by
// LS^-3, so the fits must be exact to the digits the gradient needs.  The
// backward sweeps themselves (Xbar_k = Xbar_{k+1} - omega (D^-1 A)^T Xbar_{k+1}
// and the inner products <Xbar_{k+1,i}, X_k,j>) run in the arithmetic type of
// the storage ("CS": FP64 for FP64 storage, FP32 otherwise), a well-conditioned
// linear recurrence, their inner products accumulated over the sweeps in FP64.
// The stored iterates are widened exactly.
//
// Lane layout as in the forward kernels: G lanes per row, one 16-byte vector
// of the stored block per lane (V components); the FP64 vectors (Y, Ybar,
// Xbar) use the same components per lane.
#include <type_traits>

#include "amgd_internal.cuh"
#include "rowops.cuh"

namespace amgd {
namespace adj_impl {

constexpr int kThreads = 256;

template <int G>
__device__ __forceinline__ unsigned group_mask()
{
    if constexpr (G == 32) {
        return 0xffffffffu;
    } else {
        const unsigned lane = threadIdx.x & 31u;
        return ((1u << G) - 1u) << (lane & ~(unsigned)(G - 1));
    }
}

template <int G, class T>
__device__ __forceinline__ T group_sum(T v, unsigned mask)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, G);
    return v;
}

// V consecutive arithmetic-type components (16 or 32 bytes, aligned)
template <class C, int V>
__device__ __forceinline__ void ldc(const C *p, C (&x)[V])
{
    if constexpr (sizeof(C) == 8) {
#pragma unroll
        for (int c = 0; c < V / 2; ++c) {
            const double2 v = __ldg(reinterpret_cast<const double2 *>(p) + c);
            x[2 * c] = v.x;
            x[2 * c + 1] = v.y;
        }
    } else {
#pragma unroll
        for (int c = 0; c < V / 4; ++c) {
            const float4 v = __ldg(reinterpret_cast<const float4 *>(p) + c);
            x[4 * c] = v.x;
            x[4 * c + 1] = v.y;
            x[4 * c + 2] = v.z;
            x[4 * c + 3] = v.w;
        }
    }
}

template <class C, int V>
__device__ __forceinline__ void stc(C *p, const C (&x)[V])
{
    if constexpr (sizeof(C) == 8) {
#pragma unroll
        for (int c = 0; c < V / 2; ++c)
            reinterpret_cast<double2 *>(p)[c] = make_double2(x[2 * c], x[2 * c + 1]);
    } else {
#pragma unroll
        for (int c = 0; c < V / 4; ++c)
            reinterpret_cast<float4 *>(p)[c] = make_float4(x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3]);
    }
}

// V stored components of one 16-byte vector, widened exactly to FP64
template <class TS, int V>
__device__ __forceinline__ void unpack64(const uint4 &raw, double (&x)[V])
{
    typename Store<TS>::C t[V];
    Store<TS>::unpack(raw, t);
#pragma unroll
    for (int e = 0; e < V; ++e) x[e] = (double)t[e];
}

// y_i = x_i - (1/a_ii) sum_p a_ip x_col_p (one FMA per term in CSR order) or
// y_i = x_i: this lane's V components, FP64
template <class TS, int V>
__device__ __forceinline__ void target64(const AdjArgs &A, int64_t r, int lane, int p0, int p1,
                                         double (&y)[V])
{
    const TS *__restrict__ X = (const TS *)A.x;
    const int Kp = A.Kp;
    unpack64<TS, V>(ldg16(X + r * Kp + lane * V), y);
    if (A.target != 0) return;
    const double *__restrict__ val = (const double *)A.val;
    double acc[V];
#pragma unroll
    for (int e = 0; e < V; ++e) acc[e] = 0.0;
    for (int pb = p0; pb < p1; pb += 4) {
        uint4 raw[4];
        double v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (pb + u < p1) {
                raw[u] = ldg16(X + (int64_t)__ldg(A.col + pb + u) * Kp + lane * V);
                v[u] = __ldg(val + pb + u);
            }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (pb + u >= p1) break;
            double x[V];
            unpack64<TS, V>(raw[u], x);
#pragma unroll
            for (int e = 0; e < V; ++e) acc[e] = fma(v[u], x[e], acc[e]);
        }
    }
    const double d = 1.0 / __ldg((const double *)A.diag + r);
#pragma unroll
    for (int e = 0; e < V; ++e) y[e] = fma(-d, acc[e], y[e]);
}

// fixed-order block sum of one double per thread (result valid in thread 0)
__device__ __forceinline__ double block_sum(double v)
{
    __shared__ double wsum[kThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x / 32] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < kThreads / 32; ++k) t += wsum[k];
    __syncthreads();
    return t;
}

// ---------------------------------------------------------------------------
// dL/dLS per slot.  A slot carries no gradient on the diagonal and, for the
// residual target, in a row with one off-diagonal (LS there is the constant
// 0).  Built-in loss: L = sum LS^-2 over kept slots with LS > 0.
// ---------------------------------------------------------------------------
template <class C>
__global__ void __launch_bounds__(kThreads)
k_upstream(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
           const C *__restrict__ ls, const uint8_t *__restrict__ flag,
           const double *__restrict__ ls_bar, double *__restrict__ lsb,
           double *__restrict__ partial, int32_t n, int32_t target)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kThreads) {
        const int p0 = __ldg(rp + i), p1 = __ldg(rp + i + 1);
        const bool fixed = target == 0 && p1 - p0 == 2;
        for (int p = p0; p < p1; ++p) {
            double g = 0.0;
            if (__ldg(col + p) != i && !fixed) {
                if (ls_bar) {
                    g = __ldg(ls_bar + p);
                } else if (__ldg(flag + p)) {
                    const double l = (double)__ldg(ls + p);
                    if (l > 0.0) {
                        // one FP64 division per slot (the FP64 pipe is narrow)
                        const double inv = 1.0 / l, inv2 = inv * inv;
                        acc += inv2;
                        g = -2.0 * inv2 * inv;
                    }
                }
            }
            lsb[p] = g;
        }
    }
    const double t = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// a = yx / xx to within a few FP64 ulps: the FP32 quotient, then one FP64
// correction with the FP32 reciprocal (its error enters only at second
// order) -- four FP64 operations instead of a full FP64 division on the
// narrow FP64 pipe.  Quotients whose operands fall outside the FP32 range
// take the FP64 division.
__device__ __forceinline__ double fit_quotient(double yx, double xx)
{
    const double ax = fabs(xx), ay = fabs(yx);
    if (ax < 1e-30 || ax > 1e30 || ay > 1e30 || (ay != 0.0 && ay < 1e-30)) return yx / xx;
    const float xf = (float)xx;
    const double q0 = (double)((float)yx / xf);
    const double r = fma(-q0, xx, yx);
    return fma(r, (double)(1.0f / xf), q0);
}

template <class C>
__global__ void __launch_bounds__(kThreads)
k_bvals(const double *__restrict__ val, const double *__restrict__ diag,
        const int32_t *__restrict__ at_row, const int32_t *__restrict__ at_slot,
        C *__restrict__ b, int64_t nnz)
{
    for (int64_t q = (int64_t)blockIdx.x * kThreads + threadIdx.x; q < nnz;
         q += (int64_t)gridDim.x * kThreads)
        b[q] = (C)(__ldg(val + __ldg(at_slot + q)) / __ldg(diag + __ldg(at_row + q)));
}

// ---------------------------------------------------------------------------
// the one-point fits of every slot of row i refitted in FP64 from the stored
// X_nu (§4.1, Eq. (4.3)): a_p = S_yx / S_xx (0 if S_xx = 0), LS_p = sum w (y_i -
// a_p x_j)^2 (two passes); the exact rule of a residual-target row with one
// off-diagonal (a = -a_ij/a_ii, LS = 0); diagonal: a = 0, LS = NaN.  Written
// to A.a and A.ls64 for the upstream gradient and the adjoint of the fits.
// ---------------------------------------------------------------------------
// one FP64 fit of this lane's V components, with (UW) or without the weight
// products, reduced over the G lanes of the row
template <int G, int V, bool UW>
__device__ __forceinline__ void fit64(const double (&x)[V], const double (&y)[V], const double (&w)[V],
                                      unsigned gmask, double &a_, double &ls_)
{
    double xx = 0.0, yx = 0.0;
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const double wx = UW ? x[e] : w[e] * x[e];
        xx = fma(wx, x[e], xx);
        yx = fma(wx, y[e], yx);
    }
    xx = group_sum<G>(xx, gmask);
    yx = group_sum<G>(yx, gmask);
    a_ = (xx == 0.0) ? 0.0 : fit_quotient(yx, xx);
    double res = 0.0;
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const double d = fma(-a_, x[e], y[e]);
        res = fma(UW ? d : w[e] * d, d, res);
    }
    ls_ = group_sum<G>(res, gmask);
}

// ---------------------------------------------------------------------------
// Double-float fits (FP32/BF16 storage, unit weights): the same two-pass fit
// carried in pairs of FP32 words (value = hi + lo: about 48 significant bits)
// with error-free products (one FMA) and sums (TwoSum), on the FP32 pipe
// instead of the GB300's narrow FP64 pipe.  The stored components x are exact
// FP32 values; the FP64 target y enters as its two-word split.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void df_two_sum(float a, float b, float &s, float &e)
{
    const float t = __fadd_rn(a, b);
    const float bp = __fsub_rn(t, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(t, bp)), __fsub_rn(b, bp));
    s = t;
}
__device__ __forceinline__ void df_two_prod(float a, float b, float &p, float &e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}
// (s, c) += t + t_err: s the running sum, c every rounding error (s + c the value)
__device__ __forceinline__ void df_acc(float &s, float &c, float t, float t_err)
{
    float e;
    df_two_sum(s, t, s, e);
    c = __fadd_rn(c, __fadd_rn(e, t_err));
}
template <int G>
__device__ __forceinline__ void df_allreduce(float &s, float &c, unsigned mask)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        const float so = __shfl_xor_sync(mask, s, o, G), co = __shfl_xor_sync(mask, c, o, G);
        float e;
        df_two_sum(s, so, s, e);
        c = __fadd_rn(__fadd_rn(c, co), e);
    }
}

// one fit of this lane's V components (unit weights), reduced over the G lanes
// of the row; a and LS as two words each (value = hi + lo)
template <int G, int V>
__device__ __forceinline__ void fit_df(const float (&x)[V], const float (&yh)[V], const float (&yl)[V],
                                       unsigned gmask, float &ah, float &al, float &lh, float &ll)
{
    float sxx = 0.f, cxx = 0.f, syx = 0.f, cyx = 0.f;
#pragma unroll
    for (int e = 0; e < V; ++e) {
        float p, pe;
        df_two_prod(x[e], x[e], p, pe);
        df_acc(sxx, cxx, p, pe);
        df_two_prod(x[e], yh[e], p, pe);
        df_acc(syx, cyx, p, __fmaf_rn(x[e], yl[e], pe));
    }
    df_allreduce<G>(sxx, cxx, gmask);
    df_allreduce<G>(syx, cyx, gmask);
    float xh, xl, qh, ql;
    df_two_sum(sxx, cxx, xh, xl);
    df_two_sum(syx, cyx, qh, ql);
    ah = 0.f;
    al = 0.f;
    if (xh != 0.f) {
        // a = yx / xx: the FP32 quotient, then the quotient of its remainder
        ah = __fdiv_rn(qh, xh);
        float p, pe;
        df_two_prod(ah, xh, p, pe);
        const float r = __fadd_rn(__fsub_rn(__fsub_rn(qh, p), pe), __fmaf_rn(-ah, xl, ql));
        al = __fdiv_rn(r, xh);
    }
    float sls = 0.f, cls = 0.f;
#pragma unroll
    for (int e = 0; e < V; ++e) {
        // d = y - a x as two words, then d^2 = dh^2 + 2 dh dl
        float p, pe, t, te;
        df_two_prod(ah, x[e], p, pe);
        df_two_sum(yh[e], -p, t, te);
        const float dl0 = __fadd_rn(__fsub_rn(te, pe), __fmaf_rn(-al, x[e], yl[e]));
        float dh, dl;
        df_two_sum(t, dl0, dh, dl);
        float q, qe;
        df_two_prod(dh, dh, q, qe);
        df_acc(sls, cls, q, __fmaf_rn(__fmul_rn(2.f, dh), dl, qe));
    }
    df_allreduce<G>(sls, cls, gmask);
    df_two_sum(sls, cls, lh, ll);
}

template <class TS, int G>
__global__ void __launch_bounds__(kThreads) k_refit(AdjArgs A)
{
    using S = Store<TS>;
    constexpr int V = S::V;
    const int lane = threadIdx.x & (G - 1);
    const int64_t r = (int64_t)blockIdx.x * (kThreads / G) + threadIdx.x / G;
    if (r >= A.n) return;
    const unsigned gmask = group_mask<G>();
    const TS *__restrict__ X = (const TS *)A.x;
    const int Kp = A.Kp;
    const int p0 = __ldg(A.rp + r), p1 = __ldg(A.rp + r + 1);
    double w[V], y[V];
    ldc<double, V>((const double *)A.w + lane * V, w);
    target64<TS, V>(A, r, lane, p0, p1, y);
    stc<double, V>((double *)A.y + r * Kp + lane * V, y);     // for the adjoint of the fits
    double *a_out = (double *)A.a_fit;
    double *ls_out = A.ls64;
    const bool fixed = A.target == 0 && p1 - p0 == 2;
    const double diag = __ldg((const double *)A.diag + r);
    // mixed storage with unit weights: the fits in double-float (FP32 pipe)
    constexpr bool kMixed = !std::is_same<TS, double>::value;
    const bool df = kMixed && A.unit_w;
    float yh[V], yl[V];
    if (df) {
#pragma unroll
        for (int e = 0; e < V; ++e) {
            yh[e] = (float)y[e];
            yl[e] = (float)(y[e] - (double)yh[e]);
        }
    }
    for (int p = p0; p < p1; ++p) {
        const int64_t j = __ldg(A.col + p);
        double a_, ls_;
        if (j == r) {
            a_ = 0.0;
            ls_ = NAN;
        } else if (fixed) {
            a_ = -__ldg((const double *)A.val + p) / diag;
            ls_ = 0.0;
        } else if (df) {
            if constexpr (kMixed) {
                float xf[V], ah, al, lh, ll;
                Store<TS>::unpack(ldg16(X + j * Kp + lane * V), xf);
                fit_df<G, V>(xf, yh, yl, gmask, ah, al, lh, ll);
                a_ = (double)ah + (double)al;
                ls_ = (double)lh + (double)ll;
            }
        } else {
            double x[V];
            unpack64<TS, V>(ldg16(X + j * Kp + lane * V), x);
            if (A.unit_w) fit64<G, V, true>(x, y, w, gmask, a_, ls_);
            else fit64<G, V, false>(x, y, w, gmask, a_, ls_);
        }
        if (lane == 0) {
            a_out[p] = a_;
            ls_out[p] = ls_;
        }
    }
}

// ---------------------------------------------------------------------------
// row i (Y_i as k_refit left it): Ybar_i = 2 w (y_i sum_p lsb_p - sum_p lsb_p a_p x_j), and for
// the residual target gt_p = <Ybar_i, X_col_p> over all slots
// ---------------------------------------------------------------------------
template <class TS, int G>
__global__ void __launch_bounds__(kThreads) k_edge_bwd(AdjArgs A)
{
    using S = Store<TS>;
    using C = double;
    constexpr int V = S::V;
    const int lane = threadIdx.x & (G - 1);
    const int64_t r = (int64_t)blockIdx.x * (kThreads / G) + threadIdx.x / G;
    if (r >= A.n) return;
    const unsigned gmask = group_mask<G>();
    const TS *__restrict__ X = (const TS *)A.x;
    const int Kp = A.Kp;
    const int p0 = __ldg(A.rp + r), p1 = __ldg(A.rp + r + 1);
    const int64_t off = r * Kp + lane * V;

    C w[V], y[V];
    ldc<C, V>((const C *)A.w + lane * V, w);
    ldc<C, V>((const C *)A.y + off, y);            // the target, left by k_refit

    C v[V];
#pragma unroll
    for (int e = 0; e < V; ++e) v[e] = C(0);
    double L = 0.0;
    for (int p = p0; p < p1; ++p) {
        const double g = __ldg(A.lsb + p);
        if (g == 0.0) continue;
        const int j = __ldg(A.col + p);
        const C c = (C)(g * (double)__ldg((const C *)A.a + p));
        C xj[V];
        unpack64<TS, V>(ldg16(X + (int64_t)j * Kp + lane * V), xj);
#pragma unroll
        for (int e = 0; e < V; ++e) v[e] = fma(c, xj[e], v[e]);
        L += g;
    }
    C yb[V];
    const C Lc = (C)L;
#pragma unroll
    for (int e = 0; e < V; ++e) yb[e] = C(2) * w[e] * fma(Lc, y[e], -v[e]);
    stc<C, V>((C *)A.ybar + off, yb);

    if (A.target == 0) {
        C *gt = (C *)A.gt;
        for (int p = p0; p < p1; ++p) {
            const int j = __ldg(A.col + p);
            C xj[V];
            unpack64<TS, V>(ldg16(X + (int64_t)j * Kp + lane * V), xj);
            C part = C(0);
#pragma unroll
            for (int e = 0; e < V; ++e) part = fma(yb[e], xj[e], part);
            part = group_sum<G>(part, gmask);
            if (lane == 0) gt[p] = part;
        }
    }
}

// ---------------------------------------------------------------------------
// column j (rows i of the transposed pattern):
//   Xbar_nu,j = sum_{i != j} [ -2 lsb_p a_p w (y_i - a_p x_j)  - b_q Ybar_i ]
//   (+ Ybar_j for the plain target, whose adjoint is the identity; for the
//   residual target the identity and the diagonal entry b_jj = 1 cancel)
// ---------------------------------------------------------------------------
template <class TS, int G>
__global__ void __launch_bounds__(kThreads) k_xbar_nu(AdjArgs A)
{
    using S = Store<TS>;
    using C = double;
    constexpr int V = S::V;
    const int lane = threadIdx.x & (G - 1);
    const int64_t jr = (int64_t)blockIdx.x * (kThreads / G) + threadIdx.x / G;
    if (jr >= A.n) return;
    const TS *__restrict__ X = (const TS *)A.x;
    const C *__restrict__ Y = (const C *)A.y;
    const C *__restrict__ Yb = (const C *)A.ybar;
    const int Kp = A.Kp;
    const int64_t off = jr * Kp + lane * V;

    C w[V], xj[V], acc[V];
    ldc<C, V>((const C *)A.w + lane * V, w);
    unpack64<TS, V>(ldg16(X + off), xj);
    if (A.target == 1) {
        ldc<C, V>(Yb + off, acc);
    } else {
#pragma unroll
        for (int e = 0; e < V; ++e) acc[e] = C(0);
    }
    const int q0 = __ldg(A.at_rp + jr), q1 = __ldg(A.at_rp + jr + 1);
    for (int q = q0; q < q1; ++q) {
        const int i = __ldg(A.at_row + q);
        if (i == jr) continue;
        const int p = __ldg(A.at_slot + q);
        const double g = __ldg(A.lsb + p);
        if (g != 0.0) {
            const C ap = __ldg((const C *)A.a + p);
            const C c = (C)(-2.0 * g * (double)ap);
            C yi[V];
            ldc<C, V>(Y + (int64_t)i * Kp + lane * V, yi);
            if (A.unit_w) {
#pragma unroll
                for (int e = 0; e < V; ++e) acc[e] = fma(c, fma(-ap, xj[e], yi[e]), acc[e]);
            } else {
#pragma unroll
                for (int e = 0; e < V; ++e) acc[e] = fma(c * w[e], fma(-ap, xj[e], yi[e]), acc[e]);
            }
        }
        if (A.target == 0) {
            const C b = (C)__ldg((const typename S::C *)A.at_b + q);   // the sweeps' type
            C ybi[V];
            ldc<C, V>(Yb + (int64_t)i * Kp + lane * V, ybi);
#pragma unroll
            for (int e = 0; e < V; ++e) acc[e] = fma(-b, ybi[e], acc[e]);
        }
    }
    {
        using CS = typename S::C;        // the sweeps' arithmetic type
        CS out[V];
#pragma unroll
        for (int e = 0; e < V; ++e) out[e] = (CS)acc[e];
        stc<CS, V>((CS *)A.xbar_out + off, out);
    }
}

// ---------------------------------------------------------------------------
// row i of sweep k:  gs_p (+)= <Xbar_{k+1,i}, X_k,col_p>, neighbours gathered
// four at a time
// ---------------------------------------------------------------------------
template <class TS, int G>
__global__ void __launch_bounds__(kThreads) k_gram(AdjArgs A)
{
    using S = Store<TS>;
    using C = typename S::C;        // the sweeps' arithmetic type
    constexpr int V = S::V;
    constexpr int U = 4;
    const int lane = threadIdx.x & (G - 1);
    const int64_t r = (int64_t)blockIdx.x * (kThreads / G) + threadIdx.x / G;
    if (r >= A.n) return;
    const unsigned gmask = group_mask<G>();
    const TS *__restrict__ X = (const TS *)A.x;
    double *gs = (double *)A.gs;
    const int Kp = A.Kp;
    const int p0 = __ldg(A.rp + r), p1 = __ldg(A.rp + r + 1);
    C xb[V];
    ldc<C, V>((const C *)A.xbar_in + r * Kp + lane * V, xb);
    for (int pb = p0; pb < p1; pb += U) {
        uint4 raw[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (pb + u < p1) raw[u] = ldg16(X + (int64_t)__ldg(A.col + pb + u) * Kp + lane * V);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (pb + u >= p1) break;
            C xj[V];
            S::unpack(raw[u], xj);
            C part = C(0);
#pragma unroll
            for (int e = 0; e < V; ++e) part = fma(xb[e], xj[e], part);
            part = group_sum<G>(part, gmask);
            if (lane == 0) gs[pb + u] = A.first ? (double)part : gs[pb + u] + (double)part;
        }
    }
}

// column j of sweep k:  Xbar_k,j = Xbar_{k+1,j} - omega sum_q b_q Xbar_{k+1,at_row[q]}
template <class TS, int G>
__global__ void __launch_bounds__(kThreads) k_spmm_t(AdjArgs A)
{
    using S = Store<TS>;
    using C = typename S::C;        // the sweeps' arithmetic type
    constexpr int V = S::V;
    constexpr int U = 4;
    const int lane = threadIdx.x & (G - 1);
    const int64_t jr = (int64_t)blockIdx.x * (kThreads / G) + threadIdx.x / G;
    if (jr >= A.n) return;
    const C *__restrict__ Xb = (const C *)A.xbar_in;
    const C *__restrict__ b = (const C *)A.at_b;
    const int Kp = A.Kp;
    const C om = (C)A.omega;
    C acc[V];
    ldc<C, V>(Xb + jr * Kp + lane * V, acc);
    const int q0 = __ldg(A.at_rp + jr), q1 = __ldg(A.at_rp + jr + 1);
    for (int qb = q0; qb < q1; qb += U) {
        C xi[U][V];
        C c[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (qb + u < q1) {
                c[u] = om * __ldg(b + qb + u);
                ldc<C, V>(Xb + (int64_t)__ldg(A.at_row + qb + u) * Kp + lane * V, xi[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (qb + u >= q1) break;
#pragma unroll
            for (int e = 0; e < V; ++e) acc[e] = fma(-c[u], xi[u][e], acc[e]);
        }
    }
    stc<C, V>((C *)A.xbar_out + jr * Kp + lane * V, acc);
}

// Structurally symmetric pattern: both products of one reverse sweep in one
// pass over row j, whose columns i are exactly the rows of column j:
//   gs_p (+)= <Xbar_{k+1,j}, X_k,i>                    (slot p = (j, i))
//   Xbar_k,j = Xbar_{k+1,j} - omega sum_p bm_p Xbar_{k+1,i},  bm_p = a_ij / a_ii
// (the diagonal slot has bm = 1).  Neighbours are taken four at a time.
template <class TS, int G>
__global__ void __launch_bounds__(kThreads) k_sweep_sym(AdjArgs A)
{
    using S = Store<TS>;
    using C = typename S::C;        // the sweeps' arithmetic type
    constexpr int V = S::V;
    constexpr int U = 4;
    const int lane = threadIdx.x & (G - 1);
    const int64_t r = (int64_t)blockIdx.x * (kThreads / G) + threadIdx.x / G;
    if (r >= A.n) return;
    const unsigned gmask = group_mask<G>();
    const TS *__restrict__ X = (const TS *)A.x;
    const C *__restrict__ Xb = (const C *)A.xbar_in;
    const C *__restrict__ bm = (const C *)A.bm;
    double *gs = (double *)A.gs;
    const int Kp = A.Kp;
    const C om = (C)A.omega;
    const int p0 = __ldg(A.rp + r), p1 = __ldg(A.rp + r + 1);
    C xb[V], acc[V];
    ldc<C, V>(Xb + r * Kp + lane * V, xb);
#pragma unroll
    for (int e = 0; e < V; ++e) acc[e] = xb[e];
    for (int pb = p0; pb < p1; pb += U) {
        uint4 raw[U];
        C xbi[U][V];
        C c[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (pb + u < p1) {
                const int64_t i = __ldg(A.col + pb + u);
                raw[u] = ldg16(X + i * Kp + lane * V);
                ldc<C, V>(Xb + i * Kp + lane * V, xbi[u]);
                c[u] = om * __ldg(bm + pb + u);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (pb + u >= p1) break;
            C xi[V];
            S::unpack(raw[u], xi);
            C part = C(0);
#pragma unroll
            for (int e = 0; e < V; ++e) {
                part = fma(xb[e], xi[e], part);
                acc[e] = fma(-c[u], xbi[u][e], acc[e]);
            }
            part = group_sum<G>(part, gmask);
            if (lane == 0) gs[pb + u] = A.first ? (double)part : gs[pb + u] + (double)part;
        }
    }
    stc<C, V>((C *)A.xbar_out + r * Kp + lane * V, acc);
}

// ---------------------------------------------------------------------------
// row i: dL/dval_p = -(omega gs_p + gt_p) / a_ii on every slot, and on the
// diagonal slot + (qt_i + omega qs_i) / a_ii with q_i = sum_p val_p g_p / a_ii;
// dL/domega = -sum_i qs_i (per-block partials)
// ---------------------------------------------------------------------------
template <class C>
__global__ void __launch_bounds__(kThreads)
k_finish(const int32_t *__restrict__ rp, const double *__restrict__ val,
         const double *__restrict__ diag, const int32_t *__restrict__ dslot,
         const C *__restrict__ gs, const C *__restrict__ gt, double omega, int32_t n,
         double *__restrict__ vb, double *__restrict__ partial)
{
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kThreads) {
        const int p0 = __ldg(rp + i), p1 = __ldg(rp + i + 1);
        // one FP64 division per row (the GB300's FP64 pipe is narrow): every
        // quotient by a_ii below is a product with its reciprocal
        const double inv = 1.0 / __ldg(diag + i);
        double qs = 0.0, qt = 0.0;
        for (int p = p0; p < p1; ++p) {
            const double s = gs ? (double)__ldg(gs + p) : 0.0;
            const double t = gt ? (double)__ldg(gt + p) : 0.0;
            const double v = __ldg(val + p);
            vb[p] = -(omega * s + t) * inv;
            qs += v * s;
            qt += v * t;
        }
        qs *= inv;
        qt *= inv;
        vb[__ldg(dslot + i)] += (qt + omega * qs) * inv;
        acc -= qs;
    }
    const double t = block_sum(acc);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kThreads)
k_reduce(const double *__restrict__ partial, int32_t nblocks, double *__restrict__ out)
{
    double v = 0.0;
    for (int k = threadIdx.x; k < nblocks; k += kThreads) v += partial[(int64_t)blockIdx.x * nblocks + k];
    const double t = block_sum(v);
    if (threadIdx.x == 0) out[blockIdx.x] = t;
}

inline int64_t grid_rows(int64_t n, int G) { return (n + kThreads / G - 1) / (kThreads / G); }

}  // namespace adj_impl

using namespace adj_impl;

// lanes per row = 16-byte vectors per row
static int lanes(int storage, int Kp) { return Kp / (storage == ST_FP64 ? 2 : storage == ST_FP32 ? 4 : 8); }

#define AMGD_ADJ_SWITCH_G(KERNEL, TS)                                                   \
    switch (G) {                                                                         \
    case 1: KERNEL<TS, 1><<<(unsigned)grid_rows(a.n, 1), kThreads, 0, s>>>(a); break;    \
    case 2: KERNEL<TS, 2><<<(unsigned)grid_rows(a.n, 2), kThreads, 0, s>>>(a); break;    \
    case 4: KERNEL<TS, 4><<<(unsigned)grid_rows(a.n, 4), kThreads, 0, s>>>(a); break;    \
    case 8: KERNEL<TS, 8><<<(unsigned)grid_rows(a.n, 8), kThreads, 0, s>>>(a); break;    \
    case 16: KERNEL<TS, 16><<<(unsigned)grid_rows(a.n, 16), kThreads, 0, s>>>(a); break; \
    case 32: KERNEL<TS, 32><<<(unsigned)grid_rows(a.n, 32), kThreads, 0, s>>>(a); break; \
    default: return cudaErrorInvalidValue;                                               \
    }

#define AMGD_ADJ_LAUNCHER(NAME, KERNEL)                                                  \
    cudaError_t NAME(int storage, const AdjArgs &a, cudaStream_t s)                      \
    {                                                                                    \
        if (a.n == 0) return cudaSuccess;                                                \
        const int G = lanes(storage, a.Kp);                                              \
        if (storage == ST_FP64) {                                                        \
            AMGD_ADJ_SWITCH_G(KERNEL, double)                                            \
        } else if (storage == ST_FP32) {                                                 \
            AMGD_ADJ_SWITCH_G(KERNEL, float)                                             \
        } else {                                                                         \
            AMGD_ADJ_SWITCH_G(KERNEL, __nv_bfloat16)                                     \
        }                                                                                \
        return cudaGetLastError();                                                       \
    }

AMGD_ADJ_LAUNCHER(launch_adj_refit, k_refit)
AMGD_ADJ_LAUNCHER(launch_adj_edge, k_edge_bwd)
AMGD_ADJ_LAUNCHER(launch_adj_xbar_nu, k_xbar_nu)
AMGD_ADJ_LAUNCHER(launch_adj_gram, k_gram)
AMGD_ADJ_LAUNCHER(launch_adj_spmm_t, k_spmm_t)
AMGD_ADJ_LAUNCHER(launch_adj_sweep_sym, k_sweep_sym)

cudaError_t launch_adj_upstream(int storage, const int32_t *rp, const int32_t *col,
                                const void *ls, const uint8_t *flag, const double *ls_bar,
                                double *lsb, double *partial, int32_t nblocks, int32_t n,
                                int32_t target, cudaStream_t s)
{
    (void)storage;                       // LS refitted in FP64 for every storage
    k_upstream<double><<<nblocks, kThreads, 0, s>>>(rp, col, (const double *)ls, flag, ls_bar,
                                                    lsb, partial, n, target);
    return cudaGetLastError();
}

cudaError_t launch_adj_bvals(int storage, const double *val64, const double *diag64,
                             const int32_t *at_row, const int32_t *at_slot, void *at_b,
                             int64_t nnz, cudaStream_t s)
{
    if (nnz == 0) return cudaSuccess;
    const int64_t want = (nnz + kThreads - 1) / kThreads;
    const unsigned grid = (unsigned)(want < 152 * 16 ? want : 152 * 16);
    if (storage == ST_FP64)              // the sweeps' arithmetic type
        k_bvals<double><<<grid, kThreads, 0, s>>>(val64, diag64, at_row, at_slot, (double *)at_b, nnz);
    else
        k_bvals<float><<<grid, kThreads, 0, s>>>(val64, diag64, at_row, at_slot, (float *)at_b, nnz);
    return cudaGetLastError();
}

cudaError_t launch_adj_finish(int storage, const AdjArgs &a, bool have_gs, const double *val64,
                              const double *diag64, const int32_t *diag_slot, double *val_bar,
                              double *partial, int32_t nblocks, cudaStream_t s)
{
    const bool have_gt = a.target == 0;
    (void)storage;                       // FP64 reverse pass for every storage
    k_finish<double><<<nblocks, kThreads, 0, s>>>(
        a.rp, val64, diag64, diag_slot, have_gs ? (const double *)a.gs : nullptr,
        have_gt ? (const double *)a.gt : nullptr, a.omega, a.n, val_bar, partial);
    return cudaGetLastError();
}

cudaError_t launch_adj_reduce(const double *partial, int32_t nblocks, int32_t nsums, double *out,
                              cudaStream_t s)
{
    k_reduce<<<nsums, kThreads, 0, s>>>(partial, nblocks, out);
    return cudaGetLastError();
}

}  // namespace amgd
