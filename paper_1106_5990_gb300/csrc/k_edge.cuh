// k_edge.cuh -- fused pass over the stored entries: LS target, one-point
// least-squares fit for every stored off-diagonal, row-relative threshold
// and strength flags.
//
// For row i and its stored entries p = (i, j):
//   1. y_i = x_i - (1/a_ii) sum_p a(i,col_p) x(col_p)     (Eqs. (3.2), (4.1):
//      the residual-corrected target, one local Jacobi step; same rounding
//      as the relaxation sweep with omega = 1), or y_i = x_i (Eq. (3.1)).
//   2. for every off-diagonal (§4.1, Eq. (4.3)):
//        S_xx = sum_k w_k x_jk^2, S_yx = sum_k w_k y_ik x_jk
//        a_ij = S_yx / S_xx (0 if S_xx = 0)
//        LS_ij = sum_k w_k (y_ik - a_ij x_jk)^2   (second pass over the K
//        components, each residual one fused multiply-add: no cancellation
//        of S_yy - a S_yx; an error in a_ij enters LS only to second order)
//      A residual-target row with one off-diagonal has y_i proportional to
//      x_j exactly: a = -a_ij/a_ii, LS = 0.
//      Mixed precisions (FP32 arithmetic on FP32/BF16 vectors): the three
//      sums are compensated (AMGD_SUM_COMPENSATED, below) or plain FMA
//      chains; a row with an edge of LS < 1e-4 S_yy is recomputed in FP64
//      (k_edge_fixup), with y_i rebuilt from the FP64 values of A, so
//      cancellation never decides a distance.
//   3. m_i = min_p LS_ip; slot p is strong iff LS_p = 0 or theta LS_p < m_i
//      (§4.2, Eq. (4.4), r = 1/LS); per-row strong count.
// The pass works in the caller's numbering, so every output lands where the
// caller expects it.  Its kernels compute the same thing (the edge shape's
// stage selects one; the autotuner times them): stage 0, k_edge_rows, G
// lanes per row through all steps, on a caller-order copy of a row-permuted
// vector block; stage 1, k_edge_tiles, rows cut into tiles with one thread
// per stored entry for the fits, on the same copy; stage 2, k_edge_rows
// reading the permuted block in place through renumbered column indices
// (no copy; search depth 1); stage 3, k_edge_warp (k_edge_warp.cuh), on the
// same in-place order, gathering every neighbour row once into a per-warp
// shared-memory window and fitting one stored entry per lane.
#pragma once
#include <type_traits>

#include "amgd_internal.cuh"
#include "rowops.cuh"

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

template <class C> __device__ __forceinline__ C divide(C a, C b) { return a / b; }
// the mixed path's coefficient only needs FP32 relative accuracy (its error
// enters LS at second order): the fast division is enough
template <> __device__ __forceinline__ float divide<float>(float a, float b)
{
    return __fdividef(a, b);
}

// sums over one 16-byte piece of (w) x x and (w) y x; FP32 pieces in packed pairs
template <class C, int V, bool UW> struct PieceSums;

template <int V, bool UW> struct PieceSums<double, V, UW> {
    double xx = 0.0, yx = 0.0;
    __device__ __forceinline__ void add(const double (&x)[V], const double (&y)[V], const double (&w)[V]) {
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const double wx = UW ? x[e] : w[e] * x[e];
            xx = fma(wx, x[e], xx);
            yx = fma(wx, y[e], yx);
        }
    }
    __device__ __forceinline__ double sxx() const { return xx; }
    __device__ __forceinline__ double syx() const { return yx; }
};

template <int V, bool UW> struct PieceSums<float, V, UW> {
    float2 xx = make_float2(0.f, 0.f), yx = make_float2(0.f, 0.f);
    __device__ __forceinline__ void add(const float (&x)[V], const float (&y)[V], const float (&w)[V]) {
#pragma unroll
        for (int e = 0; e < V / 2; ++e) {
            float2 x2 = make_float2(x[2 * e], x[2 * e + 1]);
            const float2 wx = UW ? x2 : make_float2(w[2 * e] * x2.x, w[2 * e + 1] * x2.y);
            xx = __ffma2_rn(wx, x2, xx);
            yx = __ffma2_rn(wx, make_float2(y[2 * e], y[2 * e + 1]), yx);
        }
    }
    __device__ __forceinline__ float sxx() const { return xx.x + xx.y; }
    __device__ __forceinline__ float syx() const { return yx.x + yx.y; }
};

// sum over one piece of w (y - a x)^2, each residual one fused multiply-add
template <class C, int V, bool UW>
__device__ __forceinline__ void residual_add(C a, const C (&x)[V], const C (&y)[V], const C (&w)[V], C &res)
{
    if constexpr (std::is_same<C, float>::value) {
        const float2 na = make_float2(-a, -a);
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int e = 0; e < V / 2; ++e) {
            const float2 d = __ffma2_rn(na, make_float2(x[2 * e], x[2 * e + 1]),
                                        make_float2(y[2 * e], y[2 * e + 1]));
            const float2 wd = UW ? d : make_float2(w[2 * e] * d.x, w[2 * e + 1] * d.y);
            acc = __ffma2_rn(wd, d, acc);
        }
        res += acc.x + acc.y;
    } else {
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const C d = fma(-a, x[e], y[e]);
            res = fma(UW ? d : w[e] * d, d, res);
        }
    }
}

// ---------------------------------------------------------------------------
// Compensated FP32 sums (mixed paths, AMGD_SUM_COMPENSATED).  Each sum is two
// FP32 words: a running sum and the exact rounding error of every addition,
// taken by TwoSum (six IEEE additions, no fusion) -- the Kahan-Babuska-
// Neumaier scheme.  S_xx and S_yx travel together as one packed pair; the LS
// terms of even and odd components as the halves of another (FP32x2
// instructions).  Lanes combine their pairs in the shuffle butterfly with
// TwoSum again, adding the error words; the two words are added once at the
// end.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);     // a - b, one rounding
}
// s + e == a + b exactly (Knuth's TwoSum, both halves of the pair)
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &s, float2 &e)
{
    s = __fadd2_rn(a, b);
    const float2 bp = sub2(s, a);
    const float2 ap = sub2(s, bp);
    e = __fadd2_rn(sub2(a, ap), sub2(b, bp));
}
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    const float ap = __fsub_rn(s, bp);
    e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}
struct Comp2 {
    float2 s = make_float2(0.f, 0.f), c = make_float2(0.f, 0.f);
    __device__ __forceinline__ void add(float2 t)
    {
        float2 sn, e;
        two_sum2(s, t, sn, e);
        s = sn;
        c = __fadd2_rn(c, e);
    }
};
// pairs of the G lanes of a row combined (xor butterfly: every lane ends with
// the total)
template <int G>
__device__ __forceinline__ void comp2_allreduce(Comp2 &v, unsigned mask)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        float2 so, co;
        so.x = __shfl_xor_sync(mask, v.s.x, o, G);
        so.y = __shfl_xor_sync(mask, v.s.y, o, G);
        co.x = __shfl_xor_sync(mask, v.c.x, o, G);
        co.y = __shfl_xor_sync(mask, v.c.y, o, G);
        float2 sn, e;
        two_sum2(v.s, so, sn, e);
        v.s = sn;
        v.c = __fadd2_rn(__fadd2_rn(v.c, co), e);
    }
}
// (S_xx, S_yx) of one piece, added to a compensated pair
template <int V, bool UW>
__device__ __forceinline__ void comp_piece_sums(const float (&x)[V], const float (&y)[V],
                                                const float (&w)[V], Comp2 &acc)
{
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const float wx = UW ? x[e] : w[e] * x[e];
        acc.add(__fmul2_rn(make_float2(wx, wx), make_float2(x[e], y[e])));
    }
}
// w (y - a x)^2 of one piece, even and odd components as the pair's halves
template <int V, bool UW>
__device__ __forceinline__ void comp_residual(float a, const float (&x)[V], const float (&y)[V],
                                              const float (&w)[V], Comp2 &acc)
{
    const float2 na = make_float2(-a, -a);
#pragma unroll
    for (int e = 0; e < V; e += 2) {
        const float2 d = __ffma2_rn(na, make_float2(x[e], x[e + 1]), make_float2(y[e], y[e + 1]));
        const float2 wd = UW ? d : make_float2(w[e] * d.x, w[e + 1] * d.y);
        acc.add(__fmul2_rn(wd, d));
    }
}
// the LS pair's two halves joined, then the lanes: one FP32 value
template <int G>
__device__ __forceinline__ float comp_ls_total(const Comp2 &acc, unsigned mask)
{
    float s, e;
    two_sum(acc.s.x, acc.s.y, s, e);
    Comp2 one;
    one.s = make_float2(s, 0.f);
    one.c = make_float2(__fadd_rn(__fadd_rn(acc.c.x, acc.c.y), e), 0.f);
    comp2_allreduce<G>(one, mask);
    return one.s.x + one.c.x;
}

// ---------------------------------------------------------------------------
// Row kernel (edge shape stages 0 and 2).  G lanes own one row through all three
// steps: the target from the row's gathers, then the fits with the row's
// neighbours gathered again (mostly L1/L2 hits), K-component sums reduced
// across the G lanes with shuffles, then the flags.
// Stage 2 (PX): the vectors stay in the sweeps' row order (no caller-order
// copy is made); row i's own vector is read at xrow[i] and the neighbour of
// slot p at xcol[p] -- the caller CSR with every column index mapped to the
// sweeps' numbering -- and the mixed paths may sum with compensation (COMP).
// Per-warp output staging: a warp owns 32/G consecutive rows of the caller's
// numbering, i.e. one contiguous run of CSR slots.  a, LS and the flags of
// that run are collected in shared memory and written out with coalesced
// stores (a run wider than warp_slots<G>() -- 16 slots per row on average --
// is written directly).
template <int G>
constexpr int warp_slots()
{
    return (32 / G) * 16;
}

template <class C, int G>
constexpr int edge_smem_bytes()
{
    return (kEdgeThreads / 32) * warp_slots<G>() * (2 * (int)sizeof(C) + 1);
}

// resident blocks per SM asked of the compiler: three for the plain sums
// (occupancy hides the gathers), two for the compensated ones (their extra
// live words would otherwise spill)
template <bool COMP>
constexpr int edge_rows_min_blocks()
{
    return COMP ? 2 : 3;
}

template <class TS, int G, int NV, int U, bool UW, bool PX, bool COMP>
__global__ void __launch_bounds__(kEdgeThreads, edge_rows_min_blocks<COMP>()) k_edge_rows(EdgeArgs A)
{
    using S = Store<TS>;
    using C = typename S::C;
    using AV = typename S::A;
    constexpr int V = S::V;
    constexpr bool kMixed = !std::is_same<C, double>::value;
    constexpr int kWarpSlots = warp_slots<G>();
    extern __shared__ __align__(16) unsigned char esm[];

    const int lane = threadIdx.x % G, lane32 = threadIdx.x % 32, warp = threadIdx.x / 32;
    const int grp_in_warp = lane32 / G;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (grp_in_warp * G));
    const int64_t r = (int64_t)blockIdx.x * (kEdgeThreads / G) + threadIdx.x / G;
    const int64_t wr0 = (int64_t)blockIdx.x * (kEdgeThreads / G) + (int64_t)warp * (32 / G);
    if (wr0 >= A.n) return;                      // whole warp past the end
    const bool active = r < A.n;

    C *a_s = reinterpret_cast<C *>(esm) + (size_t)warp * kWarpSlots;
    C *ls_s = reinterpret_cast<C *>(esm) + (size_t)(kEdgeThreads / 32) * kWarpSlots + (size_t)warp * kWarpSlots;
    uint8_t *fl_s = esm + (size_t)(kEdgeThreads / 32) * kWarpSlots * 2 * sizeof(C) + (size_t)warp * kWarpSlots;

    const int32_t *__restrict__ col = A.col;
    const int32_t *__restrict__ xcol = PX ? A.xcol : A.col;   // gather index of each slot
    const AV *__restrict__ val = (const AV *)A.val;
    const TS *__restrict__ X = (const TS *)A.x;
    const int Kp = A.Kp;
    const int64_t wr1 = min((int64_t)A.n, wr0 + 32 / G);
    const int wbase = __ldg(A.prp + wr0), wend = __ldg(A.prp + wr1);
    const bool staged = wend - wbase <= kWarpSlots;
    C *a_out = (C *)A.a_out;
    C *ls_out = (C *)A.ls_out;

    C w[NV][V];
    if constexpr (!UW) {
#pragma unroll
        for (int t = 0; t < NV; ++t)
#pragma unroll
            for (int e = 0; e < V; ++e) w[t][e] = ((const C *)A.w)[piece_of<G, NV>(lane, t) * V + e];
    }

    int q0 = 0, q1 = 0;       // the row's entries in the pattern of the fits
    C m = C(INFINITY), diag = C(1);
    bool defer = false;       // a fit of this row cancelled in FP32: redo the row in FP64
    if (active) {
        const int p0 = __ldg(A.rp + r), p1 = __ldg(A.rp + r + 1);
        q0 = __ldg(A.prp + r);
        q1 = __ldg(A.prp + r + 1);
        diag = (C)__ldg((const AV *)A.diag + r);

        // ---- 1. target --------------------------------------------------
        C y[NV][V];
        {
            Acc<C, V> acc[NV];
            row_sum<TS, G, NV, U, false>(xcol, val, X, X, 0, Kp, lane, p0, p1, acc, A.n, A.status);
            const C d = C(1) / diag;
            const int64_t xr = (PX && A.xrow) ? checked_row(__ldg(A.xrow + r), A.n, A.status) : r;
#pragma unroll
            for (int t = 0; t < NV; ++t) {
                S::unpack(ldg16(X + xr * Kp + piece_of<G, NV>(lane, t) * V), y[t]);     // x_i
                if (A.target == 0) {
#pragma unroll
                    for (int e = 0; e < V; ++e) y[t][e] = fma(-d, acc[t].get(e), y[t][e]);
                }
            }
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
        // a residual-target row of A with one off-diagonal j1: y_i is exactly
        // -(a_ij1 / a_ii) x_j1
        int j1 = -1;
        C v1 = C(0);
        if (A.target == 0 && p1 - p0 == 2) {
            const int pj = __ldg(col + p0) == r ? p0 + 1 : p0;
            j1 = __ldg(col + pj);
            v1 = (C)__ldg(val + pj);
        }

        // ---- 2. one-point LS per off-diagonal -----------------------------
        for (int pb = q0; pb < q1; pb += U) {
            int jj[U];
#pragma unroll
            for (int u = 0; u < U; ++u) jj[u] = (pb + u < q1) ? __ldg(A.pcol + pb + u) : -1;
            uint4 raw[U][NV];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (jj[u] >= 0 && jj[u] != r) {
                    const int64_t xj = checked_row(PX ? (int64_t)__ldg(xcol + pb + u) : (int64_t)jj[u],
                                                   A.n, A.status);
                    if constexpr (NV % 2 == 0) {                 // side-by-side pieces: 32-byte pairs
#pragma unroll
                        for (int t = 0; t < NV; t += 2)
                            ldg32(X + xj * Kp + piece_of<G, NV>(lane, t) * V, raw[u][t], raw[u][t + 1]);
                    } else {
#pragma unroll
                        for (int t = 0; t < NV; ++t)
                            raw[u][t] = ldg16(X + xj * Kp + piece_of<G, NV>(lane, t) * V);
                    }
                }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (jj[u] < 0) break;
                const int p = pb + u;
                C a_, ls_;
                if (jj[u] == r) {
                    a_ = C(0);
                    ls_ = C(NAN);
                } else if (jj[u] == j1) {
                    a_ = -v1 / diag;
                    ls_ = C(0);
                } else if constexpr (COMP && kMixed) {
                    Comp2 sx;
#pragma unroll
                    for (int t = 0; t < NV; ++t) {
                        C xj[V];
                        S::unpack(raw[u][t], xj);
                        comp_piece_sums<V, UW>(xj, y[t], w[t], sx);
                    }
                    comp2_allreduce<G>(sx, gmask);
                    const C sxx = sx.s.x + sx.c.x, syx = sx.s.y + sx.c.y;
                    a_ = (sxx == C(0)) ? C(0) : divide(syx, sxx);
                    Comp2 sl;
#pragma unroll
                    for (int t = 0; t < NV; ++t) {
                        C xj[V];
                        S::unpack(raw[u][t], xj);
                        comp_residual<V, UW>(a_, xj, y[t], w[t], sl);
                    }
                    ls_ = comp_ls_total<G>(sl, gmask);
                    defer = defer || ls_ < C(1e-4) * syy;
                } else {
                    // x_j is unpacked from the gathered bits once per use, so only one
                    // 16-byte piece of it is live in registers at a time
                    PieceSums<C, V, UW> ps;
#pragma unroll
                    for (int t = 0; t < NV; ++t) {
                        C xj[V];
                        S::unpack(raw[u][t], xj);
                        ps.add(xj, y[t], w[t]);
                    }
                    const C sxx = group_sum<G>(ps.sxx(), gmask);
                    const C syx = group_sum<G>(ps.syx(), gmask);
                    a_ = (sxx == C(0)) ? C(0) : divide(syx, sxx);
                    C res = C(0);
#pragma unroll
                    for (int t = 0; t < NV; ++t) {
                        C xj[V];
                        S::unpack(raw[u][t], xj);
                        residual_add<C, V, UW>(a_, xj, y[t], w[t], res);
                    }
                    ls_ = group_sum<G>(res, gmask);
                    if constexpr (kMixed) defer = defer || ls_ < C(1e-4) * syy;
                }
                if (jj[u] != r) m = fmin(m, ls_);
                if (lane == 0) {
                    if (staged) { a_s[p - wbase] = a_; ls_s[p - wbase] = ls_; }
                    else { a_out[p] = a_; ls_out[p] = ls_; }
                }
            }
        }
    }
    __syncwarp();

    // ---- 3. strength flags (from the LS values just produced) ----------------
    const C theta = (C)A.theta;
    int cnt = 0;
    if (active) {
        for (int p = q0 + lane; p < q1; p += G) {
            const int j = __ldg(A.pcol + p);
            const C l = staged ? ls_s[p - wbase] : ls_out[p];
            const int strong = (j != r) && (l == C(0) || theta * l < m);
            if (staged) fl_s[p - wbase] = (uint8_t)strong;
            else A.flag_out[p] = (uint8_t)strong;
            cnt += strong;
        }
        cnt = group_sum<G>(cnt, gmask);
        if (lane == 0) A.count_out[r] = cnt;
        if (kMixed && defer && lane == 0) A.defer_list[atomicAdd(A.defer_count, 1u)] = (int32_t)r;
    }
    __syncwarp();

    // ---- coalesced write-out of the warp's slot run --------------------------
    if (staged) {
        for (int q = lane32; q < wend - wbase; q += 32) {
            a_out[wbase + q] = a_s[q];
            ls_out[wbase + q] = ls_s[q];
            A.flag_out[wbase + q] = fl_s[q];
        }
    }
}

// ---------------------------------------------------------------------------
// Tile kernel (edge shape stage 1).  A block owns one tile of consecutive caller rows (at most
// kEdgeTileRows rows and kEdgeTileSlots stored entries; a longer row is a
// tile of its own), i.e. one contiguous run of CSR slots:
//   A. targets: G lanes per row form y_i (the same row sums and rounding as
//      the sweeps) into shared memory, plus S_yy per row on the mixed paths;
//   B. fits: one thread per stored entry gathers x_j once, reads y_i from
//      shared memory and forms S_xx, S_yx, a_ij and the residual sum LS_ij
//      over all K components itself -- no cross-lane reductions, whole-warp
//      use for the per-edge scalar work, coalesced a/LS writes; the row
//      minimum of LS is an atomic minimum on the (non-negative) bit patterns
//      in shared memory, which is order independent;
//   C. flags and per-row counts from the row minima.
// ---------------------------------------------------------------------------
template <class C> struct MinBits;
template <> struct MinBits<float> {
    using T = unsigned int;
    static constexpr T kInf = 0x7f800000u;
    __device__ __forceinline__ static T bits(float v) { return __float_as_uint(v); }
    __device__ __forceinline__ static float value(T b) { return __uint_as_float(b); }
};
template <> struct MinBits<double> {
    using T = unsigned long long;
    static constexpr T kInf = 0x7ff0000000000000ull;
    __device__ __forceinline__ static T bits(double v) { return (T)__double_as_longlong(v); }
    __device__ __forceinline__ static double value(T b) { return __longlong_as_double((long long)b); }
};

// shared-memory layout of one tile
template <class TS, int KP>
struct EdgeTileLayout {
    using C = typename Store<TS>::C;
    using M = typename MinBits<C>::T;
    static constexpr int TR = kEdgeTileRows;
    static constexpr int YS = 0;                                        // TR x KP targets
    static constexpr int DG = YS + TR * KP * (int)sizeof(C);            // TR diagonals
    static constexpr int SY = DG + TR * (int)sizeof(C);                 // TR S_yy
    static constexpr int MN = (SY + TR * (int)sizeof(C) + 7) & ~7;      // TR row minima (bits)
    static constexpr int RP = MN + TR * (int)sizeof(M);                 // TR + 1 slot offsets
    static constexpr int CN = RP + (TR + 1) * 4;                        // TR strong counts
    static constexpr int DF = CN + TR * 4;                              // TR defer marks
    static constexpr int J1 = DF + TR * 4;                              // TR exact-rule neighbours
    static constexpr int V1 = (J1 + TR * 4 + 7) & ~7;                   // TR their values a_ij1
    static constexpr int SR = V1 + TR * (int)sizeof(C);                 // slot -> local row (u8)
    static constexpr int BYTES = SR + kEdgeTileSlots;
};

template <class TS, int G, int NV, int U, bool UW, bool COMP>
__global__ void __launch_bounds__(kEdgeThreads) k_edge_tiles(EdgeArgs A)
{
    using S = Store<TS>;
    using C = typename S::C;
    using AV = typename S::A;
    using MB = MinBits<C>;
    constexpr int V = S::V;
    constexpr int P = G * NV;           // 16-byte pieces per row
    constexpr int KP = P * V;           // padded components per row
    using L = EdgeTileLayout<TS, KP>;
    constexpr bool kMixed = !std::is_same<C, double>::value;
    constexpr int HOLD = P <= 4 ? P : 1;     // pieces of x_j kept in registers between the sums
    extern __shared__ __align__(16) unsigned char esm[];
    C *ys = reinterpret_cast<C *>(esm + L::YS);
    C *dg = reinterpret_cast<C *>(esm + L::DG);
    C *syy = reinterpret_cast<C *>(esm + L::SY);
    typename MB::T *rmin = reinterpret_cast<typename MB::T *>(esm + L::MN);
    int32_t *rps = reinterpret_cast<int32_t *>(esm + L::RP);
    int32_t *cnt = reinterpret_cast<int32_t *>(esm + L::CN);
    int32_t *dfr = reinterpret_cast<int32_t *>(esm + L::DF);
    int32_t *j1s = reinterpret_cast<int32_t *>(esm + L::J1);
    C *v1s = reinterpret_cast<C *>(esm + L::V1);
    uint8_t *srow = esm + L::SR;

    const int32_t R0 = __ldg(A.tiles + blockIdx.x), R1 = __ldg(A.tiles + blockIdx.x + 1);
    const int nr = R1 - R0;
    const bool single = nr == 1;                 // possibly longer than kEdgeTileSlots
    const int32_t *__restrict__ col = A.col;
    const AV *__restrict__ val = (const AV *)A.val;
    const TS *__restrict__ X = (const TS *)A.x;
    const C *__restrict__ wv = (const C *)A.w;

    for (int q = threadIdx.x; q <= nr; q += kEdgeThreads) rps[q] = __ldg(A.prp + R0 + q);
    for (int q = threadIdx.x; q < nr; q += kEdgeThreads) {
        dg[q] = (C)__ldg((const AV *)A.diag + R0 + q);
        rmin[q] = MB::kInf;
        cnt[q] = 0;
        dfr[q] = 0;
    }
    __syncthreads();
    const int S0 = rps[0], S1 = rps[nr];

    // ---- A. targets -----------------------------------------------------------
    {
        const int lane = threadIdx.x % G;
        const unsigned gmask = (G == 32) ? 0xffffffffu
                                         : (((1u << G) - 1u) << ((threadIdx.x % 32) / G * G));
        for (int rl = threadIdx.x / G; rl < nr; rl += kEdgeThreads / G) {
            const int64_t r = R0 + rl;
            if (!single)
                for (int q = rps[rl] + lane; q < rps[rl + 1]; q += G) srow[q - S0] = (uint8_t)rl;
            const int p0 = __ldg(A.rp + r), p1 = __ldg(A.rp + r + 1);   // row of A
            if (lane == 0) {
                // a residual-target row of A with one off-diagonal j1: y_i is
                // exactly -(a_ij1 / a_ii) x_j1
                int j1 = -1;
                C v1 = C(0);
                if (A.target == 0 && p1 - p0 == 2) {
                    const int pj = __ldg(col + p0) == r ? p0 + 1 : p0;
                    j1 = __ldg(col + pj);
                    v1 = (C)__ldg(val + pj);
                }
                j1s[rl] = j1;
                v1s[rl] = v1;
            }
            C y[NV][V];
#pragma unroll
            for (int t = 0; t < NV; ++t) S::unpack(ldg16(X + r * KP + piece_of<G, NV>(lane, t) * V), y[t]);
            if (A.target == 0) {
                Acc<C, V> acc[NV];
                row_sum<TS, G, NV, U, false>(col, val, X, X, 0, KP, lane, p0, p1, acc, A.n, A.status);
                const C d = C(1) / dg[rl];
#pragma unroll
                for (int t = 0; t < NV; ++t)
#pragma unroll
                    for (int e = 0; e < V; ++e) y[t][e] = fma(-d, acc[t].get(e), y[t][e]);
            }
            C s = C(0);
#pragma unroll
            for (int t = 0; t < NV; ++t) {
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    ys[rl * KP + piece_of<G, NV>(lane, t) * V + e] = y[t][e];
                    if constexpr (kMixed)
                        s = fma(UW ? y[t][e] : wv[piece_of<G, NV>(lane, t) * V + e] * y[t][e], y[t][e], s);
                }
            }
            if constexpr (kMixed) {
                s = group_sum<G>(s, gmask);
                if (lane == 0) syy[rl] = s;
            }
        }
    }
    __syncthreads();

    // ---- B. one-point fits, one stored entry per thread -------------------------
    // one entry of a thread at a time (two in flight, their x_j gathered together,
    // measured slower: the registers cost more occupancy than the overlap gains)
    constexpr int E = 1;
    C *a_out = (C *)A.a_out;
    C *ls_out = (C *)A.ls_out;
    // the fit of slot p (row rl, column j) from the pieces `hold` of x_j
    auto fit = [&](int rl, int j, const uint4 (&hold)[HOLD], C &a_, C &ls_) {
        const TS *xj = X + checked_row(j, A.n, A.status) * KP;
        const C *yr = ys + rl * KP;
        if constexpr (COMP && kMixed) {
            // compensated sums over all K components in this thread
            Comp2 sx;
#pragma unroll
            for (int c = 0; c < P; ++c) {
                const uint4 raw = (P <= 4) ? hold[c < HOLD ? c : 0] : ldg16(xj + c * V);
                C x[V], y[V], w[V];
                S::unpack(raw, x);
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    y[e] = yr[c * V + e];
                    w[e] = UW ? C(1) : wv[c * V + e];
                }
                comp_piece_sums<V, UW>(x, y, w, sx);
            }
            const C sxx = sx.s.x + sx.c.x, syx = sx.s.y + sx.c.y;
            a_ = (sxx == C(0)) ? C(0) : divide(syx, sxx);
            Comp2 sl;
#pragma unroll
            for (int c = 0; c < P; ++c) {
                const uint4 raw = (P <= 4) ? hold[c < HOLD ? c : 0] : ldg16(xj + c * V);
                C x[V], y[V], w[V];
                S::unpack(raw, x);
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    y[e] = yr[c * V + e];
                    w[e] = UW ? C(1) : wv[c * V + e];
                }
                comp_residual<V, UW>(a_, x, y, w, sl);
            }
            ls_ = comp_ls_total<1>(sl, 0xffffffffu);
        } else {
            PieceSums<C, V, UW> ps;
#pragma unroll
            for (int c = 0; c < P; ++c) {
                const uint4 raw = (P <= 4) ? hold[c < HOLD ? c : 0] : ldg16(xj + c * V);
                C x[V], y[V], w[V];
                S::unpack(raw, x);
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    y[e] = yr[c * V + e];
                    w[e] = UW ? C(1) : wv[c * V + e];
                }
                ps.add(x, y, w);
            }
            const C sxx = ps.sxx(), syx = ps.syx();
            a_ = (sxx == C(0)) ? C(0) : divide(syx, sxx);
            C res = C(0);
#pragma unroll
            for (int c = 0; c < P; ++c) {
                const uint4 raw = (P <= 4) ? hold[c < HOLD ? c : 0] : ldg16(xj + c * V);
                C x[V], y[V], w[V];
                S::unpack(raw, x);
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    y[e] = yr[c * V + e];
                    w[e] = UW ? C(1) : wv[c * V + e];
                }
                residual_add<C, V, UW>(a_, x, y, w, res);
            }
            ls_ = res;
        }
    };
    for (int pb = S0 + threadIdx.x; pb < S1; pb += E * kEdgeThreads) {
        int rls[E], js[E];
        uint4 hold[E][HOLD];
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const int p = pb + q * kEdgeThreads;
            js[q] = -1;
            if (p < S1) {
                rls[q] = single ? 0 : srow[p - S0];
                js[q] = __ldg(A.pcol + p);
                if (P <= 4 && js[q] != R0 + rls[q] && js[q] != j1s[rls[q]]) {
                    const TS *xj = X + checked_row(js[q], A.n, A.status) * KP;
                    if constexpr (HOLD % 2 == 0) {                  // 32-byte pairs
#pragma unroll
                        for (int c = 0; c < HOLD; c += 2) ldg32(xj + c * V, hold[q][c], hold[q][c + 1]);
                    } else {
#pragma unroll
                        for (int c = 0; c < HOLD; ++c) hold[q][c] = ldg16(xj + c * V);
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < E; ++q) {
            if (js[q] < 0) break;
            const int p = pb + q * kEdgeThreads;
            const int rl = rls[q], j = js[q];
            const int64_t r = R0 + rl;
            C a_, ls_;
            if (j == r) {
                a_ = C(0);
                ls_ = C(NAN);
            } else if (j == j1s[rl]) {
                a_ = -v1s[rl] / dg[rl];                 // y_i = -(a_ij/a_ii) x_j exactly
                ls_ = C(0);
            } else {
                fit(rl, j, hold[q], a_, ls_);
                if constexpr (kMixed)
                    if (ls_ < C(1e-4) * syy[rl]) dfr[rl] = 1;    // cancellation: redo the row in FP64
            }
            a_out[p] = a_;
            ls_out[p] = ls_;
            if (j != r) atomicMin(&rmin[rl], MB::bits(ls_));
        }
    }
    __syncthreads();

    // ---- C. strength flags (Eq. (4.4) in LS form) and counts -------------------
    const C theta = (C)A.theta;
    for (int p = S0 + threadIdx.x; p < S1; p += kEdgeThreads) {
        const int rl = single ? 0 : srow[p - S0];
        const C l = ls_out[p];                       // written by this block in B; NaN on the diagonal
        const C m = MB::value(rmin[rl]);
        const int strong = l == C(0) || theta * l < m;   // false for the diagonal's NaN
        A.flag_out[p] = (uint8_t)strong;
        if (strong) atomicAdd(&cnt[rl], 1);
    }
    __syncthreads();
    for (int rl = threadIdx.x; rl < nr; rl += kEdgeThreads) {
        A.count_out[R0 + rl] = cnt[rl];
        if (kMixed && dfr[rl]) A.defer_list[atomicAdd(A.defer_count, 1u)] = R0 + rl;
    }
}

// Mixed paths: rows listed by k_edge (a fit cancelled in FP32, LS < 1e-4 S_yy)
// are recomputed here entirely in FP64 from the stored vectors (widened
// exactly) and the FP64 values of A: target with the FP64 path's rounding,
// every one-point fit, the row minimum, flags and count.  One warp per row,
// lanes over the K components (K <= 64: two per lane).
template <class TS>
__device__ __forceinline__ double elem64(const TS *p)
{
    if constexpr (std::is_same<TS, __nv_bfloat16>::value)
        return (double)__bfloat162float(*p);
    else
        return (double)*p;
}

template <class TS, bool PX>
__global__ void __launch_bounds__(256) k_edge_fixup(EdgeArgs A)
{
    using C = typename Store<TS>::C;
    const unsigned count = *A.defer_count;
    const int lane = threadIdx.x % 32;
    const TS *X = (const TS *)A.x;
    const int Kp = A.Kp;
    // vector row of caller row i and of the neighbour of slot p (stage 2: the
    // sweeps' row order; search depth 1, so the fit slots are A's slots)
    auto xrow = [&](int64_t i) -> int64_t { return (PX && A.xrow) ? checked_row(A.xrow[i], A.n, A.status) : i; };
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t q = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; q < count; q += warps) {
        const int64_t r = A.defer_list[q];
        const int p0 = A.rp[r], p1 = A.rp[r + 1];         // row of A: target
        const int q0 = A.prp[r], q1 = A.prp[r + 1];       // entries of the fits
        double diag = 1.0;
        int j1 = -1;
        double v1 = 0.0;
        for (int p = p0; p < p1; ++p) {
            if (A.col[p] == r) diag = A.val64[p];
            else if (A.target == 0 && p1 - p0 == 2) { j1 = A.col[p]; v1 = A.val64[p]; }
        }
        const double d = 1.0 / diag;
        double y[2], w[2];
        for (int h = 0; h < 2; ++h) {
            const int k = lane + 32 * h;
            w[h] = k < Kp ? A.w64[k] : 0.0;
            double acc = 0.0;
            const double xi = k < Kp ? elem64(X + xrow(r) * Kp + k) : 0.0;
            if (k < Kp)
                for (int p = p0; p < p1; ++p)
                    acc = fma(A.val64[p], elem64(X + checked_row(PX ? A.xcol[p] : A.col[p], A.n, A.status) * Kp + k), acc);
            y[h] = (A.target == 0) ? fma(-d, acc, xi) : xi;
        }
        double m = INFINITY;
        C *a_out = (C *)A.a_out;
        C *ls_out = (C *)A.ls_out;
        for (int p = q0; p < q1; ++p) {
            const int64_t j = A.pcol[p];
            double a64, ls64;
            if (j == r) {
                a64 = 0.0;
                ls64 = NAN;
            } else if (j == j1) {
                a64 = -v1 / diag;
                ls64 = 0.0;
            } else {
                double xj[2], sxx = 0.0, syx = 0.0;
                const int64_t xjr = checked_row(PX ? (int64_t)A.xcol[p] : j, A.n, A.status);
                for (int h = 0; h < 2; ++h) {
                    const int k = lane + 32 * h;
                    xj[h] = k < Kp ? elem64(X + xjr * Kp + k) : 0.0;
                    sxx = fma(w[h] * xj[h], xj[h], sxx);
                    syx = fma(w[h] * xj[h], y[h], syx);
                }
                for (int o = 16; o > 0; o >>= 1) {
                    sxx += __shfl_xor_sync(0xffffffffu, sxx, o);
                    syx += __shfl_xor_sync(0xffffffffu, syx, o);
                }
                a64 = (sxx == 0.0) ? 0.0 : syx / sxx;
                double res = 0.0;
                for (int h = 0; h < 2; ++h) {
                    const double e = fma(-a64, xj[h], y[h]);
                    res = fma(w[h] * e, e, res);
                }
                for (int o = 16; o > 0; o >>= 1) res += __shfl_xor_sync(0xffffffffu, res, o);
                ls64 = res;
            }
            if (j != r) m = fmin(m, ls64);
            if (lane == 0) {
                a_out[p] = (C)a64;
                ls_out[p] = (C)ls64;
            }
        }
        __syncwarp();
        int cnt = 0;
        for (int p = q0 + lane; p < q1; p += 32) {
            const double l = (double)ls_out[p];
            const int strong = (A.pcol[p] != r) && (l == 0.0 || A.theta * l < m);
            A.flag_out[p] = (uint8_t)strong;
            cnt += strong;
        }
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0) A.count_out[r] = cnt;
        __syncwarp();
    }
}

template <class TS, int G, int NV, int U, bool UW, bool PX, bool COMP>
cudaError_t go_rows(const EdgeArgs &a, cudaStream_t s)
{
    if constexpr (NV % 2 == 0)
        if (!rows_aligned32(a.x, a.Kp, sizeof(TS))) return cudaErrorMisalignedAddress;
    const int rows_per_block = kEdgeThreads / G;
    const unsigned grid = (unsigned)(((int64_t)a.n + rows_per_block - 1) / rows_per_block);
    constexpr int smem = edge_smem_bytes<typename Store<TS>::C, G>();
    static PerDevice opted;                  // shared-memory opt-in made on each device
    const int dev = current_device_index();
    if (smem > 48 * 1024 && opted.get(dev) == 0) {
        const cudaError_t e = cudaFuncSetAttribute(k_edge_rows<TS, G, NV, U, UW, PX, COMP>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        opted.set(dev, 1);
    }
    k_edge_rows<TS, G, NV, U, UW, PX, COMP><<<grid, kEdgeThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <class TS, int G, int NV, int U, bool UW, bool COMP>
cudaError_t go_tiles(const EdgeArgs &a, cudaStream_t s)
{
    constexpr int KP = G * NV * Store<TS>::V;
    if (a.Kp != KP || a.ntiles <= 0) return cudaErrorInvalidValue;
    if constexpr ((G * NV) % 2 == 0)          // 32-byte row reads (row sums at G = 1, fits)
        if (!rows_aligned32(a.x, a.Kp, sizeof(TS))) return cudaErrorMisalignedAddress;
    constexpr int smem = EdgeTileLayout<TS, KP>::BYTES;
    static PerDevice opted;                  // shared-memory opt-in made on each device
    const int dev = current_device_index();
    if (smem > 48 * 1024 && opted.get(dev) == 0) {
        const cudaError_t e = cudaFuncSetAttribute(k_edge_tiles<TS, G, NV, U, UW, COMP>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        opted.set(dev, 1);
    }
    k_edge_tiles<TS, G, NV, U, UW, COMP><<<(unsigned)a.ntiles, kEdgeThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace edge_impl
}  // namespace amgd

#include "k_edge_warp.cuh"

namespace amgd {
namespace edge_impl {

// one storage type and summation form; the plain and the compensated forms
// are instantiated in separate translation units (parallel compilation)
template <class TS, bool COMP, int G, int NV, int U, bool UW>
cudaError_t go(int stage, const EdgeArgs &a, cudaStream_t s)
{
    if (a.n <= 0) return cudaSuccess;
    if (stage == 1) return go_tiles<TS, G, NV, U, UW, COMP>(a, s);
    if (stage == 2) return go_rows<TS, G, NV, U, UW, true, COMP>(a, s);
    if (stage == 3) {
        if constexpr (U >= 4) return go_warp<TS, G, NV, U, UW, COMP>(a, s);
        return cudaErrorInvalidValue;
    }
    return go_rows<TS, G, NV, U, UW, false, COMP>(a, s);
}

template <class TS, bool COMP, int G, int NV, bool UW>
cudaError_t dispatch_u(int stage, int U, const EdgeArgs &a, cudaStream_t s)
{
    switch (U) {
    case 2: return go<TS, COMP, G, NV, 2, UW>(stage, a, s);
    case 4: return go<TS, COMP, G, NV, 4, UW>(stage, a, s);
    case 8: return go<TS, COMP, G, NV, 8, UW>(stage, a, s);
    }
    return cudaErrorInvalidValue;
}

template <class TS, bool COMP, int G, int NV>
cudaError_t dispatch_w(int stage, int U, bool unit_w, const EdgeArgs &a, cudaStream_t s)
{
    return unit_w ? dispatch_u<TS, COMP, G, NV, true>(stage, U, a, s)
                  : dispatch_u<TS, COMP, G, NV, false>(stage, U, a, s);
}

template <class TS, bool COMP, int G>
cudaError_t dispatch_nv(int stage, int NV, int U, bool unit_w, const EdgeArgs &a, cudaStream_t s)
{
    constexpr int V = Store<TS>::V;
    switch (NV) {
    case 1: return dispatch_w<TS, COMP, G, 1>(stage, U, unit_w, a, s);
    case 2: if constexpr (G * 2 * V <= 64) return dispatch_w<TS, COMP, G, 2>(stage, U, unit_w, a, s); break;
    case 4: if constexpr (G * 4 * V <= 64) return dispatch_w<TS, COMP, G, 4>(stage, U, unit_w, a, s); break;
    }
    return cudaErrorInvalidValue;
}

template <class TS, bool COMP>
cudaError_t dispatch_g(Shape sh, bool unit_w, const EdgeArgs &a, cudaStream_t s)
{
    constexpr int V = Store<TS>::V;
    switch (sh.G) {
    case 1: return dispatch_nv<TS, COMP, 1>(sh.stage, sh.NV, sh.U, unit_w, a, s);
    case 2: return dispatch_nv<TS, COMP, 2>(sh.stage, sh.NV, sh.U, unit_w, a, s);
    case 4: return dispatch_nv<TS, COMP, 4>(sh.stage, sh.NV, sh.U, unit_w, a, s);
    case 8: if constexpr (8 * V <= 64) return dispatch_nv<TS, COMP, 8>(sh.stage, sh.NV, sh.U, unit_w, a, s); break;
    case 16: if constexpr (16 * V <= 64) return dispatch_nv<TS, COMP, 16>(sh.stage, sh.NV, sh.U, unit_w, a, s); break;
    case 32: if constexpr (32 * V <= 64) return dispatch_nv<TS, COMP, 32>(sh.stage, sh.NV, sh.U, unit_w, a, s); break;
    }
    return cudaErrorInvalidValue;
}

}  // namespace edge_impl
}  // namespace amgd
