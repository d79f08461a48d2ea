// k_edge_warp.cuh -- warp-staged distance kernel (edge shape stage 3, search
// depth 1): the same three steps as k_edge_rows (target, one-point fits,
// threshold; §4.1 Eq. (4.3), §4.2 Eq. (4.4)), on the sweeps' row order read
// in place, with the neighbour rows gathered ONCE.
//
// A warp owns R = 32/G consecutive caller rows (one contiguous run of CSR
// slots) and walks them in three steps:
//   1. targets, G lanes per row: every stored entry's vector row is gathered
//      (16-byte pieces spread over the row's G lanes -- side by side and moved
//      two per 32-byte access when a lane holds an even number -- so one warp
//      load covers whole rows),
//      folded into the row sum with the sweeps' rounding, and parked in the
//      warp's shared-memory window, slot by slot;
//   2. fits, one lane per stored entry: x_j and y_i are read back from shared
//      memory and S_xx, S_yx, a_ij and the residual sum LS_ij are formed over
//      all K components inside the lane -- no cross-lane reductions, so the
//      compensated sums cost only their own arithmetic; a and LS leave with
//      coalesced stores;
//   3. row minimum, flags and counts, G lanes per row again.
// A warp whose run holds more than kWarpSlotsPerRow * R entries (long rows)
// skips the window: its fits gather x_j from global memory instead.
//
// A plain fit computes the same operations in the same order as k_edge_rows
// with G = 1 (pieces in order, components in order); a compensated fit keeps
// S_xx and S_yx as two compensated pairs over even and odd components, which
// changes only the rounding of the compensated sums.
#pragma once
#include <type_traits>

namespace amgd {
namespace edge_impl {

constexpr int kWarpEdgeWarps = 4;              // warps per block
constexpr int kWarpEdgeThreads = 32 * kWarpEdgeWarps;
constexpr int kWarpSlotsPerRow = 12;           // window capacity, entries per row on average

// shared-memory layout of one warp's window (bytes)
template <class TS, int G, int NV>
struct WarpEdgeLayout {
    using C = typename Store<TS>::C;
    static constexpr int P = G * NV;                         // 16-byte pieces per row
    static constexpr int V = Store<TS>::V;
    static constexpr int KP = P * V;
    static constexpr int R = 32 / G;                         // rows per warp
    static constexpr int CAP = kWarpSlotsPerRow * R;         // parked entries
    static constexpr int YST = KP + 16 / (int)sizeof(C);     // target row stride (padded: no bank conflicts)
    static constexpr int XS = 0;                             // CAP x P pieces (swizzled)
    static constexpr int YS = XS + CAP * P * 16;             // R targets
    static constexpr int LS = YS + R * YST * (int)sizeof(C); // CAP LS values
    static constexpr int SY = LS + CAP * (int)sizeof(C);     // R S_yy
    static constexpr int DG = SY + R * (int)sizeof(C);       // R diagonals
    static constexpr int V1 = DG + R * (int)sizeof(C);       // R values a_ij1
    static constexpr int RS = V1 + R * (int)sizeof(C);       // R + 1 slot offsets
    static constexpr int J1 = RS + (R + 1) * 4;              // R exact-rule neighbours
    static constexpr int DF = J1 + R * 4;                    // R defer marks
    static constexpr int SR = DF + R * 4;                    // CAP slot -> row (u8)
    static constexpr int BYTES = (SR + CAP + 15) & ~15;
    // the block: kWarpEdgeWarps windows, then the LS weights (non-unit weights)
    static constexpr int block_bytes(bool unit_w)
    {
        return kWarpEdgeWarps * BYTES + (unit_w ? 0 : KP * (int)sizeof(C));
    }
};

// piece c of parked slot s: the pieces of eight consecutive slots land in
// eight different 16-byte bank groups (conflict-free reads, one lane per slot)
template <int P>
__device__ __forceinline__ int park_index(int s, int c)
{
    if constexpr (P >= 8)
        return s * P + (c ^ (s & 7));
    else
        return s * P + (c ^ ((s / (8 / P)) & (P - 1)));
}

// 16-byte pieces of an arithmetic-type row in shared memory
template <class C, int V>
__device__ __forceinline__ void st_piece(C *dst, const C (&x)[V])
{
    if constexpr (std::is_same<C, double>::value) {
        static_assert(V == 2, "FP64 piece");
        *reinterpret_cast<double2 *>(dst) = make_double2(x[0], x[1]);
    } else {
#pragma unroll
        for (int e = 0; e < V; e += 4)
            *reinterpret_cast<float4 *>(dst + e) = make_float4(x[e], x[e + 1], x[e + 2], x[e + 3]);
    }
}
template <class C, int V>
__device__ __forceinline__ void ld_piece(const C *src, C (&x)[V])
{
    if constexpr (std::is_same<C, double>::value) {
        const double2 v = *reinterpret_cast<const double2 *>(src);
        x[0] = v.x;
        x[1] = v.y;
    } else {
#pragma unroll
        for (int e = 0; e < V; e += 4) {
            const float4 v = *reinterpret_cast<const float4 *>(src + e);
            x[e] = v.x;
            x[e + 1] = v.y;
            x[e + 2] = v.z;
            x[e + 3] = v.w;
        }
    }
}

template <int G, class T>
__device__ __forceinline__ T group_min(T v, unsigned mask)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(mask, v, o, G));
    return v;
}

template <class TS, int G, int NV, int U, bool UW, bool COMP>
__global__ void __launch_bounds__(kWarpEdgeThreads) k_edge_warp(EdgeArgs A)
{
    using S = Store<TS>;
    using C = typename S::C;
    using AV = typename S::A;
    using L = WarpEdgeLayout<TS, G, NV>;
    constexpr int V = S::V;
    constexpr int P = L::P;
    constexpr int KP = L::KP;
    constexpr int R = L::R;
    constexpr bool kMixed = !std::is_same<C, double>::value;
    constexpr int HOLD = P <= 4 ? P : 1;     // pieces of x_j kept in registers between the sums
    extern __shared__ __align__(16) unsigned char esm[];

    // LS weights of the block (non-unit weights), before any warp leaves
    C *wv = reinterpret_cast<C *>(esm + kWarpEdgeWarps * L::BYTES);
    if constexpr (!UW) {
        for (int k = threadIdx.x; k < KP; k += kWarpEdgeThreads) wv[k] = ((const C *)A.w)[k];
        __syncthreads();
    }

    const int warp = threadIdx.x / 32, lane32 = threadIdx.x % 32;
    const int rw = lane32 / G, lane = lane32 % G;
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (rw * G));
    const int64_t r0 = ((int64_t)blockIdx.x * kWarpEdgeWarps + warp) * R;
    if (r0 >= A.n) return;                     // whole warp past the end
    const int64_t r = r0 + rw;
    const bool active = r < A.n;

    unsigned char *wb = esm + warp * L::BYTES;
    uint4 *xs = reinterpret_cast<uint4 *>(wb + L::XS);
    C *ys = reinterpret_cast<C *>(wb + L::YS);
    C *lss = reinterpret_cast<C *>(wb + L::LS);
    C *syy_s = reinterpret_cast<C *>(wb + L::SY);
    C *dg_s = reinterpret_cast<C *>(wb + L::DG);
    C *v1_s = reinterpret_cast<C *>(wb + L::V1);
    int32_t *rs = reinterpret_cast<int32_t *>(wb + L::RS);
    int32_t *j1_s = reinterpret_cast<int32_t *>(wb + L::J1);
    int32_t *df_s = reinterpret_cast<int32_t *>(wb + L::DF);
    uint8_t *sr = wb + L::SR;

    const int32_t *__restrict__ col = A.col;
    const int32_t *__restrict__ xcol = A.xcol;      // gather row of each slot
    const AV *__restrict__ val = (const AV *)A.val;
    const TS *__restrict__ X = (const TS *)A.x;
    const int Kp = A.Kp;
    const int wbase = __ldg(A.rp + r0);
    const int nslot = __ldg(A.rp + min(r0 + R, (int64_t)A.n)) - wbase;
    const bool parked = nslot <= L::CAP;            // warp-uniform
    for (int k = lane32; k <= R; k += 32)       // R + 1 offsets (33 when G = 1)
        rs[k] = __ldg(A.rp + min(r0 + k, (int64_t)A.n)) - wbase;

    // ---- 1. targets; every gathered row parked by slot ----------------------------
    if (active) {
        const int p0 = __ldg(A.rp + r), p1 = __ldg(A.rp + r + 1);
        const C diag = (C)__ldg((const AV *)A.diag + r);
        Acc<C, V> acc[NV];
#pragma unroll
        for (int t = 0; t < NV; ++t) acc[t].zero();
        for (int pb = p0; pb < p1; pb += U) {
            int jj[U];
            C vv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool ok = pb + u < p1;
                jj[u] = ok ? ld_csr(xcol + pb + u) : -1;
                vv[u] = ok ? (C)ld_csr(val + pb + u) : C(0);
            }
            uint4 raw[U][NV];
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (jj[u] >= 0) {
                    const TS *src = X + checked_row(jj[u], A.n, A.status) * Kp;
                    if constexpr (NV % 2 == 0) {         // side-by-side pieces: 32-byte pairs
#pragma unroll
                        for (int t = 0; t < NV; t += 2)
                            ldg32(src + piece_of<G, NV>(lane, t) * V, raw[u][t], raw[u][t + 1]);
                    } else {
#pragma unroll
                        for (int t = 0; t < NV; ++t) raw[u][t] = ldg16(src + piece_of<G, NV>(lane, t) * V);
                    }
                }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (jj[u] < 0) break;
                const int s = pb + u - wbase;
#pragma unroll
                for (int t = 0; t < NV; ++t) {
                    C x[V];
                    S::unpack(raw[u][t], x);
                    acc[t].fma_piece(vv[u], x);
                    if (parked) xs[park_index<P>(s, piece_of<G, NV>(lane, t))] = raw[u][t];
                }
                if (parked && lane == 0) sr[s] = (uint8_t)rw;
            }
        }
        const C d = C(1) / diag;
        const int64_t xr = A.xrow ? checked_row(__ldg(A.xrow + r), A.n, A.status) : r;
        C y[NV][V];
#pragma unroll
        for (int t = 0; t < NV; ++t) {
            S::unpack(ldg16(X + xr * Kp + piece_of<G, NV>(lane, t) * V), y[t]);     // x_i
            if (A.target == 0) {
#pragma unroll
                for (int e = 0; e < V; ++e) y[t][e] = fma(-d, acc[t].get(e), y[t][e]);
            }
            st_piece<C, V>(ys + rw * L::YST + piece_of<G, NV>(lane, t) * V, y[t]);
        }
        if constexpr (kMixed) {
            C syy = C(0);
#pragma unroll
            for (int t = 0; t < NV; ++t)
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    const C wk = UW ? C(1) : wv[piece_of<G, NV>(lane, t) * V + e];
                    syy = fma(UW ? y[t][e] : wk * y[t][e], y[t][e], syy);
                }
            syy = group_sum<G>(syy, gmask);
            if (lane == 0) syy_s[rw] = syy;
        }
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
            dg_s[rw] = diag;
            j1_s[rw] = j1;
            v1_s[rw] = v1;
            df_s[rw] = 0;
        }
    }
    __syncwarp();

    // ---- 2. one-point fits, one lane per stored entry -----------------------------
    // the fit of slot s (row rl of the warp) from its x_j pieces (parked window or
    // global memory: a warp-uniform choice, so each loop below is straight code)
    C *a_out = (C *)A.a_out;
    C *ls_out = (C *)A.ls_out;
    auto fits = [&](auto parked_tag) {
        constexpr bool PK = decltype(parked_tag)::value;
        for (int s = lane32; s < nslot; s += 32) {
            const int p = wbase + s;
            int rl = 0;
            if constexpr (PK) {
                rl = sr[s];
            } else {
#pragma unroll
                for (int b = R / 2; b >= 1; b >>= 1)
                    if (rl + b < R && rs[rl + b] <= s) rl += b;      // last row starting at or before s
            }
            const int i = (int)r0 + rl;
            const int j = __ldg(A.pcol + p);
            C a_, ls_;
            if (j == i) {
                a_ = C(0);
                ls_ = C(NAN);
            } else if (j == j1_s[rl]) {
                a_ = -v1_s[rl] / dg_s[rl];                     // y_i = -(a_ij/a_ii) x_j exactly
                ls_ = C(0);
            } else {
                const C *yr = ys + rl * L::YST;
                const TS *xg = PK ? nullptr : X + checked_row(__ldg(xcol + p), A.n, A.status) * Kp;
                auto piece = [&](int c) -> uint4 {
                    if constexpr (PK) return xs[park_index<P>(s, c)];
                    else return ldg16(xg + c * V);
                };
                uint4 hold[HOLD];
#pragma unroll
                for (int c = 0; c < HOLD; ++c) hold[c] = piece(c);
                auto held = [&](int c) -> uint4 { return (P <= 4) ? hold[c < HOLD ? c : 0] : piece(c); };
                auto weights = [&](int c, C (&w)[V]) {
#pragma unroll
                    for (int e = 0; e < V; ++e) w[e] = UW ? C(1) : wv[c * V + e];
                };
                if constexpr (COMP && kMixed) {
                    // S_xx and S_yx as two compensated pairs over (even, odd)
                    // components: the products need no regrouping of registers
                    Comp2 xx, yx;
#pragma unroll
                    for (int c = 0; c < P; ++c) {
                        C x[V], y[V], w[V];
                        S::unpack(held(c), x);
                        ld_piece<C, V>(yr + c * V, y);
                        weights(c, w);
#pragma unroll
                        for (int e = 0; e < V; e += 2) {
                            const float2 x2 = make_float2(x[e], x[e + 1]);
                            const float2 wx = UW ? x2 : make_float2(w[e] * x[e], w[e + 1] * x[e + 1]);
                            xx.add(__fmul2_rn(wx, x2));
                            yx.add(__fmul2_rn(wx, make_float2(y[e], y[e + 1])));
                        }
                    }
                    const C sxx = comp_ls_total<1>(xx, 0xffffffffu), syx = comp_ls_total<1>(yx, 0xffffffffu);
                    a_ = (sxx == C(0)) ? C(0) : divide(syx, sxx);
                    Comp2 sl;
#pragma unroll
                    for (int c = 0; c < P; ++c) {
                        C x[V], y[V], w[V];
                        S::unpack(held(c), x);
                        ld_piece<C, V>(yr + c * V, y);
                        weights(c, w);
                        comp_residual<V, UW>(a_, x, y, w, sl);
                    }
                    ls_ = comp_ls_total<1>(sl, 0xffffffffu);
                } else {
                    PieceSums<C, V, UW> ps;
#pragma unroll
                    for (int c = 0; c < P; ++c) {
                        C x[V], y[V], w[V];
                        S::unpack(held(c), x);
                        ld_piece<C, V>(yr + c * V, y);
                        weights(c, w);
                        ps.add(x, y, w);
                    }
                    const C sxx = ps.sxx(), syx = ps.syx();
                    a_ = (sxx == C(0)) ? C(0) : divide(syx, sxx);
                    C res = C(0);
#pragma unroll
                    for (int c = 0; c < P; ++c) {
                        C x[V], y[V], w[V];
                        S::unpack(held(c), x);
                        ld_piece<C, V>(yr + c * V, y);
                        weights(c, w);
                        residual_add<C, V, UW>(a_, x, y, w, res);
                    }
                    ls_ = res;
                }
                if constexpr (kMixed)
                    if (ls_ < C(1e-4) * syy_s[rl]) df_s[rl] = 1;   // cancellation: redo the row in FP64
            }
            a_out[p] = a_;
            ls_out[p] = ls_;
            if constexpr (PK) lss[s] = ls_;
        }
    };
    if (parked) fits(std::true_type{});
    else fits(std::false_type{});
    __syncwarp();

    // ---- 3. row minimum, strength flags and counts (Eq. (4.4) in LS form) --------
    if (active) {
        const C theta = (C)A.theta;
        const int s0 = rs[rw], s1 = rs[rw + 1];
        C m = C(INFINITY);                         // the diagonal's NaN never wins fmin
        for (int s = s0 + lane; s < s1; s += G) m = fmin(m, parked ? lss[s] : ls_out[wbase + s]);
        m = group_min<G>(m, gmask);
        int cnt = 0;
        for (int s = s0 + lane; s < s1; s += G) {
            const C l = parked ? lss[s] : ls_out[wbase + s];
            const int strong = l == C(0) || theta * l < m;    // false for the diagonal's NaN
            A.flag_out[wbase + s] = (uint8_t)strong;
            cnt += strong;
        }
        cnt = group_sum<G>(cnt, gmask);
        if (lane == 0) {
            A.count_out[r] = cnt;
            if (kMixed && df_s[rw]) A.defer_list[atomicAdd(A.defer_count, 1u)] = (int32_t)r;
        }
    }
}

template <class TS, int G, int NV, int U, bool UW, bool COMP>
cudaError_t go_warp(const EdgeArgs &a, cudaStream_t s)
{
    using L = WarpEdgeLayout<TS, G, NV>;
    if (a.Kp != L::KP || !a.xcol) return cudaErrorInvalidValue;
    if constexpr (NV % 2 == 0)                    // 32-byte row reads
        if (!rows_aligned32(a.x, a.Kp, sizeof(TS))) return cudaErrorMisalignedAddress;
    constexpr int smem = L::block_bytes(UW);
    static_assert(smem <= 227 * 1024, "warp windows exceed the shared memory of a block");
    const int64_t rows_per_block = (int64_t)kWarpEdgeWarps * L::R;
    const unsigned grid = (unsigned)((a.n + rows_per_block - 1) / rows_per_block);
    static PerDevice opted;                  // shared-memory opt-in made on each device
    const int dev = current_device_index();
    if (smem > 48 * 1024 && opted.get(dev) == 0) {
        const cudaError_t e = cudaFuncSetAttribute(k_edge_warp<TS, G, NV, U, UW, COMP>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        opted.set(dev, 1);
    }
    k_edge_warp<TS, G, NV, U, UW, COMP><<<grid, kWarpEdgeThreads, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace edge_impl
}  // namespace amgd
