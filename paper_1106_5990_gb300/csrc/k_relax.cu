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
// Thread mapping (Shape): G lanes own one row; lane l holds NV of the row's
// 16-byte vectors -- side by side (l*NV, ..., l*NV+NV-1), moved two per
// 32-byte access, when NV is even (direct and chunked kernels; piece_of in
// rowops.cuh), else l, l+G, ..., l+(NV-1)G (the staged kernels always) -- so
// each neighbour row is read as fully used pieces.  Nonzeros are
// taken U at a time: U column indices and values are loaded, then all U*NV
// vector pieces are requested before any is consumed, which keeps U*NV loads
// per lane in flight (the kernel is bound by HBM latency and bandwidth: CSR
// once, vectors read and written once per phase).  The sums still run in CSR
// order.  This is a CSR SpMM with K right-hand sides; no tensor cores.
#include "amgd_internal.cuh"
#include "staging.cuh"
#include "rowops.cuh"

namespace amgd {
namespace {

constexpr int kRelaxThreads = 256;

// AMGD_RELAX_MINB: minimum resident blocks per SM asked of the compiler (0:
// none -- an explicit minimum, even 1, changes the compiler's register target)
#ifndef AMGD_RELAX_MINB
#define AMGD_RELAX_MINB 0
#endif
#if AMGD_RELAX_MINB > 0
#define AMGD_RELAX_BOUNDS __launch_bounds__(kRelaxThreads, AMGD_RELAX_MINB)
#else
#define AMGD_RELAX_BOUNDS __launch_bounds__(kRelaxThreads)
#endif

template <class TS, int G, int NV, int U, bool SPLIT>
__global__ void AMGD_RELAX_BOUNDS k_relax(RelaxArgs A)
{
    using S = Store<TS>;
    using C = typename S::C;
    using AV = typename S::A;
    constexpr int V = S::V;
    const int lane = threadIdx.x % G;
    const int64_t r = (int64_t)A.r0 + (int64_t)blockIdx.x * (kRelaxThreads / G) + threadIdx.x / G;
    if (r >= A.r1) return;
    const TS *xold = (const TS *)A.xold;
    TS *xnew = (TS *)A.xnew;
    const int Kp = A.Kp;

    const int p0 = ld_csr(A.rp + r), p1 = ld_csr(A.rp + r + 1);
    Acc<C, V> acc[NV];
    row_sum<TS, G, NV, U, SPLIT>(A.col, (const AV *)A.val, xold, xnew, A.split, Kp, lane, p0, p1, acc,
                                 A.nrows, A.status);
    const C c = (C)A.omega / ld_csr((const AV *)A.diag + r);
#pragma unroll
    for (int t = 0; t < NV; ++t) {
        C xi[V], out[V];
        S::unpack(ldg16(xold + r * Kp + piece_of<G, NV>(lane, t) * V), xi);   // row r is never of an earlier color
#pragma unroll
        for (int e = 0; e < V; ++e) out[e] = fma(-c, acc[t].get(e), xi[e]);
        S::store(xnew + r * Kp + piece_of<G, NV>(lane, t) * V, out);
    }
}

// Persistent, pipelined variant.  The block walks tiles of RT = kRelaxThreads/G
// consecutive rows; three tiles are in flight at once:
//   * tile k+2: its CSR slice (row pointers, column indices, values) is
//     being bulk-copied into a shared-memory stage by the TMA (staging.cuh);
//   * tile k+1: every lane has issued cp.async copies of its 16-byte pieces
//     of all neighbour rows into a shared-memory landing buffer;
//   * tile k:   computed from the landed pieces and the staged CSR.
// No register is held by a load in flight, so the number of gathers in
// flight per SM is bounded by shared memory, not by registers; the chain of
// dependent global round trips per row (row pointer -> column index ->
// gather) is gone.  A row with more than MAXR stored entries, or a tile
// whose slice does not fit a stage, is read from global memory directly.
// Results are the same bits as k_relax (same row sums in the same order).
constexpr int kStageRowsAvg = 20;   // CSR stage capacity per row of the tile
constexpr int kLandRows = 12;       // landing slots per row (MAXR)

template <class TS, int G>
constexpr int stage_cap()
{
    return ((kRelaxThreads / G) * kStageRowsAvg + 8 + 3) & ~3;
}

template <class TS, int G, int NV>
struct StagedLayout {
    static constexpr int RT = kRelaxThreads / G;
    static constexpr int CAP = stage_cap<TS, G>();
    static constexpr int RPW = ((RT + 1 + 3 + 4) + 3) & ~3;      // widened row-pointer slice
    static constexpr int STAGE = RPW * 4 + CAP * 4 + CAP * (int)sizeof(typename Store<TS>::A);
    static constexpr int LAND = RT * kLandRows * G * NV * 16;      // one landing buffer
    static constexpr int BYTES = 16 + 2 * STAGE + 2 * LAND;
};

template <class TS, int G, int NV>
constexpr int stage_smem_bytes()
{
    return StagedLayout<TS, G, NV>::BYTES;
}

template <class TS, int G, int NV, int U>
__global__ void __launch_bounds__(kRelaxThreads)
k_relax_staged(RelaxArgs A)
{
    using S = Store<TS>;
    using C = typename S::C;
    using AV = typename S::A;
    using L = StagedLayout<TS, G, NV>;
    constexpr int V = S::V;
    constexpr int RT = L::RT, CAP = L::CAP, RPW = L::RPW;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    int32_t *rp_s[2], *col_s[2];
    AV *val_s[2];
    uint4 *land[2];
    for (int k = 0; k < 2; ++k) {
        unsigned char *base = smem + 16 + k * L::STAGE;
        rp_s[k] = reinterpret_cast<int32_t *>(base);
        col_s[k] = rp_s[k] + RPW;
        val_s[k] = reinterpret_cast<AV *>(col_s[k] + CAP);
        land[k] = reinterpret_cast<uint4 *>(smem + 16 + 2 * L::STAGE + k * L::LAND);
    }

    const int32_t *__restrict__ rp = A.rp;
    const int32_t *__restrict__ col = A.col;
    const AV *__restrict__ val = (const AV *)A.val;
    const TS *__restrict__ xold = (const TS *)A.xold;
    TS *__restrict__ xnew = (TS *)A.xnew;
    const int Kp = A.Kp;
    const C omega = (C)A.omega;
    const int lane = threadIdx.x % G, grp = threadIdx.x / G;
    const int64_t nrows = (int64_t)A.r1 - A.r0;
    const int64_t ntiles = (nrows + RT - 1) / RT;
    const int64_t T = gridDim.x;

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // the tile's rows, its row-pointer slice [q0, q1) and CSR slice [s0a, s1a),
    // both widened to 16-byte boundaries; staged iff the slice fits a stage
    struct Tile {
        int64_t r0, r1, q0, s0a, s1a;
        bool staged;
    };
    auto tile_of = [&](int64_t t) {
        Tile tl;
        tl.r0 = A.r0 + t * RT;
        tl.r1 = min((int64_t)A.r1, tl.r0 + RT);
        tl.q0 = tl.r0 & ~(int64_t)3;
        tl.s0a = (int64_t)__ldg(rp + tl.r0) & ~(int64_t)3;
        tl.s1a = ((int64_t)__ldg(rp + tl.r1) + 3) & ~(int64_t)3;
        tl.staged = tl.s1a - tl.s0a <= CAP;
        return tl;
    };
    uint32_t parity[2] = {0u, 0u};
    bool issued[2] = {false, false};     // thread 0: copies issued, completion not yet seen
    auto issue_csr = [&](int64_t t, int stg, uint32_t extra) {   // thread 0 only
        const Tile tl = tile_of(t);
        if (!tl.staged) return;
        const int64_t q1 = (tl.r1 + 1 + 3) & ~(int64_t)3;
        const uint32_t nb_rp = (uint32_t)((q1 - tl.q0) * 4);
        const uint32_t nb_col = (uint32_t)((tl.s1a - tl.s0a) * 4);
        const uint32_t nb_val = (uint32_t)((tl.s1a - tl.s0a) * sizeof(AV));
        fence_proxy_async();
        mbar_arrive_expect_tx(&bar[stg], nb_rp + nb_col + nb_val + extra);
        issued[stg] = true;
        bulk_g2s(rp_s[stg], rp + tl.q0, nb_rp, &bar[stg]);
        bulk_g2s(col_s[stg], col + tl.s0a, nb_col, &bar[stg]);
        bulk_g2s(val_s[stg], val + tl.s0a, nb_val, &bar[stg]);
    };
    // wait for stage stg of tile t (if it was staged); false on time-out
    auto wait_csr = [&](const Tile &tl, int stg) {
        if (!tl.staged) return true;
        if (!mbar_wait_bounded(&bar[stg], parity[stg], A.wait_limit, A.status,
                               kStatusStagingTimeout))
            return false;
        parity[stg] ^= 1u;
        issued[stg] = false;
        return true;
    };
    // this thread's gathers for its row of tile tl into landing buffer lb
    auto issue_gathers = [&](const Tile &tl, int stg, int lb) {
        const int64_t r = tl.r0 + grp;
        if (r < tl.r1 && tl.staged) {
            const int p0 = rp_s[stg][r - tl.q0], p1 = rp_s[stg][r + 1 - tl.q0];
            if (p1 - p0 <= kLandRows) {
                uint4 *dst = land[lb] + (size_t)grp * kLandRows * (G * NV);
                for (int p = p0; p < p1; ++p) {
                    const int j = col_s[stg][p - tl.s0a];
                    const TS *src = (j < A.split ? (const TS *)xnew : xold) + checked_row(j, A.nrows, A.status) * Kp;
#pragma unroll
                    for (int tt = 0; tt < NV; ++tt)
                        cp_async16(dst + (p - p0) * (G * NV) + tt * G + lane, src + (tt * G + lane) * V);
                }
            }
        }
        cp_async_commit();
    };
    // leave after a time-out: thread 0 gives every bulk copy it issued a
    // bounded chance to land (shared memory must not be released under a copy
    // in flight); every thread drains its own cp.async groups
    auto bail = [&]() {
        for (int k = 0; k < 2; ++k)
            if (issued[k])
                mbar_wait_bounded(&bar[k], parity[k], A.wait_limit, A.status, kStatusStagingTimeout);
        cp_async_wait<0>();
    };

    // prologue: CSR of the first two tiles, gathers of the first
    int64_t t = blockIdx.x;
    if (t >= ntiles) return;
    if (threadIdx.x == 0) {
        issue_csr(t, 0, A.extra_tx);
        if (t + T < ntiles) issue_csr(t + T, 1, 0);
    }
    Tile cur = tile_of(t);
    if (__syncthreads_or(!wait_csr(cur, 0))) { bail(); return; }
    issue_gathers(cur, 0, 0);

    for (int it = 0; t < ntiles; t += T, ++it) {
        const int stg = it & 1;
        const int64_t tn = t + T;
        Tile nxt;
        bool ok = true;
        if (tn < ntiles) {
            nxt = tile_of(tn);
            ok = wait_csr(nxt, stg ^ 1);
        }
        if (__syncthreads_or(!ok)) { bail(); return; }
        if (tn < ntiles) issue_gathers(nxt, stg ^ 1, stg ^ 1);
        else cp_async_commit();
        cp_async_wait<1>();            // this thread's gathers of tile t have landed

        const int64_t r = cur.r0 + grp;
        if (r < cur.r1) {
            int p0, p1;
            if (cur.staged) { p0 = rp_s[stg][r - cur.q0]; p1 = rp_s[stg][r + 1 - cur.q0]; }
            else { p0 = __ldg(rp + r); p1 = __ldg(rp + r + 1); }
            const bool landed = cur.staged && p1 - p0 <= kLandRows;
            const uint4 *lsrc = land[stg] + (size_t)grp * kLandRows * (G * NV);
            C acc[NV][V], xi[NV][V];
#pragma unroll
            for (int tt = 0; tt < NV; ++tt)
#pragma unroll
                for (int e = 0; e < V; ++e) { acc[tt][e] = C(0); xi[tt][e] = C(0); }
            C diag = C(1);
            for (int p = p0; p < p1; ++p) {
                int j;
                C v;
                if (cur.staged) { j = col_s[stg][p - cur.s0a]; v = (C)val_s[stg][p - cur.s0a]; }
                else { j = __ldg(col + p); v = (C)__ldg(val + p); }
                const TS *src = (j < A.split ? (const TS *)xnew : xold) + checked_row(j, A.nrows, A.status) * Kp;
#pragma unroll
                for (int tt = 0; tt < NV; ++tt) {
                    const uint4 raw = landed ? lsrc[(p - p0) * (G * NV) + tt * G + lane]
                                             : ldg16(src + (tt * G + lane) * V);
                    C x[V];
                    S::unpack(raw, x);
                    if (j == r) {
#pragma unroll
                        for (int e = 0; e < V; ++e) xi[tt][e] = x[e];
                    }
#pragma unroll
                    for (int e = 0; e < V; ++e) acc[tt][e] = fma(v, x[e], acc[tt][e]);
                }
                if (j == r) diag = v;
            }
            const C c = omega / diag;
#pragma unroll
            for (int tt = 0; tt < NV; ++tt) {
                C out[V];
#pragma unroll
                for (int e = 0; e < V; ++e) out[e] = fma(-c, acc[tt][e], xi[tt][e]);
                S::store(xnew + r * Kp + (tt * G + lane) * V, out);
            }
        }
        __syncthreads();               // stage stg and landing stg are read out
        if (threadIdx.x == 0 && tn + T < ntiles) issue_csr(tn + T, stg, 0);
        cur = nxt;
    }
    cp_async_wait<0>();
}

// Warp-pipelined variant (stage 2).  Every warp walks its own contiguous
// chunk of rows in groups of RG = 32/G rows (one row per G lanes) and keeps
// three groups in flight, with no block barrier and no spin-wait:
//   * group k+2: its CSR slice (column indices, values) is being copied into
//     the warp's shared memory with cp.async (16-byte pieces, all lanes);
//   * group k+1: every lane has issued cp.async copies of its pieces of all
//     neighbour rows into the warp's landing buffer;
//   * group k:   computed from shared memory.
// Row pointers are prefetched into registers three groups ahead.  The loads
// in flight hold no registers, so a warp overlaps the HBM latency of two
// groups with the arithmetic of a third.  Rows with more than kPipeMaxNnz
// stored entries, or groups whose slice exceeds the buffer, are computed from
// global memory directly.  Same row sums in the same order as k_relax.
constexpr int kPipeMaxNnz = 12;
constexpr int kPipeWarps = 4;                // warps per block

template <class TS, int G, int NV>
struct PipeLayout {
    static constexpr int RG = 32 / G;
    static constexpr int MAXE = RG * kPipeMaxNnz + 8;                 // multiple of 4
    static constexpr int CSR = MAXE * (4 + (int)sizeof(typename Store<TS>::A));
    static constexpr int LAND = RG * kPipeMaxNnz * G * NV * 16;
    static constexpr int WARP = 3 * CSR + 2 * LAND;
    static constexpr int BYTES = kPipeWarps * WARP;
};

template <class TS, int G, int NV>
__global__ void __launch_bounds__(kPipeWarps * 32)
k_relax_pipe(RelaxArgs A, int64_t chunk)
{
    using S = Store<TS>;
    using C = typename S::C;
    using AV = typename S::A;
    using L = PipeLayout<TS, G, NV>;
    constexpr int V = S::V, RG = L::RG, MAXE = L::MAXE, P = G * NV;
    extern __shared__ __align__(16) unsigned char smem[];
    const int wib = threadIdx.x / 32, lane32 = threadIdx.x % 32;
    const int lane = lane32 % G, rig = lane32 / G;          // row inside the group
    unsigned char *wbase = smem + (size_t)wib * L::WARP;
    int32_t *col_b[3];
    AV *val_b[3];
    for (int k = 0; k < 3; ++k) {
        col_b[k] = reinterpret_cast<int32_t *>(wbase + k * L::CSR);
        val_b[k] = reinterpret_cast<AV *>(col_b[k] + MAXE);
    }
    uint4 *land_b[2];
    for (int k = 0; k < 2; ++k) land_b[k] = reinterpret_cast<uint4 *>(wbase + 3 * L::CSR + k * L::LAND);

    const int32_t *__restrict__ rp = A.rp;
    const int32_t *__restrict__ col = A.col;
    const AV *__restrict__ val = (const AV *)A.val;
    const TS *__restrict__ xold = (const TS *)A.xold;
    TS *__restrict__ xnew = (TS *)A.xnew;
    const int Kp = A.Kp;
    const int split = A.split;
    const C omega = (C)A.omega;

    if (RG + 1 > 32) return;              // never launched (see go_pipe)
    const int64_t gw = (int64_t)blockIdx.x * kPipeWarps + wib;
    const int64_t c0 = A.r0 + gw * chunk;
    const int64_t c1 = min((int64_t)A.r1, c0 + chunk);
    if (c0 >= c1) return;
    const int ngroups = (int)((c1 - c0 + RG - 1) / RG);

    // row pointer of row g0(k) + lane32 (lanes 0..RG hold the group's bounds)
    auto rp_of = [&](int k) -> int {
        const int64_t r = min(c0 + (int64_t)k * RG + lane32, c1);
        return (k < ngroups && lane32 <= RG) ? __ldg(rp + r) : 0;
    };
    // a group is buffered when its widened slice fits
    auto slice = [&](int rpv, int &s0a, int &s1a) {
        const int s0 = __shfl_sync(0xffffffffu, rpv, 0);
        const int s1 = __shfl_sync(0xffffffffu, rpv, RG);
        s0a = s0 & ~3;
        s1a = (s1 + 3) & ~3;
        return s1a - s0a <= MAXE;
    };
    auto issue_csr = [&](int k, int rpv) {
        if (k >= ngroups) return;
        int s0a, s1a;
        if (!slice(rpv, s0a, s1a)) return;
        const int b = k % 3;
        const int nc = (s1a - s0a) / 4;                       // 16-byte pieces of col
        for (int q = lane32; q < nc; q += 32) cp_async16(col_b[b] + 4 * q, col + s0a + 4 * q);
        constexpr int EPP = 16 / (int)sizeof(AV);             // values per piece
        const int nv = (s1a - s0a) / EPP;
        for (int q = lane32; q < nv; q += 32) cp_async16(val_b[b] + EPP * q, val + s0a + EPP * q);
    };
    auto issue_gathers = [&](int k, int rpv) {
        if (k >= ngroups) return;
        int s0a, s1a;
        if (!slice(rpv, s0a, s1a)) return;
        const int64_t r = c0 + (int64_t)k * RG + rig;
        const int p0 = __shfl_sync(0xffffffffu, rpv, rig), p1 = __shfl_sync(0xffffffffu, rpv, rig + 1);
        if (r >= c1 || p1 - p0 > kPipeMaxNnz) return;
        const int32_t *cb = col_b[k % 3];
        uint4 *dst = land_b[k & 1] + (size_t)rig * kPipeMaxNnz * P;
        for (int p = p0; p < p1; ++p) {
            const int j = cb[p - s0a];
            const TS *src = (j < split ? (const TS *)xnew : xold) + checked_row(j, A.nrows, A.status) * Kp;
#pragma unroll
            for (int tt = 0; tt < NV; ++tt)
                cp_async16(dst + (p - p0) * P + tt * G + lane, src + (tt * G + lane) * V);
        }
    };

    int rq0 = rp_of(0), rq1 = rp_of(1), rq2 = rp_of(2);
    issue_csr(0, rq0);
    issue_csr(1, rq1);
    cp_async_commit();
    cp_async_wait<0>();
    __syncwarp();
    issue_gathers(0, rq0);
    cp_async_commit();
    int rq3 = rp_of(3);

    for (int k = 0; k < ngroups; ++k) {
        cp_async_wait<0>();            // gathers of k and CSR of k+1 have landed
        __syncwarp();
        issue_csr(k + 2, rq2);
        issue_gathers(k + 1, rq1);
        cp_async_commit();
        const int rq4 = rp_of(k + 4);

        const int64_t r = c0 + (int64_t)k * RG + rig;
        const int p0 = __shfl_sync(0xffffffffu, rq0, rig), p1 = __shfl_sync(0xffffffffu, rq0, rig + 1);
        int s0a, s1a;
        const bool buffered = slice(rq0, s0a, s1a);
        if (r < c1) {
            const bool landed = buffered && p1 - p0 <= kPipeMaxNnz;
            const int32_t *cb = col_b[k % 3];
            const AV *vb = val_b[k % 3];
            const uint4 *lsrc = land_b[k & 1] + (size_t)rig * kPipeMaxNnz * P;
            C acc[NV][V], xi[NV][V];
#pragma unroll
            for (int tt = 0; tt < NV; ++tt)
#pragma unroll
                for (int e = 0; e < V; ++e) { acc[tt][e] = C(0); xi[tt][e] = C(0); }
            C diag = C(1);
            for (int p = p0; p < p1; ++p) {
                const int j = buffered ? cb[p - s0a] : __ldg(col + p);
                const C v = buffered ? (C)vb[p - s0a] : (C)__ldg(val + p);
#pragma unroll
                for (int tt = 0; tt < NV; ++tt) {
                    uint4 raw;
                    if (landed) {
                        raw = lsrc[(p - p0) * P + tt * G + lane];
                    } else {
                        const TS *src = (j < split ? (const TS *)xnew : xold) + checked_row(j, A.nrows, A.status) * Kp;
                        raw = ldg16(src + (tt * G + lane) * V);
                    }
                    C x[V];
                    S::unpack(raw, x);
                    if (j == r) {
#pragma unroll
                        for (int e = 0; e < V; ++e) xi[tt][e] = x[e];
                    }
#pragma unroll
                    for (int e = 0; e < V; ++e) acc[tt][e] = fma(v, x[e], acc[tt][e]);
                }
                if (j == r) diag = v;
            }
            const C c = omega / diag;
#pragma unroll
            for (int tt = 0; tt < NV; ++tt) {
                C out[V];
#pragma unroll
                for (int e = 0; e < V; ++e) out[e] = fma(-c, acc[tt][e], xi[tt][e]);
                S::store(xnew + r * Kp + (tt * G + lane) * V, out);
            }
        }
        __syncwarp();                  // buffers of group k are read out
        rq0 = rq1; rq1 = rq2; rq2 = rq3; rq3 = rq4;
    }
    cp_async_wait<0>();
}

// Chunked persistent variant (stage 3).  One block of kChunkThreads threads
// per SM owns one contiguous chunk of rows; its warps walk the chunk side by
// side in groups of RW = 32/G rows (group g of the chunk goes to warp g mod W),
// so the whole SM moves through consecutive rows together.  On matrices whose
// neighbours are close in the row order (stencils on grid lines, banded and
// mesh orderings) the rows an SM gathers are then the few grid lines around
// its current position, and a line fetched into L1 for one row serves the
// rows of the next lines too: the L2 -> L1 traffic of the gathers drops from
// one copy of each vector row per block that touches it towards one per SM.
// Each warp also asks the L2 for the row-pointer line of its group after next
// and for the column-index and value lines of its next group (their bounds
// come from the row pointers prefetched one group earlier), so a row's first
// two dependent round trips hit L2.  L2 policy: the test-vector block (read
// by the gathers, written by the update) is loaded and stored with an
// evict-last hint and the CSR, which streams through once per sweep, with an
// evict-first hint, so the vectors of the next color phase and sweep tend to
// stay in the 129 MB L2 instead of being pushed out by the matrix.  Same row
// sums in the same order as k_relax: same bits.  896 threads (28 warps): the
// register budget of 72 per thread holds a batch of four 64-byte rows per lane
// pair without spilling (at 1024 threads, 64 registers spilled and the sweep
// was 10% slower; 768 threads were 4% slower, and at 640 the direct kernel
// wins).
constexpr int kChunkThreads = 896;

__device__ __forceinline__ void prefetch_l2(const void *p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
__device__ __forceinline__ uint64_t policy_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_first()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint4 ldg16_hint(const void *p, uint64_t pol)
{
    uint4 v;
    asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void st16_hint(void *p, const uint4 &v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1,%2,%3,%4}, %5;" ::"l"(p), "r"(v.x),
                 "r"(v.y), "r"(v.z), "r"(v.w), "l"(pol)
                 : "memory");
}
// 32-byte vector load / store (sm_100 and later; the address is 32-byte aligned)
__device__ __forceinline__ void ldg32_hint(const void *p, uint64_t pol, uint4 &a, uint4 &b)
{
    asm volatile("ld.global.nc.L2::cache_hint.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], %9;"
                 : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w), "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
                 : "l"(p), "l"(pol));
}
__device__ __forceinline__ void st32_hint(void *p, const uint4 &a, const uint4 &b, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.v8.u32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8}, %9;" ::"l"(p),
                 "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b.x), "r"(b.y), "r"(b.z), "r"(b.w), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ int32_t ld32_hint(const int32_t *p, uint64_t pol)
{
    int32_t v;
    asm volatile("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ float ldv_hint(const float *p, uint64_t pol)
{
    float v;
    asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ double ldv_hint(const double *p, uint64_t pol)
{
    double v;
    asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}

template <class TS, int G, int NV, int U, bool SPLIT>
__global__ void __launch_bounds__(kChunkThreads, 1) k_relax_chunk(RelaxArgs A, int32_t chunk)
{
    using S = Store<TS>;
    using C = typename S::C;
    using AV = typename S::A;
    constexpr int V = S::V, RW = 32 / G, NW = kChunkThreads / 32;
    constexpr int64_t STEP = (int64_t)NW * RW;            // rows between a warp's groups
    const int warp = threadIdx.x / 32, lane32 = threadIdx.x % 32;
    const int lane = lane32 % G, rig = lane32 / G;
    const TS *xold = (const TS *)A.xold;
    TS *xnew = (TS *)A.xnew;
    const AV *val = (const AV *)A.val;
    const int32_t *col = A.col;
    const int Kp = A.Kp;
    const int64_t c0 = (int64_t)A.r0 + (int64_t)blockIdx.x * chunk;
    const int64_t c1 = min((int64_t)A.r1, c0 + chunk);
    const uint64_t keep = policy_evict_last(), stream = policy_evict_first();
    // a lane holding an even number of pieces holds them side by side and moves
    // them two at a time (32-byte accesses: half the load instructions and
    // cache wavefronts of a gather); otherwise the pieces interleave over the
    // G lanes.  Every component keeps its own FMA chain, so both layouts give
    // the same bits.
    constexpr bool W32 = NV % 2 == 0;
    auto piece = [&](int tt) { return W32 ? lane * NV + tt : tt * G + lane; };

    for (int64_t wr0 = c0 + (int64_t)warp * RW; wr0 < c1; wr0 += STEP) {
        // row pointers of this warp's group after next, into L2
        if (lane32 == 0 && wr0 + 2 * STEP < c1) prefetch_l2(A.rp + wr0 + 2 * STEP);
        // bounds of this warp's next group (its row pointers were prefetched)
        int n0 = 0, n1 = 0;
        if (wr0 + STEP < c1) {
            n0 = ld32_hint(A.rp + wr0 + STEP, stream);
            n1 = ld32_hint(A.rp + min(wr0 + STEP + RW, c1), stream);
        }
        const int64_t r = wr0 + rig;
        if (r < c1) {
            const int p0 = ld32_hint(A.rp + r, stream), p1 = ld32_hint(A.rp + r + 1, stream);
            Acc<C, V> acc[NV];
#pragma unroll
            for (int tt = 0; tt < NV; ++tt) acc[tt].zero();
            for (int pb = p0; pb < p1; pb += U) {
                int jj[U];
                C vv[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const bool ok = pb + u < p1;
                    jj[u] = ok ? ld32_hint(col + pb + u, stream) : -1;
                    vv[u] = ok ? (C)ldv_hint(val + pb + u, stream) : C(0);
                }
                uint4 raw[U][NV];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (jj[u] >= 0) {
                        const TS *src = (SPLIT && jj[u] < A.split ? (const TS *)xnew : xold) +
                                        checked_row(jj[u], A.nrows, A.status) * Kp;
                        if constexpr (W32) {
#pragma unroll
                            for (int tt = 0; tt < NV; tt += 2)
                                ldg32_hint(src + piece(tt) * V, keep, raw[u][tt], raw[u][tt + 1]);
                        } else {
#pragma unroll
                            for (int tt = 0; tt < NV; ++tt) raw[u][tt] = ldg16_hint(src + piece(tt) * V, keep);
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
            const C c = (C)A.omega / ldv_hint((const AV *)A.diag + r, stream);
            // x_i - (omega / a_ii) s_i, a pair of pieces (W32) or one piece at a time
            constexpr int PW = W32 ? 2 : 1;
#pragma unroll
            for (int t0 = 0; t0 < NV; t0 += PW) {
                uint4 own[PW];
                if constexpr (W32) ldg32_hint(xold + r * Kp + piece(t0) * V, keep, own[0], own[1]);
                else own[0] = ldg16_hint(xold + r * Kp + piece(t0) * V, keep);
#pragma unroll
                for (int h = 0; h < PW; ++h) {
                    C xi[V], out[V];
                    S::unpack(own[h], xi);
#pragma unroll
                    for (int e = 0; e < V; ++e) out[e] = fma(-c, acc[t0 + h].get(e), xi[e]);
                    own[h] = S::pack(out);
                }
                if constexpr (W32) st32_hint(xnew + r * Kp + piece(t0) * V, own[0], own[1], keep);
                else st16_hint(xnew + r * Kp + piece(t0) * V, own[0], keep);
            }
        }
        // column-index and value lines of this warp's next group, into L2
        if (n1 > n0) {
            const int64_t q0 = n0 & ~31, nq = ((int64_t)n1 - q0 + 31) / 32;     // 128-byte lines
            for (int64_t q = lane32; q < nq; q += 32) prefetch_l2(col + q0 + 32 * q);
            constexpr int EPL = 128 / (int)sizeof(AV);                          // values per line
            const int64_t v0 = n0 & ~(int64_t)(EPL - 1), nv = ((int64_t)n1 - v0 + EPL - 1) / EPL;
            for (int64_t q = lane32; q < nv; q += 32) prefetch_l2(val + v0 + EPL * q);
        }
    }
}

template <class TS, int G, int NV, int U>
cudaError_t go_chunk(const RelaxArgs &a, cudaStream_t s)
{
    const int64_t rows = (int64_t)a.r1 - a.r0;
    if (rows <= 0) return cudaSuccess;
    constexpr int RW = 32 / G;
    auto kern = a.split > 0 ? k_relax_chunk<TS, G, NV, U, true> : k_relax_chunk<TS, G, NV, U, false>;
    static PerDevice sm_count;
    const int dev = current_device_index();
    int sms = sm_count.get(dev);
    if (sms == 0) {
        int d = 0;
        cudaGetDevice(&d);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
        if (sms <= 0) sms = 1;
        sm_count.set(dev, sms);
    }
    // 32-byte accesses (NV even) need 32-byte aligned rows: always true of the
    // handle's buffers (P even), refused rather than faulted otherwise
    if constexpr (NV % 2 == 0) {
        if (!rows_aligned32(a.xold, a.Kp, sizeof(TS)) || !rows_aligned32(a.xnew, a.Kp, sizeof(TS)))
            return cudaErrorMisalignedAddress;
    }
    // one chunk per SM, a whole number of warp groups each
    int64_t chunk = (rows + sms - 1) / sms;
    chunk = (chunk + RW - 1) / RW * RW;
    const int64_t blocks = (rows + chunk - 1) / chunk;
    kern<<<(unsigned)blocks, kChunkThreads, 0, s>>>(a, (int32_t)chunk);
    return cudaGetLastError();
}

template <class TS, int G, int NV>
cudaError_t go_pipe(const RelaxArgs &a, cudaStream_t s)
{
    // a group's row pointers (RG + 1 of them) live in one warp's lanes, so a
    // group has at most 16 rows: G >= 2
    if constexpr (PipeLayout<TS, G, NV>::BYTES > 227 * 1024 || G < 2) {
        return cudaErrorInvalidConfiguration;
    } else {
    const int64_t rows = (int64_t)a.r1 - a.r0;
    if (rows <= 0) return cudaSuccess;
    constexpr int smem = PipeLayout<TS, G, NV>::BYTES;
    static PerDevice cache;                  // resident blocks on each device
    const int dev = current_device_index();
    int grid_cap = cache.get(dev);
    if (grid_cap == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_relax_pipe<TS, G, NV>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        int d = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&d);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_relax_pipe<TS, G, NV>,
                                                          kPipeWarps * 32, smem);
        if (e != cudaSuccess) return e;
        grid_cap = sms * (per_sm > 0 ? per_sm : 1);
        cache.set(dev, grid_cap);
    }
    // contiguous chunks, a whole number of groups each, one per warp
    constexpr int RG = PipeLayout<TS, G, NV>::RG;
    const int64_t warps = (int64_t)grid_cap * kPipeWarps;
    int64_t chunk = (rows + warps - 1) / warps;
    chunk = (chunk + RG - 1) / RG * RG;
    const int64_t used = (rows + chunk - 1) / chunk;
    const unsigned grid = (unsigned)((used + kPipeWarps - 1) / kPipeWarps);
    k_relax_pipe<TS, G, NV><<<grid, kPipeWarps * 32, smem, s>>>(a, chunk);
    return cudaGetLastError();
    }
}

constexpr int kMaxDynSmem = 227 * 1024;    // per-block dynamic shared memory on sm_103a

template <class TS, int G, int NV, int U>
cudaError_t go_staged(const RelaxArgs &a, cudaStream_t s)
{
    if constexpr (stage_smem_bytes<TS, G, NV>() > kMaxDynSmem) {
        return cudaErrorInvalidConfiguration;
    } else {
    const int64_t rows = (int64_t)a.r1 - a.r0;
    if (rows <= 0) return cudaSuccess;
    constexpr int smem = stage_smem_bytes<TS, G, NV>();
    static PerDevice cache;                  // resident blocks on each device
    const int dev = current_device_index();
    int grid_cap = cache.get(dev);
    if (grid_cap == 0) {
        cudaError_t e = cudaFuncSetAttribute(k_relax_staged<TS, G, NV, U>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        int d = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&d);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_relax_staged<TS, G, NV, U>,
                                                          kRelaxThreads, smem);
        if (e != cudaSuccess) return e;
        grid_cap = sms * (per_sm > 0 ? per_sm : 1);
        cache.set(dev, grid_cap);
    }
    const int64_t ntiles = (rows + kRelaxThreads / G - 1) / (kRelaxThreads / G);
    const unsigned grid = (unsigned)(ntiles < grid_cap ? ntiles : grid_cap);
    k_relax_staged<TS, G, NV, U><<<grid, kRelaxThreads, smem, s>>>(a);
    return cudaGetLastError();
    }
}

// shared memory of the staged kernel for a shape (0 if not instantiated)
template <class TS>
int staged_smem(int G, int NV)
{
    constexpr int V = Store<TS>::V;
    switch (G * 8 + NV) {
#define AMGD_SM(g, nv) case g * 8 + nv: if constexpr (g * nv * V <= 64) return stage_smem_bytes<TS, g, nv>(); break;
    AMGD_SM(1, 1) AMGD_SM(1, 2) AMGD_SM(1, 4) AMGD_SM(2, 1) AMGD_SM(2, 2) AMGD_SM(2, 4)
    AMGD_SM(4, 1) AMGD_SM(4, 2) AMGD_SM(4, 4) AMGD_SM(8, 1) AMGD_SM(8, 2) AMGD_SM(8, 4)
    AMGD_SM(16, 1) AMGD_SM(16, 2) AMGD_SM(16, 4) AMGD_SM(32, 1) AMGD_SM(32, 2) AMGD_SM(32, 4)
#undef AMGD_SM
    }
    return 0;
}

template <class TS, int G, int NV, int U>
cudaError_t go(const RelaxArgs &a, cudaStream_t s)
{
    const int64_t rows = (int64_t)a.r1 - a.r0;
    if (rows <= 0) return cudaSuccess;
    if constexpr (NV % 2 == 0) {                    // 32-byte row reads
        if (!rows_aligned32(a.xold, a.Kp, sizeof(TS)) || !rows_aligned32(a.xnew, a.Kp, sizeof(TS)))
            return cudaErrorMisalignedAddress;
    }
    const int rows_per_block = kRelaxThreads / G;
    const unsigned grid = (unsigned)((rows + rows_per_block - 1) / rows_per_block);
    if (a.split > 0)
        k_relax<TS, G, NV, U, true><<<grid, kRelaxThreads, 0, s>>>(a);
    else
        k_relax<TS, G, NV, U, false><<<grid, kRelaxThreads, 0, s>>>(a);
    return cudaGetLastError();
}

template <class TS, int G, int NV>
cudaError_t dispatch_u(int U, int stage, const RelaxArgs &a, cudaStream_t s)
{
    if (stage == 3) {
        switch (U) {
        case 4: return go_chunk<TS, G, NV, 4>(a, s);
        case 8: return go_chunk<TS, G, NV, 8>(a, s);
        }
        return cudaErrorInvalidValue;
    }
    switch (U) {
    case 4: return stage == 2 ? go_pipe<TS, G, NV>(a, s)
                 : stage ? go_staged<TS, G, NV, 4>(a, s) : go<TS, G, NV, 4>(a, s);
    case 8: return stage == 2 ? go_pipe<TS, G, NV>(a, s)
                 : stage ? go_staged<TS, G, NV, 8>(a, s) : go<TS, G, NV, 8>(a, s);
    }
    return cudaErrorInvalidValue;
}

template <class TS, int G>
cudaError_t dispatch_nv(int NV, int U, int stage, const RelaxArgs &a, cudaStream_t s)
{
    constexpr int V = Store<TS>::V;
    switch (NV) {
    case 1: return dispatch_u<TS, G, 1>(U, stage, a, s);
    case 2: if constexpr (G * 2 * V <= 64) return dispatch_u<TS, G, 2>(U, stage, a, s); break;
    case 4: if constexpr (G * 4 * V <= 64) return dispatch_u<TS, G, 4>(U, stage, a, s); break;
    }
    return cudaErrorInvalidValue;
}

template <class TS>
cudaError_t dispatch_g(Shape sh, const RelaxArgs &a, cudaStream_t s)
{
    constexpr int V = Store<TS>::V;
    switch (sh.G) {
    case 1: return dispatch_nv<TS, 1>(sh.NV, sh.U, sh.stage, a, s);
    case 2: return dispatch_nv<TS, 2>(sh.NV, sh.U, sh.stage, a, s);
    case 4: return dispatch_nv<TS, 4>(sh.NV, sh.U, sh.stage, a, s);
    case 8: if constexpr (8 * V <= 64) return dispatch_nv<TS, 8>(sh.NV, sh.U, sh.stage, a, s); break;
    case 16: if constexpr (16 * V <= 64) return dispatch_nv<TS, 16>(sh.NV, sh.U, sh.stage, a, s); break;
    case 32: if constexpr (32 * V <= 64) return dispatch_nv<TS, 32>(sh.NV, sh.U, sh.stage, a, s); break;
    }
    return cudaErrorInvalidValue;
}

}  // namespace

// shared memory of the pipelined kernel for a shape (0 if not instantiated)
template <class TS>
int pipe_smem(int G, int NV)
{
    constexpr int V = Store<TS>::V;
    switch (G * 8 + NV) {
#define AMGD_SM(g, nv) case g * 8 + nv: if constexpr (g * nv * V <= 64) return PipeLayout<TS, g, nv>::BYTES; break;
    AMGD_SM(1, 1) AMGD_SM(1, 2) AMGD_SM(1, 4) AMGD_SM(2, 1) AMGD_SM(2, 2) AMGD_SM(2, 4)
    AMGD_SM(4, 1) AMGD_SM(4, 2) AMGD_SM(4, 4) AMGD_SM(8, 1) AMGD_SM(8, 2) AMGD_SM(8, 4)
    AMGD_SM(16, 1) AMGD_SM(16, 2) AMGD_SM(16, 4) AMGD_SM(32, 1) AMGD_SM(32, 2) AMGD_SM(32, 4)
#undef AMGD_SM
    }
    return 0;
}

bool relax_shape_available(int storage, Shape sh)
{
    if (sh.U != 4 && sh.U != 8) return false;   // the sweeps gather 4 or 8 entries per batch
    if (!sh.stage || sh.stage == 3) return true;
    if (sh.stage == 2 && (sh.U != 4 || sh.G < 2)) return false;   // no batch size; RG <= 16
    int b = 0;
    switch (storage) {
    case ST_FP64: b = sh.stage == 2 ? pipe_smem<double>(sh.G, sh.NV) : staged_smem<double>(sh.G, sh.NV); break;
    case ST_FP32: b = sh.stage == 2 ? pipe_smem<float>(sh.G, sh.NV) : staged_smem<float>(sh.G, sh.NV); break;
    case ST_BF16:
        b = sh.stage == 2 ? pipe_smem<__nv_bfloat16>(sh.G, sh.NV) : staged_smem<__nv_bfloat16>(sh.G, sh.NV);
        break;
    }
    return b > 0 && b <= kMaxDynSmem;
}

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
