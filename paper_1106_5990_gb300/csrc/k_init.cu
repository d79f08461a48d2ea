// k_init.cu -- test-vector start (counter-based Philox4x64-10), layout and
// precision conversions of the vector block, per-slot output export and the
// permutation of A's values.
#include "amgd_internal.cuh"

namespace amgd {
namespace {

constexpr int kThreads = 256;

// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 64x64->128 multiplies with the published 4x64 multipliers, Weyl key
// schedule with the published increments.
struct U64x4 { uint64_t v[4]; };

__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                               uint64_t k0, uint64_t k1)
{
    constexpr uint64_t kMulA = 0xD2E7470EE14C6C93ull, kMulB = 0xCA5A826395121157ull;
    constexpr uint64_t kWeylA = 0x9E3779B97F4A7C15ull, kWeylB = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint64_t hiA = __umul64hi(kMulA, c0), loA = kMulA * c0;
        const uint64_t hiB = __umul64hi(kMulB, c2), loB = kMulB * c2;
        const uint64_t n0 = hiB ^ c1 ^ k0;
        const uint64_t n2 = hiA ^ c3 ^ k1;
        c0 = n0;
        c1 = loB;
        c2 = n2;
        c3 = loA;
        k0 += kWeylA;
        k1 += kWeylB;
    }
    U64x4 o;
    o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
    return o;
}

template <class TS> __device__ __forceinline__ TS from_double(double x);
template <> __device__ __forceinline__ double from_double<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_double<float>(double x) { return (float)x; }
template <> __device__ __forceinline__ __nv_bfloat16 from_double<__nv_bfloat16>(double x)
{
    return __double2bfloat16(x);
}
template <class TS> __device__ __forceinline__ double to_double(TS x) { return (double)x; }
template <> __device__ __forceinline__ double to_double<__nv_bfloat16>(__nv_bfloat16 x)
{
    return (double)__bfloat162float(x);
}

// The start value of a component is x = d * 2^-32 with the odd integer
// d = 2m + 1 - 2^32, m the component's 32-bit random integer.  |d| < 2^32,
// so the magnitude a = |d| fits 32 bits: a = 2(m - 2^31) + 1 for m >= 2^31
// (d > 0), a = 2(2^31 - 1 - m) + 1 otherwise (d < 0).  The FP64 and BF16
// values are built as raw bits with 32-bit integer work (the GPU's FP64 pipe
// is narrow; an FP32 step before BF16 would round twice), the FP32 value by
// the hardware's integer-to-FP32 conversion; either way rounded to nearest
// even exactly once.
__device__ __forceinline__ uint32_t start_magnitude(uint32_t m, bool &neg)
{
    neg = (m & 0x80000000u) == 0u;
    return neg ? (((0x7fffffffu - m) << 1) | 1u) : (((m & 0x7fffffffu) << 1) | 1u);
}

// round the odd integer a (1 <= a < 2^32) to P+1 significant bits (nearest,
// ties to even) and return the IEEE fields of a * 2^-32 for a format with P
// stored mantissa bits and exponent bias B: every value here is normal
template <int P, int B>
__device__ __forceinline__ uint32_t encode_fields(uint32_t a, uint32_t &mant)
{
    int lead = 31 - __clz((int)a);                 // 2^lead <= a < 2^(lead+1)
    uint32_t q;
    if (lead <= P) {
        q = a << (P - lead);                       // exact
    } else {
        const int sh = lead - P;
        q = a >> sh;
        const uint32_t rem = a & ((1u << sh) - 1u), half = 1u << (sh - 1);
        if (rem > half || (rem == half && (q & 1u))) ++q;
        if (q == (2u << P)) { q = 1u << P; ++lead; }   // rounded up to the next power of two
    }
    mant = q - (1u << P);
    return (uint32_t)(lead - 32 + B);             // biased exponent
}

// raw bits of the start value of one component in the storage type
template <class TS> struct StartBits;
template <> struct StartBits<double> {
    using Raw = unsigned long long;
    __device__ __forceinline__ static Raw get(uint32_t m) {
        bool neg;
        const uint32_t a = start_magnitude(m, neg);    // < 2^32: exact in FP64
        const int lead = 31 - __clz((int)a);
        const unsigned long long mant = ((unsigned long long)a << (52 - lead)) & ((1ull << 52) - 1ull);
        const unsigned long long expo = (unsigned long long)(lead - 32 + 1023);
        return (neg ? (1ull << 63) : 0ull) | (expo << 52) | mant;
    }
};
template <> struct StartBits<float> {
    using Raw = uint32_t;
    // the odd integer d = 2m + 1 - 2^32 converted to FP32 by the hardware's
    // correctly rounded (nearest-even) integer conversion, then scaled by
    // 2^-32 exactly (|d| >= 1: every value is normal): the same single
    // rounding as the bit assembly of the other storages, in two instructions
    __device__ __forceinline__ static Raw get(uint32_t m) {
        const long long d = 2ll * (long long)m + 1ll - (1ll << 32);
        return __float_as_uint(__ll2float_rn(d) * 0x1p-32f);
    }
};
template <> struct StartBits<__nv_bfloat16> {
    using Raw = uint32_t;                               // low 16 bits used
    __device__ __forceinline__ static Raw get(uint32_t m) {
        bool neg;
        uint32_t mant;
        const uint32_t e = encode_fields<7, 127>(start_magnitude(m, neg), mant);
        return (neg ? 0x8000u : 0u) | (e << 7) | mant;
    }
};

// one thread per (row, block of 8 components): one Philox4x64-10 call gives
// 4 x 64 bits = 8 components of 32 bits (low half first).  Kp is a power of
// two; lq = log2(max(1, Kp / 8)).  Values are assembled as raw bits with
// integer operations and written with 16-byte stores (or per component for
// rows shorter than 8 components).
template <class TS>
__global__ void __launch_bounds__(kThreads) k_tv_init(InitArgs A, int lq)
{
    using SB = StartBits<TS>;
    const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const int64_t r = t >> lq;
    if (r >= A.n) return;
    const int q = (int)(t & ((1 << lq) - 1));
    const int64_t o = A.perm ? A.perm[r] : r;
    int lo = 0, hi = A.nmat;                 // matrix b with mat_off[b] <= o < mat_off[b+1]
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (A.mat_off[mid] <= o) lo = mid; else hi = mid;
    }
    const uint64_t li = (uint64_t)(o - A.mat_off[lo]);
    const uint64_t key1 = A.mat_id ? (uint64_t)A.mat_id[lo] : (uint64_t)lo;
    const U64x4 u = philox4x64_10(li, (uint64_t)q, 0ull, 0ull, A.seed, key1);
    typename SB::Raw v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const uint32_t m = (k & 1) ? (uint32_t)(u.v[k / 2] >> 32) : (uint32_t)u.v[k / 2];
        v[k] = 8 * q + k < A.K ? SB::get(m) : 0;     // padding: +0
    }
    TS *x = (TS *)A.x + r * A.Kp + 8 * q;
    if (A.Kp >= 8) {
        uint4 *x4 = reinterpret_cast<uint4 *>(x);
        if constexpr (sizeof(TS) == 2) {
            x4[0] = make_uint4(v[0] | (v[1] << 16), v[2] | (v[3] << 16), v[4] | (v[5] << 16),
                               v[6] | (v[7] << 16));
        } else if constexpr (sizeof(TS) == 4) {
            x4[0] = make_uint4(v[0], v[1], v[2], v[3]);
            x4[1] = make_uint4(v[4], v[5], v[6], v[7]);
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c)
                x4[c] = make_uint4((uint32_t)v[2 * c], (uint32_t)(v[2 * c] >> 32),
                                   (uint32_t)v[2 * c + 1], (uint32_t)(v[2 * c + 1] >> 32));
        }
    } else {
        typename SB::Raw *xr = reinterpret_cast<typename SB::Raw *>(x);
        if constexpr (sizeof(TS) == 2) {
            uint16_t *x16 = reinterpret_cast<uint16_t *>(x);
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (k < A.Kp) x16[k] = (uint16_t)v[k];
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (k < A.Kp) xr[k] = v[k];
        }
    }
}

template <class TS>
__global__ void k_import(const double *__restrict__ src, TS *__restrict__ x,
                         const int32_t *__restrict__ perm, int32_t n, int32_t K, int32_t Kp)
{
    const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (t >= (int64_t)n * Kp) return;
    const int64_t r = t / Kp;
    const int kappa = (int)(t % Kp);
    const int64_t o = perm ? perm[r] : r;
    x[t] = from_double<TS>(kappa < K ? src[o * K + kappa] : 0.0);
}

template <class TS>
__global__ void k_export(const TS *__restrict__ x, double *__restrict__ dst,
                         const int32_t *__restrict__ perm, int32_t n, int32_t K, int32_t Kp)
{
    const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (t >= (int64_t)n * K) return;
    const int64_t r = t / K;
    const int kappa = (int)(t % K);
    const int64_t o = perm ? perm[r] : r;
    dst[o * K + kappa] = to_double<TS>(x[r * Kp + kappa]);
}

template <class TF, class TT>
__global__ void k_convert(const TF *__restrict__ src, TT *__restrict__ dst, int64_t count)
{
    const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (t < count) dst[t] = from_double<TT>(to_double<TF>(src[t]));
}

template <class C>
__global__ void k_export_slots(const C *__restrict__ a_in, const C *__restrict__ ls_in,
                               double *__restrict__ a, double *__restrict__ dist,
                               double *__restrict__ ls, int64_t nnz)
{
    const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (t >= nnz) return;
    const double l = (double)ls_in[t];
    if (a) a[t] = (double)a_in[t];
    if (ls) ls[t] = l;
    if (dist) dist[t] = 1.0 / l;   // +inf for LS = 0, NaN stays NaN
}

__global__ void k_permute_values(const double *__restrict__ v, const int32_t *__restrict__ rp_orig,
                                 const int32_t *__restrict__ perm, const int32_t *__restrict__ rp_perm,
                                 double *__restrict__ vp64, float *__restrict__ vp32, int32_t n)
{
    const int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (r >= n) return;
    const int64_t o = perm ? perm[r] : r;
    const int64_t s = rp_orig[o], d = rp_perm[r];
    const int len = rp_orig[o + 1] - rp_orig[o];
    for (int k = 0; k < len; ++k) {
        const double x = v[s + k];
        if (vp64) vp64[d + k] = x;
        if (vp32) vp32[d + k] = (float)x;
    }
}

__global__ void k_unpermute(const uint4 *__restrict__ x, uint4 *__restrict__ xc,
                            const int32_t *__restrict__ perm, int32_t n, int32_t pieces)
{
    const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (t >= (int64_t)n * pieces) return;
    const int64_t r = t / pieces;
    const int q = (int)(t % pieces);
    xc[(int64_t)perm[r] * pieces + q] = x[t];
}

__global__ void k_diagonal(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                           const double *__restrict__ v, double *__restrict__ d64,
                           float *__restrict__ d32, int32_t n)
{
    const int64_t r = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (r >= n) return;
    double d = 0.0;
    for (int p = rp[r]; p < rp[r + 1]; ++p)
        if (col[p] == r) d = v[p];
    if (d64) d64[r] = d;
    if (d32) d32[r] = (float)d;
}

__global__ void k_check_values(const double *__restrict__ v, int64_t nnz,
                               const int32_t *__restrict__ diag_slot, int32_t n,
                               uint32_t *__restrict__ err)
{
    const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    uint32_t e = 0;
    if (t < nnz && !isfinite(v[t])) e |= 1u;
    if (t < n && v[diag_slot[t]] == 0.0) e |= 2u;
    e = __reduce_or_sync(0xffffffffu, e);
    if (e && (threadIdx.x % 32) == 0) atomicOr(err, e);
}

// one pass over the stored values in caller order (coalesced): the FP64
// caller copy, the FP32 caller copy and the row-permuted FP64 / FP32 copies
// (slot_perm[p] = permuted slot of caller slot p); NULL targets are skipped.
// err (NULL: no check): bit 0 set when a value is not finite.
__global__ void k_scatter_values(const double *__restrict__ src, int64_t nnz,
                                 const int32_t *__restrict__ slot_perm, double *__restrict__ val_o,
                                 float *__restrict__ val32_o, double *__restrict__ vp64,
                                 float *__restrict__ vp32, uint32_t *__restrict__ err)
{
    bool bad = false;
    for (int64_t p = (int64_t)blockIdx.x * kThreads + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * kThreads) {
        const double x = src[p];
        bad = bad || !isfinite(x);
        const float f = (float)x;
        if (val_o) val_o[p] = x;
        if (val32_o) val32_o[p] = f;
        const int64_t q = slot_perm ? slot_perm[p] : p;
        if (vp64) vp64[q] = x;
        if (vp32) vp32[q] = f;
    }
    if (err && __any_sync(0xffffffffu, bad) && (threadIdx.x % 32) == 0) atomicOr(err, 1u);
}

// diagonals in caller order and in permuted order (perm[r] = caller row of r);
// NULL targets are skipped.  err (NULL: no check): bit 1 set on a zero
// diagonal.
__global__ void k_diag_values(const double *__restrict__ v, const int32_t *__restrict__ diag_slot,
                              const int32_t *__restrict__ perm, int32_t n, double *__restrict__ d64_o,
                              float *__restrict__ d32_o, double *__restrict__ d64_p,
                              float *__restrict__ d32_p, uint32_t *__restrict__ err)
{
    const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    bool zero = false;
    if (t < n) {
        const double d = v[diag_slot[t]];
        zero = d == 0.0;
        if (d64_o) d64_o[t] = d;
        if (d32_o) d32_o[t] = (float)d;
        if (d64_p || d32_p) {
            const double dp = perm ? v[diag_slot[perm[t]]] : d;
            if (d64_p) d64_p[t] = dp;
            if (d32_p) d32_p[t] = (float)dp;
        }
    }
    if (err && __any_sync(0xffffffffu, zero) && (threadIdx.x % 32) == 0) atomicOr(err, 2u);
}

inline unsigned blocks(int64_t work) { return (unsigned)((work + kThreads - 1) / kThreads); }

// priority keys of the coarse-point selection: one Philox4x64-10 block per
// point, counter (i, stage, 1, 0) (word 2 = 1 keeps them apart from the
// test-vector draws), key (seed, 0); word 0 is the key
__global__ void k_cr_keys(int32_t n, int32_t stage, uint64_t seed, uint64_t *__restrict__ key)
{
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        key[i] = philox4x64_10((uint64_t)i, (uint64_t)stage, 1ull, 0ull, seed, 0ull).v[0];
}

}  // namespace

cudaError_t launch_cr_keys(int32_t n, int32_t stage, uint64_t seed, uint64_t *key, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_cr_keys<<<blocks(n), kThreads, 0, s>>>(n, stage, seed, key);
    return cudaGetLastError();
}

cudaError_t launch_init(int storage, const InitArgs &a, cudaStream_t s)
{
    if (a.Kp & (a.Kp - 1)) return cudaErrorInvalidValue;     // Kp is a power of two
    int lq = 0;
    while ((8 << lq) < a.Kp) ++lq;
    const int64_t work = (int64_t)a.n << lq;
    if (work == 0) return cudaSuccess;
    switch (storage) {
    case ST_FP64: k_tv_init<double><<<blocks(work), kThreads, 0, s>>>(a, lq); break;
    case ST_FP32: k_tv_init<float><<<blocks(work), kThreads, 0, s>>>(a, lq); break;
    case ST_BF16: k_tv_init<__nv_bfloat16><<<blocks(work), kThreads, 0, s>>>(a, lq); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_import(int storage, const double *src, void *x, const int32_t *perm,
                          int32_t n, int32_t K, int32_t Kp, cudaStream_t s)
{
    const int64_t work = (int64_t)n * Kp;
    if (work == 0) return cudaSuccess;
    switch (storage) {
    case ST_FP64: k_import<<<blocks(work), kThreads, 0, s>>>(src, (double *)x, perm, n, K, Kp); break;
    case ST_FP32: k_import<<<blocks(work), kThreads, 0, s>>>(src, (float *)x, perm, n, K, Kp); break;
    case ST_BF16:
        k_import<<<blocks(work), kThreads, 0, s>>>(src, (__nv_bfloat16 *)x, perm, n, K, Kp);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_export(int storage, const void *x, double *dst, const int32_t *perm,
                          int32_t n, int32_t K, int32_t Kp, cudaStream_t s)
{
    const int64_t work = (int64_t)n * K;
    if (work == 0) return cudaSuccess;
    switch (storage) {
    case ST_FP64:
        k_export<<<blocks(work), kThreads, 0, s>>>((const double *)x, dst, perm, n, K, Kp);
        break;
    case ST_FP32:
        k_export<<<blocks(work), kThreads, 0, s>>>((const float *)x, dst, perm, n, K, Kp);
        break;
    case ST_BF16:
        k_export<<<blocks(work), kThreads, 0, s>>>((const __nv_bfloat16 *)x, dst, perm, n, K, Kp);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

namespace {
template <class TF>
cudaError_t convert_to(const TF *src, int to, void *dst, int64_t count, cudaStream_t s)
{
    switch (to) {
    case ST_FP64: k_convert<<<blocks(count), kThreads, 0, s>>>(src, (double *)dst, count); break;
    case ST_FP32: k_convert<<<blocks(count), kThreads, 0, s>>>(src, (float *)dst, count); break;
    case ST_BF16:
        k_convert<<<blocks(count), kThreads, 0, s>>>(src, (__nv_bfloat16 *)dst, count);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_convert(int from, const void *src, int to, void *dst, int64_t count,
                           cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    switch (from) {
    case ST_FP64: return convert_to((const double *)src, to, dst, count, s);
    case ST_FP32: return convert_to((const float *)src, to, dst, count, s);
    case ST_BF16: return convert_to((const __nv_bfloat16 *)src, to, dst, count, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_export_slots(int storage, const void *a_in, const void *ls_in, double *a,
                                double *dist, double *ls, int64_t nnz, cudaStream_t s)
{
    if (nnz == 0) return cudaSuccess;
    if (storage == ST_FP64)
        k_export_slots<<<blocks(nnz), kThreads, 0, s>>>((const double *)a_in,
                                                        (const double *)ls_in, a, dist, ls, nnz);
    else
        k_export_slots<<<blocks(nnz), kThreads, 0, s>>>((const float *)a_in, (const float *)ls_in,
                                                        a, dist, ls, nnz);
    return cudaGetLastError();
}

cudaError_t launch_unpermute(int storage, const void *x, void *x_caller, const int32_t *perm,
                             int32_t n, int32_t Kp, cudaStream_t s)
{
    const int esz = storage == ST_FP64 ? 8 : (storage == ST_FP32 ? 4 : 2);
    const int32_t pieces = (int32_t)((int64_t)Kp * esz / 16);
    const int64_t work = (int64_t)n * pieces;
    if (work == 0) return cudaSuccess;
    k_unpermute<<<blocks(work), kThreads, 0, s>>>((const uint4 *)x, (uint4 *)x_caller, perm, n, pieces);
    return cudaGetLastError();
}

cudaError_t launch_diagonal(const int32_t *rp_perm, const int32_t *col_perm, const double *vp64,
                            double *d64, float *d32, int32_t n, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_diagonal<<<blocks(n), kThreads, 0, s>>>(rp_perm, col_perm, vp64, d64, d32, n);
    return cudaGetLastError();
}

cudaError_t launch_check_values(const double *v, int64_t nnz, const int32_t *diag_slot,
                                int32_t n, uint32_t *err, cudaStream_t s)
{
    const int64_t work = nnz > n ? nnz : n;
    if (work == 0) return cudaSuccess;
    k_check_values<<<blocks(work), kThreads, 0, s>>>(v, nnz, diag_slot, n, err);
    return cudaGetLastError();
}

cudaError_t launch_scatter_values(const double *src, int64_t nnz, const int32_t *slot_perm,
                                  double *val_o, float *val32_o, double *vp64, float *vp32,
                                  cudaStream_t s, uint32_t *err)
{
    if (nnz == 0) return cudaSuccess;
    const int64_t want = (nnz + kThreads - 1) / kThreads;
    k_scatter_values<<<(unsigned)(want < 152 * 16 ? want : 152 * 16), kThreads, 0, s>>>(
        src, nnz, slot_perm, val_o, val32_o, vp64, vp32, err);
    return cudaGetLastError();
}

cudaError_t launch_diag_values(const double *v, const int32_t *diag_slot, const int32_t *perm,
                               int32_t n, double *d64_o, float *d32_o, double *d64_p, float *d32_p,
                               cudaStream_t s, uint32_t *err)
{
    if (n == 0) return cudaSuccess;
    k_diag_values<<<blocks(n), kThreads, 0, s>>>(v, diag_slot, perm, n, d64_o, d32_o, d64_p, d32_p,
                                                err);
    return cudaGetLastError();
}

cudaError_t launch_permute_values(const double *v, const int32_t *rp_orig, const int32_t *perm,
                                  const int32_t *rp_perm, double *vp64, float *vp32, int32_t n,
                                  cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_permute_values<<<blocks(n), kThreads, 0, s>>>(v, rp_orig, perm, rp_perm, vp64, vp32, n);
    return cudaGetLastError();
}

}  // namespace amgd
