// k_cr.cu -- compatible-relaxation coarsening (§3.2 Eqs. (3.4), (3.5); §4.2
// Eq. (4.4); Algorithm 1 and the candidate measure of the Remark after it).
//
// One stage, all on the device except the scalar decision of Algorithm 1's
// loop: F-relaxation of one vector from the constant start with the coarse
// rows held at zero (on the color-ordered copy of A that the test-vector
// sweeps use, so a color phase is one contiguous range of rows), the max norm
// of the result (exact: a maximum of bit patterns), the candidates
// sigma_i = |u_i| / ||u|| > tol, the strength graph restricted to F, and an
// independent set of the candidates.  The set is the greedy set in a fixed
// priority order (more candidates depending strongly on the point first, then
// a Philox key, then the smaller index); it is reached by rounds of local
// maxima, which select exactly the points the greedy order selects, so the
// result does not depend on the thread schedule.
//
// Rounding follows the sweeps of the test vectors: a row sum is a chain of
// fused multiply-adds in CSR order and the update is x_i - (omega/a_ii) s as
// one fused multiply-add, so the F-relaxation is bit-exact with a sequential
// FP64 evaluation in the same order.
#include "amgd_internal.cuh"

namespace amgd {
namespace {

constexpr int kThreads = 256;

int grid_for(int64_t n)
{
    const int64_t b = (n + kThreads - 1) / kThreads;
    return (int)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

// coarse mask into color order, u = 1 on F, 0 on C
__global__ void k_cr_start(const int32_t *__restrict__ perm, const uint8_t *__restrict__ coarse,
                           uint8_t *__restrict__ coarse_p, double *__restrict__ u, int32_t n)
{
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const uint8_t c = coarse[perm ? perm[r] : r];
        coarse_p[r] = c;
        u[r] = c ? 0.0 : 1.0;
    }
}

// The row weight omega / a_rr is the same correctly rounded quotient in every
// sweep, so it is formed once per call rather than per sweep: on this part a
// double division costs about as much as the row's sum.
__global__ void k_cr_cdiag(const double *__restrict__ diag, double omega,
                           double *__restrict__ cdiag, int32_t n)
{
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
        cdiag[r] = omega / diag[r];
}

// one F-relaxation phase over the color-ordered rows [r0, r1): weighted
// Jacobi (r0 = 0, r1 = n, every neighbour from u), or one color of a
// multicolor Gauss-Seidel sweep (neighbours of earlier colors -- rows below
// r0 -- from un, all others from u).  Coarse rows stay 0 (Eq. (3.4)).
__global__ void k_cr_sweep(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                           const double *__restrict__ val, const double *__restrict__ cdiag,
                           const uint8_t *__restrict__ coarse_p, int32_t r0, int32_t r1,
                           const double *__restrict__ u, double *un)
{
    for (int32_t r = r0 + blockIdx.x * blockDim.x + threadIdx.x; r < r1;
         r += gridDim.x * blockDim.x) {
        if (coarse_p[r]) { un[r] = 0.0; continue; }
        const double c = cdiag[r];
        double acc = 0.0;
        const int32_t e = rp[r + 1];
        for (int32_t p = rp[r]; p < e; ++p) {
            const int32_t j = col[p];
            acc = fma(val[p], j < r0 ? un[j] : u[j], acc);
        }
        un[r] = fma(-c, acc, u[r]);
    }
}

// scal[0] = bits of max_{i in F} |u_i| (non-negative doubles order like their
// bit patterns), scal[1] = |F|
__global__ void k_cr_norm(const double *__restrict__ u, const uint8_t *__restrict__ coarse,
                          int32_t n, unsigned long long *scal)
{
    unsigned long long m = 0ull, cnt = 0ull;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (coarse[i]) continue;
        const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(u[i]));
        m = b > m ? b : m;
        ++cnt;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long mo = __shfl_xor_sync(0xffffffffu, m, o);
        m = mo > m ? mo : m;
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    __shared__ unsigned long long sm[kThreads / 32], sc[kThreads / 32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { sm[w] = m; sc[w] = cnt; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < kThreads / 32; ++k) {
            m = sm[k] > m ? sm[k] : m;
            cnt += sc[k];
        }
        if (m) atomicMax(&scal[0], m);
        if (cnt) atomicAdd(&scal[1], cnt);
    }
}

// candidates (state 1, caller order) from the color-ordered u; cleared
// counters; every candidate starts as a possible local maximum
__global__ void k_cr_cand(const double *__restrict__ u, const uint8_t *__restrict__ coarse_p,
                          const int32_t *__restrict__ perm,
                          const unsigned long long *__restrict__ scal, double tol,
                          uint8_t *__restrict__ state, uint8_t *__restrict__ ismax,
                          int32_t *__restrict__ lam, int32_t n)
{
    const double unorm = __longlong_as_double((long long)scal[0]);
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const int32_t i = perm ? perm[r] : r;
        const uint8_t z = (!coarse_p[r] && fabs(u[r]) / unorm > tol) ? 1 : 0;
        state[i] = z;
        ismax[i] = z;
        lam[i] = 0;
    }
}

// strength graph on F (Eq. (4.4) with i, j in F and the minimum LS over the
// F neighbours), and lambda_j += 1 for every strong (i, j) between candidates
__global__ void k_cr_strength(const int32_t *__restrict__ prp, const int32_t *__restrict__ pcol,
                              const double *__restrict__ ls, const uint8_t *__restrict__ coarse,
                              const uint8_t *__restrict__ state, double theta,
                              uint8_t *__restrict__ strong, int32_t *lam, int32_t n)
{
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int32_t b = prp[i], e = prp[i + 1];
        if (coarse[i]) {
            for (int32_t q = b; q < e; ++q) strong[q] = 0;
            continue;
        }
        double m = __longlong_as_double(0x7ff0000000000000ll);   // +inf
        for (int32_t q = b; q < e; ++q) {
            const int32_t j = pcol[q];
            if (j != i && !coarse[j] && ls[q] < m) m = ls[q];
        }
        const bool zi = state[i] == 1;
        for (int32_t q = b; q < e; ++q) {
            const int32_t j = pcol[q];
            const double l = ls[q];
            const bool s = j != i && !coarse[j] && (l == 0.0 || theta * l < m);
            strong[q] = s;
            if (s && zi && state[j] == 1) atomicAdd(&lam[j], 1);
        }
    }
}

__device__ __forceinline__ bool cr_before(int32_t la, uint64_t ka, int32_t a, int32_t lb,
                                          uint64_t kb, int32_t b)
{
    if (la != lb) return la > lb;
    if (ka != kb) return ka > kb;
    return a < b;
}

// of every strong pair of undecided points the later one in the order is not
// a local maximum (each pair is seen from the row that stores the slot)
__global__ void k_mis_compare(const int32_t *__restrict__ prp, const int32_t *__restrict__ pcol,
                              const uint8_t *__restrict__ strong, const uint8_t *__restrict__ state,
                              const int32_t *__restrict__ lam, const uint64_t *__restrict__ key,
                              uint8_t *ismax, int32_t n)
{
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (state[i] != 1) continue;
        const int32_t li = lam[i];
        const uint64_t ki = key[i];
        const int32_t e = prp[i + 1];
        for (int32_t q = prp[i]; q < e; ++q) {
            if (!strong[q]) continue;
            const int32_t j = pcol[q];
            if (state[j] != 1) continue;
            if (cr_before(li, ki, i, lam[j], key[j], j)) ismax[j] = 0;
            else ismax[i] = 0;
        }
    }
}

__global__ void k_mis_select(uint8_t *__restrict__ state, const uint8_t *__restrict__ ismax, int32_t n)
{
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (state[i] == 1 && ismax[i]) state[i] = 2;
}

// undecided neighbours of selected points (either direction) leave the set.
// Selected points (2) are never written: two strong neighbours are never both
// selected, so only 1 -> 0 transitions race, and they write the same value.
// A point that finds no selected out-neighbour re-arms its local-maximum flag
// for the next round (if a selected in-neighbour removes it meanwhile, the
// flag is ignored: the next rounds only read it for undecided points).
__global__ void k_mis_remove(const int32_t *__restrict__ prp, const int32_t *__restrict__ pcol,
                             const uint8_t *__restrict__ strong, uint8_t *state,
                             uint8_t *__restrict__ ismax, int32_t n)
{
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint8_t st = state[i];
        if (st == 0) continue;
        const int32_t e = prp[i + 1];
        bool removed = false;
        for (int32_t q = prp[i]; q < e; ++q) {
            if (!strong[q]) continue;
            const int32_t j = pcol[q];
            if (st == 2) {
                if (state[j] == 1) state[j] = 0;
            } else if (state[j] == 2) {
                state[i] = 0;
                removed = true;
                break;
            }
        }
        if (st == 1 && !removed) ismax[i] = 1;
    }
}

__global__ void k_cr_count(const uint8_t *__restrict__ state, int32_t n, unsigned long long *out)
{
    unsigned long long cnt = 0ull;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        cnt += state[i] == 1;
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(out, cnt);
}

__global__ void k_cr_add(const uint8_t *__restrict__ state, const int32_t *__restrict__ perm,
                         uint8_t *__restrict__ coarse, uint8_t *__restrict__ coarse_p, int32_t n)
{
    for (int32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const int32_t i = perm ? perm[r] : r;
        if (state[i] == 2) {
            coarse[i] = 1;
            coarse_p[r] = 1;
        }
    }
}

}  // namespace

cudaError_t launch_cr_start(const CrArgs &a, double *u, cudaStream_t s)
{
    k_cr_start<<<grid_for(a.n), kThreads, 0, s>>>(a.perm, a.coarse, a.coarse_p, u, a.n);
    return cudaGetLastError();
}

cudaError_t launch_cr_cdiag(const CrArgs &a, cudaStream_t s)
{
    k_cr_cdiag<<<grid_for(a.n), kThreads, 0, s>>>(a.diag, a.omega, a.cdiag, a.n);
    return cudaGetLastError();
}

cudaError_t launch_cr_sweep(const CrArgs &a, bool mcgs, const int64_t *color_start,
                            int32_t ncolors, const double *u, double *un, cudaStream_t s)
{
    if (!mcgs) {
        k_cr_sweep<<<grid_for(a.n), kThreads, 0, s>>>(a.rp, a.col, a.val, a.cdiag, a.coarse_p, 0,
                                                      a.n, u, un);
        return cudaGetLastError();
    }
    for (int32_t cc = 0; cc < ncolors; ++cc) {
        const int32_t r0 = (int32_t)color_start[cc], r1 = (int32_t)color_start[cc + 1];
        if (r1 <= r0) continue;
        k_cr_sweep<<<grid_for(r1 - r0), kThreads, 0, s>>>(a.rp, a.col, a.val, a.cdiag, a.coarse_p,
                                                         r0, r1, u, un);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_cr_norm(const double *u, const uint8_t *coarse_p, int32_t n,
                           unsigned long long *scal, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(scal, 0, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_cr_norm<<<grid_for(n), kThreads, 0, s>>>(u, coarse_p, n, scal);
    return cudaGetLastError();
}

cudaError_t launch_cr_candidates(const CrArgs &a, const double *u, double tol, cudaStream_t s)
{
    const int g = grid_for(a.n);
    k_cr_cand<<<g, kThreads, 0, s>>>(u, a.coarse_p, a.perm, a.scal, tol, a.state, a.ismax, a.lam,
                                     a.n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_cr_strength<<<g, kThreads, 0, s>>>(a.prp, a.pcol, a.ls, a.coarse, a.state, a.theta, a.strong,
                                         a.lam, a.n);
    return cudaGetLastError();
}

cudaError_t launch_cr_mis_rounds(const CrArgs &a, int32_t rounds, cudaStream_t s)
{
    const int g = grid_for(a.n);
    for (int32_t r = 0; r < rounds; ++r) {
        k_mis_compare<<<g, kThreads, 0, s>>>(a.prp, a.pcol, a.strong, a.state, a.lam, a.key, a.ismax,
                                             a.n);
        k_mis_select<<<g, kThreads, 0, s>>>(a.state, a.ismax, a.n);
        k_mis_remove<<<g, kThreads, 0, s>>>(a.prp, a.pcol, a.strong, a.state, a.ismax, a.n);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(a.scal + 2, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_cr_count<<<g, kThreads, 0, s>>>(a.state, a.n, a.scal + 2);
    return cudaGetLastError();
}

cudaError_t launch_cr_add(const CrArgs &a, cudaStream_t s)
{
    k_cr_add<<<grid_for(a.n), kThreads, 0, s>>>(a.state, a.perm, a.coarse, a.coarse_p, a.n);
    return cudaGetLastError();
}

}  // namespace amgd
