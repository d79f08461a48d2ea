/*
 * amgd_oracle.c -- plain, slow, FP64 CPU oracle for the algebraic-distance
 * strength-of-connection build of Brandt, Brannick, Kahl and Livshits,
 * "An algebraic distances measure of AMG strength of connection".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  The product path (the
 * CUDA library and its Python binding) never calls it, links it or shares
 * a line of code, a header or a constant table with it.
 *
 * What it computes, step by step (one row at a time, CSR order):
 *   1. test vectors X0: Philox4x64-10 counter-based random numbers mapped
 *      to uniform(-1,1), 32 bits per element      (§3: relax Ax=0 from random
 *                                                 starting vectors)
 *   2. nu relaxation sweeps on A x = 0: weighted Jacobi, or multicolor
 *      Gauss-Seidel with snapshot semantics      (§3, §2: Gauss-Seidel)
 *   3. the LS target y_i: plain x_i (Eq. (3.1)) or the residual-corrected
 *      x_i - r_i / a_ii with r = A x (Eqs. (3.2), (4.1), (4.3))
 *   4. per stored off-diagonal (i,j): the one-point LS fit p_ij and the
 *      minimal functional LS_ij; algebraic distance r_ij = 1/LS_ij
 *                                                 (§4.1, Eq. (4.3))
 *   5. row-relative threshold r_ij > theta * max_k r_ik  (§4.2, Eq. (4.4))
 *   6. the strength graph as CSR                  (§4.2)
 *   7. (extension) the reverse pass of steps 2-5 for Jacobi sweeps: the
 *      gradient of a loss on LS with respect to A's values, omega and X0
 *   8. search depth d > 1: the graph G_d of A^d from the graph of A, and the
 *      fits of step 4 over its entries (§4.1, Eq. (4.2); §4.2)
 *   9. (extension) least-squares interpolation of a given caliber over sets
 *      of coarse points, with the size penalty gamma (§4.3)
 *  10. compatible-relaxation coarsening: F-relaxation, the convergence
 *      estimate, candidates and independent sets of the strength graph on F
 *      (§3.2, §4.2, Algorithm 1)
 *
 * Rounding conventions (the paper fixes none): every multiply-accumulate of
 * a row sum is one fused multiply-add (C99 fma, a single rounding), sums run
 * in CSR order (row sums) or in test-vector order (LS sums), and the update
 * x_i - c_i * s is one fused multiply-add with c_i = omega / a_ii.  All other
 * operations are plain IEEE double operations; the file is compiled with
 * -ffp-contract=off so the compiler adds no fusion of its own.
 *
 * Parity pins (see tests/): Philox against numpy's Philox4x64-10; sweeps
 * against dense matrix powers and a triangular solve; LS against a library
 * least-squares solve, brute-force minimisation, its normal equation and
 * closed forms (exact fits, scaling, integer weights as repeated vectors);
 * the reverse pass against central finite differences; G_d against 0/1
 * matrix powers; interpolation against brute force over all subsets; CR
 * stages against dense powers, numpy's Philox and parallel local-maximum
 * rounds, its estimate against the spectral radius and the closed form
 * |1 - omega| of a red-black split; the stencil generators against the
 * worked stencils S_A and S~_xy of §5.1.  Every function has a pin; planted
 * mistakes in a copy of this file must each fail one (test_oracle_mutants).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* 1. Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:  */
/*    as easy as 1, 2, 3", SC'11).  Multipliers and Weyl key increments are */
/*    the ones published for the 4x64 variant.                              */
/* ------------------------------------------------------------------------ */
static void orc_mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t hi0, lo0, hi1, lo1;
        orc_mulhilo64(M0, c0, &hi0, &lo0);
        orc_mulhilo64(M1, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        uint64_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/*
 * Test vectors X0 (n x K, row-major): §3 starts each test vector from a
 * random vector before relaxing A x = 0.  Element (i, kappa) takes the
 * 32-bit half (kappa mod 2; 0 = low half) of word ((kappa / 2) mod 4) of
 * Philox4x64-10 at counter (i, kappa / 8, 0, 0) and key (seed, stream): with
 * that 32-bit integer m, x = (2m + 1) 2^-32 - 1, the midpoint of the m-th of
 * 2^32 equal cells of (-1, 1).  Exact in double precision.
 * stream distinguishes the matrices of a batch (0 for a single matrix).
 */
void orc_tv_init(int64_t n, int32_t K, uint64_t seed, uint64_t stream, double *X)
{
    const uint64_t key[2] = {seed, stream};
    for (int64_t i = 0; i < n; ++i) {
        for (int32_t kappa = 0; kappa < K; ++kappa) {
            uint64_t ctr[4] = {(uint64_t)i, (uint64_t)(kappa / 8), 0, 0};
            uint64_t out[4];
            orc_philox4x64_10(ctr, key, out);
            uint64_t word = out[(kappa / 2) % 4];
            uint64_t m = (kappa % 2 == 0) ? (word & 0xffffffffULL) : (word >> 32);
            X[i * K + kappa] = ((double)(2 * m + 1)) * 0x1.0p-32 - 1.0;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Input checks.  A is the graph G=(V,E) of §4.1: (i,j) in E iff a_ij != 0, */
/* stored as CSR with an explicit, nonzero diagonal in every row.           */
/* Returns 0, or: 1 bad row_ptr, 2 column out of range, 3 duplicate (i,j),  */
/* 4 missing or zero diagonal, 5 non-finite value.                          */
/* ------------------------------------------------------------------------ */
int orc_check_csr(int64_t n, const int64_t *rp, const int32_t *col, const double *val)
{
    if (n < 0) return 1;
    if (rp[0] != 0) return 1;
    for (int64_t i = 0; i < n; ++i)
        if (rp[i + 1] < rp[i]) return 1;
    for (int64_t i = 0; i < n; ++i) {
        int have_diag = 0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            if (col[p] < 0 || (int64_t)col[p] >= n) return 2;
            if (!isfinite(val[p])) return 5;
            for (int64_t q = rp[i]; q < p; ++q)
                if (col[q] == col[p]) return 3;
            if (col[p] == i) {
                if (val[p] == 0.0) return 4;
                have_diag = 1;
            }
        }
        if (!have_diag) return 4;
    }
    return 0;
}

static double orc_diag(const int64_t *rp, const int32_t *col, const double *val, int64_t i)
{
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
        if (col[p] == i) return val[p];
    return NAN; /* unreachable for checked input */
}

/* ------------------------------------------------------------------------ */
/* 2. Relaxation of the homogeneous system A x = 0 (§3: "relaxing the       */
/*    homogeneous system Ax=0 with a different starting vector").           */
/* ------------------------------------------------------------------------ */

/*
 * One weighted-Jacobi sweep on all K vectors at once:
 *   x_i <- x_i - (omega / a_ii) * sum_p a_{i,col_p} x_{col_p}
 * using only the values from before the sweep.
 */
void orc_jacobi_sweep(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                      int32_t K, double omega, const double *X, double *Xn)
{
    for (int64_t i = 0; i < n; ++i) {
        double c = omega / orc_diag(rp, col, val, i);
        for (int32_t kappa = 0; kappa < K; ++kappa) {
            double s = 0.0;
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
                s = fma(val[p], X[(int64_t)col[p] * K + kappa], s);
            Xn[i * K + kappa] = fma(-c, s, X[i * K + kappa]);
        }
    }
}

/*
 * One multicolor Gauss-Seidel sweep (§2 names Gauss-Seidel as the smoother
 * and §5.2 relaxes the test vectors with it).  Colors are processed in
 * increasing order.  A row of color c is updated from the new values of
 * rows of smaller colors and the values from the start of the sweep of all
 * other rows, itself included ("snapshot" semantics: for a proper coloring
 * this is Gauss-Seidel in color order; when same-colored rows touch, they
 * see each other's old values).  omega is the over-relaxation weight
 * (1 = plain Gauss-Seidel).
 */
void orc_mcgs_sweep(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                    const int32_t *color, int32_t ncolors, int32_t K, double omega,
                    const double *X, double *Xn)
{
    memcpy(Xn, X, (size_t)n * (size_t)K * sizeof(double));
    for (int32_t c = 0; c < ncolors; ++c) {
        for (int64_t i = 0; i < n; ++i) {
            if (color[i] != c) continue;
            double ci = omega / orc_diag(rp, col, val, i);
            for (int32_t kappa = 0; kappa < K; ++kappa) {
                double s = 0.0;
                for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
                    int64_t j = col[p];
                    double xj = (color[j] < c) ? Xn[j * K + kappa] : X[j * K + kappa];
                    s = fma(val[p], xj, s);
                }
                Xn[i * K + kappa] = fma(-ci, s, X[i * K + kappa]);
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* 3. LS target.                                                            */
/*   mode 0 (residual-corrected, default): y_i = x_i - r_i / a_ii, r = A x  */
/*          -- the target of Eqs. (3.2), (4.1) and (4.3); the Remark in     */
/*          §3.1 identifies it with one local Jacobi step, and with         */
/*          omega = 1 it equals one orc_jacobi_sweep bit for bit.           */
/*   mode 1 (plain): y_i = x_i -- the target of Eq. (3.1).                  */
/* ------------------------------------------------------------------------ */
void orc_target(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                int32_t K, int32_t mode, const double *X, double *Y)
{
    if (mode == 1) {
        memcpy(Y, X, (size_t)n * (size_t)K * sizeof(double));
        return;
    }
    orc_jacobi_sweep(n, rp, col, val, K, 1.0, X, Y);
}

/* ------------------------------------------------------------------------ */
/* 4. One-point least squares per stored off-diagonal (§4.1, Eq. (4.3)):    */
/*   LS_ij(p) = sum_kappa w_kappa (y_i^k - p x_j^k)^2, p_ij its minimiser,  */
/*   r_ij = 1 / LS_ij(p_ij).  With S_xx = sum w x_j^2 and S_yx = sum w y x_j */
/*   the minimiser is p = S_yx / S_xx (S_xx = 0: every p is a minimiser;   */
/*   p = 0 is taken, LS = sum w y^2).  LS is evaluated as the weighted sum */
/*   of squared residuals at p (two passes over the K vectors).            */
/*   Residual-corrected target with exactly one off-diagonal in row i:     */
/*   y_i = -(a_ij / a_ii) x_j holds exactly, so p = -a_ij/a_ii and LS = 0  */
/*   are returned rather than a rounding residue.                          */
/*   Diagonal slots get a = 0, ls = NaN.  Outputs are aligned with A's CSR */
/*   slots.                                                                */
/* ------------------------------------------------------------------------ */
void orc_edge_ls(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                 int32_t K, const double *w, int32_t mode, const double *X, const double *Y,
                 double *a, double *ls)
{
    for (int64_t i = 0; i < n; ++i) {
        int64_t off = 0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
            if (col[p] != i) ++off;
        double aii = orc_diag(rp, col, val, i);
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            int64_t j = col[p];
            if (j == i) {
                a[p] = 0.0;
                ls[p] = NAN;
                continue;
            }
            if (mode == 0 && off == 1) {
                a[p] = -val[p] / aii;
                ls[p] = 0.0;
                continue;
            }
            const double *y = Y + i * K;
            const double *x = X + j * K;
            double sxx = 0.0, syx = 0.0;
            for (int32_t kappa = 0; kappa < K; ++kappa) {
                sxx += w[kappa] * x[kappa] * x[kappa];
                syx += w[kappa] * y[kappa] * x[kappa];
            }
            double pij = (sxx == 0.0) ? 0.0 : syx / sxx;
            double res = 0.0;
            for (int32_t kappa = 0; kappa < K; ++kappa) {
                double e = y[kappa] - pij * x[kappa];
                res += w[kappa] * e * e;
            }
            a[p] = pij;
            ls[p] = res;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* 5. Strength graph (§4.2, Eq. (4.4)): keep (i,j) iff                      */
/*      r_ij > theta * max_k r_ik,  k over the off-diagonals of row i.      */
/*   With r = 1/LS and m_i = min_k LS_ik this is LS_ij = 0 (r = +inf is     */
/*   always kept) or theta * LS_ij < m_i; evaluated in LS form so that no   */
/*   division by zero occurs.  The comparison is strict.                    */
/*   count[i] = number of kept slots of row i.                              */
/* ------------------------------------------------------------------------ */
void orc_threshold(int64_t n, const int64_t *rp, const int32_t *col, const double *ls,
                   double theta, uint8_t *flag, int64_t *count)
{
    for (int64_t i = 0; i < n; ++i) {
        double m = INFINITY;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
            if (col[p] != i && ls[p] < m) m = ls[p];
        int64_t cnt = 0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            int strong = 0;
            if (col[p] != i)
                strong = (ls[p] == 0.0) || (theta * ls[p] < m);
            flag[p] = (uint8_t)strong;
            cnt += strong;
        }
        count[i] = cnt;
    }
}

/* 6. The strength graph M^1 as CSR: kept slots, rows in order, CSR order  */
/*    within a row.  Returns the number of kept edges.                      */
int64_t orc_strength_csr(int64_t n, const int64_t *rp, const int32_t *col, const uint8_t *flag,
                         int64_t *s_rp, int32_t *s_col)
{
    int64_t k = 0;
    s_rp[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
            if (flag[p]) s_col[k++] = col[p];
        s_rp[i + 1] = k;
    }
    return k;
}

/* ------------------------------------------------------------------------ */
/* 7. Reverse pass.  The paper differentiates nothing; this is the chain    */
/*    rule applied to steps 2-5 for weighted-Jacobi sweeps, written out     */
/*    term by term.  Forward:                                               */
/*      X_{s+1} = X_s - omega D^{-1} A X_s          (s = 0 .. nu-1)         */
/*      Y       = X_nu - D^{-1} A X_nu  (mode 0)    or Y = X_nu (mode 1)    */
/*      a_p, LS_p from (y_i, x_j) per off-diagonal slot p = (i,j)           */
/*    and a scalar loss L(LS) whose gradient ls_bar = dL/dLS is given, or   */
/*    (ls_bar == NULL) L = sum of r_p^2 = LS_p^-2 over the slots the        */
/*    threshold keeps with LS_p > 0 (the kept set is held fixed).          */
/*    Since a_p minimises LS_p(a), dLS_p/da_p = 0 there and                 */
/*      dLS_p/dy_i = 2 w (y_i - a_p x_j),  dLS_p/dx_j = -2 w a_p (y_i - a_p x_j). */
/*    LS_p of a one-off-diagonal row in mode 0 is the constant 0: no        */
/*    gradient flows through it.  A diagonal value a_ii enters both A and   */
/*    D; val_bar holds the sum of both contributions.                       */
/*    Outputs: val_bar (nnz, aligned with A's slots), omega_bar, loss (only */
/*    for the built-in loss), x0_bar (n*K, may be NULL).  Returns 0, or -5  */
/*    when memory runs out.                                                 */
/* ------------------------------------------------------------------------ */
int orc_adjoint_jacobi(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                       int32_t K, const double *w, int32_t mode, const double *X0, int32_t nu,
                       double omega, double theta, const double *ls_bar, double *val_bar,
                       double *omega_bar, double *loss, double *x0_bar)
{
    const int64_t nnz = rp[n];
    const size_t nk = (size_t)n * (size_t)K;
    double *Xs = (double *)malloc((size_t)(nu + 1) * nk * sizeof(double) + 1);
    double *Y = (double *)malloc(nk * sizeof(double) + 1);
    double *Ybar = (double *)calloc(nk + 1, sizeof(double));
    double *Xbar = (double *)calloc(nk + 1, sizeof(double));
    double *Xnext = (double *)malloc(nk * sizeof(double) + 1);
    double *a = (double *)malloc((size_t)nnz * sizeof(double) + 1);
    double *ls = (double *)malloc((size_t)nnz * sizeof(double) + 1);
    double *lsb = (double *)calloc((size_t)nnz + 1, sizeof(double));
    uint8_t *flag = (uint8_t *)malloc((size_t)nnz + 1);
    int64_t *count = (int64_t *)malloc((size_t)n * sizeof(int64_t) + 1);
    int rc = 0;
    if (!Xs || !Y || !Ybar || !Xbar || !Xnext || !a || !ls || !lsb || !flag || !count) {
        rc = -5;
        goto done;
    }

    /* forward, keeping every iterate */
    memcpy(Xs, X0, nk * sizeof(double));
    for (int32_t s = 0; s < nu; ++s)
        orc_jacobi_sweep(n, rp, col, val, K, omega, Xs + (size_t)s * nk, Xs + (size_t)(s + 1) * nk);
    const double *Xnu = Xs + (size_t)nu * nk;
    orc_target(n, rp, col, val, K, mode, Xnu, Y);
    orc_edge_ls(n, rp, col, val, K, w, mode, Xnu, Y, a, ls);
    orc_threshold(n, rp, col, ls, theta, flag, count);

    /* upstream gradient dL/dLS */
    double L = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t off = 0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
            if (col[p] != i) ++off;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            if (col[p] == i || (mode == 0 && off == 1)) continue;
            if (ls_bar) {
                lsb[p] = ls_bar[p];
            } else if (flag[p] && ls[p] > 0.0) {
                L += 1.0 / (ls[p] * ls[p]);
                lsb[p] = -2.0 / (ls[p] * ls[p] * ls[p]);
            }
        }
    }
    if (loss) *loss = ls_bar ? NAN : L;

    /* through the one-point fits: Ybar and the direct part of Xbar(nu) */
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            int64_t j = col[p];
            if (j == i || lsb[p] == 0.0) continue;
            for (int32_t kappa = 0; kappa < K; ++kappa) {
                double e = Y[i * K + kappa] - a[p] * Xnu[j * K + kappa];
                Ybar[i * K + kappa] += lsb[p] * 2.0 * w[kappa] * e;
                Xbar[j * K + kappa] += -lsb[p] * 2.0 * w[kappa] * a[p] * e;
            }
        }
    }

    for (int64_t p = 0; p < nnz; ++p) val_bar[p] = 0.0;
    double wbar = 0.0;

    /* through the target */
    if (mode == 1) {
        for (size_t q = 0; q < nk; ++q) Xbar[q] += Ybar[q];
    } else {
        for (int64_t i = 0; i < n; ++i) {
            double aii = orc_diag(rp, col, val, i);
            int64_t pd = -1;
            double yr = 0.0;                 /* <Ybar_i, (A X_nu)_i> */
            for (int32_t kappa = 0; kappa < K; ++kappa) {
                double r = 0.0;
                for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
                    r += val[p] * Xnu[(int64_t)col[p] * K + kappa];
                yr += Ybar[i * K + kappa] * r;
                Xbar[i * K + kappa] += Ybar[i * K + kappa];
            }
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
                int64_t j = col[p];
                if (j == i) pd = p;
                double g = 0.0;              /* <Ybar_i, X_nu,j> */
                for (int32_t kappa = 0; kappa < K; ++kappa) {
                    g += Ybar[i * K + kappa] * Xnu[j * K + kappa];
                    Xbar[j * K + kappa] -= (val[p] / aii) * Ybar[i * K + kappa];
                }
                val_bar[p] -= g / aii;
            }
            val_bar[pd] += yr / (aii * aii);
        }
    }

    /* through the sweeps, last to first: Xbar holds Xbar(s+1) on entry */
    for (int32_t s = nu - 1; s >= 0; --s) {
        const double *Xc = Xs + (size_t)s * nk;
        memcpy(Xnext, Xbar, nk * sizeof(double));   /* Xbar(s+1) */
        for (int64_t i = 0; i < n; ++i) {
            double aii = orc_diag(rp, col, val, i);
            int64_t pd = -1;
            double xr = 0.0;                 /* <Xbar_i(s+1), (A X_s)_i> */
            for (int32_t kappa = 0; kappa < K; ++kappa) {
                double r = 0.0;
                for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
                    r += val[p] * Xc[(int64_t)col[p] * K + kappa];
                xr += Xnext[i * K + kappa] * r;
            }
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
                int64_t j = col[p];
                if (j == i) pd = p;
                double g = 0.0;              /* <Xbar_i(s+1), X_s,j> */
                for (int32_t kappa = 0; kappa < K; ++kappa) {
                    g += Xnext[i * K + kappa] * Xc[j * K + kappa];
                    Xbar[j * K + kappa] -= omega * (val[p] / aii) * Xnext[i * K + kappa];
                }
                val_bar[p] -= omega * g / aii;
            }
            val_bar[pd] += omega * xr / (aii * aii);
            wbar -= xr / aii;
        }
    }
    if (omega_bar) *omega_bar = wbar;
    if (x0_bar) memcpy(x0_bar, Xbar, nk * sizeof(double));

done:
    free(Xs); free(Y); free(Ybar); free(Xbar); free(Xnext);
    free(a); free(ls); free(lsb); free(flag); free(count);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* 8. Search depth d > 1 (§4.1, Eq. (4.2); §4.2: the strength graph M^d).  */
/*    V_i = { j : (A^d)_ij != 0 }, taken structurally (no numerical       */
/*    cancellation) and built from the graph of A alone, as the Remark of  */
/*    §4.2 suggests: j is in V_i iff a walk of length d joins i and j in   */
/*    the graph of A.  Every row of A holds its diagonal, so walks may     */
/*    pause and V_i is the set of vertices within d steps of i (i itself   */
/*    included).  Columns of a row are listed in ascending order.          */
/*    out_col may be NULL (count only); returns the number of entries, or  */
/*    -5 when memory runs out.                                             */
/* ------------------------------------------------------------------------ */
static int orc_cmp_i32(const void *a, const void *b)
{
    const int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

int64_t orc_distance_graph(int64_t n, const int64_t *rp, const int32_t *col, int32_t d,
                           int64_t *out_rp, int32_t *out_col)
{
    int64_t *seen = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int32_t *list = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!seen || !list) {
        free(seen);
        free(list);
        return -5;
    }
    for (int64_t v = 0; v < n; ++v) seen[v] = -1;
    int64_t total = 0;
    if (out_rp) out_rp[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        /* breadth-first search from i, d levels deep */
        int64_t len = 0, level_begin = 0;
        seen[i] = i;
        list[len++] = (int32_t)i;
        for (int32_t step = 0; step < d; ++step) {
            const int64_t level_end = len;
            for (int64_t q = level_begin; q < level_end; ++q) {
                const int64_t u = list[q];
                for (int64_t p = rp[u]; p < rp[u + 1]; ++p) {
                    const int32_t v = col[p];
                    if (seen[v] != i) {
                        seen[v] = i;
                        list[len++] = v;
                    }
                }
            }
            level_begin = level_end;
        }
        if (out_col) {
            qsort(list, (size_t)len, sizeof(int32_t), orc_cmp_i32);
            memcpy(out_col + total, list, (size_t)len * sizeof(int32_t));
        }
        total += len;
        if (out_rp) out_rp[i + 1] = total;
    }
    free(seen);
    free(list);
    return total;
}

/*
 * One-point fits over the entries of a pattern P (the graph G_d) with the
 * target of A (Eq. (4.3): y_i is built from row i of A, whatever d is).
 * As in step 4, a residual-target row of A with exactly one off-diagonal j1
 * has y_i = -(a_ij1 / a_ii) x_j1 exactly: the entry (i, j1) gets
 * a = -a_ij1 / a_ii and LS = 0; every other entry of row i in P is fitted.
 * Diagonal entries of P get a = 0, ls = NaN.  With P = A this is step 4.
 */
void orc_edge_ls_graph(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                       const int64_t *prp, const int32_t *pcol, int32_t K, const double *w,
                       int32_t mode, const double *X, const double *Y, double *a, double *ls)
{
    for (int64_t i = 0; i < n; ++i) {
        int64_t off = 0, p1 = -1;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
            if (col[p] != i) {
                ++off;
                p1 = p;
            }
        double aii = orc_diag(rp, col, val, i);
        for (int64_t q = prp[i]; q < prp[i + 1]; ++q) {
            int64_t j = pcol[q];
            if (j == i) {
                a[q] = 0.0;
                ls[q] = NAN;
                continue;
            }
            if (mode == 0 && off == 1 && j == col[p1]) {
                a[q] = -val[p1] / aii;
                ls[q] = 0.0;
                continue;
            }
            const double *y = Y + i * K;
            const double *x = X + j * K;
            double sxx = 0.0, syx = 0.0;
            for (int32_t kappa = 0; kappa < K; ++kappa) {
                sxx += w[kappa] * x[kappa] * x[kappa];
                syx += w[kappa] * y[kappa] * x[kappa];
            }
            double pij = (sxx == 0.0) ? 0.0 : syx / sxx;
            double res = 0.0;
            for (int32_t kappa = 0; kappa < K; ++kappa) {
                double e = y[kappa] - pij * x[kappa];
                res += w[kappa] * e * e;
            }
            a[q] = pij;
            ls[q] = res;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* 9. Least-squares interpolation (§4.3; the functional of Eqs. (3.1),     */
/*    (3.2) with a set W of coarse points).  For a fine row i (coarse[i] =  */
/*    0) the candidates are the coarse points of V_i in the pattern prp /  */
/*    pcol (the graph G_{d_LS}); every subset W of at most c candidates is */
/*    fitted: p_W solves the weighted normal equations                     */
/*      sum_b G_ab p_b = b_a,  G_ab = sum_k w x_a x_b,  b_a = sum_k w y x_a  */
/*    (Gaussian elimination with partial pivoting; a pivot below 1e-13 of  */
/*    the largest diagonal entry marks the set singular and it is skipped),*/
/*    and LS_W = sum_k w (y_i - sum_{a in W} p_a x_a)^2.  For each size m   */
/*    the first set (lexicographic over the ascending candidate list) with */
/*    the smallest LS_W is kept.  Sizes are then compared with the penalty  */
/*    of §4.3 on LS normalised by S_yy = sum_k w y_i^2: starting from the   */
/*    empty set (normalised LS 1), size m replaces the current size m' <  m */
/*    when LS_m / S_yy < (LS_m' / S_yy)^(gamma (m - m')).  (S_yy = 0 keeps   */
/*    the empty set.)  A coarse row interpolates itself: (i, 1).            */
/*    Outputs: P as CSR (p_rp[n+1], p_col, p_val; columns ascending) and   */
/*    the chosen LS per row (0 for coarse rows).  Returns the entry count, */
/*    -7 when it exceeds cap (p_rp still written), -5 when out of memory.  */
/* ------------------------------------------------------------------------ */
static int orc_solve_small(int m, double *G, double *b, double *p)
{
    /* G (m x m, row-major) p = b, partial pivoting; G and b are destroyed */
    double dmax = 0.0;
    for (int a = 0; a < m; ++a)
        if (fabs(G[a * m + a]) > dmax) dmax = fabs(G[a * m + a]);
    for (int k = 0; k < m; ++k) {
        int piv = k;
        for (int a = k + 1; a < m; ++a)
            if (fabs(G[a * m + k]) > fabs(G[piv * m + k])) piv = a;
        if (!(fabs(G[piv * m + k]) > 1e-13 * dmax)) return -1;
        if (piv != k) {
            for (int c2 = 0; c2 < m; ++c2) {
                double t = G[k * m + c2];
                G[k * m + c2] = G[piv * m + c2];
                G[piv * m + c2] = t;
            }
            double t = b[k];
            b[k] = b[piv];
            b[piv] = t;
        }
        for (int a = k + 1; a < m; ++a) {
            double f = G[a * m + k] / G[k * m + k];
            for (int c2 = k; c2 < m; ++c2) G[a * m + c2] -= f * G[k * m + c2];
            b[a] -= f * b[k];
        }
    }
    for (int k = m - 1; k >= 0; --k) {
        double s = b[k];
        for (int c2 = k + 1; c2 < m; ++c2) s -= G[k * m + c2] * p[c2];
        p[k] = s / G[k * m + k];
    }
    return 0;
}

int64_t orc_ls_interp(int64_t n, int32_t K, const double *w, const double *X, const double *Y,
                      const int64_t *prp, const int32_t *pcol, const uint8_t *coarse, int32_t c,
                      double gamma, int64_t *p_rp, int32_t *p_col, double *p_val, double *ls_out,
                      int64_t cap)
{
    enum { MAXC = 8 };
    if (c > MAXC) c = MAXC;
    int64_t total = 0;
    int64_t maxcand = 1;
    for (int64_t i = 0; i < n; ++i)
        if (prp[i + 1] - prp[i] > maxcand) maxcand = prp[i + 1] - prp[i];
    int32_t *cand = (int32_t *)malloc((size_t)maxcand * sizeof(int32_t));
    if (!cand) return -5;
    p_rp[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t bestset[MAXC + 1][MAXC];
        double bestp[MAXC + 1][MAXC];
        double bestls[MAXC + 1];
        int have[MAXC + 1];
        int chosen = 0;
        if (coarse[i]) {
            if (total < cap) {
                p_col[total] = (int32_t)i;
                p_val[total] = 1.0;
            }
            ++total;
            p_rp[i + 1] = total;
            if (ls_out) ls_out[i] = 0.0;
            continue;
        }
        const double *y = Y + i * K;
        int nc = 0;
        for (int64_t q = prp[i]; q < prp[i + 1]; ++q)
            if (coarse[pcol[q]]) cand[nc++] = pcol[q];
        double syy = 0.0;
        for (int32_t k = 0; k < K; ++k) syy += w[k] * y[k] * y[k];
        for (int m = 0; m <= c; ++m) have[m] = 0;
        have[0] = 1;
        bestls[0] = syy;
        for (int m = 1; m <= c && m <= nc; ++m) {
            int idx[MAXC];
            for (int a = 0; a < m; ++a) idx[a] = a;
            for (;;) {
                double G[MAXC * MAXC], b[MAXC], p[MAXC];
                for (int a = 0; a < m; ++a) {
                    const double *xa = X + (int64_t)cand[idx[a]] * K;
                    double s = 0.0;
                    for (int32_t k = 0; k < K; ++k) s += w[k] * y[k] * xa[k];
                    b[a] = s;
                    for (int bb = 0; bb < m; ++bb) {
                        const double *xb = X + (int64_t)cand[idx[bb]] * K;
                        double g = 0.0;
                        for (int32_t k = 0; k < K; ++k) g += w[k] * xa[k] * xb[k];
                        G[a * m + bb] = g;
                    }
                }
                if (orc_solve_small(m, G, b, p) == 0) {
                    double res = 0.0;
                    for (int32_t k = 0; k < K; ++k) {
                        double e = y[k];
                        for (int a = 0; a < m; ++a) e -= p[a] * X[(int64_t)cand[idx[a]] * K + k];
                        res += w[k] * e * e;
                    }
                    if (!have[m] || res < bestls[m]) {
                        have[m] = 1;
                        bestls[m] = res;
                        for (int a = 0; a < m; ++a) {
                            bestset[m][a] = cand[idx[a]];
                            bestp[m][a] = p[a];
                        }
                    }
                }
                /* next combination in lexicographic order */
                int a = m - 1;
                while (a >= 0 && idx[a] == nc - m + a) --a;
                if (a < 0) break;
                ++idx[a];
                for (int bb = a + 1; bb < m; ++bb) idx[bb] = idx[bb - 1] + 1;
            }
        }
        if (syy > 0.0) {
            for (int m = 1; m <= c; ++m) {
                if (!have[m]) continue;
                double cur = bestls[chosen] / syy;
                if (bestls[m] / syy < pow(cur, gamma * (double)(m - chosen))) chosen = m;
            }
        }
        for (int a = 0; a < chosen; ++a) {
            if (total < cap) {
                p_col[total] = bestset[chosen][a];
                p_val[total] = bestp[chosen][a];
            }
            ++total;
        }
        p_rp[i + 1] = total;
        if (ls_out) ls_out[i] = bestls[chosen];
    }
    free(cand);
    return total > cap ? -7 : total;
}

/* ------------------------------------------------------------------------ */
/* 10. Compatible-relaxation coarsening (§3.2 Eqs. (3.4), (3.5); §4.2 Eq.   */
/*     (4.4); Algorithm 1 with the candidate measure of the Remark after    */
/*     it).  One stage:                                                     */
/*     (a) nu F-relaxation sweeps of the homogeneous system from the        */
/*         constant start u = 1 on F (Eq. (3.4)): the sweep of section 2    */
/*         (weighted Jacobi, or multicolor Gauss-Seidel) applied to the     */
/*         rows of F only, with u = 0 held on C, which is                   */
/*         u_f <- (I - M_ff^{-1} A_ff) u_f;                                 */
/*     (b) the convergence estimate of Eq. (3.5) in the max norm,           */
/*         rho_f = (||u^nu|| / ||u^0||)^(1/nu)  (0 when F is empty);         */
/*     (c) stop when rho_f <= delta, or when max_sets sets were added;      */
/*     (d) candidates Z = { i in F : sigma_i = |u_i| / ||u^nu|| > tol };    */
/*     (e) the strength graph M on F (Eq. (4.4) restricted to i, j in F,    */
/*         the maximum over the neighbours k in F): slot (i, j) of the      */
/*         pattern is strong iff i, j in F, j != i and LS_ij = 0 or         */
/*         theta LS_ij < min_k LS_ik;                                       */
/*     (f) an independent set of Z in M (edges in either direction): the   */
/*         greedy set in decreasing priority, where the priority of i is    */
/*         lambda_i = |{ j in Z : (j, i) strong }| (the number of           */
/*         candidates that depend strongly on i, as in the classical first  */
/*         pass), then a random 64-bit key (word 0 of Philox4x64-10 with    */
/*         counter (i, stage, 1, 0) and key (seed, 0)), then the smaller    */
/*         index;                                                           */
/*     (g) C <- C + the set; the next stage starts again at (a).            */
/*     coarse[n] is C_0 on entry and C on exit.  rho[] gets one estimate    */
/*     per stage (at most max_sets + 1).  nu >= 1.  Returns the number of   */
/*     estimates, or -5 when out of memory.                                 */
/* ------------------------------------------------------------------------ */
static int orc_cr_before(int32_t la, uint64_t ra, int64_t a, int32_t lb, uint64_t rb, int64_t b)
{
    /* 1 if vertex a comes before vertex b in the greedy order */
    if (la != lb) return la > lb;
    if (ra != rb) return ra > rb;
    return a < b;
}

static const int32_t *orc_cr_lam;
static const uint64_t *orc_cr_key;

static int orc_cr_cmp(const void *pa, const void *pb)
{
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    if (a == b) return 0;
    return orc_cr_before(orc_cr_lam[a], orc_cr_key[a], a, orc_cr_lam[b], orc_cr_key[b], b) ? -1 : 1;
}

int32_t orc_cr_coarsen(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                       const int64_t *prp, const int32_t *pcol, const double *ls, int32_t sweep,
                       double omega, const int32_t *color, int32_t ncolors, int32_t nu,
                       double theta, double delta, double tol, int32_t max_sets, uint64_t seed,
                       uint8_t *coarse, double *rho)
{
    int64_t nnz_p = prp[n];
    double *u = (double *)malloc((size_t)(n ? n : 1) * sizeof(double));
    double *un = (double *)malloc((size_t)(n ? n : 1) * sizeof(double));
    uint8_t *inz = (uint8_t *)malloc((size_t)(n ? n : 1));
    uint8_t *inset = (uint8_t *)malloc((size_t)(n ? n : 1));
    int32_t *lam = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    uint64_t *key = (uint64_t *)malloc((size_t)(n ? n : 1) * sizeof(uint64_t));
    int64_t *order = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    uint8_t *strong = (uint8_t *)malloc((size_t)(nnz_p ? nnz_p : 1));
    int64_t *trp = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
    int64_t *tsrc = (int64_t *)malloc((size_t)(nnz_p ? nnz_p : 1) * sizeof(int64_t));
    int32_t stage = 0;
    if (!u || !un || !inz || !inset || !lam || !key || !order || !strong || !trp || !tsrc) {
        stage = -5;
        goto done;
    }
    for (;;) {
        /* (a) nu F-relaxation sweeps from the constant start */
        int64_t nf = 0;
        for (int64_t i = 0; i < n; ++i) {
            u[i] = coarse[i] ? 0.0 : 1.0;
            nf += !coarse[i];
        }
        for (int32_t s = 0; s < nu; ++s) {
            if (sweep == 0) {
                for (int64_t i = 0; i < n; ++i) {
                    if (coarse[i]) { un[i] = 0.0; continue; }
                    double c = omega / orc_diag(rp, col, val, i);
                    double acc = 0.0;
                    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) acc = fma(val[p], u[col[p]], acc);
                    un[i] = fma(-c, acc, u[i]);
                }
            } else {
                memcpy(un, u, (size_t)n * sizeof(double));
                for (int32_t cc = 0; cc < ncolors; ++cc) {
                    for (int64_t i = 0; i < n; ++i) {
                        if (color[i] != cc || coarse[i]) continue;
                        double c = omega / orc_diag(rp, col, val, i);
                        double acc = 0.0;
                        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
                            int64_t j = col[p];
                            acc = fma(val[p], color[j] < cc ? un[j] : u[j], acc);
                        }
                        un[i] = fma(-c, acc, u[i]);
                    }
                }
            }
            double *t = u;
            u = un;
            un = t;
        }
        /* (b) rho_f in the max norm; ||u^0|| = 1 when F is not empty */
        double unorm = 0.0;
        for (int64_t i = 0; i < n; ++i)
            if (!coarse[i] && fabs(u[i]) > unorm) unorm = fabs(u[i]);
        double r = nf == 0 ? 0.0 : pow(unorm, 1.0 / (double)nu);
        rho[stage] = r;
        /* (c) */
        if (!(r > delta) || stage >= max_sets) { ++stage; break; }
        /* (d) candidates */
        for (int64_t i = 0; i < n; ++i)
            inz[i] = (uint8_t)(!coarse[i] && fabs(u[i]) / unorm > tol);
        /* (e) strength graph on F */
        for (int64_t i = 0; i < n; ++i) {
            double m = INFINITY;
            for (int64_t q = prp[i]; q < prp[i + 1]; ++q) {
                strong[q] = 0;
                int64_t j = pcol[q];
                if (j != i && !coarse[j] && ls[q] < m) m = ls[q];
            }
            if (coarse[i]) continue;
            for (int64_t q = prp[i]; q < prp[i + 1]; ++q) {
                int64_t j = pcol[q];
                if (j != i && !coarse[j] && (ls[q] == 0.0 || theta * ls[q] < m)) strong[q] = 1;
            }
        }
        /* (f) priorities and the greedy independent set of Z */
        for (int64_t i = 0; i < n; ++i) lam[i] = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (!inz[j]) continue;
            for (int64_t q = prp[j]; q < prp[j + 1]; ++q)
                if (strong[q] && inz[pcol[q]]) ++lam[pcol[q]];
        }
        {
            const uint64_t k2[2] = {seed, 0};
            for (int64_t i = 0; i < n; ++i) {
                uint64_t ctr[4] = {(uint64_t)i, (uint64_t)stage, 1, 0};
                uint64_t out[4];
                orc_philox4x64_10(ctr, k2, out);
                key[i] = out[0];
            }
        }
        /* in-edges of the strong graph: the transpose of the strong slots */
        for (int64_t i = 0; i <= n; ++i) trp[i] = 0;
        for (int64_t q = 0; q < nnz_p; ++q)
            if (strong[q]) ++trp[pcol[q] + 1];
        for (int64_t i = 0; i < n; ++i) trp[i + 1] += trp[i];
        {
            int64_t *fill = order;   /* scratch: next free in-edge position per row */
            for (int64_t i = 0; i < n; ++i) fill[i] = trp[i];
            for (int64_t i = 0; i < n; ++i)
                for (int64_t q = prp[i]; q < prp[i + 1]; ++q)
                    if (strong[q]) tsrc[fill[pcol[q]]++] = i;
        }
        int64_t nz = 0;
        for (int64_t i = 0; i < n; ++i) {
            inset[i] = 0;
            if (inz[i]) order[nz++] = i;
        }
        orc_cr_lam = lam;
        orc_cr_key = key;
        qsort(order, (size_t)nz, sizeof(int64_t), orc_cr_cmp);
        for (int64_t t = 0; t < nz; ++t) {
            int64_t v = order[t];
            int blocked = 0;
            for (int64_t q = prp[v]; q < prp[v + 1] && !blocked; ++q)
                if (strong[q] && inset[pcol[q]]) blocked = 1;
            for (int64_t e = trp[v]; e < trp[v + 1] && !blocked; ++e)
                if (inset[tsrc[e]]) blocked = 1;
            if (!blocked) inset[v] = 1;
        }
        /* (g) */
        for (int64_t i = 0; i < n; ++i)
            if (inset[i]) coarse[i] = 1;
        ++stage;
    }
done:
    free(u); free(un); free(inz); free(inset); free(lam); free(key); free(order);
    free(strong); free(trp); free(tsrc);
    return stage;
}
