// amgd_api.cu -- host side of the C ABI declared in include/amgd.h:
// argument and CSR validation, device memory of a handle, the row
// permutation that makes every Gauss-Seidel color a contiguous row range,
// kernel dispatch, and CUDA-graph capture of a whole build.
#include "../../include/amgd.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "amgd_internal.cuh"

#include <nvtx3/nvToolsExt.h>

using namespace amgd;

struct amgd_ctx {
    int device = 0;
    int64_t n = 0, nnz = 0, E = 0;
    int32_t K = 0, nmat = 1;
    int storage = ST_FP64, target = AMGD_TARGET_RESIDUAL;
    std::vector<int64_t> row_off, slot_off;
    std::vector<int32_t> h_rp, h_col;          // caller CSR pattern (int32)
    std::vector<int32_t> h_diag_slot;           // slot of each row's diagonal
    // device: caller numbering
    int32_t *rp_o = nullptr, *col_o = nullptr;
    double *val_o = nullptr;
    int64_t *mat_off = nullptr;
    int32_t *diag_slot = nullptr;                // slot of each row's diagonal
    uint32_t *err_word = nullptr;                // device error bits of value checks
    uint32_t *status = nullptr;                  // device status bits of bounded waits
    bool perm64_stale = false;                   // row-permuted FP64 values / diagonal out of date
    long long wait_limit = 2000000000LL;         // cycles (about 1 s) per staged wait
    uint32_t test_extra_tx = 0;                  // test hook, see amgd_create
    // device: row-permuted matrix (aliases of the caller arrays without coloring)
    int32_t *rp_p = nullptr, *col_p = nullptr, *perm = nullptr;
    int32_t *slot_perm = nullptr;                // permuted slot of every caller slot
    double *val64 = nullptr;
    float *val32 = nullptr;
    double *diag64 = nullptr;                    // permuted diagonal
    float *diag32 = nullptr;
    float *val32_o = nullptr;                    // caller-order FP32 values (edge pass)
    double *diag64_o = nullptr;                  // caller-order diagonal (edge pass)
    float *diag32_o = nullptr;
    void *x_caller = nullptr;                    // caller-order copy of permuted vectors
    int64_t *mat_id = nullptr;                   // Philox key word 1 per matrix (NULL: index)
    int32_t *pinv = nullptr;                     // caller row -> permuted row
    int32_t *colx = nullptr;                     // caller CSR, columns in permuted numbering
    uint32_t *defer_count = nullptr;             // rows the mixed edge pass redoes in FP64
    int32_t *defer_list = nullptr;
    std::vector<int64_t> color_start;           // permuted row start of each color
    // vectors
    void *x[2] = {nullptr, nullptr};
    int cur = 0;
    std::vector<double> h_w;
    double *w64 = nullptr;
    float *w32 = nullptr;
    // outputs
    void *a = nullptr, *ls = nullptr;
    uint8_t *flag = nullptr;
    int32_t *count = nullptr, *tile = nullptr;
    int64_t *s_rp_tmp = nullptr;
    int32_t *s_col_tmp = nullptr;
    double *tmp64 = nullptr;                     // n*K or nnz doubles, staging
    size_t tmp64_len = 0;
    bool have_dist = false;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int graph_cur_after = 0;
    Shape relax_shape[3], edge_shape[3];         // per storage type
    // reverse pass: trajectory of the last recorded Jacobi relaxation
    int32_t ckpt_every = 0;                      // 0: amgd_relax records nothing
    bool traj_valid = false;
    int32_t traj_nu = 0;
    double traj_omega = 0.0;
    void *ckpt = nullptr;                        // X_0, X_s, X_2s, ... (storage type)
    size_t ckpt_bytes = 0;
    void *seg = nullptr;                         // X_{cs+1} .. X_{cs+s-1}, recomputed
    size_t seg_bytes = 0;
    void *adj_vec = nullptr;                     // Y, Ybar, Xbar[2]  (arithmetic type)
    size_t adj_vec_bytes = 0;
    void *adj_slot = nullptr;                    // gs, gt, at_b     (arithmetic type)
    size_t adj_slot_bytes = 0;
    double *lsb = nullptr;                       // dL/dLS per slot
    double *adj_part = nullptr;                  // 2 x kAdjReduceBlocks partials + 2 sums
    int32_t *at_rp = nullptr, *at_row = nullptr, *at_slot = nullptr;   // transposed pattern
    int32_t *mirror = nullptr;                   // slot of (j, i) for slot (i, j); symmetric patterns
    // least-squares interpolation working buffers
    uint8_t *ip_coarse = nullptr;
    int32_t *ip_sel_col = nullptr, *ip_cnt = nullptr;
    double *ip_sel_val = nullptr, *ip_ls = nullptr;
    int64_t *ip_rp = nullptr;
    int32_t *ip_pos = nullptr, *ip_list = nullptr, *ip_bcnt = nullptr;
    uint8_t *ip_bkt = nullptr;
    void *ip_out = nullptr;
    size_t ip_out_bytes = 0;
    // compatible-relaxation coarsening working buffers
    double *cr_u[2] = {nullptr, nullptr};
    uint8_t *cr_coarse = nullptr, *cr_state = nullptr, *cr_ismax = nullptr, *cr_strong = nullptr;
    uint8_t *cr_coarse_p = nullptr;              // coarse mask in the sweeps' row order
    double *cr_cdiag = nullptr;                  // omega / a_rr in the sweeps' row order
    size_t cr_strong_len = 0;
    int32_t *cr_lam = nullptr;
    uint64_t *cr_key = nullptr;
    unsigned long long *cr_scal = nullptr;
    int32_t cr_rounds = 0;                       // selection rounds of the last amgd_cr_coarsen
    int64_t cr_launches = 0;                     // kernels it launched
    // asynchronous value updates and results (stream-ordered, double-buffered)
    cudaStream_t up_stream = nullptr, down_stream = nullptr;
    cudaEvent_t ev_up[2] = {nullptr, nullptr}, ev_used[2] = {nullptr, nullptr};
    cudaEvent_t ev_res[2] = {nullptr, nullptr}, ev_down[2] = {nullptr, nullptr};
    double *stage[2] = {nullptr, nullptr};
    int64_t *res_rp[2] = {nullptr, nullptr};
    int32_t *res_col[2] = {nullptr, nullptr};
    int64_t res_col_len = 0;
    uint32_t *async_err = nullptr;               // value-check bits of asynchronous updates
    int up_slot = 0, res_slot = 0;
    bool async_pending = false;
    struct PendingOut { int64_t *rp; int mem; int64_t cap; };
    std::vector<PendingOut> pending_out;         // strength outputs checked at amgd_sync
    int32_t *edge_tiles = nullptr;               // row tiles of the edge pass (over the pattern)
    int32_t n_edge_tiles = 0;
    // pattern of the fits, threshold and strength graph: the graph G_d of A^d
    // (search depth d); for d = 1 these alias A's caller-order pattern
    int32_t depth = 1;
    int32_t summation = AMGD_SUM_COMPENSATED;   // LS sums of the mixed paths (edge stage 2)
    int32_t *prp = nullptr, *pcol = nullptr;
    int64_t nnz_p = 0, E_p = 0;
    bool last_backward_builtin = false;          // the last reverse pass used the built-in loss
    bool graph_is_backward = false;              // the captured graph ends with a reverse pass
    int32_t graph_traj_nu = 0;
    double graph_traj_omega = 0.0;
    bool phase_timing = false, graph_timed = false;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    std::string err;
};

namespace {

thread_local std::string g_create_err;

int V_of(int st) { return st == ST_FP64 ? 2 : (st == ST_FP32 ? 4 : 8); }
size_t esize(int st) { return st == ST_FP64 ? 8 : (st == ST_FP32 ? 4 : 2); }

// 16-byte vectors per row: ceil(K / V) rounded up to a power of two
int P_of(int st, int K)
{
    const int V = V_of(st);
    const int need = (K + V - 1) / V;
    int P = 1;
    while (P < need) P <<= 1;
    return P;
}
int Kp_of(int st, int K) { return P_of(st, K) * V_of(st); }

// a shape is valid when it tiles the row exactly and stays within the
// compiled instantiations (NV in {1,2,4}, U in {4,8}, G*NV*V <= 64)
bool shape_ok(int st, int K, Shape sh)
{
    const int P = P_of(st, K);
    if (sh.NV != 1 && sh.NV != 2 && sh.NV != 4) return false;
    if (sh.U != 2 && sh.U != 4 && sh.U != 8) return false;     // U = 2: edge pass only
    if (sh.G < 1 || sh.G > 32 || (sh.G & (sh.G - 1))) return false;
    if (sh.stage < 0 || sh.stage > 3) return false;
    return sh.G * sh.NV == P;
}

// the distance pass: stages 0 (rows) and 1 (tiles) take every valid shape;
// stage 2 (the row kernel on the sweeps' row order) 2 or 4 entries per batch,
// stage 3 (the warp-staged kernel on that order) 4 or 8
bool edge_shape_ok(Shape sh)
{
    if (sh.stage < 0 || sh.stage > 3) return false;
    if (sh.stage == 2) return sh.U == 2 || sh.U == 4;
    if (sh.stage == 3) return sh.U == 4 || sh.U == 8;
    return true;
}

// untuned default: one vector per lane, four nonzeros per batch (the
// lightest shape in registers), CSR read directly
Shape default_shape(int st, int K)
{
    return Shape{P_of(st, K), 1, 4, 0};
}



// NVTX range over one C-ABI call (header-only NVTX v3: free when no tool is
// attached, named ranges in ncu / Nsight timelines when one is)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
#define AMGD_RANGE(name) NvtxRange amgd_nvtx_range_(name)

int fail(amgd_ctx *h, int code, const std::string &msg)
{
    if (h) h->err = msg; else g_create_err = msg;
    return code;
}

int cuda_fail(amgd_ctx *h, cudaError_t e, const char *where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(h, e == cudaErrorMemoryAllocation ? AMGD_ERR_OOM : AMGD_ERR_CUDA, m);
}

#define CK(h, expr)                                              \
    do {                                                         \
        cudaError_t e__ = (expr);                                \
        if (e__ != cudaSuccess) return cuda_fail((h), e__, #expr); \
    } while (0)

// read and clear the device status word (synchronises the stream)
// drop a captured graph whose device pointers are about to change
void drop_graph(amgd_ctx *h)
{
    if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
    if (h->graph) { cudaGraphDestroy(h->graph); h->graph = nullptr; }
    h->graph_timed = false;
}

int poll_status(amgd_ctx *h)
{
    uint32_t st = 0;
    CK(h, cudaMemcpyAsync(&st, h->status, sizeof st, cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (st) {
        CK(h, cudaMemsetAsync(h->status, 0, sizeof st, h->stream));
        if (st & kStatusIndexRange)
            return fail(h, AMGD_ERR_CHECK,
                        "a gather index (a column index or row map of the matrix) was out of "
                        "range; the results are not valid (checked build)");
        return fail(h, AMGD_ERR_TIMEOUT,
                    "a staged relaxation kernel gave up waiting for its shared-memory copies; "
                    "the test vectors are not valid");
    }
    return AMGD_OK;
}

template <class T>
cudaError_t dalloc(T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void **)p, count * sizeof(T));
}

cudaError_t dfree(void *p) { return p ? cudaFree(p) : cudaSuccess; }

// copy `bytes` from host or device memory `src` into host vector storage
cudaError_t fetch(void *dst, const void *src, size_t bytes, int mem)
{
    if (bytes == 0) return cudaSuccess;
    if (mem == AMGD_MEM_HOST) {
        std::memcpy(dst, src, bytes);
        return cudaSuccess;
    }
    return cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost);
}

// CSR check of one matrix: returns AMGD_OK or an error with message
int check_csr(const int64_t *rp, const int32_t *col, const double *val, int64_t n,
              std::vector<int32_t> &marker, std::vector<int32_t> &diag_slot, int64_t slot_base,
              std::string &msg)
{
    if (rp[0] != 0) { msg = "row_ptr[0] != 0"; return AMGD_ERR_CSR; }
    for (int64_t i = 0; i < n; ++i)
        if (rp[i + 1] < rp[i]) { msg = "row_ptr decreases at row " + std::to_string(i); return AMGD_ERR_CSR; }
    marker.assign((size_t)n, -1);
    diag_slot.resize((size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        int64_t d = -1;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            const int64_t j = col[p];
            if (j < 0 || j >= n) { msg = "column out of range in row " + std::to_string(i); return AMGD_ERR_CSR; }
            if (!std::isfinite(val[p])) { msg = "non-finite value in row " + std::to_string(i); return AMGD_ERR_CSR; }
            if (marker[(size_t)j] == (int32_t)i) { msg = "duplicate column in row " + std::to_string(i); return AMGD_ERR_CSR; }
            marker[(size_t)j] = (int32_t)i;
            if (j == i) d = p;
        }
        if (d < 0 || val[d] == 0.0) { msg = "missing or zero diagonal in row " + std::to_string(i); return AMGD_ERR_ZERO_DIAG; }
        diag_slot[(size_t)i] = (int32_t)(slot_base + d);
    }
    return AMGD_OK;
}

cudaError_t ensure_tmp64(amgd_ctx *h, size_t count)
{
    if (h->tmp64_len >= count && h->tmp64) return cudaSuccess;
    dfree(h->tmp64);
    h->tmp64_len = 0;
    cudaError_t e = dalloc(&h->tmp64, count);
    if (e == cudaSuccess) h->tmp64_len = count;
    return e;
}

// allocate the two vector buffers and the weights for the current storage
int alloc_vectors(amgd_ctx *h, int st, void **x0, void **x1)
{
    const size_t bytes = (size_t)h->n * Kp_of(st, h->K) * esize(st);
    CK(h, cudaMalloc(x0, bytes ? bytes : 16));
    cudaError_t e = cudaMalloc(x1, bytes ? bytes : 16);
    if (e != cudaSuccess) { cudaFree(*x0); *x0 = nullptr; return cuda_fail(h, e, "cudaMalloc(x1)"); }
    return AMGD_OK;
}

int upload_weights(amgd_ctx *h)
{
    const int Kp = Kp_of(ST_FP64, h->K) > Kp_of(ST_FP32, h->K) ? Kp_of(ST_FP64, h->K)
                                                                : Kp_of(ST_FP32, h->K);
    const int KpMax = Kp > Kp_of(ST_BF16, h->K) ? Kp : Kp_of(ST_BF16, h->K);
    std::vector<double> w64((size_t)KpMax, 0.0);
    std::vector<float> w32((size_t)KpMax, 0.0f);
    for (int k = 0; k < h->K; ++k) { w64[(size_t)k] = h->h_w[(size_t)k]; w32[(size_t)k] = (float)h->h_w[(size_t)k]; }
    if (!h->w64) CK(h, dalloc(&h->w64, (size_t)KpMax));
    if (!h->w32) CK(h, dalloc(&h->w32, (size_t)KpMax));
    CK(h, cudaMemcpyAsync(h->w64, w64.data(), KpMax * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaMemcpyAsync(h->w32, w32.data(), KpMax * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return AMGD_OK;
}

// Values from src (caller order; NULL: h->val_o itself) into every copy the
// kernels read -- the caller FP64 array, the FP32 copies and, with a
// coloring, the row-permuted arrays -- in one coalesced pass, then the
// diagonals in caller and permuted order.
// Every value copy from the caller-order values (src, or the handle's own
// FP64 copy when NULL).  The row-permuted FP64 copy and diagonal feed only the
// FP64 sweeps and the coarsening; with mixed storage they are left stale here
// and refreshed by refresh_perm64 when one of those next runs.  err (NULL:
// none) collects the value checks of an asynchronous update.
int permute_values(amgd_ctx *h, const double *src = nullptr, uint32_t *err = nullptr)
{
    const bool in_place = src == nullptr;
    const bool mixed = h->storage != ST_FP64;
    float *v32o = (h->val32_o && h->val32_o != h->val32) ? h->val32_o : nullptr;
    double *vp64 = (h->perm && !mixed) ? h->val64 : nullptr;   // without a coloring val64 is val_o
    CK(h, launch_scatter_values(in_place ? h->val_o : src, h->nnz, h->perm ? h->slot_perm : nullptr,
                                in_place ? nullptr : h->val_o, v32o, vp64, h->val32, h->stream, err));
    CK(h, launch_diag_values(h->val_o, h->diag_slot, h->perm, (int32_t)h->n, h->diag64_o,
                             h->diag32_o, mixed ? nullptr : h->diag64, h->diag32, h->stream, err));
    h->perm64_stale = mixed;
    return AMGD_OK;
}

// bring the row-permuted FP64 values and diagonal up to date (stream order)
int refresh_perm64(amgd_ctx *h, cudaStream_t s)
{
    if (!h->perm64_stale) return AMGD_OK;
    if (h->perm)
        CK(h, launch_scatter_values(h->val_o, h->nnz, h->slot_perm, nullptr, nullptr, h->val64,
                                    nullptr, s));
    CK(h, launch_diag_values(h->val_o, h->diag_slot, h->perm, (int32_t)h->n, nullptr, nullptr,
                             h->diag64, nullptr, s));
    h->perm64_stale = false;
    return AMGD_OK;
}

int run_init(amgd_ctx *h, uint64_t seed, cudaStream_t s)
{
    InitArgs a;
    a.x = h->x[h->cur];
    a.perm = h->perm;
    a.mat_off = h->mat_off;
    a.mat_id = h->mat_id;
    a.nmat = h->nmat;
    a.n = (int32_t)h->n;
    a.K = h->K;
    a.Kp = Kp_of(h->storage, h->K);
    a.seed = seed;
    CK(h, launch_init(h->storage, a, s));
    h->have_dist = false;
    h->traj_valid = false;
    return AMGD_OK;
}

int run_relax(amgd_ctx *h, int32_t nu, double omega, int sweep, cudaStream_t s)
{
    const Shape sh = h->relax_shape[h->storage];
    if (h->storage == ST_FP64 && nu > 0) {
        const int rc = refresh_perm64(h, s);
        if (rc != AMGD_OK) return rc;
    }
    RelaxArgs a;
    a.status = h->status;
    a.wait_limit = h->wait_limit;
    a.extra_tx = h->test_extra_tx;
    a.rp = h->rp_p;
    a.col = h->col_p;
    a.val = h->storage == ST_FP64 ? (const void *)h->val64 : (const void *)h->val32;
    a.diag = h->storage == ST_FP64 ? (const void *)h->diag64 : (const void *)h->diag32;
    a.Kp = Kp_of(h->storage, h->K);
    a.omega = omega;
    a.avg_nnz = h->n ? (float)((double)h->nnz / (double)h->n) : 0.f;
    a.nrows = (int32_t)h->n;
    for (int32_t it = 0; it < nu; ++it) {
        a.xold = h->x[h->cur];
        a.xnew = h->x[1 - h->cur];
        if (sweep == AMGD_SWEEP_JACOBI) {
            a.r0 = 0;
            a.r1 = (int32_t)h->n;
            a.split = 0;
            CK(h, launch_relax(h->storage, sh, a, s));
        } else {
            for (size_t c = 0; c + 1 < h->color_start.size(); ++c) {
                a.r0 = (int32_t)h->color_start[c];
                a.r1 = (int32_t)h->color_start[c + 1];
                a.split = a.r0;
                CK(h, launch_relax(h->storage, sh, a, s));
            }
        }
        h->cur = 1 - h->cur;
    }
    if (nu > 0) h->have_dist = false;
    h->traj_valid = false;
    return AMGD_OK;
}

// grow a device buffer to at least `bytes` (contents not kept)
cudaError_t ensure_buf(void **p, size_t &have, size_t bytes)
{
    if (*p && have >= bytes) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr;
    have = 0;
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e == cudaSuccess) have = bytes;
    return e;
}

// One Jacobi sweep X_dst = X_src - omega D^{-1} A X_src with the handle's
// relaxation shape (bit-identical to the sweeps of run_relax).
int jacobi_step(amgd_ctx *h, const void *src, void *dst, double omega, cudaStream_t s)
{
    if (h->storage == ST_FP64) {
        const int rc = refresh_perm64(h, s);
        if (rc != AMGD_OK) return rc;
    }
    RelaxArgs a;
    a.status = h->status;
    a.wait_limit = h->wait_limit;
    a.extra_tx = h->test_extra_tx;
    a.rp = h->rp_p;
    a.col = h->col_p;
    a.val = h->storage == ST_FP64 ? (const void *)h->val64 : (const void *)h->val32;
    a.diag = h->storage == ST_FP64 ? (const void *)h->diag64 : (const void *)h->diag32;
    a.Kp = Kp_of(h->storage, h->K);
    a.omega = omega;
    a.avg_nnz = h->n ? (float)((double)h->nnz / (double)h->n) : 0.f;
    a.nrows = (int32_t)h->n;
    a.xold = src;
    a.xnew = dst;
    a.r0 = 0;
    a.r1 = (int32_t)h->n;
    a.split = 0;
    CK(h, launch_relax(h->storage, h->relax_shape[h->storage], a, s));
    return AMGD_OK;
}

// Jacobi sweeps that keep the trajectory for amgd_backward: X_0, X_s, X_2s,
// ... go to checkpoint slots (written by the sweeps themselves), the other
// iterates ping-pong through the two vector buffers, and X_nu ends where
// run_relax would leave it.
int run_relax_recorded(amgd_ctx *h, int32_t nu, double omega, cudaStream_t s)
{
    const int32_t S = h->ckpt_every;
    const size_t xb = (size_t)h->n * Kp_of(h->storage, h->K) * esize(h->storage);
    const int32_t nck = (nu + S - 1) / S;
    CK(h, ensure_buf(&h->ckpt, h->ckpt_bytes, (size_t)nck * xb));
    const int c0 = h->cur;
    auto loc = [&](int32_t m) -> void * {
        if (m == 0) return h->x[c0];
        if (m == nu) return h->x[(c0 + nu) & 1];
        if (m % S == 0) return (char *)h->ckpt + (size_t)(m / S) * xb;
        return h->x[(c0 + m) & 1];
    };
    if (nck > 0) CK(h, cudaMemcpyAsync(h->ckpt, h->x[c0], xb, cudaMemcpyDeviceToDevice, s));
    for (int32_t k = 0; k < nu; ++k) {
        const int rc = jacobi_step(h, loc(k), loc(k + 1), omega, s);
        if (rc != AMGD_OK) return rc;
    }
    h->cur = (c0 + nu) & 1;
    if (nu > 0) h->have_dist = false;
    h->traj_valid = true;
    h->traj_nu = nu;
    h->traj_omega = omega;
    return AMGD_OK;
}

int run_edge(amgd_ctx *h, double theta, cudaStream_t s)
{
    Shape sh = h->edge_shape[h->storage];
    if (sh.stage >= 2 && h->depth > 1) sh.stage = 0;    // stages 2 and 3 cover A's own pattern
    // stages 0 and 1 run on the caller's numbering: bring a row-permuted vector
    // block back to caller order first; stages 2 and 3 read the sweeps' row order
    const void *xc = h->x[h->cur];
    if (h->perm && sh.stage < 2) {
        if (!h->x_caller) return fail(h, AMGD_ERR_STATE, "caller-order vector buffer missing");
        CK(h, launch_unpermute(h->storage, h->x[h->cur], h->x_caller, h->perm, (int32_t)h->n,
                               Kp_of(h->storage, h->K), s));
        xc = h->x_caller;
    }
    EdgeArgs a;
    a.rp = h->rp_o;
    a.col = h->col_o;
    a.val = h->storage == ST_FP64 ? (const void *)h->val_o : (const void *)h->val32_o;
    a.diag = h->storage == ST_FP64 ? (const void *)h->diag64_o : (const void *)h->diag32_o;
    a.val64 = h->val_o;
    a.x = xc;
    a.w = h->storage == ST_FP64 ? (const void *)h->w64 : (const void *)h->w32;
    a.w64 = h->w64;
    a.a_out = h->a;
    a.ls_out = h->ls;
    a.flag_out = h->flag;
    a.count_out = h->count;
    a.defer_count = h->defer_count;
    a.defer_list = h->defer_list;
    a.prp = h->prp;
    a.pcol = h->pcol;
    a.tiles = h->edge_tiles;
    a.ntiles = h->n_edge_tiles;
    a.n = (int32_t)h->n;
    a.Kp = Kp_of(h->storage, h->K);
    a.target = h->target;
    a.theta = theta;
    if (sh.stage >= 2) {
        a.x = h->x[h->cur];                  // the sweeps' row order, read in place
        a.xrow = h->perm ? h->pinv : nullptr;
        a.xcol = h->perm ? h->colx : h->col_o;
    }
    a.compensated = h->summation == AMGD_SUM_COMPENSATED;
    a.status = h->status;
    bool unit_w = true;
    for (double wk : h->h_w) unit_w = unit_w && wk == 1.0;
    CK(h, launch_edge(h->storage, sh, unit_w, a, s));
    h->have_dist = true;
    return AMGD_OK;
}

// (re)allocate the per-slot a/LS buffers for the arithmetic type of `st`
int alloc_slot_outputs(amgd_ctx *h, int st)
{
    dfree(h->a);
    dfree(h->ls);
    h->a = h->ls = nullptr;
    const size_t es = st == ST_FP64 ? 8 : 4;
    CK(h, cudaMalloc(&h->a, (h->nnz_p ? h->nnz_p : 1) * es));
    CK(h, cudaMalloc(&h->ls, (h->nnz_p ? h->nnz_p : 1) * es));
    return AMGD_OK;
}

// row tiles of the edge pass over a caller-order pattern row pointer (host)
int build_edge_tiles(amgd_ctx *h, const std::vector<int32_t> &prp)
{
    std::vector<int32_t> tiles(1, 0);
    int64_t rows = 0, slots = 0;
    const int64_t n = h->n;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t len = prp[(size_t)i + 1] - prp[(size_t)i];
        if (rows > 0 && (rows == kEdgeTileRows || slots + len > kEdgeTileSlots)) {
            tiles.push_back((int32_t)i);
            rows = slots = 0;
        }
        ++rows;
        slots += len;
    }
    if (n > 0) tiles.push_back((int32_t)n);
    dfree(h->edge_tiles);
    h->edge_tiles = nullptr;
    h->n_edge_tiles = (int32_t)tiles.size() - 1;
    CK(h, dalloc(&h->edge_tiles, tiles.size()));
    CK(h, cudaMemcpy(h->edge_tiles, tiles.data(), tiles.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    return AMGD_OK;
}

int create_impl(int32_t nmat, const int64_t *const *rp_in, const int32_t *const *col_in,
                const double *const *val_in, const int64_t *n_in, int32_t K, uint64_t seed,
                int mem, amgd_handle *out)
{
    if (!out) return fail(nullptr, AMGD_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nmat < 1) return fail(nullptr, AMGD_ERR_ARG, "nmat < 1");
    if (K < 1 || K > 64) return fail(nullptr, AMGD_ERR_UNSUPPORTED, "K must be in 1..64");
    if (mem != AMGD_MEM_HOST && mem != AMGD_MEM_DEVICE) return fail(nullptr, AMGD_ERR_ARG, "bad mem");
    if (!rp_in || !col_in || !val_in || !n_in) return fail(nullptr, AMGD_ERR_ARG, "NULL array list");

    // gather every matrix on the host, validate, concatenate block-diagonally
    std::vector<int64_t> row_off(1, 0), slot_off(1, 0);
    for (int32_t b = 0; b < nmat; ++b) {
        if (n_in[b] < 0) return fail(nullptr, AMGD_ERR_ARG, "n < 0");
        row_off.push_back(row_off.back() + n_in[b]);
    }
    const int64_t n = row_off.back();
    if (n >= (int64_t)1 << 31) return fail(nullptr, AMGD_ERR_UNSUPPORTED, "n >= 2^31");
    std::vector<int32_t> h_rp(1, 0), h_col, diag_slot;
    std::vector<double> h_val;
    std::vector<int32_t> marker, dslot;
    for (int32_t b = 0; b < nmat; ++b) {
        const int64_t nb = n_in[b];
        if (!rp_in[b]) return fail(nullptr, AMGD_ERR_ARG, "NULL row_ptr");
        std::vector<int64_t> rp((size_t)nb + 1);
        cudaError_t e = fetch(rp.data(), rp_in[b], (nb + 1) * sizeof(int64_t), mem);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "copy row_ptr");
        if (rp[0] != 0) return fail(nullptr, AMGD_ERR_CSR, "row_ptr[0] != 0");
        const int64_t nnzb = rp[(size_t)nb];
        if (nnzb < 0) return fail(nullptr, AMGD_ERR_CSR, "negative nnz");
        if (slot_off.back() + nnzb >= ((int64_t)1 << 31) - 16)
            return fail(nullptr, AMGD_ERR_UNSUPPORTED, "nnz >= 2^31");
        if (nnzb > 0 && (!col_in[b] || !val_in[b])) return fail(nullptr, AMGD_ERR_ARG, "NULL col/val");
        std::vector<int32_t> col((size_t)nnzb);
        std::vector<double> val((size_t)nnzb);
        e = fetch(col.data(), col_in[b], nnzb * sizeof(int32_t), mem);
        if (e == cudaSuccess) e = fetch(val.data(), val_in[b], nnzb * sizeof(double), mem);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "copy col/val");
        std::string msg;
        const int rc = check_csr(rp.data(), col.data(), val.data(), nb, marker, dslot,
                                 slot_off.back(), msg);
        if (rc != AMGD_OK) return fail(nullptr, rc, "matrix " + std::to_string(b) + ": " + msg);
        const int64_t ro = row_off[(size_t)b], so = slot_off.back();
        for (int64_t i = 1; i <= nb; ++i) h_rp.push_back((int32_t)(so + rp[(size_t)i]));
        for (int64_t p = 0; p < nnzb; ++p) h_col.push_back((int32_t)(ro + col[(size_t)p]));
        h_val.insert(h_val.end(), val.begin(), val.end());
        diag_slot.insert(diag_slot.end(), dslot.begin(), dslot.end());
        slot_off.push_back(so + nnzb);
    }

    amgd_ctx *h = new amgd_ctx();
    h->n = n;
    h->nnz = slot_off.back();
    h->E = h->nnz - n;
    h->K = K;
    h->nmat = nmat;
    h->row_off = row_off;
    h->slot_off = slot_off;
    h->h_rp = std::move(h_rp);
    h->h_col = std::move(h_col);
    h->h_diag_slot = std::move(diag_slot);
    h->h_w.assign((size_t)K, 1.0);
    for (int st = 0; st < 3; ++st) {
        h->relax_shape[st] = default_shape(st, K);
        // distances: the sweeps' row order, one vector per lane, two gathers per batch
        h->edge_shape[st] = Shape{P_of(st, K), 1, 2, 2};
    }
    cudaGetDevice(&h->device);

    auto bail = [&](int rc) {
        g_create_err = h->err;
        amgd_destroy(h);
        return rc;
    };
    int rc;
#define TRY(expr)                                                          \
    do {                                                                   \
        cudaError_t e__ = (expr);                                          \
        if (e__ != cudaSuccess) return bail(cuda_fail(h, e__, #expr));     \
    } while (0)
    TRY(dalloc(&h->rp_o, (size_t)n + 1 + 4));      // +16 bytes: widened bulk copies
    TRY(dalloc(&h->col_o, (size_t)h->nnz + 16));  // +64 bytes: widened bulk copies, 16-slot loads
    TRY(dalloc(&h->val_o, (size_t)h->nnz + 4));
    TRY(dalloc(&h->mat_off, (size_t)nmat + 1));
    TRY(cudaMemcpy(h->rp_o, h->h_rp.data(), (n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
    if (h->nnz) {
        TRY(cudaMemcpy(h->col_o, h->h_col.data(), h->nnz * sizeof(int32_t), cudaMemcpyHostToDevice));
        TRY(cudaMemcpy(h->val_o, h_val.data(), h->nnz * sizeof(double), cudaMemcpyHostToDevice));
    }
    TRY(cudaMemcpy(h->mat_off, row_off.data(), (nmat + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    TRY(dalloc(&h->diag_slot, (size_t)n));
    TRY(dalloc(&h->err_word, 1));
    TRY(dalloc(&h->status, 1));
    TRY(cudaMemset(h->status, 0, sizeof(uint32_t)));
    // test hooks for the bounded-wait path (never set in normal use):
    // AMGD_TEST_STAGING_EXTRA_TX declares bytes that no copy delivers, so the
    // first staged wait runs out; AMGD_TEST_WAIT_LIMIT shortens the waits.
    if (const char *e = getenv("AMGD_TEST_STAGING_EXTRA_TX")) h->test_extra_tx = (uint32_t)atoi(e);
    if (const char *e = getenv("AMGD_TEST_WAIT_LIMIT")) h->wait_limit = atoll(e);
    if (n) TRY(cudaMemcpy(h->diag_slot, h->h_diag_slot.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice));
    h->prp = h->rp_o;
    h->pcol = h->col_o;
    h->nnz_p = h->nnz;
    h->E_p = h->E;
    if ((rc = build_edge_tiles(h, h->h_rp)) != AMGD_OK) return bail(rc);
    h->rp_p = h->rp_o;
    h->col_p = h->col_o;
    h->val64 = h->val_o;
    TRY(dalloc(&h->diag64, (size_t)n));
    TRY(dalloc(&h->diag32, (size_t)n));
    TRY(dalloc(&h->diag64_o, (size_t)n));
    TRY(dalloc(&h->diag32_o, (size_t)n));
    {
        cudaError_t e = launch_diagonal(h->rp_p, h->col_p, h->val64, h->diag64, h->diag32,
                                        (int32_t)n, h->stream);
        if (e == cudaSuccess)
            e = launch_diagonal(h->rp_o, h->col_o, h->val_o, h->diag64_o, h->diag32_o, (int32_t)n,
                                h->stream);
        if (e != cudaSuccess) return bail(cuda_fail(h, e, "launch_diagonal"));
    }
    h->color_start = {0, n};
    TRY(dalloc(&h->flag, (size_t)h->nnz_p + 16));   // 16-byte loads past the end
    TRY(dalloc(&h->defer_count, 1));
    TRY(dalloc(&h->defer_list, (size_t)n));
    TRY(dalloc(&h->count, (size_t)n));
    TRY(dalloc(&h->tile, (size_t)(n / kTileRows + 2)));
    if ((rc = alloc_slot_outputs(h, ST_FP64)) != AMGD_OK) return bail(rc);
    if ((rc = alloc_vectors(h, ST_FP64, &h->x[0], &h->x[1])) != AMGD_OK) return bail(rc);
    if ((rc = upload_weights(h)) != AMGD_OK) return bail(rc);
    if ((rc = run_init(h, seed, h->stream)) != AMGD_OK) return bail(rc);
    TRY(cudaStreamSynchronize(h->stream));
#if AMGD_CHECKS
    // checked build only: AMGD_TEST_BAD_COLUMN=<slot> stores the out-of-range
    // column index n + 1000 at that slot of the sweeps' pattern after every
    // setup kernel has run, so a test can watch a gather's bounds test fire
    // (the next synchronising call returns AMGD_ERR_CHECK)
    if (const char *e = getenv("AMGD_TEST_BAD_COLUMN")) {
        const long long slot = atoll(e);
        if (slot >= 0 && slot < h->nnz) {
            const int32_t bad = (int32_t)n + 1000;
            TRY(cudaMemcpy(h->col_p + slot, &bad, sizeof bad, cudaMemcpyHostToDevice));
        }
    }
#endif
#undef TRY
    *out = h;
    return AMGD_OK;
}

}  // namespace

void amgd::set_thread_error(const std::string &msg) { g_create_err = msg; }

extern "C" {

int amgd_create(const int64_t *row_ptr, const int32_t *col, const double *val, int64_t n,
                int32_t K, uint64_t seed, int mem, amgd_handle *out)
{
    return create_impl(1, &row_ptr, &col, &val, &n, K, seed, mem, out);
}

int amgd_create_batch(int32_t nmat, const int64_t *const *row_ptr, const int32_t *const *col,
                      const double *const *val, const int64_t *n, int32_t K, uint64_t seed,
                      int mem, amgd_handle *out)
{
    return create_impl(nmat, row_ptr, col, val, n, K, seed, mem, out);
}

int amgd_batch_offsets(amgd_handle h, int64_t *row_off, int64_t *slot_off)
{
    if (!h) return AMGD_ERR_ARG;
    if (row_off) std::memcpy(row_off, h->row_off.data(), h->row_off.size() * sizeof(int64_t));
    if (slot_off) std::memcpy(slot_off, h->slot_off.data(), h->slot_off.size() * sizeof(int64_t));
    return AMGD_OK;
}

int amgd_sizes(amgd_handle h, int64_t *n, int64_t *nnz, int64_t *E, int32_t *K, int32_t *nmat)
{
    if (!h) return AMGD_ERR_ARG;
    if (n) *n = h->n;
    if (nnz) *nnz = h->nnz;
    if (E) *E = h->E;
    if (K) *K = h->K;
    if (nmat) *nmat = h->nmat;
    return AMGD_OK;
}

int amgd_set_stream(amgd_handle h, void *stream)
{
    if (!h) return AMGD_ERR_ARG;
    h->stream = (cudaStream_t)stream;
    return AMGD_OK;
}

int amgd_set_precision(amgd_handle h, int storage)
{
    AMGD_RANGE("amgd_set_precision");
    if (!h) return AMGD_ERR_ARG;
    if (h->async_pending) return fail(h, AMGD_ERR_STATE, "asynchronous work pending: call amgd_sync first");
    if (storage != AMGD_FP64 && storage != AMGD_FP32 && storage != AMGD_BF16)
        return fail(h, AMGD_ERR_ARG, "unknown storage precision");
    if (storage == h->storage) return AMGD_OK;
    CK(h, cudaStreamSynchronize(h->stream));
    drop_graph(h);                       // vector and output buffers are reallocated
    if (storage != ST_FP64 && !h->val32) {
        CK(h, dalloc(&h->val32, (size_t)h->nnz + 4));
        CK(h, dalloc(&h->val32_o, (size_t)h->nnz + 4));
        int rc = permute_values(h);
        if (rc != AMGD_OK) return rc;
    }
    // re-layout the current vectors: export to caller-order doubles, import
    CK(h, ensure_tmp64(h, (size_t)h->n * h->K));
    CK(h, launch_export(h->storage, h->x[h->cur], h->tmp64, h->perm, (int32_t)h->n, h->K,
                        Kp_of(h->storage, h->K), h->stream));
    void *nx[2] = {nullptr, nullptr};
    int rc = alloc_vectors(h, storage, &nx[0], &nx[1]);
    if (rc != AMGD_OK) return rc;
    cudaError_t e = launch_import(storage, h->tmp64, nx[0], h->perm, (int32_t)h->n, h->K,
                                  Kp_of(storage, h->K), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        cudaFree(nx[0]);
        cudaFree(nx[1]);
        return cuda_fail(h, e, "import vectors");
    }
    const bool slot_type_changes = (storage == ST_FP64) != (h->storage == ST_FP64);
    cudaFree(h->x[0]);
    cudaFree(h->x[1]);
    h->x[0] = nx[0];
    h->x[1] = nx[1];
    if (h->x_caller) {
        cudaFree(h->x_caller);
        h->x_caller = nullptr;
        const size_t bytes = (size_t)h->n * Kp_of(storage, h->K) * esize(storage);
        CK(h, cudaMalloc(&h->x_caller, bytes ? bytes : 16));
    }
    h->cur = 0;
    h->storage = storage;
    if (slot_type_changes) {
        rc = alloc_slot_outputs(h, storage);
        if (rc != AMGD_OK) return rc;
    }
    h->have_dist = false;
    h->traj_valid = false;
    return AMGD_OK;
}

int amgd_set_target(amgd_handle h, int target)
{
    if (!h) return AMGD_ERR_ARG;
    if (target != AMGD_TARGET_RESIDUAL && target != AMGD_TARGET_PLAIN)
        return fail(h, AMGD_ERR_ARG, "unknown target");
    h->target = target;
    h->have_dist = false;
    h->traj_valid = false;
    return AMGD_OK;
}

int amgd_set_summation(amgd_handle h, int mode)
{
    if (!h) return AMGD_ERR_ARG;
    if (mode != AMGD_SUM_PLAIN && mode != AMGD_SUM_COMPENSATED)
        return fail(h, AMGD_ERR_ARG, "unknown summation mode");
    if (mode != h->summation) {
        drop_graph(h);
        h->summation = mode;
    }
    h->have_dist = false;
    h->traj_valid = false;
    return AMGD_OK;
}

int amgd_set_weights(amgd_handle h, const double *w)
{
    if (!h) return AMGD_ERR_ARG;
    std::vector<double> nw((size_t)h->K, 1.0);
    if (w) {
        for (int k = 0; k < h->K; ++k) {
            if (!(w[k] > 0.0) || !std::isfinite(w[k])) return fail(h, AMGD_ERR_ARG, "weights must be > 0 and finite");
            nw[(size_t)k] = w[k];
        }
    }
    h->h_w = nw;
    h->have_dist = false;
    h->traj_valid = false;
    return upload_weights(h);
}

int amgd_set_coloring(amgd_handle h, const int32_t *color, int32_t ncolors, int mem)
{
    AMGD_RANGE("amgd_set_coloring");
    if (!h) return AMGD_ERR_ARG;
    if (h->async_pending) return fail(h, AMGD_ERR_STATE, "asynchronous work pending: call amgd_sync first");
    if (ncolors < 1 || (!color && h->n > 0)) return fail(h, AMGD_ERR_ARG, "bad coloring arguments");
    const int64_t n = h->n;
    std::vector<int32_t> c((size_t)n);
    CK(h, fetch(c.data(), color, n * sizeof(int32_t), mem));
    std::vector<int64_t> start((size_t)ncolors + 1, 0);
    for (int64_t i = 0; i < n; ++i) {
        if (c[(size_t)i] < 0 || c[(size_t)i] >= ncolors) return fail(h, AMGD_ERR_ARG, "color out of range");
        ++start[(size_t)c[(size_t)i] + 1];
    }
    for (int32_t k = 0; k < ncolors; ++k) start[(size_t)k + 1] += start[(size_t)k];
    // stable counting sort: perm[new] = old, inv[old] = new
    std::vector<int32_t> perm((size_t)n), inv((size_t)n);
    std::vector<int64_t> next(start.begin(), start.end() - 1);
    for (int64_t i = 0; i < n; ++i) {
        const int64_t r = next[(size_t)c[(size_t)i]]++;
        perm[(size_t)r] = (int32_t)i;
        inv[(size_t)i] = (int32_t)r;
    }
    CK(h, cudaStreamSynchronize(h->stream));
    drop_graph(h);                       // the row order of the sweeps changes
    std::vector<int32_t> rp_p((size_t)n + 1, 0), col_p((size_t)h->nnz);
    for (int64_t r = 0; r < n; ++r) {
        const int32_t o = perm[(size_t)r];
        const int32_t len = h->h_rp[(size_t)o + 1] - h->h_rp[(size_t)o];
        rp_p[(size_t)r + 1] = rp_p[(size_t)r] + len;
        for (int32_t k = 0; k < len; ++k)
            col_p[(size_t)(rp_p[(size_t)r] + k)] = inv[(size_t)h->h_col[(size_t)(h->h_rp[(size_t)o] + k)]];
    }
    // current vectors out in caller order before the layout changes
    CK(h, ensure_tmp64(h, (size_t)n * h->K));
    CK(h, launch_export(h->storage, h->x[h->cur], h->tmp64, h->perm, (int32_t)n, h->K,
                        Kp_of(h->storage, h->K), h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (!h->perm) {
        CK(h, dalloc(&h->perm, (size_t)n));
        CK(h, dalloc(&h->rp_p, (size_t)n + 1 + 4));
        CK(h, dalloc(&h->col_p, (size_t)h->nnz + 4));
        CK(h, dalloc(&h->val64, (size_t)h->nnz + 4));
    }
    if (!h->x_caller) {
        const size_t bytes = (size_t)n * Kp_of(h->storage, h->K) * esize(h->storage);
        CK(h, cudaMalloc(&h->x_caller, bytes ? bytes : 16));
    }
    CK(h, cudaMemcpy(h->perm, perm.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->rp_p, rp_p.data(), (n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->col_p, col_p.data(), h->nnz * sizeof(int32_t), cudaMemcpyHostToDevice));
    {
        // the distance pass reads the sweeps' row order in place: the caller CSR
        // with its columns renumbered, and the permuted row of every caller row
        std::vector<int32_t> cx((size_t)h->nnz);
        for (int64_t p = 0; p < h->nnz; ++p) cx[(size_t)p] = inv[(size_t)h->h_col[(size_t)p]];
        if (!h->pinv) CK(h, dalloc(&h->pinv, (size_t)(n ? n : 1)));
        if (!h->colx) CK(h, dalloc(&h->colx, (size_t)h->nnz + 16));
        CK(h, cudaMemcpy(h->pinv, inv.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice));
        CK(h, cudaMemcpy(h->colx, cx.data(), h->nnz * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    {
        std::vector<int32_t> sp((size_t)h->nnz);
        for (int64_t r = 0; r < n; ++r) {
            const int32_t o = perm[(size_t)r];
            for (int32_t k = 0; k < h->h_rp[(size_t)o + 1] - h->h_rp[(size_t)o]; ++k)
                sp[(size_t)(h->h_rp[(size_t)o] + k)] = rp_p[(size_t)r] + k;
        }
        if (!h->slot_perm) CK(h, dalloc(&h->slot_perm, (size_t)(h->nnz ? h->nnz : 1)));
        if (h->nnz)
            CK(h, cudaMemcpy(h->slot_perm, sp.data(), h->nnz * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    int rc = permute_values(h);
    if (rc != AMGD_OK) return rc;
    CK(h, launch_import(h->storage, h->tmp64, h->x[h->cur], h->perm, (int32_t)n, h->K,
                        Kp_of(h->storage, h->K), h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    h->color_start = start;
    h->have_dist = false;
    h->traj_valid = false;
    return AMGD_OK;
}

int amgd_set_matrix_ids(amgd_handle h, const int64_t *ids)
{
    AMGD_RANGE("amgd_set_matrix_ids");
    if (!h) return AMGD_ERR_ARG;
    if (h->async_pending) return fail(h, AMGD_ERR_STATE, "asynchronous work pending: call amgd_sync first");
    CK(h, cudaStreamSynchronize(h->stream));
    drop_graph(h);                       // a captured start uses the old keys
    if (!ids) {
        dfree(h->mat_id);
        h->mat_id = nullptr;
        return AMGD_OK;
    }
    for (int32_t b = 0; b < h->nmat; ++b)
        if (ids[b] < 0) return fail(h, AMGD_ERR_ARG, "matrix id < 0");
    if (!h->mat_id) CK(h, dalloc(&h->mat_id, (size_t)h->nmat));
    CK(h, cudaMemcpy(h->mat_id, ids, (size_t)h->nmat * sizeof(int64_t), cudaMemcpyHostToDevice));
    return AMGD_OK;
}

int amgd_init_vectors(amgd_handle h, uint64_t seed)
{
    AMGD_RANGE("amgd_init_vectors");
    if (!h) return AMGD_ERR_ARG;
    return run_init(h, seed, h->stream);
}

int amgd_set_vectors(amgd_handle h, const double *X, int mem)
{
    if (!h) return AMGD_ERR_ARG;
    if (!X && h->n) return fail(h, AMGD_ERR_ARG, "X is NULL");
    const size_t cnt = (size_t)h->n * h->K;
    const double *src = X;
    if (mem == AMGD_MEM_HOST) {
        CK(h, ensure_tmp64(h, cnt));
        CK(h, cudaMemcpyAsync(h->tmp64, X, cnt * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        src = h->tmp64;
    } else if (mem != AMGD_MEM_DEVICE) {
        return fail(h, AMGD_ERR_ARG, "bad mem");
    }
    CK(h, launch_import(h->storage, src, h->x[h->cur], h->perm, (int32_t)h->n, h->K,
                        Kp_of(h->storage, h->K), h->stream));
    if (mem == AMGD_MEM_HOST) CK(h, cudaStreamSynchronize(h->stream));
    h->have_dist = false;
    h->traj_valid = false;
    return AMGD_OK;
}

int amgd_get_vectors(amgd_handle h, double *X, int mem)
{
    if (!h) return AMGD_ERR_ARG;
    if (!X && h->n) return fail(h, AMGD_ERR_ARG, "X is NULL");
    const size_t cnt = (size_t)h->n * h->K;
    if (mem == AMGD_MEM_DEVICE) {
        CK(h, launch_export(h->storage, h->x[h->cur], X, h->perm, (int32_t)h->n, h->K,
                            Kp_of(h->storage, h->K), h->stream));
        return AMGD_OK;
    }
    if (mem != AMGD_MEM_HOST) return fail(h, AMGD_ERR_ARG, "bad mem");
    CK(h, ensure_tmp64(h, cnt));
    CK(h, launch_export(h->storage, h->x[h->cur], h->tmp64, h->perm, (int32_t)h->n, h->K,
                        Kp_of(h->storage, h->K), h->stream));
    CK(h, cudaMemcpyAsync(X, h->tmp64, cnt * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return poll_status(h);
}

int amgd_set_values(amgd_handle h, const double *val, int mem)
{
    AMGD_RANGE("amgd_set_values");
    if (!h) return AMGD_ERR_ARG;
    if (!val && h->nnz) return fail(h, AMGD_ERR_ARG, "val is NULL");
    if (mem != AMGD_MEM_HOST && mem != AMGD_MEM_DEVICE) return fail(h, AMGD_ERR_ARG, "bad mem");
    // stage on the device, check there, then swap the staging buffer in
    CK(h, ensure_tmp64(h, (size_t)h->nnz + 4));
    CK(h, cudaMemcpyAsync(h->tmp64, val, h->nnz * sizeof(double),
                          mem == AMGD_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                          h->stream));
    CK(h, cudaMemsetAsync(h->err_word, 0, sizeof(uint32_t), h->stream));
    CK(h, launch_check_values(h->tmp64, h->nnz, h->diag_slot, (int32_t)h->n, h->err_word, h->stream));
    uint32_t err = 0;
    CK(h, cudaMemcpyAsync(&err, h->err_word, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (err & 1u) return fail(h, AMGD_ERR_CSR, "non-finite value");
    if (err & 2u) return fail(h, AMGD_ERR_ZERO_DIAG, "zero diagonal");
    // written in place: device pointers held by a captured graph stay valid
    int rc = permute_values(h, h->tmp64);
    if (rc != AMGD_OK) return rc;
    h->have_dist = false;
    h->traj_valid = false;
    return AMGD_OK;
}

namespace {

int async_setup(amgd_ctx *h)
{
    if (h->up_stream) return AMGD_OK;
    CK(h, cudaStreamCreateWithFlags(&h->up_stream, cudaStreamNonBlocking));
    CK(h, cudaStreamCreateWithFlags(&h->down_stream, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
        CK(h, cudaEventCreateWithFlags(&h->ev_up[k], cudaEventDisableTiming));
        CK(h, cudaEventCreateWithFlags(&h->ev_used[k], cudaEventDisableTiming));
        CK(h, cudaEventCreateWithFlags(&h->ev_res[k], cudaEventDisableTiming));
        CK(h, cudaEventCreateWithFlags(&h->ev_down[k], cudaEventDisableTiming));
    }
    CK(h, dalloc(&h->async_err, 1));
    CK(h, cudaMemset(h->async_err, 0, sizeof(uint32_t)));
    return AMGD_OK;
}

}  // namespace

int amgd_set_values_async(amgd_handle h, const double *val, int mem)
{
    AMGD_RANGE("amgd_set_values_async");
    if (!h) return AMGD_ERR_ARG;
    if (!val && h->nnz) return fail(h, AMGD_ERR_ARG, "val is NULL");
    if (mem != AMGD_MEM_HOST && mem != AMGD_MEM_DEVICE) return fail(h, AMGD_ERR_ARG, "bad mem");
    int rc = async_setup(h);
    if (rc != AMGD_OK) return rc;
    if (!h->stage[0]) {
        CK(h, dalloc(&h->stage[0], (size_t)h->nnz + 4));
        CK(h, dalloc(&h->stage[1], (size_t)h->nnz + 4));
    }
    const int k = h->up_slot;
    h->up_slot ^= 1;
    // the slot's previous contents must have been applied before it is refilled
    CK(h, cudaStreamWaitEvent(h->up_stream, h->ev_used[k], 0));
    CK(h, cudaMemcpyAsync(h->stage[k], val, h->nnz * sizeof(double),
                          mem == AMGD_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                          h->up_stream));
    CK(h, cudaEventRecord(h->ev_up[k], h->up_stream));
    CK(h, cudaStreamWaitEvent(h->stream, h->ev_up[k], 0));
    // the value checks ride on the copies (their bits land in the error word
    // the next synchronising call reads)
    rc = permute_values(h, h->stage[k], h->async_err);
    if (rc != AMGD_OK) return rc;
    CK(h, cudaEventRecord(h->ev_used[k], h->stream));
    h->async_pending = true;
    h->have_dist = false;
    h->traj_valid = false;
    return AMGD_OK;
}

int amgd_strength_async(amgd_handle h, int64_t *s_row_ptr, int32_t *s_col, int64_t cap, int mem)
{
    AMGD_RANGE("amgd_strength_async");
    if (!h) return AMGD_ERR_ARG;
    if (!h->have_dist) return fail(h, AMGD_ERR_STATE, "amgd_distances or a captured build must run first");
    if (!s_row_ptr || (!s_col && cap > 0) || cap < 0) return fail(h, AMGD_ERR_ARG, "bad output buffers");
    if (mem != AMGD_MEM_HOST && mem != AMGD_MEM_DEVICE) return fail(h, AMGD_ERR_ARG, "bad mem");
    int rc = async_setup(h);
    if (rc != AMGD_OK) return rc;
    if (!h->res_rp[0] || h->res_col_len < h->E_p) {
        CK(h, cudaStreamSynchronize(h->down_stream));
        CK(h, cudaStreamSynchronize(h->stream));
        for (int k = 0; k < 2; ++k) {
            dfree(h->res_col[k]);
            h->res_col[k] = nullptr;
            if (!h->res_rp[k]) CK(h, dalloc(&h->res_rp[k], (size_t)h->n + 1));
        }
        h->res_col_len = 0;
        for (int k = 0; k < 2; ++k) CK(h, dalloc(&h->res_col[k], (size_t)(h->E_p > 0 ? h->E_p : 1)));
        h->res_col_len = h->E_p;
    }
    const int k = h->res_slot;
    h->res_slot ^= 1;
    // the slot's previous copy to the caller must be done before it is rewritten
    CK(h, cudaStreamWaitEvent(h->stream, h->ev_down[k], 0));
    CK(h, launch_strength(h->count, h->prp, h->pcol, h->flag, (int32_t)h->n, h->tile, h->res_rp[k],
                          h->res_col[k], h->stream));
    CK(h, cudaEventRecord(h->ev_res[k], h->stream));
    CK(h, cudaStreamWaitEvent(h->down_stream, h->ev_res[k], 0));
    const cudaMemcpyKind kind = mem == AMGD_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    CK(h, cudaMemcpyAsync(s_row_ptr, h->res_rp[k], ((size_t)h->n + 1) * sizeof(int64_t), kind, h->down_stream));
    const int64_t ncol = cap < h->E_p ? cap : h->E_p;
    if (ncol > 0)
        CK(h, cudaMemcpyAsync(s_col, h->res_col[k], (size_t)ncol * sizeof(int32_t), kind, h->down_stream));
    CK(h, cudaEventRecord(h->ev_down[k], h->down_stream));
    h->pending_out.push_back({s_row_ptr, mem, cap});
    h->async_pending = true;
    return AMGD_OK;
}

int amgd_sync(amgd_handle h)
{
    AMGD_RANGE("amgd_sync");
    if (!h) return AMGD_ERR_ARG;
    CK(h, cudaStreamSynchronize(h->stream));
    if (h->up_stream) {
        CK(h, cudaStreamSynchronize(h->up_stream));
        CK(h, cudaStreamSynchronize(h->down_stream));
    }
    h->async_pending = false;
    std::vector<amgd_ctx::PendingOut> outs;
    outs.swap(h->pending_out);
    if (h->async_err) {
        uint32_t err = 0;
        CK(h, cudaMemcpy(&err, h->async_err, sizeof err, cudaMemcpyDeviceToHost));
        if (err) {
            CK(h, cudaMemset(h->async_err, 0, sizeof err));
            h->have_dist = false;
            if (err & 1u) return fail(h, AMGD_ERR_CSR, "an asynchronous value update had a non-finite value");
            return fail(h, AMGD_ERR_ZERO_DIAG, "an asynchronous value update had a zero diagonal");
        }
    }
    for (const auto &o : outs) {
        int64_t total = 0;
        if (o.mem == AMGD_MEM_HOST) total = o.rp[h->n];
        else CK(h, cudaMemcpy(&total, o.rp + h->n, sizeof total, cudaMemcpyDeviceToHost));
        if (total > o.cap)
            return fail(h, AMGD_ERR_CAPACITY, "strength output needs " + std::to_string(total) + " columns");
    }
    return poll_status(h);
}

int amgd_relax(amgd_handle h, int32_t nu, double omega, int sweep_type)
{
    AMGD_RANGE("amgd_relax");
    if (!h) return AMGD_ERR_ARG;
    if (nu < 0 || !std::isfinite(omega)) return fail(h, AMGD_ERR_ARG, "nu < 0 or omega not finite");
    if (sweep_type != AMGD_SWEEP_JACOBI && sweep_type != AMGD_SWEEP_MCGS)
        return fail(h, AMGD_ERR_ARG, "unknown sweep type");
    if (sweep_type == AMGD_SWEEP_MCGS && !h->perm)
        return fail(h, AMGD_ERR_STATE, "MCGS needs amgd_set_coloring first");
    if (h->ckpt_every > 0 && sweep_type == AMGD_SWEEP_JACOBI && !h->perm)
        return run_relax_recorded(h, nu, omega, h->stream);
    return run_relax(h, nu, omega, sweep_type, h->stream);
}

int amgd_distances(amgd_handle h, double theta, double *a, double *dist, double *ls, int mem)
{
    AMGD_RANGE("amgd_distances");
    if (!h) return AMGD_ERR_ARG;
    if (!(theta >= 0.0) || !std::isfinite(theta)) return fail(h, AMGD_ERR_ARG, "theta must be finite and >= 0");
    if (mem != AMGD_MEM_HOST && mem != AMGD_MEM_DEVICE) return fail(h, AMGD_ERR_ARG, "bad mem");
    int rc = run_edge(h, theta, h->stream);
    if (rc != AMGD_OK) return rc;
    double *outs[3] = {a, dist, ls};
    if (mem == AMGD_MEM_DEVICE) {
        if (a || dist || ls)
            CK(h, launch_export_slots(h->storage, h->a, h->ls, a, dist, ls, h->nnz_p, h->stream));
        return AMGD_OK;
    }
    for (int k = 0; k < 3; ++k) {
        if (!outs[k]) continue;
        CK(h, ensure_tmp64(h, (size_t)h->nnz_p));
        CK(h, launch_export_slots(h->storage, h->a, h->ls, k == 0 ? h->tmp64 : nullptr,
                                  k == 1 ? h->tmp64 : nullptr, k == 2 ? h->tmp64 : nullptr,
                                  h->nnz_p, h->stream));
        CK(h, cudaMemcpyAsync(outs[k], h->tmp64, h->nnz_p * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CK(h, cudaStreamSynchronize(h->stream));
    }
    return poll_status(h);
}

int amgd_strength(amgd_handle h, int64_t *s_row_ptr, int32_t *s_col, int64_t cap,
                  int64_t *nnz_s, int mem)
{
    AMGD_RANGE("amgd_strength");
    if (!h) return AMGD_ERR_ARG;
    if (!h->have_dist) return fail(h, AMGD_ERR_STATE, "amgd_distances must run first");
    if (!s_row_ptr || (!s_col && cap > 0) || cap < 0) return fail(h, AMGD_ERR_ARG, "bad output buffers");
    if (mem != AMGD_MEM_HOST && mem != AMGD_MEM_DEVICE) return fail(h, AMGD_ERR_ARG, "bad mem");
    if (mem == AMGD_MEM_DEVICE && cap >= h->E_p) {
        CK(h, launch_strength(h->count, h->prp, h->pcol, h->flag, (int32_t)h->n, h->tile,
                              s_row_ptr, s_col, h->stream));
        if (nnz_s) {
            CK(h, cudaMemcpyAsync(nnz_s, s_row_ptr + h->n, sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream));
            CK(h, cudaStreamSynchronize(h->stream));
        }
        return AMGD_OK;
    }
    if (!h->s_rp_tmp) CK(h, dalloc(&h->s_rp_tmp, (size_t)h->n + 1));
    if (!h->s_col_tmp) CK(h, dalloc(&h->s_col_tmp, (size_t)(h->E_p > 0 ? h->E_p : 1)));
    CK(h, launch_strength(h->count, h->prp, h->pcol, h->flag, (int32_t)h->n, h->tile,
                          h->s_rp_tmp, h->s_col_tmp, h->stream));
    int64_t total = 0;
    CK(h, cudaMemcpyAsync(&total, h->s_rp_tmp + h->n, sizeof(int64_t), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    {
        const int rc = poll_status(h);
        if (rc != AMGD_OK) return rc;
    }
    if (nnz_s) *nnz_s = total;
    if (total > cap) return fail(h, AMGD_ERR_CAPACITY, "strength output needs " + std::to_string(total) + " columns");
    const cudaMemcpyKind k = mem == AMGD_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    CK(h, cudaMemcpyAsync(s_row_ptr, h->s_rp_tmp, (h->n + 1) * sizeof(int64_t), k, h->stream));
    if (total) CK(h, cudaMemcpyAsync(s_col, h->s_col_tmp, total * sizeof(int32_t), k, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    return AMGD_OK;
}

int amgd_graph_capture(amgd_handle h, uint64_t seed, int32_t nu, double omega, int sweep_type,
                       double theta, int64_t *s_row_ptr, int32_t *s_col, int64_t cap)
{
    AMGD_RANGE("amgd_graph_capture");
    if (!h) return AMGD_ERR_ARG;
    if (h->async_pending) return fail(h, AMGD_ERR_STATE, "asynchronous work pending: call amgd_sync first");
    if (nu < 0 || !std::isfinite(omega)) return fail(h, AMGD_ERR_ARG, "nu < 0 or omega not finite");
    if (!(theta >= 0.0) || !std::isfinite(theta)) return fail(h, AMGD_ERR_ARG, "theta must be finite and >= 0");
    if (sweep_type != AMGD_SWEEP_JACOBI && sweep_type != AMGD_SWEEP_MCGS)
        return fail(h, AMGD_ERR_ARG, "unknown sweep type");
    if (sweep_type == AMGD_SWEEP_MCGS && !h->perm)
        return fail(h, AMGD_ERR_STATE, "MCGS needs amgd_set_coloring first");
    if (!s_row_ptr || (!s_col && h->E_p > 0)) return fail(h, AMGD_ERR_ARG, "bad output buffers");
    if (cap < h->E_p) return fail(h, AMGD_ERR_CAPACITY, "graph capture needs cap >= the pattern's off-diagonal count");
    if (!h->cap_stream) CK(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
    if (h->graph) { cudaGraphDestroy(h->graph); h->graph = nullptr; }
    CK(h, cudaStreamSynchronize(h->stream));
    const int cur0 = h->cur;
    h->cur = 0;
    if (h->phase_timing && !h->ev[0])
        for (auto &e : h->ev) CK(h, cudaEventCreate(&e));
    const bool timed = h->phase_timing;
    auto mark = [&](int k) {
        return timed ? cudaEventRecordWithFlags(h->ev[k], h->cap_stream, cudaEventRecordExternal)
                     : cudaSuccess;
    };
    CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = AMGD_OK;
    cudaError_t me = mark(0);
    if (me == cudaSuccess) rc = run_init(h, seed, h->cap_stream);
    if (me == cudaSuccess && rc == AMGD_OK) me = mark(1);
    if (me == cudaSuccess && rc == AMGD_OK) rc = run_relax(h, nu, omega, sweep_type, h->cap_stream);
    if (me == cudaSuccess && rc == AMGD_OK) me = mark(2);
    if (me == cudaSuccess && rc == AMGD_OK) rc = run_edge(h, theta, h->cap_stream);
    if (me == cudaSuccess && rc == AMGD_OK) me = mark(3);
    if (me == cudaSuccess && rc == AMGD_OK) {
        cudaError_t e = launch_strength(h->count, h->prp, h->pcol, h->flag, (int32_t)h->n,
                                        h->tile, s_row_ptr, s_col, h->cap_stream);
        if (e != cudaSuccess) rc = cuda_fail(h, e, "launch_strength (capture)");
    }
    if (me == cudaSuccess && rc == AMGD_OK) me = mark(4);
    if (me != cudaSuccess && rc == AMGD_OK) rc = cuda_fail(h, me, "cudaEventRecordWithFlags (capture)");
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    h->graph_cur_after = h->cur;
    h->cur = cur0;
    h->have_dist = false;
    h->traj_valid = false;
    if (rc != AMGD_OK) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    h->graph = g;
    CK(h, cudaGraphInstantiate(&h->gexec, h->graph, 0));
    h->graph_timed = timed;
    h->graph_is_backward = false;
    return AMGD_OK;
}

int amgd_set_kernel_shape(amgd_handle h, int kernel, int G, int NV, int U, int staged)
{
    if (!h) return AMGD_ERR_ARG;
    const Shape sh{G, NV, U, staged};
    if ((kernel != AMGD_KERNEL_RELAX && kernel != AMGD_KERNEL_EDGE) || !shape_ok(h->storage, h->K, sh) ||
        (kernel == AMGD_KERNEL_EDGE && !edge_shape_ok(sh)) ||
        (kernel == AMGD_KERNEL_RELAX && !relax_shape_available(h->storage, sh)))
        return fail(h, AMGD_ERR_ARG, "invalid kernel shape for this storage and K");
    (kernel == AMGD_KERNEL_RELAX ? h->relax_shape : h->edge_shape)[h->storage] = sh;
    return AMGD_OK;
}

int amgd_get_kernel_shape(amgd_handle h, int kernel, int *G, int *NV, int *U, int *staged)
{
    if (!h || (kernel != AMGD_KERNEL_RELAX && kernel != AMGD_KERNEL_EDGE)) return AMGD_ERR_ARG;
    const Shape sh = (kernel == AMGD_KERNEL_RELAX ? h->relax_shape : h->edge_shape)[h->storage];
    if (G) *G = sh.G;
    if (NV) *NV = sh.NV;
    if (U) *U = sh.U;
    if (staged) *staged = sh.stage;
    return AMGD_OK;
}

}  // extern "C"

namespace {

std::string tune_key(amgd_ctx *h, int sweep_type)
{
    cudaDeviceProp prop;
    std::string gpu = "unknown";
    if (cudaGetDeviceProperties(&prop, h->device) == cudaSuccess) gpu = prop.name;
    for (char &c : gpu)
        if (c == ';' || c == '=' || c == '\n') c = '_';
    int nb = 0;
    while (((int64_t)1 << (nb + 1)) <= h->n) ++nb;
    const long db = h->n ? (long)((h->nnz + h->n / 2) / h->n) : 0;
    return "gpu=" + gpu + ";st=" + std::to_string(h->storage) + ";K=" + std::to_string(h->K) +
           ";nb=" + std::to_string(nb) + ";db=" + std::to_string(db) +
           ";sweep=" + std::to_string(sweep_type) + ";colors=" +
           std::to_string(h->color_start.size() - 1) + ";sum=" + std::to_string(h->summation) +
           ";depth=" + std::to_string(h->depth);
}

bool parse_shape(const std::string &line, const char *tag, Shape &sh)
{
    const std::string t = std::string(";") + tag + "=";
    const size_t p = line.find(t);
    if (p == std::string::npos) return false;
    return sscanf(line.c_str() + p + t.size(), "%d,%d,%d,%d", &sh.G, &sh.NV, &sh.U, &sh.stage) == 4;
}

// median of `reps` timings (ms) of fn() on the handle's stream
template <class F>
int time_ms(amgd_ctx *h, F fn, int reps, float &out)
{
    cudaEvent_t a, b;
    CK(h, cudaEventCreate(&a));
    CK(h, cudaEventCreate(&b));
    std::vector<float> t;
    int rc = fn();                       // warm-up
    for (int k = 0; k < reps && rc == AMGD_OK; ++k) {
        cudaEventRecord(a, h->stream);
        rc = fn();
        cudaEventRecord(b, h->stream);
        cudaEventSynchronize(b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, a, b);
        t.push_back(ms);
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc != AMGD_OK) return rc;
    std::sort(t.begin(), t.end());
    out = t[t.size() / 2];
    return AMGD_OK;
}

}  // namespace

extern "C" {

int amgd_autotune(amgd_handle h, int sweep_type, double omega, const char *cache_path)
{
    AMGD_RANGE("amgd_autotune");
    if (!h) return AMGD_ERR_ARG;
    if (h->async_pending) return fail(h, AMGD_ERR_STATE, "asynchronous work pending: call amgd_sync first");
    if (sweep_type != AMGD_SWEEP_JACOBI && sweep_type != AMGD_SWEEP_MCGS)
        return fail(h, AMGD_ERR_ARG, "unknown sweep type");
    if (sweep_type == AMGD_SWEEP_MCGS && !h->perm)
        return fail(h, AMGD_ERR_STATE, "MCGS needs amgd_set_coloring first");
    if (!std::isfinite(omega)) return fail(h, AMGD_ERR_ARG, "omega not finite");
    const std::string key = tune_key(h, sweep_type);
    if (cache_path) {
        FILE *f = fopen(cache_path, "r");
        if (f) {
            char buf[1024];
            Shape r{0, 0, 0, 0}, e{0, 0, 0, 0};
            bool found = false;
            while (fgets(buf, sizeof buf, f)) {
                std::string line(buf);
                if (line.compare(0, key.size(), key) == 0 && line.size() > key.size() &&
                    line[key.size()] == ';' && parse_shape(line, "relax", r) &&
                    parse_shape(line, "edge", e) && shape_ok(h->storage, h->K, r) &&
                    shape_ok(h->storage, h->K, e) && edge_shape_ok(e) &&
                    relax_shape_available(h->storage, r))
                    found = true;       // the last matching line wins
            }
            fclose(f);
            if (found) {
                h->relax_shape[h->storage] = r;
                h->edge_shape[h->storage] = e;
                return AMGD_OK;
            }
        }
    }
    std::vector<Shape> cands;
    const int P = P_of(h->storage, h->K);
    for (int stage : {0, 1, 2, 3})
        for (int NV : {1, 2, 4})
            for (int U : {4, 8})
                if (P % NV == 0 && shape_ok(h->storage, h->K, Shape{P / NV, NV, U, stage}) &&
                    relax_shape_available(h->storage, Shape{P / NV, NV, U, stage}))
                    cands.push_back(Shape{P / NV, NV, U, stage});
    const Shape keep_r = h->relax_shape[h->storage], keep_e = h->edge_shape[h->storage];
    const int cur = h->cur;
    Shape best_r = keep_r, best_e = keep_e;
    float tr = 1e30f, te = 1e30f;
    for (const Shape &c : cands) {
        float ms = 0.f;
        h->relax_shape[h->storage] = c;
        // one sweep from the current vectors into the spare buffer (the
        // current vectors are not touched), then restore the buffer index
        int rc = time_ms(h, [&]() { int q = run_relax(h, 1, omega, sweep_type, h->stream); h->cur = cur; return q; }, 5, ms);
        if (rc != AMGD_OK) { h->relax_shape[h->storage] = keep_r; return rc; }
        if (ms < tr) { tr = ms; best_r = c; }
        {
            const int prc = poll_status(h);
            if (prc != AMGD_OK) { h->relax_shape[h->storage] = keep_r; return prc; }
        }
    }
    // edge pass: stage 0 row kernel, stage 1 tile kernel, stage 2 the row
    // kernel and stage 3 the warp-staged kernel on the sweeps' row order
    // (search depth 1)
    for (int stage : {0, 1, 2, 3})
        for (int NV : {1, 2, 4})
            for (int U : {2, 4, 8}) {
                const Shape c{P / NV, NV, U, stage};
                if (P % NV != 0 || !shape_ok(h->storage, h->K, c) || !edge_shape_ok(c)) continue;
                if (stage >= 2 && h->depth > 1) continue;
                float ms = 0.f;
                h->edge_shape[h->storage] = c;
                const int rc = time_ms(h, [&]() { return run_edge(h, 0.5, h->stream); }, 5, ms);
                if (rc != AMGD_OK) { h->edge_shape[h->storage] = keep_e; return rc; }
                if (ms < te) { te = ms; best_e = c; }
            }
    h->relax_shape[h->storage] = best_r;
    h->edge_shape[h->storage] = best_e;
    h->cur = cur;
    h->have_dist = false;
    h->traj_valid = false;
    if (cache_path) {
        FILE *f = fopen(cache_path, "a");
        if (f) {
            fprintf(f, "%s;relax=%d,%d,%d,%d;edge=%d,%d,%d,%d;relax_ms=%.5f;edge_ms=%.5f\n",
                    key.c_str(), best_r.G, best_r.NV, best_r.U, best_r.stage, best_e.G, best_e.NV,
                    best_e.U, best_e.stage, tr, te);
            fclose(f);
        }
    }
    return AMGD_OK;
}

int amgd_enable_phase_timing(amgd_handle h, int enable)
{
    if (!h) return AMGD_ERR_ARG;
    h->phase_timing = enable != 0;
    return AMGD_OK;
}

int amgd_phase_times(amgd_handle h, float *ms)
{
    if (!h || !ms) return AMGD_ERR_ARG;
    if (!h->gexec || !h->graph_timed) return fail(h, AMGD_ERR_STATE, "no timed graph captured");
    CK(h, cudaEventSynchronize(h->ev[4]));
    for (int k = 0; k < 4; ++k) CK(h, cudaEventElapsedTime(&ms[k], h->ev[k], h->ev[k + 1]));
    return poll_status(h);
}

int amgd_graph_launch(amgd_handle h)
{
    AMGD_RANGE("amgd_graph_launch");
    if (!h) return AMGD_ERR_ARG;
    if (!h->gexec) return fail(h, AMGD_ERR_STATE, "no captured graph");
    CK(h, cudaGraphLaunch(h->gexec, h->stream));
    h->cur = h->graph_cur_after;
    h->have_dist = true;
    if (h->graph_is_backward) {
        h->traj_valid = true;
        h->traj_nu = h->graph_traj_nu;
        h->traj_omega = h->graph_traj_omega;
    }
    return AMGD_OK;
}

namespace {

// V_i = { j : (A^d)_ij != 0 } (§4.1, Eq. (4.2)) without forming A^d: every
// row of A holds its diagonal, so j is in V_i exactly when the graph of A has
// a path of at most d steps from i to j (d-level breadth-first search;
// columns ascending).  Returns false if the pattern exceeds `limit` entries.
bool depth_pattern(const std::vector<int32_t> &rp, const std::vector<int32_t> &col, int64_t n,
                   int32_t d, int64_t limit, std::vector<int32_t> &prp, std::vector<int32_t> &pcol)
{
    std::vector<int32_t> mark((size_t)n, -1), frontier, next;
    prp.assign((size_t)n + 1, 0);
    pcol.clear();
    for (int64_t i = 0; i < n; ++i) {
        const size_t start = pcol.size();
        mark[(size_t)i] = (int32_t)i;
        pcol.push_back((int32_t)i);
        frontier.assign(1, (int32_t)i);
        for (int32_t level = 0; level < d && !frontier.empty(); ++level) {
            next.clear();
            for (int32_t u : frontier)
                for (int32_t p = rp[(size_t)u]; p < rp[(size_t)u + 1]; ++p) {
                    const int32_t v = col[(size_t)p];
                    if (mark[(size_t)v] != (int32_t)i) {
                        mark[(size_t)v] = (int32_t)i;
                        pcol.push_back(v);
                        next.push_back(v);
                    }
                }
            frontier.swap(next);
        }
        std::sort(pcol.begin() + (std::ptrdiff_t)start, pcol.end());
        if ((int64_t)pcol.size() > limit) return false;
        prp[(size_t)i + 1] = (int32_t)pcol.size();
    }
    return true;
}

}  // namespace

int amgd_set_search_depth(amgd_handle h, int32_t d)
{
    AMGD_RANGE("amgd_set_search_depth");
    if (!h) return AMGD_ERR_ARG;
    if (h->async_pending) return fail(h, AMGD_ERR_STATE, "asynchronous work pending: call amgd_sync first");
    if (d < 1 || d > 16) return fail(h, AMGD_ERR_ARG, "search depth must be in 1..16");
    if (d == h->depth) return AMGD_OK;
    std::vector<int32_t> prp, pcol;
    if (d > 1 && !depth_pattern(h->h_rp, h->h_col, h->n, d, ((int64_t)1 << 31) - 64, prp, pcol))
        return fail(h, AMGD_ERR_UNSUPPORTED, "the graph of A^d has 2^31 entries or more");
    CK(h, cudaStreamSynchronize(h->stream));
    drop_graph(h);
    if (h->depth > 1) {
        dfree(h->prp);
        dfree(h->pcol);
    }
    h->prp = h->rp_o;
    h->pcol = h->col_o;
    h->nnz_p = h->nnz;
    h->depth = 1;
    if (d > 1) {
        const int64_t nnz_p = (int64_t)pcol.size();
        int32_t *dp = nullptr, *dc = nullptr;
        CK(h, dalloc(&dp, (size_t)h->n + 1 + 4));
        cudaError_t e = dalloc(&dc, (size_t)nnz_p + 16);
        if (e != cudaSuccess) { dfree(dp); return cuda_fail(h, e, "cudaMalloc(pattern)"); }
        CK(h, cudaMemcpy(dp, prp.data(), (h->n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
        CK(h, cudaMemcpy(dc, pcol.data(), nnz_p * sizeof(int32_t), cudaMemcpyHostToDevice));
        h->prp = dp;
        h->pcol = dc;
        h->nnz_p = nnz_p;
        h->depth = d;
    }
    h->E_p = h->nnz_p - h->n;
    int rc = build_edge_tiles(h, d > 1 ? prp : h->h_rp);
    if (rc != AMGD_OK) return rc;
    if ((rc = alloc_slot_outputs(h, h->storage)) != AMGD_OK) return rc;
    dfree(h->flag);
    h->flag = nullptr;
    CK(h, dalloc(&h->flag, (size_t)h->nnz_p + 16));
    dfree(h->s_col_tmp);
    h->s_col_tmp = nullptr;
    h->have_dist = false;
    h->traj_valid = false;
    return AMGD_OK;
}

int amgd_distance_pattern(amgd_handle h, int64_t *row_ptr, int32_t *col, int64_t cap,
                          int64_t *nnz_p, int mem)
{
    if (!h) return AMGD_ERR_ARG;
    if (mem != AMGD_MEM_HOST && mem != AMGD_MEM_DEVICE) return fail(h, AMGD_ERR_ARG, "bad mem");
    if (nnz_p) *nnz_p = h->nnz_p;
    if (col && cap < h->nnz_p) return fail(h, AMGD_ERR_CAPACITY, "col needs the pattern's entry count");
    const cudaMemcpyKind k = mem == AMGD_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (row_ptr) {
        std::vector<int32_t> r32((size_t)h->n + 1);
        CK(h, cudaMemcpy(r32.data(), h->prp, (h->n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost));
        std::vector<int64_t> r64(r32.begin(), r32.end());
        CK(h, cudaMemcpy(row_ptr, r64.data(), (h->n + 1) * sizeof(int64_t),
                         mem == AMGD_MEM_HOST ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice));
    }
    if (col && h->nnz_p) CK(h, cudaMemcpy(col, h->pcol, h->nnz_p * sizeof(int32_t), k));
    return AMGD_OK;
}

int amgd_ls_interpolation(amgd_handle h, const uint8_t *coarse, int coarse_mem, int32_t caliber,
                          double gamma, int64_t *p_row_ptr, int32_t *p_col, double *p_val,
                          int64_t cap, int64_t *nnz_p, double *ls, int mem)
{
    AMGD_RANGE("amgd_ls_interpolation");
    if (!h) return AMGD_ERR_ARG;
    if (caliber < 1 || caliber > kInterpMaxCaliber) return fail(h, AMGD_ERR_ARG, "caliber must be in 1..4");
    if (!(gamma >= 0.0) || !std::isfinite(gamma)) return fail(h, AMGD_ERR_ARG, "gamma must be finite and >= 0");
    if (h->K > 64) return fail(h, AMGD_ERR_UNSUPPORTED, "interpolation needs K <= 64");
    if ((!coarse && h->n) || !p_row_ptr) return fail(h, AMGD_ERR_ARG, "NULL coarse mask or row_ptr");
    if ((coarse_mem != AMGD_MEM_HOST && coarse_mem != AMGD_MEM_DEVICE) ||
        (mem != AMGD_MEM_HOST && mem != AMGD_MEM_DEVICE))
        return fail(h, AMGD_ERR_ARG, "bad mem");
    cudaStream_t s = h->stream;
    const int64_t n = h->n;
    // working buffers (kept by the handle)
    if (!h->ip_coarse) {
        CK(h, dalloc(&h->ip_coarse, (size_t)n + 16));
        CK(h, dalloc(&h->ip_sel_col, (size_t)n * kInterpMaxCaliber + 1));
        CK(h, dalloc(&h->ip_sel_val, (size_t)n * kInterpMaxCaliber + 1));
        CK(h, dalloc(&h->ip_cnt, (size_t)n + 8));
        CK(h, dalloc(&h->ip_ls, (size_t)n + 1));
        CK(h, dalloc(&h->ip_rp, (size_t)n + 1));
        CK(h, dalloc(&h->ip_pos, (size_t)n));
        CK(h, dalloc(&h->ip_list, (size_t)n));
        CK(h, dalloc(&h->ip_bkt, (size_t)n));
        CK(h, dalloc(&h->ip_bcnt, (size_t)kInterpBuckets));
    }
    CK(h, cudaMemcpyAsync(h->ip_coarse, coarse, (size_t)n,
                          coarse_mem == AMGD_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    CK(h, cudaMemsetAsync(h->ip_cnt, 0, ((size_t)n + 8) * sizeof(int32_t), s));
    const void *xc = h->x[h->cur];
    if (h->perm) {
        if (!h->x_caller) return fail(h, AMGD_ERR_STATE, "caller-order vector buffer missing");
        CK(h, launch_unpermute(h->storage, h->x[h->cur], h->x_caller, h->perm, (int32_t)n,
                               Kp_of(h->storage, h->K), s));
        xc = h->x_caller;
    }
    InterpArgs a;
    a.rp = h->rp_o;
    a.col = h->col_o;
    a.val64 = h->val_o;
    a.prp = h->prp;
    a.pcol = h->pcol;
    a.coarse = h->ip_coarse;
    a.x = xc;
    a.w64 = h->w64;
    a.sel_col = h->ip_sel_col;
    a.sel_val = h->ip_sel_val;
    a.cnt = h->ip_cnt;
    a.ls = h->ip_ls;
    a.err = h->err_word;
    a.n = (int32_t)n;
    a.K = h->K;
    a.Kp = Kp_of(h->storage, h->K);
    a.target = h->target;
    a.caliber = caliber;
    a.gamma = gamma;
    a.pos = h->ip_pos;
    a.bkt = h->ip_bkt;
    a.list = h->ip_list;
    a.bcnt = h->ip_bcnt;
    a.unit_w = true;
    for (double wk : h->h_w) a.unit_w = a.unit_w && wk == 1.0;
    CK(h, cudaMemsetAsync(h->err_word, 0, sizeof(uint32_t), s));
    CK(h, launch_ls_interp(h->storage, a, s));
    CK(h, launch_row_ptr(h->ip_cnt, (int32_t)n, h->tile, h->ip_rp, s));
    uint32_t err = 0;
    int64_t total = 0;
    CK(h, cudaMemcpyAsync(&err, h->err_word, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    CK(h, cudaMemcpyAsync(&total, h->ip_rp + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CK(h, cudaStreamSynchronize(s));
    if (err & 1u)
        return fail(h, AMGD_ERR_UNSUPPORTED, "a fine row has more than 32 coarse candidates");
    if (nnz_p) *nnz_p = total;
    if ((p_col || p_val) && cap < total)
        return fail(h, AMGD_ERR_CAPACITY, "P needs " + std::to_string(total) + " entries");
    const cudaMemcpyKind k = mem == AMGD_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    CK(h, cudaMemcpyAsync(p_row_ptr, h->ip_rp, (n + 1) * sizeof(int64_t), k, s));
    if (ls) CK(h, cudaMemcpyAsync(ls, h->ip_ls, n * sizeof(double), k, s));
    if (p_col && p_val && total > 0) {
        int32_t *dc = p_col;
        double *dv = p_val;
        if (mem == AMGD_MEM_HOST) {
            CK(h, ensure_buf(&h->ip_out, h->ip_out_bytes, (size_t)total * (sizeof(int32_t) + sizeof(double))));
            dv = (double *)h->ip_out;
            dc = (int32_t *)(dv + total);
        }
        CK(h, launch_interp_fill(h->ip_rp, h->ip_sel_col, h->ip_sel_val, (int32_t)n, dc, dv, s));
        if (mem == AMGD_MEM_HOST) {
            CK(h, cudaMemcpyAsync(p_col, dc, total * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            CK(h, cudaMemcpyAsync(p_val, dv, total * sizeof(double), cudaMemcpyDeviceToHost, s));
        }
    }
    CK(h, cudaStreamSynchronize(s));
    return poll_status(h);
}

int amgd_cr_coarsen(amgd_handle h, uint8_t *coarse, int coarse_mem, const double *ls, int ls_mem,
                    int sweep, double omega, int32_t nu, double theta, double delta, double tol,
                    int32_t max_sets, uint64_t seed, double *rho, int32_t *n_rho)
{
    AMGD_RANGE("amgd_cr_coarsen");
    if (!h) return AMGD_ERR_ARG;
    if (n_rho) *n_rho = 0;
    if (h->nmat != 1) return fail(h, AMGD_ERR_UNSUPPORTED, "coarsening needs a single-matrix handle");
    if (nu < 1 || max_sets < 0) return fail(h, AMGD_ERR_ARG, "nu must be >= 1 and max_sets >= 0");
    if (!std::isfinite(omega) || omega == 0.0 || !(theta >= 0.0) || !std::isfinite(theta) ||
        !std::isfinite(delta) || !std::isfinite(tol))
        return fail(h, AMGD_ERR_ARG, "omega, theta, delta and tol must be finite (omega != 0, theta >= 0)");
    if (sweep != AMGD_SWEEP_JACOBI && sweep != AMGD_SWEEP_MCGS) return fail(h, AMGD_ERR_ARG, "unknown sweep type");
    if (sweep == AMGD_SWEEP_MCGS && !h->perm)
        return fail(h, AMGD_ERR_STATE, "MCGS needs amgd_set_coloring first");
    if (!coarse && h->n) return fail(h, AMGD_ERR_ARG, "NULL coarse mask");
    if ((coarse_mem != AMGD_MEM_HOST && coarse_mem != AMGD_MEM_DEVICE) ||
        (ls && ls_mem != AMGD_MEM_HOST && ls_mem != AMGD_MEM_DEVICE))
        return fail(h, AMGD_ERR_ARG, "bad mem");
    if (!ls && !h->have_dist) return fail(h, AMGD_ERR_STATE, "no LS given and amgd_distances has not run");
    cudaStream_t s = h->stream;
    const int64_t n = h->n;
    if (!h->cr_u[0]) {
        CK(h, dalloc(&h->cr_u[0], (size_t)n));
        CK(h, dalloc(&h->cr_u[1], (size_t)n));
        CK(h, dalloc(&h->cr_coarse, (size_t)n));
        CK(h, dalloc(&h->cr_state, (size_t)n));
        CK(h, dalloc(&h->cr_ismax, (size_t)n));
        CK(h, dalloc(&h->cr_lam, (size_t)n));
        CK(h, dalloc(&h->cr_key, (size_t)n));
        CK(h, dalloc(&h->cr_scal, 4));
    }
    if (h->cr_strong_len < (size_t)h->nnz_p || !h->cr_strong) {
        dfree(h->cr_strong);
        h->cr_strong = nullptr;
        h->cr_strong_len = 0;
        CK(h, dalloc(&h->cr_strong, (size_t)h->nnz_p));
        h->cr_strong_len = (size_t)h->nnz_p;
    }
    // LS per pattern slot, FP64, on the device
    const double *d_ls = ls;
    if (!ls || ls_mem == AMGD_MEM_HOST) {
        CK(h, ensure_tmp64(h, (size_t)h->nnz_p));
        if (ls)
            CK(h, cudaMemcpyAsync(h->tmp64, ls, h->nnz_p * sizeof(double), cudaMemcpyHostToDevice, s));
        else
            CK(h, launch_export_slots(h->storage, h->a, h->ls, nullptr, nullptr, h->tmp64, h->nnz_p, s));
        d_ls = h->tmp64;
    }
    CK(h, cudaMemcpyAsync(h->cr_coarse, coarse, (size_t)n,
                          coarse_mem == AMGD_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    if (!h->cr_coarse_p) CK(h, dalloc(&h->cr_coarse_p, (size_t)n));
    if (!h->cr_cdiag) CK(h, dalloc(&h->cr_cdiag, (size_t)n));
    {
        const int rc = refresh_perm64(h, s);
        if (rc != AMGD_OK) return rc;
    }
    CrArgs a;
    a.rp = h->rp_p;
    a.col = h->col_p;
    a.val = h->val64;
    a.diag = h->diag64;
    a.cdiag = h->cr_cdiag;
    a.perm = h->perm;
    a.coarse_p = h->cr_coarse_p;
    a.prp = h->prp;
    a.pcol = h->pcol;
    a.ls = d_ls;
    a.coarse = h->cr_coarse;
    a.state = h->cr_state;
    a.ismax = h->cr_ismax;
    a.strong = h->cr_strong;
    a.lam = h->cr_lam;
    a.key = h->cr_key;
    a.scal = h->cr_scal;
    a.n = (int32_t)n;
    a.omega = omega;
    a.theta = theta;
    int32_t stage = 0;
    unsigned long long scal[3] = {0, 0, 0};
    const int32_t ncolors = (int32_t)h->color_start.size() - 1;
    const int64_t sweep_launches = sweep == AMGD_SWEEP_MCGS ? ncolors : 1;
    h->cr_rounds = 0;
    h->cr_launches = ls ? 0 : 1;                  // the LS export
    CK(h, launch_cr_cdiag(a, s));
    ++h->cr_launches;
    for (;;) {
        // nu F-relaxation sweeps from the constant start (Eq. (3.4))
        CK(h, launch_cr_start(a, h->cr_u[0], s));
        int cu = 0;
        for (int32_t it = 0; it < nu; ++it) {
            CK(h, launch_cr_sweep(a, sweep == AMGD_SWEEP_MCGS, h->color_start.data(), ncolors,
                                  h->cr_u[cu], h->cr_u[cu ^ 1], s));
            cu ^= 1;
        }
        // the convergence estimate of Eq. (3.5) in the max norm (||u^0|| = 1)
        CK(h, launch_cr_norm(h->cr_u[cu], h->cr_coarse_p, (int32_t)n, h->cr_scal, s));
        CK(h, cudaMemcpyAsync(scal, h->cr_scal, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        CK(h, cudaStreamSynchronize(s));
        double unorm;
        std::memcpy(&unorm, &scal[0], sizeof unorm);
        h->cr_launches += 2 + nu * sweep_launches;
        const double r = scal[1] == 0 ? 0.0 : std::pow(unorm, 1.0 / (double)nu);
        if (rho) rho[stage] = r;
        if (!(r > delta) || stage >= max_sets) { ++stage; break; }
        // candidates, strength graph on F, priorities
        CK(h, launch_cr_candidates(a, h->cr_u[cu], tol, s));
        CK(h, launch_cr_keys((int32_t)n, stage, seed, h->cr_key, s));
        // independent set: rounds of local maxima until no candidate is undecided;
        // every round selects at least the first undecided point of the order
        int64_t rounds = 0;
        for (;;) {
            const int32_t batch = rounds < 8 ? 4 : 8;
            CK(h, launch_cr_mis_rounds(a, batch, s));
            rounds += batch;
            h->cr_launches += 3 * (int64_t)batch + 1;
            CK(h, cudaMemcpyAsync(&scal[2], h->cr_scal + 2, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
            CK(h, cudaStreamSynchronize(s));
            if (scal[2] == 0) break;
            if (rounds > n + 8) return fail(h, AMGD_ERR_CUDA, "independent-set rounds did not finish");
        }
        CK(h, launch_cr_add(a, s));
        h->cr_launches += 4;                      // candidates, strength, keys, add
        h->cr_rounds += (int32_t)rounds;
        ++stage;
    }
    CK(h, cudaMemcpyAsync(coarse, h->cr_coarse, (size_t)n,
                          coarse_mem == AMGD_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    CK(h, cudaStreamSynchronize(s));
    if (n_rho) *n_rho = stage;
    return poll_status(h);
}

int amgd_cr_stats(amgd_handle h, int32_t *rounds, int64_t *launches)
{
    if (!h) return AMGD_ERR_ARG;
    if (rounds) *rounds = h->cr_rounds;
    if (launches) *launches = h->cr_launches;
    return AMGD_OK;
}

int amgd_set_checkpointing(amgd_handle h, int32_t every)
{
    if (!h) return AMGD_ERR_ARG;
    if (every < 0) return fail(h, AMGD_ERR_ARG, "checkpoint interval < 0");
    h->ckpt_every = every;
    if (every == 0) h->traj_valid = false;
    return AMGD_OK;
}

namespace {

// transposed pattern of A (host counting sort, entries of a column in
// ascending row order), built once per handle
int ensure_transpose(amgd_ctx *h)
{
    if (h->at_rp) return AMGD_OK;
    const int64_t n = h->n, nnz = h->nnz;
    std::vector<int32_t> trp((size_t)n + 1, 0), trow((size_t)nnz), tslot((size_t)nnz);
    for (int64_t p = 0; p < nnz; ++p) ++trp[(size_t)h->h_col[(size_t)p] + 1];
    for (int64_t j = 0; j < n; ++j) trp[(size_t)j + 1] += trp[(size_t)j];
    std::vector<int32_t> next(trp.begin(), trp.end() - 1);
    for (int64_t i = 0; i < n; ++i)
        for (int32_t p = h->h_rp[(size_t)i]; p < h->h_rp[(size_t)i + 1]; ++p) {
            const int32_t q = next[(size_t)h->h_col[(size_t)p]]++;
            trow[(size_t)q] = (int32_t)i;
            tslot[(size_t)q] = p;
        }
    CK(h, dalloc(&h->at_rp, (size_t)n + 1));
    CK(h, dalloc(&h->at_row, (size_t)(nnz ? nnz : 1)));
    CK(h, dalloc(&h->at_slot, (size_t)(nnz ? nnz : 1)));
    CK(h, cudaMemcpy(h->at_rp, trp.data(), (n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
    if (nnz) {
        CK(h, cudaMemcpy(h->at_row, trow.data(), nnz * sizeof(int32_t), cudaMemcpyHostToDevice));
        CK(h, cudaMemcpy(h->at_slot, tslot.data(), nnz * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    // structurally symmetric pattern with ascending columns: row j's columns
    // are column j's rows in the same order, and slot p = (j, i) has the
    // mirror slot (i, j); the reverse sweeps then need one kernel per sweep
    bool sym = true;
    for (int64_t j = 0; j < n && sym; ++j) {
        const int32_t p0 = h->h_rp[(size_t)j], p1 = h->h_rp[(size_t)j + 1];
        if (p1 - p0 != trp[(size_t)j + 1] - trp[(size_t)j]) { sym = false; break; }
        for (int32_t k = 0; k < p1 - p0; ++k)
            if (h->h_col[(size_t)(p0 + k)] != trow[(size_t)(trp[(size_t)j] + k)]) { sym = false; break; }
    }
    if (sym && nnz) {
        std::vector<int32_t> mirror((size_t)nnz);
        for (int64_t j = 0; j < n; ++j)
            for (int32_t k = 0; k < h->h_rp[(size_t)j + 1] - h->h_rp[(size_t)j]; ++k)
                mirror[(size_t)(h->h_rp[(size_t)j] + k)] = tslot[(size_t)(trp[(size_t)j] + k)];
        CK(h, dalloc(&h->mirror, (size_t)nnz));
        CK(h, cudaMemcpy(h->mirror, mirror.data(), nnz * sizeof(int32_t), cudaMemcpyHostToDevice));
    }
    return AMGD_OK;
}

}  // namespace

namespace {

// device buffers of the reverse pass (allocated before any capture)
int prepare_backward(amgd_ctx *h)
{
    const size_t cs = 8;                 // the reverse pass computes in FP64
    const size_t nk = (size_t)h->n * Kp_of(h->storage, h->K);
    const size_t xb = nk * esize(h->storage);
    const int32_t S = h->ckpt_every > 0 ? h->ckpt_every : 1;
    int rc = ensure_transpose(h);
    if (rc != AMGD_OK) return rc;
    CK(h, ensure_buf(&h->adj_vec, h->adj_vec_bytes, 4 * nk * cs));
    CK(h, ensure_buf(&h->adj_slot, h->adj_slot_bytes, 6 * (size_t)(h->nnz ? h->nnz : 1) * cs));
    CK(h, ensure_buf(&h->seg, h->seg_bytes, (size_t)(S - 1) * xb));
    if (!h->lsb) CK(h, dalloc(&h->lsb, (size_t)(h->nnz ? h->nnz : 1)));
    if (!h->adj_part) CK(h, dalloc(&h->adj_part, (size_t)2 * kAdjReduceBlocks + 2));
    CK(h, ensure_tmp64(h, (size_t)h->nnz));
    return AMGD_OK;
}

// Enqueue the whole reverse pass on stream s (nothing synchronises).
// lsb_in: device dL/dLS or NULL (built-in loss); vb: device dL/dval.
// The two sums (loss, dL/domega) land in adj_part[2 nb], adj_part[2 nb + 1].
int run_backward(amgd_ctx *h, const double *lsb_in, double *vb, cudaStream_t s)
{
    const int st = h->storage;
    const int32_t n = (int32_t)h->n;
    const int64_t nnz = h->nnz;
    const int Kp = Kp_of(st, h->K);
    const size_t cs = 8;                 // FP64 reverse pass
    const size_t nk = (size_t)n * Kp;
    const size_t xb = nk * esize(st);
    const int32_t S = h->ckpt_every > 0 ? h->ckpt_every : 1;
    const int32_t nu = h->traj_nu;
    const int nb = kAdjReduceBlocks;
    char *vecs = (char *)h->adj_vec;
    void *Y = vecs, *Ybar = vecs + nk * cs;
    void *Xbar[2] = {vecs + 2 * nk * cs, vecs + 3 * nk * cs};
    char *slots = (char *)h->adj_slot;
    void *gs = slots, *gt = slots + nnz * cs, *at_b = slots + 2 * nnz * cs;
    void *bm = slots + 3 * nnz * cs;
    double *a64 = (double *)(slots + 4 * nnz * cs), *ls64 = (double *)(slots + 5 * nnz * cs);

    AdjArgs a;
    a.rp = h->rp_o;
    a.col = h->col_o;
    a.val = h->val_o;                    // FP64 values, diagonal and weights
    a.diag = h->diag64_o;
    a.at_rp = h->at_rp;
    a.at_row = h->at_row;
    a.at_slot = h->at_slot;
    a.at_b = at_b;
    a.bm = h->mirror ? bm : nullptr;
    a.x = h->x[h->cur];
    a.w = h->w64;
    a.a = a64;
    a.a_fit = a64;
    a.ls64 = ls64;
    a.lsb = h->lsb;
    a.n = n;
    a.Kp = Kp;
    a.target = h->target;
    a.unit_w = true;
    for (double wk : h->h_w) a.unit_w = a.unit_w && wk == 1.0;
    a.y = Y;                             // the refit leaves the FP64 target here for the adjoint
    // the fits of X_nu in FP64 (the forward pass's own a and LS may be FP32)
    CK(h, launch_adj_refit(st, a, s));
    CK(h, launch_adj_upstream(st, h->rp_o, h->col_o, ls64, h->flag, lsb_in, h->lsb, h->adj_part,
                              nb, n, h->target, s));
    CK(h, launch_adj_bvals(st, h->val_o, h->diag64_o, h->at_row, h->at_slot, at_b, nnz, s));
    if (h->mirror)   // per slot (j, i): a_ij / a_ii, the mirror entry over its row's diagonal
        CK(h, launch_adj_bvals(st, h->val_o, h->diag64_o, h->col_o, h->mirror, bm, nnz, s));

    a.y = Y;
    a.ybar = Ybar;
    a.xbar_in = nullptr;
    a.xbar_out = Xbar[0];
    a.gs = gs;
    a.gt = gt;
    a.n = n;
    a.Kp = Kp;
    a.target = h->target;
    a.first = 1;
    a.omega = h->traj_omega;
    CK(h, launch_adj_edge(st, a, s));
    CK(h, launch_adj_xbar_nu(st, a, s));

    // sweeps, last to first, one checkpoint segment at a time: the iterates
    // between two checkpoints are recomputed by the forward kernel
    int xc = 0;
    const int32_t nseg = (nu + S - 1) / S;
    for (int32_t c = nseg - 1; c >= 0; --c) {
        const int32_t k0 = c * S, k1 = std::min(k0 + S, nu);
        void *base = (char *)h->ckpt + (size_t)c * xb;
        auto iterate = [&](int32_t k) -> void * {
            return k == k0 ? base : (char *)h->seg + (size_t)(k - k0 - 1) * xb;
        };
        for (int32_t k = k0; k + 1 < k1; ++k) {
            const int rc = jacobi_step(h, iterate(k), iterate(k + 1), h->traj_omega, s);
            if (rc != AMGD_OK) return rc;
        }
        for (int32_t k = k1 - 1; k >= k0; --k) {
            a.x = iterate(k);
            a.xbar_in = Xbar[xc];
            a.xbar_out = Xbar[1 - xc];
            a.first = k == nu - 1;
            if (a.bm) {
                CK(h, launch_adj_sweep_sym(st, a, s));
            } else {
                CK(h, launch_adj_gram(st, a, s));
                CK(h, launch_adj_spmm_t(st, a, s));
            }
            xc = 1 - xc;
        }
    }
    CK(h, launch_adj_finish(st, a, nu > 0, h->val_o, h->diag64_o, h->diag_slot, vb,
                            h->adj_part + nb, nb, s));
    CK(h, launch_adj_reduce(h->adj_part, nb, 2, h->adj_part + 2 * nb, s));
    return AMGD_OK;
}

int backward_checks(amgd_ctx *h)
{
    if (h->depth != 1)
        return fail(h, AMGD_ERR_UNSUPPORTED, "the reverse pass covers search depth 1");
    if (h->perm)
        return fail(h, AMGD_ERR_UNSUPPORTED, "the reverse pass covers Jacobi sweeps without a coloring");
    if (!h->traj_valid)
        return fail(h, AMGD_ERR_STATE, "no recorded trajectory: amgd_set_checkpointing, then a Jacobi amgd_relax");
    if (!h->have_dist) return fail(h, AMGD_ERR_STATE, "amgd_distances must run after amgd_relax");
    return AMGD_OK;
}

}  // namespace

int amgd_backward(amgd_handle h, const double *ls_bar, int mem, double *val_bar,
                  double *omega_bar, double *loss)
{
    AMGD_RANGE("amgd_backward");
    if (!h) return AMGD_ERR_ARG;
    if (mem != AMGD_MEM_HOST && mem != AMGD_MEM_DEVICE) return fail(h, AMGD_ERR_ARG, "bad mem");
    if (!val_bar && h->nnz) return fail(h, AMGD_ERR_ARG, "val_bar is NULL");
    int rc = backward_checks(h);
    if (rc != AMGD_OK) return rc;
    if ((rc = prepare_backward(h)) != AMGD_OK) return rc;
    cudaStream_t s = h->stream;
    const int64_t nnz = h->nnz;
    const double *lsb_in = ls_bar;
    double *vb = val_bar;
    if (mem == AMGD_MEM_HOST) {
        // one staging buffer serves both: dL/dLS is consumed by the first
        // kernel, dL/dval written by the last
        if (ls_bar)
            CK(h, cudaMemcpyAsync(h->tmp64, ls_bar, nnz * sizeof(double), cudaMemcpyHostToDevice, s));
        lsb_in = ls_bar ? h->tmp64 : nullptr;
        vb = h->tmp64;
    }
    if ((rc = run_backward(h, lsb_in, vb, s)) != AMGD_OK) return rc;
    if (mem == AMGD_MEM_HOST && nnz)
        CK(h, cudaMemcpyAsync(val_bar, vb, nnz * sizeof(double), cudaMemcpyDeviceToHost, s));
    h->last_backward_builtin = ls_bar == nullptr;
    if (omega_bar || loss || mem == AMGD_MEM_HOST) return amgd_backward_scalars(h, omega_bar, loss);
    return AMGD_OK;
}

int amgd_backward_scalars(amgd_handle h, double *omega_bar, double *loss)
{
    if (!h) return AMGD_ERR_ARG;
    if (!h->adj_part) return fail(h, AMGD_ERR_STATE, "no reverse pass has run");
    double sums[2] = {0.0, 0.0};
    CK(h, cudaMemcpyAsync(sums, h->adj_part + 2 * kAdjReduceBlocks, 2 * sizeof(double),
                          cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    if (loss) *loss = h->last_backward_builtin ? sums[0] : NAN;
    if (omega_bar) *omega_bar = sums[1];
    return poll_status(h);
}

int amgd_graph_capture_backward(amgd_handle h, uint64_t seed, int32_t nu, double omega,
                                double theta, double *val_bar)
{
    AMGD_RANGE("amgd_graph_capture_backward");
    if (!h) return AMGD_ERR_ARG;
    if (h->async_pending) return fail(h, AMGD_ERR_STATE, "asynchronous work pending: call amgd_sync first");
    if (nu < 0 || !std::isfinite(omega)) return fail(h, AMGD_ERR_ARG, "nu < 0 or omega not finite");
    if (!(theta >= 0.0) || !std::isfinite(theta)) return fail(h, AMGD_ERR_ARG, "theta must be finite and >= 0");
    if (!val_bar && h->nnz) return fail(h, AMGD_ERR_ARG, "val_bar is NULL");
    if (h->perm || h->depth != 1)
        return fail(h, AMGD_ERR_UNSUPPORTED,
                    "the reverse pass covers Jacobi sweeps without a coloring at search depth 1");
    if (h->ckpt_every <= 0) return fail(h, AMGD_ERR_STATE, "amgd_set_checkpointing must come first");
    // every buffer the captured work touches exists before the capture
    {
        const size_t xb = (size_t)h->n * Kp_of(h->storage, h->K) * esize(h->storage);
        const int32_t nck = (nu + h->ckpt_every - 1) / h->ckpt_every;
        CK(h, ensure_buf(&h->ckpt, h->ckpt_bytes, (size_t)nck * xb));
        const int rc = prepare_backward(h);
        if (rc != AMGD_OK) return rc;
    }
    if (!h->cap_stream) CK(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
    if (h->graph) { cudaGraphDestroy(h->graph); h->graph = nullptr; }
    CK(h, cudaStreamSynchronize(h->stream));
    const int cur0 = h->cur;
    h->cur = 0;
    if (h->phase_timing && !h->ev[0])
        for (auto &e : h->ev) CK(h, cudaEventCreate(&e));
    const bool timed = h->phase_timing;
    auto mark = [&](int k) {
        return timed ? cudaEventRecordWithFlags(h->ev[k], h->cap_stream, cudaEventRecordExternal)
                     : cudaSuccess;
    };
    CK(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal));
    int rc = AMGD_OK;
    cudaError_t me = mark(0);
    if (me == cudaSuccess) rc = run_init(h, seed, h->cap_stream);
    if (me == cudaSuccess && rc == AMGD_OK) me = mark(1);
    if (me == cudaSuccess && rc == AMGD_OK) rc = run_relax_recorded(h, nu, omega, h->cap_stream);
    if (me == cudaSuccess && rc == AMGD_OK) me = mark(2);
    if (me == cudaSuccess && rc == AMGD_OK) rc = run_edge(h, theta, h->cap_stream);
    if (me == cudaSuccess && rc == AMGD_OK) me = mark(3);
    if (me == cudaSuccess && rc == AMGD_OK) rc = run_backward(h, nullptr, val_bar, h->cap_stream);
    if (me == cudaSuccess && rc == AMGD_OK) me = mark(4);
    if (me != cudaSuccess && rc == AMGD_OK) rc = cuda_fail(h, me, "cudaEventRecordWithFlags (capture)");
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
    h->graph_cur_after = h->cur;
    h->cur = cur0;
    h->have_dist = false;
    h->traj_valid = false;
    if (rc != AMGD_OK) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    h->graph = g;
    CK(h, cudaGraphInstantiate(&h->gexec, h->graph, 0));
    h->graph_timed = timed;
    h->graph_is_backward = true;
    h->graph_traj_nu = nu;
    h->graph_traj_omega = omega;
    h->last_backward_builtin = true;
    return AMGD_OK;
}

int amgd_destroy(amgd_handle h)
{
    if (!h) return AMGD_OK;
    if (h->stream || h->x[0]) cudaStreamSynchronize(h->stream);
    if (h->up_stream) {
        cudaStreamSynchronize(h->up_stream);
        cudaStreamSynchronize(h->down_stream);
        cudaStreamDestroy(h->up_stream);
        cudaStreamDestroy(h->down_stream);
        for (int k = 0; k < 2; ++k) {
            cudaEventDestroy(h->ev_up[k]);
            cudaEventDestroy(h->ev_used[k]);
            cudaEventDestroy(h->ev_res[k]);
            cudaEventDestroy(h->ev_down[k]);
        }
    }
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->graph) cudaGraphDestroy(h->graph);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    for (auto e : h->ev)
        if (e) cudaEventDestroy(e);
    if (h->perm) {
        dfree(h->perm);
        dfree(h->rp_p);
        dfree(h->col_p);
        dfree(h->val64);
        dfree(h->slot_perm);
        dfree(h->pinv);
        dfree(h->colx);
    }
    dfree(h->mat_id);
    if (h->depth > 1) {
        dfree(h->prp);
        dfree(h->pcol);
    }
    void *ptrs[] = {h->rp_o, h->col_o, h->val_o, h->mat_off, h->diag_slot, h->err_word, h->status,
                    h->diag64, h->diag32, h->val32_o, h->diag64_o, h->diag32_o, h->x_caller,
                    h->defer_count, h->defer_list,
                    h->val32, h->x[0], h->x[1],
                    h->w64, h->w32, h->a, h->ls, h->flag, h->count, h->tile, h->s_rp_tmp,
                    h->s_col_tmp, h->tmp64, h->ckpt, h->seg, h->adj_vec, h->adj_slot, h->lsb,
                    h->adj_part, h->at_rp, h->at_row, h->at_slot, h->edge_tiles, h->mirror,
                    h->ip_coarse, h->ip_sel_col, h->ip_cnt, h->ip_sel_val, h->ip_ls, h->ip_rp,
                    h->ip_out, h->ip_pos, h->ip_list, h->ip_bcnt, h->ip_bkt, h->cr_u[0], h->cr_u[1], h->cr_coarse, h->cr_coarse_p, h->cr_cdiag, h->stage[0], h->stage[1], h->res_rp[0],
                    h->res_rp[1], h->res_col[0], h->res_col[1], h->async_err, h->cr_state,
                    h->cr_ismax, h->cr_strong, h->cr_lam, h->cr_key, h->cr_scal};
    for (void *p : ptrs) dfree(p);
    delete h;
    return AMGD_OK;
}

int amgd_checked_build(void)
{
    return AMGD_CHECKS ? 1 : 0;
}

const char *amgd_status_string(int status)
{
    switch (status) {
    case AMGD_OK: return "AMGD_OK";
    case AMGD_ERR_ARG: return "AMGD_ERR_ARG: bad argument";
    case AMGD_ERR_CSR: return "AMGD_ERR_CSR: malformed CSR matrix";
    case AMGD_ERR_ZERO_DIAG: return "AMGD_ERR_ZERO_DIAG: missing or zero diagonal";
    case AMGD_ERR_CUDA: return "AMGD_ERR_CUDA: CUDA runtime error";
    case AMGD_ERR_OOM: return "AMGD_ERR_OOM: device allocation failed";
    case AMGD_ERR_STATE: return "AMGD_ERR_STATE: call out of order";
    case AMGD_ERR_CAPACITY: return "AMGD_ERR_CAPACITY: output buffer too small";
    case AMGD_ERR_TIMEOUT: return "AMGD_ERR_TIMEOUT: bounded device wait gave up";
    case AMGD_ERR_UNSUPPORTED: return "AMGD_ERR_UNSUPPORTED: size or mode not supported";
    case AMGD_ERR_CHECK: return "AMGD_ERR_CHECK: an index failed its bounds test (checked build)";
    }
    return "unknown status";
}

const char *amgd_last_error(amgd_handle h)
{
    return h ? h->err.c_str() : g_create_err.c_str();
}

}  // extern "C"
