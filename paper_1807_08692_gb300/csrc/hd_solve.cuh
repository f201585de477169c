// Shared declarations of the online query path (Eq. 17-20).
#pragma once
#include <cuda_fp16.h>

#include "hd_internal.cuh"

// Per-column CG state, fp64 scalars.
struct ColState {
    double rho;     // r^T z (z = r without preconditioner)
    double sigma;   // p^T A p
    double a;       // step length rho / sigma (0 when inactive)
    double beta;    // rho' / rho (0 when inactive)
    double rr;      // ||r||^2
    double bb;      // ||b||^2
    double tol2;    // tol^2 ||b||^2
    int active;
    int iters;
    int status;
    int confirms;   // residual replacements so far (true residual above tol at a stop)
    int restart;    // 1: r was just replaced by b - A x; the direction restarts from it
    // serving (continuous batching inside the iteration):
    int refill;     // 1: a request was installed at the last scalar step; the direction
                    // that follows drops R (p0 = M^-1 y), the next update starts x, r afresh
    int free_col;   // 1: no request holds the column (it may take a staged one)
    double rr_fix;  // ||y - a q||^2 - ||a q||^2 of a refilled column's first update (exact)
};

// Requests staged for a server lane's next scalar step: a column that stops
// there (or is free) takes the next one (atomic claim), its old request's
// statistics are kept for the host, and the iteration's direction forms the
// new request's p0 = M^-1 y.  Device pointers; all null outside the server.
struct Refill {
    const int32_t* off = nullptr;     // staged request s: entries off[s] .. off[s + 1]
    const int32_t* yidx = nullptr;    // of yidx / yval
    const float* yval = nullptr;
    const double* bb = nullptr;       // ||y_s||^2
    const double* tol2 = nullptr;     // tol_s^2 ||y_s||^2
    const double* C = nullptr;        // [nstage][rpad] U^T y_s (with eigenpairs)
    const int* nstage = nullptr;
    const int32_t* pre = nullptr;     // [Bp] staged request given to a free column by the host (-1: none)
    int* next = nullptr;              // the next staged request for a column that stops (starts after
                                      // the host's assignments)
    int32_t* assign = nullptr;        // [Bp] staged request installed in column j (-1: none)
    int32_t* ret_iters = nullptr;     // [Bp] iterations / status / ||r||^2 of the request
    int32_t* ret_status = nullptr;    //      column j gave up for the new one
    double* ret_rr = nullptr;
    int32_t* col_cnt = nullptr;       // [Bp] the installed request's y, kept per column
    int32_t* col_idx = nullptr;       // [Bp][REFILL_MAX_NNZ]
    float* col_val = nullptr;
    int32_t rpad = 0;
    int32_t live = 0;                 // columns at or above this take no request from `next`
};
constexpr int REFILL_MAX_NNZ = 512;

// Low-rank product helpers (storage-specific implementations).
//  reduce: part[c][k][j] = sum over rows of chunk c of U[i][k] * V[i][j]
//  expand: out = f(U H) for each row (see ExpandOp)
enum ExpandOp {
    EXP_SET_X = 0,      // x_i   = U_i H
    EXP_SUB_R = 1,      // r_i  -= U_i H
    EXP_ADD_Q = 2,      // q_i  += U_i H
    EXP_DIRECTION = 3,  // p_i   = r_i + U_i H + beta p_i
};

struct LowRank {
    const hd_eig* e;
    int32_t rpad;       // r rounded up to 64
    int32_t nchunk;     // row chunks of the reduction partials
    float* part;        // [nchunk][rpad][Bp]
    double* C;          // [rpad][Bp] fp64
    float* H;           // [rpad][Bp] fp32
    __nv_bfloat16* Hhi; // [Bp16][rpad] bf16 (transposed, K-major) high part of H
    __nv_bfloat16* Hlo; // low part
    int32_t Bp16;
    int32_t live = 0;   // > 0: only columns below this can be active (tensor-core paths skip the rest)
};

// `gate` (device int, may be null): the kernels return at once when it is 0
// (no column active), so iterations past convergence cost only their launch.
int lr_reduce(hd_ctx* ctx, const LowRank& lr, const float* V, int64_t n, int32_t Bp, const int* gate = nullptr);
int lr_finish(hd_ctx* ctx, const LowRank& lr, int32_t Bp, const double* coef);
int lr_expand(hd_ctx* ctx, const LowRank& lr, int op, float* out, const float* Rv, const float* Pv, int64_t n,
              int32_t Bp, const ColState* st, const int* gate = nullptr);
bool lr_use_tensor_cores(const hd_eig* e);
// HD_ERR_TIMEOUT (flags cleared) if a tensor-core kernel gave up a bounded wait
// since the last check; synchronises the context's stream
int lr_tc_check_flags(hd_ctx* ctx);
// partial-sum chunks of the reduction for this embedding and batch width
int lr_nchunk(hd_ctx* ctx, const hd_eig* e, int32_t Bp);
int lr_sparse_nchunk(hd_ctx* ctx, const hd_eig* e);
int lr_sparse_reduce(hd_ctx* ctx, const LowRank& lr, const float* V, int64_t n, int32_t Bp, const int* gate);
int lr_sparse_expand(hd_ctx* ctx, const LowRank& lr, int op, float* out, const float* Rv, const float* Pv, int64_t n,
                     int32_t Bp, const ColState* st, const int* gate);
int lr_tc_reduce(hd_ctx* ctx, const LowRank& lr, const float* V, int64_t n, int32_t Bp, const int* gate);
int lr_tc_expand(hd_ctx* ctx, const LowRank& lr, int op, float* out, const float* Rv, const float* Pv, int64_t n,
                 int32_t Bp, const ColState* st, const int* gate);
int lr_tc_nchunk(hd_ctx* ctx, int64_t n);

// ------------------------------------------------------------------ iteration engine
struct VecLaunch {
    int S;       // columns per row-group slab
    int nblk;    // grid.x
    int slabs;   // grid.y
};

// Truncated temporal systems (one per column): row t of column j has the
// entries off[j * smax + t] .. off[j * smax + t + 1] of (ci, wv), ci a row
// index of the same column's system; columns j >= B are empty.
struct TruncSys {
    const int64_t* off = nullptr;
    const int32_t* ci = nullptr;
    const float* wv = nullptr;
    int32_t B = 0;
    int64_t smax = 0;
};

struct Engine {
    hd_ctx* ctx = nullptr;
    const hd_graph* g = nullptr;
    const TruncSys* ts = nullptr;   // per-column operators instead of g (truncated temporal)
    int64_t n = 0;
    int32_t B = 0, Bp = 0;
    VecLaunch vl{};
    int rch = 64;                      // rows per reduction chunk (depends on n only)
    int64_t nch = 0;                   // reduction chunks: column partials are [nch][Bp]
    int segK = 1;                      // SpMM node-range segments (1: one pass)
    const int32_t* seg = nullptr;      // their row bounds [segK + 1][n]
    // a 4-column batch may use k_spmm_n4 (its sums run in another order than
    // k_spmm's; the server keeps one order at every lane width)
    bool narrow4 = true;
    float *R = nullptr, *P = nullptr, *Q = nullptr, *X = nullptr;
    float2* part = nullptr;
    ColState* st = nullptr;
    int* num_active = nullptr;
    int* err = nullptr;
    // the staged observations (device), scattered again for the true residual
    const int32_t* yp = nullptr;
    const int32_t* yi = nullptr;
    const float* yv = nullptr;
    double* Cy = nullptr;       // U^T y [rpad][Bp] (paper and projected forms: x^s and b)
    // fp16 copy of P for the SpMM gathers of late iterations (hd_query_batch
    // only: the decision covers the whole batch, so a column's bits would
    // depend on its neighbours, which the server avoids)
    bool allow_half = false;
    const Refill* refill = nullptr;   // a server lane: requests installed inside the iteration
    __half* P16 = nullptr;      // n x Bp
    unsigned* p16_max = nullptr;  // [Bp] max |P_j| as float bits
    int* use_half = nullptr;    // 1: the next SpMM gathers P16
    double* negop = nullptr;    // -(a / (1 - a)) lambda: the deflation term of -L_a(W_r)
    LowRank lr{};
    bool has_lr = false;
    double *gcoef = nullptr, *hcoef = nullptr, *opcoef = nullptr, *dcoef = nullptr, *ones = nullptr;
    int eff_mode = HD_MODE_PAPER;
    float c1 = 0.f, c2 = 0.f, xs = 1.f;
    int r = 0;
    int32_t max_iter = 0;
};

VecLaunch vec_launch(hd_ctx* ctx, int64_t n, int32_t Bp, int S = 0);
// Column-slab width of the SpMM for this graph and batch width: measured once
// per (graph, Bp) over the widths dividing Bp (HD_SLAB overrides).
int tune_slab(hd_ctx* ctx, const hd_graph* g, int32_t Bp, const float* P, float* Q);
int simt_nchunk(hd_ctx* ctx, int64_t n, int rpad, int Bp);
// Node-range segments for the SpMM with slab width S: measured once per
// (graph, Bp) over K in {1, 2, 4, 8} (HD_SEGMENTS overrides); sets E.segK / E.seg.
int tune_segments(hd_ctx* ctx, Engine& E);
int engine_iteration(Engine& E, int (*after_update)(void*), void* arg);
// r += y for the columns of a server lane that took a request at the last
// scalar step (after their first update), with the exact ||r||^2 correction
int launch_refill_r(Engine& E);
// rows per reduction chunk for n rows, and the engine's chunk count from it
int reduction_chunk_rows(int64_t n);
void engine_set_reduction(Engine& E);
int hd_query_impl(hd_ctx* ctx, const hd_graph* g, const TruncSys* ts, const hd_eig* eig, int mode, int32_t B,
                  const int32_t* y_ptr, const int32_t* y_idx, const float* y_val, double alpha, const float* tol,
                  int32_t max_iter, float* X, int32_t ldx, int32_t* iters, float* relres, int32_t* status);
