// Continuous-batching query server over the multi-RHS CG engine.
//
// A server owns persistent batches ("lanes") of columns (R, P, Q, X of n x Bp):
// the wide lane of `slots` columns and, when there is room, a narrow lane of
// four.  Requests queue on the host.  Before each step the host stages queued
// requests (their observations and U^T y); inside the step's scalar kernel a
// column whose request stops there -- or a free column -- claims the next
// staged request, so the same iteration's direction already forms the new
// request's p0 = M^-1 y and a column never spends an iteration idle between two
// requests.  The stopped request's x stays in the column until the next update,
// which starts the new one from scratch; between the two the host ranks it
// (top-K copied out).  Staged requests that found no column go back to the
// front of the queue.
//
// A lightly loaded server (wide lane idle, queue no longer than the narrow
// lane's free columns) stages into the narrow lane: its rows are 16 bytes
// instead of 4 x slots bytes, so one request moves far fewer bytes per
// iteration.  Otherwise requests go to the wide lane.  A column's arithmetic
// never depends on its lane, slot or the other columns (per-element SpMM order
// is the same for every slab width, reductions are chunked by rows, the
// tensor-core products treat columns independently, every request starts the
// same way), so a request gets the same bits alone or in a mix.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <deque>
#include <unordered_map>
#include <vector>

#include "hd_solve.cuh"

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Req {
    uint64_t ticket = 0;
    std::vector<int32_t> idx;
    std::vector<float> val;
    double bb = 0.0;
    float tol = 0.f;
    int32_t K = 0;
    int32_t slot = -1;      // reported slot (narrow-lane slots follow the wide ones)
    double submit_s = 0, admit_s = 0, done_s = 0;
    int32_t iters = 0, status = 0;
    float relres = 0.f;
    bool done = false;
    std::vector<int32_t> out_idx;
    std::vector<float> out_score;
};

// U^T y of each staged request (fp64, in entry order; zero beyond r): the
// spectral part of its first preconditioned residual z0 = y + U D U^T y.
// One block per request, threads over the eigen-index k.
template <typename T>
__device__ __forceinline__ double u_entry(const T* U, const float* scale, int64_t i, int ldu, int k);
template <>
__device__ __forceinline__ double u_entry<float>(const float* U, const float*, int64_t i, int ldu, int k) {
    return (double)U[i * ldu + k];
}
template <>
__device__ __forceinline__ double u_entry<__nv_bfloat16>(const __nv_bfloat16* U, const float*, int64_t i, int ldu,
                                                         int k) {
    return (double)__bfloat162float(U[i * ldu + k]);
}
template <>
__device__ __forceinline__ double u_entry<__nv_fp8_e4m3>(const __nv_fp8_e4m3* U, const float* scale, int64_t i,
                                                         int ldu, int k) {
    return (double)(float(U[i * ldu + k]) * scale[i]);
}

template <typename T>
__global__ void k_stage_c(const T* U, const float* scale, int ldu, int r, int rpad, const int32_t* off,
                          const int32_t* yidx, const float* yval, double* C) {
    const int s = blockIdx.x;
    for (int k = threadIdx.x; k < rpad; k += blockDim.x) {
        double c = 0.0;
        if (k < r)
            for (int32_t t = off[s]; t < off[s + 1]; ++t) c += (double)yval[t] * u_entry<T>(U, scale, yidx[t], ldu, k);
        C[(int64_t)s * rpad + k] = c;
    }
}

// the same from a sparsified U (rows in CSR): one thread per request
__global__ void k_stage_c_sparse(const int64_t* rp, const int32_t* col, const float* val, int rpad, int nstage,
                                 const int32_t* off, const int32_t* yidx, const float* yval, double* C) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nstage) return;
    double* c = C + (int64_t)s * rpad;
    for (int k = 0; k < rpad; ++k) c[k] = 0.0;
    for (int32_t t = off[s]; t < off[s + 1]; ++t) {
        const int64_t i = yidx[t];
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) c[col[q]] += (double)yval[t] * (double)val[q];
    }
}

// a cancelled request's column: inactive and free from the next kernel on
__global__ void k_cancel_col(ColState* st, int j) {
    st[j].active = 0;
    st[j].refill = 0;
    st[j].free_col = 1;
    st[j].a = 0.0;
    st[j].beta = 0.0;
    st[j].status = HD_COL_CANCELLED;
}

}  // namespace


// One persistent batch of columns and everything it needs on both sides.
struct Lane {
    Engine E;
    Refill rf;              // device pointers of the staging below (E.refill points here)
    int32_t slots = 0;
    int32_t slot_base = 0;  // reported slot number of column 0
    int S_full = 4;         // SpMM slab width measured for the whole lane
    void* dev = nullptr;
    hd_ctx* ctx = nullptr;
    // staging for the next step: device arrays and their pinned host sources
    int32_t cap_nnz = 0;
    int32_t *d_off = nullptr, *d_yidx = nullptr;
    float* d_yval = nullptr;
    double *d_bb = nullptr, *d_tol2 = nullptr, *d_C = nullptr;
    int* d_ctl = nullptr;   // [0] requests claimable this iteration, [1] next one for a stopping column
    int32_t* d_pre = nullptr;  // [Bp] staged request assigned to a free column (-1: none)
    int32_t* h_pre = nullptr;
    int32_t *h_off = nullptr, *h_yidx = nullptr;
    float* h_yval = nullptr;
    double *h_bb = nullptr, *h_tol2 = nullptr;
    int* h_ctl = nullptr;
    // what the step's scalar kernels recorded
    int32_t* h_assign = nullptr;
    int32_t* h_ret_iters = nullptr;
    int32_t* h_ret_status = nullptr;
    double* h_ret_rr = nullptr;
    std::vector<Req*> staged;
    // ranking outputs
    int32_t* d_idx = nullptr;
    float* d_sc = nullptr;
    int32_t* h_idx = nullptr;
    float* h_sc = nullptr;
    ColState* h_st = nullptr;
    std::vector<Req*> slot_req;

    bool running() const {
        for (Req* r : slot_req)
            if (r) return true;
        return false;
    }
    int32_t free_slots() const {
        int32_t f = 0;
        for (Req* r : slot_req) f += r == nullptr;
        return f;
    }
};

struct hd_server {
    hd_ctx* ctx = nullptr;
    const hd_graph* g = nullptr;
    const hd_eig* eig = nullptr;
    int32_t Kmax = 0, max_iter = 0;
    Lane lanes[2];  // [0] wide, [1] narrow (slots == 0 when absent)
    std::deque<Req*> queue;
    std::unordered_map<uint64_t, Req*> reqs;
    std::deque<uint64_t> finished;  // tickets retired and not yet reported by hd_serve_completed
    uint64_t next_ticket = 1;
};

static void lane_free(hd_ctx* ctx, Lane& L) {
    if (ctx) cudaStreamSynchronize(ctx->stream);
    cudaFree(L.dev);
    for (void* h : {(void*)L.h_off, (void*)L.h_yidx, (void*)L.h_yval, (void*)L.h_bb, (void*)L.h_tol2,
                    (void*)L.h_ctl, (void*)L.h_pre, (void*)L.h_assign, (void*)L.h_idx, (void*)L.h_sc,
                    (void*)L.h_st})
        cudaFreeHost(h);
    L = Lane();
}

static void server_free(hd_server* s) {
    if (!s) return;
    for (Lane& L : s->lanes) lane_free(s->ctx, L);
    for (auto& kv : s->reqs) delete kv.second;
    delete s;
}

// after the update: a column that took a request at the last scalar step gets
// its y (r = y - a q) and the exact correction of ||r||^2
static int refill_cb(void* arg) {
    return launch_refill_r(((Lane*)arg)->E);
}

// Buffers and engine of one lane of `slots` columns.
static int lane_open(hd_ctx* ctx, const hd_graph* g, const hd_eig* eig, double alpha, int32_t slots, int32_t max_iter,
                     int32_t Kmax, int32_t slot_base, Lane& L) {
    const bool lr_on = eig && eig->r > 0;
    const int64_t n = g->n;
    L.ctx = ctx;
    L.slots = slots;
    L.slot_base = slot_base;
    Engine& E = L.E;
    E.ctx = ctx;
    E.g = g;
    E.n = n;
    engine_set_reduction(E);
    E.B = slots;
    E.Bp = (slots + 3) / 4 * 4;
    E.has_lr = lr_on;
    E.r = lr_on ? eig->r : 0;
    E.eff_mode = lr_on ? HD_MODE_PCG : HD_MODE_PAPER;
    E.c1 = (float)(1.0 / (1.0 - alpha));
    E.c2 = (float)(alpha / (1.0 - alpha));
    E.xs = 1.0f;
    E.max_iter = max_iter;
    // one SpMM order in every lane: k_spmm's thread-per-row sums, one pass
    E.narrow4 = false;
    E.segK = 1;
    E.seg = nullptr;
    const int32_t Bp = E.Bp;
    const int rpad = lr_on ? (eig->r + 63) / 64 * 64 : 0;
    const int Bp16 = (Bp + 15) / 16 * 16;
    const int nchunk = lr_on ? lr_nchunk(ctx, eig, Bp) : 0;
    L.cap_nnz = Bp * REFILL_MAX_NNZ;
    const size_t vec = (size_t)n * Bp * 4;
    size_t bytes = 4 * ws_size(vec) + ws_size((size_t)E.nch * Bp * 8) + ws_size(Bp * sizeof(ColState)) +
                   ws_size(64) + 2 * ws_size((size_t)Bp * Kmax * 4) +
                   // staging: offsets, entries, bb, tol2, U^T y, control; per column: assignment,
                   // retired statistics, the installed request's y
                   ws_size((Bp + 1) * 4) + 2 * ws_size((size_t)L.cap_nnz * 4) + 2 * ws_size(Bp * 8) +
                   ws_size((size_t)Bp * std::max(rpad, 1) * 8) + ws_size(64) + 3 * ws_size(Bp * 4) +
                   ws_size(Bp * 8) + ws_size(Bp * 4) + 2 * ws_size((size_t)Bp * REFILL_MAX_NNZ * 4) +
                   ws_size(Bp * 4);
    if (lr_on)
        bytes += ws_size((size_t)nchunk * rpad * Bp * 4) + ws_size((size_t)rpad * Bp * 8) +
                 ws_size((size_t)rpad * Bp * 4) + 2 * ws_size((size_t)Bp16 * rpad * 2) + ws_size(rpad * 8);
    if (cudaMalloc(&L.dev, bytes) != cudaSuccess) {
        cudaGetLastError();
        L.dev = nullptr;
        return hd_fail(ctx, HD_ERR_OOM, "server buffers: %zu bytes", bytes);
    }
    L.slot_req.assign(slots, nullptr);
    WsCarver cv(L.dev);
    E.R = cv.take<float>((size_t)n * Bp);
    E.P = cv.take<float>((size_t)n * Bp);
    E.Q = cv.take<float>((size_t)n * Bp);
    E.X = cv.take<float>((size_t)n * Bp);
    E.part = cv.take<float2>((size_t)E.nch * Bp);
    E.st = cv.take<ColState>(Bp);
    E.num_active = cv.take<int>(16);
    E.err = E.num_active + 1;
    E.vl = vec_launch(ctx, n, Bp, tune_slab(ctx, g, Bp, E.P, E.Q));
    L.S_full = E.vl.S;
    L.d_idx = cv.take<int32_t>((size_t)Bp * Kmax);
    L.d_sc = cv.take<float>((size_t)Bp * Kmax);
    L.d_off = cv.take<int32_t>(Bp + 1);
    L.d_yidx = cv.take<int32_t>(L.cap_nnz);
    L.d_yval = cv.take<float>(L.cap_nnz);
    L.d_bb = cv.take<double>(Bp);
    L.d_tol2 = cv.take<double>(Bp);
    L.d_C = cv.take<double>((size_t)Bp * std::max(rpad, 1));
    L.d_ctl = cv.take<int>(16);
    Refill& rf = L.rf;
    rf.off = L.d_off;
    rf.yidx = L.d_yidx;
    rf.yval = L.d_yval;
    rf.bb = L.d_bb;
    rf.tol2 = L.d_tol2;
    rf.C = lr_on ? L.d_C : nullptr;
    rf.nstage = L.d_ctl;
    rf.next = L.d_ctl + 1;
    // assignment and retired statistics in one block (one copy to the host per
    // step): [assign | ret_iters | ret_status] int32[Bp] each, then ret_rr f64[Bp]
    uint8_t* ret = cv.take<uint8_t>((size_t)Bp * 20);
    rf.assign = (int32_t*)ret;
    rf.ret_iters = rf.assign + Bp;
    rf.ret_status = rf.ret_iters + Bp;
    rf.ret_rr = (double*)(rf.ret_status + Bp);
    rf.col_cnt = cv.take<int32_t>(Bp);
    rf.col_idx = cv.take<int32_t>((size_t)Bp * REFILL_MAX_NNZ);
    rf.col_val = cv.take<float>((size_t)Bp * REFILL_MAX_NNZ);
    L.d_pre = cv.take<int32_t>(Bp);
    rf.pre = L.d_pre;
    rf.rpad = rpad;
    rf.live = slots;
    E.refill = &L.rf;
    if (lr_on) {
        E.lr.e = eig;
        E.lr.rpad = rpad;
        E.lr.nchunk = nchunk;
        E.lr.Bp16 = Bp16;
        E.lr.part = cv.take<float>((size_t)nchunk * rpad * Bp);
        E.lr.C = cv.take<double>((size_t)rpad * Bp);
        E.lr.H = cv.take<float>((size_t)rpad * Bp);
        E.lr.Hhi = cv.take<__nv_bfloat16>((size_t)Bp16 * rpad);
        E.lr.Hlo = cv.take<__nv_bfloat16>((size_t)Bp16 * rpad);
        E.dcoef = cv.take<double>(rpad);
        std::vector<double> dc(rpad, 0.0);
        for (int k = 0; k < eig->r; ++k) {
            const double l = std::max(0.0, eig->lambda_h[k]);
            dc[k] = alpha * l / (1.0 - alpha * l);
        }
        HD_CUDA(ctx, cudaMemcpyAsync(E.dcoef, dc.data(), rpad * 8, cudaMemcpyHostToDevice, ctx->stream));
        HD_CUDA(ctx, cudaMemsetAsync(E.lr.Hhi, 0, (size_t)Bp16 * rpad * 2, ctx->stream));
        HD_CUDA(ctx, cudaMemsetAsync(E.lr.Hlo, 0, (size_t)Bp16 * rpad * 2, ctx->stream));
    }
    HD_CUDA(ctx, cudaMemsetAsync(L.dev, 0, 4 * ws_size(vec), ctx->stream));
    HD_CUDA(ctx, cudaMemsetAsync(E.num_active, 0, 16 * sizeof(int), ctx->stream));
    HD_CUDA(ctx, cudaMemsetAsync(L.d_ctl, 0, 16 * sizeof(int), ctx->stream));
    HD_CUDA(ctx, cudaMemsetAsync(rf.assign, 0xff, Bp * sizeof(int32_t), ctx->stream));
    HD_CUDA(ctx, cudaMemsetAsync(L.d_pre, 0xff, Bp * sizeof(int32_t), ctx->stream));
    std::vector<ColState> st0(Bp);
    for (int j = 0; j < Bp; ++j) {
        memset(&st0[j], 0, sizeof st0[j]);
        st0[j].status = HD_COL_EMPTY;
        st0[j].free_col = j < slots ? 1 : 0;
    }
    HD_CUDA(ctx, cudaMemcpyAsync(E.st, st0.data(), Bp * sizeof(ColState), cudaMemcpyHostToDevice, ctx->stream));
    if (cudaMallocHost(&L.h_off, (Bp + 1) * 4) || cudaMallocHost(&L.h_yidx, (size_t)L.cap_nnz * 4) ||
        cudaMallocHost(&L.h_yval, (size_t)L.cap_nnz * 4) || cudaMallocHost(&L.h_bb, Bp * 8) ||
        cudaMallocHost(&L.h_tol2, Bp * 8) || cudaMallocHost(&L.h_ctl, 16 * sizeof(int)) ||
        cudaMallocHost(&L.h_pre, Bp * 4) ||
        cudaMallocHost(&L.h_assign, (size_t)Bp * 20) ||
        cudaMallocHost(&L.h_idx, (size_t)Bp * Kmax * 4) || cudaMallocHost(&L.h_sc, (size_t)Bp * Kmax * 4) ||
        cudaMallocHost(&L.h_st, Bp * sizeof(ColState))) {
        cudaGetLastError();
        return hd_fail(ctx, HD_ERR_OOM, "pinned host buffers");
    }
    L.h_ret_iters = L.h_assign + Bp;
    L.h_ret_status = L.h_ret_iters + Bp;
    L.h_ret_rr = (double*)(L.h_ret_status + Bp);
    return HD_OK;
}

// A request that needs no iteration (y = 0, or tol >= 1 so that x = 0
// already meets it) finishes on the host: its x is 0, ranked as ids 0 .. K-1.
static void finish_trivial(hd_server* s, Req* r, double now) {
    r->iters = 0;
    r->status = r->bb == 0.0 ? HD_COL_EMPTY : HD_COL_CONVERGED;
    r->relres = r->bb == 0.0 ? 0.f : 1.f;
    r->out_idx.resize(r->K);
    r->out_score.assign(r->K, 0.f);
    for (int32_t k = 0; k < r->K; ++k) r->out_idx[k] = k < s->g->n ? k : -1;
    r->admit_s = r->done_s = now;
    r->done = true;
    s->finished.push_back(r->ticket);
}

// Stage up to a lane's width of queued requests for its next step: their
// observations and ||y||^2, tol^2 ||y||^2, and U^T y on the device.
static int lane_stage(hd_server* s, Lane& L) {
    hd_ctx* ctx = s->ctx;
    L.staged.clear();
    int32_t off = 0;
    const double now = now_s();
    while (!s->queue.empty() && (int32_t)L.staged.size() < L.slots) {
        Req* r = s->queue.front();
        if (off + (int32_t)r->idx.size() > L.cap_nnz) break;
        s->queue.pop_front();
        if (r->bb == 0.0 || r->bb <= (double)r->tol * r->tol * r->bb) {
            finish_trivial(s, r, now);
            continue;
        }
        const int c = (int)L.staged.size();
        L.staged.push_back(r);
        L.h_off[c] = off;
        L.h_bb[c] = r->bb;
        L.h_tol2[c] = (double)r->tol * (double)r->tol * r->bb;
        std::copy(r->idx.begin(), r->idx.end(), L.h_yidx + off);
        std::copy(r->val.begin(), r->val.end(), L.h_yval + off);
        off += (int32_t)r->idx.size();
    }
    const int ns = (int)L.staged.size();
    if (!ns) return HD_OK;
    L.h_off[ns] = off;
    HD_CUDA(ctx, cudaMemcpyAsync(L.d_off, L.h_off, (ns + 1) * 4, cudaMemcpyHostToDevice, ctx->stream));
    HD_CUDA(ctx, cudaMemcpyAsync(L.d_yidx, L.h_yidx, (size_t)off * 4, cudaMemcpyHostToDevice, ctx->stream));
    HD_CUDA(ctx, cudaMemcpyAsync(L.d_yval, L.h_yval, (size_t)off * 4, cudaMemcpyHostToDevice, ctx->stream));
    HD_CUDA(ctx, cudaMemcpyAsync(L.d_bb, L.h_bb, ns * 8, cudaMemcpyHostToDevice, ctx->stream));
    HD_CUDA(ctx, cudaMemcpyAsync(L.d_tol2, L.h_tol2, ns * 8, cudaMemcpyHostToDevice, ctx->stream));
    const hd_eig* e = s->eig;
    if (L.E.has_lr) {
        const int rpad = L.rf.rpad;
        if (e->sparse) {
            k_stage_c_sparse<<<ceil_div(ns, 32), 32, 0, ctx->stream>>>(e->sp_rp, e->sp_col, e->sp_val, rpad, ns,
                                                                       L.d_off, L.d_yidx, L.d_yval, L.d_C);
        } else if (e->storage == HD_F32) {
            k_stage_c<float><<<ns, 128, 0, ctx->stream>>>((const float*)e->U, e->scale, e->ldu, e->r, rpad, L.d_off,
                                                          L.d_yidx, L.d_yval, L.d_C);
        } else if (e->storage == HD_BF16) {
            k_stage_c<__nv_bfloat16><<<ns, 128, 0, ctx->stream>>>((const __nv_bfloat16*)e->U, e->scale, e->ldu, e->r,
                                                                  rpad, L.d_off, L.d_yidx, L.d_yval, L.d_C);
        } else {
            k_stage_c<__nv_fp8_e4m3><<<ns, 128, 0, ctx->stream>>>((const __nv_fp8_e4m3*)e->U, e->scale, e->ldu, e->r,
                                                                  rpad, L.d_off, L.d_yidx, L.d_yval, L.d_C);
        }
        HD_CHECK_LAUNCH(ctx);
    }
    return HD_OK;
}

// `iters` CG iterations of lane L; staged requests may be taken at the last
// one's scalar step; then retirement: the rankings of the requests that
// stopped, copied to the host.
static int lane_step(hd_server* s, Lane& L, int32_t iters) {
    hd_ctx* ctx = s->ctx;
    Engine& E = L.E;
    const int32_t Bp = E.Bp;
    const int ns = (int)L.staged.size();
    if (!L.running() && ns == 0) return HD_OK;
    if (ns > 0 && iters < 1) iters = 1;
    // staged requests go first to the lowest free columns (assigned here), the
    // rest to columns that stop in the last iteration; the tensor-core products
    // skip the columns above `live`, the highest column that can be occupied
    // (per-column arithmetic is unchanged)
    int32_t live = 0, npre = 0;
    for (int j = 0; j < L.slots; ++j)
        if (L.slot_req[j]) live = j + 1;
    if (ns > 0) {
        for (int j = 0; j < Bp; ++j) {
            L.h_pre[j] = -1;
            if (j < L.slots && !L.slot_req[j] && npre < ns) {
                L.h_pre[j] = npre++;
                live = std::max(live, j + 1);
            }
        }
        HD_CUDA(ctx, cudaMemcpyAsync(L.d_pre, L.h_pre, Bp * 4, cudaMemcpyHostToDevice, ctx->stream));
    }
    E.lr.live = live;
    L.rf.live = live;
    // the narrowest slab that holds every column that can be occupied (at most
    // the width measured for the full lane): a lightly loaded lane gathers less
    // per SpMM row.  Results do not depend on it: the reductions are chunked by
    // rows, and every slab width sums a row's entries in the same order.
    int S = L.S_full;
    for (int c : {4, 8, 16, 32, 64, 128})
        if (c >= live && c <= L.S_full && Bp % c == 0) {
            S = c;
            break;
        }
    if (S != E.vl.S) E.vl = vec_launch(ctx, E.n, Bp, S);
    HD_CUDA(ctx, cudaMemsetAsync(L.rf.assign, 0xff, Bp * sizeof(int32_t), ctx->stream));
    HD_CUDA(ctx, cudaMemsetAsync(L.d_ctl, 0, 2 * sizeof(int), ctx->stream));
    for (int t = 0; t < iters; ++t) {
        if (t == iters - 1 && ns > 0) {
            // staged requests can be taken at the last iteration only: a column's
            // stopped x must reach the host's ranking before an update resets it
            L.h_ctl[0] = ns;
            L.h_ctl[1] = npre;
            HD_CUDA(ctx, cudaMemcpyAsync(L.d_ctl, L.h_ctl, 2 * sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
        }
        int rc = engine_iteration(E, refill_cb, &L);
        if (rc) return rc;
    }
    // ---- poll and retire
    HD_CUDA(ctx, cudaMemcpyAsync(L.h_st, E.st, Bp * sizeof(ColState), cudaMemcpyDeviceToHost, ctx->stream));
    HD_CUDA(ctx, cudaMemcpyAsync(L.h_assign, L.rf.assign, (size_t)Bp * 20, cudaMemcpyDeviceToHost, ctx->stream));
    HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (E.has_lr && lr_use_tensor_cores(E.lr.e)) {
        const int frc = lr_tc_check_flags(ctx);
        if (frc) return frc;
    }
    const double t_step = now_s();
    std::vector<int32_t> Kc(Bp, 0);
    std::vector<std::pair<int, Req*>> fin;  // (column, request that stopped there)
    std::vector<char> taken(ns, 0);
    for (int j = 0; j < L.slots; ++j) {
        Req* old = L.slot_req[j];
        const int a = L.h_assign[j];
        if (a >= 0 && a < ns) {
            if (old) {
                old->iters = L.h_ret_iters[j];
                old->status = L.h_ret_status[j];
                old->relres = old->bb > 0 ? (float)std::sqrt(L.h_ret_rr[j] / old->bb) : 0.f;
                Kc[j] = old->K;
                fin.push_back({j, old});
            }
            Req* r = L.staged[a];
            r->slot = L.slot_base + j;
            r->admit_s = t_step;
            L.slot_req[j] = r;
            taken[a] = 1;
        } else if (old && !L.h_st[j].active) {
            const ColState& c = L.h_st[j];
            old->iters = c.iters;
            old->status = c.status;
            old->relres = c.bb > 0 ? (float)std::sqrt(c.rr / c.bb) : 0.f;
            Kc[j] = old->K;
            fin.push_back({j, old});
            L.slot_req[j] = nullptr;
        }
    }
    // staged requests no column took go back to the front of the queue, in order
    for (int a = ns - 1; a >= 0; --a)
        if (!taken[a]) s->queue.push_front(L.staged[a]);
    L.staged.clear();
    if (fin.empty()) return HD_OK;
    int rc;
    {
        HD_PROF(ctx, "rank");
        rc = hd_rank_impl(ctx, E.X, E.n, Bp, Bp, Kc.data(), s->Kmax, 0, L.d_idx, L.d_sc);
    }
    if (rc) return rc;
    // the rankings of the retiring columns: one copy per array, of the rows
    // from the first to the last retiring column (a few hundred KB at most)
    int jlo = Bp, jhi = -1;
    for (auto& f : fin) {
        jlo = std::min(jlo, f.first);
        jhi = std::max(jhi, f.first);
    }
    const size_t off = (size_t)jlo * s->Kmax, cnt = (size_t)(jhi - jlo + 1) * s->Kmax * 4;
    HD_CUDA(ctx, cudaMemcpyAsync(L.h_idx + off, L.d_idx + off, cnt, cudaMemcpyDeviceToHost, ctx->stream));
    HD_CUDA(ctx, cudaMemcpyAsync(L.h_sc + off, L.d_sc + off, cnt, cudaMemcpyDeviceToHost, ctx->stream));
    HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const double t_done = now_s();
    for (auto& f : fin) {
        const int j = f.first;
        Req* r = f.second;
        r->out_idx.assign(L.h_idx + (size_t)j * s->Kmax, L.h_idx + (size_t)j * s->Kmax + r->K);
        r->out_score.assign(L.h_sc + (size_t)j * s->Kmax, L.h_sc + (size_t)j * s->Kmax + r->K);
        r->done_s = t_done;
        r->done = true;
        s->finished.push_back(r->ticket);
    }
    return HD_OK;
}

// Launch, once, every kernel a lane can use later (one iteration per slab
// width with no column active and nothing staged, so every kernel returns at
// once, and a ranking with K = 0): the first launch of a kernel loads its
// module, which would otherwise stall the first steps that need it; the
// ranking also reserves its workspace at the lane's size here.
static int lane_warm(hd_server* s, Lane& L) {
    hd_ctx* ctx = s->ctx;
    Engine& E = L.E;
    for (int c : {4, 8, 16, 32, 64, 128}) {
        if (c > L.S_full || E.Bp % c) continue;
        E.vl = vec_launch(ctx, E.n, E.Bp, c);
        int rc = engine_iteration(E, refill_cb, &L);
        if (rc) return rc;
    }
    E.vl = vec_launch(ctx, E.n, E.Bp, L.S_full);
    std::vector<int32_t> K0(E.Bp, 0);
    return hd_rank_impl(ctx, E.X, E.n, E.Bp, E.Bp, K0.data(), s->Kmax, 0, L.d_idx, L.d_sc);
}

extern "C" {

int hd_serve_open(hd_ctx* ctx, const hd_graph* g, const hd_eig* eig, int mode, double alpha, int32_t max_slots,
                  size_t mem_budget, int32_t max_iter, int32_t Kmax, hd_server** out) {
    if (!ctx || !g || !out || max_slots < 1 || max_slots > 256 || Kmax < 1 || Kmax > 2048 || max_iter < 1)
        return HD_ERR_INVALID_ARG;
    if (!(alpha >= 0.0 && alpha < 1.0)) return hd_fail(ctx, HD_ERR_INVALID_ARG, "alpha=%g", alpha);
    const bool lr_on = eig && eig->r > 0;
    if (lr_on && mode != HD_MODE_PCG)
        return hd_fail(ctx, HD_ERR_INVALID_ARG, "the server runs PCG with eigenpairs (mode %d unsupported)", mode);
    *out = nullptr;
    HD_CUDA(ctx, cudaSetDevice(ctx->device));
    const int64_t n = g->n;
    // admission by device memory: each slot holds R, P, Q, X columns and its ranking
    const size_t per_slot = (size_t)4 * n * 4 + (size_t)Kmax * 8;
    int32_t slots = max_slots;
    if (mem_budget > 0) slots = (int32_t)std::min<size_t>(max_slots, mem_budget / per_slot);
    if (slots < 1) return hd_fail(ctx, HD_ERR_OOM, "memory budget %zu below one slot (%zu bytes)", mem_budget, per_slot);
    // the narrow lane: four more columns when the wide lane has at least eight
    // and the budget (if any) holds them too
    const bool narrow = slots >= 8 && (mem_budget == 0 || mem_budget / per_slot >= (size_t)slots + 4);
    hd_server* s = new hd_server();
    s->ctx = ctx;
    s->g = g;
    s->eig = eig;
    s->Kmax = Kmax;
    s->max_iter = max_iter;
    int rc = lane_open(ctx, g, eig, alpha, slots, max_iter, Kmax, 0, s->lanes[0]);
    if (!rc && narrow) rc = lane_open(ctx, g, eig, alpha, 4, max_iter, Kmax, slots, s->lanes[1]);
    // the wide lane last: the shared workspace is reserved at its (larger) size
    if (!rc && narrow) rc = lane_warm(s, s->lanes[1]);
    if (!rc) rc = lane_warm(s, s->lanes[0]);
    if (!rc) rc = hd_check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "server set-up", __FILE__, __LINE__);
    if (rc) {
        server_free(s);
        return rc;
    }
    *out = s;
    return HD_OK;
}

int hd_serve_slots(const hd_server* s) { return s ? s->lanes[0].slots : 0; }

int hd_serve_submit(hd_server* s, int32_t nnz_y, const int32_t* idx, const float* val, float tol, int32_t K,
                    uint64_t* ticket) {
    if (!s || !ticket || nnz_y < 0 || (nnz_y > 0 && (!idx || !val)) || K < 0 || K > s->Kmax || nnz_y > 512)
        return s ? hd_fail(s->ctx, HD_ERR_INVALID_ARG, "bad request (nnz %d, K %d)", nnz_y, K) : HD_ERR_INVALID_ARG;
    Req* r = new Req();
    // duplicates are summed; ||y||^2 is the norm of the summed vector
    std::vector<std::pair<int32_t, float>> e(nnz_y);
    for (int t = 0; t < nnz_y; ++t) {
        if (idx[t] < 0 || idx[t] >= s->g->n) {
            delete r;
            return hd_fail(s->ctx, HD_ERR_INVALID_ARG, "observation index %d out of range", idx[t]);
        }
        if (!std::isfinite(val[t])) {
            delete r;
            return hd_fail(s->ctx, HD_ERR_INVALID_ARG, "observation value %d is not finite", t);
        }
        e[t] = {idx[t], val[t]};
    }
    r->idx.assign(idx, idx + nnz_y);
    r->val.assign(val, val + nnz_y);
    std::stable_sort(e.begin(), e.end(), [](auto& a, auto& b) { return a.first < b.first; });
    double bb = 0.0;
    for (size_t t = 0; t < e.size();) {
        float acc = 0.0f;
        size_t u = t;
        for (; u < e.size() && e[u].first == e[t].first; ++u) acc += e[u].second;
        bb += (double)acc * (double)acc;
        t = u;
    }
    r->bb = bb;
    r->tol = tol;
    r->K = K;
    r->ticket = s->next_ticket++;
    r->submit_s = now_s();
    s->queue.push_back(r);
    s->reqs[r->ticket] = r;
    *ticket = r->ticket;
    return HD_OK;
}

int hd_serve_step(hd_server* s, int32_t iters, int32_t* busy) {
    if (!s || iters < 0) return HD_ERR_INVALID_ARG;
    Lane& W = s->lanes[0];
    Lane& N = s->lanes[1];
    // staging: a lightly loaded server uses the narrow lane
    if (!s->queue.empty()) {
        const bool narrow = N.slots > 0 && !W.running() && (int32_t)s->queue.size() <= N.free_slots();
        int rc = lane_stage(s, narrow ? N : W);
        if (rc) return rc;
    }
    for (int l = 0; l < 2; ++l) {
        if (s->lanes[l].slots == 0) continue;
        int rc = lane_step(s, s->lanes[l], iters);
        if (rc) return rc;
    }
    if (busy) {
        int32_t b = (int32_t)s->queue.size();
        for (const Lane& L : s->lanes)
            for (Req* r : L.slot_req) b += r != nullptr;
        *busy = b;
    }
    return HD_OK;
}

int hd_serve_cancel(hd_server* s, uint64_t ticket) {
    if (!s) return HD_ERR_INVALID_ARG;
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return HD_ERR_NOT_FOUND;
    Req* r = it->second;
    if (r->done) return HD_OK;
    auto q = std::find(s->queue.begin(), s->queue.end(), r);
    if (q != s->queue.end()) {
        s->queue.erase(q);
    } else {
        // running: free its column now; the column stops iterating at once
        for (Lane& L : s->lanes)
            for (int j = 0; j < L.slots; ++j)
                if (L.slot_req[j] == r) {
                    k_cancel_col<<<1, 1, 0, s->ctx->stream>>>(L.E.st, j);
                    HD_CHECK_LAUNCH(s->ctx);
                    L.slot_req[j] = nullptr;
                }
    }
    r->status = HD_COL_CANCELLED;
    r->done_s = now_s();
    r->done = true;
    s->finished.push_back(r->ticket);
    return HD_OK;
}

int hd_serve_poll(hd_server* s, uint64_t ticket, int32_t* idx_out, float* score_out, hd_req_stats* st) {
    if (!s) return HD_ERR_INVALID_ARG;
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return HD_ERR_NOT_FOUND;
    Req* r = it->second;
    if (!r->done) return HD_PENDING;
    if (idx_out) std::copy(r->out_idx.begin(), r->out_idx.end(), idx_out);
    if (score_out) std::copy(r->out_score.begin(), r->out_score.end(), score_out);
    if (st) {
        st->submit_s = r->submit_s;
        st->admit_s = r->admit_s;
        st->done_s = r->done_s;
        st->iters = r->iters;
        st->status = r->status;
        st->relres = r->relres;
        st->slot = r->slot;
    }
    s->reqs.erase(it);
    delete r;
    return HD_OK;
}

int hd_serve_completed(hd_server* s, uint64_t* tickets, int32_t max_tickets, int32_t* count) {
    if (!s || !count || max_tickets < 0 || (max_tickets > 0 && !tickets)) return HD_ERR_INVALID_ARG;
    int32_t c = 0;
    while (c < max_tickets && !s->finished.empty()) {
        tickets[c++] = s->finished.front();
        s->finished.pop_front();
    }
    *count = c;
    return HD_OK;
}

int hd_serve_close(hd_server* s) {
    server_free(s);
    return HD_OK;
}

}  // extern "C"
