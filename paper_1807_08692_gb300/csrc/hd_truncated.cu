// Temporal filtering on truncated graphs, "Temporal†" (Sec. 3.1, Sec. 5.1,
// Table 1): for query j only the shortlist S_j of database items is kept, the
// affinity restricted to S_j x S_j is normalised again by its own degrees,
// W_j = D_j^-1/2 A_{S_j S_j} D_j^-1/2, and L_alpha(W_j) x_j = y_j is solved by
// the same multi-column CG as the full query (one system per column).
//
// The affinity is recovered from the stored graph as A_ik = W_ik / (d_i^-1/2
// d_k^-1/2).  Building the B systems:
//   pos[j][i]  = position of id i in S_j, or -1           (one int32 map per column)
//   row (j, t) = the entries of A's row S_j[t] whose column is in S_j, in the
//                graph's column order, with their local positions
//   offsets by an exclusive scan of the row counts; values rescaled by the
//   subgraph's D^-1/2 on both sides.
// Observations outside the shortlist are dropped (index 0, value 0).
#include <algorithm>
#include <cmath>
#include <vector>

#include "hd_solve.cuh"

namespace {

// thread (t, j): pos[j][S_j[t]] = t; bad ids and duplicates raise the error flag
__global__ void k_ts_mark(const int32_t* sl_ptr, const int32_t* sl_idx, int32_t B, int64_t n, int32_t* pos,
                          int* err) {
    const int j = blockIdx.y;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int32_t b = sl_ptr[j], e = sl_ptr[j + 1];
    if (t >= e - b) return;
    const int32_t i = sl_idx[b + t];
    if (i < 0 || i >= n) {
        atomicExch(err, 1);
        return;
    }
    if (atomicCAS(&pos[(int64_t)j * n + i], -1, (int32_t)t) != -1) atomicExch(err, 2);
}

// one warp per (j, t): kept entries and the subgraph degree of row t
__global__ void k_ts_rowcount(const int32_t* rp, const int32_t* col, const float* val, const float* dinv,
                              const int32_t* sl_ptr, const int32_t* sl_idx, int32_t B, int64_t n, int64_t smax,
                              const int32_t* pos, int32_t* cnt, float* deg) {
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= (int64_t)B * smax) return;
    const int j = (int)(w / smax);
    const int64_t t = w - (int64_t)j * smax;
    const int32_t b = sl_ptr[j];
    int c = 0;
    float d = 0.0f;
    if (t < sl_ptr[j + 1] - b) {
        const int32_t i = sl_idx[b + t];
        const float di = dinv[i];
        const int32_t* pj = pos + (int64_t)j * n;
        for (int32_t q0 = rp[i]; q0 < rp[i + 1]; q0 += 32) {
            const int32_t q = q0 + lane;
            bool keep = false;
            float a = 0.0f;
            if (q < rp[i + 1]) {
                const int32_t k = col[q];
                keep = pj[k] >= 0;
                if (keep) a = val[q] / (di * dinv[k]);
            }
            c += __popc(__ballot_sync(0xffffffffu, keep));
            d += a;
        }
    }
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if (lane == 0) {
        cnt[w] = c;
        deg[w] = d;
    }
}

// one warp per (j, t): the kept entries with their local column, in order;
// values already scaled by D^-1/2 of the subgraph on both sides
__global__ void k_ts_fill(const int32_t* rp, const int32_t* col, const float* val, const float* dinv,
                          const int32_t* sl_ptr, const int32_t* sl_idx, int32_t B, int64_t n, int64_t smax,
                          const int32_t* pos, const float* sdinv, const int64_t* off, int32_t* ci, float* wv) {
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= (int64_t)B * smax) return;
    const int j = (int)(w / smax);
    const int64_t t = w - (int64_t)j * smax;
    const int32_t b = sl_ptr[j];
    if (t >= sl_ptr[j + 1] - b) return;
    const int32_t i = sl_idx[b + t];
    const float di = dinv[i];
    const float si = sdinv[w];
    const int32_t* pj = pos + (int64_t)j * n;
    const float* sj = sdinv + (int64_t)j * smax;
    const uint32_t below = (1u << lane) - 1u;
    int64_t at = off[w];
    for (int32_t q0 = rp[i]; q0 < rp[i + 1]; q0 += 32) {
        const int32_t q = q0 + lane;
        int32_t u = -1;
        float a = 0.0f;
        if (q < rp[i + 1]) {
            const int32_t k = col[q];
            u = pj[k];
            if (u >= 0) a = val[q] / (di * dinv[k]);
        }
        const uint32_t kb = __ballot_sync(0xffffffffu, u >= 0);
        if (u >= 0) {
            const int64_t o = at + __popc(kb & below);
            ci[o] = u;
            wv[o] = si * a * sj[u];
        }
        at += __popc(kb);
    }
}

__global__ void k_ts_sdinv(const float* deg, int64_t count, float* sdinv) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < count) sdinv[e] = deg[e] > 0.0f ? 1.0f / sqrtf(deg[e]) : 0.0f;
}

// observations of column j -> local positions (outside S_j: position 0, value 0)
__global__ void k_ts_map_y(const int32_t* y_ptr, const int32_t* y_idx, const float* y_val, int32_t B, int64_t n,
                           const int32_t* pos, int32_t* y_loc, float* y_lv, int* err) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= B) return;
    for (int32_t q = y_ptr[j]; q < y_ptr[j + 1]; ++q) {
        const int32_t i = y_idx[q];
        if (i < 0 || i >= n || !isfinite(y_val[q])) {
            atomicExch(err, 3);
            y_loc[q] = 0;
            y_lv[q] = 0.0f;
            continue;
        }
        const int32_t u = pos[(int64_t)j * n + i];
        y_loc[q] = u >= 0 ? u : 0;
        y_lv[q] = u >= 0 ? y_val[q] : 0.0f;
    }
}

// exclusive scan, part 1: sums of 1024-element blocks
__global__ void k_scan_sums(const int32_t* in, int64_t count, int64_t* bsum) {
    __shared__ int64_t sm[32];
    const int64_t e = blockIdx.x * 1024ll + threadIdx.x;
    int64_t v = e < count ? in[e] : 0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t s = 0;
        for (int w = 0; w < 32; ++w) s += sm[w];
        bsum[blockIdx.x] = s;
    }
}

// part 2: out[e] = boff[block] + sum of in[block start .. e - 1]; out[count] = total
__global__ void k_scan_apply(const int32_t* in, int64_t count, const int64_t* boff, int64_t* out) {
    __shared__ int64_t sm[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t e = blockIdx.x * 1024ll + threadIdx.x;
    const int64_t v = e < count ? in[e] : 0;
    int64_t x = v;  // inclusive scan within the warp
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t s = sm[lane];
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sm[lane] = s;  // inclusive over warps
    }
    __syncthreads();
    const int64_t before = boff[blockIdx.x] + (warp > 0 ? sm[warp - 1] : 0) + x - v;
    if (e < count) out[e] = before;
    if (e == count - 1) out[count] = before + v;
}

}  // namespace

extern "C" int hd_temporal_truncated(hd_ctx* ctx, const hd_graph* g, int32_t B, const int32_t* sl_ptr,
                                     const int32_t* sl_idx, const int32_t* y_ptr, const int32_t* y_idx,
                                     const float* y_val, double alpha, const float* tol, int32_t max_iter, float* X,
                                     int32_t ldx, int32_t* iters, float* relres, int32_t* status) {
    if (!ctx || !g || !sl_ptr || !sl_idx || !y_ptr || !tol || !X || B <= 0 || B > 4096) return HD_ERR_INVALID_ARG;
    HD_CUDA(ctx, cudaSetDevice(ctx->device));
    const int64_t n = g->n;
    // shortlist sizes on the host
    std::vector<int32_t> hp(B + 1);
    if (hd_is_device_ptr(sl_ptr)) {
        HD_CUDA(ctx, cudaMemcpy(hp.data(), sl_ptr, (B + 1) * 4, cudaMemcpyDeviceToHost));
    } else {
        std::copy(sl_ptr, sl_ptr + B + 1, hp.begin());
    }
    int64_t smax = 0;
    for (int j = 0; j < B; ++j) {
        if (hp[j + 1] < hp[j] || hp[j] < 0) return hd_fail(ctx, HD_ERR_INVALID_ARG, "shortlist pointers not monotone");
        smax = std::max<int64_t>(smax, hp[j + 1] - hp[j]);
    }
    if (smax <= 0) return hd_fail(ctx, HD_ERR_INVALID_ARG, "empty shortlists");
    if (smax > n) return hd_fail(ctx, HD_ERR_INVALID_ARG, "shortlist longer than the graph");
    if (ldx < B) return hd_fail(ctx, HD_ERR_INVALID_ARG, "ldx=%d < B=%d", ldx, B);
    const int64_t nsl = hp[B];
    int32_t nnz_y;
    if (hd_is_device_ptr(y_ptr)) {
        HD_CUDA(ctx, cudaMemcpy(&nnz_y, y_ptr + B, 4, cudaMemcpyDeviceToHost));
    } else {
        nnz_y = y_ptr[B];
    }
    if (nnz_y < 0 || (nnz_y > 0 && (!y_idx || !y_val))) return HD_ERR_INVALID_ARG;
    const int64_t rows = (int64_t)B * smax;
    const int64_t nblk = (rows + 1023) / 1024;

    // inputs on the device; everything here is this call's own allocation (the
    // solve below uses the context workspace)
    std::vector<void*> own;
    auto dalloc = [&](void** p, size_t bytes) -> int {
        if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
            cudaGetLastError();
            return hd_fail(ctx, HD_ERR_OOM, "truncated systems: %zu bytes", bytes);
        }
        own.push_back(*p);
        return HD_OK;
    };
    auto release = [&]() {
        cudaStreamSynchronize(ctx->stream);
        for (void* p : own) cudaFree(p);
        own.clear();
    };
    int rc = HD_OK;
#define TS_TRY(x)         \
    do {                  \
        if ((rc = (x))) { \
            release();    \
            return rc;    \
        }                 \
    } while (0)
#define TS_CUDA(x) TS_TRY(hd_check_cuda(ctx, (x), #x, __FILE__, __LINE__))
#define TS_LAUNCH() TS_TRY(hd_check_launch(ctx, __FILE__, __LINE__))
    int32_t *d_slp, *d_sli, *pos, *cnt, *d_yp, *d_yi, *y_loc;
    float *d_yv, *y_lv, *deg, *sdinv;
    int64_t *bsum, *off;
    int* err;
    TS_TRY(dalloc((void**)&d_slp, (B + 1) * 4));
    TS_TRY(dalloc((void**)&d_sli, (size_t)nsl * 4));
    TS_TRY(dalloc((void**)&pos, (size_t)B * n * 4));
    TS_TRY(dalloc((void**)&cnt, (size_t)rows * 4));
    TS_TRY(dalloc((void**)&deg, (size_t)rows * 4));
    TS_TRY(dalloc((void**)&sdinv, (size_t)rows * 4));
    TS_TRY(dalloc((void**)&bsum, (size_t)nblk * 8));
    TS_TRY(dalloc((void**)&off, (size_t)(rows + 1) * 8));
    TS_TRY(dalloc((void**)&d_yp, (B + 1) * 4));
    TS_TRY(dalloc((void**)&d_yi, (size_t)nnz_y * 4));
    TS_TRY(dalloc((void**)&d_yv, (size_t)nnz_y * 4));
    TS_TRY(dalloc((void**)&y_loc, (size_t)nnz_y * 4));
    TS_TRY(dalloc((void**)&y_lv, (size_t)nnz_y * 4));
    TS_TRY(dalloc((void**)&err, 16));
    auto copy_in = [&](void* dst, const void* src, size_t bytes) -> int {
        if (!bytes) return HD_OK;
        return hd_check_cuda(ctx, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, ctx->stream), "copy in",
                             __FILE__, __LINE__);
    };
    TS_TRY(copy_in(d_slp, hp.data(), (B + 1) * 4));
    TS_TRY(copy_in(d_sli, sl_idx, (size_t)nsl * 4));
    TS_TRY(copy_in(d_yp, y_ptr, (B + 1) * 4));
    TS_TRY(copy_in(d_yi, y_idx, (size_t)nnz_y * 4));
    TS_TRY(copy_in(d_yv, y_val, (size_t)nnz_y * 4));
    TS_CUDA(cudaMemsetAsync(err, 0, 16, ctx->stream));
    TS_CUDA(cudaMemsetAsync(pos, 0xff, (size_t)B * n * 4, ctx->stream));
    {
        HD_PROF(ctx, "trunc_build");
        k_ts_mark<<<dim3((unsigned)((smax + 255) / 256), B), 256, 0, ctx->stream>>>(d_slp, d_sli, B, n, pos, err);
        TS_LAUNCH();
        k_ts_rowcount<<<ceil_div(rows * 32, 256), 256, 0, ctx->stream>>>(g->row_ptr, g->col, g->val, g->dinv, d_slp,
                                                                         d_sli, B, n, smax, pos, cnt, deg);
        TS_LAUNCH();
        k_scan_sums<<<(unsigned)nblk, 1024, 0, ctx->stream>>>(cnt, rows, bsum);
        TS_LAUNCH();
    }
    std::vector<int64_t> hb(nblk);
    TS_CUDA(cudaMemcpyAsync(hb.data(), bsum, (size_t)nblk * 8, cudaMemcpyDeviceToHost, ctx->stream));
    TS_CUDA(cudaMemcpyAsync(ctx->h_poll, err, 4, cudaMemcpyDeviceToHost, ctx->stream));
    TS_CUDA(cudaStreamSynchronize(ctx->stream));
    if (ctx->h_poll[0]) {
        const int e = ctx->h_poll[0];
        release();
        return hd_fail(ctx, HD_ERR_INVALID_ARG, e == 2 ? "duplicate id in a shortlist" : "shortlist id out of range");
    }
    int64_t run = 0;
    for (int64_t b = 0; b < nblk; ++b) {
        const int64_t s = hb[b];
        hb[b] = run;
        run += s;
    }
    const int64_t nnz = run;
    TS_CUDA(cudaMemcpyAsync(bsum, hb.data(), (size_t)nblk * 8, cudaMemcpyHostToDevice, ctx->stream));
    int32_t* ci;
    float* wv;
    TS_TRY(dalloc((void**)&ci, (size_t)nnz * 4));
    TS_TRY(dalloc((void**)&wv, (size_t)nnz * 4));
    {
        HD_PROF(ctx, "trunc_build");
        k_scan_apply<<<(unsigned)nblk, 1024, 0, ctx->stream>>>(cnt, rows, bsum, off);
        TS_LAUNCH();
        k_ts_sdinv<<<ceil_div(rows, 256), 256, 0, ctx->stream>>>(deg, rows, sdinv);
        TS_LAUNCH();
        k_ts_fill<<<ceil_div(rows * 32, 256), 256, 0, ctx->stream>>>(g->row_ptr, g->col, g->val, g->dinv, d_slp, d_sli,
                                                                     B, n, smax, pos, sdinv, off, ci, wv);
        TS_LAUNCH();
        k_ts_map_y<<<ceil_div(B, 128), 128, 0, ctx->stream>>>(d_yp, d_yi, d_yv, B, n, pos, y_loc, y_lv, err);
        TS_LAUNCH();
    }
    TruncSys ts;
    ts.off = off;
    ts.ci = ci;
    ts.wv = wv;
    ts.B = B;
    ts.smax = smax;
    rc = hd_query_impl(ctx, g, &ts, nullptr, HD_MODE_PAPER, B, d_yp, y_loc, y_lv, alpha, tol, max_iter, X, ldx, iters,
                       relres, status);
    if (!rc) {
        TS_CUDA(cudaMemcpyAsync(ctx->h_poll, err, 4, cudaMemcpyDeviceToHost, ctx->stream));
        TS_CUDA(cudaStreamSynchronize(ctx->stream));
        if (ctx->h_poll[0]) rc = hd_fail(ctx, HD_ERR_INVALID_ARG, "bad observation: index out of range or non-finite value");
    }
    release();
    return rc;
#undef TS_LAUNCH
#undef TS_CUDA
#undef TS_TRY
}
