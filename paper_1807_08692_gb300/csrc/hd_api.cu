// Context, memory staging, graph and eigenpair handles of the C ABI (include/hd.h).
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cmath>
#include <vector>

#include "hd_internal.cuh"

int hd_fail(hd_ctx* ctx, int code, const char* fmt, ...) {
    if (ctx) {
        char buf[1024];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return code;
}

cudaEvent_t hd_prof_event(hd_ctx* ctx) {
    if (!ctx->ev_pool.empty()) {
        cudaEvent_t e = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

bool hd_is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int hd_ws_reserve(hd_ctx* ctx, size_t bytes, void** out) {
    if (bytes == 0) bytes = 256;
    if (bytes > ctx->ws_bytes) {
        if (ctx->ws) {
            HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
            HD_CUDA(ctx, cudaFree(ctx->ws));
            ctx->ws = nullptr;
            ctx->ws_bytes = 0;
        }
        size_t want = bytes + bytes / 8;
        cudaError_t e = cudaMalloc(&ctx->ws, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return hd_fail(ctx, HD_ERR_OOM, "workspace of %zu bytes: %s", want, cudaGetErrorString(e));
        }
        ctx->ws_bytes = want;
    }
    *out = ctx->ws;
    return HD_OK;
}

int hd_stage_in(hd_ctx* ctx, const void* src, size_t bytes, void* dev_scratch, const void** dev_out) {
    if (bytes == 0 || hd_is_device_ptr(src)) {
        *dev_out = src;
        return HD_OK;
    }
    HD_CUDA(ctx, cudaMemcpyAsync(dev_scratch, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
    *dev_out = dev_scratch;
    return HD_OK;
}

static int copy_out(hd_ctx* ctx, void* dst, const void* src_dev, size_t bytes) {
    if (!dst || bytes == 0) return HD_OK;
    cudaMemcpyKind kind = hd_is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    HD_CUDA(ctx, cudaMemcpyAsync(dst, src_dev, bytes, kind, ctx->stream));
    if (kind == cudaMemcpyDeviceToHost) HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return HD_OK;
}

extern "C" {

int hd_create(hd_ctx** out, int device, void* cuda_stream) {
    if (!out) return HD_ERR_INVALID_ARG;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return HD_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return HD_ERR_CUDA;
    hd_ctx* c = new hd_ctx();
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaMallocHost(&c->h_poll, 64 * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&c->d_flags, 64 * sizeof(int)) != cudaSuccess ||
        cudaMemset(c->d_flags, 0, 64 * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        delete c;
        return HD_ERR_CUDA;
    }
    *out = c;
    return HD_OK;
}

int hd_set_stream(hd_ctx* ctx, void* cuda_stream) {
    if (!ctx) return HD_ERR_INVALID_ARG;
    HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->stream = (cudaStream_t)cuda_stream;
    return HD_OK;
}

int hd_destroy(hd_ctx* ctx) {
    if (!ctx) return HD_OK;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    hd_rank_static_forget(ctx->device);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->h_poll) cudaFreeHost(ctx->h_poll);
    if (ctx->d_flags) cudaFree(ctx->d_flags);
    for (auto& kv : ctx->iter_graphs) cudaGraphExecDestroy(kv.second.exec);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    for (auto& kv : ctx->prof_ev)
        for (auto& pr : kv.second) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
    for (auto e : ctx->ev_pool) cudaEventDestroy(e);
    delete ctx;
    return HD_OK;
}

const char* hd_last_error(const hd_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int hd_profile_enable(hd_ctx* ctx, int on) {
    if (!ctx) return HD_ERR_INVALID_ARG;
    ctx->prof = on != 0;
    return HD_OK;
}

int hd_profile_read(hd_ctx* ctx, const char* name, int64_t* launches, double* total_ms, int64_t* busy_launches) {
    if (!ctx || !name) return HD_ERR_INVALID_ARG;
    HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    double tot = 0.0, mx = 0.0;
    int64_t cnt = 0, busy = 0;
    std::vector<float> each;
    auto it = ctx->prof_ev.find(name);
    if (it != ctx->prof_ev.end()) {
        for (auto& pr : it->second) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, pr.first, pr.second) != cudaSuccess) ms = 0.0f;
            each.push_back(ms);
            tot += ms;
            mx = ms > mx ? ms : mx;
            ++cnt;
            ctx->ev_pool.push_back(pr.first);
            ctx->ev_pool.push_back(pr.second);
        }
        it->second.clear();
    }
    for (float ms : each) busy += ms >= 0.05 * mx;
    cudaGetLastError();
    if (launches) *launches = cnt;
    if (total_ms) *total_ms = tot;
    if (busy_launches) *busy_launches = busy;
    return HD_OK;
}
int64_t hd_launch_count(const hd_ctx* ctx) { return ctx ? ctx->launches : 0; }
int hd_workspace_bytes(const hd_ctx* ctx, size_t* bytes) {
    if (!ctx || !bytes) return HD_ERR_INVALID_ARG;
    *bytes = ctx->ws_bytes;
    return HD_OK;
}
int hd_num_sms(const hd_ctx* ctx) { return ctx ? ctx->num_sms : 0; }

}  // extern "C"

// ------------------------------------------------------------------ graph kernels

__global__ void k_check_csr(const int32_t* rp, const int32_t* col, int64_t n, int64_t nnz, int* flag) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        int32_t b = rp[i], e = rp[i + 1];
        if (b > e || b < 0 || e > nnz) atomicExch(flag, 1);
        if (i == 0 && b != 0) atomicExch(flag, 1);
        if (i == n - 1 && e != nnz) atomicExch(flag, 1);
    }
    for (int64_t t = i; t < nnz; t += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = col[t];
        if (c < 0 || c >= n) atomicExch(flag, 2);
    }
}

// One thread per row: insertion sort of (col, val) by column.
__global__ void k_sort_rows(const int32_t* rp, int32_t* col, float* val, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t b = rp[i], e = rp[i + 1];
    for (int32_t t = b + 1; t < e; ++t) {
        int32_t c = col[t];
        float v = val[t];
        int32_t s = t - 1;
        while (s >= b && col[s] > c) {
            col[s + 1] = col[s];
            val[s + 1] = val[s];
            --s;
        }
        col[s + 1] = c;
        val[s + 1] = v;
    }
}

// D = diag(A 1) in fp64 per row; dinv = D^-1/2 (0 for degree 0).
__global__ void k_degrees(const int32_t* rp, const float* val, int64_t n, float* dinv, double* dinv64) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int32_t t = rp[i]; t < rp[i + 1]; ++t) s += (double)val[t];
    double di = s > 0.0 ? 1.0 / sqrt(s) : 0.0;
    dinv64[i] = di;
    dinv[i] = (float)di;
}

// W_ij = D_i^-1/2 A_ij D_j^-1/2, one warp per row.
__global__ void k_scale_rows(const int32_t* rp, const int32_t* col, float* val, int64_t n,
                             const double* dinv64) {
    int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (row >= n) return;
    double di = dinv64[row];
    for (int32_t t = rp[row] + lane; t < rp[row + 1]; t += 32)
        val[t] = (float)((double)val[t] * di * dinv64[col[t]]);
}

int hd_normalize_graph(hd_ctx* ctx, hd_graph* g) {
    void* ws;
    int rc = hd_ws_reserve(ctx, ws_size(g->n * sizeof(double)), &ws);
    if (rc) return rc;
    double* dinv64 = (double*)ws;
    k_degrees<<<ceil_div(g->n, 256), 256, 0, ctx->stream>>>(g->row_ptr, g->val, g->n, g->dinv, dinv64);
    HD_CHECK_LAUNCH(ctx);
    k_scale_rows<<<ceil_div(g->n * 32, 256), 256, 0, ctx->stream>>>(g->row_ptr, g->col, g->val, g->n, dinv64);
    HD_CHECK_LAUNCH(ctx);
    return HD_OK;
}

static void graph_free(hd_graph* g) {
    if (!g) return;
    cudaFree(g->row_ptr);
    cudaFree(g->col);
    cudaFree(g->val);
    cudaFree(g->dinv);
    for (auto& kv : g->seg_bounds) cudaFree(kv.second);
    delete g;
}

static int graph_alloc(hd_ctx* ctx, int64_t n, int64_t nnz, hd_graph** out) {
    hd_graph* g = new hd_graph();
    g->n = n;
    g->nnz = nnz;
    g->device = ctx->device;
    cudaError_t e1 = cudaMalloc(&g->row_ptr, (n + 1) * sizeof(int32_t));
    cudaError_t e2 = cudaMalloc(&g->col, (nnz > 0 ? nnz : 1) * sizeof(int32_t));
    cudaError_t e3 = cudaMalloc(&g->val, (nnz > 0 ? nnz : 1) * sizeof(float));
    cudaError_t e4 = cudaMalloc(&g->dinv, n * sizeof(float));
    if (e1 || e2 || e3 || e4) {
        cudaGetLastError();
        graph_free(g);
        return hd_fail(ctx, HD_ERR_OOM, "graph n=%lld nnz=%lld", (long long)n, (long long)nnz);
    }
    *out = g;
    return HD_OK;
}

int hd_graph_alloc_internal(hd_ctx* ctx, int64_t n, int64_t nnz, hd_graph** out) {
    return graph_alloc(ctx, n, nnz, out);
}
void hd_graph_free_internal(hd_graph* g) { graph_free(g); }

// row_ptr monotone from 0 to nnz and every column in [0, n) (checked on the device)
int hd_graph_check(hd_ctx* ctx, const hd_graph* g) {
    const int64_t n = g->n, nnz = g->nnz;
    HD_CUDA(ctx, cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), ctx->stream));
    const int64_t m = n > nnz ? n : nnz;
    k_check_csr<<<ceil_div(m, 256) > 4096 ? 4096 : ceil_div(m, 256), 256, 0, ctx->stream>>>(g->row_ptr, g->col, n,
                                                                                        nnz, ctx->d_flags);
    HD_CHECK_LAUNCH(ctx);
    HD_CUDA(ctx, cudaMemcpyAsync(ctx->h_poll, ctx->d_flags, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->h_poll[0])
        return hd_fail(ctx, HD_ERR_INVALID_ARG,
                       ctx->h_poll[0] == 1 ? "row_ptr not monotone from 0 to nnz" : "column index out of range");
    return HD_OK;
}

extern "C" {

int hd_graph_from_csr(hd_ctx* ctx, int64_t n, int64_t nnz, const int32_t* row_ptr, const int32_t* col,
                      const float* val, int normalized, hd_graph** out) {
    if (!ctx || !out || !row_ptr || (nnz > 0 && (!col || !val))) return HD_ERR_INVALID_ARG;
    *out = nullptr;
    if (n <= 0 || nnz < 0 || nnz >= (1ll << 31) || n >= (1ll << 31))
        return hd_fail(ctx, HD_ERR_INVALID_ARG, "bad sizes n=%lld nnz=%lld", (long long)n, (long long)nnz);
    HD_CUDA(ctx, cudaSetDevice(ctx->device));
    hd_graph* g;
    int rc = graph_alloc(ctx, n, nnz, &g);
    if (rc) return rc;
    auto kind = [](const void* p) { return hd_is_device_ptr(p) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; };
    if (cudaMemcpyAsync(g->row_ptr, row_ptr, (n + 1) * 4, kind(row_ptr), ctx->stream) ||
        (nnz && cudaMemcpyAsync(g->col, col, nnz * 4, kind(col), ctx->stream)) ||
        (nnz && cudaMemcpyAsync(g->val, val, nnz * 4, kind(val), ctx->stream))) {
        graph_free(g);
        return hd_fail(ctx, HD_ERR_CUDA, "graph upload: %s", cudaGetErrorString(cudaGetLastError()));
    }
    cudaMemsetAsync(ctx->d_flags, 0, sizeof(int), ctx->stream);
    k_check_csr<<<ceil_div(n > nnz ? n : nnz, 256) > 4096 ? 4096 : ceil_div(n > nnz ? n : nnz, 256), 256, 0,
                  ctx->stream>>>(g->row_ptr, g->col, n, nnz, ctx->d_flags);
    ctx->launches++;
    cudaMemcpyAsync(ctx->h_poll, ctx->d_flags, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        graph_free(g);
        return hd_fail(ctx, HD_ERR_CUDA, "graph check: %s", cudaGetErrorString(cudaGetLastError()));
    }
    if (ctx->h_poll[0]) {
        graph_free(g);
        return hd_fail(ctx, HD_ERR_INVALID_ARG, ctx->h_poll[0] == 1 ? "row_ptr not monotone from 0 to nnz"
                                                                     : "column index out of range");
    }
    k_sort_rows<<<ceil_div(n, 128), 128, 0, ctx->stream>>>(g->row_ptr, g->col, g->val, n);
    ctx->launches++;
    if (normalized) {
        // dinv is not known for a pre-normalised W; report 1 (unused by the solver).
        std::vector<float> ones(n, 1.0f);
        cudaMemcpyAsync(g->dinv, ones.data(), n * 4, cudaMemcpyHostToDevice, ctx->stream);
        cudaStreamSynchronize(ctx->stream);
    } else {
        rc = hd_normalize_graph(ctx, g);
        if (rc) {
            graph_free(g);
            return rc;
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        graph_free(g);
        return hd_fail(ctx, HD_ERR_CUDA, "graph_from_csr: %s", cudaGetErrorString(e));
    }
    *out = g;
    return HD_OK;
}

int hd_graph_tuning(const hd_graph* g, int32_t Bp, int32_t* slab, int32_t* segments) {
    if (!g) return HD_ERR_INVALID_ARG;
    auto it = g->slab_cache.find(Bp);
    if (it == g->slab_cache.end()) return HD_ERR_INVALID_ARG;
    if (slab) *slab = it->second;
    auto is = g->seg_cache.find(Bp);
    if (segments) *segments = is == g->seg_cache.end() ? 1 : is->second;
    return HD_OK;
}

int hd_graph_info(const hd_graph* g, int64_t* n, int64_t* nnz) {
    if (!g) return HD_ERR_INVALID_ARG;
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    return HD_OK;
}

int hd_graph_export(hd_ctx* ctx, const hd_graph* g, int32_t* row_ptr, int32_t* col, float* val, float* dinv) {
    if (!ctx || !g) return HD_ERR_INVALID_ARG;
    int rc;
    if ((rc = copy_out(ctx, row_ptr, g->row_ptr, (g->n + 1) * 4))) return rc;
    if ((rc = copy_out(ctx, col, g->col, g->nnz * 4))) return rc;
    if ((rc = copy_out(ctx, val, g->val, g->nnz * 4))) return rc;
    if ((rc = copy_out(ctx, dinv, g->dinv, g->n * 4))) return rc;
    HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return HD_OK;
}

int hd_graph_destroy(hd_graph* g) {
    graph_free(g);
    return HD_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ eigenpairs

__global__ void k_store_u(const float* src, int32_t lds, int64_t n, int32_t r, int32_t ldu, int storage,
                          void* dst, float* scale, __nv_bfloat16* split, int32_t ldsplit) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* s = src + i * lds;
    if (storage == HD_F32) {
        float* d = (float*)dst + i * ldu;
        for (int k = 0; k < ldu; ++k) d[k] = k < r ? s[k] : 0.0f;
        if (split) {
            const int half = ldsplit / 2;
            __nv_bfloat16* h = split + i * ldsplit;
            for (int k = 0; k < half; ++k) {
                const float v = k < r ? s[k] : 0.0f;
                const __nv_bfloat16 hi = __float2bfloat16_rn(v);
                h[k] = hi;
                h[half + k] = __float2bfloat16_rn(v - __bfloat162float(hi));
            }
        }
    } else if (storage == HD_BF16) {
        __nv_bfloat16* d = (__nv_bfloat16*)dst + i * ldu;
        for (int k = 0; k < ldu; ++k) d[k] = __float2bfloat16_rn(k < r ? s[k] : 0.0f);
    } else {
        float m = 0.0f;
        for (int k = 0; k < r; ++k) m = fmaxf(m, fabsf(s[k]));
        float sc = m > 0.0f ? m / 448.0f : 1.0f;
        scale[i] = sc;
        __nv_fp8_e4m3* d = (__nv_fp8_e4m3*)dst + i * ldu;
        for (int k = 0; k < ldu; ++k) d[k] = __nv_fp8_e4m3(k < r ? s[k] / sc : 0.0f);
    }
}

__global__ void k_load_u(const void* U, const float* scale, int64_t n, int32_t r, int32_t ldu, int storage,
                         float* dst) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int k = 0; k < r; ++k) {
        float v;
        if (storage == HD_F32) v = ((const float*)U)[i * ldu + k];
        else if (storage == HD_BF16) v = __bfloat162float(((const __nv_bfloat16*)U)[i * ldu + k]);
        else v = float(((const __nv_fp8_e4m3*)U)[i * ldu + k]) * scale[i];
        dst[i * r + k] = v;
    }
}

static void eig_free(hd_eig* e) {
    if (!e) return;
    cudaFree(e->U);
    cudaFree(e->Usplit);
    cudaFree(e->scale);
    cudaFree(e->lambda_d);
    cudaFree(e->sp_rp);
    cudaFree(e->sp_col);
    cudaFree(e->sp_val);
    cudaFree(e->sp_cp);
    cudaFree(e->sp_row);
    cudaFree(e->sp_cval);
    delete e;
}

int hd_check_launch(hd_ctx* ctx, const char* file, int line) {
    ctx->launches++;
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 0 : hd_fail(ctx, HD_ERR_CUDA, "%s:%d launch: %s", file, line, cudaGetErrorString(e));
}

int hd_eig_alloc(hd_ctx* ctx, int64_t n, int32_t r, int storage, hd_eig** out) {
    hd_eig* e = new hd_eig();
    e->n = n;
    e->r = r;
    e->storage = storage;
    e->ldu = ((r + 15) / 16) * 16;
    if (e->ldu == 0) e->ldu = 16;
    size_t es = storage == HD_F32 ? 4 : storage == HD_BF16 ? 2 : 1;
    cudaError_t a = cudaMalloc(&e->U, (size_t)n * e->ldu * es);
    cudaError_t b = cudaMalloc(&e->scale, n * sizeof(float));
    cudaError_t c = cudaMalloc(&e->lambda_d, (r > 0 ? r : 1) * sizeof(double));
    cudaError_t d = cudaSuccess;
    if (storage == HD_F32 && r > 0) {
        e->lds = 2 * ((r + 127) / 128 * 128);
        d = cudaMalloc(&e->Usplit, (size_t)n * e->lds * 2);
    }
    if (a || b || c || d) {
        cudaGetLastError();
        eig_free(e);
        return hd_fail(ctx, HD_ERR_OOM, "eigenpairs n=%lld r=%d", (long long)n, r);
    }
    *out = e;
    return HD_OK;
}

int hd_eig_store_from_device_f32(hd_ctx* ctx, hd_eig* e, const float* U_d, int32_t ldsrc) {
    k_store_u<<<ceil_div(e->n, 256), 256, 0, ctx->stream>>>(U_d, ldsrc, e->n, e->r, e->ldu, e->storage, e->U,
                                                            e->scale, (__nv_bfloat16*)e->Usplit, e->lds);
    HD_CHECK_LAUNCH(ctx);
    return HD_OK;
}

extern "C" {

int hd_eig_from_host(hd_ctx* ctx, const hd_graph* g, int32_t r, const double* lambda, const float* U, int storage,
                     hd_eig** out) {
    if (!ctx || !g || !out || r < 0 || (r > 0 && (!lambda || !U))) return HD_ERR_INVALID_ARG;
    if (storage != HD_F32 && storage != HD_BF16 && storage != HD_FP8)
        return hd_fail(ctx, HD_ERR_INVALID_ARG, "storage %d", storage);
    if (r > 1024) return hd_fail(ctx, HD_ERR_INVALID_ARG, "r=%d > 1024", r);
    *out = nullptr;
    hd_eig* e;
    int rc = hd_eig_alloc(ctx, g->n, r, storage, &e);
    if (rc) return rc;
    e->lambda_h.assign(lambda, lambda + r);
    if (r > 0) {
        HD_CUDA(ctx, cudaMemcpyAsync(e->lambda_d, lambda, r * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
        const float* Ud = U;
        float* tmp = nullptr;
        if (!hd_is_device_ptr(U)) {
            HD_CUDA(ctx, cudaMalloc(&tmp, (size_t)g->n * r * sizeof(float)));
            HD_CUDA(ctx, cudaMemcpyAsync(tmp, U, (size_t)g->n * r * sizeof(float), cudaMemcpyHostToDevice,
                                         ctx->stream));
            Ud = tmp;
        }
        rc = hd_eig_store_from_device_f32(ctx, e, Ud, r);
        cudaStreamSynchronize(ctx->stream);
        if (tmp) cudaFree(tmp);
        if (rc) {
            eig_free(e);
            return rc;
        }
    }
    *out = e;
    return HD_OK;
}

int hd_eig_info(const hd_eig* e, int32_t* r, int* storage) {
    if (!e) return HD_ERR_INVALID_ARG;
    if (r) *r = e->r;
    if (storage) *storage = e->storage;
    return HD_OK;
}

int hd_eig_restarts(const hd_eig* e, int32_t* restarts) {
    if (!e || !restarts) return HD_ERR_INVALID_ARG;
    *restarts = e->restarts;
    return HD_OK;
}

int hd_eig_export(hd_ctx* ctx, const hd_eig* e, double* lambda, float* U) {
    if (!ctx || !e) return HD_ERR_INVALID_ARG;
    if (lambda) memcpy(lambda, e->lambda_h.data(), e->r * sizeof(double));
    if (U && e->r > 0) {
        float* Ud = U;
        float* tmp = nullptr;
        if (!hd_is_device_ptr(U)) {
            HD_CUDA(ctx, cudaMalloc(&tmp, (size_t)e->n * e->r * sizeof(float)));
            Ud = tmp;
        }
        if (e->sparse) {
            int rc = hd_eig_sparse_export(ctx, e, Ud);
            if (rc) {
                if (tmp) cudaFree(tmp);
                return rc;
            }
        } else {
            k_load_u<<<ceil_div(e->n, 256), 256, 0, ctx->stream>>>(e->U, e->scale, e->n, e->r, e->ldu, e->storage, Ud);
            HD_CHECK_LAUNCH(ctx);
        }
        if (tmp) {
            HD_CUDA(ctx, cudaMemcpyAsync(U, tmp, (size_t)e->n * e->r * 4, cudaMemcpyDeviceToHost, ctx->stream));
            HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
            cudaFree(tmp);
        }
    }
    HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return HD_OK;
}

int hd_eig_destroy(hd_eig* e) {
    eig_free(e);
    return HD_OK;
}

}  // extern "C"
