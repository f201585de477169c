// SHybrid (Sec. 5.3): the spectral embedding U with its smallest entries set to
// zero, stored sparse, and the two low-rank products of every query mode on it.
//
// Selection: the round(s * n * r) entries of smallest |U_ij| over the whole
// n x r matrix are dropped; among equal magnitudes the later row-major entry
// goes first.  Equivalently the kept set is the top (n r - drop) of |U_ij| with
// ties kept in row-major order, found here by a radix select over the fp32 bit
// patterns of |U_ij| (monotone for non-negative floats) and a tie rank taken
// from a scan over rows.
//
// Storage: CSR (rows of U, for U H) and CSC (columns of U, for U^T V), fp32
// values equal to the dequantised stored entries, 64-bit offsets.
//
//  expand : out_i = op(sum_{(k, u) in row i} u H_k)     thread per (row, 4 columns)
//  reduce : part_c[k] = sum_{(i, u) in chunk c of column k} u V_i   warp per (chunk, k);
//           each column's entries are split into nchunk equal ranges, summed in
//           row order, so the result does not depend on the launch.
#include <algorithm>
#include <cmath>
#include <vector>

#include "hd_solve.cuh"

namespace {

constexpr int CHR = 2048;  // rows per chunk when the CSC is filled

__device__ __forceinline__ float u_entry(const void* U, const float* scale, int storage, int ldu, int64_t i, int k) {
    if (storage == HD_F32) return ((const float*)U)[i * ldu + k];
    if (storage == HD_BF16) return __bfloat162float(((const __nv_bfloat16*)U)[i * ldu + k]);
    return float(((const __nv_fp8_e4m3*)U)[i * ldu + k]) * scale[i];
}

__device__ __forceinline__ uint32_t mag_key(float v) { return __float_as_uint(fabsf(v)); }

// 256-bin histogram of digit (key >> shift) & 255 over the keys whose bits under
// `mask` equal `prefix`
__global__ void k_sp_hist(const void* U, const float* scale, int storage, int ldu, int64_t n, int r, uint32_t prefix,
                          uint32_t mask, int shift, unsigned long long* hist) {
    __shared__ unsigned int sh[256];
    for (int b = threadIdx.x; b < 256; b += blockDim.x) sh[b] = 0;
    __syncthreads();
    const int64_t tot = n * r;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / r;
        const int k = (int)(e - i * r);
        const uint32_t key = mag_key(u_entry(U, scale, storage, ldu, i, k));
        if ((key & mask) == prefix) atomicAdd(&sh[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += blockDim.x)
        if (sh[b]) atomicAdd(&hist[b], (unsigned long long)sh[b]);
}

// per row (one warp): entries above the threshold and entries equal to it
__global__ void k_sp_rowcount(const void* U, const float* scale, int storage, int ldu, int64_t n, int r, uint32_t T,
                              int32_t* gt, int32_t* tie) {
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    int g = 0, t = 0;
    for (int k0 = 0; k0 < r; k0 += 32) {
        const int k = k0 + lane;
        const uint32_t key = k < r ? mag_key(u_entry(U, scale, storage, ldu, i, k)) : 0u;
        g += __popc(__ballot_sync(0xffffffffu, k < r && key > T));
        t += __popc(__ballot_sync(0xffffffffu, k < r && key == T));
    }
    if (lane == 0) {
        gt[i] = g;
        tie[i] = t;
    }
}

// CSR fill (one warp per row), entries in column order
__global__ void k_sp_fill_rows(const void* U, const float* scale, int storage, int ldu, int64_t n, int r, uint32_t T,
                               int64_t m, const int64_t* tie_before, const int64_t* rp, int32_t* col, float* val) {
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    const uint32_t below = (1u << lane) - 1u;
    int64_t pos = rp[i];
    int64_t ties = tie_before[i];
    for (int k0 = 0; k0 < r; k0 += 32) {
        const int k = k0 + lane;
        const float v = k < r ? u_entry(U, scale, storage, ldu, i, k) : 0.0f;
        const uint32_t key = mag_key(v);
        const bool is_tie = k < r && key == T;
        const uint32_t tb = __ballot_sync(0xffffffffu, is_tie);
        const bool keep = k < r && (key > T || (is_tie && ties + __popc(tb & below) < m));
        const uint32_t kb = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const int64_t q = pos + __popc(kb & below);
            col[q] = k;
            val[q] = v;
        }
        pos += __popc(kb);
        ties += __popc(tb);
    }
}

// entries per (chunk of CHR rows, column)
__global__ void k_sp_colcount(const int64_t* rp, const int32_t* col, int64_t n, int r, int32_t* cnt) {
    extern __shared__ int32_t sc[];
    for (int k = threadIdx.x; k < r; k += blockDim.x) sc[k] = 0;
    __syncthreads();
    const int64_t i0 = (int64_t)blockIdx.x * CHR, i1 = min(n, i0 + CHR);
    for (int64_t t = rp[i0] + threadIdx.x; t < rp[i1]; t += blockDim.x) atomicAdd(&sc[col[t]], 1);
    __syncthreads();
    for (int k = threadIdx.x; k < r; k += blockDim.x) cnt[(int64_t)blockIdx.x * r + k] = sc[k];
}

// CSC fill: thread k of the chunk's block walks the chunk's rows in order
__global__ void k_sp_fill_cols(const int64_t* rp, const int32_t* col, const float* val, int64_t n, int r,
                               const int64_t* base, int32_t* rowidx, float* cval) {
    const int64_t i0 = (int64_t)blockIdx.x * CHR, i1 = min(n, i0 + CHR);
    for (int k = threadIdx.x; k < r; k += blockDim.x) {
        int64_t pos = base[(int64_t)blockIdx.x * r + k];
        for (int64_t i = i0; i < i1; ++i)
            for (int64_t t = rp[i]; t < rp[i + 1]; ++t)
                if (col[t] == k) {
                    rowidx[pos] = (int32_t)i;
                    cval[pos] = val[t];
                    ++pos;
                }
    }
}

// dense n x r fp32 from the CSR (zeros elsewhere)
__global__ void k_sp_export(const int64_t* rp, const int32_t* col, const float* val, int64_t n, int r, float* dst) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float* d = dst + i * r;
    for (int k = 0; k < r; ++k) d[k] = 0.0f;
    for (int64_t t = rp[i]; t < rp[i + 1]; ++t) d[col[t]] = val[t];
}

__device__ __forceinline__ float4 ld4c(const float* p) { return *reinterpret_cast<const float4*>(p); }

__global__ void __launch_bounds__(256) k_sp_expand(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                   const float* __restrict__ val, const float* __restrict__ H, int op,
                                                   float* __restrict__ out, const float* __restrict__ Rv,
                                                   const float* __restrict__ Pv, int64_t n, int32_t Bp,
                                                   const ColState* __restrict__ st, const int* gate) {
    if (gate && *gate == 0) return;
    const int nq = Bp >> 2;
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t row = e / nq;
    if (row >= n) return;
    const int cq = 4 * (int)(e - row * nq);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t t = rp[row]; t < rp[row + 1]; ++t) {
        const float u = val[t];
        const float4 h = ld4c(H + (int64_t)col[t] * Bp + cq);
        acc.x = fmaf(u, h.x, acc.x);
        acc.y = fmaf(u, h.y, acc.y);
        acc.z = fmaf(u, h.z, acc.z);
        acc.w = fmaf(u, h.w, acc.w);
    }
    const int64_t o = row * Bp + cq;
    float4 v;
    if (op == EXP_SET_X) {
        v = acc;
    } else if (op == EXP_SUB_R) {
        v = ld4c(out + o);
        v.x -= acc.x; v.y -= acc.y; v.z -= acc.z; v.w -= acc.w;
    } else if (op == EXP_ADD_Q) {
        v = ld4c(out + o);
        v.x += acc.x; v.y += acc.y; v.z += acc.z; v.w += acc.w;
    } else {
        const float4 rr = ld4c(Rv + o), pp = ld4c(Pv + o);
        const float b0 = (float)st[cq].beta, b1 = (float)st[cq + 1].beta;
        const float b2 = (float)st[cq + 2].beta, b3 = (float)st[cq + 3].beta;
        // a served column that just took a new request drops r (p0 = U D U^T y + y)
        const bool f0 = st[cq].refill, f1 = st[cq + 1].refill, f2 = st[cq + 2].refill, f3 = st[cq + 3].refill;
        v.x = (f0 ? 0.0f : rr.x) + acc.x + (b0 == 0.0f ? 0.0f : b0 * pp.x);
        v.y = (f1 ? 0.0f : rr.y) + acc.y + (b1 == 0.0f ? 0.0f : b1 * pp.y);
        v.z = (f2 ? 0.0f : rr.z) + acc.z + (b2 == 0.0f ? 0.0f : b2 * pp.z);
        v.w = (f3 ? 0.0f : rr.w) + acc.w + (b3 == 0.0f ? 0.0f : b3 * pp.w);
    }
    *reinterpret_cast<float4*>(out + o) = v;
}

__global__ void __launch_bounds__(256) k_sp_reduce(const int64_t* __restrict__ cp, const int32_t* __restrict__ rowidx,
                                                   const float* __restrict__ cval, const float* __restrict__ V,
                                                   int32_t Bp, int r, int rpad, int nchunk, float* __restrict__ part,
                                                   const int* gate) {
    if (gate && *gate == 0) return;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= (int64_t)nchunk * rpad) return;
    const int c = (int)(w / rpad), k = (int)(w % rpad);
    int64_t a = 0, b = 0;
    if (k < r) {
        const int64_t s = cp[k], len = cp[k + 1] - s;
        a = s + len * c / nchunk;
        b = s + len * (c + 1) / nchunk;
    }
    float* dst = part + ((int64_t)c * rpad + k) * Bp;
    for (int g0 = 0; g0 < Bp; g0 += 128) {
        const int j = g0 + 4 * lane;
        if (j >= Bp) break;
        float4 acc0 = make_float4(0.f, 0.f, 0.f, 0.f), acc1 = acc0;
        int64_t t = a;
        for (; t + 1 < b; t += 2) {
            const float u0 = cval[t], u1 = cval[t + 1];
            const float4 v0 = ld4c(V + (int64_t)rowidx[t] * Bp + j);
            const float4 v1 = ld4c(V + (int64_t)rowidx[t + 1] * Bp + j);
            acc0.x = fmaf(u0, v0.x, acc0.x); acc0.y = fmaf(u0, v0.y, acc0.y);
            acc0.z = fmaf(u0, v0.z, acc0.z); acc0.w = fmaf(u0, v0.w, acc0.w);
            acc1.x = fmaf(u1, v1.x, acc1.x); acc1.y = fmaf(u1, v1.y, acc1.y);
            acc1.z = fmaf(u1, v1.z, acc1.z); acc1.w = fmaf(u1, v1.w, acc1.w);
        }
        if (t < b) {
            const float u0 = cval[t];
            const float4 v0 = ld4c(V + (int64_t)rowidx[t] * Bp + j);
            acc0.x = fmaf(u0, v0.x, acc0.x); acc0.y = fmaf(u0, v0.y, acc0.y);
            acc0.z = fmaf(u0, v0.z, acc0.z); acc0.w = fmaf(u0, v0.w, acc0.w);
        }
        *reinterpret_cast<float4*>(dst + j) =
            make_float4(acc0.x + acc1.x, acc0.y + acc1.y, acc0.z + acc1.z, acc0.w + acc1.w);
    }
}

}  // namespace

int lr_sparse_nchunk(hd_ctx* ctx, const hd_eig* e) {
    const int rpad = (e->r + 63) / 64 * 64;
    const int warps = ctx->num_sms * 64;
    return std::max(1, std::min(256, warps / std::max(rpad, 1)));
}

int lr_sparse_reduce(hd_ctx* ctx, const LowRank& lr, const float* V, int64_t n, int32_t Bp, const int* gate) {
    (void)n;
    const hd_eig* e = lr.e;
    const int64_t warps = (int64_t)lr.nchunk * lr.rpad;
    k_sp_reduce<<<ceil_div(warps * 32, 256), 256, 0, ctx->stream>>>(e->sp_cp, e->sp_row, e->sp_cval, V, Bp, e->r,
                                                                     lr.rpad, lr.nchunk, lr.part, gate);
    HD_CHECK_LAUNCH(ctx);
    return HD_OK;
}

int lr_sparse_expand(hd_ctx* ctx, const LowRank& lr, int op, float* out, const float* Rv, const float* Pv, int64_t n,
                     int32_t Bp, const ColState* st, const int* gate) {
    const hd_eig* e = lr.e;
    const int64_t thr = n * (Bp / 4);
    k_sp_expand<<<ceil_div(thr, 256), 256, 0, ctx->stream>>>(e->sp_rp, e->sp_col, e->sp_val, lr.H, op, out, Rv, Pv, n,
                                                              Bp, st, gate);
    HD_CHECK_LAUNCH(ctx);
    return HD_OK;
}

int hd_eig_sparse_export(hd_ctx* ctx, const hd_eig* e, float* dst) {
    k_sp_export<<<ceil_div(e->n, 256), 256, 0, ctx->stream>>>(e->sp_rp, e->sp_col, e->sp_val, e->n, e->r, dst);
    HD_CHECK_LAUNCH(ctx);
    return HD_OK;
}

extern "C" int hd_eig_sparsify(hd_ctx* ctx, const hd_eig* src, double sparsity, hd_eig** out) {
    if (!ctx || !src || !out || !(sparsity >= 0.0 && sparsity <= 1.0)) return HD_ERR_INVALID_ARG;
    if (src->sparse) return hd_fail(ctx, HD_ERR_INVALID_ARG, "eigenpairs are already sparse");
    if (src->r <= 0) return hd_fail(ctx, HD_ERR_INVALID_ARG, "r = 0");
    *out = nullptr;
    HD_CUDA(ctx, cudaSetDevice(ctx->device));
    const int64_t n = src->n;
    const int r = src->r;
    const int64_t total = n * r;
    // round half to even, as the product of the two doubles
    const int64_t drop = (int64_t)std::nearbyint(sparsity * (double)total);
    const int64_t keep = total - drop;
    const int grid = ctx->num_sms * 8;

    std::vector<void*> tmp;
    auto dalloc = [&](void** p, size_t bytes) -> int {
        if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
            cudaGetLastError();
            return hd_fail(ctx, HD_ERR_OOM, "sparsify: %zu bytes", bytes);
        }
        tmp.push_back(*p);
        return HD_OK;
    };
    auto release = [&]() {
        cudaStreamSynchronize(ctx->stream);
        for (void* p : tmp) cudaFree(p);
        tmp.clear();
    };
    int rc = HD_OK;
#define SP_TRY(x)          \
    do {                   \
        if ((rc = (x))) {  \
            release();     \
            return rc;     \
        }                  \
    } while (0)
#define SP_CUDA(x) SP_TRY(hd_check_cuda(ctx, (x), #x, __FILE__, __LINE__))

    // ---- threshold key T and the number m of entries equal to T that stay
    uint32_t T = 0xffffffffu;
    int64_t m = 0;
    if (keep > 0) {
        unsigned long long* hist;
        SP_TRY(dalloc((void**)&hist, 256 * 8));
        std::vector<unsigned long long> hh(256);
        uint32_t prefix = 0, mask = 0;
        int64_t need = keep;  // largest keys still to place at or below the current prefix
        for (int shift = 24; shift >= 0; shift -= 8) {
            SP_CUDA(cudaMemsetAsync(hist, 0, 256 * 8, ctx->stream));
            k_sp_hist<<<grid, 256, 0, ctx->stream>>>(src->U, src->scale, src->storage, src->ldu, n, r, prefix, mask,
                                                     shift, hist);
            SP_TRY(hd_check_launch(ctx, __FILE__, __LINE__));
            SP_CUDA(cudaMemcpyAsync(hh.data(), hist, 256 * 8, cudaMemcpyDeviceToHost, ctx->stream));
            SP_CUDA(cudaStreamSynchronize(ctx->stream));
            int d = 255;
            for (; d >= 0; --d) {
                if ((int64_t)hh[d] >= need) break;
                need -= (int64_t)hh[d];
            }
            if (d < 0) {
                release();
                return hd_fail(ctx, HD_ERR_CUDA, "sparsify: radix select lost count");
            }
            prefix |= (uint32_t)d << shift;
            mask |= 255u << shift;
        }
        T = prefix;
        m = need;
    }

    // ---- row counts, tie ranks and row pointers
    int32_t *gt, *tie;
    SP_TRY(dalloc((void**)&gt, n * 4));
    SP_TRY(dalloc((void**)&tie, n * 4));
    std::vector<int32_t> hg(n, 0), ht(n, 0);
    if (keep > 0) {
        k_sp_rowcount<<<ceil_div(n * 32, 256), 256, 0, ctx->stream>>>(src->U, src->scale, src->storage, src->ldu, n, r,
                                                                      T, gt, tie);
        SP_TRY(hd_check_launch(ctx, __FILE__, __LINE__));
        SP_CUDA(cudaMemcpyAsync(hg.data(), gt, n * 4, cudaMemcpyDeviceToHost, ctx->stream));
        SP_CUDA(cudaMemcpyAsync(ht.data(), tie, n * 4, cudaMemcpyDeviceToHost, ctx->stream));
        SP_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    std::vector<int64_t> rp(n + 1), tb(n);
    int64_t tacc = 0;
    rp[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        tb[i] = tacc;
        const int64_t kt = std::max<int64_t>(0, std::min<int64_t>(ht[i], m - tacc));
        tacc += ht[i];
        rp[i + 1] = rp[i] + hg[i] + kt;
    }
    const int64_t nnz = rp[n];
    if (nnz != keep) {
        release();
        return hd_fail(ctx, HD_ERR_CUDA, "sparsify: kept %lld entries, expected %lld", (long long)nnz, (long long)keep);
    }

    hd_eig* e = new hd_eig();
    e->n = n;
    e->r = r;
    e->ldu = src->ldu;
    e->storage = src->storage;
    e->sparse = true;
    e->nnz = nnz;
    e->lambda_h = src->lambda_h;
    auto ealloc = [&](void** p, size_t bytes) -> int {
        if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) {
            cudaGetLastError();
            return hd_fail(ctx, HD_ERR_OOM, "sparse eigenpairs: %zu bytes", bytes);
        }
        return HD_OK;
    };
    int ea = ealloc((void**)&e->lambda_d, (size_t)r * 8);
    if (!ea) ea = ealloc((void**)&e->sp_rp, (size_t)(n + 1) * 8);
    if (!ea) ea = ealloc((void**)&e->sp_col, (size_t)nnz * 4);
    if (!ea) ea = ealloc((void**)&e->sp_val, (size_t)nnz * 4);
    if (!ea) ea = ealloc((void**)&e->sp_cp, (size_t)(r + 1) * 8);
    if (!ea) ea = ealloc((void**)&e->sp_row, (size_t)nnz * 4);
    if (!ea) ea = ealloc((void**)&e->sp_cval, (size_t)nnz * 4);
    if (ea) {
        hd_eig_destroy(e);
        release();
        return ea;
    }
    auto fail_e = [&](int code) {
        hd_eig_destroy(e);
        release();
        return code;
    };
#define SP_E(x)                                                              \
    do {                                                                     \
        int c_ = hd_check_cuda(ctx, (x), #x, __FILE__, __LINE__);            \
        if (c_) return fail_e(c_);                                           \
    } while (0)
    SP_E(cudaMemcpyAsync(e->lambda_d, src->lambda_d, (size_t)r * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    SP_E(cudaMemcpyAsync(e->sp_rp, rp.data(), (size_t)(n + 1) * 8, cudaMemcpyHostToDevice, ctx->stream));
    int64_t* tb_d;
    if ((rc = dalloc((void**)&tb_d, (size_t)n * 8))) return fail_e(rc);
    SP_E(cudaMemcpyAsync(tb_d, tb.data(), (size_t)n * 8, cudaMemcpyHostToDevice, ctx->stream));
    if (nnz > 0) {
        k_sp_fill_rows<<<ceil_div(n * 32, 256), 256, 0, ctx->stream>>>(src->U, src->scale, src->storage, src->ldu, n,
                                                                       r, T, m, tb_d, e->sp_rp, e->sp_col, e->sp_val);
        if ((rc = hd_check_launch(ctx, __FILE__, __LINE__))) return fail_e(rc);
    }
    // ---- CSC: per-chunk column counts -> offsets -> ordered fill
    const int64_t nch = (n + CHR - 1) / CHR;
    int32_t* cnt;
    int64_t* base_d;
    if ((rc = dalloc((void**)&cnt, (size_t)nch * r * 4))) return fail_e(rc);
    if ((rc = dalloc((void**)&base_d, (size_t)nch * r * 8))) return fail_e(rc);
    std::vector<int32_t> hc((size_t)nch * r, 0);
    if (nnz > 0) {
        k_sp_colcount<<<(unsigned)nch, 256, (size_t)r * 4, ctx->stream>>>(e->sp_rp, e->sp_col, n, r, cnt);
        if ((rc = hd_check_launch(ctx, __FILE__, __LINE__))) return fail_e(rc);
        SP_E(cudaMemcpyAsync(hc.data(), cnt, (size_t)nch * r * 4, cudaMemcpyDeviceToHost, ctx->stream));
        SP_E(cudaStreamSynchronize(ctx->stream));
    }
    std::vector<int64_t> cp(r + 1, 0), base((size_t)nch * r);
    for (int k = 0; k < r; ++k) {
        int64_t s = 0;
        for (int64_t c = 0; c < nch; ++c) s += hc[(size_t)c * r + k];
        cp[k + 1] = cp[k] + s;
    }
    for (int k = 0; k < r; ++k) {
        int64_t at = cp[k];
        for (int64_t c = 0; c < nch; ++c) {
            base[(size_t)c * r + k] = at;
            at += hc[(size_t)c * r + k];
        }
    }
    SP_E(cudaMemcpyAsync(e->sp_cp, cp.data(), (size_t)(r + 1) * 8, cudaMemcpyHostToDevice, ctx->stream));
    SP_E(cudaMemcpyAsync(base_d, base.data(), (size_t)nch * r * 8, cudaMemcpyHostToDevice, ctx->stream));
    if (nnz > 0) {
        const int thr = std::min(1024, (r + 31) / 32 * 32);
        k_sp_fill_cols<<<(unsigned)nch, thr, 0, ctx->stream>>>(e->sp_rp, e->sp_col, e->sp_val, n, r, base_d,
                                                               e->sp_row, e->sp_cval);
        if ((rc = hd_check_launch(ctx, __FILE__, __LINE__))) return fail_e(rc);
    }
    SP_E(cudaStreamSynchronize(ctx->stream));
    release();
    *out = e;
    return HD_OK;
#undef SP_E
#undef SP_CUDA
#undef SP_TRY
}

extern "C" int hd_eig_nnz(const hd_eig* e, int64_t* nnz) {
    if (!e || !nnz) return HD_ERR_INVALID_ARG;
    *nnz = e->sparse ? e->nnz : e->n * (int64_t)e->r;
    return HD_OK;
}
