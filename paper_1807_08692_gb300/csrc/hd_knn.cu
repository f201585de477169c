// k-NN search and graph construction (Sec. 3; Sec. 5.1).
//
// Similarities s = q^T x are accumulated in fp32: bf16 descriptors on the 5th
// generation tensor cores (tcgen05.mma, TMA-fed shared memory, accumulators in
// TMEM) with the per-row top-k selection fused into the TMEM epilogue, so the
// n x n similarity matrix never leaves the SM; fp32 descriptors on CUDA cores
// (exact fp32 products).  Neighbour lists are ordered by decreasing s, ties to
// the smaller database index; self is excluded when the query set is the
// database.  The graph keeps weight max(s, 0)^gamma, symmetrised (union or
// mutual), then W = D^-1/2 A D^-1/2.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include <cudaTypedefs.h>

#include "hd_internal.cuh"
#include "tc.cuh"

int hd_graph_alloc_internal(hd_ctx* ctx, int64_t n, int64_t nnz, hd_graph** out);
void hd_graph_free_internal(hd_graph* g);

// ------------------------------------------------------------------ tensor maps
int hd_make_tmap_2d(CUtensorMap* map, const void* base, int elem_bytes, uint64_t rows, uint64_t cols,
                    uint64_t ld_elems, uint32_t box_rows, uint32_t box_cols, int swizzle128) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return -1;
        encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    CUtensorMapDataType dt = elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                             : elem_bytes == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                                               : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    cuuint64_t gdim[2] = {cols, rows};
    cuuint64_t gstride[1] = {ld_elems * (uint64_t)elem_bytes};
    cuuint32_t box[2] = {box_cols, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(map, dt, 2, const_cast<void*>(base), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -2;
}

// ------------------------------------------------------------------ list insertion
// Insert (s, id) into a row's list kept sorted by (-s, id).  Returns new k-th score.
__device__ __noinline__ float list_insert_ordered(float* ls, int32_t* li, int k, float s, int32_t id) {
    int p = k - 1;
    while (p > 0 && (ls[p - 1] < s || (ls[p - 1] == s && li[p - 1] > id))) {
        ls[p] = ls[p - 1];
        li[p] = li[p - 1];
        --p;
    }
    ls[p] = s;
    li[p] = id;
    return ls[k - 1];
}

// ------------------------------------------------------------------ fp32 CUDA-core kNN
namespace {
constexpr int FB = 64;   // queries and database rows per tile
constexpr int FK = 16;   // depth chunk
constexpr int KMAX = 64;
}

__global__ void __launch_bounds__(256) k_knn_f32(const float* __restrict__ X, int64_t n, int d,
                                                 const float* __restrict__ Q, int64_t nq, int k, int excl,
                                                 int32_t* __restrict__ idx_out, float* __restrict__ sim_out) {
    __shared__ float As[FK][FB + 4];
    __shared__ float Bs[FK][FB + 4];
    __shared__ float ls[FB][KMAX];
    __shared__ int32_t li[FB][KMAX];
    __shared__ float cs[FB][FB];
    __shared__ int32_t cidx[FB][FB];
    __shared__ int cnt[FB];
    __shared__ float tau[FB];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t q0 = (int64_t)blockIdx.x * FB;
    for (int t = tid; t < FB * KMAX; t += 256) {
        ls[t / KMAX][t % KMAX] = -INFINITY;
        li[t / KMAX][t % KMAX] = -1;
    }
    if (tid < FB) {
        cnt[tid] = 0;
        tau[tid] = -INFINITY;
    }
    __syncthreads();
    for (int64_t t0 = 0; t0 < n; t0 += FB) {
        float acc[4][4] = {};
        for (int kc = 0; kc < d; kc += FK) {
            for (int e = tid; e < FB * FK; e += 256) {
                int r = e / FK, c = e % FK;
                int64_t qr = q0 + r, xr = t0 + r;
                As[c][r] = (qr < nq && kc + c < d) ? Q[qr * d + kc + c] : 0.0f;
                Bs[c][r] = (xr < n && kc + c < d) ? X[xr * d + kc + c] : 0.0f;
            }
            __syncthreads();
#pragma unroll
            for (int c = 0; c < FK; ++c) {
                float a[4], b[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    a[i] = As[c][ty * 4 + i];
                    b[i] = Bs[c][tx * 4 + i];
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int r = ty * 4 + i;
            int64_t qr = q0 + r;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                int64_t id = t0 + tx * 4 + j;
                float s = acc[i][j];
                if (qr < nq && id < n && !(excl && id == qr) && s > tau[r]) {
                    int p = atomicAdd(&cnt[r], 1);
                    cs[r][p] = s;
                    cidx[r][p] = (int32_t)id;
                }
            }
        }
        __syncthreads();
        if (tid < FB) {
            int r = tid;
            float th = tau[r];
            for (int c = 0; c < cnt[r]; ++c) {
                float s = cs[r][c];
                int32_t id = cidx[r][c];
                if (s > ls[r][k - 1] || (s == ls[r][k - 1] && id < li[r][k - 1]))
                    th = list_insert_ordered(&ls[r][0], &li[r][0], k, s, id);
            }
            tau[r] = th;
            cnt[r] = 0;
        }
        __syncthreads();
    }
    for (int t = tid; t < FB * k; t += 256) {
        int r = t / k, c = t % k;
        int64_t qr = q0 + r;
        if (qr < nq) {
            idx_out[qr * k + c] = li[r][c];
            sim_out[qr * k + c] = ls[r][c];
        }
    }
}

// ------------------------------------------------------------------ bf16 tcgen05 kNN
namespace knntc {
constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;   // 16 KB
constexpr int B_BYTES = BN * BK * 2;   // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr int THREADS = 192;
}  // namespace knntc

__global__ void __launch_bounds__(knntc::THREADS, 1)
    k_knn_tc(const __grid_constant__ CUtensorMap tmQ, const __grid_constant__ CUtensorMap tmX, int64_t n, int d,
             int64_t nq, int k, int excl, int32_t* __restrict__ idx_out, float* __restrict__ sim_out,
             int* __restrict__ err) {
    using namespace knntc;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* acc_full = empty + STAGES;
    uint64_t* acc_empty = acc_full + 2;
    uint64_t* drain = acc_empty + 2;
    uint32_t* tmem_slot = (uint32_t*)(drain + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nkb = (d + BK - 1) / BK;
    const int ntile = (int)((n + BN - 1) / BN);
    const int nwork = (int)((nq + BM - 1) / BM);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&acc_full[b], 1);
            tc::mbar_init(&acc_empty[b], 128);
        }
        tc::mbar_init(drain, 1);
        *abort_flag = 0;
        tc::fence_barrier_init();
    }
    if (warp == 1) tc::tmem_alloc<512>(tmem_slot);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            tc::prefetch_tmap(&tmQ);
            tc::prefetch_tmap(&tmX);
            uint32_t it = 0;
            bool ok = true;
            for (int w = blockIdx.x; w < nwork && ok; w += gridDim.x)
                for (int t = 0; t < ntile && ok; ++t)
                    for (int kb = 0; kb < nkb; ++kb, ++it) {
                        int s = it % STAGES;
                        uint32_t ph = (it / STAGES) & 1;
                        if (!tc::mbar_wait(&empty[s], ph ^ 1, abort_flag)) {
                            ok = false;
                            break;
                        }
                        uint8_t* a = smem + s * STAGE_BYTES;
                        tc::mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                        tc::tma_load_2d(a, &tmQ, &full[s], kb * BK, w * BM);
                        tc::tma_load_2d(a + A_BYTES, &tmX, &full[s], kb * BK, t * BN);
                    }
            if (!ok) {
                *abort_flag = 1;
                atomicExch(err, 1);
            }
            // drain: the latest load issued into each stage must land before the CTA may exit
            for (uint32_t j = 0; j < (uint32_t)STAGES && j < it; ++j) {
                uint32_t last = it - 1 - j;
                tc::mbar_wait(&full[last % STAGES], (last / STAGES) & 1, nullptr, 200000000ull);
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t IDESC = tc::idesc_bf16(BM, BN, 0, 0);
            uint32_t it = 0, tcount = 0;
            bool ok = true;
            for (int w = blockIdx.x; w < nwork && ok; w += gridDim.x)
                for (int t = 0; t < ntile && ok; ++t, ++tcount) {
                    int ab = tcount & 1;
                    uint32_t aph = (tcount >> 1) & 1;
                    if (!tc::mbar_wait(&acc_empty[ab], aph ^ 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    uint32_t dt = tmem + ab * BN;
                    for (int kb = 0; kb < nkb; ++kb, ++it) {
                        int s = it % STAGES;
                        uint32_t ph = (it / STAGES) & 1;
                        if (!tc::mbar_wait(&full[s], ph, abort_flag)) {
                            ok = false;
                            break;
                        }
                        tc::fence_after_sync();
                        uint32_t a = tc::smem_u32(smem + s * STAGE_BYTES);
                        uint32_t b = a + A_BYTES;
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk) {
                            uint64_t ad = tc::smem_desc(a + kk * 32, 16, 1024, tc::SWIZZLE_128B);
                            uint64_t bd = tc::smem_desc(b + kk * 32, 16, 1024, tc::SWIZZLE_128B);
                            tc::mma_bf16(dt, ad, bd, IDESC, (kb | kk) ? 1u : 0u);
                        }
                        tc::mma_commit(&empty[s]);
                    }
                    if (ok) tc::mma_commit(&acc_full[ab]);
                }
            if (!ok) {
                *abort_flag = 1;
                atomicExch(err, 2);
                // wait for every MMA this thread issued before TMEM is released
                tc::mma_commit(drain);
                tc::mbar_wait(drain, 0, nullptr, 200000000ull);
            }
        }
    } else {
        // ---------------- epilogue: warps 2..5, one query row per thread
        const int quarter = warp & 3;
        const int rloc = quarter * 32 + lane;
        uint32_t tcount = 0;
        bool ok = true;
        for (int w = blockIdx.x; w < nwork && ok; w += gridDim.x) {
            const int64_t row = (int64_t)w * BM + rloc;
            const bool live = row < nq;
            float* ls = sim_out + (live ? row : 0) * k;
            int32_t* li = idx_out + (live ? row : 0) * k;
            if (live)
                for (int c = 0; c < k; ++c) {
                    ls[c] = -INFINITY;
                    li[c] = -1;
                }
            float tau = -INFINITY;
            for (int t = 0; t < ntile; ++t, ++tcount) {
                int ab = tcount & 1;
                uint32_t aph = (tcount >> 1) & 1;
                if (!tc::mbar_wait(&acc_full[ab], aph, abort_flag)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                for (int c = 0; c < BN / 32; ++c) {
                    float v[32];
                    tc::tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + ab * BN + c * 32, v);
                    tc::tmem_ld_wait();
                    if (live) {
                        const int64_t base = (int64_t)t * BN + c * 32;
#pragma unroll
                        for (int i = 0; i < 32; ++i) {
                            const int64_t id = base + i;
                            if (v[i] > tau && id < n && !(excl && id == row))
                                tau = list_insert_ordered(ls, li, k, v[i], (int32_t)id);
                        }
                    }
                }
                tc::fence_before_sync();
                tc::mbar_arrive(&acc_empty[ab]);
            }
        }
        if (!ok) {
            *abort_flag = 1;
            atomicExch(err, 3);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc<512>(tmem);
    }
}

int hd_knn_impl(hd_ctx* ctx, const void* Xd, int64_t n, int32_t d, int dtype, const void* Qd, int64_t nq, int32_t k,
                int exclude_self, int32_t* idx_d, float* sim_d) {
    if (k < 1 || k > KMAX) return hd_fail(ctx, HD_ERR_INVALID_ARG, "k=%d outside [1, %d]", k, KMAX);
    if (nq <= 0 || n <= 0) return HD_OK;
    if (dtype == HD_F32) {
        k_knn_f32<<<ceil_div(nq, FB), 256, 0, ctx->stream>>>((const float*)Xd, n, d, (const float*)Qd, nq, k,
                                                             exclude_self, idx_d, sim_d);
        HD_CHECK_LAUNCH(ctx);
        return HD_OK;
    }
    if (dtype != HD_BF16) return hd_fail(ctx, HD_ERR_INVALID_ARG, "dtype %d", dtype);
    if (d % 8) return hd_fail(ctx, HD_ERR_INVALID_ARG, "bf16 descriptors need d %% 8 == 0 (d=%d)", d);
    using namespace knntc;
    CUtensorMap tq, tx;
    if (hd_make_tmap_2d(&tq, Qd, 2, nq, d, d, BM, BK, 1) || hd_make_tmap_2d(&tx, Xd, 2, n, d, d, BN, BK, 1))
        return hd_fail(ctx, HD_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    static uint64_t attr = 0;
    if (hd_first_on_device(attr, ctx->device)) {
        HD_CUDA(ctx, cudaFuncSetAttribute(k_knn_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    }
    int nwork = ceil_div(nq, BM);
    int grid = nwork < ctx->num_sms ? nwork : ctx->num_sms;
    HD_CUDA(ctx, cudaMemsetAsync(ctx->d_flags + 1, 0, sizeof(int), ctx->stream));
    HD_PROF(ctx, "knn");
    k_knn_tc<<<grid, THREADS, SMEM_BYTES, ctx->stream>>>(tq, tx, n, d, nq, k, exclude_self, idx_d, sim_d,
                                                         ctx->d_flags + 1);
    HD_CHECK_LAUNCH(ctx);
    HD_CUDA(ctx, cudaMemcpyAsync(ctx->h_poll + 1, ctx->d_flags + 1, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->h_poll[1]) return hd_fail(ctx, HD_ERR_TIMEOUT, "k-NN tensor-core pipeline wait timed out (%d)", ctx->h_poll[1]);
    return HD_OK;
}

// ------------------------------------------------------------------ symmetrisation
__device__ __forceinline__ float edge_weight(float s, float gamma) {
    float m = fmaxf(s, 0.0f);
    return gamma == 3.0f ? m * m * m : powf(m, gamma);
}

// For each directed entry i -> j: is i in j's list (reciprocal), and j's weight for it.
__global__ void k_recip(const int32_t* idx, const float* sim, int64_t n, int k, float gamma, int8_t* recip,
                        float* wrev, int32_t* extra) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * k) return;
    int64_t i = e / k;
    int32_t j = idx[e];
    float w = j >= 0 ? edge_weight(sim[e], gamma) : 0.0f;
    int8_t found = 0;
    float wr = 0.0f;
    if (j >= 0 && w > 0.0f) {
        for (int u = 0; u < k; ++u)
            if (idx[(int64_t)j * k + u] == (int32_t)i) {
                float w2 = edge_weight(sim[(int64_t)j * k + u], gamma);
                if (w2 > 0.0f) {
                    found = 1;
                    wr = w2;
                }
                break;
            }
        if (!found) atomicAdd(&extra[j], 1);
    }
    recip[e] = found;
    wrev[e] = wr;
}

__global__ void k_rowlen(const int32_t* idx, const float* sim, const int8_t* recip, const int32_t* extra, int64_t n,
                         int k, float gamma, int sym, int32_t* len, int32_t* own) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c = 0;
    for (int u = 0; u < k; ++u) {
        int64_t e = i * k + u;
        bool valid = idx[e] >= 0 && edge_weight(sim[e], gamma) > 0.0f;
        if (valid && (sym == HD_SYM_UNION || recip[e])) ++c;
    }
    own[i] = c;
    len[i] = c + (sym == HD_SYM_UNION ? extra[i] : 0);
}

__global__ void k_fill(const int32_t* idx, const float* sim, const int8_t* recip, const float* wrev,
                       const int32_t* row_ptr, const int32_t* own, int32_t* cursor, int64_t n, int k, float gamma,
                       int sym, int32_t* col, float* val) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t pos = row_ptr[i];
    for (int u = 0; u < k; ++u) {
        int64_t e = i * k + u;
        int32_t j = idx[e];
        float w = j >= 0 ? edge_weight(sim[e], gamma) : 0.0f;
        if (!(w > 0.0f)) continue;
        if (recip[e]) {
            col[pos] = j;
            val[pos] = sym == HD_SYM_UNION ? fmaxf(w, wrev[e]) : fminf(w, wrev[e]);
            ++pos;
        } else if (sym == HD_SYM_UNION) {
            col[pos] = j;
            val[pos] = w;
            ++pos;
            int32_t q = row_ptr[j] + own[j] + atomicAdd(&cursor[j], 1);
            col[q] = (int32_t)i;
            val[q] = w;
        }
    }
}

__global__ void k_sort_rows2(const int32_t* rp, int32_t* col, float* val, int64_t n) {
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

int hd_graph_from_lists(hd_ctx* ctx, int64_t n, int32_t k, const int32_t* idx_d, const float* sim_d, float gamma,
                        int sym, hd_graph** out) {
    int8_t* recip;
    float* wrev;
    int32_t *extra, *len, *own, *cursor;
    size_t nk = (size_t)n * k;
    HD_CUDA(ctx, cudaMalloc(&recip, nk));
    HD_CUDA(ctx, cudaMalloc(&wrev, nk * 4));
    HD_CUDA(ctx, cudaMalloc(&extra, n * 4));
    HD_CUDA(ctx, cudaMalloc(&len, n * 4));
    HD_CUDA(ctx, cudaMalloc(&own, n * 4));
    HD_CUDA(ctx, cudaMalloc(&cursor, n * 4));
    HD_CUDA(ctx, cudaMemsetAsync(extra, 0, n * 4, ctx->stream));
    HD_CUDA(ctx, cudaMemsetAsync(cursor, 0, n * 4, ctx->stream));
    k_recip<<<ceil_div(nk, 256), 256, 0, ctx->stream>>>(idx_d, sim_d, n, k, gamma, recip, wrev, extra);
    HD_CHECK_LAUNCH(ctx);
    k_rowlen<<<ceil_div(n, 256), 256, 0, ctx->stream>>>(idx_d, sim_d, recip, extra, n, k, gamma, sym, len, own);
    HD_CHECK_LAUNCH(ctx);
    std::vector<int32_t> h_len(n), h_ptr(n + 1);
    HD_CUDA(ctx, cudaMemcpyAsync(h_len.data(), len, n * 4, cudaMemcpyDeviceToHost, ctx->stream));
    HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    int64_t acc = 0;
    for (int64_t i = 0; i < n; ++i) {
        h_ptr[i] = (int32_t)acc;
        acc += h_len[i];
    }
    h_ptr[n] = (int32_t)acc;
    if (acc >= (1ll << 31)) return hd_fail(ctx, HD_ERR_INVALID_ARG, "graph too large: nnz=%lld", (long long)acc);
    hd_graph* g;
    int rc = hd_graph_alloc_internal(ctx, n, acc, &g);
    if (rc) return rc;
    HD_CUDA(ctx, cudaMemcpyAsync(g->row_ptr, h_ptr.data(), (n + 1) * 4, cudaMemcpyHostToDevice, ctx->stream));
    k_fill<<<ceil_div(n, 256), 256, 0, ctx->stream>>>(idx_d, sim_d, recip, wrev, g->row_ptr, own, cursor, n, k, gamma,
                                                      sym, g->col, g->val);
    HD_CHECK_LAUNCH(ctx);
    k_sort_rows2<<<ceil_div(n, 128), 128, 0, ctx->stream>>>(g->row_ptr, g->col, g->val, n);
    HD_CHECK_LAUNCH(ctx);
    rc = hd_normalize_graph(ctx, g);
    HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(recip);
    cudaFree(wrev);
    cudaFree(extra);
    cudaFree(len);
    cudaFree(own);
    cudaFree(cursor);
    if (rc) {
        hd_graph_free_internal(g);
        return rc;
    }
    *out = g;
    return HD_OK;
}

// ------------------------------------------------------------------ C ABI
static int stage_matrix(hd_ctx* ctx, const void* p, size_t bytes, void** owned, const void** dev) {
    *owned = nullptr;
    if (hd_is_device_ptr(p)) {
        *dev = p;
        return HD_OK;
    }
    HD_CUDA(ctx, cudaMalloc(owned, bytes));
    HD_CUDA(ctx, cudaMemcpyAsync(*owned, p, bytes, cudaMemcpyHostToDevice, ctx->stream));
    *dev = *owned;
    return HD_OK;
}

extern "C" {

int hd_knn(hd_ctx* ctx, const void* X, int64_t n, int32_t d, int dtype, const void* Q, int64_t nq, int32_t k,
           int exclude_self, int32_t* idx_out, float* sim_out) {
    if (!ctx || !X || !Q || !idx_out || !sim_out || n <= 0 || nq <= 0 || d <= 0) return HD_ERR_INVALID_ARG;
    if (dtype != HD_F32 && dtype != HD_BF16) return hd_fail(ctx, HD_ERR_INVALID_ARG, "dtype %d", dtype);
    HD_CUDA(ctx, cudaSetDevice(ctx->device));
    size_t es = dtype == HD_F32 ? 4 : 2;
    void *ox, *oq;
    const void *xd, *qd;
    int rc = stage_matrix(ctx, X, (size_t)n * d * es, &ox, &xd);
    if (!rc) rc = stage_matrix(ctx, Q, (size_t)nq * d * es, &oq, &qd);
    if (rc) return rc;
    bool dev_out = hd_is_device_ptr(idx_out) && hd_is_device_ptr(sim_out);
    int32_t* idd = idx_out;
    float* sdd = sim_out;
    if (!dev_out) {
        HD_CUDA(ctx, cudaMalloc(&idd, (size_t)nq * k * 4));
        HD_CUDA(ctx, cudaMalloc(&sdd, (size_t)nq * k * 4));
    }
    rc = hd_knn_impl(ctx, xd, n, d, dtype, qd, nq, k, exclude_self, idd, sdd);
    if (!rc && !dev_out) {
        HD_CUDA(ctx, cudaMemcpyAsync(idx_out, idd, (size_t)nq * k * 4, cudaMemcpyDeviceToHost, ctx->stream));
        HD_CUDA(ctx, cudaMemcpyAsync(sim_out, sdd, (size_t)nq * k * 4, cudaMemcpyDeviceToHost, ctx->stream));
    }
    HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (!dev_out) {
        cudaFree(idd);
        cudaFree(sdd);
    }
    if (ox) cudaFree(ox);
    if (oq) cudaFree(oq);
    return rc;
}

int hd_build_graph(hd_ctx* ctx, const void* X, int64_t n, int32_t d, int dtype, int32_t k, float gamma, int sym,
                   hd_graph** out) {
    if (!ctx || !X || !out || n <= 1 || d <= 0 || k < 1 || k >= n) return HD_ERR_INVALID_ARG;
    if (sym != HD_SYM_UNION && sym != HD_SYM_MUTUAL) return hd_fail(ctx, HD_ERR_INVALID_ARG, "sym %d", sym);
    if (dtype != HD_F32 && dtype != HD_BF16) return hd_fail(ctx, HD_ERR_INVALID_ARG, "dtype %d", dtype);
    *out = nullptr;
    HD_CUDA(ctx, cudaSetDevice(ctx->device));
    size_t es = dtype == HD_F32 ? 4 : 2;
    void* ox;
    const void* xd;
    int rc = stage_matrix(ctx, X, (size_t)n * d * es, &ox, &xd);
    if (rc) return rc;
    int32_t* idx;
    float* sim;
    HD_CUDA(ctx, cudaMalloc(&idx, (size_t)n * k * 4));
    HD_CUDA(ctx, cudaMalloc(&sim, (size_t)n * k * 4));
    rc = hd_knn_impl(ctx, xd, n, d, dtype, xd, n, k, 1, idx, sim);
    if (!rc) rc = hd_graph_from_lists(ctx, n, k, idx, sim, gamma, sym, out);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(idx);
    cudaFree(sim);
    if (ox) cudaFree(ox);
    return rc;
}

int hd_observe(hd_ctx* ctx, const void* X, int64_t n, int32_t d, int dtype, const void* Q, int32_t nq, int32_t k_y,
               float gamma, int32_t* y_ptr, int32_t* y_idx, float* y_val) {
    if (!ctx || !X || !Q || !y_ptr || !y_idx || !y_val || nq <= 0 || k_y < 1 || k_y > n) return HD_ERR_INVALID_ARG;
    std::vector<int32_t> li((size_t)nq * k_y);
    std::vector<float> ls((size_t)nq * k_y);
    int rc = hd_knn(ctx, X, n, d, dtype, Q, nq, k_y, 0, li.data(), ls.data());
    if (rc) return rc;
    std::vector<int32_t> ptr(nq + 1), ids;
    std::vector<float> vals;
    ptr[0] = 0;
    for (int32_t q = 0; q < nq; ++q) {
        std::vector<std::pair<int32_t, float>> row;
        for (int u = 0; u < k_y; ++u) {
            int32_t j = li[(size_t)q * k_y + u];
            float s = ls[(size_t)q * k_y + u];
            float m = s > 0.0f ? s : 0.0f;
            float w = gamma == 3.0f ? m * m * m : powf(m, gamma);
            if (j >= 0 && w > 0.0f) row.push_back({j, w});
        }
        std::sort(row.begin(), row.end(), [](auto& a, auto& b) { return a.first < b.first; });
        for (auto& e : row) {
            ids.push_back(e.first);
            vals.push_back(e.second);
        }
        ptr[q + 1] = (int32_t)ids.size();
    }
    auto put = [&](void* dst, const void* src, size_t bytes) -> int {
        if (!bytes) return HD_OK;
        cudaMemcpyKind kd = hd_is_device_ptr(dst) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
        HD_CUDA(ctx, cudaMemcpy(dst, src, bytes, kd));
        return HD_OK;
    };
    if ((rc = put(y_ptr, ptr.data(), ptr.size() * 4))) return rc;
    if ((rc = put(y_idx, ids.data(), ids.size() * 4))) return rc;
    if ((rc = put(y_val, vals.data(), vals.size() * 4))) return rc;
    return HD_OK;
}

}  // extern "C"
