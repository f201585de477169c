// Ranking by decreasing score (Sec. 3): per-column top-K of an n x B score block.
//
// The usual path is the sampled-threshold one below (one pass over the scores
// collects the candidates above a threshold drawn from a sample, and only the
// candidates are selected and sorted).  The exact fallback, and the path of the
// allocation-free entry point, is a radix select over the whole column:
// per column j the K_j-th largest score is found by a most-significant-digit
// radix select over the 32-bit order-preserving key of each float (4 passes of
// 8 bits, histograms in shared memory).  If scores tie at the boundary, a
// second radix select over the inverted row ids picks the smallest ids among
// the tied scores, so the selected set is exactly the first K of the order
// (score descending, id ascending).  The K survivors are then sorted per column
// with a bitonic sort on (key, ~id).
#include <algorithm>
#include <atomic>
#include <vector>

#include "hd_internal.cuh"

struct SelState {
    uint32_t prefix;   // digits decided so far (keys), then (~ids) in the tie phase
    uint32_t prefix2;
    int32_t k_rem;     // how many still to take among those matching the prefix
    int32_t greater;   // taken: key > threshold
    int32_t eq;        // number of elements equal to the key threshold
    int32_t K;
    int32_t tie;       // 1 when the id phase is needed
    int32_t count;     // collected so far
};

constexpr int CG = 64;  // columns per histogram block

__global__ void k_pool(const float* X, int64_t n_img, int32_t B, int32_t ldx, int32_t pool, float* Y) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_img * B) return;
    int64_t i = e / B;
    int j = (int)(e % B);
    float s = 0.0f;
    for (int t = 0; t < pool; ++t) s += X[(i * pool + t) * ldx + j];
    Y[i * B + j] = s;
}

__global__ void k_sel_init(SelState* st, const int32_t* K, int32_t B, int64_t n) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= B) return;
    SelState s;
    s.prefix = 0;
    s.prefix2 = 0;
    s.K = (int32_t)((int64_t)K[j] < n ? (int64_t)K[j] : n);
    s.k_rem = s.K;
    s.greater = 0;
    s.eq = 0;
    s.tie = 0;
    s.count = 0;
    st[j] = s;
}

// Histogram of digit `shift` among elements whose higher digits match the prefix.
// phase 0: keys of scores; phase 1: ~id among elements whose key equals the threshold.
__global__ void __launch_bounds__(256) k_hist(const float* X, int64_t n, int32_t B, int32_t ld, const SelState* st,
                                              int phase, int shift, uint32_t* hist) {
    extern __shared__ uint32_t h[];  // [cg][256]
    const int c0 = blockIdx.y * CG;
    const int cg = min(CG, B - c0);
    for (int t = threadIdx.x; t < cg * 256; t += blockDim.x) h[t] = 0;
    __syncthreads();
    const uint32_t hi_mask = shift == 24 ? 0u : (0xFFFFFFFFu << (shift + 8));
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * cg; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / cg;
        const int jl = (int)(e % cg);
        const int j = c0 + jl;
        const SelState& s = st[j];
        if (s.K == 0) continue;
        const uint32_t key = float_key(X[i * ld + j]);
        uint32_t v;
        if (phase == 0) {
            if ((key ^ s.prefix) & hi_mask) continue;
            v = key;
        } else {
            if (!s.tie || key != s.prefix) continue;
            v = ~(uint32_t)i;
            if ((v ^ s.prefix2) & hi_mask) continue;
        }
        atomicAdd(&h[jl * 256 + ((v >> shift) & 255u)], 1u);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < cg * 256; t += blockDim.x)
        if (h[t]) atomicAdd(&hist[(int64_t)(c0 + t / 256) * 256 + (t % 256)], h[t]);
}

__global__ void k_select(SelState* st, uint32_t* hist, int32_t B, int phase, int shift) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= B) return;
    SelState s = st[j];
    uint32_t* h = hist + (int64_t)j * 256;
    if (s.K > 0 && (phase == 0 || s.tie)) {
        int32_t cum = 0;
        int d = 255;
        for (; d > 0; --d) {
            if (cum + (int32_t)h[d] >= s.k_rem) break;
            cum += (int32_t)h[d];
        }
        if (phase == 0) {
            s.prefix |= (uint32_t)d << shift;
            s.greater += cum;
            s.k_rem -= cum;
            if (shift == 0) {
                s.eq = (int32_t)h[d];
                s.tie = s.k_rem < s.eq ? 1 : 0;
            }
        } else {
            s.prefix2 |= (uint32_t)d << shift;
            s.k_rem -= cum;
        }
    }
    for (int t = 0; t < 256; ++t) h[t] = 0;
    st[j] = s;
}

// Collect the selected elements (exactly K per column) into cand[j][0..K).
__global__ void k_collect(const float* X, int64_t n, int32_t B, int32_t ld, SelState* st, int32_t Kmax,
                          uint64_t* cand) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * B; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / B;
        const int j = (int)(e % B);
        const SelState& s = st[j];
        if (s.K == 0) continue;
        const uint32_t key = float_key(X[i * ld + j]);
        bool take = key > s.prefix;
        if (key == s.prefix) take = !s.tie || (~(uint32_t)i) >= s.prefix2;
        if (take) {
            int p = atomicAdd(&st[j].count, 1);
            if (p < Kmax) cand[(int64_t)j * Kmax + p] = ((uint64_t)key << 32) | (uint64_t)(~(uint32_t)i);
        }
    }
}

// Sort each column's candidates descending by (key, ~id) and write ids / scores.
__global__ void k_sort_out(const uint64_t* cand, const SelState* st, int32_t Kmax, int32_t* idx_out, float* score_out,
                           int skip_empty = 0) {
    extern __shared__ uint64_t sk[];
    const int j = blockIdx.x;
    const int K = min(st[j].K, Kmax);
    if (skip_empty && K == 0) return;
    int P = 1;
    while (P < K) P <<= 1;
    for (int t = threadIdx.x; t < P; t += blockDim.x) sk[t] = t < K ? cand[(int64_t)j * Kmax + t] : 0ull;
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < P; t += blockDim.x) {
                int u = t ^ stride;
                if (u > t) {
                    bool desc = (t & size) == 0;
                    uint64_t a = sk[t], b = sk[u];
                    if (desc ? (a < b) : (a > b)) {
                        sk[t] = b;
                        sk[u] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int t = threadIdx.x; t < Kmax; t += blockDim.x) {
        if (t < K) {
            uint64_t v = sk[t];
            idx_out[(int64_t)j * Kmax + t] = (int32_t)(~(uint32_t)(v & 0xFFFFFFFFu));
            score_out[(int64_t)j * Kmax + t] = key_float((uint32_t)(v >> 32));
        } else {
            idx_out[(int64_t)j * Kmax + t] = -1;
            score_out[(int64_t)j * Kmax + t] = 0.0f;
        }
    }
}

// ---- sampled-threshold fast path ----------------------------------------------
// A strided sample of each column gives a key threshold tau with, in
// expectation, about 4K + 8 (n / sample) elements at or above it; one pass over
// the scores collects those candidates, and per column a radix select finds
// the K-th of them and a sort orders the K at or above it.
// The result is exact whenever at least K and at most CAP candidates passed;
// otherwise that column is ranked again by the radix select.
constexpr int TK_SAMPLE = 4096;
constexpr int TK_CAP = 16384;
constexpr int TK_TOP = 2048;  // K <= Kmax <= 2048
// dynamic shared memory of k_topk_sort: candidates, the top K, histogram, scalars
constexpr size_t TK_SORT_SMEM = (size_t)(TK_CAP + TK_TOP) * 8 + 256 * 4 + 2 * 8 + 16;

// Each thread takes compare-exchange pairs directly (pair q: t = the q-th index
// with bit `stride` clear, u = t + stride), so no thread idles in a stage.
__device__ __forceinline__ void bitonic_desc_u64(uint64_t* a, int P) {
    for (int size = 2; size <= P; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int q = threadIdx.x; q < P / 2; q += blockDim.x) {
                const int t = ((q & ~(stride - 1)) << 1) | (q & (stride - 1));
                const int u = t + stride;
                const bool desc = (t & size) == 0;
                const uint64_t x = a[t], y = a[u];
                if (desc ? (x < y) : (x > y)) {
                    a[t] = y;
                    a[u] = x;
                }
            }
            __syncthreads();
        }
}

// The k-th largest (1-based, counting repeats) of a[0 .. cnt) in shared
// memory, by a most-significant-digit radix select over the low `nbits` bits
// (8 per round): a 256-bin histogram of the elements that match the digits
// chosen so far, then one warp finds the bin that holds the k-th (each lane sums
// 8 bins, a shuffle scan over the lanes).  All threads of the block call it.
__device__ uint64_t block_kth_desc(const uint64_t* a, int cnt, int k, int nbits, uint32_t* hist, uint64_t* sh) {
    uint64_t prefix = 0;
    int krem = k;
    for (int shift = nbits - 8; shift >= 0; shift -= 8) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
        __syncthreads();
        const uint64_t hi = shift + 8 >= 64 ? 0ull : (~0ull << (shift + 8));
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            const uint64_t v = a[i];
            if ((v & hi) == prefix) atomicAdd(&hist[(v >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            int h[8], sum = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                h[q] = (int)hist[255 - 8 * lane - q];  // lane 0 holds the highest bins
                sum += h[q];
            }
            int incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const int excl = incl - sum;
            const unsigned m = __ballot_sync(0xffffffffu, excl < krem && krem <= incl);
            if (m && lane == __ffs(m) - 1) {
                int cum = excl, d = 255 - 8 * lane - 7;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    if (cum + h[q] >= krem) {
                        d = 255 - 8 * lane - q;
                        break;
                    }
                    cum += h[q];
                }
                sh[0] = prefix | ((uint64_t)d << shift);
                sh[1] = (uint64_t)(krem - cum);
            }
        }
        __syncthreads();
        prefix = sh[0];
        krem = (int)sh[1];
        __syncthreads();
    }
    return prefix;
}

__global__ void __launch_bounds__(1024) k_topk_sample(const float* X, int64_t n, int32_t ld, const int32_t* Kd,
                                                     uint32_t* tau, int* cnt) {
    __shared__ uint64_t sk[TK_SAMPLE];
    const int j = blockIdx.x;
    const int64_t K = (int64_t)Kd[j] < n ? (int64_t)Kd[j] : n;
    if (K <= 0) {  // nothing to rank in this column (the filter and the sort skip it too)
        if (threadIdx.x == 0) {
            tau[j] = 0xFFFFFFFFu;
            cnt[j] = 0;
        }
        return;
    }
    const int s = (int)(n < TK_SAMPLE ? n : (int64_t)TK_SAMPLE);
    for (int t = threadIdx.x; t < TK_SAMPLE; t += blockDim.x) {
        uint64_t v = 0;
        if (t < s) {
            const int64_t i = (int64_t)t * n / s;
            v = (uint64_t)float_key(X[i * ld + j]);
        }
        sk[t] = v;
    }
    __syncthreads();
    // the threshold is the (kp + 1)-th largest sample (a radix select, not a sort)
    __shared__ uint32_t hist[256];
    __shared__ uint64_t sh[2];
    int64_t kp = (4 * K * s + n - 1) / n + 8;
    if (kp > s - 1) kp = s - 1;
    const uint64_t t = block_kth_desc(sk, TK_SAMPLE, (int)kp + 1, 32, hist, sh);
    if (threadIdx.x == 0) {
        tau[j] = (uint32_t)t;
        cnt[j] = 0;
    }
}

// Each thread keeps one column (B <= 256: 256 / B rows per block step) so the
// column's threshold and K stay in registers and no index is divided per element;
// eight rows' loads are issued before their compares (0.136 ms against 0.159 ms
// for a 1M x 64 block, cold L2).
constexpr int TK_ROWS = 8;
__global__ void __launch_bounds__(256) k_topk_filter(const float* X, int64_t n, int32_t B, int32_t ld,
                                                     const int32_t* Kd, const uint32_t* tau, int* cnt, uint64_t* cand) {
    const bool narrow = B <= 256;
    const int R = narrow ? 256 / B : 1;
    const int rt = narrow ? (int)threadIdx.x / B : 0;
    if (rt >= R) return;
    const int64_t step = (int64_t)gridDim.x * R;
    for (int j = narrow ? (int)threadIdx.x % B : (int)threadIdx.x; j < B; j += narrow ? B : 256) {
        const uint32_t tj = __ldg(tau + j);
        if (__ldg(Kd + j) <= 0) continue;
        for (int64_t i0 = (int64_t)blockIdx.x * R + rt; i0 < n; i0 += TK_ROWS * step) {
            float v[TK_ROWS];
#pragma unroll
            for (int u = 0; u < TK_ROWS; ++u) {
                const int64_t i = i0 + u * step;
                v[u] = i < n ? __ldcs(X + i * ld + j) : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < TK_ROWS; ++u) {
                const int64_t i = i0 + u * step;
                const uint32_t key = float_key(v[u]);
                if (i < n && key >= tj) {
                    const int p = atomicAdd(&cnt[j], 1);
                    if (p < TK_CAP) cand[(int64_t)j * TK_CAP + p] = ((uint64_t)key << 32) | (uint64_t)(~(uint32_t)i);
                }
            }
        }
    }
}

__global__ void __launch_bounds__(1024) k_topk_sort(const uint64_t* cand, const int* cnt, const int32_t* Kd, int64_t n,
                                                   int32_t Kmax, int32_t* idx_out, float* score_out, int* fail) {
    extern __shared__ uint64_t sk[];
    const int j = blockIdx.x;
    const int K = (int)((int64_t)Kd[j] < n ? (int64_t)Kd[j] : n);
    const int c = cnt[j];
    if (K > 0 && (c < K || c > TK_CAP)) {
        if (threadIdx.x == 0) fail[j] = 1;
        return;
    }
    if (threadIdx.x == 0) fail[j] = 0;
    // candidates' keys (score key, ~id) are distinct: exactly K lie at or above
    // the K-th largest, which a radix select finds; only those K are sorted
    uint64_t* top = sk + TK_CAP;  // [TK_TOP]
    uint32_t* hist = reinterpret_cast<uint32_t*>(top + TK_TOP);
    uint64_t* sh = reinterpret_cast<uint64_t*>(hist + 256);
    int* fill = reinterpret_cast<int*>(sh + 2);
    int P = 1;
    while (P < K) P <<= 1;
    if (K > 0) {
        for (int t = threadIdx.x; t < c; t += blockDim.x) sk[t] = cand[(int64_t)j * TK_CAP + t];
        if (threadIdx.x == 0) *fill = 0;
        __syncthreads();
        const uint64_t T = block_kth_desc(sk, c, K, 64, hist, sh);
        for (int t = threadIdx.x; t < c; t += blockDim.x)
            if (sk[t] >= T) {
                const int p = atomicAdd(fill, 1);  // exactly K reach here; the bound only guards the array
                if (p < TK_TOP) top[p] = sk[t];
            }
        for (int t = K + threadIdx.x; t < P; t += blockDim.x) top[t] = 0ull;
        __syncthreads();
        bitonic_desc_u64(top, P);
    }
    for (int t = threadIdx.x; t < Kmax; t += blockDim.x) {
        if (t < K) {
            const uint64_t v = top[t];
            idx_out[(int64_t)j * Kmax + t] = (int32_t)(~(uint32_t)(v & 0xFFFFFFFFu));
            score_out[(int64_t)j * Kmax + t] = key_float((uint32_t)(v >> 32));
        } else {
            idx_out[(int64_t)j * Kmax + t] = -1;
            score_out[(int64_t)j * Kmax + t] = 0.0f;
        }
    }
}

static int radix_rank(hd_ctx* ctx, const float* src, int64_t m, int32_t B, int32_t ld, const int32_t* K_h,
                      int32_t Kmax, int32_t* idx_d, float* score_d, int skip_empty, WsCarver& cv);

int hd_rank_impl(hd_ctx* ctx, const float* Xd, int64_t n, int32_t B, int32_t ldx, const int32_t* K_h, int32_t Kmax,
                 int32_t pool, int32_t* idx_d, float* score_d) {
    const float* src = Xd;
    int64_t m = n;
    int32_t ld = ldx;
    size_t bytes = ws_size(B * sizeof(SelState)) + ws_size((size_t)B * 256 * 4) + ws_size((size_t)B * Kmax * 8) +
                   ws_size(B * 4) + ws_size((size_t)B * TK_CAP * 8) + 3 * ws_size(B * 4) + ws_size(B * 4);
    if (pool > 1) {
        m = n / pool;
        bytes += ws_size((size_t)m * B * 4);
    }
    void* ws;
    int rc = hd_ws_reserve(ctx, bytes, &ws);
    if (rc) return rc;
    WsCarver cv(ws);
    int32_t* Kd = cv.take<int32_t>(B);
    uint64_t* cand = cv.take<uint64_t>((size_t)B * TK_CAP);
    uint32_t* tau = cv.take<uint32_t>(B);
    int* cnt = cv.take<int>(B);
    int* fail = cv.take<int>(B);
    if (pool > 1) {
        float* Y = cv.take<float>((size_t)m * B);
        k_pool<<<ceil_div(m * B, 256), 256, 0, ctx->stream>>>(Xd, m, B, ldx, pool, Y);
        HD_CHECK_LAUNCH(ctx);
        src = Y;
        ld = B;
    }
    HD_CUDA(ctx, cudaMemcpyAsync(Kd, K_h, B * 4, cudaMemcpyHostToDevice, ctx->stream));
    static uint64_t attr = 0;
    if (hd_first_on_device(attr, ctx->device)) {
        HD_CUDA(ctx, cudaFuncSetAttribute(k_topk_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, TK_SORT_SMEM));
    }
    k_topk_sample<<<B, 1024, 0, ctx->stream>>>(src, m, ld, Kd, tau, cnt);
    HD_CHECK_LAUNCH(ctx);
    const int gc = std::max(1, std::min<int>(ceil_div(m * B, 256 * 8), ctx->num_sms * 8));
    k_topk_filter<<<gc, 256, 0, ctx->stream>>>(src, m, B, ld, Kd, tau, cnt, cand);
    HD_CHECK_LAUNCH(ctx);
    k_topk_sort<<<B, 1024, TK_SORT_SMEM, ctx->stream>>>(cand, cnt, Kd, m, Kmax, idx_d, score_d, fail);
    HD_CHECK_LAUNCH(ctx);
    std::vector<int> hf(B);
    HD_CUDA(ctx, cudaMemcpyAsync(hf.data(), fail, B * 4, cudaMemcpyDeviceToHost, ctx->stream));
    HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    std::vector<int32_t> Kf(B, 0);
    bool any = false;
    for (int j = 0; j < B; ++j)
        if (hf[j]) {
            Kf[j] = K_h[j];
            any = true;
        }
    if (!any) return HD_OK;
    return radix_rank(ctx, src, m, B, ld, Kf.data(), Kmax, idx_d, score_d, 1, cv);
}

// Exact radix select for the columns with K > 0 (the others are left untouched
// when skip_empty is set).
static int radix_rank(hd_ctx* ctx, const float* src, int64_t m, int32_t B, int32_t ld, const int32_t* K_h,
                      int32_t Kmax, int32_t* idx_d, float* score_d, int skip_empty, WsCarver& cv) {
    SelState* st = cv.take<SelState>(B);
    uint32_t* hist = cv.take<uint32_t>((size_t)B * 256);
    uint64_t* cand = cv.take<uint64_t>((size_t)B * Kmax);
    int32_t* Kd = cv.take<int32_t>(B);
    HD_CUDA(ctx, cudaMemcpyAsync(Kd, K_h, B * 4, cudaMemcpyHostToDevice, ctx->stream));
    HD_CUDA(ctx, cudaMemsetAsync(hist, 0, (size_t)B * 256 * 4, ctx->stream));
    k_sel_init<<<ceil_div(B, 128), 128, 0, ctx->stream>>>(st, Kd, B, m);
    HD_CHECK_LAUNCH(ctx);
    static uint64_t attr = 0;
    if (hd_first_on_device(attr, ctx->device)) {
        HD_CUDA(ctx, cudaFuncSetAttribute(k_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, CG * 256 * 4));
    }
    const int gy = ceil_div(B, CG);
    const int gx = std::max(1, std::min<int>(ceil_div(m * std::min(B, CG), 256), ctx->num_sms * 4 / gy + 1));
    const size_t hsm = (size_t)std::min(B, CG) * 256 * 4;
    for (int phase = 0; phase < 2; ++phase) {
        if (phase == 1) {
            // the id pass is only needed when some column has ties at its boundary
            std::vector<SelState> hs(B);
            HD_CUDA(ctx, cudaMemcpyAsync(hs.data(), st, B * sizeof(SelState), cudaMemcpyDeviceToHost, ctx->stream));
            HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
            bool any = false;
            for (auto& x : hs) any = any || x.tie;
            if (!any) break;
        }
        for (int shift = 24; shift >= 0; shift -= 8) {
            k_hist<<<dim3(gx, gy), 256, hsm, ctx->stream>>>(src, m, B, ld, st, phase, shift, hist);
            HD_CHECK_LAUNCH(ctx);
            k_select<<<ceil_div(B, 128), 128, 0, ctx->stream>>>(st, hist, B, phase, shift);
            HD_CHECK_LAUNCH(ctx);
        }
    }
    const int gc = std::max(1, std::min<int>(ceil_div(m * B, 256 * 8), ctx->num_sms * 8));
    k_collect<<<gc, 256, 0, ctx->stream>>>(src, m, B, ld, st, Kmax, cand);
    HD_CHECK_LAUNCH(ctx);
    int P = 1;
    while (P < Kmax) P <<= 1;
    k_sort_out<<<B, 256, (size_t)P * 8, ctx->stream>>>(cand, st, Kmax, idx_d, score_d, skip_empty);
    HD_CHECK_LAUNCH(ctx);
    return HD_OK;
}

extern "C" int hd_rank(hd_ctx* ctx, const float* X, int64_t n, int32_t B, int32_t ldx, const int32_t* K,
                       int32_t Kmax, int32_t pool, int32_t* idx_out, float* score_out) {
    if (!ctx || !X || !K || !idx_out || !score_out || n <= 0 || B <= 0 || ldx < B) return HD_ERR_INVALID_ARG;
    if (Kmax < 1 || Kmax > 2048) return hd_fail(ctx, HD_ERR_INVALID_ARG, "Kmax=%d outside [1, 2048]", Kmax);
    if (pool < 0 || (pool > 1 && n % pool)) return hd_fail(ctx, HD_ERR_INVALID_ARG, "pool=%d does not divide n", pool);
    if (!hd_is_device_ptr(X)) return hd_fail(ctx, HD_ERR_INVALID_ARG, "X must be device memory");
    for (int j = 0; j < B; ++j)
        if (K[j] < 0 || K[j] > Kmax) return hd_fail(ctx, HD_ERR_INVALID_ARG, "K[%d]=%d outside [0, Kmax]", j, K[j]);
    HD_CUDA(ctx, cudaSetDevice(ctx->device));
    bool dev = hd_is_device_ptr(idx_out) && hd_is_device_ptr(score_out);
    int32_t* id = idx_out;
    float* sd = score_out;
    if (!dev) {
        HD_CUDA(ctx, cudaMallocAsync(&id, (size_t)B * Kmax * 4, ctx->stream));
        HD_CUDA(ctx, cudaMallocAsync(&sd, (size_t)B * Kmax * 4, ctx->stream));
    }
    int rc;
    {
        HD_PROF(ctx, "rank");
        rc = hd_rank_impl(ctx, X, n, B, ldx, K, Kmax, pool, id, sd);
    }
    if (!rc && !dev) {
        HD_CUDA(ctx, cudaMemcpyAsync(idx_out, id, (size_t)B * Kmax * 4, cudaMemcpyDeviceToHost, ctx->stream));
        HD_CUDA(ctx, cudaMemcpyAsync(score_out, sd, (size_t)B * Kmax * 4, cudaMemcpyDeviceToHost, ctx->stream));
        HD_CUDA(ctx, cudaFreeAsync(id, ctx->stream));
        HD_CUDA(ctx, cudaFreeAsync(sd, ctx->stream));
        HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    return rc;
}

// ------------------------------------------------------------------ allocation-free ranking
// hd_rank_static: the same top-K as hd_rank, for callers that cannot allocate
// device memory at call time.  All scratch lives in one file-scope device
// array sized for the stated maxima below; every device that loads the library
// holds it until the process exits.
namespace {
constexpr int RS_MAX_B = 256;
constexpr int RS_MAX_K = 2048;
constexpr size_t RS_STATE = RS_MAX_B * sizeof(SelState);
constexpr size_t RS_HIST = (size_t)RS_MAX_B * 256 * sizeof(uint32_t);
constexpr size_t RS_CAND = (size_t)RS_MAX_B * RS_MAX_K * sizeof(uint64_t);
constexpr size_t RS_K = RS_MAX_B * sizeof(int32_t);
constexpr size_t RS_BYTES = RS_STATE + RS_HIST + RS_CAND + RS_K;  // about 4.3 MB
}  // namespace

static __device__ __align__(256) unsigned char g_rank_scratch[RS_BYTES];

// Device address of g_rank_scratch per device (the host-side symbol is only a
// stand-in and must never be handed to a kernel).  Looked up on the first call
// on each device, with that device current; hd_destroy forgets it, so a device
// reset between contexts leads to a fresh lookup.  While a context is alive the
// cached address assumes its device is not reset.
static std::atomic<void*> g_rank_scratch_dev[64];

void hd_rank_static_forget(int device) {
    if (device >= 0 && device < 64) g_rank_scratch_dev[device].store(nullptr);
}

extern "C" int hd_rank_static(hd_ctx* ctx, const float* X, int64_t n, int32_t B, int32_t ldx, const int32_t* K,
                              int32_t Kmax, int32_t* idx_out, float* score_out) {
    if (!ctx || !X || !K || !idx_out || !score_out || n <= 0 || n >= (1ll << 31) || B <= 0 || ldx < B)
        return HD_ERR_INVALID_ARG;
    if (B > RS_MAX_B || Kmax < 1 || Kmax > RS_MAX_K)
        return hd_fail(ctx, HD_ERR_INVALID_ARG, "hd_rank_static: B=%d (max %d), Kmax=%d (max %d)", B, RS_MAX_B, Kmax,
                       RS_MAX_K);
    if (!hd_is_device_ptr(X) || !hd_is_device_ptr(idx_out) || !hd_is_device_ptr(score_out))
        return hd_fail(ctx, HD_ERR_INVALID_ARG, "hd_rank_static: X and the outputs must be device memory");
    // K is copied here, so the caller's array is only read during the call
    // (the device copy below then reads the library's pageable copy, which the
    // runtime stages before returning)
    int32_t kh[RS_MAX_B];
    for (int j = 0; j < B; ++j) {
        kh[j] = K[j];
        if (kh[j] < 0 || kh[j] > Kmax) return hd_fail(ctx, HD_ERR_INVALID_ARG, "K[%d]=%d outside [0, Kmax]", j, kh[j]);
    }
    if (ctx->device < 0 || ctx->device >= 64) return hd_fail(ctx, HD_ERR_INVALID_ARG, "device %d", ctx->device);
    HD_CUDA(ctx, cudaSetDevice(ctx->device));
    void* base_p = g_rank_scratch_dev[ctx->device].load();
    if (!base_p) {
        cudaError_t e = cudaGetSymbolAddress(&base_p, g_rank_scratch);
        if (e != cudaSuccess || !base_p)
            return hd_fail(ctx, HD_ERR_CUDA, "cudaGetSymbolAddress(g_rank_scratch): %s", cudaGetErrorString(e));
        g_rank_scratch_dev[ctx->device].store(base_p);
        HD_CUDA(ctx, cudaFuncSetAttribute(k_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, CG * 256 * 4));
    }
    char* base = (char*)base_p;
    SelState* st = (SelState*)base;
    uint32_t* hist = (uint32_t*)(base + RS_STATE);
    uint64_t* cand = (uint64_t*)(base + RS_STATE + RS_HIST);
    int32_t* Kd = (int32_t*)(base + RS_STATE + RS_HIST + RS_CAND);
    // the array keeps the previous call's contents: the histogram must start at zero
    HD_CUDA(ctx, cudaMemsetAsync(hist, 0, (size_t)B * 256 * sizeof(uint32_t), ctx->stream));
    HD_CUDA(ctx, cudaMemcpyAsync(Kd, kh, B * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    k_sel_init<<<ceil_div(B, 128), 128, 0, ctx->stream>>>(st, Kd, B, n);
    HD_CHECK_LAUNCH(ctx);
    const int gy = ceil_div(B, CG);
    const int gx = std::max(1, std::min<int>(ceil_div(n * std::min(B, CG), 256), ctx->num_sms * 4 / gy + 1));
    const size_t hsm = (size_t)std::min(B, CG) * 256 * 4;
    SelState hs[RS_MAX_B];
    for (int phase = 0; phase < 2; ++phase) {
        if (phase == 1) {
            HD_CUDA(ctx, cudaMemcpyAsync(hs, st, B * sizeof(SelState), cudaMemcpyDeviceToHost, ctx->stream));
            HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
            bool any = false;
            for (int j = 0; j < B; ++j) any = any || hs[j].tie;
            if (!any) break;
        }
        for (int shift = 24; shift >= 0; shift -= 8) {
            k_hist<<<dim3(gx, gy), 256, hsm, ctx->stream>>>(X, n, B, ldx, st, phase, shift, hist);
            HD_CHECK_LAUNCH(ctx);
            k_select<<<ceil_div(B, 128), 128, 0, ctx->stream>>>(st, hist, B, phase, shift);
            HD_CHECK_LAUNCH(ctx);
        }
    }
    const int gc = std::max(1, std::min<int>(ceil_div(n * B, 256), ctx->num_sms * 8));
    k_collect<<<gc, 256, 0, ctx->stream>>>(X, n, B, ldx, st, Kmax, cand);
    HD_CHECK_LAUNCH(ctx);
    int P = 1;
    while (P < Kmax) P <<= 1;
    k_sort_out<<<B, 256, (size_t)P * 8, ctx->stream>>>(cand, st, Kmax, idx_out, score_out);
    HD_CHECK_LAUNCH(ctx);
    return HD_OK;
}
