// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "../../include/hd.h"

struct hd_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    std::string err;
    int64_t launches = 0;
    // grow-only device workspace, carved per call (stream ordered)
    void* ws = nullptr;
    size_t ws_bytes = 0;
    // pinned host words for polling device counters
    int* h_poll = nullptr;
    int* d_flags = nullptr;   // [0]: device-side error flag, [1..]: misc counters
    // CUDA graphs of runs of CG iterations, keyed by everything the kernels
    // take as arguments plus the run length (a few kept; re-captured when the
    // solve's pointers or scalars change); launched on `stream`
    struct IterGraph {
        cudaGraphExec_t exec = nullptr;
        int64_t launches = 0;
    };
    cudaStream_t cap_stream = nullptr;
    std::map<std::vector<uint64_t>, IterGraph> iter_graphs;
    // iterations the previous solve with the same key (run length left out) took
    std::vector<uint64_t> hint_key;
    int iter_hint = 0;
    // per-kernel event timing (hd_profile_enable)
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::map<std::string, std::vector<std::pair<cudaEvent_t, cudaEvent_t>>> prof_ev;
};

// Bracket a launch with profiling events when enabled.
cudaEvent_t hd_prof_event(hd_ctx* ctx);
struct ProfScope {
    hd_ctx* ctx;
    const char* name;
    cudaEvent_t a = nullptr;
    ProfScope(hd_ctx* c, const char* n) : ctx(c), name(n) {
        if (ctx->prof) {
            a = hd_prof_event(ctx);
            cudaEventRecord(a, ctx->stream);
        }
    }
    ~ProfScope() {
        if (a) {
            cudaEvent_t b = hd_prof_event(ctx);
            cudaEventRecord(b, ctx->stream);
            ctx->prof_ev[name].push_back({a, b});
        }
    }
};
#define HD_CAT2(a, b) a##b
#define HD_CAT(a, b) HD_CAT2(a, b)
#define HD_PROF(ctx, name) ProfScope HD_CAT(hd_prof_scope_, __LINE__)((ctx), (name))

struct hd_graph {
    int64_t n = 0, nnz = 0;
    int device = 0;
    int32_t* row_ptr = nullptr;
    int32_t* col = nullptr;
    float* val = nullptr;     // normalised W
    float* dinv = nullptr;    // D^-1/2
    // autotuned SpMM column-slab width per padded batch width (Bp -> S)
    mutable std::map<int, int> slab_cache;
    // node-range segments of the SpMM: per segment count K, the entry bounds
    // [K + 1][n] of every row's part in each range of ceil(n / K) columns
    // (rows are sorted by column, so each part is contiguous); and the K
    // chosen per padded batch width
    mutable std::map<int, int32_t*> seg_bounds;
    mutable std::map<int, int> seg_cache;
    // entries in the longest row (measured on first use; -1 until then)
    mutable int32_t max_row = -1;
};

struct hd_eig {
    int64_t n = 0;
    int32_t r = 0;
    int32_t ldu = 0;          // leading dimension of U in elements (multiple of 16)
    int storage = HD_F32;
    void* U = nullptr;        // n x ldu, storage type
    float* scale = nullptr;   // per-row fp8 scale (HD_FP8 only)
    // HD_F32 only: bf16 copy of U split as [hi | lo] per row (each half
    // r rounded up to 128 wide, zero padded), hi = bf16(U), lo = bf16(U - hi),
    // read by the tensor-core products; lds = row length in elements
    void* Usplit = nullptr;
    int32_t lds = 0;
    double* lambda_d = nullptr;
    std::vector<double> lambda_h;
    int32_t restarts = -1;    // thick restarts of the Lanczos run that made it (-1: not from Lanczos)
    // sparsified embedding (hd_eig_sparsify): U is not stored densely then
    bool sparse = false;
    int64_t nnz = 0;
    int64_t* sp_rp = nullptr;   // CSR row offsets [n + 1]
    int32_t* sp_col = nullptr;  // CSR column (eigen-index) [nnz]
    float* sp_val = nullptr;    // CSR values [nnz]
    int64_t* sp_cp = nullptr;   // CSC column offsets [r + 1]
    int32_t* sp_row = nullptr;  // CSC row [nnz]
    float* sp_cval = nullptr;   // CSC values [nnz]
};

// ---------------------------------------------------------------- errors
int hd_fail(hd_ctx* ctx, int code, const char* fmt, ...);
// True the first time it is called for `device` with this flag word (function
// attributes such as the dynamic shared-memory limit are set per device).
inline bool hd_first_on_device(uint64_t& mask, int device) {
    const uint64_t b = 1ull << (device & 63);
    if (mask & b) return false;
    mask |= b;
    return true;
}
#define HD_CUDA(ctx, call)                                                            \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return hd_fail((ctx), HD_ERR_CUDA, "%s:%d %s: %s", __FILE__, __LINE__, #call, \
                           cudaGetErrorString(e_));                                   \
    } while (0)
// Function forms of the two checks, for code that must release resources
// before returning: 0 or the error code (the message is recorded).
inline int hd_check_cuda(hd_ctx* ctx, cudaError_t e, const char* what, const char* file, int line) {
    return e == cudaSuccess ? 0 : hd_fail(ctx, HD_ERR_CUDA, "%s:%d %s: %s", file, line, what, cudaGetErrorString(e));
}
int hd_check_launch(hd_ctx* ctx, const char* file, int line);
#define HD_CHECK_LAUNCH(ctx)                                                          \
    do {                                                                              \
        (ctx)->launches++;                                                            \
        cudaError_t e_ = cudaGetLastError();                                          \
        if (e_ != cudaSuccess)                                                        \
            return hd_fail((ctx), HD_ERR_CUDA, "%s:%d launch: %s", __FILE__, __LINE__,   \
                           cudaGetErrorString(e_));                                   \
    } while (0)

// ---------------------------------------------------------------- memory
bool hd_is_device_ptr(const void* p);
// Workspace: returns a device pointer of at least `bytes`, 256-aligned,
// valid until the next hd_ws_reserve on the same context.
int hd_ws_reserve(hd_ctx* ctx, size_t bytes, void** out);
// drop the cached device address of hd_rank_static's scratch on a device
void hd_rank_static_forget(int device);
struct WsCarver {
    char* base;
    size_t off = 0;
    explicit WsCarver(void* b) : base((char*)b) {}
    template <class T>
    T* take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T* p = (T*)(base + off);
        off += count * sizeof(T);
        return p;
    }
};
inline size_t ws_size(size_t bytes) { return (bytes + 255) & ~size_t(255); }

// Copy a caller buffer (host or device) to a device pointer (or alias it).
int hd_stage_in(hd_ctx* ctx, const void* src, size_t bytes, void* dev_scratch, const void** dev_out);

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------- device helpers
// Compensated (Knuth TwoSum) accumulation in fp32: value s + c.
struct KSum {
    float s, c;
};
__device__ __forceinline__ void ksum_add(KSum& a, float x) {
    float t = a.s + x;
    float bp = t - a.s;
    float e = (a.s - (t - bp)) + (x - bp);
    a.s = t;
    a.c += e;
}
__device__ __forceinline__ void ksum_merge(KSum& a, KSum b) {
    float t = a.s + b.s;
    float bp = t - a.s;
    float e = (a.s - (t - bp)) + (b.s - bp);
    a.s = t;
    a.c += b.c + e;
}

// Monotone map float -> uint32 (larger float, larger key).
__device__ __forceinline__ uint32_t float_key(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_float(uint32_t k) {
    uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(u);
}

// ---------------------------------------------------------------- cross-TU entry points
int hd_knn_impl(hd_ctx* ctx, const void* Xd, int64_t n, int32_t d, int dtype, const void* Qd,
                int64_t nq, int32_t k, int exclude_self, int32_t* idx_d, float* sim_d);
int hd_graph_from_lists(hd_ctx* ctx, int64_t n, int32_t k, const int32_t* idx_d, const float* sim_d,
                        float gamma, int sym, hd_graph** out);
int hd_normalize_graph(hd_ctx* ctx, hd_graph* g);
int hd_graph_alloc_internal(hd_ctx* ctx, int64_t n, int64_t nnz, hd_graph** out);
int hd_graph_check(hd_ctx* ctx, const hd_graph* g);
int hd_eig_alloc(hd_ctx* ctx, int64_t n, int32_t r, int storage, hd_eig** out);
int hd_eig_store_from_device_f32(hd_ctx* ctx, hd_eig* e, const float* U_d, int32_t ldsrc);
int hd_eig_sparse_export(hd_ctx* ctx, const hd_eig* e, float* dst);
int hd_spmm_apply(hd_ctx* ctx, const hd_graph* g, const float* P, float* Q, int32_t ld, int32_t B,
                  float c1, float c2);
int hd_rank_impl(hd_ctx* ctx, const float* Xd, int64_t n, int32_t B, int32_t ldx, const int32_t* K_h,
                 int32_t Kmax, int32_t pool, int32_t* idx_d, float* score_d);
