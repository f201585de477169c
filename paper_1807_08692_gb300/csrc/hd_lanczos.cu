// Offline eigenpairs: largest r eigenpairs of W by block Lanczos (Sec. 4.3
// names Lanczos as the way to get the few top eigenpairs the hybrid needs).
//
// Block Krylov basis Q (n x m, fp64, column-major) grown one block of b at a
// time from W Q_j, where the product with W runs in the library's fp32 SpMM.
// Every new block is orthogonalised against the whole basis twice (classical
// Gram-Schmidt twice, fp64 GEMMs) and normalised by Cholesky QR twice; the
// projections Q^T W Q_j are kept, so T = Q^T W Q is known explicitly.  When the
// basis is full, the Rayleigh-Ritz problem T = S Theta S^T (fp64, dense) gives
// Ritz pairs; residuals ||W y - theta y|| are measured with one more SpMM.
// Thick restart keeps the top k Ritz vectors plus the orthogonalised remainder.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include <cublas_v2.h>
#include <cusolverDn.h>

#include "hd_internal.cuh"

namespace {

struct Handles {
    cublasHandle_t blas = nullptr;
    cusolverDnHandle_t sol = nullptr;
    ~Handles() {
        if (blas) cublasDestroy(blas);
        if (sol) cusolverDnDestroy(sol);
    }
};

__device__ __forceinline__ uint64_t splitmix(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

// Uniform(-1, 1) start block from a counter-based hash of (seed, row, column).
__global__ void k_rand_block(double* V, int64_t n, int b, int64_t ld, uint64_t seed, int salt) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * b) return;
    int64_t i = e % n;
    int64_t j = e / n;
    uint64_t h = splitmix(seed ^ splitmix((uint64_t)i * 0x100000001B3ull + (uint64_t)j * 7919ull + (uint64_t)salt));
    V[j * ld + i] = ((double)(h >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;
}

// column-major fp64 (n x b, ld) -> row-major fp32 (n x bp)
__global__ void k_cm64_to_rm32(const double* V, int64_t n, int b, int64_t ld, float* out, int bp) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * bp) return;
    int64_t i = e / bp;
    int j = (int)(e % bp);
    out[e] = j < b ? (float)V[j * ld + i] : 0.0f;
}

// row-major fp32 (n x bp) -> column-major fp64 (n x b, ld)
__global__ void k_rm32_to_cm64(const float* in, int64_t n, int b, int bp, double* V, int64_t ld) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * b) return;
    int64_t i = e % n;
    int j = (int)(e / n);
    V[j * ld + i] = (double)in[i * bp + j];
}

// res[j] = || WY[:, j] - theta_j Y[:, j] ||^2 partial sums by atomics (fp64)
__global__ void k_resid(const double* WY, const double* Y, const double* theta, int64_t n, int k, int64_t ld,
                        double* res) {
    int j = blockIdx.y;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double d = WY[j * ld + i] - theta[j] * Y[j * ld + i];
        s += d * d;
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double sm[32];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[w];
        atomicAdd(&res[j], t);
    }
}

// column-major fp64 n x r -> row-major fp32 n x r
__global__ void k_cm64_to_rm32_r(const double* Y, int64_t n, int r, int64_t ld, float* U) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * r) return;
    int64_t i = e / r;
    int j = (int)(e % r);
    U[e] = (float)Y[j * ld + i];
}

// Sd[:, t] = S[:, m - 1 - t] for t < k (descending eigenvalue order)
__global__ void k_top_cols(const double* S, int m, int k, double* Sd) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)m * k) return;
    int t = (int)(e / m), i = (int)(e % m);
    Sd[e] = S[(int64_t)(m - 1 - t) * m + i];
}

}  // namespace

#define BL(call)                                                                               \
    do {                                                                                       \
        cublasStatus_t s_ = (call);                                                            \
        if (s_ != CUBLAS_STATUS_SUCCESS) return hd_fail(ctx, HD_ERR_CUDA, "cublas %d at %s:%d", (int)s_, __FILE__, __LINE__); \
    } while (0)
#define SL(call)                                                                               \
    do {                                                                                       \
        cusolverStatus_t s_ = (call);                                                          \
        if (s_ != CUSOLVER_STATUS_SUCCESS) return hd_fail(ctx, HD_ERR_CUDA, "cusolver %d at %s:%d", (int)s_, __FILE__, __LINE__); \
    } while (0)

struct Lanczos {
    hd_ctx* ctx;
    const hd_graph* g;
    int64_t n;
    int b, m;
    Handles h;
    double* Q;      // n x (m + b) column-major: basis plus the remainder block
    double* T;      // m x m
    double* W;      // n x max(b, k) work
    double* Y;      // n x k Ritz vectors
    double* WY;     // n x k
    double* G;      // small (m x max(b,k)) projections
    float* f_in;    // n x bp fp32 row-major
    float* f_out;
    double* S;      // m x m eigenvectors of T
    double* Sd;     // m x k, top-k in descending order
    double* theta;  // m
    double* resd;   // k
    int* info;
    double* work;
    int lwork = 0;
    int bp;
    float c2 = -1.0f;  // SpMM coefficient: -1 multiplies by W, +1 by -W (smallest end)
};

static int spmm_block(Lanczos& L, const double* V, int cols, double* out) {
    hd_ctx* ctx = L.ctx;
    // process in chunks of at most bp columns
    for (int c0 = 0; c0 < cols; c0 += L.bp) {
        int c = std::min(L.bp, cols - c0);
        int bp = (c + 3) / 4 * 4;
        k_cm64_to_rm32<<<ceil_div(L.n * bp, 256), 256, 0, ctx->stream>>>(V + (int64_t)c0 * L.n, L.n, c, L.n, L.f_in, bp);
        HD_CHECK_LAUNCH(ctx);
        int rc = hd_spmm_apply(ctx, L.g, L.f_in, L.f_out, bp, c, 0.0f, L.c2);
        if (rc) return rc;
        k_rm32_to_cm64<<<ceil_div(L.n * c, 256), 256, 0, ctx->stream>>>(L.f_out, L.n, c, bp, out + (int64_t)c0 * L.n, L.n);
        HD_CHECK_LAUNCH(ctx);
    }
    return HD_OK;
}

// W (n x b) -= Q[:, :cols] (Q[:, :cols]^T W), twice; returns the first projection in G (cols x b).
static int cgs2(Lanczos& L, int cols, double* Wb, int b, double* Gout) {
    hd_ctx* ctx = L.ctx;
    const double one = 1.0, zero = 0.0, mone = -1.0;
    for (int pass = 0; pass < 2; ++pass) {
        double* Gp = pass == 0 ? Gout : L.G + (size_t)L.m * b;
        BL(cublasDgemm(L.h.blas, CUBLAS_OP_T, CUBLAS_OP_N, cols, b, (int)L.n, &one, L.Q, (int)L.n, Wb, (int)L.n, &zero,
                       Gp, cols));
        BL(cublasDgemm(L.h.blas, CUBLAS_OP_N, CUBLAS_OP_N, (int)L.n, b, cols, &mone, L.Q, (int)L.n, Gp, cols, &one, Wb,
                       (int)L.n));
    }
    return HD_OK;
}

// Orthonormalise W (n x b) in place by Cholesky QR twice.  Returns 1 if rank deficient.
static int chol_qr2(Lanczos& L, double* Wb, int b, int* deficient) {
    hd_ctx* ctx = L.ctx;
    const double one = 1.0, zero = 0.0;
    *deficient = 0;
    std::vector<double> Gh((size_t)b * b);
    for (int pass = 0; pass < 2; ++pass) {
        BL(cublasDgemm(L.h.blas, CUBLAS_OP_T, CUBLAS_OP_N, b, b, (int)L.n, &one, Wb, (int)L.n, Wb, (int)L.n, &zero, L.G, b));
        HD_CUDA(ctx, cudaMemcpyAsync(Gh.data(), L.G, (size_t)b * b * 8, cudaMemcpyDeviceToHost, ctx->stream));
        HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        // upper Cholesky G = R^T R (column-major), in place
        double mx = 0.0;
        for (int i = 0; i < b; ++i) mx = std::max(mx, Gh[(size_t)i * b + i]);
        for (int j = 0; j < b; ++j) {
            for (int i = 0; i <= j; ++i) {
                double s = Gh[(size_t)j * b + i];
                for (int t = 0; t < i; ++t) s -= Gh[(size_t)i * b + t] * Gh[(size_t)j * b + t];
                if (i == j) {
                    if (!(s > 1e-24 * std::max(mx, 1e-300))) {
                        *deficient = 1;
                        return HD_OK;
                    }
                    Gh[(size_t)j * b + j] = std::sqrt(s);
                } else {
                    Gh[(size_t)j * b + i] = s / Gh[(size_t)i * b + i];
                }
            }
            for (int i = j + 1; i < b; ++i) Gh[(size_t)j * b + i] = 0.0;
        }
        HD_CUDA(ctx, cudaMemcpyAsync(L.G, Gh.data(), (size_t)b * b * 8, cudaMemcpyHostToDevice, ctx->stream));
        BL(cublasDtrsm(L.h.blas, CUBLAS_SIDE_RIGHT, CUBLAS_FILL_MODE_UPPER, CUBLAS_OP_N, CUBLAS_DIAG_NON_UNIT, (int)L.n, b,
                       &one, L.G, b, Wb, (int)L.n));
    }
    return HD_OK;
}

// Make block W orthonormal and orthogonal to Q[:, :cols]; replaces it by random
// directions when the Krylov space is exhausted.
static int new_block(Lanczos& L, int cols, double* Wb, uint64_t seed, int salt) {
    hd_ctx* ctx = L.ctx;
    for (int attempt = 0; attempt < 4; ++attempt) {
        int def = 0;
        int rc = chol_qr2(L, Wb, L.b, &def);
        if (rc) return rc;
        if (!def) return HD_OK;
        k_rand_block<<<ceil_div(L.n * L.b, 256), 256, 0, ctx->stream>>>(Wb, L.n, L.b, L.n, seed, salt * 16 + attempt + 1);
        HD_CHECK_LAUNCH(ctx);
        if (cols > 0 && (rc = cgs2(L, cols, Wb, L.b, L.G + (size_t)2 * L.m * L.b))) return rc;
    }
    return hd_fail(ctx, HD_ERR_NOT_CONVERGED, "could not extend the Krylov basis (n=%lld too small?)", (long long)L.n);
}

// Top-r eigenpairs of sign * W (sign = +1: W; -1: the smallest end of W).  With
// out == nullptr only the Ritz values and residuals are returned.
static int lanczos_top(hd_ctx* ctx, const hd_graph* g, int32_t r, int32_t block, int32_t max_basis, double tol,
                       int32_t max_restarts, int storage, uint64_t seed, int sign, hd_eig** out, double* eigvals_out,
                       double* resid_out) {
    if (out) *out = nullptr;
    HD_CUDA(ctx, cudaSetDevice(ctx->device));
    Lanczos L;
    L.ctx = ctx;
    L.g = g;
    L.c2 = sign > 0 ? -1.0f : 1.0f;
    L.n = g->n;
    L.b = block > 0 ? block : 32;
    if (L.b > 128) L.b = 128;
    const int k = std::min<int64_t>(r + L.b, L.n);     // Ritz vectors kept at a restart
    int m = max_basis > 0 ? max_basis : std::max(2 * r + 2 * L.b, 4 * L.b);
    m = (m + L.b - 1) / L.b * L.b;
    if (m > L.n) m = (int)(L.n / L.b) * L.b;
    if (m < k + L.b || m <= r) return hd_fail(ctx, HD_ERR_INVALID_ARG, "basis %d too small for r=%d, block %d (n=%lld)",
                                              m, r, L.b, (long long)L.n);
    L.m = m;
    L.bp = 64;
    const int64_t n = L.n;
    auto dmalloc = [&](void** p, size_t bytes) -> int {
        if (cudaMalloc(p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return hd_fail(ctx, HD_ERR_OOM, "Lanczos: %zu bytes", bytes);
        }
        return HD_OK;
    };
    int rc = 0;
    std::vector<void*> owned;
    auto take = [&](void** p, size_t bytes) {
        if (!rc) rc = dmalloc(p, bytes);
        if (!rc) owned.push_back(*p);
    };
    take((void**)&L.Q, (size_t)n * (m + L.b) * 8);
    take((void**)&L.T, (size_t)m * m * 8);
    take((void**)&L.W, (size_t)n * std::max(L.b, k) * 8);
    take((void**)&L.Y, (size_t)n * k * 8);
    take((void**)&L.WY, (size_t)n * k * 8);
    take((void**)&L.G, (size_t)3 * m * std::max(L.b, k) * 8 + (size_t)k * k * 8);
    take((void**)&L.f_in, (size_t)n * L.bp * 4);
    take((void**)&L.f_out, (size_t)n * L.bp * 4);
    take((void**)&L.theta, (size_t)m * 8);
    take((void**)&L.S, (size_t)m * m * 8);
    take((void**)&L.Sd, (size_t)m * k * 8);
    take((void**)&L.resd, (size_t)k * 8);
    take((void**)&L.info, 64);
    auto cleanup = [&]() {
        cudaStreamSynchronize(ctx->stream);
        for (void* p : owned) cudaFree(p);
    };
    if (rc) {
        cleanup();
        return rc;
    }
#define TRY(x)            \
    do {                  \
        rc = (x);         \
        if (rc) {         \
            cleanup();    \
            return rc;    \
        }                 \
    } while (0)
    if (cublasCreate(&L.h.blas) != CUBLAS_STATUS_SUCCESS || cusolverDnCreate(&L.h.sol) != CUSOLVER_STATUS_SUCCESS) {
        cleanup();
        return hd_fail(ctx, HD_ERR_CUDA, "cublas/cusolver init failed");
    }
    cublasSetStream(L.h.blas, ctx->stream);
    cusolverDnSetStream(L.h.sol, ctx->stream);
    if (cusolverDnDsyevd_bufferSize(L.h.sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, m, L.T, m, L.theta,
                                    &L.lwork) != CUSOLVER_STATUS_SUCCESS) {
        cleanup();
        return hd_fail(ctx, HD_ERR_CUDA, "syevd buffer size");
    }
    take((void**)&L.work, (size_t)L.lwork * 8);
    if (rc) {
        cleanup();
        return rc;
    }

    const double one = 1.0, zero = 0.0;
    // start block
    k_rand_block<<<ceil_div(n * L.b, 256), 256, 0, ctx->stream>>>(L.Q, n, L.b, n, seed, 0);
    HD_CHECK_LAUNCH(ctx);
    TRY(new_block(L, 0, L.Q, seed, 1));
    HD_CUDA(ctx, cudaMemsetAsync(L.T, 0, (size_t)m * m * 8, ctx->stream));
    int cols = L.b;
    int salt = 2;
    std::vector<double> th(m), res(k), Th;
    bool converged = false;
    for (int restart = 0;; ++restart) {
        // ---- grow the basis while a block fits in m columns; the orthogonalised
        // remainder of the last product stays in the next slot Q[:, cols : cols + b]
        while (true) {
            double* V = L.Q + (size_t)(cols - L.b) * n;
            double* Wn = L.Q + (size_t)cols * n;  // next block slot
            TRY(spmm_block(L, V, L.b, Wn));
            // T[0:cols, cols-b:cols] = Q^T W V ; W -= Q (Q^T W) twice
            TRY(cgs2(L, cols, Wn, L.b, L.G));
            BL(cublasDgeam(L.h.blas, CUBLAS_OP_N, CUBLAS_OP_N, cols, L.b, &one, L.G, cols, &zero, L.G, cols,
                           L.T + (size_t)(cols - L.b) * m, m));
            BL(cublasDgeam(L.h.blas, CUBLAS_OP_T, CUBLAS_OP_N, L.b, cols, &one, L.G, cols, &zero, L.G, L.b,
                           L.T + (cols - L.b), m));
            if (cols + L.b > m) break;
            TRY(new_block(L, cols, Wn, seed, salt++));
            cols += L.b;
        }
        // ---- Rayleigh-Ritz on the leading mc x mc block of T (mc = basis size reached)
        const int mc = cols;
        HD_CUDA(ctx, cudaMemcpy2DAsync(L.S, (size_t)mc * 8, L.T, (size_t)m * 8, (size_t)mc * 8, mc,
                                       cudaMemcpyDeviceToDevice, ctx->stream));
        SL(cusolverDnDsyevd(L.h.sol, CUSOLVER_EIG_MODE_VECTOR, CUBLAS_FILL_MODE_LOWER, mc, L.S, mc, L.theta, L.work,
                            L.lwork, L.info));
        HD_CUDA(ctx, cudaMemcpyAsync(th.data(), L.theta, (size_t)mc * 8, cudaMemcpyDeviceToHost, ctx->stream));
        // eigenvalues ascending: the top k are the last k columns of S, taken in reverse
        k_top_cols<<<ceil_div((int64_t)mc * k, 256), 256, 0, ctx->stream>>>(L.S, mc, k, L.Sd);
        HD_CHECK_LAUNCH(ctx);
        BL(cublasDgemm(L.h.blas, CUBLAS_OP_N, CUBLAS_OP_N, (int)n, k, mc, &one, L.Q, (int)n, L.Sd, mc, &zero, L.Y,
                       (int)n));
        HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        std::vector<double> thk(k);
        for (int t = 0; t < k; ++t) thk[t] = th[mc - 1 - t];
        HD_CUDA(ctx, cudaMemcpyAsync(L.theta, thk.data(), (size_t)k * 8, cudaMemcpyHostToDevice, ctx->stream));
        // residuals with one SpMM of the Ritz block
        TRY(spmm_block(L, L.Y, k, L.WY));
        HD_CUDA(ctx, cudaMemsetAsync(L.resd, 0, (size_t)k * 8, ctx->stream));
        k_resid<<<dim3(std::max(1, std::min(ceil_div(n, 256), 64)), k), 256, 0, ctx->stream>>>(L.WY, L.Y, L.theta, n, k,
                                                                                             n, L.resd);
        HD_CHECK_LAUNCH(ctx);
        HD_CUDA(ctx, cudaMemcpyAsync(res.data(), L.resd, (size_t)k * 8, cudaMemcpyDeviceToHost, ctx->stream));
        HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        double worst = 0.0;
        for (int t = 0; t < r; ++t) worst = std::max(worst, std::sqrt(res[t]));
        converged = worst <= tol;
        if (getenv("HD_LANCZOS_TRACE"))
            fprintf(stderr, "lanczos restart %d cols %d worst %.3e theta %.8f %.8f %.8f\n", restart, cols, worst,
                    thk[0], thk[1], thk[std::min(r, k) - 1]);
        if (converged || restart >= max_restarts) {
            for (int t = 0; t < r; ++t) {
                if (eigvals_out) eigvals_out[t] = thk[t];
                if (resid_out) resid_out[t] = std::sqrt(res[t]);
            }
            if (!out) {
                cleanup();
                return converged ? HD_OK : hd_fail(ctx, HD_ERR_NOT_CONVERGED, "max residual %.3e > tol %.1e", worst, tol);
            }
            hd_eig* e;
            TRY(hd_eig_alloc(ctx, n, r, storage, &e));
            e->restarts = restart;
            e->lambda_h.assign(thk.begin(), thk.begin() + r);
            HD_CUDA(ctx, cudaMemcpyAsync(e->lambda_d, thk.data(), (size_t)r * 8, cudaMemcpyHostToDevice, ctx->stream));
            float* U32;
            TRY(dmalloc((void**)&U32, (size_t)n * r * 4));
            owned.push_back(U32);
            k_cm64_to_rm32_r<<<ceil_div(n * r, 256), 256, 0, ctx->stream>>>(L.Y, n, r, n, U32);
            HD_CHECK_LAUNCH(ctx);
            TRY(hd_eig_store_from_device_f32(ctx, e, U32, r));
            cleanup();
            *out = e;
            return converged ? HD_OK : hd_fail(ctx, HD_ERR_NOT_CONVERGED, "max residual %.3e > tol %.1e", worst, tol);
        }
        // ---- thick restart: Q = [Y (k), remainder (b)], T = Q^T W Q for the first k + b columns
        double* rem = L.Q + (size_t)mc * n;                  // remainder block (already orthogonal to Q[:, :mc])
        HD_CUDA(ctx, cudaMemcpyAsync(L.W, rem, (size_t)n * L.b * 8, cudaMemcpyDeviceToDevice, ctx->stream));
        HD_CUDA(ctx, cudaMemcpyAsync(L.Q, L.Y, (size_t)n * k * 8, cudaMemcpyDeviceToDevice, ctx->stream));
        double* nb = L.Q + (size_t)k * n;
        HD_CUDA(ctx, cudaMemcpyAsync(nb, L.W, (size_t)n * L.b * 8, cudaMemcpyDeviceToDevice, ctx->stream));
        TRY(cgs2(L, k, nb, L.b, L.G + (size_t)2 * L.m * L.b));
        TRY(new_block(L, k, nb, seed, salt++));
        cols = k + L.b;
        HD_CUDA(ctx, cudaMemsetAsync(L.T, 0, (size_t)m * m * 8, ctx->stream));
        // T[0:k+b, 0:k] = Q[:, :k+b]^T (W Y)
        double* P = L.G;
        BL(cublasDgemm(L.h.blas, CUBLAS_OP_T, CUBLAS_OP_N, cols, k, (int)n, &one, L.Q, (int)n, L.WY, (int)n, &zero, P, cols));
        BL(cublasDgeam(L.h.blas, CUBLAS_OP_N, CUBLAS_OP_N, cols, k, &one, P, cols, &zero, P, cols, L.T, m));
        BL(cublasDgeam(L.h.blas, CUBLAS_OP_T, CUBLAS_OP_N, k, cols, &one, P, cols, &zero, P, k, L.T, m));
    }
#undef TRY
}

extern "C" int hd_eigendecompose(hd_ctx* ctx, const hd_graph* g, int32_t r, int32_t block, int32_t max_basis,
                                 double tol, int32_t max_restarts, int storage, uint64_t seed, hd_eig** out,
                                 double* eigvals_out, double* resid_out) {
    if (!ctx || !g || !out || r <= 0 || r > 1024) return HD_ERR_INVALID_ARG;
    if (storage != HD_F32 && storage != HD_BF16 && storage != HD_FP8)
        return hd_fail(ctx, HD_ERR_INVALID_ARG, "storage %d", storage);
    return lanczos_top(ctx, g, r, block, max_basis, tol, max_restarts, storage, seed, +1, out, eigvals_out, resid_out);
}

extern "C" int hd_spectrum_min(hd_ctx* ctx, const hd_graph* g, double tol, int32_t max_restarts, uint64_t seed,
                               double* lam_min) {
    if (!ctx || !g || !lam_min) return HD_ERR_INVALID_ARG;
    if (g->n < 32) return hd_fail(ctx, HD_ERR_INVALID_ARG, "n=%lld too small for the Lanczos estimate", (long long)g->n);
    double th = 0.0, rs = 0.0;
    // one Ritz value of -W with a block of 4 and a basis of 64 columns
    const int rc = lanczos_top(ctx, g, 1, 4, 64, tol, max_restarts, HD_F32, seed, -1, nullptr, &th, &rs);
    *lam_min = -th;
    return rc;
}

// Eq. 21-23: kappa of the system CG runs on and the iterations the bound needs.
extern "C" int hd_cg_bound(int mode, double alpha, double lam_next, double lam_min, double tol, double* kappa_out,
                           int32_t* iters_anorm, int32_t* iters_resid) {
    if (!(alpha >= 0.0 && alpha < 1.0) || !(tol > 0.0) || !(lam_next <= 1.0) || !(lam_min >= -1.0) ||
        lam_min > lam_next || (mode != HD_MODE_PAPER && mode != HD_MODE_PROJ && mode != HD_MODE_PCG))
        return HD_ERR_INVALID_ARG;
    // the deflated operator keeps r zero eigenvalues, so its extremes are
    // max(0, lambda_{r+1}) and min(0, lambda_n)
    const double top = std::max(0.0, lam_next), bot = std::min(0.0, lam_min);
    const double kappa = (1.0 - alpha * bot) / (1.0 - alpha * top);
    // the residual criterion ||r|| <= tol ||b|| follows from the A-norm bound
    // through sqrt(kappa(A)) of the matrix the residual belongs to: the deflated
    // operator for Forms P and N, L_alpha(W) itself (Eq. 22) for the
    // preconditioned solve
    const double kappa_a = mode == HD_MODE_PCG ? (1.0 - alpha * bot) / (1.0 - alpha) : kappa;
    const double sk = std::sqrt(kappa);
    const double q = (sk - 1.0) / (sk + 1.0);
    auto first = [&](double target) -> int32_t {
        if (q <= 0.0) return 1;
        const double need = std::log(target / 2.0) / std::log(q);
        int32_t i = need <= 0.0 ? 0 : (int32_t)std::ceil(need);
        // settle rounding of the logarithms against the bound itself
        while (i > 0 && 2.0 * std::pow(q, i - 1) <= target) --i;
        while (2.0 * std::pow(q, i) > target) ++i;
        return i;
    };
    if (kappa_out) *kappa_out = kappa;
    if (iters_anorm) *iters_anorm = first(tol);
    if (iters_resid) *iters_resid = first(tol / std::sqrt(kappa_a));
    return HD_OK;
}
