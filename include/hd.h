/*
 * hd.h - C ABI of the GB300 (sm_103a) hybrid spectral-temporal diffusion library.
 *
 * The library computes, for sparse observation vectors y over a k-NN graph,
 * the ranking vector x = h_alpha(W) y = (1 - alpha)(I - alpha W)^-1 y
 * (Iscen et al., "Hybrid Diffusion: Spectral-Temporal Graph Filtering for
 * Manifold Ranking", Eq. 3) as the sum of a spectral term from r precomputed
 * eigenpairs and a temporal term solved by conjugate gradient (Eq. 17-20),
 * and returns a top-K ranking of the database (Sec. 3).
 *
 * Conventions for every entry point:
 *  - Return value: HD_OK (0) or a negative HD_ERR_* code; the message of the
 *    last failure on a context is available from hd_last_error().
 *  - Pointers marked "host or device" are classified with
 *    cudaPointerGetAttributes; host buffers are copied in or out inside the
 *    call.  Pointers marked "device" must be device memory on the context's
 *    device.  All input buffers stay owned by the caller and are only read
 *    during the call; output buffers are caller-provided.
 *  - Handles (hd_ctx, hd_graph, hd_eig, hd_server) are allocated by the
 *    library and released with the matching *_destroy call (hd_serve_close
 *    for a server, before hd_destroy of its context).
 *  - All device work of a context is issued on the context's stream, in
 *    order.  Calls are thread-compatible per context, not thread-safe.
 *  - Dense n x B blocks are row-major: element (i, j) at i * ld + j.
 *  - There is no CPU fallback: without a usable CUDA device every call that
 *    needs one returns HD_ERR_CUDA.
 */
#ifndef HD_H
#define HD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------- */
#define HD_OK 0
#define HD_ERR_INVALID_ARG (-1)
#define HD_ERR_OOM (-2)
#define HD_ERR_CUDA (-3)
#define HD_ERR_TIMEOUT (-4)      /* a bounded device-side wait ran out */
#define HD_ERR_NOT_CONVERGED (-5)
#define HD_PENDING (-6)          /* serving: request not finished yet */
#define HD_ERR_NOT_FOUND (-7)

/* ---- element types ---------------------------------------------------- */
#define HD_F32 0
#define HD_BF16 1
#define HD_FP8 2                 /* e4m3 with one fp32 scale per row */

/* ---- graph symmetrisation --------------------------------------------- */
#define HD_SYM_UNION 0           /* edge if either end lists the other; larger weight */
#define HD_SYM_MUTUAL 1          /* edge if both ends list each other; smaller weight */

/* ---- query modes -------------------------------------------------------- */
#define HD_MODE_PAPER 0          /* Eq. 17-20: x = U1 g(L1) U1^T y + CG on L_a(W - U1 L1 U1^T) x^t = y */
#define HD_MODE_PROJ 1           /* x = U1 h(L1) U1^T y + (1-a) x2, (I - a W_r) x2 = (I - U1 U1^T) y */
#define HD_MODE_PCG 2            /* PCG on L_a(W) x = y, M^-1 = I + U1 diag(a l/(1 - a l)) U1^T */
/* Or-ed into HD_MODE_PAPER or HD_MODE_PROJ: X receives the temporal term alone
 * (x^t of Eq. 19, or (1-a) x2 of the projected form) instead of x^s + x^t, so
 * the temporal solve can be checked on its own (Eq. 19-20).  Invalid with
 * HD_MODE_PCG, which has no separate terms. */
#define HD_MODE_TEMPORAL_ONLY 0x100

/* ---- per-column status --------------------------------------------------- */
#define HD_COL_CONVERGED 0
#define HD_COL_MAX_ITER 1
#define HD_COL_BREAKDOWN 2       /* p^T A p <= 0 or not finite */
#define HD_COL_EMPTY 3           /* y == 0: x = 0 after 0 iterations */
#define HD_COL_CANCELLED 4       /* serving: withdrawn by hd_serve_cancel, no ranking */
#define HD_COL_STAGNATED 5       /* the recursive residual met tol, the true residual did not, even
                                    after the allowed residual replacements (fp32 floor) */

typedef struct hd_ctx hd_ctx;
typedef struct hd_graph hd_graph;
typedef struct hd_eig hd_eig;
typedef struct hd_server hd_server;

/* ---- context ------------------------------------------------------------- */

/* Create a context on CUDA device `device` issuing work on `cuda_stream`
 * (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream; NULL = the
 * legacy default stream).  Errors: HD_ERR_CUDA if the device is unusable. */
int hd_create(hd_ctx** out, int device, void* cuda_stream);
int hd_set_stream(hd_ctx* ctx, void* cuda_stream);
int hd_destroy(hd_ctx* ctx);
const char* hd_last_error(const hd_ctx* ctx);
/* Number of library kernel launches issued on this context so far. */
int64_t hd_launch_count(const hd_ctx* ctx);
/* Bytes of device workspace the context currently holds (grown on demand by
 * the calls that need scratch, released by hd_destroy). */
int hd_workspace_bytes(const hd_ctx* ctx, size_t* bytes);
/* Number of streaming multiprocessors of the context's device. */
int hd_num_sms(const hd_ctx* ctx);
/* Per-kernel device timing: while enabled, every launch of the library's
 * main kernels is bracketed by CUDA events on the context's stream.
 * hd_profile_read synchronises the stream and returns, for the kernel family
 * `name` ("spmm", "spmm_h" (the SpMM on the fp16 copy of P), "to_half" (making
 * that copy), "resid" (the true-residual SpMM), "dot", "update", "direction",
 * "colsq", "lr_reduce", "lr_expand", "scalar", "rank", "knn", "trunc_build"),
 * the number of
 * launches and their summed duration since the
 * last read, then clears that family.  busy_launches (may be NULL) counts the
 * launches that took at least 5% of the family's longest one: kernels of an
 * iteration return at once when none of their columns is active, and those
 * idle launches are left out of it. */
int hd_profile_enable(hd_ctx* ctx, int on);
int hd_profile_read(hd_ctx* ctx, const char* name, int64_t* launches, double* total_ms,
                    int64_t* busy_launches);

/* ---- graph (Sec. 3; Sec. 5.1) -------------------------------------------- */

/* Graph from a CSR matrix (host or device arrays).  row_ptr[n+1], col[nnz],
 * val[nnz] (fp32).  normalized = 0: val holds the raw symmetric adjacency A
 * (sparse, symmetric, nonnegative, zero diagonal) and the library forms
 * W = D^-1/2 A D^-1/2 with D = diag(A 1) (Sec. 3; a degree-0 node gets
 * D^-1/2 = 0).  normalized = 1: val already holds W.  Column indices must be
 * in [0, n); within a row they need not be sorted.
 * Errors: HD_ERR_INVALID_ARG on n <= 0, nnz < 0, nnz >= 2^31, or a
 * row_ptr that is not monotone from 0 to nnz. */
int hd_graph_from_csr(hd_ctx* ctx, int64_t n, int64_t nnz, const int32_t* row_ptr,
                      const int32_t* col, const float* val, int normalized, hd_graph** out);

/* k-NN graph of n descriptors X (n x d row-major, dtype HD_F32 or HD_BF16,
 * host or device): neighbours are the top k by dot product with self
 * excluded, ties to the smaller index (Sec. 5.1); weights max(s, 0)^gamma;
 * symmetrised by `sym`; edges of weight 0 dropped; normalised to W.
 * Similarities accumulate in fp32 (bf16 products on tensor cores).
 * Requires 1 <= k <= 64, k < n, d a multiple of 8 (bf16) or 4 (f32). */
int hd_build_graph(hd_ctx* ctx, const void* X, int64_t n, int32_t d, int dtype, int32_t k,
                   float gamma, int sym, hd_graph** out);

/* k nearest database rows of each of nq query rows (the neighbour search of
 * hd_build_graph on its own).  Q == X with exclude_self = 1 gives the graph's
 * directed lists.  idx_out[nq*k] (int32), sim_out[nq*k] (fp32) are host or
 * device; row q holds its neighbours by decreasing similarity, ties to the
 * smaller index, -1 / -inf past the end when fewer than k exist. */
int hd_knn(hd_ctx* ctx, const void* X, int64_t n, int32_t d, int dtype, const void* Q,
           int64_t nq, int32_t k, int exclude_self, int32_t* idx_out, float* sim_out);

/* Observation vectors (Sec. 3; Sec. 5.1): for each of nq queries Q (nq x d),
 * y has its non-zeros at the top-k_y database rows with value max(s, 0)^gamma.
 * Output in CSC-like form: y_ptr[nq+1], y_idx[nq*k_y], y_val[nq*k_y]
 * (host or device), ids ascending within a query; zero values are dropped,
 * so y_ptr[q+1] - y_ptr[q] <= k_y. */
int hd_observe(hd_ctx* ctx, const void* X, int64_t n, int32_t d, int dtype, const void* Q,
               int32_t nq, int32_t k_y, float gamma, int32_t* y_ptr, int32_t* y_idx,
               float* y_val);

int hd_graph_info(const hd_graph* g, int64_t* n, int64_t* nnz);
/* The SpMM launch shape the library measured for this graph at padded batch
 * width Bp (B rounded up to 4) during an earlier solve: *slab = columns per
 * row group (4..128), *segments = node-range passes.  HD_ERR_INVALID_ARG if no
 * solve with that width has run on the graph yet. */
int hd_graph_tuning(const hd_graph* g, int32_t Bp, int32_t* slab, int32_t* segments);
/* Copy the normalised graph out (any pointer may be NULL; host or device):
 * row_ptr[n+1], col[nnz], val[nnz] = W, dinv[n] = D^-1/2. Rows sorted by column. */
int hd_graph_export(hd_ctx* ctx, const hd_graph* g, int32_t* row_ptr, int32_t* col, float* val,
                    float* dinv);
int hd_graph_destroy(hd_graph* g);

/* ---- eigenpairs (Sec. 3.2, Sec. 4.1, Sec. 4.3) ------------------------------ */

/* Eigenpairs supplied by the caller: lambda[r] (host, descending), U
 * (n x r row-major fp32, host or device), stored on the device as `storage`
 * (HD_F32, HD_BF16 round-to-nearest-even, or HD_FP8 e4m3 with per-row scale
 * max_k |U_ik| / 448).  HD_F32 keeps, besides the fp32 values, a bf16
 * [hi | lo] copy (4 more bytes per entry) that the tensor-core products read;
 * their results carry about 16 significant bits of U and of the fp32 operand.
 * r may be 0. */
int hd_eig_from_host(hd_ctx* ctx, const hd_graph* g, int32_t r, const double* lambda,
                     const float* U, int storage, hd_eig** out);

/* Largest r (algebraic) eigenpairs of W by block Lanczos with full fp64
 * reorthogonalisation and thick restarts (Sec. 4.3 names Lanczos).  block = block
 * size b, max_basis = largest Krylov basis kept (multiple of b, > r), tol =
 * residual tolerance ||W u - l u|| on each pair, max_restarts bounds the outer
 * loop.  eigvals_out[r] and resid_out[r] (host, may be NULL) receive the Ritz
 * values and residual norms; returns HD_ERR_NOT_CONVERGED (with a usable
 * *out) if some residual stays above tol. */
int hd_eigendecompose(hd_ctx* ctx, const hd_graph* g, int32_t r, int32_t block,
                      int32_t max_basis, double tol, int32_t max_restarts, int storage,
                      uint64_t seed, hd_eig** out, double* eigvals_out, double* resid_out);

/* ---- convergence analysis (Sec. 4.4, Eq. 21-23) ---------------------------- */

/* Smallest eigenvalue lambda_n of W, the other end of the spectrum that sets
 * kappa in Eq. 22-23, by the same block Lanczos run on -W (block 4, basis 64
 * columns).  *lam_min (host) receives the Ritz value; HD_ERR_NOT_CONVERGED
 * (with the estimate written) if its residual ||W u - l u|| stays above tol
 * after max_restarts restarts.  Needs n >= 32. */
int hd_spectrum_min(hd_ctx* ctx, const hd_graph* g, double tol, int32_t max_restarts,
                    uint64_t seed, double* lam_min);

/* Host arithmetic, no device work.  For a solve in `mode` with the top r
 * eigenpairs removed, lam_next = lambda_{r+1}(W) (lambda_1 = 1 for r = 0) and
 * lam_min = lambda_n(W):
 *  *kappa_out   = kappa of the operator CG iterates on, Eq. 23 (Eq. 22 at
 *                 r = 0); the deflated operator's extremes are
 *                 max(0, lambda_{r+1}) and min(0, lambda_n).  For HD_MODE_PCG
 *                 the same number is kappa(M^-1 L_alpha(W)) with exact U.
 *  *iters_anorm = smallest i with phi_i(kappa) <= tol (Eq. 21): A-norm error
 *                 reduction by tol.
 *  *iters_resid = smallest i with sqrt(kappa_A) phi_i(kappa) <= tol, an upper
 *                 bound on the iterations the solver's stopping rule
 *                 ||r|| <= tol ||b|| needs in exact arithmetic (kappa_A: the
 *                 condition number of the matrix whose residual is measured,
 *                 L_alpha(W) for HD_MODE_PCG, the deflated operator otherwise).
 * Any output may be NULL.  HD_ERR_INVALID_ARG unless 0 <= alpha < 1, tol > 0
 * and -1 <= lam_min <= lam_next <= 1. */
int hd_cg_bound(int mode, double alpha, double lam_next, double lam_min, double tol,
                double* kappa_out, int32_t* iters_anorm, int32_t* iters_resid);

int hd_eig_info(const hd_eig* e, int32_t* r, int* storage);
/* Thick restarts the block Lanczos run that computed e took (-1 for
 * eigenpairs given by the caller, loaded or sparsified). */
int hd_eig_restarts(const hd_eig* e, int32_t* restarts);

/* SHybrid (Sec. 5.3, Table 1, Fig. 2): a new eigenpair handle whose U keeps
 * only the largest-magnitude entries of src's stored U.  The
 * round(sparsity * n * r) entries of smallest |U_ij| over the whole n x r
 * matrix are set to zero (round half to even); among equal magnitudes the
 * later entry in row-major order is dropped first, so the kept set is unique.
 * The kept entries keep their dequantised fp32 values and are stored twice,
 * by rows and by columns (12 bytes per entry plus offsets); lambda is
 * unchanged.  Every query mode and hd_eig_project / hd_eig_expand accept the
 * result (their low-rank products then run on the sparse entries);
 * hd_eig_export returns it densely with zeros.  sparsity in [0, 1]; src must
 * be dense with r > 0.  src stays valid and independent. */
int hd_eig_sparsify(hd_ctx* ctx, const hd_eig* src, double sparsity, hd_eig** out);
/* Stored entries of U: nnz of a sparsified handle, n * r otherwise. */
int hd_eig_nnz(const hd_eig* e, int64_t* nnz);
/* lambda[r] (host), U n x r fp32 (host or device; dequantised). */
int hd_eig_export(hd_ctx* ctx, const hd_eig* e, double* lambda, float* U);
int hd_eig_destroy(hd_eig* e);

/* The two halves of the right-to-left spectral product of Eq. 4, on the
 * stored (possibly quantised) U, with the library's own kernels:
 *  hd_eig_project: C = U^T V  for V n x B fp32 (device, leading dimension B),
 *                  C_out r x B fp64 (host or device).
 *  hd_eig_expand : X = U H    for H r x B fp64 (host or device),
 *                  X_out n x B fp32 (device, leading dimension B).
 * B must be a multiple of 4 and at most 256. */
int hd_eig_project(hd_ctx* ctx, const hd_eig* e, const float* V, int32_t B, double* C_out);
int hd_eig_expand(hd_ctx* ctx, const hd_eig* e, const double* H, int32_t B, float* X_out);

/* ---- truncated temporal filtering, "Temporal†" (Sec. 3.1, Sec. 5.1) ------- */

/* The baseline the paper compares against at large scale: for query j only
 * the shortlist S_j (its nearest database items, chosen by the caller) is
 * kept; the affinity restricted to S_j x S_j is normalised again by its own
 * degrees, W_j = D_j^-1/2 A_{S_j S_j} D_j^-1/2, and L_alpha(W_j) x_j = y_j
 * (Eq. 2 on the subgraph) is solved by CG, one system per column.  A is
 * recovered from the stored graph as W_ik / (d_i^-1/2 d_k^-1/2) (for a graph
 * given already normalised, A = W).
 *  sl_ptr[B+1], sl_idx : shortlists (host or device), ids in [0, n), no
 *             duplicate within a shortlist; s_j = sl_ptr[j+1] - sl_ptr[j] >= 0,
 *             s_max = max_j s_j >= 1.
 *  y_ptr, y_idx, y_val : observations as for hd_query_batch, by database id;
 *             entries outside S_j are dropped.
 *  X        : output s_max x B (leading dimension ldx >= B), host or device:
 *             X[t][j] is the score of sl_idx[sl_ptr[j] + t]; rows t >= s_j
 *             are 0.
 *  tol, max_iter, iters, relres, status : as for hd_query_batch.
 * Temporary device memory of about B n 4 bytes (the position maps) plus the B
 * subsystems is allocated for the call.  Errors: HD_ERR_INVALID_ARG for a bad
 * or duplicated shortlist id or observation index, HD_ERR_OOM. */
int hd_temporal_truncated(hd_ctx* ctx, const hd_graph* g, int32_t B, const int32_t* sl_ptr,
                          const int32_t* sl_idx, const int32_t* y_ptr, const int32_t* y_idx,
                          const float* y_val, double alpha, const float* tol, int32_t max_iter,
                          float* X, int32_t ldx, int32_t* iters, float* relres, int32_t* status);

/* ---- general transfer functions (Appendix A) ------------------------------ */

/* x = h(W) y for a transfer function given by its series coefficients
 * h(A) = sum_{i < ncoef} c_i A^i (Eq. 31, truncated by the caller), computed
 * by Theorem 2 (Eq. 32-33): x = U g(Lambda) U^T y + h(W - U Lambda U^T) y with
 * g(x) = h(x) - h(0); the second term by Horner's rule on the black box
 * z -> W z - U (Lambda (U^T z)) (ncoef - 1 SpMMs and low-rank products).
 *  eig      : NULL or r = 0 gives h(W) y by Horner's rule on W alone.
 *  y_ptr[B+1], y_idx, y_val : sparse observations as for hd_query_batch.
 *  coeffs[ncoef] : host, fp64, finite; 1 <= ncoef <= 100000.
 *  X        : output n x B (leading dimension ldx >= B), host or device.
 * Arithmetic is fp32 on the device (g(Lambda) in fp64 on the host).  With
 * c_i = (1 - alpha) alpha^i the result is the truncated series of Eq. 3. */
int hd_filter_poly(hd_ctx* ctx, const hd_graph* g, const hd_eig* eig, int32_t B,
                   const int32_t* y_ptr, const int32_t* y_idx, const float* y_val,
                   const double* coeffs, int32_t ncoef, float* X, int32_t ldx);

/* ---- checkpoints of the offline artefacts (Sec. 3, Sec. 4.1) -------------- */

/* The graph W and the eigenpairs are computed once offline and reused for
 * every query; these write them to a flat file and read them back (host
 * paths; little-endian; the arrays exactly as stored on the device, so a
 * loaded handle gives bit-identical results).  Files are not portable across
 * format versions (a magic string is checked).  hd_eig_save rejects
 * sparsified eigenpairs (sparsify again after loading).  Loading checks the
 * CSR structure like hd_graph_from_csr.  Errors: HD_ERR_INVALID_ARG (file
 * missing, short or not a checkpoint), HD_ERR_OOM. */
int hd_graph_save(hd_ctx* ctx, const hd_graph* g, const char* path);
int hd_graph_load(hd_ctx* ctx, const char* path, hd_graph** out);
int hd_eig_save(hd_ctx* ctx, const hd_eig* e, const char* path);
int hd_eig_load(hd_ctx* ctx, const char* path, hd_eig** out);

/* ---- failure detection (no counterpart in the paper) ---------------------- */

/* Self-test of the bounded waits that keep the tensor-core kernels from
 * hanging a shared GPU: a one-warp kernel waits on a barrier that nothing
 * completes (it must give up after limit_us microseconds, 1..1,000,000) and
 * then on one whose abort flag another lane raises (it must give up at once).
 * gave_up[2] (host) receives 1 for each wait that gave up.  Returns
 * HD_ERR_TIMEOUT when both gave up, which is the expected outcome; the
 * context stays usable. */
int hd_selftest_wait(hd_ctx* ctx, uint32_t limit_us, int32_t* gave_up);

/* ---- online query (Eq. 17-20) -------------------------------------------- */

/* Solve for B ranking vectors at once (one column per query).
 *  eig      : NULL or r = 0 gives temporal filtering (Eq. 2) in every mode.
 *  mode     : HD_MODE_PAPER / HD_MODE_PROJ / HD_MODE_PCG (see above), the
 *             first two optionally or-ed with HD_MODE_TEMPORAL_ONLY.
 *  y_ptr[B+1], y_idx, y_val : the sparse observations (host or device);
 *             indices in [0, n); duplicates are summed.
 *  alpha    : in [0, 1).
 *  tol[B]   : per-column relative residual tolerance (host or device).
 *  max_iter : maximum operator applications per column.
 *  X        : output, n x B scores with leading dimension ldx >= B
 *             (host or device).  X = x^s + x^t.
 *  iters[B], relres[B], status[B] : per column (host or device, may be NULL).
 * Stopping (x0 = 0, Sec. 4.4): a column stops iterating when its recursive
 * residual r satisfies ||r||_2 <= tol ||b||_2.  The true residual b - A x of
 * the system the column solves (A = L_a(W) for HD_MODE_PCG and temporal
 * filtering, L_a(W - U1 L1 U1^T) for the paper's form, b = y, or
 * (I - U1 U1^T) y for the projected form) is then computed once for the whole
 * batch with the same kernels.  A column whose true residual is above
 * tol ||b||_2 is restarted from its x with r := b - A x (residual
 * replacement), at most 3 times per call and within max_iter; if it still
 * misses, its status is HD_COL_STAGNATED.  relres[j] is the final TRUE
 * relative residual ||b - A x|| / ||b||, computed in fp32 on the device.
 * The solve runs without host synchronisation except polls of an active-
 * column count: the first after as many iterations as the previous solve on
 * the context took (same graph, eigenpairs, mode and batch width; 4 otherwise,
 * at most 8), then every 2.  Each such run of iterations is one CUDA graph,
 * captured on the context's own side stream the first time and replayed on
 * the context's stream while the graph, eigenpairs, mode, batch width, alpha
 * and max_iter stay the same (any change re-captures it; with
 * hd_profile_enable on, kernels launch one by one instead).  The call is
 * therefore not itself capturable into a caller's graph.  Errors: HD_ERR_INVALID_ARG for bad
 * sizes, indices out of range or non-finite observation values (checked on
 * the device before any iteration; X is then undefined),
 * HD_ERR_TIMEOUT if a tensor-core kernel gave up one of its bounded pipeline
 * waits (the kernels never hang; X is then undefined),
 * HD_ERR_NOT_CONVERGED is NOT returned: per-column status says it. */
int hd_query_batch(hd_ctx* ctx, const hd_graph* g, const hd_eig* eig, int mode, int32_t B,
                   const int32_t* y_ptr, const int32_t* y_idx, const float* y_val, double alpha,
                   const float* tol, int32_t max_iter, float* X, int32_t ldx, int32_t* iters,
                   float* relres, int32_t* status);

/* ---- ranking (Sec. 3) ------------------------------------------------------ */

/* Per column j of X (n x B, leading dimension ldx, device), the K[j] largest
 * scores in decreasing order, ties to the smaller row id.  pool > 1 first sums
 * each run of `pool` consecutive rows (regional descriptors: one image per run,
 * n a multiple of pool) and ranks the n/pool sums.  K[B] (host), K[j] <= Kmax
 * <= 2048.  idx_out[B*Kmax], score_out[B*Kmax] (host or device): column j at
 * offset j*Kmax; entries past K[j] are -1 / 0. */
int hd_rank(hd_ctx* ctx, const float* X, int64_t n, int32_t B, int32_t ldx, const int32_t* K,
            int32_t Kmax, int32_t pool, int32_t* idx_out, float* score_out);

/* Top-K ranking that allocates nothing (no counterpart in the paper): the
 * results equal hd_rank's for the same inputs.  For callers that cannot call
 * cudaMalloc at request time -- a real-time serving thread that must not block
 * on the allocator's device synchronisation, a host whose device memory is
 * entirely reserved by another framework's caching allocator, or a plugin that
 * may only use memory handed to it.  Scratch is one file-scope device array of
 * about 4.3 MB (B <= 256 columns, Kmax <= 2048) that every device using the
 * library holds until the process exits.  The first call on a device (again
 * after hd_destroy of a context on it) looks up that array's device address
 * with cudaGetSymbolAddress; the cached address assumes the device is not
 * reset while a context on it is alive.  The call cannot be captured into a
 * CUDA graph: it copies K from host memory and, when ties fall at a column's
 * K-th place, reads state back and synchronises the stream.  K is read during
 * the call only (the library copies it).  All calls share the array: calls
 * whose work overlaps on the GPU (different streams or contexts, or host
 * threads) race and must be serialised by the caller.  X (n x B, leading
 * dimension ldx), idx_out and score_out (B x Kmax) must be device memory; K[B]
 * is host.  No pooling.
 * Errors: HD_ERR_INVALID_ARG beyond the limits or for host X/outputs. */
int hd_rank_static(hd_ctx* ctx, const float* X, int64_t n, int32_t B, int32_t ldx,
                   const int32_t* K, int32_t Kmax, int32_t* idx_out, float* score_out);

/* ---- serving: continuous batching (no counterpart in the paper) ------------- */

typedef struct hd_req_stats {
    double submit_s;    /* host steady clock (s) at hd_serve_submit */
    double admit_s;     /* end of the step in which a column took the request */
    double done_s;      /* when its ranking had been copied to the host */
    int32_t iters;      /* CG iterations the request used */
    int32_t status;     /* HD_COL_* */
    float relres;       /* final relative residual ||r|| / ||y|| of the recursion: a served
                           column stops on it (no separate b - A x pass per retirement) */
    int32_t slot;       /* batch column it ran in (narrow-lane columns follow the wide ones) */
} hd_req_stats;

/* Open a server over a graph and optional eigenpairs.  The server owns one
 * persistent batch of up to max_slots columns (<= 256); with mem_budget > 0
 * the slot count is cut to what fits (each slot needs 4*n*4 + Kmax*8 bytes for
 * its R, P, Q, X columns and ranking).  When that batch has at least 8
 * columns and the budget (if any) holds 4 more, a second, narrow batch of 4
 * columns is kept too: a lightly loaded server (wide batch idle, queue no
 * longer than the narrow batch's free columns) admits there, where a request
 * moves 16 bytes per row instead of 4 x slots; results are the same bits in
 * either batch.  With eigenpairs the mode must be HD_MODE_PCG (the paper's
 * form needs a per-request spectral term at admission); without, it is
 * temporal CG.  Kmax <= 2048 bounds per-request K.
 * Errors: HD_ERR_OOM when not even one slot fits the budget or the device. */
int hd_serve_open(hd_ctx* ctx, const hd_graph* g, const hd_eig* eig, int mode, double alpha,
                  int32_t max_slots, size_t mem_budget, int32_t max_iter, int32_t Kmax,
                  hd_server** out);
/* Columns of the wide persistent batch. */
int hd_serve_slots(const hd_server* s);
/* Queue one request: its observation (nnz_y <= 512 host entries, indices in
 * [0, n), finite values, duplicates summed), residual tolerance and K <= Kmax.
 * Copies the arrays; returns a ticket.  Errors: HD_ERR_INVALID_ARG. */
int hd_serve_submit(hd_server* s, int32_t nnz_y, const int32_t* idx, const float* val, float tol,
                    int32_t K, uint64_t* ticket);
/* One step of the server: stage up to a batch's width of queued requests
 * (their observations and, with eigenpairs, U^T y), run `iters` CG
 * iterations of the whole batch, then retire every column that stopped
 * (converged, max_iter, breakdown): its top-K is ranked on the device and
 * copied to the host.  Admission happens inside the last iteration: in its
 * scalar step a column whose request stops there, or a free column, takes the
 * next staged request, and the same iteration's direction forms the new
 * request's p0 = M^-1 y, so no column spends an iteration between two requests
 * (a request's first update comes in the next step).  Staged requests no
 * column took go back to the front of the queue.  A request with y = 0 or
 * tol >= 1 finishes at staging (x = 0, ids 0 .. K-1 with score 0).
 * iters = 0 with requests queued runs one iteration.  *busy (may be NULL)
 * receives the number of queued plus running requests. */
int hd_serve_step(hd_server* s, int32_t iters, int32_t* busy);
/* HD_PENDING while the request runs; then copies its K ids / scores (host)
 * and stats, forgets the ticket and returns HD_OK.  HD_ERR_NOT_FOUND for an
 * unknown ticket.  A cancelled request reports status HD_COL_CANCELLED and
 * writes no ids or scores. */
int hd_serve_poll(hd_server* s, uint64_t ticket, int32_t* idx_out, float* score_out,
                  hd_req_stats* st);
/* Withdraw a request: a queued one leaves the queue, a running one frees its
 * column at once (the column is marked inactive on the context's stream, so
 * the batch's next iterations skip it and the column can take the next
 * request).  The request then polls as finished with status
 * HD_COL_CANCELLED and is reported by hd_serve_completed.  HD_OK also for a
 * request that had already finished (its results stay); HD_ERR_NOT_FOUND for
 * an unknown or already polled ticket. */
int hd_serve_cancel(hd_server* s, uint64_t ticket);
/* Tickets retired by hd_serve_step since the last call, in retirement order
 * (at most max_tickets; the rest stay for the next call): lets a caller with
 * many requests in flight poll only the finished ones.  *count receives the
 * number written to tickets[] (host). */
int hd_serve_completed(hd_server* s, uint64_t* tickets, int32_t max_tickets, int32_t* count);
/* Frees the server's buffers.  A server uses its context until it is closed:
 * close every server before hd_destroy of its context. */
int hd_serve_close(hd_server* s);

#ifdef __cplusplus
}
#endif
#endif /* HD_H */
