// Online query path: spectral term + temporal term by multi-RHS CG (Eq. 17-20).
//
// Layout: every n x B block (R, P, Q, X) is row-major with a padded width Bp
// (B rounded up to a multiple of 4) so that one gathered row of P is Bp
// contiguous fp32 values: a group of Bp/4 lanes moves it with float4 loads.
//
// One CG iteration for B columns at once (per-column scalars in fp64):
//   Q = c1 P - c2 W P [+ U (c3 Lambda o (U^T P))]                 Eq. 20
//   sigma = P^T Q  (SpMM partials + c3 sum_k lambda_k C_k^2, C = U^T P)
//   a = rho / sigma; X += a P; R -= a Q; rr = ||R||^2               (CG, Sec. 4.4)
//   [PCG: C = U^T R, rho' = rr + sum_k D_k C_k^2, Z = R + U (D o C)]
//   beta = rho' / rho; P = Z + beta P
// Columns stop individually (||r|| <= tol ||b||, max_iter, breakdown); a
// stopped column keeps X and R bit-for-bit (its step length is 0).  When every
// column has stopped, the true residual b - A x is formed for the batch; a
// column whose recursive residual met tol but whose true residual did not is
// restarted from x with r := b - A x (residual replacement, at most
// MAX_CONFIRM times), and the true value is what the solve reports.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <vector>

#include <cuda_fp16.h>

#include "hd_solve.cuh"

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ float4 ld4v(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

// ------------------------------------------------------------------ kernels
// R[:, j] += y_j (one thread per column: duplicates summed in input order).
__global__ void k_scatter_y(const int32_t* y_ptr, const int32_t* y_idx, const float* y_val, int32_t B, int64_t n,
                            int32_t ld, float* R, int* err) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= B) return;
    int32_t b = y_ptr[j], e = y_ptr[j + 1];
    if (b > e || b < 0) {
        atomicExch(err, 1);
        return;
    }
    for (int32_t t = b; t < e; ++t) {
        const int32_t i = y_idx[t];
        const float v = y_val[t];
        if (i < 0 || i >= n || !isfinite(v)) {
            atomicExch(err, 1);
            continue;
        }
        R[(int64_t)i * ld + j] += v;
    }
}

// True when some column of this block's S-column slab is active; with
// st == nullptr every slab works.
template <int S>
__device__ __forceinline__ bool slab_has_work(const ColState* st) {
    if (!st) return true;
    int w = 0;
    if (threadIdx.x < S) w = st[blockIdx.y * S + threadIdx.x].active;
    return __syncthreads_or(w) != 0;
}

#define FMA4(acc_, wt_, vec_)                  \
    acc_.x = fmaf(wt_, vec_.x, acc_.x);       \
    acc_.y = fmaf(wt_, vec_.y, acc_.y);       \
    acc_.z = fmaf(wt_, vec_.z, acc_.z);       \
    acc_.w = fmaf(wt_, vec_.w, acc_.w)

// 4-column slabs: two lanes per row, which compute the same two chains as a
// thread per row (chain s: entries 8c + {0, 2, 4, 6} of the full chunks of 8,
// then every tail entry in order; chain s2: entries 8c + {1, 3, 5, 7}; the row
// sum s + s2), so the bits do not change; the pairs halve each lane's serial
// gathers and read the row's indices two at a time (0.28 ms against 0.38 ms
// on the 1M-node graph, the same bits).  128 rows per block step.
__device__ __forceinline__ void spmm_rows_pair4(const int32_t* rp, const int32_t* ci, const float* wv,
                                                const float* P, float* Q, int64_t n, int32_t ld, float c1, float c2) {
    const int lane = threadIdx.x & 31, h = lane & 1;
    const int col = blockIdx.y * 4;
    // rows advance warp-uniformly (the shuffle needs every lane); a lane past
    // the last row works on an empty row and writes nothing
    for (int64_t r0 = (int64_t)blockIdx.x * 128 + (threadIdx.x >> 5) * 16; r0 < n; r0 += (int64_t)gridDim.x * 128) {
        const int64_t row = r0 + (lane >> 1);
        const bool ok = row < n;
        const int32_t b = ok ? rp[row] : 0, e = ok ? rp[row + 1] : 0;
        const int32_t full = b + (e - b) / 8 * 8;
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        int32_t t = b;
        for (; t + 16 <= full; t += 16) {  // two chunks: this lane's 8 entries
            float w[8];
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int32_t k = t + 2 * u + h;
                w[u] = __ldg(wv + k);
                v[u] = ld4(P + (int64_t)__ldg(ci + k) * ld + col);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                FMA4(s, w[u], v[u]);
            }
        }
        if (t < full) {  // one chunk left
            float w[4];
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int32_t k = t + 2 * u + h;
                w[u] = __ldg(wv + k);
                v[u] = ld4(P + (int64_t)__ldg(ci + k) * ld + col);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                FMA4(s, w[u], v[u]);
            }
            t += 8;
        }
        if (h == 0) {  // the tail belongs to chain s, in masked batches of 4
            for (; t < e; t += 4) {
                const int m = e - t;
                float4 v[4];
                float w[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    w[u] = u < m ? __ldg(wv + t + u) : 0.f;
                    v[u] = u < m ? ld4(P + (int64_t)__ldg(ci + t + u) * ld + col) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (u < m) {
                        FMA4(s, w[u], v[u]);
                    }
                }
            }
        }
        const float ox = __shfl_xor_sync(0xffffffffu, s.x, 1), oy = __shfl_xor_sync(0xffffffffu, s.y, 1);
        const float oz = __shfl_xor_sync(0xffffffffu, s.z, 1), ow = __shfl_xor_sync(0xffffffffu, s.w, 1);
        if (ok && h == 0) {
            s.x += ox;
            s.y += oy;
            s.z += oz;
            s.w += ow;
            const float4 own = ld4(P + row * ld + col);
            float4 q;
            q.x = c1 * own.x - c2 * s.x;
            q.y = c1 * own.y - c2 * s.y;
            q.z = c1 * own.z - c2 * s.z;
            q.w = c1 * own.w - c2 * s.w;
            st4(Q + row * ld + col, q);
        }
    }
}

// Q = c1 P - c2 W P for the S-column slab blockIdx.y: S/4 threads per row, each
// over all of the row's entries (chains as above), 8 gathers in flight.  The
// P^T Q partials of CG come from k_dot below: kept out of this kernel, its
// register count allows eight 256-thread blocks per SM, and the extra warps
// keep more of the random row gathers in flight (measured on the 1M-node graph:
// 1.58 ms + 0.08 ms for the separate pass against 2.06 ms with the partials
// fused).  The summation order is the same at every slab width.
// `skip` (may be null): the launch returns at once when *skip is not 0.
template <int S>
__global__ void __launch_bounds__(256, 8) k_spmm(const int32_t* rp, const int32_t* ci, const float* wv, const float* P,
                                              float* Q, int64_t n, int32_t ld, float c1, float c2,
                                              const ColState* st, const int* skip = nullptr) {
    constexpr int L = S / 4;
    constexpr int RPB = 256 / L;
    if (skip && *skip) return;
    if (!slab_has_work<S>(st)) return;
    if constexpr (S == 4) {
        spmm_rows_pair4(rp, ci, wv, P, Q, n, ld, c1, c2);
        return;
    }
    const int g = (threadIdx.x & 31) % L;
    const int col = blockIdx.y * S + 4 * g;
    for (int64_t row = (int64_t)blockIdx.x * RPB + threadIdx.x / L; row < n; row += (int64_t)gridDim.x * RPB) {
        const int32_t b = rp[row], e = rp[row + 1];
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 s2 = make_float4(0.f, 0.f, 0.f, 0.f);
        int32_t t = b;
        for (; t + 8 <= e; t += 8) {
            int32_t j[8];
            float w[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                j[u] = __ldg(ci + t + u);
                w[u] = __ldg(wv + t + u);
            }
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = ld4(P + (int64_t)j[u] * ld + col);
#pragma unroll
            for (int u = 0; u < 8; u += 2) {
                FMA4(s, w[u], v[u]);
                FMA4(s2, w[u + 1], v[u + 1]);
            }
        }
        // the last e - t < 8 entries, four gathers issued before their
        // multiply-adds, which still run one entry after another
        for (; t < e; t += 4) {
            const int m = e - t;
            float4 v[4];
            float w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                w[u] = u < m ? __ldg(wv + t + u) : 0.f;
                v[u] = u < m ? ld4(P + (int64_t)__ldg(ci + t + u) * ld + col) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (u < m) {
                    FMA4(s, w[u], v[u]);
                }
            }
        }
        s.x += s2.x;
        s.y += s2.y;
        s.z += s2.z;
        s.w += s2.w;
        const float4 own = ld4(P + row * ld + col);
        float4 q;
        q.x = c1 * own.x - c2 * s.x;
        q.y = c1 * own.y - c2 * s.y;
        q.z = c1 * own.z - c2 * s.z;
        q.w = c1 * own.w - c2 * s.w;
        st4(Q + row * ld + col, q);
    }
}

// A batch of at most 4 columns (one 4-column slab, hd_query_batch only): four
// lanes per row, lane e summing entries b + e, b + e + 4, ... in order (four
// loads in flight), the four sums meeting as (v0 + v2) + (v1 + v3).  The
// row's index / weight reads are coalesced and eight rows gather per warp:
// 0.24 ms on the 1M-node benchmark graph against 0.28 ms for k_spmm<4> (two
// lanes per row), 0.38 ms for a thread per row and 0.32 ms for a warp per row.
// Its sums run in another order than k_spmm's, so the server, whose results
// must not depend on the lane width, keeps k_spmm.
constexpr int N4_ROWS = 64;  // rows per 256-thread block
__global__ void __launch_bounds__(256, 8) k_spmm_n4(const int32_t* rp, const int32_t* ci, const float* wv,
                                                    const float* P, float* Q, int64_t n, float c1, float c2,
                                                    const ColState* st) {
    if (!slab_has_work<4>(st)) return;
    const int lane = threadIdx.x & 31, e = lane & 3;
    // rows advance warp-uniformly (the shuffles need every lane); a lane past
    // the last row works on an empty row and writes nothing
    for (int64_t r0 = (int64_t)blockIdx.x * N4_ROWS + (threadIdx.x >> 5) * 8; r0 < n;
         r0 += (int64_t)gridDim.x * N4_ROWS) {
        const int64_t row = r0 + (lane >> 2);
        const bool ok = row < n;
        const int32_t b = ok ? rp[row] : 0, end = ok ? rp[row + 1] : 0;
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int32_t t = b + e; t < end; t += 16) {
            const int m = (end - t + 3) / 4;
            float w[4];
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                w[u] = u < m ? __ldg(wv + t + 4 * u) : 0.f;
                v[u] = u < m ? ld4(P + (int64_t)__ldg(ci + t + 4 * u) * 4) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (u < m) {
                    FMA4(s, w[u], v[u]);
                }
        }
#pragma unroll
        for (int o = 2; o > 0; o >>= 1) {
            s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
            s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
            s.z += __shfl_xor_sync(0xffffffffu, s.z, o);
            s.w += __shfl_xor_sync(0xffffffffu, s.w, o);
        }
        if (ok && e == 0) {
            const float4 own = ld4(P + row * 4);
            float4 q;
            q.x = c1 * own.x - c2 * s.x;
            q.y = c1 * own.y - c2 * s.y;
            q.z = c1 * own.z - c2 * s.z;
            q.w = c1 * own.w - c2 * s.w;
            st4(Q + row * 4, q);
        }
    }
}

// ---- a 16-bit copy of P for the SpMM gathers of late iterations
// Inexact Krylov methods (Simoncini and Szyld, SIAM J. Sci. Comput. 2003; van
// den Eshof and Sleijpen, SIAM J. Matrix Anal. Appl. 2004): the operator may be
// applied less accurately as the residual shrinks; the gap between recursive
// and true residual grows by |a_k| ||E_k p_k|| per iteration.  Here E_k p =
// c2 W (p~ - p) with p~ the fp16 copy (relative rounding u16 = 2^-11 per
// entry), and |a_k| ||p_k|| = ||x_{k+1} - x_k|| <= 2 ||r_k|| (L_a(W) >= I), so
// the gap added by an fp16 iteration is at most 2 c2 u16 ||W (p~ - p)|| / u16
// ||p|| times ||r_k||: 0.1 ||r_k|| in the worst case, ~0.008 ||r_k|| for rounding
// errors of random sign over ~54 neighbours.  The next SpMM gathers the fp16
// copy once every active column has ||r|| <= HALF_THETA tol ||b||, which keeps
// the typical gap near a quarter of tol ||b||; the true-residual confirmation
// certifies the result either way.  Each column is scaled by a power of two so
// that its largest entry lies in [2^13, 2^14) (exact, no overflow); the own-row
// term c1 p, the dot products and the updates stay fp32.
constexpr double HALF_THETA = 25.0;

// per-column max |P| (the bits of a non-negative float order like the value);
// runs when the next SpMM gathers the fp16 copy and some column is active
__global__ void __launch_bounds__(256) k_colmax(const float* __restrict__ P, int64_t n, int32_t ld,
                                                unsigned* __restrict__ mx, const int* __restrict__ use_half,
                                                const int* __restrict__ num_active) {
    if (!*use_half || !*num_active) return;
    __shared__ unsigned bmax[256];  // per column of this block (ld <= 256)
    const int nq = ld >> 2;
    const int rpb = blockDim.x / nq;  // rows per block step
    for (int c = threadIdx.x; c < ld; c += blockDim.x) bmax[c] = 0u;
    __syncthreads();
    if ((int)threadIdx.x < rpb * nq) {
        const int q = threadIdx.x % nq;
        float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;
        for (int64_t row = (int64_t)blockIdx.x * rpb + threadIdx.x / nq; row < n; row += (int64_t)gridDim.x * rpb) {
            const float4 v = ld4(P + row * ld + 4 * q);
            m0 = fmaxf(m0, fabsf(v.x));
            m1 = fmaxf(m1, fabsf(v.y));
            m2 = fmaxf(m2, fabsf(v.z));
            m3 = fmaxf(m3, fabsf(v.w));
        }
        // one global atomic per column and block: same-address atomics from
        // every thread would serialise in the one L2 slice holding mx
        atomicMax(bmax + 4 * q, __float_as_uint(m0));
        atomicMax(bmax + 4 * q + 1, __float_as_uint(m1));
        atomicMax(bmax + 4 * q + 2, __float_as_uint(m2));
        atomicMax(bmax + 4 * q + 3, __float_as_uint(m3));
    }
    __syncthreads();
    for (int c = threadIdx.x; c < ld; c += blockDim.x) atomicMax(mx + c, bmax[c]);
}

// 2^k with max|P_j| 2^k in [2^13, 2^14) (1 for a zero column), and its inverse
__device__ __forceinline__ float half_scale(unsigned mbits, bool inverse) {
    const float m = __uint_as_float(mbits);
    if (!(m > 0.f)) return 1.f;
    int ex;
    frexpf(m, &ex);  // m = f 2^ex, f in [0.5, 1)
    return ldexpf(1.f, inverse ? ex - 14 : 14 - ex);
}

// P16 = fp16(P_j 2^k_j) column by column
__global__ void __launch_bounds__(256) k_to_half(const float* __restrict__ P, int64_t n, int32_t ld,
                                                 const unsigned* __restrict__ mx, __half* __restrict__ P16,
                                                 const int* __restrict__ use_half,
                                                 const int* __restrict__ num_active) {
    if (!*use_half || !*num_active) return;
    const int nq = ld >> 2;
    const int rpb = blockDim.x / nq;
    if ((int)threadIdx.x >= rpb * nq) return;
    const int q = threadIdx.x % nq;
    const float s0 = half_scale(mx[4 * q], false), s1 = half_scale(mx[4 * q + 1], false);
    const float s2 = half_scale(mx[4 * q + 2], false), s3 = half_scale(mx[4 * q + 3], false);
    for (int64_t row = (int64_t)blockIdx.x * rpb + threadIdx.x / nq; row < n; row += (int64_t)gridDim.x * rpb) {
        const float4 v = ld4(P + row * ld + 4 * q);
        const __half2 a = __floats2half2_rn(v.x * s0, v.y * s1);
        const __half2 b = __floats2half2_rn(v.z * s2, v.w * s3);
        uint2 o;
        o.x = *reinterpret_cast<const unsigned*>(&a);
        o.y = *reinterpret_cast<const unsigned*>(&b);
        *reinterpret_cast<uint2*>(P16 + row * ld + 4 * q) = o;
    }
}

#define FMA8H(acc_, wt_, raw_)                                                    \
    {                                                                             \
        const __half2* h_ = reinterpret_cast<const __half2*>(&(raw_));            \
        _Pragma("unroll") for (int k_ = 0; k_ < 4; ++k_) {                        \
            const float2 f_ = __half22float2(h_[k_]);                             \
            acc_[2 * k_] = fmaf(wt_, f_.x, acc_[2 * k_]);                         \
            acc_[2 * k_ + 1] = fmaf(wt_, f_.y, acc_[2 * k_ + 1]);                 \
        }                                                                         \
    }

// Q = c1 P - c2 W P with the W P gathers from the fp16 copy (S columns per
// slab, 8 per lane: a row's slab is S 2 bytes); the sums are fp32, unscaled by
// the column's power of two at the end.  Runs when *use_half is set.
template <int S>
__global__ void __launch_bounds__(256, 4) k_spmm_h(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                   const float* __restrict__ wv, const __half* __restrict__ P16,
                                                   const unsigned* __restrict__ mx, const float* __restrict__ P,
                                                   float* __restrict__ Q, int64_t n, int32_t ld, float c1, float c2,
                                                   const ColState* st, const int* __restrict__ use_half) {
    constexpr int L = S / 8;
    constexpr int RPB = 256 / L;
    if (!*use_half) return;
    if (!slab_has_work<S>(st)) return;
    const int g = (threadIdx.x & 31) % L;
    const int col = blockIdx.y * S + 8 * g;
    float inv[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) inv[c] = half_scale(mx[col + c], true);
    for (int64_t row = (int64_t)blockIdx.x * RPB + threadIdx.x / L; row < n; row += (int64_t)gridDim.x * RPB) {
        const int32_t b = rp[row], e = rp[row + 1];
        float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        int32_t t = b;
        for (; t + 8 <= e; t += 8) {
            int32_t j[8];
            float w[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                j[u] = __ldg(ci + t + u);
                w[u] = __ldg(wv + t + u);
            }
            uint4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldg(reinterpret_cast<const uint4*>(P16 + (int64_t)j[u] * ld + col));
#pragma unroll
            for (int u = 0; u < 8; ++u) FMA8H(acc, w[u], v[u]);
        }
        for (; t < e; t += 4) {
            const int m = e - t;
            uint4 v[4];
            float w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                w[u] = u < m ? __ldg(wv + t + u) : 0.f;
                v[u] = u < m ? __ldg(reinterpret_cast<const uint4*>(P16 + (int64_t)__ldg(ci + t + u) * ld + col))
                             : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (u < m) FMA8H(acc, w[u], v[u]);
            }
        }
        const float4 o0 = ld4(P + row * ld + col), o1 = ld4(P + row * ld + col + 4);
        const float own[8] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w};
        float q[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) q[c] = c1 * own[c] - c2 * (acc[c] * inv[c]);
        st4(Q + row * ld + col, make_float4(q[0], q[1], q[2], q[3]));
        st4(Q + row * ld + col + 4, make_float4(q[4], q[5], q[6], q[7]));
    }
}

// ---- the true residual, accumulated in two fp32 words
// b - A x with A = c1 I - c2 W cancels: c1 x and c2 W x are ~1/(1 - a) times
// larger than the result, so the fp32 rounding of W x (relative ~u per term)
// would reach the residual magnified 1/(1 - a) times (about 7e-7 ||y|| on the
// 2,000-node graph, as large as a 1e-6 tolerance).  The residual kernels below
// carry W x as an unevaluated sum hi + lo of two fp32 numbers, built with
// error-free transformations: the product w v = p + e exactly (e from one fma;
// Ogita, Rump and Oishi, "Accurate sum and dot product", 2005) and the sum
// hi + p = s + e exactly (Knuth's TwoSum).  The _rn intrinsics keep the
// compiler from contracting these into other fma operations.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
}

// hi + lo += w v
__device__ __forceinline__ void df_fma(float& hi, float& lo, float w, float v) {
    const float p = __fmul_rn(w, v);
    const float pe = __fmaf_rn(w, v, -p);
    float s, e;
    two_sum(hi, p, s, e);
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(e, pe));
}

// -(c1 x - c2 (hi + lo)), rounded once at the end
__device__ __forceinline__ float neg_operator(float c1, float x, float c2, float hi, float lo) {
    const float p1 = __fmul_rn(c1, x), e1 = __fmaf_rn(c1, x, -p1);
    const float p2 = __fmul_rn(c2, hi), e2 = __fmaf_rn(c2, hi, -p2);
    float d, e3;
    two_sum(p1, -p2, d, e3);
    const float tail = __fsub_rn(__fsub_rn(__fadd_rn(e3, e1), e2), __fmul_rn(c2, lo));
    return -__fadd_rn(d, tail);
}

// Q = -(c1 X - c2 W X) for the S-column slab blockIdx.y, W X in two words.
// Runs when *pick is 1 (see k_resid_pick).
template <int S>
__global__ void __launch_bounds__(256, 4) k_resid(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                                  const float* __restrict__ wv, const float* __restrict__ X,
                                                  float* __restrict__ Q, int64_t n, int32_t ld, float c1, float c2,
                                                  const int* __restrict__ pick) {
    constexpr int L = S / 4;
    constexpr int RPB = 256 / L;
    if (*pick != 1) return;
    const int g = (threadIdx.x & 31) % L;
    const int col = blockIdx.y * S + 4 * g;
    for (int64_t row = (int64_t)blockIdx.x * RPB + threadIdx.x / L; row < n; row += (int64_t)gridDim.x * RPB) {
        const int32_t b = rp[row], e = rp[row + 1];
        float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
        int32_t t = b;
        for (; t + 4 <= e; t += 4) {
            int32_t j[4];
            float w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                j[u] = __ldg(ci + t + u);
                w[u] = __ldg(wv + t + u);
            }
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) v[u] = ld4(X + (int64_t)j[u] * ld + col);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                df_fma(hi[0], lo[0], w[u], v[u].x);
                df_fma(hi[1], lo[1], w[u], v[u].y);
                df_fma(hi[2], lo[2], w[u], v[u].z);
                df_fma(hi[3], lo[3], w[u], v[u].w);
            }
        }
        for (; t < e; ++t) {
            const float w0 = __ldg(wv + t);
            const float4 v0 = ld4(X + (int64_t)__ldg(ci + t) * ld + col);
            df_fma(hi[0], lo[0], w0, v0.x);
            df_fma(hi[1], lo[1], w0, v0.y);
            df_fma(hi[2], lo[2], w0, v0.z);
            df_fma(hi[3], lo[3], w0, v0.w);
        }
        const float4 own = ld4(X + row * ld + col);
        float4 q;
        q.x = neg_operator(c1, own.x, c2, hi[0], lo[0]);
        q.y = neg_operator(c1, own.y, c2, hi[1], lo[1]);
        q.z = neg_operator(c1, own.z, c2, hi[2], lo[2]);
        q.w = neg_operator(c1, own.w, c2, hi[3], lo[3]);
        st4(Q + row * ld + col, q);
    }
}

// Per-column operators (truncated systems): column j's row t holds the entries
// off[j * n + t] .. off[j * n + t + 1] of (ci, wv); columns j >= B are empty.
// Q = c1 P - c2 W_j P column by column.
template <int S>
__global__ void __launch_bounds__(256) k_spmm_cols(const int64_t* __restrict__ off, const int32_t* __restrict__ ci,
                                                   const float* __restrict__ wv, int32_t B, const float* __restrict__ P,
                                                   float* __restrict__ Q, int64_t n, int32_t ld, float c1, float c2,
                                                   const ColState* __restrict__ st) {
    constexpr int L = S / 4;
    constexpr int RPB = 256 / L;
    if (!slab_has_work<S>(st)) return;
    const int g = (threadIdx.x & 31) % L;
    const int col = blockIdx.y * S + 4 * g;
    for (int64_t row = (int64_t)blockIdx.x * RPB + threadIdx.x / L; row < n; row += (int64_t)gridDim.x * RPB) {
        float s[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = col + c;
            if (j >= B) continue;
            const int64_t f = (int64_t)j * n + row;
            const int64_t b = __ldg(off + f), e = __ldg(off + f + 1);
            float s0 = 0.f, s1 = 0.f;
            int64_t t = b;
            for (; t + 2 <= e; t += 2) {
                s0 = fmaf(__ldg(wv + t), __ldg(P + (int64_t)__ldg(ci + t) * ld + j), s0);
                s1 = fmaf(__ldg(wv + t + 1), __ldg(P + (int64_t)__ldg(ci + t + 1) * ld + j), s1);
            }
            if (t < e) s0 = fmaf(__ldg(wv + t), __ldg(P + (int64_t)__ldg(ci + t) * ld + j), s0);
            s[c] = s0 + s1;
        }
        const float4 own = ld4(P + row * ld + col);
        float4 q;
        q.x = c1 * own.x - c2 * s[0];
        q.y = c1 * own.y - c2 * s[1];
        q.z = c1 * own.z - c2 * s[2];
        q.w = c1 * own.w - c2 * s[3];
        st4(Q + row * ld + col, q);
    }
}

// Q = -(c1 X - c2 W_j X) column by column (truncated systems), W_j X in two words.
template <int S>
__global__ void __launch_bounds__(256) k_resid_cols(const int64_t* __restrict__ off, const int32_t* __restrict__ ci,
                                                    const float* __restrict__ wv, int32_t B, const float* __restrict__ X,
                                                    float* __restrict__ Q, int64_t n, int32_t ld, float c1, float c2) {
    constexpr int L = S / 4;
    constexpr int RPB = 256 / L;
    const int g = (threadIdx.x & 31) % L;
    const int col = blockIdx.y * S + 4 * g;
    for (int64_t row = (int64_t)blockIdx.x * RPB + threadIdx.x / L; row < n; row += (int64_t)gridDim.x * RPB) {
        const float4 own = ld4(X + row * ld + col);
        const float ox[4] = {own.x, own.y, own.z, own.w};
        float q[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = col + c;
            float hi = 0.f, lo = 0.f;
            if (j < B) {
                const int64_t f = (int64_t)j * n + row;
                const int64_t b = __ldg(off + f), e = __ldg(off + f + 1);
                for (int64_t t = b; t < e; ++t) df_fma(hi, lo, __ldg(wv + t), __ldg(X + (int64_t)__ldg(ci + t) * ld + j));
            }
            q[c] = neg_operator(c1, ox[c], c2, hi, lo);
        }
        st4(Q + row * ld + col, make_float4(q[0], q[1], q[2], q[3]));
    }
}

// *out = the largest row length (entries) of the CSR graph
__global__ void k_max_row(const int32_t* __restrict__ rp, int64_t n, int* out) {
    int m = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, rp[i + 1] - rp[i]);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// Row i's entries in segment s (columns [s w, (s + 1) w)) are
// bounds[s n + i] .. bounds[(s + 1) n + i] (rows sorted by column).
__global__ void k_seg_bounds(const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, int64_t n, int K,
                             int64_t w, int32_t* __restrict__ bounds) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t t = rp[i];
    const int32_t e = rp[i + 1];
    bounds[i] = t;
    for (int s = 1; s < K; ++s) {
        const int64_t lim = (int64_t)s * w;
        while (t < e && ci[t] < lim) ++t;
        bounds[(int64_t)s * n + i] = t;
    }
    bounds[(int64_t)K * n + i] = e;
}

// One node-range segment of Q = c1 P - c2 W P: the gathered rows of P all lie
// in one range of the nodes, so that range stays in L2 for the pass.  The
// first segment writes Q, the others subtract into it.
template <int S>
__global__ void __launch_bounds__(256, 8) k_spmm_seg(const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                  const int32_t* __restrict__ ci, const float* __restrict__ wv,
                                                  const float* __restrict__ P, float* __restrict__ Q, int64_t n,
                                                  int32_t ld, float c1, float c2, const ColState* __restrict__ st,
                                                  int first) {
    constexpr int L = S / 4;
    constexpr int RPB = 256 / L;
    if (!slab_has_work<S>(st)) return;
    const int g = (threadIdx.x & 31) % L;
    const int col = blockIdx.y * S + 4 * g;
    for (int64_t row = (int64_t)blockIdx.x * RPB + threadIdx.x / L; row < n; row += (int64_t)gridDim.x * RPB) {
        const int32_t b = __ldg(lo + row), e = __ldg(hi + row);
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 s2 = make_float4(0.f, 0.f, 0.f, 0.f);
        int32_t t = b;
        for (; t + 8 <= e; t += 8) {
            int32_t j[8];
            float w[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                j[u] = __ldg(ci + t + u);
                w[u] = __ldg(wv + t + u);
            }
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = ld4(P + (int64_t)j[u] * ld + col);
#pragma unroll
            for (int u = 0; u < 8; u += 2) {
                FMA4(s, w[u], v[u]);
                FMA4(s2, w[u + 1], v[u + 1]);
            }
        }
        // the last e - t < 8 entries as in k_spmm (a row's part in one node
        // range is short, ~nnz/(n K) entries, so this tail is a large share)
        for (; t < e; t += 4) {
            const int m = e - t;
            float4 v[4];
            float w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                w[u] = u < m ? __ldg(wv + t + u) : 0.f;
                v[u] = u < m ? ld4(P + (int64_t)__ldg(ci + t + u) * ld + col) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (u < m) {
                    FMA4(s, w[u], v[u]);
                }
            }
        }
        s.x += s2.x;
        s.y += s2.y;
        s.z += s2.z;
        s.w += s2.w;
        float4 q;
        if (first) {
            const float4 own = ld4(P + row * ld + col);
            q.x = c1 * own.x - c2 * s.x;
            q.y = c1 * own.y - c2 * s.y;
            q.z = c1 * own.z - c2 * s.z;
            q.w = c1 * own.w - c2 * s.w;
        } else {
            q = ld4v(Q + row * ld + col);
            q.x -= c2 * s.x;
            q.y -= c2 * s.y;
            q.z -= c2 * s.z;
            q.w -= c2 * s.w;
        }
        st4(Q + row * ld + col, q);
    }
}

// ---- column reductions ----
// Every per-column sum of the solve (||r||^2, p^T q, ||y||^2) is formed the
// same way whatever the launch shape: rows are cut into chunks of `rch`
// consecutive rows (rch depends on n only); within a chunk, thread g of 8 sums
// rows g, g + 8, ... in order for one column quad (compensated fp32), the 8
// sums meet in a fixed order in shared memory, and the chunk partials
// [nch][ld] are added in chunk order by the fp64 column kernels.  A column's CG
// scalars are therefore the same bit for bit whatever the slab width, the
// batch width or the other columns of the batch.
constexpr int RG = 8;      // threads per chunk and quad
constexpr int RQ = 128;    // quads per block (at most)

int reduction_chunk_rows(int64_t n) {
    const int64_t r = (n + 4095) / 4096;
    return (int)std::max<int64_t>(512, (r + RG - 1) / RG * RG);
}

// thread -> (chunk = blockIdx.x, quad, g); false when the quad has no column to work on
__device__ __forceinline__ bool red_thread(int64_t n, int32_t ld, int rch, const ColState* st, int64_t& r0,
                                           int64_t& r1, int& col, int& g) {
    const int nq = ld >> 2;
    const int qpb = nq < RQ ? nq : RQ;
    const int quad = blockIdx.y * RQ + (int)threadIdx.x % qpb;
    g = (int)threadIdx.x / qpb;
    col = 4 * quad;
    r0 = (int64_t)blockIdx.x * rch + g;
    r1 = min(n, (int64_t)(blockIdx.x + 1) * rch);
    if (quad >= nq) return false;
    if (!st) return true;
    bool w = false;
#pragma unroll
    for (int c = 0; c < 4; ++c) w |= st[col + c].active;
    return w;
}

// combine the RG partial sums of each quad in g order and store the chunk partial
__device__ __forceinline__ void red_finish(float2* part, int32_t ld, bool work, int col, int g, const KSum (&a)[4]) {
    extern __shared__ float2 red_sm[];  // [RG][qpb * 4]
    const int nq = ld >> 2;
    const int qpb = nq < RQ ? nq : RQ;
    const int ql = (int)threadIdx.x % qpb;
#pragma unroll
    for (int c = 0; c < 4; ++c)
        red_sm[g * qpb * 4 + ql * 4 + c] = work ? make_float2(a[c].s, a[c].c) : make_float2(0.f, 0.f);
    __syncthreads();
    if (g != 0 || !work) return;
    KSum t[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        t[c] = KSum{red_sm[ql * 4 + c].x, red_sm[ql * 4 + c].y};
        for (int h = 1; h < RG; ++h)
            ksum_merge(t[c], KSum{red_sm[h * qpb * 4 + ql * 4 + c].x, red_sm[h * qpb * 4 + ql * 4 + c].y});
    }
    float4* d = reinterpret_cast<float4*>(part + (int64_t)blockIdx.x * ld + col);
    d[0] = make_float4(t[0].s, t[0].c, t[1].s, t[1].c);
    d[1] = make_float4(t[2].s, t[2].c, t[3].s, t[3].c);
}

// Partials of sum_i V_ij^2 (every column).
__global__ void __launch_bounds__(1024) k_colsq(const float* __restrict__ V, int64_t n, int32_t ld, int rch,
                                                float2* __restrict__ part) {
    int64_t r0, r1;
    int col, g;
    const bool work = red_thread(n, ld, rch, nullptr, r0, r1, col, g);
    KSum acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    // four rows' loads issued before their (row-ordered) compensated adds: one
    // load in flight per thread left this single-array pass at half the HBM rate
    if (work)
        for (int64_t row = r0; row < r1; row += 4 * RG) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                v[u] = row + u * RG < r1 ? ld4v(V + (row + u * RG) * ld + col) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (row + u * RG >= r1) break;
                ksum_add(acc[0], v[u].x * v[u].x);
                ksum_add(acc[1], v[u].y * v[u].y);
                ksum_add(acc[2], v[u].z * v[u].z);
                ksum_add(acc[3], v[u].w * v[u].w);
            }
        }
    red_finish(part, ld, work, col, g, acc);
}

// Partials of P^T Q (columns being iterated).
__global__ void __launch_bounds__(1024) k_dot(const float* __restrict__ P, const float* __restrict__ Q, int64_t n,
                                              int32_t ld, int rch, float2* __restrict__ part,
                                              const ColState* __restrict__ st) {
    int64_t r0, r1;
    int col, g;
    const bool work = red_thread(n, ld, rch, st, r0, r1, col, g);
    KSum acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    if (work)
        for (int64_t row = r0; row < r1; row += RG) {
            const float4 a = ld4(P + row * ld + col), b = ld4(Q + row * ld + col);
            ksum_add(acc[0], a.x * b.x);
            ksum_add(acc[1], a.y * b.y);
            ksum_add(acc[2], a.z * b.z);
            ksum_add(acc[3], a.w * b.w);
        }
    red_finish(part, ld, work, col, g, acc);
}

// X += xs a P; R -= a Q; partials of ||R||^2.
__global__ void __launch_bounds__(1024) k_update(float* __restrict__ X, float* __restrict__ R,
                                                 const float* __restrict__ P, const float* __restrict__ Q, int64_t n,
                                                 int32_t ld, int rch, const ColState* __restrict__ st, float xs,
                                                 float2* __restrict__ part) {
    int64_t r0, r1;
    int col, g;
    const bool work = red_thread(n, ld, rch, st, r0, r1, col, g);
    KSum acc[4] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    if (work) {
        const float a0 = (float)st[col].a, a1 = (float)st[col + 1].a, a2 = (float)st[col + 2].a,
                    a3 = (float)st[col + 3].a;
        const float x0 = xs * a0, x1 = xs * a1, x2 = xs * a2, x3 = xs * a3;
        // a served column that took a new request at the last scalar step starts
        // from x0 = 0, r0 = y: x = a p, r = -a q here, y is added next
        const bool f0 = st[col].refill, f1 = st[col + 1].refill, f2 = st[col + 2].refill, f3 = st[col + 3].refill;
        const bool any_refill = f0 | f1 | f2 | f3;
        for (int64_t row = r0; row < r1; row += RG) {
            const int64_t o = row * ld + col;
            const float4 p = ld4v(P + o), q = ld4v(Q + o);
            float4 x = ld4v(X + o), r = ld4v(R + o);
            if (any_refill) {
                if (f0) x.x = r.x = 0.0f;
                if (f1) x.y = r.y = 0.0f;
                if (f2) x.z = r.z = 0.0f;
                if (f3) x.w = r.w = 0.0f;
            }
            x.x = fmaf(x0, p.x, x.x); x.y = fmaf(x1, p.y, x.y); x.z = fmaf(x2, p.z, x.z); x.w = fmaf(x3, p.w, x.w);
            r.x = fmaf(-a0, q.x, r.x); r.y = fmaf(-a1, q.y, r.y); r.z = fmaf(-a2, q.z, r.z); r.w = fmaf(-a3, q.w, r.w);
            st4(X + o, x);
            st4(R + o, r);
            ksum_add(acc[0], r.x * r.x);
            ksum_add(acc[1], r.y * r.y);
            ksum_add(acc[2], r.z * r.z);
            ksum_add(acc[3], r.w * r.w);
        }
    }
    red_finish(part, ld, work, col, g, acc);
}

// P = R + beta P.
template <int S>
__global__ void __launch_bounds__(256) k_direction(float* __restrict__ P, const float* __restrict__ R, int64_t n,
                                                   int32_t ld, const ColState* __restrict__ st) {
    constexpr int L = S / 4;
    constexpr int RPB = 256 / L;
    if (!slab_has_work<S>(st)) return;
    const int g = (threadIdx.x & 31) % L;
    const int col = blockIdx.y * S + 4 * g;
    const float b0 = (float)st[col].beta, b1 = (float)st[col + 1].beta, b2 = (float)st[col + 2].beta,
                b3 = (float)st[col + 3].beta;
    // a served column that just took a new request: p0 = y, added after this
    const bool f0 = st[col].refill, f1 = st[col + 1].refill, f2 = st[col + 2].refill, f3 = st[col + 3].refill;
    for (int64_t row = (int64_t)blockIdx.x * RPB + threadIdx.x / L; row < n; row += (int64_t)gridDim.x * RPB) {
        const int64_t o = row * ld + col;
        const float4 r = ld4v(R + o);
        float4 p = ld4v(P + o);
        p.x = b0 == 0.0f ? (f0 ? 0.0f : r.x) : fmaf(b0, p.x, r.x);
        p.y = b1 == 0.0f ? (f1 ? 0.0f : r.y) : fmaf(b1, p.y, r.y);
        p.z = b2 == 0.0f ? (f2 ? 0.0f : r.z) : fmaf(b2, p.z, r.z);
        p.w = b3 == 0.0f ? (f3 ? 0.0f : r.w) : fmaf(b3, p.w, r.w);
        st4(P + o, p);
    }
}

// ---- per-column scalar kernels: one block per column, fp64 reductions ----
// Block-wide fp64 sum (all threads get the result).
__device__ __forceinline__ double block_sum_f64(double v) {
    __shared__ double sm[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sm[w] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sm[i];
    return t;
}

// sum over blocks of column j's compensated partials
__device__ __forceinline__ double col_sum(const float2* part, int nblk, int ld, int j) {
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        const float2 v = part[(int64_t)b * ld + j];
        s += (double)v.x + (double)v.y;
    }
    return block_sum_f64(s);
}

// sum_k coef_k C_kj^2
__device__ __forceinline__ double col_lowrank(const double* C, const double* coef, int r, int ld, int j) {
    double s = 0.0;
    if (C)
        for (int k = threadIdx.x; k < r; k += blockDim.x) {
            const double c = C[(int64_t)k * ld + j];
            s += coef[k] * c * c;
        }
    return block_sum_f64(s);
}

// Setup: bb = ||b||^2; rho = bb (+ sum D C^2 for PCG); activity and 0-iteration convergence.
__global__ void k_fin_setup(const float2* part, int nblk, int32_t Bp, int32_t B, const float* tol, ColState* st,
                            const double* C, const double* coef, int32_t r, int* num_active) {
    const int j = blockIdx.x;
    const double bb = col_sum(part, nblk, Bp, j);
    const double lrt = col_lowrank(C, coef, r, Bp, j);
    if (threadIdx.x != 0) return;
    ColState s;
    s.bb = bb;
    s.rr = bb;
    s.rho = bb + lrt;
    const double t = j < B ? (double)tol[j] : 0.0;
    s.tol2 = t * t * bb;
    s.sigma = 0.0;
    s.a = 0.0;
    s.beta = 0.0;
    s.iters = 0;
    s.confirms = 0;
    s.restart = 0;
    s.refill = 0;
    s.free_col = 0;
    s.rr_fix = 0.0;
    if (j >= B || bb == 0.0) {
        s.active = 0;
        s.status = HD_COL_EMPTY;
    } else if (bb <= s.tol2) {
        s.active = 0;
        s.status = HD_COL_CONVERGED;
    } else {
        s.active = 1;
        s.status = HD_COL_MAX_ITER;
        atomicAdd(num_active, 1);
    }
    st[j] = s;
}

// a = rho / sigma with sigma = SpMM partials (+ sum_k coef_k C_k^2).
__global__ void k_fin_sigma(const float2* part, int nblk, int32_t Bp, ColState* st, const double* C,
                            const double* coef, int32_t r) {
    const int j = blockIdx.x;
    ColState& s = st[j];
    if (!s.active) {
        if (threadIdx.x == 0) s.a = 0.0;
        return;
    }
    const double sig = col_sum(part, nblk, Bp, j) + col_lowrank(C, coef, r, Bp, j);
    if (threadIdx.x != 0) return;
    s.sigma = sig;
    if (!(sig > 0.0) || !isfinite(sig)) {
        s.active = 0;
        s.status = HD_COL_BREAKDOWN;
        s.a = 0.0;
    } else {
        s.a = s.rho / sig;
    }
}

// After the update: rr, convergence, beta.  With C: PCG rho' = rr + sum_k coef_k C_k^2.
// num_active must be zero before the launch.
// use_half (may be null; 1 before the launch): cleared when a column that stays
// active has ||r||^2 > theta2 tol^2 ||b||^2 (the next SpMM then gathers fp32).
__global__ void k_fin_rr(const float2* part, int nblk, int32_t Bp, ColState* st, int32_t max_iter,
                         const double* C, const double* coef, int32_t r, int* num_active, int* use_half = nullptr,
                         double theta2 = 0.0) {
    const int j = blockIdx.x;
    ColState& s = st[j];
    if (!s.active) {
        if (threadIdx.x == 0) s.beta = 0.0;
        return;
    }
    const double rr = col_sum(part, nblk, Bp, j);
    const double lrt = col_lowrank(C, coef, r, Bp, j);
    if (threadIdx.x != 0) return;
    const double rho = rr + lrt;
    s.iters += 1;
    s.rr = rr;
    s.beta = rho / s.rho;
    s.rho = rho;
    if (!isfinite(rr)) {
        s.active = 0;
        s.status = HD_COL_BREAKDOWN;
        s.beta = 0.0;
    } else if (rr <= s.tol2) {
        s.active = 0;
        s.status = HD_COL_CONVERGED;
    } else if (s.iters >= max_iter) {
        s.active = 0;
        s.status = HD_COL_MAX_ITER;
    } else {
        atomicAdd(num_active, 1);
        if (use_half && !(rr <= theta2 * s.tol2)) atomicExch(use_half, 0);
    }
}

// sum_k coef_k c_k^2 for one contiguous row c (block-wide)
__device__ __forceinline__ double row_lowrank(const double* c, const double* coef, int r) {
    double v = 0.0;
    if (c)
        for (int k = threadIdx.x; k < r; k += blockDim.x) v += coef[k] * c[k] * c[k];
    return block_sum_f64(v);
}

// The scalar step of a server lane (k_fin_rr plus admission inside the
// iteration).  A free column the host assigned (the lowest free ones, so that
// the occupied columns stay packed) takes its staged request, and a column that
// stops here claims the next unassigned one: the stopped request's iterations,
// status and ||r||^2 go to the
// host, the column restarts as the new request (r0 = y, rho = y^T M^-1 y from
// the staged U^T y) with `refill` set, so that the direction that follows
// forms p0 = M^-1 y and the next update starts x and r afresh.  A stopped
// column that claims nothing becomes free once the host has its ranking.
// A refilled column's first ||r||^2 adds rr_fix (the y entries, exact).
__global__ void k_fin_rr_serve(const float2* part, int nblk, int32_t Bp, ColState* st, int32_t max_iter,
                               const double* C, const double* coef, int32_t r, int* num_active, Refill rf) {
    __shared__ int claim;
    const int j = blockIdx.x;
    ColState& s = st[j];
    const bool active = s.active, was_free = s.free_col;
    if (!active && !was_free) {
        if (threadIdx.x == 0) s.beta = 0.0;
        return;
    }
    double rr = 0.0, lrt = 0.0;
    if (active) {
        rr = col_sum(part, nblk, Bp, j);
        lrt = col_lowrank(C, coef, r, Bp, j);
    }
    if (threadIdx.x == 0) {
        claim = -1;
        bool stopped = was_free;
        if (active) {
            if (s.refill) {
                rr += s.rr_fix;
                s.refill = 0;
            }
            const double rho = rr + lrt;
            s.iters += 1;
            s.rr = rr;
            s.beta = rho / s.rho;
            s.rho = rho;
            stopped = true;
            if (!isfinite(rr)) {
                s.active = 0;
                s.status = HD_COL_BREAKDOWN;
                s.beta = 0.0;
            } else if (rr <= s.tol2) {
                s.active = 0;
                s.status = HD_COL_CONVERGED;
            } else if (s.iters >= max_iter) {
                s.active = 0;
                s.status = HD_COL_MAX_ITER;
            } else {
                stopped = false;
                atomicAdd(num_active, 1);
            }
        }
        if (stopped) {
            // a free column the host assigned takes its request; a column that
            // stops here (or stopped earlier in the step) the next unassigned one
            const int ns = *rf.nstage;
            int c = INT_MAX;
            if (ns > 0) {
                const int pc = rf.pre[j];
                c = pc >= 0 ? pc : j < rf.live ? atomicAdd(rf.next, 1) : INT_MAX;
            }
            if (c < ns) claim = c;
            else if (active) s.free_col = 1;
        }
    }
    __syncthreads();
    const int c = claim;
    if (c < 0) return;
    const double lrs = row_lowrank(rf.C ? rf.C + (int64_t)c * rf.rpad : nullptr, coef, r);
    if (threadIdx.x != 0) return;
    // the request the column held (stopped here or at an earlier step's
    // iteration; the host ignores these for a column it holds as free)
    rf.ret_iters[j] = s.iters;
    rf.ret_status[j] = s.status;
    rf.ret_rr[j] = s.rr;
    rf.assign[j] = c;
    s.bb = rf.bb[c];
    s.tol2 = rf.tol2[c];
    s.rr = s.bb;
    s.rho = s.bb + lrs;
    s.beta = 0.0;
    s.a = 0.0;
    s.iters = 0;
    s.confirms = 0;
    s.restart = 0;
    s.rr_fix = 0.0;
    s.active = 1;
    s.free_col = 0;
    s.refill = 1;
    s.status = HD_COL_MAX_ITER;
    atomicAdd(num_active, 1);
}

// H = coef o (U^T y) for the columns that took a staged request (the operand
// of the direction's U H; the other columns keep theirs)
__global__ void k_refill_h(Refill rf, const double* coef, int rpad, int32_t Bp, float* H, __nv_bfloat16* Hhi,
                           __nv_bfloat16* Hlo) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)rpad * Bp) return;
    const int k = (int)(e / Bp), j = (int)(e % Bp);
    const int c = rf.assign[j];
    if (c < 0) return;
    const double h = coef[k] * rf.C[(int64_t)c * rpad + k];
    H[e] = (float)h;
    if (Hhi) {
        const __nv_bfloat16 hi = __double2bfloat16(h);
        const __nv_bfloat16 lo = __double2bfloat16(h - (double)__bfloat162float(hi));
        Hhi[(int64_t)j * rpad + k] = hi;
        Hlo[(int64_t)j * rpad + k] = lo;
    }
}

// p0 += y for the columns that took a staged request (the direction left
// U D U^T y there, or 0 without eigenpairs); y is kept with the column for its
// first update
__global__ void k_refill_p(Refill rf, float* P, int32_t Bp) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= Bp) return;
    const int c = rf.assign[j];
    if (c < 0) return;
    const int32_t b = rf.off[c], e = rf.off[c + 1];
    for (int32_t t = b; t < e; ++t) {
        const int32_t i = rf.yidx[t];
        const float v = rf.yval[t];
        P[(int64_t)i * Bp + j] += v;
        rf.col_idx[(int64_t)j * REFILL_MAX_NNZ + (t - b)] = i;
        rf.col_val[(int64_t)j * REFILL_MAX_NNZ + (t - b)] = v;
    }
    rf.col_cnt[j] = e - b;
}

// After the first update of a refilled column (r = -a q): r += y, and rr_fix =
// sum over y's entries of (r_i + y_i)^2 - r_i^2 (fp64; duplicates in turn)
__global__ void k_refill_r(Refill rf, float* R, int32_t Bp, ColState* st) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= Bp || !st[j].refill) return;
    double fix = 0.0;
    for (int t = 0; t < rf.col_cnt[j]; ++t) {
        float* a = R + (int64_t)rf.col_idx[(int64_t)j * REFILL_MAX_NNZ + t] * Bp + j;
        const float v = *a;
        const float w = v + rf.col_val[(int64_t)j * REFILL_MAX_NNZ + t];
        *a = w;
        fix += (double)w * (double)w - (double)v * (double)v;
    }
    st[j].rr_fix = fix;
}

int launch_refill_r(Engine& E) {
    k_refill_r<<<ceil_div(E.Bp, 128), 128, 0, E.ctx->stream>>>(*E.refill, E.R, E.Bp, E.st);
    HD_CHECK_LAUNCH(E.ctx);
    return HD_OK;
}

// Which residual kernel runs: the fp32 evaluation of b - A x has an error of
// at most (c2 gamma_m + 2 u c1) ||x|| + 2 u ||b|| (u = 2^-24; gamma_m = m u /
// (1 - m u) bounds the rounding of a sum of m products, m the longest row
// plus one; ||W|x||| <= ||x|| for the nonnegative W of spectral radius 1).
// When that is at most a tenth of tol ||b|| for every column, the fp32 SpMM
// runs (*pick = 0), else the two-word kernel (*pick = 1).  part: partials of
// ||x_j||^2; one block per column.
__global__ void k_resid_pick(const float2* part, int nblk, int32_t Bp, int32_t B, const ColState* st, double gamma,
                             double c1, double c2, int* pick) {
    const int j = blockIdx.x;
    if (j >= B) return;
    const double xx = col_sum(part, nblk, Bp, j);
    if (threadIdx.x != 0) return;
    const ColState& s = st[j];
    if (s.status == HD_COL_EMPTY || s.status == HD_COL_CANCELLED || s.bb <= 0.0) return;
    const double u = 1.0 / 16777216.0;
    const double bound = (c2 * gamma + 2.0 * u * c1) * sqrt(xx) + 2.0 * u * sqrt(s.bb);
    // tol2 = tol^2 ||b||^2
    if (!(bound <= 0.1 * sqrt(s.tol2))) atomicExch(pick, 1);
}

// ---- confirmation by the true residual (x0 = 0 and a residual stopping rule, Sec. 4.4)
// Residual replacements allowed per column and solve.
constexpr int MAX_CONFIRM = 3;

// part: partials of ||T||^2, T = b - A x (every column).  rr := ||T||^2, the
// value the solve reports.  A column whose recursive residual met tol while
// ||T|| > tol ||b|| is reactivated with r := T (flag `restart`) while it has
// iterations and replacements left; otherwise it is STAGNATED.
__global__ void k_fin_confirm(const float2* part, int nblk, int32_t Bp, int32_t B, ColState* st, int32_t max_iter,
                              int* num_active) {
    const int j = blockIdx.x;
    ColState& s = st[j];
    if (j >= B || s.status == HD_COL_EMPTY || s.status == HD_COL_CANCELLED) return;
    const double tt = col_sum(part, nblk, Bp, j);
    if (threadIdx.x != 0) return;
    s.rr = tt;
    s.restart = 0;
    if (!isfinite(tt)) {
        s.status = HD_COL_BREAKDOWN;
        return;
    }
    if (s.status != HD_COL_CONVERGED || tt <= s.tol2) return;
    if (s.iters < max_iter && s.confirms < MAX_CONFIRM) {
        s.confirms += 1;
        s.active = 1;
        s.status = HD_COL_MAX_ITER;
        s.restart = 1;
        atomicAdd(num_active, 1);
    } else {
        s.status = HD_COL_STAGNATED;
    }
}

// R[:, j] := T[:, j] for the columns being restarted.
__global__ void k_restart_copy(float* __restrict__ R, const float* __restrict__ T, int64_t n, int32_t ld,
                               const ColState* __restrict__ st) {
    const int nq = ld >> 2;
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // float4 index = row * nq + quad
    if (e >= n * nq) return;
    const int col = 4 * (int)(e % nq);
    const int m = st[col].restart | st[col + 1].restart << 1 | st[col + 2].restart << 2 | st[col + 3].restart << 3;
    if (!m) return;
    float4 r = ld4v(R + 4 * e);
    const float4 t = ld4v(T + 4 * e);
    if (m & 1) r.x = t.x;
    if (m & 2) r.y = t.y;
    if (m & 4) r.z = t.z;
    if (m & 8) r.w = t.w;
    st4(R + 4 * e, r);
}

// Restarted columns: rho = ||r||^2 (+ sum_k coef_k C_k^2 with the
// preconditioner, C = U^T r), a fresh direction (beta = 0); every other
// column gets beta = 0 so the direction update leaves it finite.
__global__ void k_fin_restart(ColState* st, const double* C, const double* coef, int32_t r) {
    const int j = blockIdx.x;
    ColState& s = st[j];
    if (!s.restart) {
        if (threadIdx.x == 0) s.beta = 0.0;
        return;
    }
    const double lrt = col_lowrank(C, coef, r, gridDim.x, j);
    if (threadIdx.x != 0) return;
    s.rho = s.rr + lrt;
    s.beta = 0.0;
    s.a = 0.0;
    s.restart = 0;
}

// C [rpad][Bp] (fp64) given directly: H = coef o C (fp32 and bf16 hi/lo
// transposed), the operand layout lr_finish produces from partials.
__global__ void k_lr_coef(const double* __restrict__ Csrc, int rpad, int32_t Bp, const double* __restrict__ coef,
                          float* H, __nv_bfloat16* Hhi, __nv_bfloat16* Hlo) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)rpad * Bp) return;
    const int k = (int)(e / Bp), j = (int)(e % Bp);
    const double h = coef[k] * Csrc[e];
    H[e] = (float)h;
    if (Hhi) {
        const __nv_bfloat16 hi = __double2bfloat16(h);
        const __nv_bfloat16 lo = __double2bfloat16(h - (double)__bfloat162float(hi));
        Hhi[(int64_t)j * rpad + k] = hi;
        Hlo[(int64_t)j * rpad + k] = lo;
    }
}

__global__ void k_outputs(const ColState* st, int32_t B, int32_t* iters, float* relres, int32_t* status) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= B) return;
    ColState s = st[j];
    if (iters) iters[j] = s.iters;
    if (relres) relres[j] = s.bb > 0.0 ? (float)sqrt(s.rr / s.bb) : 0.0f;
    if (status) status[j] = s.status;
}

__global__ void k_copy_out(const float* Xi, int32_t Bp, float* X, int32_t ldx, int32_t B, int64_t n) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * B) return;
    int64_t i = e / B;
    int j = (int)(e % B);
    X[i * ldx + j] = Xi[i * Bp + j];
}

// ------------------------------------------------------------------ low-rank, CUDA cores
template <typename T>
__device__ __forceinline__ float u_at(const T* U, const float* scale, int64_t i, int ldu, int k);
template <>
__device__ __forceinline__ float u_at<float>(const float* U, const float*, int64_t i, int ldu, int k) {
    return __ldg(U + i * ldu + k);
}
template <>
__device__ __forceinline__ float u_at<__nv_bfloat16>(const __nv_bfloat16* U, const float*, int64_t i, int ldu, int k) {
    return __bfloat162float(U[i * ldu + k]);
}
template <>
__device__ __forceinline__ float u_at<__nv_fp8_e4m3>(const __nv_fp8_e4m3* U, const float* scale, int64_t i, int ldu,
                                                      int k) {
    return float(U[i * ldu + k]) * __ldg(scale + i);
}

// part[c][k][j] = sum_{i in chunk c} U_ik V_ij ; grid (chunk, k-block of 64, 16-column slab)
template <typename T>
__global__ void __launch_bounds__(256) k_lr_reduce_simt(const T* __restrict__ U, const float* __restrict__ scale,
                                                        int ldu, int r, int rpad, const float* __restrict__ V,
                                                        int64_t n, int32_t Bp, int64_t rpc,
                                                        float* __restrict__ part, const int* gate) {
    if (gate && *gate == 0) return;
    const int kk = threadIdx.x >> 2, cq = 4 * (threadIdx.x & 3);
    const int k = blockIdx.y * 64 + kk;
    const int col = blockIdx.z * 16 + cq;
    const int64_t i0 = (int64_t)blockIdx.x * rpc;
    const int64_t i1 = min(n, i0 + rpc);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (k < r && col < Bp)
        for (int64_t i = i0; i < i1; ++i) {
            const float u = u_at<T>(U, scale, i, ldu, k);
            const float4 v = ld4(V + i * Bp + col);
            acc.x = fmaf(u, v.x, acc.x);
            acc.y = fmaf(u, v.y, acc.y);
            acc.z = fmaf(u, v.z, acc.z);
            acc.w = fmaf(u, v.w, acc.w);
        }
    if (k < rpad && col < Bp) st4(part + ((int64_t)blockIdx.x * rpad + k) * Bp + col, acc);
}

// C = sum over chunks (fp64); H = coef o C (fp32 and bf16 hi/lo transposed).
// Block: 32 consecutive entries x 8 warps splitting the chunks.
__global__ void __launch_bounds__(256) k_lr_finish(const float* __restrict__ part, int nchunk, int rpad, int32_t Bp,
                                                   const double* coef, double* C, float* H, __nv_bfloat16* Hhi,
                                                   __nv_bfloat16* Hlo) {
    __shared__ double sm[8][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t e = (int64_t)blockIdx.x * 32 + lane;
    const int64_t tot = (int64_t)rpad * Bp;
    double s = 0.0;
    if (e < tot)
        for (int c = w; c < nchunk; c += 8) s += (double)part[(int64_t)c * tot + e];
    sm[w][lane] = s;
    __syncthreads();
    if (w != 0 || e >= tot) return;
    s = 0.0;
    for (int i = 0; i < 8; ++i) s += sm[i][lane];
    const int k = (int)(e / Bp), j = (int)(e % Bp);
    C[e] = s;
    const double h = coef[k] * s;
    H[e] = (float)h;
    if (Hhi) {
        const __nv_bfloat16 hi = __double2bfloat16(h);
        const __nv_bfloat16 lo = __double2bfloat16(h - (double)__bfloat162float(hi));
        Hhi[(int64_t)j * rpad + k] = hi;
        Hlo[(int64_t)j * rpad + k] = lo;
    }
}

// out = op(U H) for the 16-column slab blockIdx.y; H staged in shared memory.
template <typename T>
__global__ void __launch_bounds__(256) k_lr_expand_simt(const T* __restrict__ U, const float* __restrict__ scale,
                                                        int ldu, int r, const float* __restrict__ H, int op,
                                                        float* __restrict__ out, const float* __restrict__ Rv,
                                                        const float* __restrict__ Pv, int64_t n, int32_t Bp,
                                                        const ColState* __restrict__ st, const int* gate) {
    if (gate && *gate == 0) return;
    extern __shared__ float Hs[];  // [r][16]
    const int slab = blockIdx.y;
    for (int e = threadIdx.x; e < r * 16; e += blockDim.x) {
        const int k = e >> 4, c = e & 15;
        Hs[e] = (slab * 16 + c < Bp) ? H[(int64_t)k * Bp + slab * 16 + c] : 0.0f;
    }
    __syncthreads();
    const int cq = 4 * (threadIdx.x & 3);
    const int col = slab * 16 + cq;
    if (col >= Bp) return;
    float b0 = 0.f, b1 = 0.f, b2 = 0.f, b3 = 0.f;
    bool f0 = false, f1 = false, f2 = false, f3 = false;
    if (op == EXP_DIRECTION) {
        b0 = (float)st[col].beta;
        b1 = (float)st[col + 1].beta;
        b2 = (float)st[col + 2].beta;
        b3 = (float)st[col + 3].beta;
        // a served column that just took a new request drops r (p0 = U D U^T y + y)
        f0 = st[col].refill;
        f1 = st[col + 1].refill;
        f2 = st[col + 2].refill;
        f3 = st[col + 3].refill;
    }
    for (int64_t row = (int64_t)blockIdx.x * 64 + (threadIdx.x >> 2); row < n; row += (int64_t)gridDim.x * 64) {
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int k = 0; k < r; ++k) {
            const float u = u_at<T>(U, scale, row, ldu, k);
            const float4 h = *reinterpret_cast<const float4*>(Hs + k * 16 + cq);
            acc.x = fmaf(u, h.x, acc.x);
            acc.y = fmaf(u, h.y, acc.y);
            acc.z = fmaf(u, h.z, acc.z);
            acc.w = fmaf(u, h.w, acc.w);
        }
        const int64_t o = row * Bp + col;
        float4 v;
        if (op == EXP_SET_X) {
            v = acc;
        } else if (op == EXP_SUB_R) {
            v = ld4v(out + o);
            v.x -= acc.x; v.y -= acc.y; v.z -= acc.z; v.w -= acc.w;
        } else if (op == EXP_ADD_Q) {
            v = ld4v(out + o);
            v.x += acc.x; v.y += acc.y; v.z += acc.z; v.w += acc.w;
        } else {
            const float4 rr = ld4v(Rv + o), pp = ld4v(Pv + o);
            v.x = (f0 ? 0.0f : rr.x) + acc.x + (b0 == 0.0f ? 0.0f : b0 * pp.x);
            v.y = (f1 ? 0.0f : rr.y) + acc.y + (b1 == 0.0f ? 0.0f : b1 * pp.y);
            v.z = (f2 ? 0.0f : rr.z) + acc.z + (b2 == 0.0f ? 0.0f : b2 * pp.z);
            v.w = (f3 ? 0.0f : rr.w) + acc.w + (b3 == 0.0f ? 0.0f : b3 * pp.w);
        }
        st4(out + o, v);
    }
}

int simt_nchunk(hd_ctx* ctx, int64_t n, int rpad, int Bp) {
    int blocks_per_chunk = (rpad / 64) * ceil_div(Bp, 16);
    int nc = ceil_div(4 * ctx->num_sms, blocks_per_chunk);
    int64_t maxc = std::max<int64_t>(1, n / 64);
    return (int)std::max<int64_t>(1, std::min<int64_t>(nc, maxc));
}

int lr_nchunk(hd_ctx* ctx, const hd_eig* e, int32_t Bp) {
    if (e->sparse) return lr_sparse_nchunk(ctx, e);
    return lr_use_tensor_cores(e) ? lr_tc_nchunk(ctx, e->n) : simt_nchunk(ctx, e->n, (e->r + 63) / 64 * 64, Bp);
}

int lr_reduce(hd_ctx* ctx, const LowRank& lr, const float* V, int64_t n, int32_t Bp, const int* gate) {
    HD_PROF(ctx, "lr_reduce");
    if (lr.e->sparse) return lr_sparse_reduce(ctx, lr, V, n, Bp, gate);
    if (lr_use_tensor_cores(lr.e)) return lr_tc_reduce(ctx, lr, V, n, Bp, gate);
    const hd_eig* e = lr.e;
    int64_t rpc = (n + lr.nchunk - 1) / lr.nchunk;
    dim3 grid(lr.nchunk, lr.rpad / 64, ceil_div(Bp, 16));
    if (e->storage == HD_F32)
        k_lr_reduce_simt<float><<<grid, 256, 0, ctx->stream>>>((const float*)e->U, e->scale, e->ldu, e->r, lr.rpad, V,
                                                               n, Bp, rpc, lr.part, gate);
    else if (e->storage == HD_BF16)
        k_lr_reduce_simt<__nv_bfloat16><<<grid, 256, 0, ctx->stream>>>((const __nv_bfloat16*)e->U, e->scale, e->ldu,
                                                                       e->r, lr.rpad, V, n, Bp, rpc, lr.part, gate);
    else
        k_lr_reduce_simt<__nv_fp8_e4m3><<<grid, 256, 0, ctx->stream>>>((const __nv_fp8_e4m3*)e->U, e->scale, e->ldu,
                                                                       e->r, lr.rpad, V, n, Bp, rpc, lr.part, gate);
    HD_CHECK_LAUNCH(ctx);
    return HD_OK;
}

int lr_finish(hd_ctx* ctx, const LowRank& lr, int32_t Bp, const double* coef) {
    HD_PROF(ctx, "scalar");
    int64_t tot = (int64_t)lr.rpad * Bp;
    k_lr_finish<<<ceil_div(tot, 32), 256, 0, ctx->stream>>>(lr.part, lr.nchunk, lr.rpad, Bp, coef, lr.C,
                                                             lr.H, lr.Hhi, lr.Hlo);
    HD_CHECK_LAUNCH(ctx);
    return HD_OK;
}

// H = coef o Csrc for a C kept from earlier (the operand of lr_expand)
static int lr_coef(hd_ctx* ctx, const LowRank& lr, int32_t Bp, const double* coef, const double* Csrc) {
    HD_PROF(ctx, "scalar");
    const int64_t tot = (int64_t)lr.rpad * Bp;
    k_lr_coef<<<ceil_div(tot, 256), 256, 0, ctx->stream>>>(Csrc, lr.rpad, Bp, coef, lr.H, lr.Hhi, lr.Hlo);
    HD_CHECK_LAUNCH(ctx);
    return HD_OK;
}

int lr_expand(hd_ctx* ctx, const LowRank& lr, int op, float* out, const float* Rv, const float* Pv, int64_t n,
              int32_t Bp, const ColState* st, const int* gate) {
    HD_PROF(ctx, "lr_expand");
    if (lr.e->sparse) return lr_sparse_expand(ctx, lr, op, out, Rv, Pv, n, Bp, st, gate);
    if (lr_use_tensor_cores(lr.e)) return lr_tc_expand(ctx, lr, op, out, Rv, Pv, n, Bp, st, gate);
    const hd_eig* e = lr.e;
    size_t smem = (size_t)e->r * 16 * sizeof(float);
    int gx = (int)std::min<int64_t>(ceil_div(n, 64), (int64_t)ctx->num_sms * 8);
    dim3 grid(gx, ceil_div(Bp, 16));
    static uint64_t attr = 0;
    if (hd_first_on_device(attr, ctx->device)) {
        cudaFuncSetAttribute(k_lr_expand_simt<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024 + 1024);
        cudaFuncSetAttribute(k_lr_expand_simt<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024 + 1024);
        cudaFuncSetAttribute(k_lr_expand_simt<__nv_fp8_e4m3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024 + 1024);
    }
    if (e->storage == HD_F32)
        k_lr_expand_simt<float><<<grid, 256, smem, ctx->stream>>>((const float*)e->U, e->scale, e->ldu, e->r, lr.H, op,
                                                                  out, Rv, Pv, n, Bp, st, gate);
    else if (e->storage == HD_BF16)
        k_lr_expand_simt<__nv_bfloat16><<<grid, 256, smem, ctx->stream>>>(
            (const __nv_bfloat16*)e->U, e->scale, e->ldu, e->r, lr.H, op, out, Rv, Pv, n, Bp, st, gate);
    else
        k_lr_expand_simt<__nv_fp8_e4m3><<<grid, 256, smem, ctx->stream>>>(
            (const __nv_fp8_e4m3*)e->U, e->scale, e->ldu, e->r, lr.H, op, out, Rv, Pv, n, Bp, st, gate);
    HD_CHECK_LAUNCH(ctx);
    return HD_OK;
}

// ------------------------------------------------------------------ launch helpers


static int pick_slab(int32_t Bp) {
    static int forced = -1;
    if (forced < 0) {
        const char* s = getenv("HD_SLAB");
        forced = s ? atoi(s) : 0;
    }
    int cands[] = {128, 64, 32, 16, 8, 4};
    for (int S : cands)
        if ((forced == 0 || S <= forced) && Bp % S == 0) return S;
    return 4;
}

VecLaunch vec_launch(hd_ctx* ctx, int64_t n, int32_t Bp, int S) {
    VecLaunch v;
    v.S = S > 0 ? S : pick_slab(Bp);
    int rpb = 256 / (v.S / 4);
    v.slabs = Bp / v.S;
    v.nblk = (int)std::min<int64_t>(ceil_div(n, rpb), (int64_t)ctx->num_sms * 8);
    if (v.nblk < 1) v.nblk = 1;
    return v;
}

#define HD_DISPATCH_S(S, ...)                  \
    switch (S) {                               \
        case 4: { constexpr int SS = 4; __VA_ARGS__; } break;     \
        case 8: { constexpr int SS = 8; __VA_ARGS__; } break;     \
        case 16: { constexpr int SS = 16; __VA_ARGS__; } break;   \
        case 32: { constexpr int SS = 32; __VA_ARGS__; } break;   \
        case 64: { constexpr int SS = 64; __VA_ARGS__; } break;   \
        default: { constexpr int SS = 128; __VA_ARGS__; } break;  \
    }

int tune_slab(hd_ctx* ctx, const hd_graph* g, int32_t Bp, const float* P, float* Q) {
    auto it = g->slab_cache.find(Bp);
    if (it != g->slab_cache.end()) return it->second;
    if (getenv("HD_SLAB")) return g->slab_cache[Bp] = pick_slab(Bp);
    int best = pick_slab(Bp);
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int S : {8, 16, 32, 64, 128}) {
        if (Bp % S || (S == 8 && Bp > 8 && g->n < 4096)) continue;
        VecLaunch v = vec_launch(ctx, g->n, Bp, S);
        dim3 grid(v.nblk, v.slabs);
        float tot = 0.f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, ctx->stream);
            HD_DISPATCH_S(S, (k_spmm<SS><<<grid, 256, 0, ctx->stream>>>(g->row_ptr, g->col, g->val, P, Q, g->n, Bp,
                                                                         1.f, 1.f, nullptr)));
            cudaEventRecord(e1, ctx->stream);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep) tot += ms;
        }
        ctx->launches += 3;
        if (tot < best_ms * 0.97f) {
            best_ms = tot;
            best = S;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    g->slab_cache[Bp] = best;
    return best;
}

int hd_spmm_apply(hd_ctx* ctx, const hd_graph* g, const float* P, float* Q, int32_t ld, int32_t B, float c1,
                  float c2) {
    VecLaunch v = vec_launch(ctx, g->n, ld);
    dim3 grid(v.nblk, v.slabs);
    HD_DISPATCH_S(v.S, (k_spmm<SS><<<grid, 256, 0, ctx->stream>>>(g->row_ptr, g->col, g->val, P, Q, g->n, ld, c1, c2,
                                                                   nullptr)));
    HD_CHECK_LAUNCH(ctx);
    return HD_OK;
}

// grid and block of the column reductions: one block row per chunk, up to 128 quads x 8 threads
static inline dim3 red_grid(const Engine& E) {
    const int nq = E.Bp / 4;
    return dim3((unsigned)E.nch, (unsigned)ceil_div(nq, RQ));
}
static inline unsigned red_block(const Engine& E) {
    const int nq = E.Bp / 4;
    return (unsigned)(RG * (nq < RQ ? nq : RQ));
}
static inline size_t red_smem(const Engine& E) { return (size_t)red_block(E) * 4 * sizeof(float2); }

static int launch_dot(Engine& E, float2* part, const ColState* st) {
    hd_ctx* ctx = E.ctx;
    HD_PROF(ctx, "dot");
    k_dot<<<red_grid(E), red_block(E), red_smem(E), ctx->stream>>>(E.P, E.Q, E.n, E.Bp, E.rch, part, st);
    HD_CHECK_LAUNCH(ctx);
    return HD_OK;
}

static int launch_update(Engine& E) {
    hd_ctx* ctx = E.ctx;
    HD_PROF(ctx, "update");
    k_update<<<red_grid(E), red_block(E), red_smem(E), ctx->stream>>>(E.X, E.R, E.P, E.Q, E.n, E.Bp, E.rch, E.st, E.xs, E.part);
    HD_CHECK_LAUNCH(ctx);
    return HD_OK;
}

static int launch_colsq(Engine& E, const float* V) {
    hd_ctx* ctx = E.ctx;
    HD_PROF(ctx, "colsq");
    k_colsq<<<red_grid(E), red_block(E), red_smem(E), ctx->stream>>>(V, E.n, E.Bp, E.rch, E.part);
    HD_CHECK_LAUNCH(ctx);
    return HD_OK;
}

void engine_set_reduction(Engine& E) {
    E.rch = reduction_chunk_rows(E.n);
    E.nch = (E.n + E.rch - 1) / E.rch;
}

// Q = c1 V - c2 W V (V = P unless given) with the engine's slab width and
// segments (+ P^T Q partials)
static int launch_spmm(Engine& E, float c1, float c2, float2* part, const ColState* st, const float* V = nullptr) {
    hd_ctx* ctx = E.ctx;
    const hd_graph* g = E.g;
    const float* Pin = V ? V : E.P;
    dim3 grid(E.vl.nblk, E.vl.slabs);
    if (!V && E.use_half) {
        // the iteration's SpMM: an fp16 copy of P is gathered when *use_half
        // (columns 8 per lane; 64-column slabs make a row's slab 128 bytes)
        const int S16 = E.Bp % 64 == 0 ? 64 : E.Bp % 32 == 0 ? 32 : E.Bp % 16 == 0 ? 16 : 8;
        const int nq = E.Bp / 4;
        const int rpb = 256 / nq;
        const dim3 gc((unsigned)std::min<int64_t>(ceil_div(E.n, rpb), (int64_t)ctx->num_sms * 8));
        const int rpb16 = 256 / (S16 / 8);
        const dim3 gh((unsigned)std::min<int64_t>(ceil_div(E.n, rpb16), (int64_t)ctx->num_sms * 4),
                      (unsigned)(E.Bp / S16));
        {
            HD_PROF(ctx, "to_half");
            HD_CUDA(ctx, cudaMemsetAsync(E.p16_max, 0, (size_t)E.Bp * sizeof(unsigned), ctx->stream));
            k_colmax<<<gc, 256, 0, ctx->stream>>>(E.P, E.n, E.Bp, E.p16_max, E.use_half, E.num_active);
            HD_CHECK_LAUNCH(ctx);
            k_to_half<<<gc, 256, 0, ctx->stream>>>(E.P, E.n, E.Bp, E.p16_max, E.P16, E.use_half, E.num_active);
            HD_CHECK_LAUNCH(ctx);
        }
        {
            HD_PROF(ctx, "spmm");
            HD_DISPATCH_S(E.vl.S, (k_spmm<SS><<<grid, 256, 0, ctx->stream>>>(g->row_ptr, g->col, g->val, E.P, E.Q, E.n,
                                                                              E.Bp, c1, c2, st, E.use_half)));
            HD_CHECK_LAUNCH(ctx);
        }
        {
            HD_PROF(ctx, "spmm_h");
            switch (S16) {
                case 64: k_spmm_h<64><<<gh, 256, 0, ctx->stream>>>(g->row_ptr, g->col, g->val, E.P16, E.p16_max, E.P,
                                                                    E.Q, E.n, E.Bp, c1, c2, st, E.use_half); break;
                case 32: k_spmm_h<32><<<gh, 256, 0, ctx->stream>>>(g->row_ptr, g->col, g->val, E.P16, E.p16_max, E.P,
                                                                    E.Q, E.n, E.Bp, c1, c2, st, E.use_half); break;
                case 16: k_spmm_h<16><<<gh, 256, 0, ctx->stream>>>(g->row_ptr, g->col, g->val, E.P16, E.p16_max, E.P,
                                                                    E.Q, E.n, E.Bp, c1, c2, st, E.use_half); break;
                default: k_spmm_h<8><<<gh, 256, 0, ctx->stream>>>(g->row_ptr, g->col, g->val, E.P16, E.p16_max, E.P,
                                                                   E.Q, E.n, E.Bp, c1, c2, st, E.use_half); break;
            }
            HD_CHECK_LAUNCH(ctx);
        }
        if (part) return launch_dot(E, part, st);
        return HD_OK;
    }
    {
        HD_PROF(ctx, "spmm");
        if (E.segK <= 1 && E.Bp == 4 && E.narrow4) {
            const dim3 g4((unsigned)std::max(1, ceil_div(E.n, N4_ROWS)));
            k_spmm_n4<<<g4, 256, 0, ctx->stream>>>(g->row_ptr, g->col, g->val, Pin, E.Q, E.n, c1, c2, st);
            HD_CHECK_LAUNCH(ctx);
        } else if (E.segK <= 1) {
            HD_DISPATCH_S(E.vl.S, (k_spmm<SS><<<grid, 256, 0, ctx->stream>>>(g->row_ptr, g->col, g->val, Pin, E.Q,
                                                                              E.n, E.Bp, c1, c2, st)));
            HD_CHECK_LAUNCH(ctx);
        } else {
            for (int s = 0; s < E.segK; ++s) {
                const int32_t* lo = E.seg + (int64_t)s * E.n;
                HD_DISPATCH_S(E.vl.S, (k_spmm_seg<SS><<<grid, 256, 0, ctx->stream>>>(
                                          lo, lo + E.n, g->col, g->val, Pin, E.Q, E.n, E.Bp, c1, c2, st, s == 0)));
                HD_CHECK_LAUNCH(ctx);
            }
        }
    }
    if (part) return launch_dot(E, part, st);
    return HD_OK;
}

static const int32_t* seg_bounds_for(hd_ctx* ctx, const hd_graph* g, int K) {
    auto it = g->seg_bounds.find(K);
    if (it != g->seg_bounds.end()) return it->second;
    int32_t* b = nullptr;
    if (cudaMalloc(&b, (size_t)(K + 1) * g->n * 4) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    const int64_t w = (g->n + K - 1) / K;
    k_seg_bounds<<<ceil_div(g->n, 256), 256, 0, ctx->stream>>>(g->row_ptr, g->col, g->n, K, w, b);
    ctx->launches++;
    if (cudaGetLastError() != cudaSuccess) {
        cudaFree(b);
        return nullptr;
    }
    g->seg_bounds[K] = b;
    return b;
}

int tune_segments(hd_ctx* ctx, Engine& E) {
    const hd_graph* g = E.g;
    E.segK = 1;
    E.seg = nullptr;
    static int forced = -2;
    if (forced == -2) {
        const char* s = getenv("HD_SEGMENTS");
        forced = s ? atoi(s) : -1;
    }
    int K = 1;
    auto it = g->seg_cache.find(E.Bp);
    if (forced >= 1) {
        K = forced;
        g->seg_cache[E.Bp] = K;  // reported by hd_graph_tuning
    } else if (it != g->seg_cache.end()) {
        K = it->second;
    } else if ((int64_t)g->n * E.Bp * 4 > (int64_t)64 << 20) {
        // gathered block larger than about half of L2: time the candidates
        float best_ms = 1e30f;
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        for (int k : {1, 2, 4, 8}) {
            if (k > 1 && !seg_bounds_for(ctx, g, k)) continue;
            E.segK = k;
            E.seg = k > 1 ? g->seg_bounds[k] : nullptr;
            float tot = 0.f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(e0, ctx->stream);
                launch_spmm(E, 1.f, 1.f, nullptr, nullptr);
                cudaEventRecord(e1, ctx->stream);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep) tot += ms;
            }
            if (tot < best_ms * 0.97f) {
                best_ms = tot;
                K = k;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaGetLastError();
        g->seg_cache[E.Bp] = K;
    }
    if (K > 1) {
        const int32_t* b = seg_bounds_for(ctx, g, K);
        if (!b) return hd_fail(ctx, HD_ERR_OOM, "SpMM segment bounds");
        E.segK = K;
        E.seg = b;
    } else {
        E.segK = 1;
        E.seg = nullptr;
    }
    return HD_OK;
}

// ------------------------------------------------------------------ the solve


#define LAUNCH_VEC(kernel, ...)                                                                 \
    do {                                                                                        \
        HD_PROF(S_.ctx, #kernel[2] == 's' && #kernel[3] == 'p' ? "spmm"                         \
                        : #kernel[2] == 'u' ? "update" : #kernel[2] == 'd' ? "direction" : "colsq"); \
        dim3 grid_(S_.vl.nblk, S_.vl.slabs);                                                    \
        HD_DISPATCH_S(S_.vl.S, (kernel<SS><<<grid_, 256, 0, S_.ctx->stream>>>(__VA_ARGS__)));   \
        HD_CHECK_LAUNCH(S_.ctx);                                                                \
    } while (0)


// The scalar step after the update (rr, convergence, beta; C / coef: the PCG
// term): k_fin_rr, or for a server lane k_fin_rr_serve, which also installs
// staged requests, followed by their U^T y into H for the direction.
static int launch_fin_rr(Engine& S_, const double* C, const double* coef, int r) {
    hd_ctx* ctx = S_.ctx;
    const int32_t Bp = S_.Bp;
    HD_PROF(ctx, "scalar");
    HD_CUDA(ctx, cudaMemsetAsync(S_.num_active, 0, sizeof(int), ctx->stream));
    if (S_.refill) {
        k_fin_rr_serve<<<Bp, 128, 0, ctx->stream>>>(S_.part, (int)S_.nch, Bp, S_.st, S_.max_iter, C, coef, r,
                                                   S_.num_active, *S_.refill);
        HD_CHECK_LAUNCH(ctx);
        if (S_.has_lr && S_.eff_mode == HD_MODE_PCG) {
            const int64_t tot = (int64_t)S_.lr.rpad * Bp;
            k_refill_h<<<ceil_div(tot, 256), 256, 0, ctx->stream>>>(*S_.refill, S_.dcoef, S_.lr.rpad, Bp, S_.lr.H,
                                                                     S_.lr.Hhi, S_.lr.Hlo);
            HD_CHECK_LAUNCH(ctx);
        }
        return HD_OK;
    }
    if (S_.use_half) HD_CUDA(ctx, cudaMemsetAsync(S_.use_half, 0xff, sizeof(int), ctx->stream));
    k_fin_rr<<<Bp, 128, 0, ctx->stream>>>(S_.part, (int)S_.nch, Bp, S_.st, S_.max_iter, C, coef, r, S_.num_active,
                                         S_.use_half, HALF_THETA * HALF_THETA);
    HD_CHECK_LAUNCH(ctx);
    return HD_OK;
}

// One CG iteration of every column (Eq. 20 operator, CG update, direction).
// `after_update`, if given, runs right after the X/R update (the serving loop
// scatters newly admitted observations there).
int engine_iteration(Engine& S_, int (*after_update)(void*), void* arg) {
    hd_ctx* ctx = S_.ctx;
    const int64_t n = S_.n;
    const int32_t Bp = S_.Bp;
    const int r = S_.r;
    const bool lr_on = S_.has_lr;
    const int eff_mode = S_.eff_mode;
    const float c1 = S_.c1, c2 = S_.c2;
    const int32_t max_iter = S_.max_iter;
    const double* Cd = lr_on ? S_.lr.C : nullptr;
    int rc;
    if (eff_mode == HD_MODE_PCG) {
        if ((rc = launch_spmm(S_, c1, c2, S_.part, S_.st))) return rc;
        { HD_PROF(ctx, "scalar");
        k_fin_sigma<<<Bp, 128, 0, ctx->stream>>>(S_.part, (int)S_.nch, Bp, S_.st, nullptr, nullptr, 0); }
        HD_CHECK_LAUNCH(ctx);
        if ((rc = launch_update(S_))) return rc;
    if (after_update && (rc = after_update(arg))) return rc;
        if ((rc = lr_reduce(ctx, S_.lr, S_.R, n, Bp, S_.num_active))) return rc;
        if ((rc = lr_finish(ctx, S_.lr, Bp, S_.dcoef))) return rc;
        if ((rc = launch_fin_rr(S_, Cd, S_.dcoef, r))) return rc;
        if ((rc = lr_expand(ctx, S_.lr, EXP_DIRECTION, S_.P, S_.R, S_.P, n, Bp, S_.st, S_.num_active))) return rc;
        if (S_.refill) {
            k_refill_p<<<ceil_div(Bp, 128), 128, 0, ctx->stream>>>(*S_.refill, S_.P, Bp);
            HD_CHECK_LAUNCH(ctx);
        }
    } else {
        if (S_.ts)
        {
            LAUNCH_VEC(k_spmm_cols, S_.ts->off, S_.ts->ci, S_.ts->wv, S_.ts->B, S_.P, S_.Q, n, Bp, c1, c2, S_.st);
            if ((rc = launch_dot(S_, S_.part, S_.st))) return rc;
        }
        else if ((rc = launch_spmm(S_, c1, c2, S_.part, S_.st)))
            return rc;
        if (lr_on) {
            if ((rc = lr_expand(ctx, S_.lr, EXP_ADD_Q, S_.Q, nullptr, nullptr, n, Bp, S_.st, S_.num_active)))
                return rc;
        }
        { HD_PROF(ctx, "scalar");
        k_fin_sigma<<<Bp, 128, 0, ctx->stream>>>(S_.part, (int)S_.nch, Bp, S_.st, Cd,
                                                lr_on ? S_.opcoef : nullptr, r); }
        HD_CHECK_LAUNCH(ctx);
        if ((rc = launch_update(S_))) return rc;
    if (after_update && (rc = after_update(arg))) return rc;
        if ((rc = launch_fin_rr(S_, nullptr, nullptr, 0))) return rc;
        LAUNCH_VEC(k_direction, S_.P, S_.R, n, Bp, S_.st);
        if (S_.refill) {
            k_refill_p<<<ceil_div(Bp, 128), 128, 0, ctx->stream>>>(*S_.refill, S_.P, Bp);
            HD_CHECK_LAUNCH(ctx);
        }
        if (lr_on) {
            if ((rc = lr_reduce(ctx, S_.lr, S_.P, n, Bp, S_.num_active))) return rc;
            if ((rc = lr_finish(ctx, S_.lr, Bp, S_.opcoef))) return rc;
        }
    }
    return HD_OK;
}

// Run `iters` CG iterations as one CUDA graph launch.  The graph is captured
// on a private stream (the context's stream may be the legacy default stream,
// which cannot be captured) and re-captured whenever anything the kernels take
// as an argument differs from every cached capture.
static uint64_t fbits(float f) {
    uint32_t u;
    memcpy(&u, &f, sizeof u);
    return u;
}

// Everything the iteration kernels take as arguments (the run length is added
// by the caller).
static std::vector<uint64_t> iteration_key(const Engine& E) {
    return {(uint64_t)E.g, (uint64_t)E.ts, (uint64_t)(E.ts ? E.ts->off : nullptr), (uint64_t)(E.ts ? E.ts->ci : nullptr),
            (uint64_t)(E.ts ? E.ts->wv : nullptr), (uint64_t)(E.ts ? E.ts->B : 0), (uint64_t)E.g->row_ptr,
            (uint64_t)E.g->col, (uint64_t)E.g->val, (uint64_t)E.n, (uint64_t)E.lr.e,
            (uint64_t)(E.has_lr ? E.lr.e->U : nullptr), (uint64_t)(E.has_lr ? E.lr.e->storage : -1),
            (uint64_t)(E.has_lr ? E.lr.e->sp_rp : nullptr), (uint64_t)(E.has_lr ? E.lr.e->sp_cp : nullptr),
            (uint64_t)E.R, (uint64_t)E.P, (uint64_t)E.Q, (uint64_t)E.X, (uint64_t)E.part, (uint64_t)E.st,
            (uint64_t)E.num_active, (uint64_t)E.lr.part, (uint64_t)E.lr.C, (uint64_t)E.lr.H, (uint64_t)E.lr.Hhi,
            (uint64_t)E.lr.Hlo, (uint64_t)E.dcoef, (uint64_t)E.opcoef, (uint64_t)E.segK, (uint64_t)E.seg,
            (uint64_t)E.nch, (uint64_t)E.Bp, (uint64_t)E.vl.S, (uint64_t)E.vl.nblk, (uint64_t)E.vl.slabs,
            (uint64_t)E.lr.nchunk, (uint64_t)E.lr.rpad, (uint64_t)E.lr.Bp16, (uint64_t)E.has_lr,
            (uint64_t)E.eff_mode, (uint64_t)E.r, (uint64_t)E.max_iter, fbits(E.c1), fbits(E.c2), fbits(E.xs),
            (uint64_t)E.P16, (uint64_t)E.p16_max, (uint64_t)E.use_half, (uint64_t)E.ctx->stream};
}

static int run_iterations_graph(Engine& E, int iters) {
    hd_ctx* ctx = E.ctx;
    std::vector<uint64_t> key = iteration_key(E);
    key.push_back((uint64_t)iters);
    auto it = ctx->iter_graphs.find(key);
    if (it == ctx->iter_graphs.end()) {
        if (ctx->iter_graphs.size() >= 8) {
            for (auto& kv : ctx->iter_graphs) cudaGraphExecDestroy(kv.second.exec);
            ctx->iter_graphs.clear();
        }
        if (!ctx->cap_stream) HD_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        cudaStream_t user = ctx->stream;
        // the capture stream starts after everything already queued on the user stream
        HD_CUDA(ctx, cudaStreamSynchronize(user));
        ctx->stream = ctx->cap_stream;
        const int64_t l0 = ctx->launches;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeRelaxed);
        int rc = HD_OK;
        if (e == cudaSuccess) {
            for (int t = 0; t < iters && rc == HD_OK; ++t) rc = engine_iteration(E, nullptr, nullptr);
            cudaError_t e2 = cudaStreamEndCapture(ctx->cap_stream, &graph);
            if (rc == HD_OK && e2 != cudaSuccess) e = e2;
        }
        ctx->stream = user;
        if (rc) return rc;
        if (e != cudaSuccess) {
            cudaGetLastError();
            return hd_fail(ctx, HD_ERR_CUDA, "iteration graph capture: %s", cudaGetErrorString(e));
        }
        hd_ctx::IterGraph ig;
        e = cudaGraphInstantiate(&ig.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return hd_fail(ctx, HD_ERR_CUDA, "iteration graph instantiate: %s", cudaGetErrorString(e));
        ig.launches = ctx->launches - l0;
        ctx->launches = l0;
        it = ctx->iter_graphs.emplace(key, ig).first;
    }
    HD_CUDA(ctx, cudaGraphLaunch(it->second.exec, ctx->stream));
    ctx->launches += it->second.launches;
    return HD_OK;
}

// HD_NO_HALF=1: every SpMM of the iterations gathers fp32
static bool half_gathers_off() {
    static int off = -1;
    if (off < 0) {
        const char* s = getenv("HD_NO_HALF");
        off = (s && atoi(s)) ? 1 : 0;
    }
    return off != 0;
}

static bool graphs_enabled(hd_ctx* ctx) {
    static int off = -1;
    if (off < 0) {
        const char* s = getenv("HD_NO_GRAPH");
        off = (s && atoi(s)) ? 1 : 0;
    }
    return !off && !ctx->prof;
}

extern "C" int hd_query_batch(hd_ctx* ctx, const hd_graph* g, const hd_eig* eig, int mode, int32_t B,
                              const int32_t* y_ptr, const int32_t* y_idx, const float* y_val, double alpha,
                              const float* tol, int32_t max_iter, float* X, int32_t ldx, int32_t* iters,
                              float* relres, int32_t* status) {
    return hd_query_impl(ctx, g, nullptr, eig, mode, B, y_ptr, y_idx, y_val, alpha, tol, max_iter, X, ldx, iters,
                         relres, status);
}

// Iterate until no column is active: runs of iterations (CUDA graphs when
// enabled), each followed by a poll of the active count and of the
// tensor-core kernels' wait flags.  The first run is as long as the previous
// solve with the same key took (at most 8), later runs 2, 4, 8, then 16
// iterations, so a repeated workload polls once and launches no idle
// iterations.  `ran` accumulates the iterations launched.
static int iterate_until_stopped(Engine& E, int& ran) {
    hd_ctx* ctx = E.ctx;
    const std::vector<uint64_t> hkey = iteration_key(E);
    const int first = (ctx->hint_key == hkey && ctx->iter_hint > 0) ? std::min(ctx->iter_hint, 8) : 4;
    int run = 0, next = 2;
    int active = 1;
    int rc;
    // every active column stops within max_iter iterations of its own; the
    // bound only guards the host loop
    const int64_t cap = (int64_t)(MAX_CONFIRM + 1) * E.max_iter + 8;
    while (active > 0 && ran < cap) {
        int todo = first;
        if (run > 0) {
            todo = next;
            next = std::min(2 * next, 16);
        }
        if (graphs_enabled(ctx)) {
            if ((rc = run_iterations_graph(E, todo))) return rc;
        } else {
            for (int t = 0; t < todo; ++t)
                if ((rc = engine_iteration(E, nullptr, nullptr))) return rc;
        }
        ran += todo;
        ++run;
        HD_CUDA(ctx, cudaMemcpyAsync(ctx->h_poll, E.num_active, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        HD_CUDA(ctx, cudaMemcpyAsync(ctx->h_poll + 8, ctx->d_flags + 2, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                                     ctx->stream));
        HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        active = ctx->h_poll[0];
        if (ctx->h_poll[8] || ctx->h_poll[9]) return lr_tc_check_flags(ctx);
    }
    return HD_OK;
}

// T = b - A x into Q for every column (A the operator the solve iterates on,
// applied to X; b = y, or y - U C_y for the projected form) and the partials
// of ||T||^2 in E.part.  X holds the temporal term alone at this point.
static int true_residual(Engine& E, double alpha) {
    hd_ctx* ctx = E.ctx;
    const int64_t n = E.n;
    const int32_t Bp = E.Bp;
    const double c1d = 1.0 / (1.0 - alpha), c2d = alpha / (1.0 - alpha);
    const float c1 = (float)c1d, c2 = (float)c2d;
    int rc;
    dim3 grid(E.vl.nblk, E.vl.slabs);
    if (E.ts) {
        // Q = -L_a(W_j) x column by column (truncated systems), in two words
        HD_PROF(ctx, "resid");
        HD_DISPATCH_S(E.vl.S, (k_resid_cols<SS><<<grid, 256, 0, ctx->stream>>>(E.ts->off, E.ts->ci, E.ts->wv, E.ts->B,
                                                                                E.X, E.Q, n, Bp, c1, c2)));
        HD_CHECK_LAUNCH(ctx);
    } else {
        // Q = -L_a(W) x: the fp32 SpMM when its rounding bound is small against
        // every column's tolerance, else the two-word kernel (k_resid_pick)
        const hd_graph* g = E.g;
        const double u = 1.0 / 16777216.0;
        const double m = (double)g->max_row + 1.0;
        const double gamma = m * u / (1.0 - m * u);
        int* pick = E.num_active + 2;
        if ((rc = launch_colsq(E, E.X))) return rc;
        {
            HD_PROF(ctx, "scalar");
            HD_CUDA(ctx, cudaMemsetAsync(pick, 0, sizeof(int), ctx->stream));
            k_resid_pick<<<Bp, 128, 0, ctx->stream>>>(E.part, (int)E.nch, Bp, E.B, E.st, gamma, c1d, c2d, pick);
        }
        HD_CHECK_LAUNCH(ctx);
        HD_PROF(ctx, "resid");
        HD_DISPATCH_S(E.vl.S, (k_spmm<SS><<<grid, 256, 0, ctx->stream>>>(g->row_ptr, g->col, g->val, E.X, E.Q, n, Bp,
                                                                          -c1, -c2, nullptr, pick)));
        HD_CHECK_LAUNCH(ctx);
        HD_DISPATCH_S(E.vl.S, (k_resid<SS><<<grid, 256, 0, ctx->stream>>>(g->row_ptr, g->col, g->val, E.X, E.Q, n, Bp,
                                                                           c1, c2, pick)));
        HD_CHECK_LAUNCH(ctx);
    }
    if (E.has_lr && E.eff_mode != HD_MODE_PCG) {
        // deflated operator: Q -= (a / (1 - a)) U (Lambda (U^T x))
        if ((rc = lr_reduce(ctx, E.lr, E.X, n, Bp))) return rc;
        if ((rc = lr_finish(ctx, E.lr, Bp, E.negop))) return rc;
        if ((rc = lr_expand(ctx, E.lr, EXP_ADD_Q, E.Q, nullptr, nullptr, n, Bp, nullptr))) return rc;
        if (E.eff_mode == HD_MODE_PROJ) {
            // b = y - U (U^T y)
            if ((rc = lr_coef(ctx, E.lr, Bp, E.ones, E.Cy))) return rc;
            if ((rc = lr_expand(ctx, E.lr, EXP_SUB_R, E.Q, nullptr, nullptr, n, Bp, nullptr))) return rc;
        }
    }
    k_scatter_y<<<ceil_div(E.B, 128), 128, 0, ctx->stream>>>(E.yp, E.yi, E.yv, E.B, n, Bp, E.Q, E.err);
    HD_CHECK_LAUNCH(ctx);
    return launch_colsq(E, E.Q);
}

// Restart the columns k_fin_confirm reactivated: r := T (in Q), a fresh
// direction from it (p = M^-1 r with the preconditioner, p = r otherwise), and
// for the deflated forms C = U^T p for the next operator application.
static int restart_columns(Engine& E) {
    hd_ctx* ctx = E.ctx;
    const int64_t n = E.n;
    const int32_t Bp = E.Bp;
    int rc;
    k_restart_copy<<<ceil_div(n * (Bp / 4), 256), 256, 0, ctx->stream>>>(E.R, E.Q, n, Bp, E.st);
    HD_CHECK_LAUNCH(ctx);
    if (E.use_half) HD_CUDA(ctx, cudaMemsetAsync(E.use_half, 0, sizeof(int), ctx->stream));
    if (E.eff_mode == HD_MODE_PCG) {
        if ((rc = lr_reduce(ctx, E.lr, E.R, n, Bp))) return rc;
        if ((rc = lr_finish(ctx, E.lr, Bp, E.dcoef))) return rc;
        {
            HD_PROF(ctx, "scalar");
            k_fin_restart<<<Bp, 128, 0, ctx->stream>>>(E.st, E.lr.C, E.dcoef, E.r);
        }
        HD_CHECK_LAUNCH(ctx);
        return lr_expand(ctx, E.lr, EXP_DIRECTION, E.P, E.R, E.P, n, Bp, E.st);
    }
    {
        HD_PROF(ctx, "scalar");
        k_fin_restart<<<Bp, 128, 0, ctx->stream>>>(E.st, nullptr, nullptr, 0);
    }
    HD_CHECK_LAUNCH(ctx);
    {
        HD_PROF(ctx, "direction");
        dim3 grid(E.vl.nblk, E.vl.slabs);
        HD_DISPATCH_S(E.vl.S, (k_direction<SS><<<grid, 256, 0, ctx->stream>>>(E.P, E.R, n, Bp, E.st)));
        HD_CHECK_LAUNCH(ctx);
    }
    if (E.has_lr) {
        if ((rc = lr_reduce(ctx, E.lr, E.P, n, Bp))) return rc;
        if ((rc = lr_finish(ctx, E.lr, Bp, E.opcoef))) return rc;
    }
    return HD_OK;
}

// The solve behind hd_query_batch; with `ts` the operator is the per-column
// truncated system (rows = shortlist positions) instead of the graph.
int hd_query_impl(hd_ctx* ctx, const hd_graph* g, const TruncSys* ts, const hd_eig* eig, int mode, int32_t B,
                  const int32_t* y_ptr, const int32_t* y_idx, const float* y_val, double alpha, const float* tol,
                  int32_t max_iter, float* X, int32_t ldx, int32_t* iters, float* relres, int32_t* status) {
    if (!ctx || !g || !y_ptr || !tol || !X) return HD_ERR_INVALID_ARG;
    if (ts && eig) return hd_fail(ctx, HD_ERR_INVALID_ARG, "truncated systems take no eigenpairs");
    if (B <= 0 || ldx < B) return hd_fail(ctx, HD_ERR_INVALID_ARG, "B=%d ldx=%d", B, ldx);
    if (!(alpha >= 0.0 && alpha < 1.0)) return hd_fail(ctx, HD_ERR_INVALID_ARG, "alpha=%g not in [0,1)", alpha);
    const bool temporal_only = (mode & HD_MODE_TEMPORAL_ONLY) != 0;
    mode &= ~HD_MODE_TEMPORAL_ONLY;
    if (mode != HD_MODE_PAPER && mode != HD_MODE_PROJ && mode != HD_MODE_PCG)
        return hd_fail(ctx, HD_ERR_INVALID_ARG, "mode %d", mode);
    if (temporal_only && mode == HD_MODE_PCG)
        return hd_fail(ctx, HD_ERR_INVALID_ARG, "HD_MODE_TEMPORAL_ONLY needs the paper's or the projected form");
    if (max_iter < 0) return hd_fail(ctx, HD_ERR_INVALID_ARG, "max_iter %d", max_iter);
    if (eig && eig->n != g->n) return hd_fail(ctx, HD_ERR_INVALID_ARG, "eigenpairs for n=%lld, graph n=%lld",
                                              (long long)eig->n, (long long)g->n);
    HD_CUDA(ctx, cudaSetDevice(ctx->device));
    Engine S_;
    S_.ctx = ctx;
    S_.g = g;
    S_.ts = ts;
    S_.n = ts ? ts->smax : g->n;
    engine_set_reduction(S_);
    S_.B = B;
    S_.Bp = (B + 3) / 4 * 4;
    S_.vl = vec_launch(ctx, S_.n, S_.Bp, pick_slab(S_.Bp));
    const int64_t n = S_.n;
    const int32_t Bp = S_.Bp;
    const bool lr_on = eig && eig->r > 0;
    S_.has_lr = lr_on;
    S_.lr = LowRank{};
    const int r = lr_on ? eig->r : 0;
    const int rpad = lr_on ? (r + 63) / 64 * 64 : 0;
    const int Bp16 = (Bp + 15) / 16 * 16;

    // host-side copy of y_ptr to learn nnz
    int32_t nnz_y;
    {
        int32_t last;
        if (hd_is_device_ptr(y_ptr)) {
            HD_CUDA(ctx, cudaMemcpy(&last, y_ptr + B, 4, cudaMemcpyDeviceToHost));
        } else {
            last = y_ptr[B];
        }
        nnz_y = last;
        if (nnz_y < 0) return hd_fail(ctx, HD_ERR_INVALID_ARG, "y_ptr[B] = %d", nnz_y);
        if (nnz_y > 0 && (!y_idx || !y_val)) return HD_ERR_INVALID_ARG;
    }
    const bool x_direct = hd_is_device_ptr(X) && ldx == Bp;
    int nchunk = 0;
    if (lr_on) nchunk = lr_nchunk(ctx, eig, Bp);

    size_t vec = (size_t)n * Bp * sizeof(float);
    size_t bytes = 3 * ws_size(vec) + (x_direct ? 0 : ws_size(vec)) + ws_size((size_t)S_.nch * Bp * sizeof(float2)) +
                   ws_size(Bp * sizeof(ColState)) + ws_size(64) + ws_size((B + 1) * 4) + 2 * ws_size(nnz_y * 4 + 4) +
                   ws_size(B * 4);
    if (lr_on)
        bytes += ws_size((size_t)nchunk * rpad * Bp * 4) + 2 * ws_size((size_t)rpad * Bp * 8) +
                 ws_size((size_t)rpad * Bp * 4) + 2 * ws_size((size_t)Bp16 * rpad * 2) + 6 * ws_size(rpad * 8);
    // the fp16 gather copy of P: graph solves with 8 <= Bp <= 256 columns in multiples of 8
    const bool half_ok = !ts && Bp % 8 == 0 && Bp <= 256;
    if (half_ok) bytes += ws_size((size_t)n * Bp * 2) + ws_size((size_t)Bp * 4);
    void* ws;
    int rc = hd_ws_reserve(ctx, bytes, &ws);
    if (rc) return rc;
    WsCarver cv(ws);
    S_.R = cv.take<float>((size_t)n * Bp);
    S_.P = cv.take<float>((size_t)n * Bp);
    S_.Q = cv.take<float>((size_t)n * Bp);
    S_.X = x_direct ? X : cv.take<float>((size_t)n * Bp);
    S_.part = cv.take<float2>((size_t)S_.nch * Bp);
    S_.st = cv.take<ColState>(Bp);
    S_.num_active = cv.take<int>(16);
    S_.err = S_.num_active + 1;
    int32_t* d_yptr = cv.take<int32_t>(B + 1);
    int32_t* d_yidx = cv.take<int32_t>(nnz_y + 1);
    float* d_yval = cv.take<float>(nnz_y + 1);
    float* d_tol = cv.take<float>(B);
    const void *yp, *yi, *yv, *tl;
    if ((rc = hd_stage_in(ctx, y_ptr, (B + 1) * 4, d_yptr, &yp))) return rc;
    if ((rc = hd_stage_in(ctx, y_idx, (size_t)nnz_y * 4, d_yidx, &yi))) return rc;
    if ((rc = hd_stage_in(ctx, y_val, (size_t)nnz_y * 4, d_yval, &yv))) return rc;
    if ((rc = hd_stage_in(ctx, tol, (size_t)B * 4, d_tol, &tl))) return rc;
    S_.yp = (const int32_t*)yp;
    S_.yi = (const int32_t*)yi;
    S_.yv = (const float*)yv;
    __half* p16 = half_ok ? cv.take<__half>((size_t)n * Bp) : nullptr;
    unsigned* p16_max = half_ok ? cv.take<unsigned>(Bp) : nullptr;
    if (lr_on) {
        S_.lr.e = eig;
        S_.lr.rpad = rpad;
        S_.lr.nchunk = nchunk;
        S_.lr.Bp16 = Bp16;
        S_.lr.part = cv.take<float>((size_t)nchunk * rpad * Bp);
        S_.lr.C = cv.take<double>((size_t)rpad * Bp);
        S_.Cy = cv.take<double>((size_t)rpad * Bp);
        S_.lr.H = cv.take<float>((size_t)rpad * Bp);
        S_.lr.Hhi = cv.take<__nv_bfloat16>((size_t)Bp16 * rpad);
        S_.lr.Hlo = cv.take<__nv_bfloat16>((size_t)Bp16 * rpad);
        S_.gcoef = cv.take<double>(rpad);
        S_.hcoef = cv.take<double>(rpad);
        S_.opcoef = cv.take<double>(rpad);
        S_.dcoef = cv.take<double>(rpad);
        S_.ones = cv.take<double>(rpad);
        S_.negop = cv.take<double>(rpad);
        std::vector<double> gc(rpad, 0.0), hc(rpad, 0.0), oc(rpad, 0.0), dc(rpad, 0.0), on(rpad, 0.0), ng(rpad, 0.0);
        const double a = alpha;
        const double c3 = mode == HD_MODE_PROJ ? a : a / (1.0 - a);
        for (int k = 0; k < r; ++k) {
            double l = eig->lambda_h[k];
            gc[k] = (1.0 - a) * a * l / (1.0 - a * l);  // g_alpha, Eq. 16
            hc[k] = (1.0 - a) / (1.0 - a * l);          // h_alpha, Sec. 3.2
            oc[k] = c3 * l;
            double lt = l > 0.0 ? l : 0.0;
            dc[k] = a * lt / (1.0 - a * lt);
            on[k] = 1.0;
            ng[k] = -a / (1.0 - a) * l;
        }
        HD_CUDA(ctx, cudaMemcpyAsync(S_.gcoef, gc.data(), rpad * 8, cudaMemcpyHostToDevice, ctx->stream));
        HD_CUDA(ctx, cudaMemcpyAsync(S_.hcoef, hc.data(), rpad * 8, cudaMemcpyHostToDevice, ctx->stream));
        HD_CUDA(ctx, cudaMemcpyAsync(S_.opcoef, oc.data(), rpad * 8, cudaMemcpyHostToDevice, ctx->stream));
        HD_CUDA(ctx, cudaMemcpyAsync(S_.dcoef, dc.data(), rpad * 8, cudaMemcpyHostToDevice, ctx->stream));
        HD_CUDA(ctx, cudaMemcpyAsync(S_.ones, on.data(), rpad * 8, cudaMemcpyHostToDevice, ctx->stream));
        HD_CUDA(ctx, cudaMemcpyAsync(S_.negop, ng.data(), rpad * 8, cudaMemcpyHostToDevice, ctx->stream));
        HD_CUDA(ctx, cudaMemsetAsync(S_.lr.Hhi, 0, (size_t)Bp16 * rpad * 2, ctx->stream));
        HD_CUDA(ctx, cudaMemsetAsync(S_.lr.Hlo, 0, (size_t)Bp16 * rpad * 2, ctx->stream));
    }

    // ---------------- setup
    if (!ts && g->max_row < 0) {
        // the longest row bounds the rounding of the true residual (k_resid_pick)
        HD_CUDA(ctx, cudaMemsetAsync(S_.num_active, 0, sizeof(int), ctx->stream));
        k_max_row<<<std::min<int64_t>(ceil_div(n, 256), (int64_t)ctx->num_sms * 8), 256, 0, ctx->stream>>>(
            g->row_ptr, n, S_.num_active);
        HD_CHECK_LAUNCH(ctx);
        HD_CUDA(ctx, cudaMemcpyAsync(ctx->h_poll, S_.num_active, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        g->max_row = ctx->h_poll[0];
    }
    S_.vl = vec_launch(ctx, n, Bp, ts ? pick_slab(Bp) : tune_slab(ctx, g, Bp, S_.P, S_.Q));
    if (!ts && (rc = tune_segments(ctx, S_))) return rc;
    if (half_ok && S_.segK == 1 && !half_gathers_off()) {
        S_.P16 = p16;
        S_.p16_max = p16_max;
        S_.use_half = S_.num_active + 3;  // 0: the first iteration gathers fp32
        HD_CUDA(ctx, cudaMemsetAsync(S_.use_half, 0, sizeof(int), ctx->stream));
    }
    const int eff_mode = lr_on ? mode : HD_MODE_PAPER;
    const double a = alpha;
    float c1, c2, xs = 1.0f;
    if (eff_mode == HD_MODE_PROJ) {
        c1 = 1.0f;
        c2 = (float)a;
        xs = (float)(1.0 - a);
    } else {
        c1 = (float)(1.0 / (1.0 - a));
        c2 = (float)(a / (1.0 - a));
    }
    // X accumulates the temporal term alone; the spectral term is added after
    // the true-residual confirmation
    HD_CUDA(ctx, cudaMemsetAsync(S_.R, 0, vec, ctx->stream));
    HD_CUDA(ctx, cudaMemsetAsync(S_.X, 0, vec, ctx->stream));
    HD_CUDA(ctx, cudaMemsetAsync(S_.err, 0, sizeof(int), ctx->stream));
    k_scatter_y<<<ceil_div(B, 128), 128, 0, ctx->stream>>>((const int32_t*)yp, (const int32_t*)yi, (const float*)yv,
                                                           B, n, Bp, S_.R, S_.err);
    HD_CHECK_LAUNCH(ctx);
    const double* Cd = lr_on ? S_.lr.C : nullptr;
    const size_t cbytes = (size_t)rpad * Bp * sizeof(double);
    if (eff_mode == HD_MODE_PAPER) {
        if ((rc = launch_colsq(S_, S_.R))) return rc;
        HD_CUDA(ctx, cudaMemsetAsync(S_.num_active, 0, sizeof(int), ctx->stream));
        k_fin_setup<<<Bp, 128, 0, ctx->stream>>>(S_.part, (int)S_.nch, Bp, B, (const float*)tl, S_.st, nullptr, nullptr,
                                                0, S_.num_active);
        HD_CHECK_LAUNCH(ctx);
        HD_CUDA(ctx, cudaMemcpyAsync(S_.P, S_.R, vec, cudaMemcpyDeviceToDevice, ctx->stream));
        if (lr_on) {
            // C = U^T y: kept for x^s = U g(Lambda) C (Eq. 18), and U^T P for the first operator
            if ((rc = lr_reduce(ctx, S_.lr, S_.R, n, Bp))) return rc;
            if ((rc = lr_finish(ctx, S_.lr, Bp, S_.opcoef))) return rc;
            HD_CUDA(ctx, cudaMemcpyAsync(S_.Cy, S_.lr.C, cbytes, cudaMemcpyDeviceToDevice, ctx->stream));
        }
    } else if (eff_mode == HD_MODE_PROJ) {
        // C = U^T y (kept); b = y - U C
        if ((rc = lr_reduce(ctx, S_.lr, S_.R, n, Bp))) return rc;
        if ((rc = lr_finish(ctx, S_.lr, Bp, S_.ones))) return rc;
        HD_CUDA(ctx, cudaMemcpyAsync(S_.Cy, S_.lr.C, cbytes, cudaMemcpyDeviceToDevice, ctx->stream));
        if ((rc = lr_expand(ctx, S_.lr, EXP_SUB_R, S_.R, nullptr, nullptr, n, Bp, S_.st))) return rc;
        if ((rc = launch_colsq(S_, S_.R))) return rc;
        HD_CUDA(ctx, cudaMemsetAsync(S_.num_active, 0, sizeof(int), ctx->stream));
        k_fin_setup<<<Bp, 128, 0, ctx->stream>>>(S_.part, (int)S_.nch, Bp, B, (const float*)tl, S_.st, nullptr, nullptr,
                                                0, S_.num_active);
        HD_CHECK_LAUNCH(ctx);
        HD_CUDA(ctx, cudaMemcpyAsync(S_.P, S_.R, vec, cudaMemcpyDeviceToDevice, ctx->stream));
        if ((rc = lr_reduce(ctx, S_.lr, S_.P, n, Bp))) return rc;
        if ((rc = lr_finish(ctx, S_.lr, Bp, S_.opcoef))) return rc;
    } else {  // PCG
        if ((rc = launch_colsq(S_, S_.R))) return rc;
        if ((rc = lr_reduce(ctx, S_.lr, S_.R, n, Bp))) return rc;
        if ((rc = lr_finish(ctx, S_.lr, Bp, S_.dcoef))) return rc;
        HD_CUDA(ctx, cudaMemsetAsync(S_.num_active, 0, sizeof(int), ctx->stream));
        k_fin_setup<<<Bp, 128, 0, ctx->stream>>>(S_.part, (int)S_.nch, Bp, B, (const float*)tl, S_.st, Cd, S_.dcoef, r,
                                                S_.num_active);
        HD_CHECK_LAUNCH(ctx);
        HD_CUDA(ctx, cudaMemsetAsync(S_.P, 0, vec, ctx->stream));
        if ((rc = lr_expand(ctx, S_.lr, EXP_DIRECTION, S_.P, S_.R, S_.P, n, Bp, S_.st))) return rc;
    }

    // ---------------- iterations, then confirmation by the true residual
    S_.eff_mode = eff_mode;
    S_.c1 = c1;
    S_.c2 = c2;
    S_.xs = xs;
    S_.r = r;
    S_.max_iter = max_iter;
    HD_CUDA(ctx, cudaMemcpyAsync(ctx->h_poll, S_.num_active, 2 * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->h_poll[1])
        return hd_fail(ctx, HD_ERR_INVALID_ARG, "bad observation: index out of range, non-finite value or bad y_ptr");
    int active = ctx->h_poll[0];
    int ran = 0, first_ran = -1;
    std::vector<ColState> hs(B);
    for (int round = 0; round <= MAX_CONFIRM; ++round) {
        if (active > 0 && max_iter > 0 && (rc = iterate_until_stopped(S_, ran))) return rc;
        if (first_ran < 0) first_ran = ran;
        if ((rc = true_residual(S_, a))) return rc;
        {
            HD_PROF(ctx, "scalar");
            HD_CUDA(ctx, cudaMemsetAsync(S_.num_active, 0, sizeof(int), ctx->stream));
            k_fin_confirm<<<Bp, 128, 0, ctx->stream>>>(S_.part, (int)S_.nch, Bp, B, S_.st, max_iter, S_.num_active);
        }
        HD_CHECK_LAUNCH(ctx);
        HD_CUDA(ctx, cudaMemcpyAsync(ctx->h_poll, S_.num_active, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
        HD_CUDA(ctx, cudaMemcpyAsync(hs.data(), S_.st, B * sizeof(ColState), cudaMemcpyDeviceToHost, ctx->stream));
        HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        active = ctx->h_poll[0];
        if (active == 0) break;
        if ((rc = restart_columns(S_))) return rc;
    }
    // the next solve with the same key polls first after as many iterations as
    // this one's columns took before any restart (without restarts the
    // columns' own count, else the iterations launched)
    int most = 0;
    for (int j = 0; j < B; ++j) most = std::max(most, hs[j].iters);
    ctx->hint_key = iteration_key(S_);
    ctx->iter_hint = ran == first_ran ? most : first_ran;
    for (int j = 0; j < B; ++j) {
        if (iters && !hd_is_device_ptr(iters)) iters[j] = hs[j].iters;
        if (relres && !hd_is_device_ptr(relres)) relres[j] = hs[j].bb > 0 ? (float)std::sqrt(hs[j].rr / hs[j].bb) : 0.f;
        if (status && !hd_is_device_ptr(status)) status[j] = hs[j].status;
    }
    // ---------------- spectral term (Eq. 17-18): X += U g(Lambda) U^T y, or U h(Lambda) U^T y (projected form)
    if (lr_on && eff_mode != HD_MODE_PCG && !temporal_only) {
        if ((rc = lr_coef(ctx, S_.lr, Bp, eff_mode == HD_MODE_PAPER ? S_.gcoef : S_.hcoef, S_.Cy))) return rc;
        if ((rc = lr_expand(ctx, S_.lr, EXP_ADD_Q, S_.X, nullptr, nullptr, n, Bp, nullptr))) return rc;
    }

    // ---------------- outputs
    if ((iters && hd_is_device_ptr(iters)) || (relres && hd_is_device_ptr(relres)) ||
        (status && hd_is_device_ptr(status))) {
        k_outputs<<<ceil_div(B, 128), 128, 0, ctx->stream>>>(S_.st, B, hd_is_device_ptr(iters) ? iters : nullptr,
                                                             hd_is_device_ptr(relres) ? relres : nullptr,
                                                             hd_is_device_ptr(status) ? status : nullptr);
        HD_CHECK_LAUNCH(ctx);
    }
    if (!x_direct) {
        if (hd_is_device_ptr(X)) {
            k_copy_out<<<ceil_div(n * B, 256), 256, 0, ctx->stream>>>(S_.X, Bp, X, ldx, B, n);
            HD_CHECK_LAUNCH(ctx);
        } else {
            HD_CUDA(ctx, cudaMemcpy2DAsync(X, (size_t)ldx * 4, S_.X, (size_t)Bp * 4, (size_t)B * 4, n,
                                           cudaMemcpyDeviceToHost, ctx->stream));
            HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        }
    }
    if (lr_on && lr_use_tensor_cores(eig)) return lr_tc_check_flags(ctx);
    return HD_OK;
}

// ------------------------------------------------------------------ spectral products on their own
static int lowrank_setup(hd_ctx* ctx, const hd_eig* e, int32_t Bp, LowRank& lr, double** coef_ones, WsCarver& cv) {
    lr.e = e;
    lr.rpad = (e->r + 63) / 64 * 64;
    lr.Bp16 = (Bp + 15) / 16 * 16;
    lr.nchunk = lr_nchunk(ctx, e, Bp);
    lr.part = cv.take<float>((size_t)lr.nchunk * lr.rpad * Bp);
    lr.C = cv.take<double>((size_t)lr.rpad * Bp);
    lr.H = cv.take<float>((size_t)lr.rpad * Bp);
    lr.Hhi = cv.take<__nv_bfloat16>((size_t)lr.Bp16 * lr.rpad);
    lr.Hlo = cv.take<__nv_bfloat16>((size_t)lr.Bp16 * lr.rpad);
    *coef_ones = cv.take<double>(lr.rpad);
    std::vector<double> on(lr.rpad, 0.0);
    for (int k = 0; k < e->r; ++k) on[k] = 1.0;
    HD_CUDA(ctx, cudaMemcpyAsync(*coef_ones, on.data(), lr.rpad * 8, cudaMemcpyHostToDevice, ctx->stream));
    HD_CUDA(ctx, cudaMemsetAsync(lr.Hhi, 0, (size_t)lr.Bp16 * lr.rpad * 2, ctx->stream));
    HD_CUDA(ctx, cudaMemsetAsync(lr.Hlo, 0, (size_t)lr.Bp16 * lr.rpad * 2, ctx->stream));
    return HD_OK;
}

static size_t lowrank_bytes(hd_ctx* ctx, const hd_eig* e, int32_t Bp) {
    int rpad = (e->r + 63) / 64 * 64;
    int nch = lr_nchunk(ctx, e, Bp);
    return ws_size((size_t)nch * rpad * Bp * 4) + ws_size((size_t)rpad * Bp * 8) + ws_size((size_t)rpad * Bp * 4) +
           2 * ws_size((size_t)((Bp + 15) / 16 * 16) * rpad * 2) + ws_size(rpad * 8);
}

extern "C" int hd_eig_project(hd_ctx* ctx, const hd_eig* e, const float* V, int32_t B, double* C_out) {
    if (!ctx || !e || !V || !C_out || B <= 0 || B % 4 || B > 256 || e->r <= 0) return HD_ERR_INVALID_ARG;
    if (!hd_is_device_ptr(V)) return hd_fail(ctx, HD_ERR_INVALID_ARG, "V must be device memory");
    void* ws;
    int rc = hd_ws_reserve(ctx, lowrank_bytes(ctx, e, B), &ws);
    if (rc) return rc;
    WsCarver cv(ws);
    LowRank lr;
    double* ones;
    if ((rc = lowrank_setup(ctx, e, B, lr, &ones, cv))) return rc;
    if ((rc = lr_reduce(ctx, lr, V, e->n, B))) return rc;
    if ((rc = lr_finish(ctx, lr, B, ones))) return rc;
    // rows 0..r-1 of C (fp64, r x B)
    cudaMemcpyKind kind = hd_is_device_ptr(C_out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    HD_CUDA(ctx, cudaMemcpyAsync(C_out, lr.C, (size_t)e->r * B * 8, kind, ctx->stream));
    HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (lr_use_tensor_cores(e) && (rc = lr_tc_check_flags(ctx))) return rc;
    return HD_OK;
}

// H (fp64, r x B) -> the fp32 partial layout [1][rpad][B], zero beyond r.
__global__ void k_h_to_part(const double* Hin, int r, int32_t B, int rpad, float* part) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)rpad * B) return;
    int k = (int)(e / B);
    part[e] = k < r ? (float)Hin[e] : 0.0f;
}

extern "C" int hd_eig_expand(hd_ctx* ctx, const hd_eig* e, const double* H, int32_t B, float* X_out) {
    if (!ctx || !e || !H || !X_out || B <= 0 || B % 4 || B > 256 || e->r <= 0) return HD_ERR_INVALID_ARG;
    if (!hd_is_device_ptr(X_out)) return hd_fail(ctx, HD_ERR_INVALID_ARG, "X_out must be device memory");
    void* ws;
    int rc = hd_ws_reserve(ctx, lowrank_bytes(ctx, e, B) + ws_size((size_t)e->r * B * 8), &ws);
    if (rc) return rc;
    WsCarver cv(ws);
    LowRank lr;
    double* ones;
    if ((rc = lowrank_setup(ctx, e, B, lr, &ones, cv))) return rc;
    double* Hs = cv.take<double>((size_t)e->r * B);
    const void* Hd;
    if ((rc = hd_stage_in(ctx, H, (size_t)e->r * B * 8, Hs, &Hd))) return rc;
    lr.nchunk = 1;
    k_h_to_part<<<ceil_div((int64_t)lr.rpad * B, 256), 256, 0, ctx->stream>>>((const double*)Hd, e->r, B, lr.rpad,
                                                                             lr.part);
    HD_CHECK_LAUNCH(ctx);
    if ((rc = lr_finish(ctx, lr, B, ones))) return rc;
    if ((rc = lr_expand(ctx, lr, EXP_SET_X, X_out, nullptr, nullptr, e->n, B, nullptr))) return rc;
    HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (lr_use_tensor_cores(e) && (rc = lr_tc_check_flags(ctx))) return rc;
    return HD_OK;
}

// ------------------------------------------------------------------ general transfer functions (Appendix A)

// out = (accumulate ? out : 0) + c * Y over n x Bp
__global__ void k_axpy_dense(float* __restrict__ out, const float* __restrict__ Y, float c, int64_t count4,
                             int accumulate) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= count4) return;
    const float4 y = reinterpret_cast<const float4*>(Y)[e];
    float4 o = accumulate ? reinterpret_cast<const float4*>(out)[e] : make_float4(0.f, 0.f, 0.f, 0.f);
    o.x = fmaf(c, y.x, o.x);
    o.y = fmaf(c, y.y, o.y);
    o.z = fmaf(c, y.z, o.z);
    o.w = fmaf(c, y.w, o.w);
    reinterpret_cast<float4*>(out)[e] = o;
}

extern "C" int hd_filter_poly(hd_ctx* ctx, const hd_graph* g, const hd_eig* eig, int32_t B, const int32_t* y_ptr,
                              const int32_t* y_idx, const float* y_val, const double* coeffs, int32_t ncoef,
                              float* X, int32_t ldx) {
    if (!ctx || !g || !y_ptr || !coeffs || !X) return HD_ERR_INVALID_ARG;
    if (B <= 0 || B > 4096 || ldx < B) return hd_fail(ctx, HD_ERR_INVALID_ARG, "B=%d ldx=%d", B, ldx);
    if (ncoef < 1 || ncoef > 100000) return hd_fail(ctx, HD_ERR_INVALID_ARG, "ncoef=%d", ncoef);
    for (int i = 0; i < ncoef; ++i)
        if (!std::isfinite(coeffs[i])) return hd_fail(ctx, HD_ERR_INVALID_ARG, "coefficient %d not finite", i);
    if (eig && eig->n != g->n) return hd_fail(ctx, HD_ERR_INVALID_ARG, "eigenpairs for n=%lld, graph n=%lld",
                                              (long long)eig->n, (long long)g->n);
    HD_CUDA(ctx, cudaSetDevice(ctx->device));
    const int64_t n = g->n;
    const int32_t Bp = (B + 3) / 4 * 4;
    const bool lr_on = eig && eig->r > 0;
    int32_t nnz_y;
    if (hd_is_device_ptr(y_ptr)) {
        HD_CUDA(ctx, cudaMemcpy(&nnz_y, y_ptr + B, 4, cudaMemcpyDeviceToHost));
    } else {
        nnz_y = y_ptr[B];
    }
    if (nnz_y < 0) return hd_fail(ctx, HD_ERR_INVALID_ARG, "y_ptr[B] = %d", nnz_y);
    if (nnz_y > 0 && (!y_idx || !y_val)) return HD_ERR_INVALID_ARG;
    const size_t vec = (size_t)n * Bp * 4;
    size_t bytes = 3 * ws_size(vec) + ws_size(64) + ws_size((B + 1) * 4) + 2 * ws_size((size_t)nnz_y * 4 + 4);
    if (lr_on) bytes += lowrank_bytes(ctx, eig, Bp) + 2 * ws_size((size_t)((eig->r + 63) / 64 * 64) * 8);
    void* ws;
    int rc = hd_ws_reserve(ctx, bytes, &ws);
    if (rc) return rc;
    WsCarver cv(ws);
    float* Yd = cv.take<float>((size_t)n * Bp);
    float* acc = cv.take<float>((size_t)n * Bp);
    float* Q = cv.take<float>((size_t)n * Bp);
    int* err = cv.take<int>(16);
    int32_t* d_yptr = cv.take<int32_t>(B + 1);
    int32_t* d_yidx = cv.take<int32_t>(nnz_y + 1);
    float* d_yval = cv.take<float>(nnz_y + 1);
    const void *yp, *yi, *yv;
    if ((rc = hd_stage_in(ctx, y_ptr, (B + 1) * 4, d_yptr, &yp))) return rc;
    if ((rc = hd_stage_in(ctx, y_idx, (size_t)nnz_y * 4, d_yidx, &yi))) return rc;
    if ((rc = hd_stage_in(ctx, y_val, (size_t)nnz_y * 4, d_yval, &yv))) return rc;
    LowRank lr{};
    double *ones = nullptr, *lamc = nullptr, *gc = nullptr;
    if (lr_on) {
        if ((rc = lowrank_setup(ctx, eig, Bp, lr, &ones, cv))) return rc;
        lamc = cv.take<double>(lr.rpad);
        gc = cv.take<double>(lr.rpad);
        // g(lambda) = h(lambda) - h(0) = sum_{i >= 1} c_i lambda^i (Eq. 33), Horner in fp64
        std::vector<double> lh(lr.rpad, 0.0), gh(lr.rpad, 0.0);
        for (int k = 0; k < eig->r; ++k) {
            const double l = eig->lambda_h[k];
            double s = 0.0;
            for (int i = ncoef - 1; i >= 1; --i) s = s * l + coeffs[i];
            lh[k] = l;
            gh[k] = s * l;
        }
        HD_CUDA(ctx, cudaMemcpyAsync(lamc, lh.data(), lr.rpad * 8, cudaMemcpyHostToDevice, ctx->stream));
        HD_CUDA(ctx, cudaMemcpyAsync(gc, gh.data(), lr.rpad * 8, cudaMemcpyHostToDevice, ctx->stream));
    }
    HD_CUDA(ctx, cudaMemsetAsync(Yd, 0, vec, ctx->stream));
    HD_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
    k_scatter_y<<<ceil_div(B, 128), 128, 0, ctx->stream>>>((const int32_t*)yp, (const int32_t*)yi, (const float*)yv, B,
                                                           n, Bp, Yd, err);
    HD_CHECK_LAUNCH(ctx);
    const int64_t c4 = (int64_t)n * Bp / 4;
    // h(W_r) y by Horner's rule on the black box W_r z = W z - U (Lambda (U^T z)) (Eq. 32)
    k_axpy_dense<<<ceil_div(c4, 256), 256, 0, ctx->stream>>>(acc, Yd, (float)coeffs[ncoef - 1], c4, 0);
    HD_CHECK_LAUNCH(ctx);
    for (int i = ncoef - 2; i >= 0; --i) {
        { HD_PROF(ctx, "spmm");
          if ((rc = hd_spmm_apply(ctx, g, acc, Q, Bp, B, 0.0f, -1.0f))) return rc; }
        if (lr_on) {
            if ((rc = lr_reduce(ctx, lr, acc, n, Bp))) return rc;
            if ((rc = lr_finish(ctx, lr, Bp, lamc))) return rc;
            if ((rc = lr_expand(ctx, lr, EXP_SUB_R, Q, nullptr, nullptr, n, Bp, nullptr))) return rc;
        }
        k_axpy_dense<<<ceil_div(c4, 256), 256, 0, ctx->stream>>>(Q, Yd, (float)coeffs[i], c4, 1);
        HD_CHECK_LAUNCH(ctx);
        std::swap(acc, Q);
    }
    // + U g(Lambda) U^T y (Eq. 32)
    if (lr_on) {
        if ((rc = lr_reduce(ctx, lr, Yd, n, Bp))) return rc;
        if ((rc = lr_finish(ctx, lr, Bp, gc))) return rc;
        if ((rc = lr_expand(ctx, lr, EXP_ADD_Q, acc, nullptr, nullptr, n, Bp, nullptr))) return rc;
    }
    HD_CUDA(ctx, cudaMemcpyAsync(ctx->h_poll, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->h_poll[0])
        return hd_fail(ctx, HD_ERR_INVALID_ARG, "bad observation: index out of range, non-finite value or bad y_ptr");
    if (hd_is_device_ptr(X)) {
        k_copy_out<<<ceil_div(n * B, 256), 256, 0, ctx->stream>>>(acc, Bp, X, ldx, B, n);
        HD_CHECK_LAUNCH(ctx);
    } else {
        HD_CUDA(ctx, cudaMemcpy2DAsync(X, (size_t)ldx * 4, acc, (size_t)Bp * 4, (size_t)B * 4, n,
                                       cudaMemcpyDeviceToHost, ctx->stream));
    }
    HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (lr_on && lr_use_tensor_cores(eig) && (rc = lr_tc_check_flags(ctx))) return rc;
    return HD_OK;
}
