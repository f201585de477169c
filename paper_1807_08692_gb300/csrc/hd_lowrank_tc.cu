// Tall-skinny low-rank products of the hybrid operator on 5th-generation tensor
// cores (tcgen05.mma kind::f16, TMA-fed shared memory, fp32 accumulators in TMEM).
//
//  expand : out_i = op(U_i H) for every row i    (U n x r bf16, H r x B fp32)
//  reduce : part_c = sum_{i in chunk c} U_i^T V_i  (V n x B fp32)
//
// U is exact in bf16.  The fp32 operand (H or V) is split into bf16 high and
// low parts (x = hi + lo + O(2^-16 |x|)) and both are multiplied, so the
// products keep about 16 significant bits before the fp32 accumulation.
// FP32 storage: U is also kept as a bf16 [hi | lo] copy (lo = bf16(U - hi));
// the expansion runs twice the k-blocks (the lo half meets the same H blocks)
// and the reduction twice the M tiles, adding the lo tile into the hi tile in
// the epilogue, so all four hi/lo products are formed.
// FP8 storage (e4m3 codes with a per-row fp32 scale): TMA brings the raw code
// tiles in, four converter warps widen them to bf16 (exact: every e4m3 value
// is a bf16 value) in the swizzled layout the MMA reads, and the row scale is
// applied to the fp32 side (the expansion's output rows, the reduction's V
// rows), so the MMAs are the same as for bf16 storage.
// Both products are HBM-bound (arithmetic intensity ~B flop per byte of U):
// the tensor cores only have to keep up with the U stream.
#include <algorithm>
#include <cstdio>

#include "hd_solve.cuh"
#include "tc.cuh"

namespace {
constexpr int BM = 128;           // rows of U per tile
constexpr int BK = 64;            // bf16 elements per 128-byte swizzle row
constexpr int XSTAGES = 6;
constexpr int RSTAGES = 3;
constexpr int THREADS = 320;      // warp 0: TMA, warp 1: MMA, warps 2-9: epilogue / conversion
constexpr int EPI = 256;          // epilogue threads: two warps per TMEM lane quarter, splitting the columns
constexpr int TILE_BYTES = BM * BK * 2;  // 16 KB
constexpr int CONV = 128;         // converter threads (warps 10-13) for FP8 storage
constexpr int CSTAGES = 2;        // converted bf16 A stages for FP8 storage
constexpr int RAW_X = BM * BK;    // raw fp8 expansion stage: 128 rows x 64 codes
constexpr int RAW_R = BM * 128;   // raw fp8 reduction stage: 128 rows x 128 codes
constexpr int STAGE_BYTES = (EPI / 32) * 32 * 32 * 4;  // expansion epilogue: 32 x 32 fp32 per warp
}  // namespace

// 16 e4m3 codes -> 16 bf16 values (both exact), as two 16-byte chunks
__device__ __forceinline__ void fp8x16_to_bf16(const uint4 raw, uint4& lo, uint4& hi) {
    const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
    uint32_t o[8];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[q] >> (16 * h)), __NV_E4M3);
            __half2 hv;
            memcpy(&hv, &hr, sizeof hv);
            const float2 f = __half22float2(hv);
            const __nv_bfloat162 b = __floats2bfloat162_rn(f.x, f.y);
            memcpy(&o[2 * q + h], &b, sizeof(uint32_t));
        }
    }
    lo = make_uint4(o[0], o[1], o[2], o[3]);
    hi = make_uint4(o[4], o[5], o[6], o[7]);
}

bool lr_use_tensor_cores(const hd_eig* e) {
    static int off = -1;
    if (off < 0) {
        const char* s = getenv("HD_LOWRANK_SIMT");
        off = (s && atoi(s)) ? 1 : 0;
    }
    return e && !e->sparse && (e->storage == HD_BF16 || e->storage == HD_FP8 || (e->storage == HD_F32 && e->Usplit)) &&
           !off;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t* r = reinterpret_cast<uint32_t*>(v);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

template <uint32_t NC>
__device__ __forceinline__ void tmem_alloc_dyn(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_dyn(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

static uint32_t tmem_cols_for(uint32_t need) {
    uint32_t c = 32;
    while (c < need) c <<= 1;
    return c;
}

// =====================================================================================
// expand: out = op(U H)
// =====================================================================================
struct ExpandArgs {
    int64_t n;
    int32_t Bp;
    int32_t c0;     // first column of this launch
    int32_t Nc;     // columns of this launch (multiple of 16, <= 256)
    int32_t nkb;    // k-block iterations per tile (64 eigen-indices each)
    int32_t nkb_b;  // k-blocks of H; with U stored as [hi | lo] there are 2 nkb_b iterations: iteration kb
                    // reads U block kb (kb < nkb_b) or kb + a_off (the lo half) and H block kb mod nkb_b
    int32_t a_off;
    int32_t op;
    uint32_t tmem_cols;
    float* out;
    const float* R;
    const float* P;
    const ColState* st;
    const int* gate;
    const float* scale;  // per-row scale of FP8 storage
};

// SU = 0: bf16 storage (U tiles go straight from TMA to the MMA);
// SU = 1: fp8 storage (raw code tiles, converter warps, row scale in the epilogue)
template <int SU>
__global__ void __launch_bounds__(THREADS + (SU ? CONV : 0), 1)
    k_lr_expand_tc(const __grid_constant__ CUtensorMap tmU, const __grid_constant__ CUtensorMap tmHhi,
                   const __grid_constant__ CUtensorMap tmHlo, ExpandArgs a, int* err) {
    if (a.gate && *a.gate == 0) return;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t btile = (uint32_t)a.Nc * 128;  // one k-block of H^T (Nc rows x 128 B)
    constexpr int NA = SU ? CSTAGES : XSTAGES;    // bf16 A stages the MMA reads
    uint8_t* As = smem;
    uint8_t* Raw = As + NA * TILE_BYTES;          // raw fp8 stages (SU only)
    uint8_t* Bhi = Raw + (SU ? XSTAGES * RAW_X : 0);
    uint8_t* Blo = Bhi + a.nkb_b * btile;
    float* stage = reinterpret_cast<float*>(Blo + a.nkb_b * btile);  // epilogue transposition, 4 KB per warp
    uint64_t* bars = (uint64_t*)(reinterpret_cast<uint8_t*>(stage) + STAGE_BYTES);
    uint64_t* full = bars;
    uint64_t* empty = full + XSTAGES;
    uint64_t* bfull = empty + XSTAGES;
    uint64_t* acc_full = bfull + 1;
    uint64_t* acc_empty = acc_full + 2;
    uint64_t* drain = acc_empty + 2;
    uint64_t* cfull = drain + 1;
    uint64_t* cempty = cfull + CSTAGES;
    uint32_t* tmem_slot = (uint32_t*)(cempty + CSTAGES);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntiles = (int)((a.n + BM - 1) / BM);

    if (threadIdx.x == 0) {
        for (int s = 0; s < XSTAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], SU ? CONV : 1);
        }
        for (int s = 0; s < CSTAGES; ++s) {
            tc::mbar_init(&cfull[s], CONV);
            tc::mbar_init(&cempty[s], 1);
        }
        tc::mbar_init(bfull, 1);
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&acc_full[b], 1);
            tc::mbar_init(&acc_empty[b], EPI);
        }
        tc::mbar_init(drain, 1);
        *abort_flag = 0;
        tc::fence_barrier_init();
    }
    if (warp == 1) tmem_alloc_dyn<0>(tmem_slot, a.tmem_cols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            tc::mbar_arrive_expect_tx(bfull, 2u * a.nkb_b * btile);
            for (int kb = 0; kb < a.nkb_b; ++kb) {
                tc::tma_load_2d(Bhi + kb * btile, &tmHhi, bfull, kb * BK, a.c0);
                tc::tma_load_2d(Blo + kb * btile, &tmHlo, bfull, kb * BK, a.c0);
            }
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x)
                for (int kb = 0; kb < a.nkb; ++kb, ++it) {
                    const int s = it % XSTAGES;
                    if (!tc::mbar_wait(&empty[s], ((it / XSTAGES) & 1) ^ 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    if (SU) {
                        tc::mbar_arrive_expect_tx(&full[s], RAW_X);
                        tc::tma_load_2d(Raw + s * RAW_X, &tmU, &full[s], kb * BK, t * BM);
                    } else {
                        tc::mbar_arrive_expect_tx(&full[s], TILE_BYTES);
                        tc::tma_load_2d(As + s * TILE_BYTES, &tmU, &full[s], (kb < a.nkb_b ? kb : kb + a.a_off) * BK,
                                        t * BM);
                    }
                }
            if (!ok) {
                *abort_flag = 1;
                atomicExch(err, 11);
            }
            tc::mbar_wait(bfull, 0, nullptr, 200000000ull);
            for (uint32_t j = 0; j < (uint32_t)XSTAGES && j < it; ++j) {
                const uint32_t last = it - 1 - j;
                tc::mbar_wait(&full[last % XSTAGES], (last / XSTAGES) & 1, nullptr, 200000000ull);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_bf16(BM, a.Nc, 0, 0);
            bool ok = tc::mbar_wait(bfull, 0, abort_flag);
            uint32_t it = 0, tcount = 0;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tcount) {
                const int ab = tcount & 1;
                if (!tc::mbar_wait(&acc_empty[ab], ((tcount >> 1) & 1) ^ 1, abort_flag)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t dt = tmem + ab * a.Nc;
                for (int kb = 0; kb < a.nkb; ++kb, ++it) {
                    const int s = SU ? it % CSTAGES : it % XSTAGES;
                    uint64_t* fb = SU ? &cfull[s] : &full[s];
                    if (!tc::mbar_wait(fb, (SU ? it / CSTAGES : it / XSTAGES) & 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t aa = tc::smem_u32(As + s * TILE_BYTES);
                    const int kbb = kb < a.nkb_b ? kb : kb - a.nkb_b;
                    const uint32_t bh = tc::smem_u32(Bhi + kbb * btile);
                    const uint32_t bl = tc::smem_u32(Blo + kbb * btile);
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint64_t ad = tc::smem_desc(aa + kk * 32, 16, 1024, tc::SWIZZLE_128B);
                        tc::mma_bf16(dt, ad, tc::smem_desc(bh + kk * 32, 16, 1024, tc::SWIZZLE_128B), idesc,
                                     (kb | kk) ? 1u : 0u);
                        tc::mma_bf16(dt, ad, tc::smem_desc(bl + kk * 32, 16, 1024, tc::SWIZZLE_128B), idesc, 1u);
                    }
                    tc::mma_commit(SU ? &cempty[s] : &empty[s]);
                }
                if (ok) tc::mma_commit(&acc_full[ab]);
            }
            if (!ok) {
                *abort_flag = 1;
                atomicExch(err, 12);
                tc::mma_commit(drain);
                tc::mbar_wait(drain, 0, nullptr, 200000000ull);
            }
        }
    } else if (SU && warp >= THREADS / 32) {
        // converters: raw 128 x 64 code tile -> bf16 128 x 128 B rows, 128-byte swizzle
        const int ct = threadIdx.x - THREADS;
        uint32_t it = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x)
            for (int kb = 0; kb < a.nkb; ++kb, ++it) {
                const int s = it % XSTAGES, s2 = it % CSTAGES;
                if (!tc::mbar_wait(&full[s], (it / XSTAGES) & 1, abort_flag) ||
                    !tc::mbar_wait(&cempty[s2], ((it / CSTAGES) & 1) ^ 1, abort_flag)) {
                    ok = false;
                    break;
                }
                const uint8_t* src = Raw + s * RAW_X;
                uint8_t* dst = As + s2 * TILE_BYTES;
#pragma unroll
                for (int p = 0; p < RAW_X / 16 / CONV; ++p) {
                    const int ci = p * CONV + ct;   // 16-code chunk: row ci/4, codes 16*(ci%4) ..
                    const int row = ci >> 2, lc = 2 * (ci & 3), sw = row & 7;
                    uint4 lo, hi;
                    fp8x16_to_bf16(*reinterpret_cast<const uint4*>(src + ci * 16), lo, hi);
                    *reinterpret_cast<uint4*>(dst + row * 128 + ((lc ^ sw) << 4)) = lo;
                    *reinterpret_cast<uint4*>(dst + row * 128 + (((lc + 1) ^ sw) << 4)) = hi;
                }
                tc::fence_proxy_async_smem();
                tc::mbar_arrive(&cfull[s2]);
                tc::mbar_arrive(&empty[s]);
            }
        if (!ok) {
            *abort_flag = 1;
            atomicExch(err, 14);
        }
    } else {
        // epilogue: warps 2-9; lane quarter (warp % 4) gives the TMEM lanes (rows),
        // the two warps of a quarter split the 16-column chunks, 32 columns at a
        // time.  Each thread reads its row's accumulators from TMEM and parks
        // them in a per-warp shared tile (16-byte chunks XOR-swizzled by row, so
        // both the row-wise writes and the column-wise reads are conflict-free);
        // the global side then runs with lanes across columns, 8 rows x 4
        // columns per thread, so every warp access covers 4 rows x 128 bytes.
        // The global operands of a tile's first 32 columns are loaded one tile
        // ahead, overlapping the MMAs of that tile.
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        const int rloc = quarter * 32 + lane;
        const int nch = a.Nc / 16;
        const int nh = (nch + 1) / 2;
        const int cb = half ? nh : 0, ce = half ? nch : nh;
        const int sr = lane >> 3, ch = lane & 7;  // global-side mapping: row offset, 16-byte column chunk
        float4* stg = reinterpret_cast<float4*>(stage) + (warp - 2) * 256;  // 32 rows x 8 chunks
        float4 g1[8], g2[8];
        auto load_ops = [&](int t_, int c0_) {
            const int j = a.c0 + c0_ * 16 + 4 * ch;
            const bool colok = c0_ + (ch >> 2) < ce && j < a.Bp && a.op != EXP_SET_X;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int64_t row_ = (int64_t)t_ * BM + quarter * 32 + sr + 4 * k;
                g1[k] = g2[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (!colok || row_ >= a.n) continue;
                if (a.op == EXP_DIRECTION) {
                    g1[k] = *reinterpret_cast<const float4*>(a.R + row_ * a.Bp + j);
                    g2[k] = *reinterpret_cast<const float4*>(a.P + row_ * a.Bp + j);
                } else {
                    g1[k] = *reinterpret_cast<const float4*>(a.out + row_ * a.Bp + j);
                }
            }
        };
        if ((int)blockIdx.x < ntiles && cb < ce) load_ops(blockIdx.x, cb);
        uint32_t tcount = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tcount) {
            const int ab = tcount & 1;
            const int64_t row = (int64_t)t * BM + rloc;
            const float rsc = (SU && row < a.n) ? __ldg(a.scale + row) : 1.0f;
            if (!tc::mbar_wait(&acc_full[ab], (tcount >> 1) & 1, abort_flag)) {
                ok = false;
                break;
            }
            tc::fence_after_sync();
            for (int c0 = cb; c0 < ce; c0 += 2) {
                if (c0 != cb) load_ops(t, c0);
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    if (c0 + u >= ce) break;
                    float v[16];
                    tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + ab * a.Nc + (c0 + u) * 16, v);
                    tc::tmem_ld_wait();
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float4 w4 = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                        if (SU) {
                            w4.x *= rsc;
                            w4.y *= rsc;
                            w4.z *= rsc;
                            w4.w *= rsc;
                        }
                        stg[lane * 8 + ((u * 4 + q) ^ (lane & 7))] = w4;
                    }
                }
                __syncwarp();
                const int j = a.c0 + c0 * 16 + 4 * ch;
                const bool colok = c0 + (ch >> 2) < ce && j < a.Bp;
                float b0 = 0.f, b1 = 0.f, b2 = 0.f, b3 = 0.f;
                bool f0 = false, f1 = false, f2 = false, f3 = false;
                if (colok && a.op == EXP_DIRECTION) {
                    b0 = (float)a.st[j].beta;
                    b1 = (float)a.st[j + 1].beta;
                    b2 = (float)a.st[j + 2].beta;
                    b3 = (float)a.st[j + 3].beta;
                    // a served column that just took a new request drops r (p0 = U D U^T y + y)
                    f0 = a.st[j].refill;
                    f1 = a.st[j + 1].refill;
                    f2 = a.st[j + 2].refill;
                    f3 = a.st[j + 3].refill;
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int rr = sr + 4 * k;
                    const int64_t row_g = (int64_t)t * BM + quarter * 32 + rr;
                    if (!colok || row_g >= a.n) continue;
                    const float4 acc = stg[rr * 8 + (ch ^ (rr & 7))];
                    float4 w;
                    if (a.op == EXP_SET_X) {
                        w = acc;
                    } else if (a.op == EXP_SUB_R) {
                        w = g1[k];
                        w.x -= acc.x; w.y -= acc.y; w.z -= acc.z; w.w -= acc.w;
                    } else if (a.op == EXP_ADD_Q) {
                        w = g1[k];
                        w.x += acc.x; w.y += acc.y; w.z += acc.z; w.w += acc.w;
                    } else {
                        const float4 r4 = g1[k], p4 = g2[k];
                        w.x = (f0 ? 0.0f : r4.x) + acc.x + (b0 == 0.0f ? 0.0f : b0 * p4.x);
                        w.y = (f1 ? 0.0f : r4.y) + acc.y + (b1 == 0.0f ? 0.0f : b1 * p4.y);
                        w.z = (f2 ? 0.0f : r4.z) + acc.z + (b2 == 0.0f ? 0.0f : b2 * p4.z);
                        w.w = (f3 ? 0.0f : r4.w) + acc.w + (b3 == 0.0f ? 0.0f : b3 * p4.w);
                    }
                    *reinterpret_cast<float4*>(a.out + row_g * a.Bp + j) = w;
                }
                __syncwarp();
            }
            tc::fence_before_sync();
            tc::mbar_arrive(&acc_empty[ab]);
            const int tn = t + gridDim.x;
            if (tn < ntiles && cb < ce) load_ops(tn, cb);
        }
        if (!ok) {
            *abort_flag = 1;
            atomicExch(err, 13);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tmem_dealloc_dyn(tmem, a.tmem_cols);
    }
}

// =====================================================================================
// reduce: part_c = U_chunk^T V_chunk
// =====================================================================================
struct ReduceArgs {
    int64_t n;
    int32_t Bp;
    int32_t c0;          // first column of this launch
    int32_t Nc;          // columns (multiple of 64, <= 256)
    int32_t mt;          // M tiles of 128 eigen-indices
    int32_t rpad;
    int64_t tiles_per_cta;
    int32_t fold;        // U stored as [hi | lo]: M tiles m and m + fold add into output rows of tile m (0: none)
    uint32_t lbo, sbo;   // MN-major descriptor strides (bytes)
    uint32_t tmem_cols;
    const float* V;
    float* part;         // [gridDim.x][rpad][Bp]
    const int* gate;
    const float* scale;  // per-row scale of FP8 storage
};

template <int SU>
__global__ void __launch_bounds__(THREADS + (SU ? CONV : 0), 1)
    k_lr_reduce_tc(const __grid_constant__ CUtensorMap tmU, ReduceArgs a, int* err) {
    if (a.gate && *a.gate == 0) return;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const uint32_t astage = 2 * TILE_BYTES;                 // 128 rows x 128 eigen-indices
    const uint32_t bterm = (uint32_t)(a.Nc / 64) * TILE_BYTES;  // 128 rows x Nc, one bf16 part
    constexpr int NA = SU ? CSTAGES : RSTAGES;
    uint8_t* As = smem;
    uint8_t* Raw = As + NA * astage;                        // raw fp8 stages (SU only)
    uint8_t* Bs = Raw + (SU ? RSTAGES * RAW_R : 0);         // [2 buffers][hi, lo]
    uint64_t* bars = (uint64_t*)(Bs + 4 * bterm);
    uint64_t* full = bars;
    uint64_t* empty = full + RSTAGES;
    uint64_t* bfull = empty + RSTAGES;
    uint64_t* bempty = bfull + 2;
    uint64_t* done = bempty + 2;
    uint64_t* drain = done + 1;
    uint64_t* cfull = drain + 1;
    uint64_t* cempty = cfull + CSTAGES;
    uint32_t* tmem_slot = (uint32_t*)(cempty + CSTAGES);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntiles_all = (a.n + BM - 1) / BM;
    const int64_t t0 = (int64_t)blockIdx.x * a.tiles_per_cta;
    const int64_t t1 = min(ntiles_all, t0 + a.tiles_per_cta);
    const int ntl = t1 > t0 ? (int)(t1 - t0) : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < RSTAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], SU ? CONV : 1);
        }
        for (int s = 0; s < CSTAGES; ++s) {
            tc::mbar_init(&cfull[s], CONV);
            tc::mbar_init(&cempty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&bfull[b], EPI);
            tc::mbar_init(&bempty[b], 1);
        }
        tc::mbar_init(done, 1);
        tc::mbar_init(drain, 1);
        *abort_flag = 0;
        tc::fence_barrier_init();
    }
    if (warp == 1) tmem_alloc_dyn<0>(tmem_slot, a.tmem_cols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t it = 0;
            bool ok = true;
            for (int tl = 0; tl < ntl && ok; ++tl)
                for (int m = 0; m < a.mt; ++m, ++it) {
                    const int s = it % RSTAGES;
                    if (!tc::mbar_wait(&empty[s], ((it / RSTAGES) & 1) ^ 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    const int32_t rowc = (int32_t)((t0 + tl) * BM);
                    if (SU) {
                        tc::mbar_arrive_expect_tx(&full[s], RAW_R);
                        tc::tma_load_2d(Raw + s * RAW_R, &tmU, &full[s], m * 128, rowc);
                    } else {
                        uint8_t* dst = As + s * astage;
                        tc::mbar_arrive_expect_tx(&full[s], astage);
                        tc::tma_load_2d(dst, &tmU, &full[s], m * 128, rowc);
                        tc::tma_load_2d(dst + TILE_BYTES, &tmU, &full[s], m * 128 + 64, rowc);
                    }
                }
            if (!ok) {
                *abort_flag = 1;
                atomicExch(err, 21);
            }
            for (uint32_t j = 0; j < (uint32_t)RSTAGES && j < it; ++j) {
                const uint32_t last = it - 1 - j;
                tc::mbar_wait(&full[last % RSTAGES], (last / RSTAGES) & 1, nullptr, 200000000ull);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_bf16(BM, a.Nc, 1, 1);
            uint32_t it = 0;
            bool ok = true;
            for (int tl = 0; tl < ntl && ok; ++tl) {
                const int buf = tl & 1;
                if (!tc::mbar_wait(&bfull[buf], (tl >> 1) & 1, abort_flag)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t bh = tc::smem_u32(Bs + (2 * buf) * bterm);
                const uint32_t bl = tc::smem_u32(Bs + (2 * buf + 1) * bterm);
                for (int m = 0; m < a.mt; ++m, ++it) {
                    const int s = SU ? it % CSTAGES : it % RSTAGES;
                    uint64_t* fb = SU ? &cfull[s] : &full[s];
                    if (!tc::mbar_wait(fb, (SU ? it / CSTAGES : it / RSTAGES) & 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t aa = tc::smem_u32(As + s * astage);
                    const uint32_t dt = tmem + m * a.Nc;
#pragma unroll
                    for (int kk = 0; kk < BM / 16; ++kk) {
                        const uint64_t ad = tc::smem_desc(aa + kk * 2048, a.lbo, a.sbo, tc::SWIZZLE_128B);
                        tc::mma_bf16(dt, ad, tc::smem_desc(bh + kk * 2048, a.lbo, a.sbo, tc::SWIZZLE_128B), idesc,
                                     (tl | kk) ? 1u : 0u);
                        tc::mma_bf16(dt, ad, tc::smem_desc(bl + kk * 2048, a.lbo, a.sbo, tc::SWIZZLE_128B), idesc, 1u);
                    }
                    tc::mma_commit(SU ? &cempty[s] : &empty[s]);
                }
                if (ok) tc::mma_commit(&bempty[buf]);
            }
            tc::mma_commit(done);
            if (!ok) {
                *abort_flag = 1;
                atomicExch(err, 22);
            }
        }
    } else if (SU && warp >= THREADS / 32) {
        // converters: raw 128 rows x 128 codes -> two MN-major bf16 blocks of 64
        // eigen-indices (128-byte rows, 128-byte swizzle)
        const int ct = threadIdx.x - THREADS;
        uint32_t it = 0;
        bool ok = true;
        for (int tl = 0; tl < ntl && ok; ++tl)
            for (int m = 0; m < a.mt; ++m, ++it) {
                const int s = it % RSTAGES, s2 = it % CSTAGES;
                if (!tc::mbar_wait(&full[s], (it / RSTAGES) & 1, abort_flag) ||
                    !tc::mbar_wait(&cempty[s2], ((it / CSTAGES) & 1) ^ 1, abort_flag)) {
                    ok = false;
                    break;
                }
                const uint8_t* src = Raw + s * RAW_R;
                uint8_t* dst = As + s2 * astage;
#pragma unroll
                for (int p = 0; p < RAW_R / 16 / CONV; ++p) {
                    const int ci = p * CONV + ct;   // 16-code chunk: row ci/8, eigen-indices 16*(ci%8) ..
                    const int rr = ci >> 3, c = ci & 7, sw = rr & 7;
                    const int lc = 2 * (c & 3);
                    uint8_t* blk = dst + (c >> 2) * TILE_BYTES + rr * 128;
                    uint4 lo, hi;
                    fp8x16_to_bf16(*reinterpret_cast<const uint4*>(src + ci * 16), lo, hi);
                    *reinterpret_cast<uint4*>(blk + ((lc ^ sw) << 4)) = lo;
                    *reinterpret_cast<uint4*>(blk + (((lc + 1) ^ sw) << 4)) = hi;
                }
                tc::fence_proxy_async_smem();
                tc::mbar_arrive(&cfull[s2]);
                tc::mbar_arrive(&empty[s]);
            }
        if (!ok) {
            *abort_flag = 1;
            atomicExch(err, 25);
        }
    } else {
        // conversion of V tiles into bf16 hi/lo, MN-major 128-byte swizzle, then the epilogue
        const int tid = threadIdx.x - 64;
        const int quarter = warp & 3;
        const int half = (warp - 2) >> 2;
        bool ok = true;
        // only the columns below Bp are converted: the MMA output columns beyond
        // them are never stored, so their operand bytes in shared memory do not matter
        const int live4 = (a.Bp - a.c0 + 3) / 4;
        const int cq_n = live4 < a.Nc / 4 ? (live4 > 0 ? live4 : 1) : a.Nc / 4;
        const int total = BM * cq_n;
        // V of the next tile is loaded into registers while the current one is
        // converted (one batch when a tile fits EPI x 8 float4, i.e. Nc <= 64)
        const bool one_batch = total <= EPI * 8;
        float4 v[8];
        float vs[8];
        auto load_tile = [&](int tl_, int base_) {
            const int64_t row0_ = (t0 + tl_) * BM;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = base_ + u * EPI;
                v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                vs[u] = 1.0f;
                if (e < total) {
                    const int rr = e / cq_n, j = a.c0 + 4 * (e % cq_n);
                    const int64_t i = row0_ + rr;
                    if (i < a.n && j < a.Bp) {
                        v[u] = *reinterpret_cast<const float4*>(a.V + i * a.Bp + j);
                        if (SU) vs[u] = __ldg(a.scale + i);
                    }
                }
            }
        };
        if (ntl > 0 && one_batch) load_tile(0, tid);
        for (int tl = 0; tl < ntl && ok; ++tl) {
            const int buf = tl & 1;
            if (!tc::mbar_wait(&bempty[buf], ((tl >> 1) & 1) ^ 1, abort_flag)) {
                ok = false;
                break;
            }
            uint8_t* bh = Bs + (2 * buf) * bterm;
            uint8_t* bl = Bs + (2 * buf + 1) * bterm;
            for (int base = tid; base < total; base += EPI * 8) {
                if (!one_batch) load_tile(tl, base);
                float4 cur[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    cur[u] = v[u];
                    if (SU) {
                        cur[u].x *= vs[u];
                        cur[u].y *= vs[u];
                        cur[u].z *= vs[u];
                        cur[u].w *= vs[u];
                    }
                }
                if (one_batch && tl + 1 < ntl) load_tile(tl + 1, tid);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int e = base + u * EPI;
                    if (e >= total) break;
                    const int rr = e / cq_n, jl = 4 * (e % cq_n);
                    __nv_bfloat16 h[4], l[4];
                    const float vv[4] = {cur[u].x, cur[u].y, cur[u].z, cur[u].w};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        h[q] = __float2bfloat16_rn(vv[q]);
                        l[q] = __float2bfloat16_rn(vv[q] - __bfloat162float(h[q]));
                    }
                    const int nb = jl >> 6, jj = jl & 63;
                    const uint32_t off = nb * TILE_BYTES + rr * 128 + ((((jj >> 3) ^ (rr & 7))) << 4) + (jj & 7) * 2;
                    *reinterpret_cast<uint2*>(bh + off) = *reinterpret_cast<const uint2*>(h);
                    *reinterpret_cast<uint2*>(bl + off) = *reinterpret_cast<const uint2*>(l);
                }
            }
            tc::fence_proxy_async_smem();
            tc::mbar_arrive(&bfull[buf]);
        }
        if (!ok) {
            *abort_flag = 1;
            atomicExch(err, 23);
        }
        // epilogue: lane k of M tile m holds sum_i U_{i, m*128+k} V_{i, :}
        float* dst = a.part + (int64_t)blockIdx.x * a.rpad * a.Bp;
        const bool have = ntl > 0 && ok && tc::mbar_wait(done, 0, abort_flag);
        if (ntl > 0 && !have) atomicExch(err, 24);
        tc::fence_after_sync();
        const int nch = a.Nc / 16;
        const int nh = (nch + 1) / 2;
        const int cb = half ? nh : 0, ce = half ? nch : nh;
        const int mt_out = a.fold ? a.fold : a.mt;
        for (int m = 0; m < mt_out; ++m) {
            const int k = m * 128 + quarter * 32 + lane;
            for (int c = cb; c < ce; ++c) {
                float v[16];
                if (have) {
                    tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + m * a.Nc + c * 16, v);
                    tc::tmem_ld_wait();
                    if (a.fold) {
                        float v2[16];
                        tmem_ld16(tmem + ((uint32_t)(quarter * 32) << 16) + (m + a.fold) * a.Nc + c * 16, v2);
                        tc::tmem_ld_wait();
#pragma unroll
                        for (int q = 0; q < 16; ++q) v[q] += v2[q];
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) v[q] = 0.0f;
                }
                if (k < a.rpad) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int j = a.c0 + c * 16 + 4 * q;
                        if (j < a.Bp)
                            *reinterpret_cast<float4*>(dst + (int64_t)k * a.Bp + j) =
                                make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tmem_dealloc_dyn(tmem, a.tmem_cols);
    }
}

// =====================================================================================
// host side
// =====================================================================================
int lr_tc_nchunk(hd_ctx* ctx, int64_t n) {
    int64_t tiles = (n + BM - 1) / BM;
    return (int)std::max<int64_t>(1, std::min<int64_t>(ctx->num_sms, tiles));
}

// The tensor-core kernels record a bounded wait that ran out (mbarrier timeout,
// codes 11-25) in d_flags[2] (expansion) and d_flags[3] (reduction) instead of
// hanging; callers read the flags at their next host synchronisation.
int lr_tc_check_flags(hd_ctx* ctx) {
    HD_CUDA(ctx, cudaMemcpyAsync(ctx->h_poll + 8, ctx->d_flags + 2, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                                 ctx->stream));
    HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->h_poll[8] || ctx->h_poll[9]) {
        const int e = ctx->h_poll[8], r = ctx->h_poll[9];
        HD_CUDA(ctx, cudaMemsetAsync(ctx->d_flags + 2, 0, 2 * sizeof(int), ctx->stream));
        return hd_fail(ctx, HD_ERR_TIMEOUT, "tensor-core pipeline wait ran out (expansion %d, reduction %d)", e, r);
    }
    return HD_OK;
}

int lr_tc_expand(hd_ctx* ctx, const LowRank& lr, int op, float* out, const float* Rv, const float* Pv, int64_t n,
                 int32_t Bp, const ColState* st, const int* gate) {
    const hd_eig* e = lr.e;
    const int su = e->storage == HD_FP8 ? 1 : 0;
    const bool split = e->storage == HD_F32;  // [hi | lo] bf16 copy of the fp32 U
    const int nkb_b = lr.rpad / BK;
    const int nkb = split ? 2 * nkb_b : nkb_b;
    const int a_off = split ? e->lds / 2 / BK - nkb_b : 0;
    CUtensorMap tu;
    if (split ? hd_make_tmap_2d(&tu, e->Usplit, 2, n, e->lds, e->lds, BM, BK, 1)
              : hd_make_tmap_2d(&tu, e->U, su ? 1 : 2, n, e->ldu, e->ldu, BM, BK, su ? 0 : 1))
        return hd_fail(ctx, HD_ERR_CUDA, "tensor map for U failed");
    // column chunks so that H^T (hi + lo) fits next to the A pipeline
    const int max_smem = 227 * 1024 - 2048;
    const int apipe = su ? CSTAGES * TILE_BYTES + XSTAGES * RAW_X : XSTAGES * TILE_BYTES;
    // columns that can be active (the server's occupied slots); the rest keep their values
    const int cols = lr.live > 0 ? std::min(lr.Bp16, (lr.live + 15) / 16 * 16) : lr.Bp16;
    int Nc = cols;
    while (Nc > 16 && (apipe + STAGE_BYTES + 2 * nkb_b * Nc * 128 > max_smem || Nc > 256)) Nc = (Nc / 2 + 15) / 16 * 16;
    if (apipe + STAGE_BYTES + 2 * nkb_b * Nc * 128 > max_smem)
        return hd_fail(ctx, HD_ERR_INVALID_ARG, "rank %d too large for the tensor-core expansion", e->r);
    static uint64_t attr[2] = {0, 0};
    if (hd_first_on_device(attr[su], ctx->device)) {
        HD_CUDA(ctx, cudaFuncSetAttribute(su ? k_lr_expand_tc<1> : k_lr_expand_tc<0>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    }
    for (int c0 = 0; c0 < cols; c0 += Nc) {
        const int nc = std::min(Nc, cols - c0);
        CUtensorMap th, tl;
        if (hd_make_tmap_2d(&th, lr.Hhi, 2, lr.Bp16, lr.rpad, lr.rpad, nc, BK, 1) ||
            hd_make_tmap_2d(&tl, lr.Hlo, 2, lr.Bp16, lr.rpad, lr.rpad, nc, BK, 1))
            return hd_fail(ctx, HD_ERR_CUDA, "tensor map for H failed");
        ExpandArgs a;
        a.n = n;
        a.Bp = Bp;
        a.c0 = c0;
        a.Nc = nc;
        a.nkb = nkb;
        a.nkb_b = nkb_b;
        a.a_off = a_off;
        a.op = op;
        a.tmem_cols = tmem_cols_for(2 * nc);
        a.out = out;
        a.R = Rv;
        a.P = Pv;
        a.st = st;
        a.gate = gate;
        a.scale = e->scale;
        const size_t smem = 1024 + apipe + STAGE_BYTES + 2 * (size_t)nkb_b * nc * 128 + 256;
        const int tiles = (int)((n + BM - 1) / BM);
        const int grid = std::min(tiles, ctx->num_sms);
        if (su)
            k_lr_expand_tc<1><<<grid, THREADS + CONV, smem, ctx->stream>>>(tu, th, tl, a, ctx->d_flags + 2);
        else
            k_lr_expand_tc<0><<<grid, THREADS, smem, ctx->stream>>>(tu, th, tl, a, ctx->d_flags + 2);
        HD_CHECK_LAUNCH(ctx);
    }
    return HD_OK;
}

int lr_tc_reduce(hd_ctx* ctx, const LowRank& lr, const float* V, int64_t n, int32_t Bp, const int* gate) {
    const hd_eig* e = lr.e;
    const int su = e->storage == HD_FP8 ? 1 : 0;
    const bool split = e->storage == HD_F32;
    // with the [hi | lo] copy the M tiles cover both halves (lds / 2 is a multiple of 64)
    const int fold = split ? e->lds / 256 : 0;
    const int mt = split ? 2 * fold : (e->r + 127) / 128;
    CUtensorMap tu;
    int tmrc;
    if (split) tmrc = hd_make_tmap_2d(&tu, e->Usplit, 2, n, e->lds, e->lds, BM, BK, 1);
    else if (su) tmrc = hd_make_tmap_2d(&tu, e->U, 1, n, e->ldu, e->ldu, BM, 128, 0);
    else tmrc = hd_make_tmap_2d(&tu, e->U, 2, n, e->ldu, e->ldu, BM, BK, 1);
    if (tmrc) return hd_fail(ctx, HD_ERR_CUDA, "tensor map for U failed");
    const int Bp64 = lr.live > 0 ? std::min((Bp + 63) / 64 * 64, (lr.live + 63) / 64 * 64) : (Bp + 63) / 64 * 64;
    int Nc = Bp64;
    const int max_smem = 227 * 1024 - 2048;
    const size_t apipe = su ? (size_t)CSTAGES * 2 * TILE_BYTES + (size_t)RSTAGES * RAW_R : (size_t)RSTAGES * 2 * TILE_BYTES;
    auto smem_of = [&](int nc) { return apipe + 4 * (size_t)(nc / 64) * TILE_BYTES; };
    while (Nc > 64 && (smem_of(Nc) > (size_t)max_smem || mt * Nc > 512 || Nc > 256)) Nc -= 64;
    if (mt * Nc > 512 || smem_of(Nc) > (size_t)max_smem)
        return hd_fail(ctx, HD_ERR_INVALID_ARG, "rank %d too large for the tensor-core reduction", e->r);
    static uint64_t attr[2] = {0, 0};
    if (hd_first_on_device(attr[su], ctx->device)) {
        HD_CUDA(ctx, cudaFuncSetAttribute(su ? k_lr_reduce_tc<1> : k_lr_reduce_tc<0>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
    }
    const int64_t tiles = (n + BM - 1) / BM;
    const int grid = lr.nchunk;
    for (int c0 = 0; c0 < Bp64; c0 += Nc) {
        const int nc = std::min(Nc, Bp64 - c0);
        ReduceArgs a;
        a.n = n;
        a.Bp = Bp;
        a.c0 = c0;
        a.Nc = nc;
        a.mt = mt;
        a.fold = fold;
        a.rpad = lr.rpad;
        a.tiles_per_cta = (tiles + grid - 1) / grid;
        // MN-major operands: the leading byte offset steps between the 64-element
        // blocks of M (or N), the stride byte offset between groups of 8 K rows
        a.lbo = TILE_BYTES;
        a.sbo = 1024;
        a.tmem_cols = tmem_cols_for(mt * nc);
        a.V = V;
        a.part = lr.part;
        a.gate = gate;
        a.scale = e->scale;
        const size_t smem = 1024 + smem_of(nc) + 256;
        if (su)
            k_lr_reduce_tc<1><<<grid, THREADS + CONV, smem, ctx->stream>>>(tu, a, ctx->d_flags + 3);
        else
            k_lr_reduce_tc<0><<<grid, THREADS, smem, ctx->stream>>>(tu, a, ctx->d_flags + 3);
        HD_CHECK_LAUNCH(ctx);
    }
    return HD_OK;
}

// ------------------------------------------------------------------ bounded-wait self-test
// One warp: lane 0 waits on an mbarrier that nothing completes (it must give
// up after limit_ns), then on a second one while lane 1 raises the abort flag
// (it must give up at once).  out[0] / out[1]: 1 when each wait gave up.
__global__ void k_wait_selftest(uint64_t limit_ns, int* out) {
    __shared__ uint64_t bar[2];
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
        abort_flag = 0;
        tc::fence_barrier_init();
    }
    __syncwarp();
    if (threadIdx.x == 0) out[0] = tc::mbar_wait(&bar[0], 0, nullptr, limit_ns) ? 0 : 1;
    __syncwarp();
    if (threadIdx.x == 1) *(volatile int*)&abort_flag = 1;
    __syncwarp();
    if (threadIdx.x == 0) out[1] = tc::mbar_wait(&bar[1], 0, (volatile int*)&abort_flag, 1000000000ull) ? 0 : 1;
}

extern "C" int hd_selftest_wait(hd_ctx* ctx, uint32_t limit_us, int32_t* gave_up) {
    if (!ctx || !gave_up || limit_us == 0 || limit_us > 1000000) return HD_ERR_INVALID_ARG;
    HD_CUDA(ctx, cudaSetDevice(ctx->device));
    HD_CUDA(ctx, cudaMemsetAsync(ctx->d_flags + 4, 0, 2 * sizeof(int), ctx->stream));
    k_wait_selftest<<<1, 32, 0, ctx->stream>>>((uint64_t)limit_us * 1000ull, ctx->d_flags + 4);
    HD_CHECK_LAUNCH(ctx);
    HD_CUDA(ctx, cudaMemcpyAsync(ctx->h_poll + 12, ctx->d_flags + 4, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                                 ctx->stream));
    HD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    gave_up[0] = ctx->h_poll[12];
    gave_up[1] = ctx->h_poll[13];
    return (gave_up[0] && gave_up[1]) ? HD_ERR_TIMEOUT : HD_OK;
}
