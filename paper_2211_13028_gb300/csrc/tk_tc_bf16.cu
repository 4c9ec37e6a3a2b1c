// Tensor-core mode-j contraction (TTM) for BF16 data on sm_103a.
//
//   out[l + L*(a + m*r)] = sum_i M(i, a) X[l + L*(i + n_j*r)]     (X viewed as L x n_j x R)
//
// X is BF16 in memory, so its tiles feed tcgen05.mma directly from shared
// memory: no conversion pass, no TMEM staging of A.  The factor M is split
// into BF16 parts M = M_hi + M_lo + O(2^-18 |M|) (the refinement pass: the
// second part wins back the subspace accuracy a single BF16 rounding of Q
// would lose), and one MMA per 16-deep K step computes X * [M_hi ; M_lo]
// (N = 2 NPAD, the halves land in separate TMEM columns and are summed by the
// epilogue).  Products of BF16 values are exact in the FP32 accumulator.
//
// Kernel structure (persistent, one CTA of 6 warps per SM):
//   warp 0      TMA producer: 64-deep K chunks of a 128-row tile of X (16 KB) and the
//               matching 64 x NPAD chunks of M_hi and M_lo into an SMEM ring.
//   warp 1      allocates TMEM; lane 0 issues tcgen05.mma.kind::f16 with A and B
//               read from SMEM descriptors (A K-major for a contraction over the
//               contiguous mode, MN-major otherwise; 128-byte swizzle).
//   warps 2-5   epilogue: tcgen05.ld of a double-buffered accumulator, halves
//               summed, rows written to global memory.
// Every mbarrier wait is bounded by a wall-clock limit; on expiry the CTA raises
// FLAG_TIMEOUT, stops issuing work, drains what it issued and frees its TMEM.
#include <cuda_bf16.h>

#include "tk_tc_common.cuh"

namespace tk {
namespace bf {

using tc::gtimer;
using tc::kTimeoutNs;
using tc::mbar_arrive;
using tc::mbar_expect_tx;
using tc::mbar_init;
using tc::mbar_try_wait;
using tc::mbar_wait;
using tc::smem_u32;

constexpr int kThreads = 192;
constexpr int kRows = 128;                   // tile rows (TMEM lanes)
constexpr int kChunk = 64;                   // K elements per stage: one 128-byte row of BF16
constexpr int kXBytes = kRows * kChunk * 2;  // 16 KB

// D[tmem] (+)= A[smem desc] * B[smem desc], kind::f16 (BF16 inputs, FP32 accumulate), M = 128.
__device__ __forceinline__ void mma_bf16_ss(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Instruction descriptor: D F32, A and B BF16, B K-major, A K-major or MN-major
// (bit 15), M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_bf16(int n, bool a_mn_major) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn_major ? 1u : 0u) << 15) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(kRows >> 4) << 24);
}

// Shared-memory descriptor of an MN-major operand in the 128-byte-swizzle
// layout: 64 contiguous MN elements per 128-byte row, 8 rows (K) per 1 KB
// swizzle atom; lbo = byte distance between atoms along MN, sbo = between
// 8-row groups along K.
__device__ __forceinline__ uint64_t desc_mn_sw128(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version
    d |= (uint64_t)2 << 61;  // 128-byte swizzle
    return d;
}

struct BfArgs {
    int64_t L, nj, R, m;
    int64_t ntiles, tiles_per_r, nk, nblk;  // work item = (row tile, block of NPAD output columns)
    int64_t rows_b;                         // rows of M_hi in the split factor (M_lo follows)
    float* out;
    unsigned* flags;
};

template <int NPAD>
struct BfCfg {
    static constexpr int kBBytes = NPAD * 128;  // one of M_hi / M_lo: NPAD rows of 128 B
    static constexpr int kStage = kXBytes + 2 * kBBytes;
    static constexpr int kBudget = 200 * 1024;
    static constexpr int kStages = kBudget / kStage > 12 ? 12 : kBudget / kStage;
    static constexpr int kSmem = kStages * kStage + 1024 + 256;
    static_assert(kStages >= 2, "SMEM budget");
    static_assert(kStage % 1024 == 0, "stages must keep 1 KB swizzle alignment");
    static_assert(4 * NPAD <= 512, "TMEM budget");
};

template <int NPAD, bool KMAJOR>
__global__ void __launch_bounds__(kThreads, 1)
    ttm_bf16_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmB, BfArgs args) {
    using C = BfCfg<NPAD>;
    constexpr int S = C::kStages;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * C::kStage);
    uint64_t* full = bars;            // [S] TMA landed
    uint64_t* empty = bars + S;       // [S] stage consumed (MMA commit)
    uint64_t* accfull = bars + 2 * S; // [2] accumulator complete (MMA commit)
    uint64_t* accempty = accfull + 2; // [2] accumulator drained (one arrival per epilogue warp)
    uint64_t* done = accempty + 2;    // [1] every issued MMA complete
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accfull[b], 1);
            mbar_init(&accempty[b], 4);
        }
        mbar_init(done, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        tc::tc_fence_before();
    }
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tbase = *tmem_slot;
    unsigned* flags = args.flags;
    const int64_t nk = args.nk;
    const int64_t nitems = args.ntiles * args.nblk;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            int64_t it = 0;
            bool ok = true;
            for (int64_t w = blockIdx.x; w < nitems && ok; w += gridDim.x) {
                const int64_t t = w / args.nblk, nb = w % args.nblk;
                int64_t r0 = 0, l0 = 0, rr = 0;
                if (KMAJOR) {
                    r0 = t * kRows;
                } else {
                    rr = t / args.tiles_per_r;
                    l0 = (t % args.tiles_per_r) * kRows;
                }
                for (int64_t kc = 0; kc < nk; ++kc, ++it) {
                    const int s = (int)(it % S);
                    const uint32_t ph = (uint32_t)((it / S) & 1);
                    if (!mbar_wait(&empty[s], ph ^ 1, abort, flags)) {
                        ok = false;
                        break;
                    }
                    uint8_t* xs = smem + s * C::kStage;
                    uint8_t* bs = xs + kXBytes;
                    mbar_expect_tx(&full[s], kXBytes + 2 * C::kBBytes);
                    if (KMAJOR) {
                        tc::tma_load_2d(xs, &tmX, (int)(kc * kChunk), (int)r0, &full[s]);
                    } else {
                        tc::tma_load_3d(xs, &tmX, (int)l0, (int)(kc * kChunk), (int)rr, &full[s]);
                        tc::tma_load_3d(xs + kXBytes / 2, &tmX, (int)(l0 + 64), (int)(kc * kChunk), (int)rr, &full[s]);
                    }
                    tc::tma_load_2d(bs, &tmB, (int)(kc * kChunk), (int)(nb * NPAD), &full[s]);
                    tc::tma_load_2d(bs + C::kBBytes, &tmB, (int)(kc * kChunk), (int)(args.rows_b + nb * NPAD),
                                    &full[s]);
                }
            }
            // drain: every issued load has landed before the CTA can exit
            const int64_t n_out = it < S ? it : S;
            for (int64_t q = it - n_out; q < it; ++q) {
                const uint64_t t0 = gtimer();
                while (!mbar_try_wait(&full[q % S], (uint32_t)((q / S) & 1)) && gtimer() - t0 < kTimeoutNs) {
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            int64_t it = 0, acc = 0;
            bool ok = true;
            constexpr uint32_t idesc = idesc_bf16(2 * NPAD, !KMAJOR);
            for (int64_t w = blockIdx.x; w < nitems && ok; w += gridDim.x, ++acc) {
                const int a = (int)(acc & 1);
                if (!mbar_wait(&accempty[a], (uint32_t)(((acc >> 1) & 1) ^ 1), abort, flags)) {
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t d_tmem = tbase + a * 2 * NPAD;
                for (int64_t kc = 0; kc < nk; ++kc, ++it) {
                    const int s = (int)(it % S);
                    if (!mbar_wait(&full[s], (uint32_t)((it / S) & 1), abort, flags)) {
                        ok = false;
                        break;
                    }
                    tc::tc_fence_after();
                    const uint32_t xs = smem_u32(smem + s * C::kStage);
                    const uint32_t bs = xs + kXBytes;
#pragma unroll
                    for (int k16 = 0; k16 < kChunk / 16; ++k16) {
                        // A: K-major rows of 128 B (advance 32 B per 16 elements of K), or MN-major
                        // boxes of 64 K-rows x 128 B, the second 64 rows of the tile 8 KB further
                        // (lbo) and 8-row K groups 1 KB apart (sbo; advance 2 KB per 16 of K).
                        const uint64_t adesc = KMAJOR ? tc::desc_sw128(xs + 32 * k16)
                                                      : desc_mn_sw128(xs + 2048 * k16, kXBytes / 2, 1024);
                        const uint64_t bdesc = tc::desc_sw128(bs + 32 * k16);
                        mma_bf16_ss(d_tmem, adesc, bdesc, idesc, (kc | k16) != 0);
                    }
                    tc::tc_commit(&empty[s]);
                }
                if (!ok) break;
                tc::tc_commit(&accfull[a]);
            }
            tc::tc_commit(done);
            const uint64_t t0 = gtimer();
            while (!mbar_try_wait(done, 0) && gtimer() - t0 < kTimeoutNs) {
            }
        }
    } else {
        // ------------------------------------------------ epilogue (warps 2-5: TMEM lane quarter = warp % 4)
        const int q = warp & 3;
        const int rho = 32 * q + lane;
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        int64_t acc = 0;
        for (int64_t w = blockIdx.x; w < nitems; w += gridDim.x, ++acc) {
            const int64_t t = w / args.nblk, nb = w % args.nblk;
            const int a = (int)(acc & 1);
            const bool got = mbar_wait(&accfull[a], (uint32_t)((acc >> 1) & 1), abort, flags);
            if (!__all_sync(0xffffffffu, got)) break;  // warp-uniform: tcgen05.ld below is .aligned
            tc::tc_fence_after();
            int64_t base, stride;
            bool valid;
            if (KMAJOR) {
                const int64_t r = t * kRows + rho;
                valid = r < args.R;
                base = r * args.m;
                stride = 1;
            } else {
                const int64_t rr = t / args.tiles_per_r;
                const int64_t l = (t % args.tiles_per_r) * kRows + rho;
                valid = l < args.L;
                base = l + args.L * args.m * rr;
                stride = args.L;
            }
            const int64_t col0 = nb * NPAD;
            base += col0 * stride;
            const int64_t ncol = args.m - col0;
            const uint32_t ta = tbase + lane_base + a * 2 * NPAD;
#pragma unroll
            for (int c0 = 0; c0 < NPAD; c0 += 16) {
                float h[16], g[16];
                __syncwarp();
                tc::tmem_ld16(ta + c0, h);
                tc::tmem_ld16(ta + NPAD + c0, g);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (valid) {
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (c0 + i < ncol) args.out[base + (c0 + i) * stride] = h[i] + g[i];
                }
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&accempty[a]);
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc::tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tbase) : "memory");
    }
}

// hi = rn_bf16(M(i, a)), lo = rn_bf16(M(i, a) - hi) (zero when with_lo == 0: a
// single BF16 rounding of M), K-major: hi (i, a) at i + ldo*a, lo at
// i + ldo*(rows_b + a); zero beyond nj and m.
__global__ void split_bf16_kernel(const void* M, tk_dtype dt, int64_t ldm, int mtrans, int64_t nj, int64_t m,
                                  int64_t rows_b, int64_t ldo, int with_lo, __nv_bfloat16* out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ldo * rows_b) return;
    const int64_t i = idx % ldo, a = idx / ldo;
    double v = 0.0;
    if (i < nj && a < m) {
        const int64_t o = mtrans ? a + ldm * i : i + ldm * a;
        v = dt == TK_F64 ? static_cast<const double*>(M)[o] : (double)static_cast<const float*>(M)[o];
    }
    const __nv_bfloat16 h = __double2bfloat16(v);
    const __nv_bfloat16 l = __double2bfloat16(with_lo ? v - (double)__bfloat162float(h) : 0.0);
    out[idx] = h;
    out[idx + ldo * rows_b] = l;
}

template <int NPAD, bool KMAJOR>
static void launch_kernel(const Ctx& c, const CUtensorMap& tx, const CUtensorMap& tb, const BfArgs& a) {
    using Cf = BfCfg<NPAD>;
    auto kern = ttm_bf16_kernel<NPAD, KMAJOR>;
    static bool attr_set = false;
    if (!attr_set) {
        TK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cf::kSmem));
        attr_set = true;
    }
    const int grid = (int)std::min<int64_t>(a.ntiles * a.nblk, tc::grid_sms(c));
    kern<<<grid, kThreads, Cf::kSmem, c.stream>>>(tx, tb, a);
}

}  // namespace bf

bool ttm_bf16_eligible(const Tens& X, int j, int64_t m, tk_dtype out_dt) {
    if (X.dt != TK_BF16 || out_dt != TK_F32) return false;
    if (m < 1 || m > 65535) return false;
    const int64_t L = X.left(j), nj = X.n[j], R = X.right(j);
    if (nj < 16 || ((uintptr_t)X.p % 16) != 0) return false;
    if (L >= ((int64_t)1 << 31) || R >= ((int64_t)1 << 31) || nj >= ((int64_t)1 << 31)) return false;
    if (L == 1) return nj % 8 == 0;  // K-major: 16-byte row stride
    return L % 8 == 0;               // MN-major: 16-byte stride of the i index
}

void launch_ttm_bf16(Ctx& c, const Tens& X, int j, const Mat& M, bool mtrans, int64_t m, float* out) {
    const int64_t L = X.left(j), nj = X.n[j], R = X.right(j);
    int64_t npad, nblk;
    if (m <= 96) {
        npad = (m + 15) / 16 * 16;
        nblk = 1;
    } else {
        npad = 64;
        nblk = (m + 63) / 64;
    }
    const int64_t ldo = (nj + 7) / 8 * 8;
    const int64_t rows_b = npad * nblk;
    __nv_bfloat16* split = static_cast<__nv_bfloat16*>(c.alloc_bytes(sizeof(__nv_bfloat16) * 2 * ldo * rows_b));
    if (!c.exec) return;
    {
        const int64_t tot = ldo * rows_b;
        ProfScope ps(c, "elementwise", 4.0 * tot + 8.0 * nj * m, 0.0);
        bf::split_bf16_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, c.stream>>>(M.p, M.dt, M.ld, mtrans ? 1 : 0,
                                                                                   nj, m, rows_b, ldo,
                                                                                   c.refine == -1 ? 0 : 1, split);
        c.counted();
        c.check_launch();
    }
    CUtensorMap tx, tb;
    const bool kmajor = (L == 1);
    if (kmajor) {
        const uint64_t dims[2] = {(uint64_t)nj, (uint64_t)R};
        const uint64_t str[1] = {(uint64_t)nj * 2};
        const uint32_t box[2] = {bf::kChunk, bf::kRows};
        tc::encode(&tx, X.p, 2, dims, str, box, true, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
    } else {
        const uint64_t dims[3] = {(uint64_t)L, (uint64_t)nj, (uint64_t)R};
        const uint64_t str[2] = {(uint64_t)L * 2, (uint64_t)L * nj * 2};
        const uint32_t box[3] = {64, bf::kChunk, 1};
        tc::encode(&tx, X.p, 3, dims, str, box, true, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
    }
    {
        const uint64_t dims[2] = {(uint64_t)nj, (uint64_t)(2 * rows_b)};
        const uint64_t str[1] = {(uint64_t)ldo * 2};
        const uint32_t box[2] = {bf::kChunk, (uint32_t)npad};
        tc::encode(&tb, split, 2, dims, str, box, true, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16);
    }
    bf::BfArgs a;
    a.L = L;
    a.nj = nj;
    a.R = R;
    a.m = m;
    a.nk = (nj + bf::kChunk - 1) / bf::kChunk;
    a.nblk = nblk;
    a.tiles_per_r = kmajor ? 1 : (L + bf::kRows - 1) / bf::kRows;
    a.ntiles = kmajor ? (R + bf::kRows - 1) / bf::kRows : R * a.tiles_per_r;
    a.rows_b = rows_b;
    a.out = out;
    a.flags = c.dflags;
    const char* name = ((const void*)X.p == c.xdata || L * R * m == c.xnumel) ? "xpass_tc" : "ttm_tc";
    ProfScope ps(c, name, 2.0 * (double)L * R * nj + 4.0 * nj * m + 4.0 * (double)L * R * m,
                 2.0 * (double)L * R * nj * m);
#define TK_BF_CASE(NP)                                            \
    case NP:                                                      \
        if (kmajor) bf::launch_kernel<NP, true>(c, tx, tb, a);    \
        else bf::launch_kernel<NP, false>(c, tx, tb, a);          \
        break;
    switch (npad) {
        TK_BF_CASE(16)
        TK_BF_CASE(32)
        TK_BF_CASE(48)
        TK_BF_CASE(64)
        TK_BF_CASE(80)
        TK_BF_CASE(96)
        default: fail(TK_ERR_SHAPE, "ttm_bf16: unsupported width");
    }
#undef TK_BF_CASE
    c.counted();
    c.check_launch();
}

}  // namespace tk
