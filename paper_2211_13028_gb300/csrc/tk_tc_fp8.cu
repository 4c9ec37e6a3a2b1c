// Tensor-core mode-1 contraction (TTM over the contiguous mode) for FP8 (E4M3)
// data on sm_103a.
//
//   out[a + m*r] = inv * sum_i M(i, a) Xq[i + n_1*r]     (X = Xq / x_scale, viewed as n_1 x R)
//
// X is E4M3 in memory and contiguous along the contracted mode, so its tiles
// feed tcgen05.mma.kind::f8f6f4 straight from shared memory as a K-major
// operand (128-byte rows of 128 elements, 128-byte swizzle).  Both operands of
// that MMA are 8-bit, so the factor is carried as E4M3 pieces, each with its
// own power-of-two scale: with s chosen so that max |M| s lies in (224, 448],
// r_0 = M s, q_t = e4m3(r_t 2^(4t)) and r_{t+1} = r_t - q_t 2^(-4t).  E4M3
// rounding leaves at most 2^-4 of a normal value, so every q_t stays in
// (-448, 448] and, scaled up by 2^(4t), clear of E4M3's subnormal floor for the
// larger entries: four pieces represent M s to ~4e-7 (relative Frobenius error of
// the product on orthonormal and Gaussian factors; a single scale for all pieces
// stalls near 1e-5 on that floor).  One MMA per 32-deep K step computes
// Xq [q_0 ; q_1 ; q_2 ; q_3] (N = 4 NPAD); the pieces land in separate TMEM column
// groups (products of E4M3 values are exact in the FP32 accumulator), and the
// epilogue sums them with their scales 2^(-4t), smallest first, times
// inv = 1 / (x_scale s).
//
// Kernel structure (persistent, one CTA of 6 warps per SM), as the BF16 kernel:
//   warp 0      TMA producer: 128-deep K chunks of a 128-row tile of X (16 KB) and
//               the matching 128 x NPAD chunks of the four pieces into an SMEM ring.
//   warp 1      allocates TMEM; lane 0 issues the MMAs.
//   warps 2-5   epilogue: tcgen05.ld of a double-buffered accumulator, pieces
//               summed, rows written to global memory.
// Every mbarrier wait is bounded by a wall-clock limit; on expiry the CTA raises
// FLAG_TIMEOUT, stops issuing work, drains what it issued and frees its TMEM.
#include <cuda_fp8.h>

#include "tk_tc_common.cuh"

namespace tk {
namespace f8 {

using tc::gtimer;
using tc::kTimeoutNs;
using tc::mbar_arrive;
using tc::mbar_expect_tx;
using tc::mbar_init;
using tc::mbar_try_wait;
using tc::mbar_wait;
using tc::smem_u32;

constexpr int kThreads = 192;
constexpr int kRows = 128;              // tile rows (TMEM lanes)
constexpr int kChunk = 128;             // K elements per stage: one 128-byte row of E4M3
constexpr int kXBytes = kRows * kChunk;  // 16 KB
constexpr int kPieces = 4;

// D[tmem] (+)= A[smem desc] * B[smem desc], kind::f8f6f4 (E4M3 inputs, FP32 accumulate), M = 128.
__device__ __forceinline__ void mma_f8_ss(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Instruction descriptor: D F32, A and B E4M3 (format 0), both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_e4m3(int n) {
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
}

struct F8Args {
    int64_t R, m;
    int64_t ntiles, nk, nblk;  // work item = (row tile, block of NPAD output columns)
    int64_t rows_b;            // rows of one piece in the split factor
    float x_inv;               // 1 / x_scale
    const float* m_scale;      // device: the factor's power-of-two scale s
    float* out;
    unsigned* flags;
};

template <int NPAD>
struct F8Cfg {
    static constexpr int kBBytes = NPAD * 128;  // one piece: NPAD rows of 128 B
    static constexpr int kStage = kXBytes + kPieces * kBBytes;
    static constexpr int kBudget = 200 * 1024;
    static constexpr int kStages = kBudget / kStage > 12 ? 12 : kBudget / kStage;
    static constexpr int kSmem = kStages * kStage + 1024 + 256;
    static constexpr int kAccCols = kPieces * NPAD;
    static_assert(kStages >= 2, "SMEM budget");
    static_assert(kStage % 1024 == 0, "stages must keep 1 KB swizzle alignment");
    static_assert(2 * kAccCols <= 512, "TMEM budget");
    static_assert(kAccCols <= 256, "N of one MMA");
};

template <int NPAD>
__global__ void __launch_bounds__(kThreads, 1)
    ttm_fp8_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmB, F8Args args) {
    using C = F8Cfg<NPAD>;
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
                const int64_t r0 = t * kRows;
                for (int64_t kc = 0; kc < nk; ++kc, ++it) {
                    const int s = (int)(it % S);
                    const uint32_t ph = (uint32_t)((it / S) & 1);
                    if (!mbar_wait(&empty[s], ph ^ 1, abort, flags)) {
                        ok = false;
                        break;
                    }
                    uint8_t* xs = smem + s * C::kStage;
                    uint8_t* bs = xs + kXBytes;
                    mbar_expect_tx(&full[s], kXBytes + kPieces * C::kBBytes);
                    tc::tma_load_2d(xs, &tmX, (int)(kc * kChunk), (int)r0, &full[s]);
#pragma unroll
                    for (int pc = 0; pc < kPieces; ++pc)
                        tc::tma_load_2d(bs + pc * C::kBBytes, &tmB, (int)(kc * kChunk),
                                        (int)(pc * args.rows_b + nb * NPAD), &full[s]);
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
            constexpr uint32_t idesc = idesc_e4m3(C::kAccCols);
            for (int64_t w = blockIdx.x; w < nitems && ok; w += gridDim.x, ++acc) {
                const int a = (int)(acc & 1);
                if (!mbar_wait(&accempty[a], (uint32_t)(((acc >> 1) & 1) ^ 1), abort, flags)) {
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
                const uint32_t d_tmem = tbase + a * C::kAccCols;
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
                    for (int k32 = 0; k32 < kChunk / 32; ++k32) {
                        // K-major rows of 128 B: advance 32 B per 32 elements of K; the pieces are
                        // consecutive NPAD-row groups of B (8-row groups 1 KB apart)
                        mma_f8_ss(d_tmem, tc::desc_sw128(xs + 32 * k32), tc::desc_sw128(bs + 32 * k32), idesc,
                                  (kc | k32) != 0);
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
        const float inv = args.x_inv / *args.m_scale;
        int64_t acc = 0;
        for (int64_t w = blockIdx.x; w < nitems; w += gridDim.x, ++acc) {
            const int64_t t = w / args.nblk, nb = w % args.nblk;
            const int a = (int)(acc & 1);
            const bool got = mbar_wait(&accfull[a], (uint32_t)((acc >> 1) & 1), abort, flags);
            if (!__all_sync(0xffffffffu, got)) break;  // warp-uniform: tcgen05.ld below is .aligned
            tc::tc_fence_after();
            const int64_t r = t * kRows + rho;
            const bool valid = r < args.R;
            const int64_t col0 = nb * NPAD;
            const int64_t base = r * args.m + col0;
            const int64_t ncol = args.m - col0;
            const uint32_t ta = tbase + lane_base + a * C::kAccCols;
#pragma unroll
            for (int c0 = 0; c0 < NPAD; c0 += 16) {
                float p[kPieces][16];
                __syncwarp();
#pragma unroll
                for (int pc = 0; pc < kPieces; ++pc) tc::tmem_ld16(ta + pc * NPAD + c0, p[pc]);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (valid) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        float v = p[kPieces - 1][i];
#pragma unroll
                        for (int pc = kPieces - 2; pc >= 0; --pc) v = fmaf(v, 0.0625f, p[pc][i]);  // q_t 2^(-4t)
                        if (c0 + i < ncol) args.out[base + c0 + i] = v * inv;
                    }
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

// s = 2^e with max |M| s in (224, 448] (1 when M is zero), into *scale.
__global__ void __launch_bounds__(1024) fp8_factor_scale_kernel(const void* M, tk_dtype dt, int64_t ldm, int mtrans,
                                                                int64_t nj, int64_t m, float* scale) {
    __shared__ float red[32];
    float amax = 0.f;
    for (int64_t e = threadIdx.x; e < nj * m; e += blockDim.x) {
        const int64_t i = e % nj, a = e / nj;
        const int64_t o = mtrans ? a + ldm * i : i + ldm * a;
        const float v = dt == TK_F64 ? (float)static_cast<const double*>(M)[o] : static_cast<const float*>(M)[o];
        amax = fmaxf(amax, fabsf(v));
    }
    for (int o = 16; o; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = amax;
    __syncthreads();
    if (threadIdx.x == 0) {
        float mx = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mx = fmaxf(mx, red[w]);
        int e = 0;
        if (mx > 0.f && isfinite(mx)) {
            frexpf(448.f / mx, &e);  // 448 / mx = f 2^e with f in [0.5, 1): s = 2^(e-1) <= 448 / mx < 2^e
            e -= 1;
        }
        *scale = ldexpf(1.f, e);
    }
}

// Piece t of M s (t = 0..3), E4M3, K-major: (i, a) of piece t at i + ldo (t rows_b + a); zero beyond nj
// and m.  q_t = e4m3(r_t 2^(4t)) with r_0 = M s and r_{t+1} = r_t - q_t 2^(-4t) (round to nearest even,
// saturating).
__global__ void split_fp8_kernel(const void* M, tk_dtype dt, int64_t ldm, int mtrans, int64_t nj, int64_t m,
                                 int64_t rows_b, int64_t ldo, const float* scale, __nv_fp8_e4m3* out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ldo * rows_b) return;
    const int64_t i = idx % ldo, a = idx / ldo;
    double r = 0.0;
    if (i < nj && a < m) {
        const int64_t o = mtrans ? a + ldm * i : i + ldm * a;
        r = (dt == TK_F64 ? static_cast<const double*>(M)[o] : (double)static_cast<const float*>(M)[o]) *
            (double)*scale;
    }
    double up = 1.0;
#pragma unroll
    for (int t = 0; t < kPieces; ++t) {
        const __nv_fp8_e4m3 q(r * up);
        out[idx + ldo * rows_b * t] = q;
        r -= (double)(float)q / up;
        up *= 16.0;
    }
}

template <int NPAD>
static void launch_kernel(const Ctx& c, const CUtensorMap& tx, const CUtensorMap& tb, const F8Args& a) {
    using Cf = F8Cfg<NPAD>;
    auto kern = ttm_fp8_kernel<NPAD>;
    static bool attr_set = false;
    if (!attr_set) {
        TK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cf::kSmem));
        attr_set = true;
    }
    const int grid = (int)std::min<int64_t>(a.ntiles * a.nblk, tc::grid_sms(c));
    kern<<<grid, kThreads, Cf::kSmem, c.stream>>>(tx, tb, a);
}

}  // namespace f8

bool ttm_fp8_eligible(const Tens& X, int j, int64_t m, tk_dtype out_dt) {
    if (X.dt != TK_FP8_E4M3 || out_dt != TK_F32) return false;
    if (m < 1 || m > 65535) return false;
    const int64_t L = X.left(j), nj = X.n[j], R = X.right(j);
    if (L != 1) return false;  // the contracted mode must be the contiguous one (K-major operand)
    if (nj < 32 || nj % 16 != 0 || ((uintptr_t)X.p % 16) != 0) return false;  // 16-byte row stride
    return R >= f8::kRows && R < ((int64_t)1 << 31) && nj < ((int64_t)1 << 31);
}

void launch_ttm_fp8(Ctx& c, const Tens& X, int j, const Mat& M, bool mtrans, int64_t m, float* out) {
    const int64_t nj = X.n[j], R = X.right(j);
    int64_t npad, nblk;
    if (m <= 64) {
        npad = (m + 15) / 16 * 16;
        nblk = 1;
    } else {
        npad = 64;
        nblk = (m + 63) / 64;
    }
    const int64_t ldo = (nj + 15) / 16 * 16;
    const int64_t rows_b = npad * nblk;
    __nv_fp8_e4m3* split = static_cast<__nv_fp8_e4m3*>(c.alloc_bytes((size_t)f8::kPieces * ldo * rows_b));
    float* scale = c.alloc<float>(1);
    if (!c.exec) return;
    {
        const int64_t tot = ldo * rows_b;
        ProfScope ps(c, "elementwise", 4.0 * tot + 8.0 * nj * m, 0.0);
        f8::fp8_factor_scale_kernel<<<1, 1024, 0, c.stream>>>(M.p, M.dt, M.ld, mtrans ? 1 : 0, nj, m, scale);
        c.counted();
        c.check_launch();
        f8::split_fp8_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, c.stream>>>(M.p, M.dt, M.ld, mtrans ? 1 : 0,
                                                                                   nj, m, rows_b, ldo, scale, split);
        c.counted();
        c.check_launch();
    }
    CUtensorMap tx, tb;
    {
        const uint64_t dims[2] = {(uint64_t)nj, (uint64_t)R};
        const uint64_t str[1] = {(uint64_t)nj};
        const uint32_t box[2] = {f8::kChunk, f8::kRows};
        tc::encode(&tx, X.p, 2, dims, str, box, true, CU_TENSOR_MAP_DATA_TYPE_UINT8);
    }
    {
        const uint64_t dims[2] = {(uint64_t)nj, (uint64_t)(f8::kPieces * rows_b)};
        const uint64_t str[1] = {(uint64_t)ldo};
        const uint32_t box[2] = {f8::kChunk, (uint32_t)npad};
        tc::encode(&tb, split, 2, dims, str, box, true, CU_TENSOR_MAP_DATA_TYPE_UINT8);
    }
    f8::F8Args a;
    a.R = R;
    a.m = m;
    a.nk = (nj + f8::kChunk - 1) / f8::kChunk;
    a.nblk = nblk;
    a.ntiles = (R + f8::kRows - 1) / f8::kRows;
    a.rows_b = rows_b;
    a.x_inv = 1.f / X.scale;
    a.m_scale = scale;
    a.out = out;
    a.flags = c.dflags;
    const char* name = ((const void*)X.p == c.xdata || R * m == c.xnumel) ? "xpass_tc" : "ttm_tc";
    ProfScope ps(c, name, 1.0 * (double)R * nj + 4.0 * nj * m + 4.0 * (double)R * m, 2.0 * (double)R * nj * m);
    switch (npad) {
        case 16: f8::launch_kernel<16>(c, tx, tb, a); break;
        case 32: f8::launch_kernel<32>(c, tx, tb, a); break;
        case 48: f8::launch_kernel<48>(c, tx, tb, a); break;
        case 64: f8::launch_kernel<64>(c, tx, tb, a); break;
        default: fail(TK_ERR_SHAPE, "ttm_fp8: unsupported width");
    }
    c.counted();
    c.check_launch();
}

}  // namespace tk
