// Tensor-core mode-j contraction (TTM) for FP32 data on sm_103a.
//
//   out[l + L*(a + m*r)] = sum_i M(i, a) X[l + L*(i + n_j*r)]     (X viewed as L x n_j x R)
//
// FP32 accuracy from TF32 tensor cores by the split-product ("3xTF32") method:
// x = x_hi + x_lo and M = M_hi + M_lo with every part a TF32 value (round to
// nearest), and x*M ~ x_hi*M_hi + x_hi*M_lo + x_lo*M_hi with FP32 accumulation.
//
// Kernel structure (persistent, one CTA per SM; warp counts in Warps<EPI> below):
//   warp 0      TMA producer: 32-deep K chunks of a 128-row tile of X (16 KB) plus the
//               matching 32 x NPAD chunks of M_hi and M_lo, into an SMEM ring.
//   warp 1      allocates TMEM; lane 0 issues tcgen05.mma.
//   converters  (16 warps for a plain product, 8 with the residual epilogue): each
//               lane reads its row's values of the chunk from SMEM, splits them into
//               TF32 hi / lo and writes them to TMEM with tcgen05.st.  The MMA reads A
//               from TMEM, so X is read from SMEM exactly once, and a contraction over
//               a non-contiguous mode (MN-major X) needs no transpose: only the
//               element each lane reads differs.
//   epilogue    (4 warps, 16 with the residual): tcgen05.ld of a double-buffered
//               accumulator, hi+lo column halves summed, rows written to global memory
//               (or compared with X: EPI 1, 2).
// A plain product along a strided mode with fewer than 64 rows before it packs
// several slabs into each 128-row tile, and one with too few tiles for the SMs
// splits each tile's K chunks over several work items, whose partial products a
// second kernel sums in order (TcArgs::pack, TcArgs::ksplit).
// One MMA per 8-deep K step computes A_hi * [M_hi ; M_lo] (N = 2*NPAD, the two halves
// land in separate TMEM columns); a second adds A_lo * M_hi into the second half, with
// the other small term.  The tensor core's FP32 accumulation rounds each addition
// toward zero, a bias that grows with the number of additions into the large
// A_hi * M_hi sum, so that sum receives one MMA per K step and the corrections the
// other (on the 512^3 benchmark field the core pass's relative error against the
// FP64 oracle went from 1.0e-5 to 7.3e-6).
// Every mbarrier wait is bounded by a wall-clock limit; on expiry the CTA raises
// FLAG_TIMEOUT, stops issuing work, drains what it issued and frees its TMEM.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <type_traits>

#include "tk_tc_common.cuh"

namespace tk {
namespace tc {

// Warp roles: 0 TMA producer, 1 TMEM allocation + MMA issue, 2-3 idle, then
// the converters, then the epilogue.  The plain-store kernels (EPI 0) need many
// converters (X streams through them) and a light epilogue; the residual
// kernels (EPI 1, 2) convert only the small reconstruction operand but compare
// every element of X in the epilogue, so they trade converters for epilogue warps.
template <int EPI>
struct Warps {
    static constexpr int kConv = EPI ? 8 : 16;   // converter warps: (1 or 2 chunk groups) x 2 K halves x 4 lane quarters
    static constexpr int kGroups = kConv / 8;
    static constexpr int kEpi = EPI ? 16 : 4;    // epilogue warps: 4 lane quarters x column groups
    static constexpr int kColGroups = kEpi / 4;
    static constexpr int kFirstConv = 4;
    static constexpr int kFirstEpi = 4 + kConv;
    static constexpr int kThreads = 32 * (4 + kConv + kEpi);
};
constexpr int kRows = 128;    // tile rows (TMEM lanes)
constexpr int kChunk = 32;    // K elements per pipeline stage
constexpr int kXBytes = kRows * kChunk * 4;
// D[tmem] (+)= A[tmem] * B[smem desc], kind::tf32, M = 128.
__device__ __forceinline__ void mma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t idesc,
                                            uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Instruction descriptor: D F32, A/B TF32, both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
}

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

#define TK_R32(a) "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(a[4]), "r"(a[5]), "r"(a[6]), "r"(a[7]), \
    "r"(a[8]), "r"(a[9]), "r"(a[10]), "r"(a[11]), "r"(a[12]), "r"(a[13]), "r"(a[14]), "r"(a[15]),          \
    "r"(a[16]), "r"(a[17]), "r"(a[18]), "r"(a[19]), "r"(a[20]), "r"(a[21]), "r"(a[22]), "r"(a[23]),         \
    "r"(a[24]), "r"(a[25]), "r"(a[26]), "r"(a[27]), "r"(a[28]), "r"(a[29]), "r"(a[30]), "r"(a[31])

__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, %32};" ::"r"(taddr),
        TK_R32(v)
        : "memory");
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

struct TcArgs {
    int64_t L, nj, R, m;
    int64_t ntiles, tiles_per_r, nk, nblk;  // work item = (row tile, block of NPAD output columns)
    // strided mode with L < 64 (EPI 0 only): a tile holds `pack` consecutive r of L rows each
    // (pack L <= 128 rows) instead of one r, so that short rows fill the 128-row tile; 1 otherwise
    int pack;
    uint32_t xbytes;                        // TMA bytes of one X chunk (128 x 32 x 4, or L x 32 x pack x 4)
    // EPI 0 with few row tiles: the K chunks of a tile are split over ksplit work items, each writing
    // its partial product to part + s out_numel (summed in order by a second kernel); 1 otherwise
    int ksplit;
    float* part;
    int64_t out_numel;
    void* out;                              // EPI 0: product (FP32); EPI 2: alpha * (xref - product) (XR)
    const void* xref;                       // EPI 1, 2: tensor compared with the product (same layout, XR)
    float alpha;
    float xr_scale;                         // EPI 1, 2: xref element = stored value * xr_scale (FP8: 1 / scale)
    double* partials;                       // EPI 1, 2: per CTA {sum (xref - product)^2, sum xref^2}
    unsigned* flags;
};

template <int NPAD, int EPI, typename XR = float>
struct Cfg {
    static constexpr int kBBytes = NPAD * 128;  // one of M_hi / M_lo: NPAD rows of 128 B
    static constexpr int kStage = kXBytes + 2 * kBBytes;
    static constexpr int kXrBytes = EPI ? kRows * NPAD * (int)sizeof(XR) : 0;  // X tile compared in the residual epilogue
    // X tiles in flight: about 128 KB, enough to cover HBM latency at one SM's share of
    // the bandwidth (2 to 8 tiles)
    static constexpr int kXrFit = EPI ? (128 * 1024) / (kRows * NPAD * (int)sizeof(XR)) : 0;
    static constexpr int kXrBufs = EPI ? (kXrFit > 8 ? 8 : (kXrFit < 2 ? 2 : kXrFit)) : 0;
    static constexpr int kBudget = 210 * 1024 - kXrBufs * kXrBytes;
    static constexpr int kStages = kBudget / kStage > 12 ? 12 : kBudget / kStage;
    static constexpr int kAccCols = 2 * NPAD;      // accumulators: 2 x (2*NPAD) columns
    static constexpr int kAcc0 = 0;
    static constexpr int kABuf = 2 * kAccCols;     // A buffers: NA x 64 columns (hi 32 | lo 32)
    static constexpr int kNA = (512 - kABuf) / 64 > 6 ? 6 : (512 - kABuf) / 64;  // >= 2
    static constexpr int kSmem = kStages * kStage + kXrBufs * kXrBytes + 1024 + 512;
    static_assert(kNA >= 2, "TMEM budget");
    static_assert(kStages >= 2, "SMEM budget");
};

// (hi, lo) += b with Knuth's two-sum on the high part; the low part collects
// the rounding errors (a double-float running sum of FP32 terms).
__device__ __forceinline__ void ef_add(float& hi, float& lo, float b) {
    const float s = __fadd_rn(hi, b);
    const float v = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, v)), __fsub_rn(b, v));
    hi = s;
    lo = __fadd_rn(lo, e);
}

__device__ __forceinline__ float xr_to_f32(float v) { return v; }
__device__ __forceinline__ float xr_to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float xr_to_f32(__nv_fp8_e4m3 v) { return static_cast<float>(v); }
__device__ __forceinline__ void xr_store(float* p, float v) { *p = v; }
__device__ __forceinline__ void xr_store(__nv_bfloat16* p, float v) { *p = __float2bfloat16_rn(v); }

// EPI 0: store the product; 1: accumulate the residual norms against xref;
// 2: as 1 and also store alpha * (xref - product).  XR: element type of xref
// and of the EPI 2 output (FP32, or BF16 for BF16 data).
template <int NPAD, bool KMAJOR, int EPI, typename XR = float>
__global__ void __launch_bounds__(Warps<EPI>::kThreads, 1)
    ttm_tf32x3_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmBhi,
                      const __grid_constant__ CUtensorMap tmBlo, const __grid_constant__ CUtensorMap tmXr,
                      TcArgs args) {
    using C = Cfg<NPAD, EPI, XR>;
    constexpr int S = C::kStages;
    constexpr int NA = C::kNA;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    float* xr_buf = reinterpret_cast<float*>(smem + S * C::kStage);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + S * C::kStage + C::kXrBufs * C::kXrBytes);
    uint64_t* full = bars;               // [S] TMA landed
    uint64_t* xfree = bars + S;          // [S] stage consumed (one arrival per converter warp + 1 MMA commit)
    uint64_t* afull = bars + 2 * S;      // [NA] A buffer written (one arrival per converter warp)
    uint64_t* aempty = afull + NA;       // [NA] A buffer consumed (MMA commit)
    uint64_t* accfull = aempty + NA;     // [2] accumulator complete (MMA commit)
    uint64_t* accempty = accfull + 2;    // [2] accumulator drained (one arrival per epilogue warp)
    constexpr int XB = C::kXrBufs > 0 ? C::kXrBufs : 1;
    uint64_t* xrfull = accempty + 2;     // [XB] residual X tile landed
    uint64_t* xrempty = xrfull + XB;     // [XB] residual X tile consumed (one arrival per epilogue warp)
    uint64_t* done = xrempty + XB;       // [1] every issued MMA complete
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    using W = Warps<EPI>;
    __shared__ double red[2 * W::kEpi];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&xfree[s], 9);   // 8 converter warps + 1 MMA commit
        }
        for (int b = 0; b < NA; ++b) {
            mbar_init(&afull[b], 8);   // 8 converter warps
            mbar_init(&aempty[b], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accfull[b], 1);
            mbar_init(&accempty[b], W::kEpi);   // one arrival per epilogue warp
        }
        for (int b = 0; b < XB; ++b) {
            mbar_init(&xrfull[b], 1);
            mbar_init(&xrempty[b], W::kEpi);
        }
        mbar_init(done, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tmem_slot;
    unsigned* flags = args.flags;
    const int64_t nk = args.nk;
    const int64_t nitems = args.ntiles * args.nblk * args.ksplit;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            int64_t it = 0, item = 0;
            bool ok = true;
            for (int64_t w = blockIdx.x; w < nitems && ok; w += gridDim.x, ++item) {
                const int64_t w2 = w / args.ksplit, sk = w % args.ksplit;
                const int64_t t = w2 / args.nblk, nb = w2 % args.nblk;
                const int64_t kc0 = nk * sk / args.ksplit, kc1 = nk * (sk + 1) / args.ksplit;
                int64_t r0 = 0, l0 = 0, rr = 0;
                if (KMAJOR) {
                    r0 = t * kRows;
                } else {
                    rr = (t / args.tiles_per_r) * args.pack;
                    l0 = (t % args.tiles_per_r) * kRows;
                }
                if (EPI) {  // the X tile the epilogue compares this item's product with
                    const int xb = (int)(item % XB);
                    if (!mbar_wait(&xrempty[xb], (uint32_t)(((item / XB) & 1) ^ 1), abort, flags)) break;
                    mbar_expect_tx(&xrfull[xb], C::kXrBytes);
                    tma_load_3d(reinterpret_cast<uint8_t*>(xr_buf) + xb * C::kXrBytes, &tmXr, (int)l0, (int)(nb * NPAD),
                                (int)rr, &xrfull[xb]);
                }
                for (int64_t kc = kc0; kc < kc1; ++kc, ++it) {
                    const int s = (int)(it % S);
                    const uint32_t ph = (uint32_t)((it / S) & 1);
                    if (!mbar_wait(&xfree[s], ph ^ 1, abort, flags)) {
                        ok = false;
                        break;
                    }
                    uint8_t* xs = smem + s * C::kStage;
                    uint8_t* bs = xs + kXBytes;
                    mbar_expect_tx(&full[s], args.xbytes + 2 * C::kBBytes);
                    if (KMAJOR) {
                        tma_load_2d(xs, &tmX, (int)(kc * kChunk), (int)r0, &full[s]);
                    } else {
                        // one unswizzled 128 x 32 box: rows i of 128 floats (512 B)
                        tma_load_3d(xs, &tmX, (int)l0, (int)(kc * kChunk), (int)rr, &full[s]);
                    }
                    tma_load_2d(bs, &tmBhi, (int)(kc * kChunk), (int)(nb * NPAD), &full[s]);
                    tma_load_2d(bs + C::kBBytes, &tmBlo, (int)(kc * kChunk), (int)(nb * NPAD), &full[s]);
                }
            }
            // drain: every issued load has landed before the CTA can exit
            const int64_t n_out = it < S ? it : S;
            for (int64_t q = it - n_out; q < it; ++q) {
                const uint64_t t0 = gtimer();
                while (!mbar_try_wait(&full[q % S], (uint32_t)((q / S) & 1)) && gtimer() - t0 < kTimeoutNs) {
                }
            }
            if (EPI) {
                const int64_t n_xr = item < XB ? item : XB;
                for (int64_t q = item - n_xr; q < item; ++q) {
                    const uint64_t t0 = gtimer();
                    while (!mbar_try_wait(&xrfull[q % XB], (uint32_t)((q / XB) & 1)) && gtimer() - t0 < kTimeoutNs) {
                    }
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            int64_t it = 0, ab = 0, acc = 0;
            bool ok = true;
            for (int64_t w = blockIdx.x; w < nitems && ok; w += gridDim.x, ++acc) {
                const int a = (int)(acc & 1);
                if (!mbar_wait(&accempty[a], (uint32_t)(((acc >> 1) & 1) ^ 1), abort, flags)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d_tmem = tbase + C::kAcc0 + a * C::kAccCols;
                const int64_t sk = w % args.ksplit;
                const int64_t kc0 = nk * sk / args.ksplit, kc1 = nk * (sk + 1) / args.ksplit;
                for (int64_t kc = kc0; kc < kc1; ++kc, ++it, ++ab) {
                    const int s = (int)(it % S);
                    const int b = (int)(ab % NA);
                    if (!mbar_wait(&full[s], (uint32_t)((it / S) & 1), abort, flags) ||
                        !mbar_wait(&afull[b], (uint32_t)((ab / NA) & 1), abort, flags)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t bs = smem_u32(smem + s * C::kStage + kXBytes);
                    const uint32_t a_hi = tbase + C::kABuf + 64 * b;
#pragma unroll
                    for (int k8 = 0; k8 < kChunk / 8; ++k8) {
                        const uint64_t bdesc = desc_sw128(bs + 32 * k8);
                        mma_tf32_ts(d_tmem, a_hi + 8 * k8, bdesc, idesc_tf32(2 * NPAD), (kc != kc0 || k8 != 0) ? 1u : 0u);
                        mma_tf32_ts(d_tmem + NPAD, a_hi + 32 + 8 * k8, bdesc, idesc_tf32(NPAD), 1u);
                    }
                    tc_commit(&aempty[b]);
                    tc_commit(&xfree[s]);
                }
                if (!ok) break;
                tc_commit(&accfull[a]);
            }
            tc_commit(done);
            const uint64_t t0 = gtimer();
            while (!mbar_try_wait(done, 0) && gtimer() - t0 < kTimeoutNs) {
            }
        }
    } else if (warp >= W::kFirstConv && warp < W::kFirstEpi) {
        // ------------------------------------------------ converters: X chunk -> TF32 hi / lo in TMEM
        // groups of 8 warps (with 2 groups, group g takes the even / odd chunks, so two chunks
        // are converted at once); within a group two warps per TMEM lane quarter, half hs
        // converting K columns [16 hs, 16 hs + 16).
        const int cw = warp - W::kFirstConv;
        const int q = warp & 3, hs = (cw >> 2) & 1, grp = cw >> 3;
        const int rho = 32 * q + lane;  // tile row == TMEM lane
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        const int Lp = (int)args.L;     // packed tiles only (L < 64)
        const int xoff = args.pack > 1 ? (rho < Lp * args.pack ? (rho / Lp) * kChunk * Lp + rho % Lp : -1) : rho;
        const int istride = args.pack > 1 ? Lp : kRows;
        int64_t it = 0, ab = 0;
        bool ok = true;
        for (int64_t w = blockIdx.x; w < nitems && ok; w += gridDim.x) {
            const int64_t sk = w % args.ksplit;
            const int64_t kc0 = nk * sk / args.ksplit, kc1 = nk * (sk + 1) / args.ksplit;
            for (int64_t kc = kc0; kc < kc1; ++kc, ++it, ++ab) {
                if (W::kGroups == 2 && (it & 1) != grp) continue;
                const int s = (int)(it % S);
                const int b = (int)(ab % NA);
                bool got = mbar_wait(&full[s], (uint32_t)((it / S) & 1), abort, flags) &&
                           mbar_wait(&aempty[b], (uint32_t)(((ab / NA) & 1) ^ 1), abort, flags);
                if (!__all_sync(0xffffffffu, got)) {  // warp-uniform: tcgen05.st below is .aligned
                    ok = false;
                    break;
                }
                const uint8_t* xs = smem + s * C::kStage;
                float v[16];
                if (KMAJOR) {
                    // row rho: 128 B, 16-byte chunk j stored at chunk j ^ (rho & 7)
                    const uint8_t* row = xs + rho * 128;
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        const int j = 4 * hs + jj;
                        const float4 f = *reinterpret_cast<const float4*>(row + ((j ^ (rho & 7)) << 4));
                        v[4 * jj] = f.x;
                        v[4 * jj + 1] = f.y;
                        v[4 * jj + 2] = f.z;
                        v[4 * jj + 3] = f.w;
                    }
                } else {
                    // rows i of 128 floats (512 B, no swizzle): lanes read consecutive words.  Packed
                    // tiles hold [p][i][l] (p < pack, rows of L floats): tile row rho = l + L p; the
                    // rows past L pack are padding (zero)
                    const float* xf = reinterpret_cast<const float*>(xs);
#pragma unroll
                    for (int ii = 0; ii < 16; ++ii) {
                        const int i = 16 * hs + ii;
                        v[ii] = xoff >= 0 ? xf[xoff + i * istride] : 0.f;
                    }
                }
                uint32_t hi[16], lo[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    hi[i] = tf32_rna(v[i]);
                    lo[i] = tf32_rna(v[i] - __uint_as_float(hi[i]));
                }
                const uint32_t ta = tbase + lane_base + C::kABuf + 64 * b + 16 * hs;
                __syncwarp();
                tmem_st16(ta, hi);
                tmem_st16(ta + 32, lo);
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                tc_fence_before();
                __syncwarp();  // the warp's TMEM stores and SMEM reads are ordered before lane 0's arrivals
                if (lane == 0) {
                    mbar_arrive(&afull[b]);
                    mbar_arrive(&xfree[s]);
                }
            }
        }
    } else if (warp >= W::kFirstEpi) {
        // ------------------------------------------------ epilogue
        // warp e drains TMEM lane quarter warp % 4 (the quarter a warp may access) and the
        // 16-column slices cg, cg + kColGroups, ... of the accumulator
        const int q = warp & 3;
        const int cg = (warp - W::kFirstEpi) >> 2;
        const int rho = 32 * q + lane;
        const uint32_t lane_base = (uint32_t)(32 * q) << 16;
        // running sums as double-float pairs (hi + lo, Knuth two-sum): FP32 instructions only, the FP64
        // pipe (1/64 of FP32 here) stays out of the per-item work
        float srh = 0.f, srl = 0.f, sxh = 0.f, sxl = 0.f;
        int64_t acc = 0;
        for (int64_t w = blockIdx.x; w < nitems; w += gridDim.x, ++acc) {
            const int64_t w2 = w / args.ksplit, sk = w % args.ksplit;
            const int64_t t = w2 / args.nblk, nb = w2 % args.nblk;
            float* const outp = args.ksplit > 1 ? args.part + sk * args.out_numel : static_cast<float*>(args.out);
            const int a = (int)(acc & 1);
            const int xb = (int)(acc % XB);
            bool got = mbar_wait(&accfull[a], (uint32_t)((acc >> 1) & 1), abort, flags);
            if (EPI) got = got && mbar_wait(&xrfull[xb], (uint32_t)((acc / XB) & 1), abort, flags);
            if (!__all_sync(0xffffffffu, got)) break;  // warp-uniform: tcgen05.ld below is .aligned
            tc_fence_after();
            int64_t base;
            int64_t stride;
            bool valid;
            if (KMAJOR) {
                const int64_t r = t * kRows + rho;
                valid = r < args.R;
                base = r * args.m;
                stride = 1;
            } else if (args.pack > 1) {  // packed tile: row rho = l + L p holds (l, r = pack t + p)
                const int Lp = (int)args.L;
                const int64_t rr = t * args.pack + rho / Lp;
                const int64_t l = rho % Lp;
                valid = rho < Lp * args.pack && rr < args.R;
                base = l + args.L * args.m * rr;
                stride = args.L;
            } else {
                const int64_t rr = t / args.tiles_per_r;
                const int64_t l = (t % args.tiles_per_r) * kRows + rho;
                valid = l < args.L;
                base = l + args.L * args.m * rr;
                stride = args.L;
            }
            const int64_t col0 = nb * NPAD;
            base += col0 * stride;
            const int64_t ncol = args.m - col0;  // valid columns in this block (may exceed NPAD)
            const uint32_t ta = tbase + lane_base + C::kAcc0 + a * C::kAccCols;
            // [column][row] of the residual X tile
            const XR* xt = reinterpret_cast<const XR*>(reinterpret_cast<const uint8_t*>(xr_buf) + xb * C::kXrBytes);
#pragma unroll
            for (int c0 = 16 * cg; c0 < NPAD; c0 += 16 * W::kColGroups) {
                float h[16], g[16];
                __syncwarp();
                tmem_ld16(ta + c0, h);
                tmem_ld16(ta + NPAD + c0, g);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (valid) {
                    if (EPI == 0) {
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            if (c0 + i < ncol) outp[base + (c0 + i) * stride] = h[i] + g[i];
                    } else {
                        float fr = 0.f, fx = 0.f;
                        const XR* xcol = xt + c0 * kRows + rho;
                        XR* op = EPI == 2 ? static_cast<XR*>(args.out) + base + c0 * stride : nullptr;
                        auto one = [&](int i) {
                            float xv = xr_to_f32(xcol[i * kRows]);
                            if constexpr (std::is_same<XR, __nv_fp8_e4m3>::value) xv *= args.xr_scale;  // 1 / scale
                            const float dv = xv - (h[i] + g[i]);
                            fr = fmaf(dv, dv, fr);
                            fx = fmaf(xv, xv, fx);
                            if constexpr (EPI == 2) xr_store(op + i * stride, args.alpha * dv);
                        };
                        if (c0 + 16 <= ncol) {  // a full slice: no per-column test
#pragma unroll
                            for (int i = 0; i < 16; ++i) one(i);
                        } else {
#pragma unroll
                            for (int i = 0; i < 16; ++i)
                                if (c0 + i < ncol) one(i);
                        }
                        ef_add(srh, srl, fr);
                        ef_add(sxh, sxl, fx);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&accempty[a]);
                if (EPI) mbar_arrive(&xrempty[xb]);
            }
        }
        if (EPI != 0) {
            // reduce over the epilogue threads: warp shuffles, then named barrier 1, then one
            // thread sums the warps in a fixed order
            double sr = (double)srh + (double)srl, sx = (double)sxh + (double)sxl;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                sr += __shfl_xor_sync(0xffffffffu, sr, o);
                sx += __shfl_xor_sync(0xffffffffu, sx, o);
            }
            const int e = warp - W::kFirstEpi;
            if (lane == 0) {
                red[2 * e] = sr;
                red[2 * e + 1] = sx;
            }
            asm volatile("bar.sync 1, %0;" ::"n"(32 * W::kEpi) : "memory");
            if (e == 0 && lane == 0) {
                double a0 = 0.0, a1 = 0.0;
                for (int i = 0; i < W::kEpi; ++i) {
                    a0 += red[2 * i];
                    a1 += red[2 * i + 1];
                }
                args.partials[2 * blockIdx.x] = a0;
                args.partials[2 * blockIdx.x + 1] = a1;
            }
        }
    }
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tbase) : "memory");
    }
}

// ------------------------------------------------------------------ host side

// hi = rn_tf32(M(i, a)), lo = rn_tf32(M(i, a) - hi), stored K-major: (i, a) at i + ldo*a,
// a in [0, npad) with zero padding beyond m.
__global__ void split_tf32_kernel(const void* M, tk_dtype dt, int64_t ldm, int mtrans, int64_t nj, int64_t m,
                                  int64_t npad, int64_t ldo, float* hi, float* lo) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= ldo * npad) return;
    int64_t i = idx % ldo, a = idx / ldo;
    double v = 0.0;
    if (i < nj && a < m) {
        int64_t o = mtrans ? a + ldm * i : i + ldm * a;
        v = dt == TK_F64 ? static_cast<const double*>(M)[o] : (double)static_cast<const float*>(M)[o];
    }
    float h = __uint_as_float(tf32_rna((float)v));
    float l = __uint_as_float(tf32_rna((float)(v - (double)h)));
    hi[idx] = h;
    lo[idx] = l;
}

// Several factors split in one launch (blockIdx.y = factor): the same split
// as split_tf32_kernel for each.
struct SplitJob {
    const void* M;
    int dt, mtrans;
    int64_t ldm, nj, m, rows_b, ldo;
    float* hi;
    float* lo;
};
constexpr int kMaxSplitJobs = 8;
struct SplitBatch {
    SplitJob job[kMaxSplitJobs];
};

__global__ void split_tf32_batch_kernel(SplitBatch sb) {
    const SplitJob& jb = sb.job[blockIdx.y];
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < jb.ldo * jb.rows_b;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx % jb.ldo, a = idx / jb.ldo;
        double v = 0.0;
        if (i < jb.nj && a < jb.m) {
            const int64_t o = jb.mtrans ? a + jb.ldm * i : i + jb.ldm * a;
            v = jb.dt == TK_F64 ? static_cast<const double*>(jb.M)[o] : (double)static_cast<const float*>(jb.M)[o];
        }
        const float h = __uint_as_float(tf32_rna((float)v));
        const float l = __uint_as_float(tf32_rna((float)(v - (double)h)));
        jb.hi[idx] = h;
        jb.lo[idx] = l;
    }
}

// out = the sum of the ksplit partial products part[s n .. s n + n), in order of s.
__global__ void splitk_sum_kernel(const float* __restrict__ part, int ksplit, int64_t n, float* __restrict__ out) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        float v = part[e];
        for (int sk = 1; sk < ksplit; ++sk) v += part[(int64_t)sk * n + e];
        out[e] = v;
    }
}

template <int NPAD, bool KMAJOR, int EPI, typename XR = float>
static void launch_kernel(const Ctx& c, const CUtensorMap& tx, const CUtensorMap& th, const CUtensorMap& tl,
                          const CUtensorMap& txr, const TcArgs& a) {
    using Cf = Cfg<NPAD, EPI, XR>;
    auto kern = ttm_tf32x3_kernel<NPAD, KMAJOR, EPI, XR>;
    static bool attr_set = false;
    if (!attr_set) {
        TK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Cf::kSmem));
        attr_set = true;
    }
    int grid = (int)std::min<int64_t>(a.ntiles * a.nblk * a.ksplit, grid_sms(c));
    kern<<<grid, Warps<EPI>::kThreads, Cf::kSmem, c.stream>>>(tx, th, tl, txr, a);
}

// Self-test of the bounded wait: one warp waits, through the same mbar_wait_warp
// the tcgen05 kernels use, on an mbarrier that nothing ever arrives at, so the
// wait must give up after limit_ns, raise FLAG_TIMEOUT and let the kernel
// return.  waited[0] receives the nanoseconds the wait lasted.
__global__ void __launch_bounds__(32) wait_selftest_kernel(uint64_t limit_ns, unsigned* flags, long long* waited) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort;
    if (threadIdx.x == 0) {
        abort = 0;
        mbar_init(&bar, 1);
    }
    __syncthreads();
    const uint64_t t0 = gtimer();
    const bool ok = mbar_wait_warp(&bar, 0, &abort, flags, limit_ns);
    if (threadIdx.x == 0) waited[0] = ok ? -1 : (long long)(gtimer() - t0);
}

}  // namespace tc

void launch_wait_selftest(const Ctx& c, uint64_t limit_ns, long long* waited) {
    if (!c.exec) return;
    tc::wait_selftest_kernel<<<1, 32, 0, c.stream>>>(limit_ns, c.dflags, waited);
    c.counted();
    c.check_launch();
}

// Output columns: up to 96 (64 for the residual epilogue, whose X tiles share
// shared memory with the pipeline) in one block padded to 16, else blocks of 64.
static void tc_blocks(int64_t m, int64_t& npad, int64_t& nblk, bool residual = false) {
    if (m <= (residual ? 64 : 96)) {
        npad = (m + 15) / 16 * 16;
        nblk = 1;
    } else {
        npad = 64;
        nblk = (m + 63) / 64;
    }
}

// The factor splits that tensor-core TTMs about to run will need, made in one
// launch and entered in the call's split cache (c.split_cache must be on while
// those TTMs run).  Factors already split are skipped.
void tc_presplit(Ctx& c, const std::vector<TcSplitReq>& reqs) {
    tc::SplitBatch sb;
    int nj_ = 0;
    int64_t most = 0;
    for (const TcSplitReq& q : reqs) {
        int64_t npad, nblk;
        tc_blocks(q.m, npad, nblk, q.residual);
        const int64_t ldo = (q.nj + 3) / 4 * 4, rows_b = npad * nblk;
        bool have = false;
        for (const Ctx::Split& e : c.splits)
            have = have || (e.p == q.M.p && e.dt == (int)q.M.dt && e.ld == q.M.ld && e.mtrans == (q.mtrans ? 1 : 0) &&
                            e.nj == q.nj && e.m == q.m && e.npad == npad && e.rows == rows_b);
        if (have || nj_ == tc::kMaxSplitJobs) continue;
        float* hi = c.alloc<float>(ldo * rows_b);
        float* lo = c.alloc<float>(ldo * rows_b);
        c.splits.push_back({q.M.p, q.M.ld, q.nj, q.m, npad, rows_b, (int)q.M.dt, q.mtrans ? 1 : 0, hi, lo});
        sb.job[nj_++] = {q.M.p, (int)q.M.dt, q.mtrans ? 1 : 0, q.M.ld, q.nj, q.m, rows_b, ldo, hi, lo};
        most = std::max(most, ldo * rows_b);
    }
    if (!c.exec || nj_ == 0) return;
    ProfScope ps(c, "elementwise", 16.0 * most * nj_, 0.0);
    tc::split_tf32_batch_kernel<<<dim3((unsigned)std::min<int64_t>((most + 255) / 256, 1024), (unsigned)nj_), 256, 0,
                                  c.stream>>>(sb);
    c.counted();
    c.check_launch();
}

bool ttm_tc_eligible(const Tens& X, int j, int64_t m, tk_dtype out_dt) {
    if (X.dt != TK_F32 || out_dt != TK_F32) return false;
    if (m < 1 || m > 65535) return false;
    const int64_t L = X.left(j), nj = X.n[j], R = X.right(j);
    if (nj < 32 || ((uintptr_t)X.p % 16) != 0) return false;
    if (L == 1) return nj % 4 == 0 && R >= tc::kRows && R < ((int64_t)1 << 31);
    return L % 4 == 0 && L >= 32 && L < ((int64_t)1 << 31) && R < ((int64_t)1 << 31) && nj < ((int64_t)1 << 31);
}

// Shared launcher.  epi 0: out = X x_j M^T.  epi 1/2: compare the product with
// xref (same dims as the product): partial norms per CTA into partials, and
// for epi 2 out = alpha * (xref - product).
static void ttm_tc_run(Ctx& c, const Tens& X, int j, const Mat& M, bool mtrans, int64_t m, void* out, int epi,
                       const void* xref, tk_dtype xrdt, float alpha, double* partials, const char* prof_name,
                       float xr_scale = 1.f) {
    const int64_t L = X.left(j), nj = X.n[j], R = X.right(j);
    int64_t npad, nblk;
    tc_blocks(m, npad, nblk, epi != 0);
    const int64_t ldo = (nj + 3) / 4 * 4;
    const int64_t rows_b = npad * nblk;
    float* hi = nullptr;
    float* lo = nullptr;
    bool have = false;
    if (c.split_cache) {
        for (const Ctx::Split& e : c.splits)
            if (e.p == M.p && e.dt == (int)M.dt && e.ld == M.ld && e.mtrans == (mtrans ? 1 : 0) && e.nj == nj &&
                e.m == m && e.npad == npad && e.rows == rows_b) {
                hi = e.hi;
                lo = e.lo;
                have = true;
                break;
            }
    }
    if (!have) {
        hi = c.alloc<float>(ldo * rows_b);
        lo = c.alloc<float>(ldo * rows_b);
        if (c.split_cache)
            c.splits.push_back({M.p, M.ld, nj, m, npad, rows_b, (int)M.dt, mtrans ? 1 : 0, hi, lo});
    }
    // the work items: 128-row tiles (a strided mode with under 64 rows before it packs several slabs
    // per tile) x blocks of NPAD output columns; a plain product with too few of them for half the
    // SMs splits each tile's K chunks over several items (at least two chunks each), whose partial
    // products are summed in order afterwards
    const bool kmajor = (L == 1);
    const int pack = (!kmajor && epi == 0 && L < tc::kRows / 2) ? (int)(tc::kRows / L) : 1;
    const int64_t nk = (nj + tc::kChunk - 1) / tc::kChunk;
    const int64_t tiles_per_r = kmajor ? 1 : (L + tc::kRows - 1) / tc::kRows;
    const int64_t ntiles = kmajor ? (R + tc::kRows - 1) / tc::kRows
                                  : (pack > 1 ? (R + pack - 1) / pack : R * tiles_per_r);
    int ksplit = 1;
    {
        const int64_t items = ntiles * nblk, sms = tc::grid_sms(c);
        if (epi == 0 && items * 2 <= sms && nk >= 4)
            ksplit = (int)std::max<int64_t>(1, std::min<int64_t>(nk / 2, sms / items));
    }
    float* part = ksplit > 1 ? c.alloc<float>(ksplit * L * m * R) : nullptr;
    if (!c.exec) return;
    if (!have) {
        int64_t tot = ldo * rows_b;
        ProfScope ps(c, "elementwise", 8.0 * tot + 8.0 * nj * m, 0.0);
        tc::split_tf32_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, c.stream>>>(M.p, M.dt, M.ld, mtrans ? 1 : 0,
                                                                                   nj, m, rows_b, ldo, hi, lo);
        c.counted();
        c.check_launch();
    }
    CUtensorMap tx, th, tl;
    if (kmajor) {
        uint64_t dims[2] = {(uint64_t)nj, (uint64_t)R};
        uint64_t str[1] = {(uint64_t)nj * 4};
        uint32_t box[2] = {tc::kChunk, tc::kRows};
        tc::encode(&tx, X.p, 2, dims, str, box);
    } else {
        uint64_t dims[3] = {(uint64_t)L, (uint64_t)nj, (uint64_t)R};
        uint64_t str[2] = {(uint64_t)L * 4, (uint64_t)L * nj * 4};
        uint32_t box[3] = {tc::kRows, tc::kChunk, 1};
        if (pack > 1) {  // L rows of pack consecutive r per box (L x 4 bytes: a multiple of 16)
            box[0] = (uint32_t)L;
            box[2] = (uint32_t)pack;
        }
        tc::encode(&tx, X.p, 3, dims, str, box, false);
    }
    {
        uint64_t dims[2] = {(uint64_t)nj, (uint64_t)rows_b};
        uint64_t str[1] = {(uint64_t)ldo * 4};
        uint32_t box[2] = {tc::kChunk, (uint32_t)npad};
        tc::encode(&th, hi, 2, dims, str, box);
        tc::encode(&tl, lo, 2, dims, str, box);
    }
    CUtensorMap txr = tx;  // unused when epi == 0
    const bool xr_bf16 = epi != 0 && xrdt == TK_BF16;
    const bool xr_fp8 = epi != 0 && xrdt == TK_FP8_E4M3;
    if (epi != 0) {
        TK_REQUIRE(!kmajor, TK_ERR_SHAPE, "ttm_tc: the fused residual needs a non-leading mode");
        TK_REQUIRE(xrdt == TK_F32 || xrdt == TK_BF16 || (xrdt == TK_FP8_E4M3 && epi == 1), TK_ERR_DTYPE,
                   "ttm_tc: residual reference must be F32/BF16 (FP8: norms only)");
        const uint64_t es = xr_fp8 ? 1 : (xr_bf16 ? 2 : 4);
        uint64_t dims[3] = {(uint64_t)L, (uint64_t)m, (uint64_t)R};
        uint64_t str[2] = {(uint64_t)L * es, (uint64_t)L * m * es};
        uint32_t box[3] = {tc::kRows, (uint32_t)npad, 1};
        tc::encode(&txr, xref, 3, dims, str, box, false,
                   xr_fp8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8
                          : (xr_bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32));
    }
    tc::TcArgs a;
    a.L = L;
    a.nj = nj;
    a.R = R;
    a.m = m;
    a.nk = nk;
    a.nblk = nblk;
    a.tiles_per_r = tiles_per_r;
    a.ntiles = ntiles;
    a.pack = pack;
    a.xbytes = (uint32_t)(pack > 1 ? L * tc::kChunk * pack * 4 : tc::kXBytes);
    a.ksplit = ksplit;
    a.part = part;
    a.out_numel = L * m * R;
    a.out = out;
    a.xref = xref;
    a.alpha = alpha;
    a.xr_scale = xr_scale;
    a.partials = partials;
    a.flags = c.dflags;
    const double xres = xr_fp8 ? 1.0 : (xr_bf16 ? 2.0 : 4.0);
    double bytes = 4.0 * (double)L * R * nj + 8.0 * nj * m;
    if (epi == 0) bytes += 4.0 * (double)L * R * m;
    if (epi >= 1) bytes += xres * (double)L * R * m;
    if (epi == 2) bytes += xres * (double)L * R * m;
    ProfScope ps(c, prof_name, bytes, 2.0 * (double)L * R * nj * m);
#define TK_TC_CASE(NP)                                                                             \
    case NP:                                                                                       \
        if (epi == 0) {                                                                            \
            if (kmajor) tc::launch_kernel<NP, true, 0>(c, tx, th, tl, txr, a);                          \
            else tc::launch_kernel<NP, false, 0>(c, tx, th, tl, txr, a);                                \
        } else if (xr_fp8) {                                                                       \
            tc::launch_kernel<NP, false, 1, __nv_fp8_e4m3>(c, tx, th, tl, txr, a);                      \
        } else if (xr_bf16) {                                                                      \
            if (epi == 1) tc::launch_kernel<NP, false, 1, __nv_bfloat16>(c, tx, th, tl, txr, a);         \
            else tc::launch_kernel<NP, false, 2, __nv_bfloat16>(c, tx, th, tl, txr, a);                  \
        } else if (epi == 1) {                                                                     \
            tc::launch_kernel<NP, false, 1>(c, tx, th, tl, txr, a);                                     \
        } else {                                                                                   \
            tc::launch_kernel<NP, false, 2>(c, tx, th, tl, txr, a);                                     \
        }                                                                                          \
        break;
    switch (npad) {
        TK_TC_CASE(16)
        TK_TC_CASE(32)
        TK_TC_CASE(48)
        TK_TC_CASE(64)
        TK_TC_CASE(80)
        TK_TC_CASE(96)
        default: fail(TK_ERR_SHAPE, "ttm_tc: unsupported width");
    }
#undef TK_TC_CASE
    c.counted();
    c.check_launch();
    if (ksplit > 1) {
        const int64_t n = L * m * R;
        tc::splitk_sum_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, c.stream>>>(
            part, ksplit, n, static_cast<float*>(out));
        c.counted();
        c.check_launch();
    }
}

void launch_ttm_tc(Ctx& c, const Tens& X, int j, const Mat& M, bool mtrans, int64_t m, float* out) {
    const int64_t L = X.left(j), R = X.right(j);
    // kernel classes: "xpass_tc" streams all of X (a pass over the input),
    // "ttm_tc" contracts an intermediate
    const char* name = ((const void*)X.p == c.xdata || L * R * m == c.xnumel) ? (c.background ? "xpass_tc_bg" : "xpass_tc")
                                                                              : "ttm_tc";
    ttm_tc_run(c, X, j, M, mtrans, m, out, 0, nullptr, TK_F32, 0.f, nullptr, name);
}

int tc_num_ctas(const Ctx& c, const Tens& X, int j, int64_t m, bool residual) {
    int64_t npad, nblk;
    tc_blocks(m, npad, nblk, residual);
    const int64_t L = X.left(j), R = X.right(j);
    const int64_t tiles = (L == 1) ? (R + tc::kRows - 1) / tc::kRows : R * ((L + tc::kRows - 1) / tc::kRows);
    return (int)std::min<int64_t>(tiles * nblk, tc::grid_sms(c));
}

bool ttm_tc_residual_eligible(const Tens& W, int j, int64_t m) {
    int64_t npad, nblk;
    tc_blocks(m, npad, nblk, true);
    // the residual X tile is a (128 rows x npad columns) TMA box: keep it inside the tensor
    return W.left(j) >= tc::kRows && m >= npad && ttm_tc_eligible(W, j, m, TK_F32);
}

void launch_ttm_tc_residual(Ctx& c, const Tens& W, int j, const Mat& M, bool mtrans, int64_t m, const void* xref,
                            tk_dtype xrdt, void* dx, float alpha, double* partials, float xr_scale) {
    ttm_tc_run(c, W, j, M, mtrans, m, dx, dx ? 2 : 1, xref, xrdt, alpha, partials,
               c.background ? "xpass_tc_bg" : "xpass_tc", xr_scale);
}

}  // namespace tk
