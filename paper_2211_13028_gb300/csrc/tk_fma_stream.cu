// Narrow TTMs that stream FP32 data: out = X x_j M^T with at most 8 output
// columns (the widths of the Kronecker sketch factors).  At that width each
// element needs at most 8 fused multiply-adds (one per column of M: the
// kernel is instantiated for 5..8 computed columns), well inside the FP32 pipe at HBM rate,
// so the data is streamed by TMA into a ring of shared-memory stages (as the
// tensor-core kernels do; the registers of a plain SIMT kernel cannot keep
// enough bytes in flight) and consumed by FP32 FMA warps, with M held in
// shared memory for the whole pass.  FP32 accumulation, as in the tensor-core
// path, whose tf32 instruction count at this width would bound the pass.
//
// Work item: one tile of 128 rows (the same tiling and TMA boxes as the
// tensor-core kernels).  Warp 0 issues the TMA loads; warps 1..8 consume, in
// four groups of 2 that take every fourth chunk (so four chunks are in work at
// once): thread (q, kh) of a group sums K-columns [16 kh, 16 kh + 16) of its
// chunks for the four rows q, q + 32, q + 64, q + 96, so that each row of M
// read from shared memory (a broadcast, four wavefronts per 16-byte load)
// serves four rows of X: the shared-memory pipe, not the FMA pipe, is what a
// narrow pass exhausts first.  The eight partial sums of a row are added
// through shared memory at the end of the item.  Every wait is bounded (the
// abort protocol of the tensor-core kernels); on a timeout the consumers keep
// their control flow (so that the named barriers still match) and skip the
// arithmetic.
#include <cuda.h>
#include <cuda_runtime.h>

#include "tk_internal.cuh"
#include "tk_tc_common.cuh"

namespace tk {
namespace tc {

constexpr int FS_COLS = 8;                       // output columns (zero-padded)
constexpr int FS_GROUP = 2;                      // consumer warps per group (32 row quads x 2 K halves)
constexpr int FS_NGRP = 4;                       // groups, taking chunks in turn
constexpr int FS_PARTS = 2 * FS_NGRP;            // partial sums per row
constexpr int FS_CONS = FS_NGRP * FS_GROUP;      // consumer warps
constexpr int FS_THREADS = 32 * (1 + FS_CONS);
// X bytes in flight per SM are what bounds a streaming pass here (loaded HBM
// latency is several microseconds), so the ring takes the shared memory that
// M and the partial sums leave: 11 stages of 16 KB.
constexpr int FS_STAGES = 11;
constexpr int FS_ROWS = 128;                     // tile rows
constexpr int FS_CHUNK = 32;                     // K columns per stage
constexpr int FS_XBYTES = FS_ROWS * FS_CHUNK * 4;
constexpr int FS_MAX_NJ = 512;                   // M rows held in shared memory

struct FsArgs {
    int64_t L, nj, R, m;
    int64_t ntiles, tiles_per_r, nk;
    const float* M;
    int64_t ldm;
    int mtrans;
    float* out;
    unsigned* flags;
    SignMap sm;  // SIGN instantiations: the Rademacher diagonal applied on load
};

inline size_t fs_smem(int64_t nk) {
    return 1024 + (size_t)FS_STAGES * FS_XBYTES + sizeof(float) * (size_t)nk * FS_CHUNK * FS_COLS +
           sizeof(float) * (FS_PARTS - 1) * FS_ROWS * FS_COLS + sizeof(uint64_t) * (2 * FS_STAGES + 1);
}

// NC: the output columns computed (m <= NC <= FS_COLS; M is held zero-padded to FS_COLS columns).
template <bool KMAJOR, bool SIGN, int NC>
__global__ void __launch_bounds__(FS_THREADS, 1)
    ttm_fma_stream_kernel(const __grid_constant__ CUtensorMap tmX, FsArgs args) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int64_t nk = args.nk;
    float* msm = reinterpret_cast<float*>(smem + FS_STAGES * FS_XBYTES);  // M(i, a), nk * 32 rows x 8
    float* red = msm + nk * FS_CHUNK * FS_COLS;  // [part - 1][row][col]: the partial sums but (group 0, half 0)
    uint64_t* full = reinterpret_cast<uint64_t*>(red + (FS_PARTS - 1) * FS_ROWS * FS_COLS);
    uint64_t* xfree = full + FS_STAGES;
    volatile int* abort = reinterpret_cast<volatile int*>(xfree + FS_STAGES);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int64_t e = tid; e < nk * FS_CHUNK * FS_COLS; e += blockDim.x) {
        const int64_t i = e / FS_COLS, a = e % FS_COLS;
        msm[e] = (i < args.nj && a < args.m) ? (args.mtrans ? args.M[a + args.ldm * i] : args.M[i + args.ldm * a])
                                             : 0.f;
    }
    if (tid == 0) {
        for (int s = 0; s < FS_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&xfree[s], FS_GROUP);
        }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    unsigned* flags = args.flags;
    const int64_t nitems = args.ntiles;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            int64_t it = 0;
            bool ok = true;
            for (int64_t t = blockIdx.x; t < nitems && ok; t += gridDim.x) {
                int64_t r0 = 0, l0 = 0, rr = 0;
                if (KMAJOR) {
                    r0 = t * FS_ROWS;
                } else {
                    rr = t / args.tiles_per_r;
                    l0 = (t % args.tiles_per_r) * FS_ROWS;
                }
                for (int64_t kc = 0; kc < nk; ++kc, ++it) {
                    const int s = (int)(it % FS_STAGES);
                    if (!mbar_wait(&xfree[s], (uint32_t)(((it / FS_STAGES) & 1) ^ 1), abort, flags)) {
                        ok = false;
                        break;
                    }
                    uint8_t* xs = smem + s * FS_XBYTES;
                    mbar_expect_tx(&full[s], FS_XBYTES);
                    if (KMAJOR)
                        tma_load_2d(xs, &tmX, (int)(kc * FS_CHUNK), (int)r0, &full[s]);
                    else
                        tma_load_3d(xs, &tmX, (int)l0, (int)(kc * FS_CHUNK), (int)rr, &full[s]);
                }
            }
            // drain: every issued load has landed before the CTA can exit
            const int64_t n_out = it < FS_STAGES ? it : FS_STAGES;
            for (int64_t q = it - n_out; q < it; ++q) {
                const uint64_t t0 = gtimer();
                while (!mbar_try_wait(&full[q % FS_STAGES], (uint32_t)((q / FS_STAGES) & 1)) &&
                       gtimer() - t0 < kTimeoutNs) {
                }
            }
        }
        return;
    }
    // ------------------------------------------------ FMA consumers
    const int ct = tid - 32, q = ct & 31, kh = (ct >> 5) & 1, grp = ct >> 6;
    const float4* m4 = reinterpret_cast<const float4*>(msm);
    int64_t it = 0;
    for (int64_t t = blockIdx.x; t < nitems; t += gridDim.x) {
        float acc[4][NC];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int a = 0; a < NC; ++a) acc[u][a] = 0.f;
        uint32_t c0[4];  // SIGN: unfolding column of (row, i = 0) for this item's four rows
        if (SIGN) {
            const SignMap& sm = args.sm;
            const int64_t rr = KMAJOR ? 0 : t / args.tiles_per_r;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t row = (KMAJOR ? t : t % args.tiles_per_r) * FS_ROWS + q + 32 * u;
                c0[u] = (uint32_t)(sm.C1 * (row % sm.P1) + sm.P2 * (row / sm.P3) + sm.B1 * (rr % sm.Q1) +
                                   sm.B2 * (rr / sm.Q2));
            }
        }
        for (int64_t kc = 0; kc < nk; ++kc, ++it) {
            if ((int)(it % FS_NGRP) != grp) continue;
            const int s = (int)(it % FS_STAGES);
            const bool got = mbar_wait_warp(&full[s], (uint32_t)((it / FS_STAGES) & 1), abort, flags);
            if (got) {
                const uint8_t* xs = smem + s * FS_XBYTES;
                const float4* mrow = m4 + (kc * FS_CHUNK + 16 * kh) * 2;
#pragma unroll
                for (int k4 = 0; k4 < 4; ++k4) {  // four K columns at a time
                    float v[4][4];                 // [row u][k]
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int rho = q + 32 * u;
                        if (KMAJOR) {
                            // row rho: 128 B, 16-byte chunk j stored at chunk j ^ (rho & 7)
                            const int j = 4 * kh + k4;
                            const float4 f =
                                *reinterpret_cast<const float4*>(xs + rho * 128 + ((j ^ (rho & 7)) << 4));
                            v[u][0] = f.x;
                            v[u][1] = f.y;
                            v[u][2] = f.z;
                            v[u][3] = f.w;
                        } else {
                            // rows i of 128 floats (512 B): lanes read consecutive words
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk)
                                v[u][kk] = reinterpret_cast<const float*>(xs)[(16 * kh + 4 * k4 + kk) * FS_ROWS + rho];
                        }
                        if (SIGN) {
                            const uint32_t i0 = (uint32_t)(kc * FS_CHUNK + 16 * kh + 4 * k4);
                            const uint32_t A = (uint32_t)args.sm.A;
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk)
                                v[u][kk] = __uint_as_float(__float_as_uint(v[u][kk]) ^
                                                           tk_rad_bits(args.sm.key, c0[u] + A * (i0 + kk)));
                        }
                    }
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const float4 ma = mrow[2 * (4 * k4 + kk)];
                        const float4 mb = NC > 4 ? mrow[2 * (4 * k4 + kk) + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
                        const float mv[FS_COLS] = {ma.x, ma.y, ma.z, ma.w, mb.x, mb.y, mb.z, mb.w};
#pragma unroll
                        for (int u = 0; u < 4; ++u)
#pragma unroll
                            for (int a = 0; a < NC; ++a) acc[u][a] = fmaf(v[u][kk], mv[a], acc[u][a]);
                    }
                }
            }
            __syncwarp();  // the warp's reads of the stage are done before lane 0 releases it
            if (lane == 0) mbar_arrive(&xfree[s]);
        }
        // add the partial sums, then store the rows
        const int part = 2 * grp + kh;  // 0: (group 0, half 0) ... FS_PARTS - 1
        if (part != 0) {
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int a = 0; a < NC; ++a) red[((part - 1) * FS_ROWS + q + 32 * u) * FS_COLS + a] = acc[u][a];
        }
        asm volatile("bar.sync 1, %0;" ::"n"(32 * FS_CONS) : "memory");
        if (part == 0 && !*abort) {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int rho = q + 32 * u;
                int64_t base, stride;
                bool valid;
                if (KMAJOR) {
                    const int64_t r = t * FS_ROWS + rho;
                    valid = r < args.R;
                    base = r * args.m;
                    stride = 1;
                } else {
                    const int64_t rr = t / args.tiles_per_r;
                    const int64_t l = (t % args.tiles_per_r) * FS_ROWS + rho;
                    valid = l < args.L;
                    base = l + args.L * args.m * rr;
                    stride = args.L;
                }
                if (valid) {
#pragma unroll
                    for (int a = 0; a < NC; ++a)
                        if (a < args.m) {
                            float v = acc[u][a];
#pragma unroll
                            for (int pp = 1; pp < FS_PARTS; ++pp) v += red[((pp - 1) * FS_ROWS + rho) * FS_COLS + a];
                            args.out[base + a * stride] = v;
                        }
                }
            }
        }
        asm volatile("bar.sync 1, %0;" ::"n"(32 * FS_CONS) : "memory");
    }
}

}  // namespace tc

bool ttm_narrow_eligible(const Tens& X, int j, int64_t m, tk_dtype out_dt) {
    if (X.dt != TK_F32 || out_dt != TK_F32 || m < 1 || m > tc::FS_COLS) return false;
    const int64_t L = X.left(j), nj = X.n[j], R = X.right(j);
    if (nj < 1 || nj > tc::FS_MAX_NJ || L * nj * R < (1 << 22)) return false;  // small tensors: the general kernels
    if (reinterpret_cast<uintptr_t>(X.p) % 16) return false;
    // TMA: global strides are multiples of 16 bytes
    return L == 1 ? nj % 4 == 0 : L % 4 == 0;
}

void launch_ttm_narrow(const Ctx& c, const Tens& X, int j, const Mat& M, bool mtrans, int64_t m, float* out,
                       const SignMap* sm) {
    if (!c.exec) return;
    TK_REQUIRE(M.dt == TK_F32, TK_ERR_DTYPE, "narrow ttm: F32 matrix");
    const int64_t L = X.left(j), nj = X.n[j], R = X.right(j);
    const bool kmajor = (L == 1);
    CUtensorMap tx;
    if (kmajor) {
        uint64_t dims[2] = {(uint64_t)nj, (uint64_t)R};
        uint64_t str[1] = {(uint64_t)nj * 4};
        uint32_t box[2] = {tc::FS_CHUNK, tc::FS_ROWS};
        tc::encode(&tx, X.p, 2, dims, str, box);
    } else {
        uint64_t dims[3] = {(uint64_t)L, (uint64_t)nj, (uint64_t)R};
        uint64_t str[2] = {(uint64_t)L * 4, (uint64_t)L * nj * 4};
        uint32_t box[3] = {tc::FS_ROWS, tc::FS_CHUNK, 1};
        tc::encode(&tx, X.p, 3, dims, str, box, false);
    }
    tc::FsArgs a;
    a.L = L;
    a.nj = nj;
    a.R = R;
    a.m = m;
    a.nk = (nj + tc::FS_CHUNK - 1) / tc::FS_CHUNK;
    a.tiles_per_r = kmajor ? 1 : (L + tc::FS_ROWS - 1) / tc::FS_ROWS;
    a.ntiles = kmajor ? (R + tc::FS_ROWS - 1) / tc::FS_ROWS : R * a.tiles_per_r;
    a.M = static_cast<const float*>(M.p);
    a.ldm = M.ld;
    a.mtrans = mtrans ? 1 : 0;
    a.out = out;
    a.flags = c.dflags;
    if (sm) a.sm = *sm;
    const size_t smem = tc::fs_smem(a.nk);
    const char* name = (const void*)X.p == c.xdata ? "xpass_narrow" : "ttm_narrow";
    ProfScope ps(c, name, 4.0 * (double)L * nj * R + 4.0 * (double)L * m * R + 4.0 * nj * m, 2.0 * L * nj * R * m);
    const int grid = (int)std::min<int64_t>(a.ntiles, tc::grid_sms(c));
    auto run = [&](auto kern) {
        TK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<grid, tc::FS_THREADS, smem, c.stream>>>(tx, a);
    };
    // the FMAs of the output columns the factor has (5..8; the Kronecker-SRHT path always takes 8)
    const int nc = sm ? 8 : (int)std::max<int64_t>(5, m);
    if (sm) {
        kmajor ? run(tc::ttm_fma_stream_kernel<true, true, 8>) : run(tc::ttm_fma_stream_kernel<false, true, 8>);
    } else if (kmajor) {
        nc == 5 ? run(tc::ttm_fma_stream_kernel<true, false, 5>)
                : nc == 6 ? run(tc::ttm_fma_stream_kernel<true, false, 6>)
                          : nc == 7 ? run(tc::ttm_fma_stream_kernel<true, false, 7>)
                                    : run(tc::ttm_fma_stream_kernel<true, false, 8>);
    } else {
        nc == 5 ? run(tc::ttm_fma_stream_kernel<false, false, 5>)
                : nc == 6 ? run(tc::ttm_fma_stream_kernel<false, false, 6>)
                          : nc == 7 ? run(tc::ttm_fma_stream_kernel<false, false, 7>)
                                    : run(tc::ttm_fma_stream_kernel<false, false, 8>);
    }
    c.counted();
    c.check_launch();
}

}  // namespace tk
