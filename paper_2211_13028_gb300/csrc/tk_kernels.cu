// SIMT kernels of libtucker: generic mode-j TTM, FP64 small dense linear
// algebra (Gram / GEMM, Cholesky + triangular inverse, Householder QR, Jacobi
// eigensolver) and element-wise helpers.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <math.h>

#include <type_traits>

#include "tk_internal.cuh"

namespace tk {

void Ctx::check_launch() const {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) fail(TK_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
}

// Only the streams that receive work wait on the fork (a stream that joined a
// graph recording must be joined back before the recording ends).
void ctx_fork_begin(Ctx& c, int used) {
    TK_CUDA(cudaEventRecord(c.ev_fork, c.stream));
    for (int i = 0; i < used; ++i) TK_CUDA(cudaStreamWaitEvent(c.aux[i], c.ev_fork, 0));
}

// Joins the first `used` auxiliary streams back into `main` and makes it the
// call's stream again (also on the error path, hence no throw before that).
void ctx_fork_end(Ctx& c, cudaStream_t main, int used) {
    c.stream = main;
    cudaError_t first = cudaSuccess;
    for (int i = 0; i < used; ++i) {
        cudaError_t e = cudaEventRecord(c.ev_join[i], c.aux[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(main, c.ev_join[i], 0);
        if (first == cudaSuccess) first = e;
    }
    if (first != cudaSuccess) fail(TK_ERR_CUDA, std::string("fork join: ") + cudaGetErrorString(first));
}

// The side stream (the last auxiliary stream) waits for the call's stream and
// becomes the call's stream; ctx_side_end joins it back into `main`.
void ctx_side_begin(Ctx& c) {
    TK_CUDA(cudaEventRecord(c.ev_fork, c.stream));
    TK_CUDA(cudaStreamWaitEvent(c.aux[Ctx::kFork], c.ev_fork, 0));
    c.stream = c.aux[Ctx::kFork];
}

void ctx_side_end(Ctx& c, cudaStream_t main) {
    c.stream = main;
    cudaError_t e = cudaEventRecord(c.ev_join[Ctx::kFork], c.aux[Ctx::kFork]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(main, c.ev_join[Ctx::kFork], 0);
    if (e != cudaSuccess) fail(TK_ERR_CUDA, std::string("side join: ") + cudaGetErrorString(e));
}

// ------------------------------------------------------------------ loads

__device__ __forceinline__ float ldx(const float* p, int64_t i, float) { return p[i]; }
__device__ __forceinline__ float ldx(const __nv_bfloat16* p, int64_t i, float) { return __bfloat162float(p[i]); }
__device__ __forceinline__ float ldx(const __nv_fp8_e4m3* p, int64_t i, float inv) {
    return static_cast<float>(p[i]) * inv;
}
__device__ __forceinline__ double ldx(const double* p, int64_t i, double) { return p[i]; }

__device__ __forceinline__ double ld_any(const void* p, tk_dtype dt, int64_t i, float scale_inv = 1.f) {
    switch (dt) {
        case TK_F64: return static_cast<const double*>(p)[i];
        case TK_F32: return static_cast<const float*>(p)[i];
        case TK_BF16: return __bfloat162float(static_cast<const __nv_bfloat16*>(p)[i]);
        default: return static_cast<float>(static_cast<const __nv_fp8_e4m3*>(p)[i]) * scale_inv;
    }
}
__device__ __forceinline__ void st_any(void* p, tk_dtype dt, int64_t i, double v) {
    switch (dt) {
        case TK_F64: static_cast<double*>(p)[i] = v; break;
        case TK_F32: static_cast<float*>(p)[i] = (float)v; break;
        case TK_BF16: static_cast<__nv_bfloat16*>(p)[i] = __float2bfloat16((float)v); break;
        default: static_cast<__nv_fp8_e4m3*>(p)[i] = __nv_fp8_e4m3((float)v); break;
    }
}

__device__ __forceinline__ int64_t v2off(const View2& v, int64_t a, int64_t t) {
    int64_t o = (v.A1 == INT64_MAX) ? a * v.sa1 : (a % v.A1) * v.sa1 + (a / v.A1) * v.sa2;
    o += (v.T1 == INT64_MAX) ? t * v.st1 : (t % v.T1) * v.st1 + (t / v.T1) * v.st2;
    return o;
}
__device__ __forceinline__ double v2ld(const View2& v, int64_t a, int64_t t) {
    int64_t o = v2off(v, a, t);
    return v.dt == TK_F64 ? static_cast<const double*>(v.p)[o] : (double)static_cast<const float*>(v.p)[o];
}

// Sequential walk along t of one row a of a View2 (t = 0, 1, ...).
struct V2Walk {
    const View2& v;
    int64_t base, lo, hi;
    __device__ V2Walk(const View2& vv, int64_t a) : v(vv), lo(0), hi(0) {
        base = (v.A1 == INT64_MAX) ? a * v.sa1 : (a % v.A1) * v.sa1 + (a / v.A1) * v.sa2;
    }
    __device__ __forceinline__ double load() const {
        int64_t o = base + lo * v.st1 + hi * v.st2;
        return v.dt == TK_F64 ? static_cast<const double*>(v.p)[o] : (double)static_cast<const float*>(v.p)[o];
    }
    __device__ __forceinline__ void next() {
        if (++lo == v.T1) {
            lo = 0;
            ++hi;
        }
    }
};

// ------------------------------------------------------------------ TTM
// out[l + L*(a + m*r)] = sum_i M(i, a) X[l + L*(i + nj*r)],  rows rho = l + L*r.
// 64 x 32 output tile per 256-thread block, K step 16, 4 x 2 outputs per thread.
// KFAST (L == 1): the contraction index is contiguous, so tile loads run along i.

template <typename Tx, typename Ta, bool KFAST>
__global__ void __launch_bounds__(256) ttm_simt_kernel(const Tx* __restrict__ X, int64_t L, int64_t nj, int64_t R,
                                                       const Ta* __restrict__ M, int64_t ldm, int mtrans, int64_t m,
                                                       Ta* __restrict__ out, Ta xinv) {
    constexpr int BM = 64, BN = 32, BK = 16;
    __shared__ Ta Xs[BK][BM + 1];
    __shared__ Ta Ms[BK][BN + 1];
    const int tid = threadIdx.x;
    const int tm = tid % 16, tn = tid / 16;
    const int64_t rows = L * R;
    const int64_t row0 = (int64_t)blockIdx.x * BM;
    const int64_t a0 = (int64_t)blockIdx.y * BN;

    int64_t xbase[4];
    int xk[4], xr[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int e = tid + 256 * q;
        int rr, kk;
        if (KFAST) { kk = e % BK; rr = e / BK; } else { rr = e % BM; kk = e / BM; }
        xk[q] = kk; xr[q] = rr;
        int64_t row = row0 + rr;
        if (row < rows) {
            int64_t l = row % L, r = row / L;
            xbase[q] = l + L * nj * r;
        } else {
            xbase[q] = -1;
        }
    }
    Ta acc[4][2];
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q][0] = acc[q][1] = Ta(0);

    for (int64_t k0 = 0; k0 < nj; k0 += BK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int64_t k = k0 + xk[q];
            Ta v = Ta(0);
            if (xbase[q] >= 0 && k < nj) v = ldx(X, xbase[q] + L * k, xinv);
            Xs[xk[q]][xr[q]] = v;
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            int e = tid + 256 * q;
            int kk = e % BK, aa = e / BK;
            int64_t k = k0 + kk, a = a0 + aa;
            Ta v = Ta(0);
            if (k < nj && a < m) v = mtrans ? M[a + ldm * k] : M[k + ldm * a];
            Ms[kk][aa] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            Ta xv[4], mv[2];
#pragma unroll
            for (int q = 0; q < 4; ++q) xv[q] = Xs[kk][tm + 16 * q];
#pragma unroll
            for (int q = 0; q < 2; ++q) mv[q] = Ms[kk][tn + 16 * q];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int w = 0; w < 2; ++w) acc[q][w] += xv[q] * mv[w];
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int64_t row = row0 + tm + 16 * q;
        if (row >= rows) continue;
        int64_t l = row % L, r = row / L;
#pragma unroll
        for (int w = 0; w < 2; ++w) {
            int64_t a = a0 + tn + 16 * w;
            if (a < m) out[l + L * (a + m * r)] = acc[q][w];
        }
    }
}

// Small TTMs: one thread per output element (consecutive threads along l).
template <typename Tx, typename Ta>
__global__ void __launch_bounds__(256) ttm_direct_kernel(const Tx* __restrict__ X, int64_t L, int64_t nj, int64_t R,
                                                         const Ta* __restrict__ M, int64_t ldm, int mtrans, int64_t m,
                                                         Ta* __restrict__ out, Ta xinv) {
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= L * m * R) return;
    const int64_t l = o % L, rest = o / L;
    const int64_t a = rest % m, r = rest / m;
    const Tx* x = X + l + L * nj * r;
    Ta s = Ta(0);
    for (int64_t i = 0; i < nj; ++i) s += (mtrans ? M[a + ldm * i] : M[i + ldm * a]) * ldx(x, L * i, xinv);
    out[o] = s;
}

// Few outputs per slab, long contraction (L m <= 256, e.g. the second product
// of a sketch, 6 x 512 x 512 -> 6 x 7 x 512, or a core TTM along its first
// mode): a CTA per r stages the slab X[:, :, r] in shared memory with
// coalesced loads and splits each of the L m dot products over S threads,
// summed in shared memory.  A thread per output would walk X with stride L
// and leave most SMs idle.
constexpr int SLAB_THREADS = 256;

template <typename Tx, typename Ta>
__global__ void __launch_bounds__(SLAB_THREADS) ttm_slab_kernel(const Tx* __restrict__ X, int64_t L, int64_t nj,
                                                                int64_t R, const Ta* __restrict__ M, int64_t ldm,
                                                                int mtrans, int64_t m, int S, Ta* __restrict__ out,
                                                                Ta xinv) {
    extern __shared__ __align__(16) unsigned char slab_raw[];
    Ta* xs = reinterpret_cast<Ta*>(slab_raw);  // L x nj, X[l, i] at xs[l + L i]
    Ta* part = xs + L * nj;                    // S x (L m) partial sums
    const int64_t r = blockIdx.x;
    const Tx* x = X + L * nj * r;
    for (int64_t e = threadIdx.x; e < L * nj; e += blockDim.x) xs[e] = ldx(x, e, xinv);
    __syncthreads();
    const int64_t T = L * m;
    const int64_t task = threadIdx.x % T, sp = threadIdx.x / T;
    if (sp < S) {
        const int64_t l = task % L, a = task / L;
        const int64_t i0 = nj * sp / S, i1 = nj * (sp + 1) / S;
        Ta acc = Ta(0);
        for (int64_t i = i0; i < i1; ++i) acc += (mtrans ? M[a + ldm * i] : M[i + ldm * a]) * xs[l + L * i];
        part[sp * T + task] = acc;
    }
    __syncthreads();
    for (int64_t t = threadIdx.x; t < T; t += blockDim.x) {
        Ta v = Ta(0);
        for (int q = 0; q < S; ++q) v += part[q * T + t];
        const int64_t l = t % L, a = t / L;
        out[l + L * (a + m * r)] = v;
    }
}

// FP64 TTM of FP32-class data in double-float arithmetic (defined with the
// double-float helpers below); returns false where it does not apply.
static bool ttm_direct_df(const Ctx& c, const double* X, int64_t L, int64_t nj, int64_t R, const double* M,
                          int64_t ldm, bool mtrans, int64_t m, double* out);

template <typename Tx, typename Ta>
static void ttm_dispatch(const Ctx& c, const Tx* X, int64_t L, int64_t nj, int64_t R, const Ta* M, int64_t ldm,
                         bool mtrans, int64_t m, Ta* out, Ta xinv) {
    int64_t rows = L * R;
    if constexpr (std::is_same<Tx, double>::value && std::is_same<Ta, double>::value) {
        if (c.df64 && ttm_direct_df(c, X, L, nj, R, M, ldm, mtrans, m, out)) return;
    }
    // (a slab of fewer than 256 elements leaves each CTA too little work: one thread per output then)
    if (L * m <= SLAB_THREADS && nj >= 32 && L * nj >= 256 &&
        (double)sizeof(Ta) * (L * nj + SLAB_THREADS) <= 40 * 1024 && R <= 0x7fffffff) {
        const int S = (int)std::min<int64_t>(16, SLAB_THREADS / (L * m));
        const size_t smem = sizeof(Ta) * (size_t)(L * nj + (int64_t)S * L * m);
        const char* name = (const void*)X == c.xdata ? "xpass_simt" : "ttm_simt";
        ProfScope ps(c, name, (double)rows * nj * sizeof(Tx) + (double)rows * m * sizeof(Ta), 2.0 * rows * nj * m);
        ttm_slab_kernel<Tx, Ta><<<(unsigned)R, SLAB_THREADS, smem, c.stream>>>(X, L, nj, R, M, ldm, mtrans ? 1 : 0, m,
                                                                               S, out, xinv);
        c.counted();
        c.check_launch();
        return;
    }
    if (rows * m <= (1 << 21) && nj <= 512) {
        const char* name = (const void*)X == c.xdata ? "xpass_simt" : "ttm_simt";
        ProfScope ps(c, name, (double)rows * nj * sizeof(Tx) + (double)rows * m * sizeof(Ta), 2.0 * rows * nj * m);
        ttm_direct_kernel<Tx, Ta><<<(unsigned)((rows * m + 255) / 256), 256, 0, c.stream>>>(X, L, nj, R, M, ldm,
                                                                                           mtrans, m, out, xinv);
        c.counted();
        c.check_launch();
        return;
    }
    const char* name = ((const void*)X == c.xdata || rows * m == c.xnumel) ? "xpass_simt" : "ttm_simt";
    ProfScope ps(c, name, (double)rows * nj * sizeof(Tx) + (double)rows * m * sizeof(Ta) + (double)nj * m * sizeof(Ta),
                 2.0 * rows * nj * m);
    dim3 grid((unsigned)((rows + 63) / 64), (unsigned)((m + 31) / 32));
    TK_REQUIRE(grid.y <= 65535, TK_ERR_SHAPE, "ttm: too many output columns");
    if (L == 1)
        ttm_simt_kernel<Tx, Ta, true><<<grid, 256, 0, c.stream>>>(X, L, nj, R, M, ldm, mtrans, m, out, xinv);
    else
        ttm_simt_kernel<Tx, Ta, false><<<grid, 256, 0, c.stream>>>(X, L, nj, R, M, ldm, mtrans, m, out, xinv);
    c.counted();
    c.check_launch();
}

void launch_ttm(const Ctx& c, const Tens& X, int j, const Mat& M, bool mtrans, int64_t m, void* out,
                tk_dtype out_dt) {
    if (!c.exec) return;
    int64_t L = X.left(j), nj = X.n[j], R = X.right(j);
    if (L * R == 0 || m == 0) return;
    if (X.dt == TK_F64) {
        TK_REQUIRE(M.dt == TK_F64 && out_dt == TK_F64, TK_ERR_DTYPE, "ttm: F64 data needs F64 matrix and output");
        ttm_dispatch<double, double>(c, (const double*)X.p, L, nj, R, (const double*)M.p, M.ld, mtrans, m,
                                     (double*)out, 1.0);
        return;
    }
    TK_REQUIRE(M.dt == TK_F32 && out_dt == TK_F32, TK_ERR_DTYPE, "ttm: narrow data needs F32 matrix and output");
    float inv = X.dt == TK_FP8_E4M3 ? 1.f / X.scale : 1.f;
    switch (X.dt) {
        case TK_F32:
            ttm_dispatch<float, float>(c, (const float*)X.p, L, nj, R, (const float*)M.p, M.ld, mtrans, m,
                                       (float*)out, inv);
            break;
        case TK_BF16:
            ttm_dispatch<__nv_bfloat16, float>(c, (const __nv_bfloat16*)X.p, L, nj, R, (const float*)M.p, M.ld,
                                               mtrans, m, (float*)out, inv);
            break;
        case TK_FP8_E4M3:
            ttm_dispatch<__nv_fp8_e4m3, float>(c, (const __nv_fp8_e4m3*)X.p, L, nj, R, (const float*)M.p, M.ld,
                                               mtrans, m, (float*)out, inv);
            break;
        default: fail(TK_ERR_DTYPE, "ttm: unsupported data dtype");
    }
}

// ------------------------------------------------------------------ Kronecker-SRHT signs

SignMap sign_map(const Tens& X, int n, int j0, uint64_t seed) {
    SignMap sm;
    sm.key = tk_rad_key(seed, n);
    const int64_t stride = X.left(n), nn = X.n[n], L = X.left(j0), nj0 = X.n[j0];
    const int64_t big = INT64_MAX;
    if (L == 1) {  // rows r of the unfolding along j0, i contiguous: lin = i + nj0 r
        if (n > j0) {
            const int64_t Sa = stride / nj0;
            sm.C1 = nj0; sm.P1 = Sa; sm.P2 = stride; sm.P3 = Sa * nn; sm.A = 1;
        } else {  // every mode before j0 has size 1: mode n is trivial
            sm.C1 = nj0; sm.P1 = big; sm.P2 = 0; sm.P3 = 1; sm.A = 1;
        }
    } else if (n < j0) {  // lin = l + L i + L nj0 rr, mode n inside l
        sm.C1 = 1; sm.P1 = stride; sm.P2 = stride; sm.P3 = stride * nn;
        sm.A = L / nn; sm.B1 = (L / nn) * nj0; sm.Q1 = big; sm.B2 = 0; sm.Q2 = 1;
    } else {  // mode n inside rr
        const int64_t Sb = stride / (L * nj0);
        sm.C1 = 1; sm.P1 = big; sm.P2 = 0; sm.P3 = 1;
        sm.A = L; sm.B1 = L * nj0; sm.Q1 = Sb; sm.B2 = stride; sm.Q2 = Sb * nn;
    }
    return sm;
}

// dst[lin] = d_n(c) X[lin], c = lin mod stride_n + stride_n floor(lin / (stride_n n_n)):
// the sign bit of the stored value is flipped, which is exact for every dtype.
template <typename W>
__global__ void sign_copy_kernel(const W* __restrict__ X, W* __restrict__ dst, int64_t numel, int64_t stride, int64_t nn,
                                 uint32_t key, W top) {
    for (int64_t lin = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; lin < numel;
         lin += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = (uint32_t)(lin % stride + stride * (lin / (stride * nn)));
        dst[lin] = tk_rad_bits(key, c) ? (W)(X[lin] ^ top) : X[lin];
    }
}

void launch_sign_copy(const Ctx& c, const Tens& X, int n, uint64_t seed, void* dst) {
    if (!c.exec) return;
    const int64_t numel = X.numel();
    if (numel == 0) return;
    const int64_t stride = X.left(n), nn = X.n[n];
    const uint32_t key = tk_rad_key(seed, n);
    const unsigned grid = (unsigned)std::min<int64_t>((numel + 255) / 256, 152 * 32);
    ProfScope ps(c, "elementwise", 2.0 * numel * dtype_size(X.dt), 0.0);
    switch (dtype_size(X.dt)) {
        case 8:
            sign_copy_kernel<uint64_t><<<grid, 256, 0, c.stream>>>(static_cast<const uint64_t*>(X.p),
                                                                   static_cast<uint64_t*>(dst), numel, stride, nn, key,
                                                                   (uint64_t)1 << 63);
            break;
        case 4:
            sign_copy_kernel<uint32_t><<<grid, 256, 0, c.stream>>>(static_cast<const uint32_t*>(X.p),
                                                                   static_cast<uint32_t*>(dst), numel, stride, nn, key,
                                                                   0x80000000u);
            break;
        case 2:
            sign_copy_kernel<uint16_t><<<grid, 256, 0, c.stream>>>(static_cast<const uint16_t*>(X.p),
                                                                   static_cast<uint16_t*>(dst), numel, stride, nn, key,
                                                                   (uint16_t)0x8000);
            break;
        default:
            sign_copy_kernel<uint8_t><<<grid, 256, 0, c.stream>>>(static_cast<const uint8_t*>(X.p),
                                                                  static_cast<uint8_t*>(dst), numel, stride, nn, key,
                                                                  (uint8_t)0x80);
            break;
    }
    c.counted();
    c.check_launch();
}

// ------------------------------------------------------------------ FP64 GEMM (NT) with split-K

__global__ void gemm_reduce_kernel(int64_t m, int64_t n, int nsplit, const double* P, double alpha, double beta,
                                   double* C, int64_t ldc, const int* skip) {
    if (skip && *skip) return;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m * n) return;
    double s = 0;
    for (int z = 0; z < nsplit; ++z) s += P[(int64_t)z * m * n + idx];
    int64_t a = idx % m, b = idx / m;
    double* dst = C + a + ldc * b;
    *dst = beta == 0.0 ? alpha * s : alpha * s + beta * *dst;
}

// 16 x 16 output tile per 256-thread CTA (one output per thread), K staged
// through shared memory 32 at a time for both operands (converted to FP64 on
// load).  Each operand is loaded with lanes running along whichever of its two
// indices is contiguous in memory.  Split-K: CTA z covers [z kchunk, (z+1)
// kchunk) and, with P != NULL, writes its partial tile to P[z] for a
// deterministic reduction; otherwise it applies alpha/beta to C directly.
struct TileLoader {
    // element e in [0, 512) of a 16 x 32 (row x k) tile -> (row, k)
    bool kfast;
    // k contiguous within 32-aligned runs (plain columns, or an unfolding whose
    // fastest contracted mode is a multiple of 32 long): warps read along k
    __device__ TileLoader(const View2& v) { kfast = v.st1 == 1 && (v.T1 == INT64_MAX || v.T1 % 32 == 0); }
    __device__ __forceinline__ void rk(int e, int& r, int& kk) const {
        if (kfast) { r = e >> 5; kk = e & 31; }
        else { r = e & 15; kk = e >> 4; }
    }
};

__device__ __forceinline__ int64_t v2row(const View2& v, int64_t a) {
    if (v.A1 == INT64_MAX) return a * v.sa1;
    if (a < 0x7fffffff && v.A1 < 0x7fffffff) {
        const uint32_t q = (uint32_t)a / (uint32_t)v.A1;
        return (int64_t)((uint32_t)a - q * (uint32_t)v.A1) * v.sa1 + (int64_t)q * v.sa2;
    }
    return (a % v.A1) * v.sa1 + (a / v.A1) * v.sa2;
}
__device__ __forceinline__ int64_t v2col(const View2& v, int64_t t) {
    if (v.T1 == INT64_MAX) return t * v.st1;
    if (t < 0x7fffffff && v.T1 < 0x7fffffff) {
        const uint32_t q = (uint32_t)t / (uint32_t)v.T1;
        return (int64_t)((uint32_t)t - q * (uint32_t)v.T1) * v.st1 + (int64_t)q * v.st2;
    }
    return (t % v.T1) * v.st1 + (t / v.T1) * v.st2;
}
__device__ __forceinline__ double v2get(const View2& v, int64_t o) {
    return v.dt == TK_F64 ? static_cast<const double*>(v.p)[o] : (double)static_cast<const float*>(v.p)[o];
}

// (hi, lo) += (bh, bl) for normalised double-float pairs (Knuth two-sum on
// the high parts, the low parts added into the error).
__device__ __forceinline__ void df_add(float& hi, float& lo, float bh, float bl) {
    const float s = __fadd_rn(hi, bh);
    const float v = __fadd_rn(s, -hi);
    const float e0 = __fadd_rn(__fadd_rn(hi, -__fadd_rn(s, -v)), __fadd_rn(bh, -v));  // hi + bh = s + e0 exactly
    const float e = __fadd_rn(e0, __fadd_rn(lo, bl));
    const float h2 = __fadd_rn(s, e);
    lo = __fadd_rn(e, -__fadd_rn(h2, -s));
    hi = h2;
}

// w * 2^-sh as a double-float pair, by integer splitting of the FP64
// significand (top 24 bits, then the next 29 rounded to FP32), with no FP64
// instruction.  Magnitudes below 2^-74 after scaling keep only the high part,
// below 2^-126 (outside FP32's normal range) they become zero, and at or
// above 2^128 the high part is an infinity.
__device__ __forceinline__ float2 df_from_f64(double w, int sh) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(w);
    const int ex = (int)((u >> 52) & 0x7FF);
    const int E = ex - 1023 - sh;
    if (ex == 0 || E < -126) return make_float2(0.f, 0.f);
    const unsigned sg = (unsigned)(u >> 63) << 31;
    if (E > 127) return make_float2(__uint_as_float(sg | 0x7F800000u), 0.f);
    const unsigned long long m = u & ((1ull << 52) - 1);
    const float hi = __uint_as_float(sg | ((unsigned)(E + 127) << 23) | (unsigned)(m >> 29));
    float lo = 0.f;
    if (E >= -74) {
        const float sc = __uint_as_float((unsigned)(E - 52 + 127) << 23);
        lo = __fmul_rn(__uint2float_rn((unsigned)(m & ((1u << 29) - 1))), sc);
        lo = __uint_as_float(__float_as_uint(lo) | sg);
    }
    return make_float2(hi, lo);
}

// One step of the compensated dot product Dot2 (Ogita, Rump and Oishi,
// "Accurate sum and dot product", 2005): the product is split exactly
// (p + e, e = fma(a, b, -p)), p is added to the running sum s with Knuth's
// two-sum, and both rounding errors go into the correction c.  Only s + p is
// on the loop-carried path; the result s + c is as accurate as a dot product
// carried out in twice the working precision.
__device__ __forceinline__ void dot2_step(float& s, float& c, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = fmaf(a, b, -p);
    const float t = __fadd_rn(s, p);
    const float z = __fadd_rn(t, -s);
    const float q = __fadd_rn(__fadd_rn(s, -__fadd_rn(t, -z)), __fadd_rn(p, -z));
    s = t;
    c = __fadd_rn(c, __fadd_rn(q, e));
}

// One Dot2 step for double-float operands a = a.x + a.y, b = b.x + b.y: the
// product of the high parts split exactly, the cross terms (their rounding is
// ~2^-48 of the product) and both rounding errors into the correction c; the
// low-low term (2^-48) is dropped.
__device__ __forceinline__ void df_dot_step(float& s, float& c, float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    const float t = __fadd_rn(s, p);
    const float z = __fsub_rn(t, s);
    const float q = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
    s = t;
    c = __fadd_rn(c, __fadd_rn(q, e));
}

// MODE 0: FP64 fma.  MODE 1: both operands hold FP32 values (FP32 data), and
// the products are
// accumulated on the FP32 pipe with Dot2 (as accurate as about 48 significant
// bits, several times the FP64 rate here); otherwise FP64 fma.
// One thread per output of out[l + L (a + m r)] = sum_i M(i, a) X[l + L (i + nj r)],
// FP64 operands split into double-float pairs (M staged split in shared
// memory), Dot2 accumulation: the FP64 pipe here is 1/64 of the FP32 pipe.
__global__ void __launch_bounds__(256) ttm_direct_df_kernel(const double* __restrict__ X, int64_t L, int64_t nj,
                                                            int64_t R, const double* __restrict__ M, int64_t ldm,
                                                            int mtrans, int64_t m, double* __restrict__ out) {
    extern __shared__ float2 msp[];  // nj x m: msp[i + nj a] = split M(i, a)
    for (int64_t e = threadIdx.x; e < nj * m; e += blockDim.x) {
        const int64_t i = e % nj, a = e / nj;
        msp[e] = df_from_f64(mtrans ? M[a + ldm * i] : M[i + ldm * a], 0);
    }
    __syncthreads();
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= L * m * R) return;
    const int64_t l = o % L, rest = o / L;
    const int64_t a = rest % m, r = rest / m;
    const double* x = X + l + L * nj * r;
    const float2* mc = msp + nj * a;
    float sh = 0.f, sl = 0.f;
    int64_t i = 0;
    for (; i + 8 <= nj; i += 8) {  // the eight loads issued before the products that use them
        double xv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) xv[u] = x[L * (i + u)];
#pragma unroll
        for (int u = 0; u < 8; ++u) df_dot_step(sh, sl, df_from_f64(xv[u], 0), mc[i + u]);
    }
    for (; i < nj; ++i) df_dot_step(sh, sl, df_from_f64(x[L * i], 0), mc[i]);
    out[o] = (double)sh + (double)sl;
}

static bool ttm_direct_df(const Ctx& c, const double* X, int64_t L, int64_t nj, int64_t R, const double* M,
                          int64_t ldm, bool mtrans, int64_t m, double* out) {
    const int64_t rows = L * R;
    const size_t smem = sizeof(float2) * (size_t)(nj * m);
    if (rows * m > (1 << 22) || smem > 48 * 1024) return false;
    ProfScope ps(c, "ttm_simt", 8.0 * rows * nj + 8.0 * rows * m, 2.0 * rows * nj * m);
    ttm_direct_df_kernel<<<(unsigned)((rows * m + 255) / 256), 256, smem, c.stream>>>(X, L, nj, R, M, ldm,
                                                                                     mtrans ? 1 : 0, m, out);
    c.counted();
    c.check_launch();
    return true;
}

template <typename E>
__device__ __forceinline__ E gemm_elem(double v) {
    if constexpr (std::is_same<E, float2>::value)
        return df_from_f64(v, 0);
    else
        return (E)v;
}

// MODE 2: the operands (FP64 or FP32) are split into double-float pairs on
// load and the products accumulate with df_dot_step on the FP32 pipe (~47
// significant bits; FP32's exponent range bounds the products).
template <int MODE>
__global__ void __launch_bounds__(256) gemm_tile16_kernel(int64_t m, int64_t n, int64_t K, int64_t kchunk, View2 A,
                                                          View2 B, double alpha, double beta, double* C, int64_t ldc,
                                                          double* P, unsigned* ctr, const int* skip) {
    constexpr bool DFACC = MODE != 0;
    using E = typename std::conditional<MODE == 0, double, typename std::conditional<MODE == 1, float, float2>::type>::type;
    if (skip && *skip) return;
    __shared__ E As[32][17];
    __shared__ E Bs[32][17];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t a0 = (int64_t)blockIdx.x * 16, b0 = (int64_t)blockIdx.y * 16;
    const int64_t kb = (int64_t)blockIdx.z * kchunk;
    const int64_t ke = min(K, kb + kchunk);
    const TileLoader la(A), lb(B);
    int ra[2], ka[2], rb[2], kb2[2];
    int64_t oa[2], ob[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        la.rk(tid + 256 * q, ra[q], ka[q]);
        lb.rk(tid + 256 * q, rb[q], kb2[q]);
        oa[q] = a0 + ra[q] < m ? v2row(A, a0 + ra[q]) : -1;
        ob[q] = b0 + rb[q] < n ? v2row(B, b0 + rb[q]) : -1;
    }
    double acc0 = 0.0, acc1 = 0.0;
    float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
    for (int64_t k0 = kb; k0 < ke; k0 += 32) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int64_t k1 = k0 + ka[q], k2 = k0 + kb2[q];
            As[ka[q]][ra[q]] = gemm_elem<E>((oa[q] >= 0 && k1 < ke) ? v2get(A, oa[q] + v2col(A, k1)) : 0.0);
            Bs[kb2[q]][rb[q]] = gemm_elem<E>((ob[q] >= 0 && k2 < ke) ? v2get(B, ob[q] + v2col(B, k2)) : 0.0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 32; kk += 2) {
            if constexpr (MODE == 2) {
                df_dot_step(h0, l0, As[kk][tx], Bs[kk][ty]);
                df_dot_step(h1, l1, As[kk + 1][tx], Bs[kk + 1][ty]);
            } else if constexpr (MODE == 1) {
                dot2_step(h0, l0, As[kk][tx], Bs[kk][ty]);
                dot2_step(h1, l1, As[kk + 1][tx], Bs[kk + 1][ty]);
            } else {
                acc0 = fma(As[kk][tx], Bs[kk][ty], acc0);
                acc1 = fma(As[kk + 1][tx], Bs[kk + 1][ty], acc1);
            }
        }
        __syncthreads();
    }
    const int64_t a = a0 + tx, b = b0 + ty;
    const bool in = a < m && b < n;
    const double sum = DFACC ? ((double)h0 + (double)l0) + ((double)h1 + (double)l1) : acc0 + acc1;
    if (!P) {
        if (in) {
            double* dst = C + a + ldc * b;
            *dst = beta == 0.0 ? alpha * sum : alpha * sum + beta * *dst;
        }
        return;
    }
    if (in) P[(int64_t)blockIdx.z * m * n + a + m * b] = sum;
    if (!ctr) return;  // a separate reduction kernel adds the partial tiles
    // the last CTA of this tile to arrive adds the partial tiles (and re-zeroes the counter)
    __shared__ int s_last;
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        unsigned* t = ctr + blockIdx.x + (int64_t)gridDim.x * blockIdx.y;
        const unsigned prev = atomicAdd(t, 1u);
        s_last = prev == gridDim.z - 1;
        if (s_last) *t = 0u;
    }
    __syncthreads();
    if (!s_last || !in) return;
    __threadfence();
    double tot = 0.0;
    for (int z = 0; z < (int)gridDim.z; ++z) tot += __ldcg(P + (int64_t)z * m * n + a + m * b);
    double* dst = C + a + ldc * b;
    *dst = beta == 0.0 ? alpha * tot : alpha * tot + beta * *dst;
}

// Small FP64 products (FP64 runs at 2 FMA per clock per SM here, so a
// 16 x 16 tile over 16 CTAs leaves the GPU idle): a CTA takes a T x T tile and
// splits K over G = 256 / T^2 thread groups, which are summed in shared memory
// at the end, so a k x k x k product with k ~ 50 spreads over ~170 SMs.
template <int T>
__global__ void __launch_bounds__(256) gemm_small_kernel(int64_t m, int64_t n, int64_t K, View2 A, View2 B,
                                                         double alpha, double beta, double* C, int64_t ldc,
                                                         const int* skip) {
    if (skip && *skip) return;
    constexpr int G = 256 / (T * T);
    __shared__ double As[32][T + 1];
    __shared__ double Bs[32][T + 1];
    __shared__ double red[G][T * T];
    const int tid = threadIdx.x, o = tid % (T * T), g = tid / (T * T);
    const int tx = o % T, ty = o / T;
    const int64_t a0 = (int64_t)blockIdx.x * T, b0 = (int64_t)blockIdx.y * T;
    const bool akf = A.st1 == 1 && (A.T1 == INT64_MAX || A.T1 % 32 == 0);
    const bool bkf = B.st1 == 1 && (B.T1 == INT64_MAX || B.T1 % 32 == 0);
    double acc = 0.0;
    for (int64_t k0 = 0; k0 < K; k0 += 32) {
        for (int e = tid; e < 64 * T; e += 256) {
            const bool isb = e >= 32 * T;
            const int f = isb ? e - 32 * T : e;
            const bool kf = isb ? bkf : akf;
            const int r = kf ? f >> 5 : f % T, kk = kf ? f & 31 : f / T;
            const View2& V = isb ? B : A;
            const int64_t row = (isb ? b0 : a0) + r, k = k0 + kk;
            const double v = (row < (isb ? n : m) && k < K) ? v2get(V, v2row(V, row) + v2col(V, k)) : 0.0;
            if (isb)
                Bs[kk][r] = v;
            else
                As[kk][r] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = g; kk < 32; kk += G) acc = fma(As[kk][tx], Bs[kk][ty], acc);
        __syncthreads();
    }
    red[g][o] = acc;
    __syncthreads();
    if (g != 0) return;
    double sum = 0.0;
#pragma unroll
    for (int q = 0; q < G; ++q) sum += red[q][o];
    const int64_t a = a0 + tx, b = b0 + ty;
    if (a >= m || b >= n) return;
    double* dst = C + a + ldc * b;
    *dst = beta == 0.0 ? alpha * sum : alpha * sum + beta * *dst;
}

void gemm_nt_f64(Ctx& c, int64_t m, int64_t n, int64_t K, const View2& A, const View2& B, double alpha, double beta,
                 double* C, int64_t ldc, const int* skip, bool df_ok) {
    // Dot2 accumulation where the caller allows it and both operands are FP32; double-float
    // operands throughout a call on FP32-class data (c.df64)
    const int mode = (df_ok && A.dt == TK_F32 && B.dt == TK_F32) ? 1 : (c.df64 ? 2 : 0);
    const bool df = mode != 0;
    // short K and few 16 x 16 tiles: smaller tiles with K split inside the CTA
    if (mode != 1 && K < 128 && ((m + 15) / 16) * ((n + 15) / 16) < 152) {
        if (!c.exec || m == 0 || n == 0) return;
        const bool t8 = ((m + 7) / 8) * ((n + 7) / 8) >= 152;
        const int T = t8 ? 8 : 4;
        dim3 grid((unsigned)((m + T - 1) / T), (unsigned)((n + T - 1) / T));
        ProfScope ps(c, "gemm_f64", 8.0 * (double)(m * ((n + T - 1) / T) + n * ((m + T - 1) / T)) * K + 8.0 * m * n,
                     2.0 * m * n * K);
        if (t8)
            gemm_small_kernel<8><<<grid, 256, 0, c.stream>>>(m, n, K, A, B, alpha, beta, C, ldc, skip);
        else
            gemm_small_kernel<4><<<grid, 256, 0, c.stream>>>(m, n, K, A, B, alpha, beta, C, ldc, skip);
        c.counted();
        c.check_launch();
        return;
    }
    // 16 x 16 tiles; split K only when the tiles alone leave most SMs idle and
    // each split still has at least 64 terms.
    const int64_t tiles = ((m + 15) / 16) * ((n + 15) / 16);
    int64_t nsplit = 1;
    if (K >= 128 && tiles < 2 * 152) {
        nsplit = std::min<int64_t>((2 * 152 + tiles - 1) / tiles, K / 64);
        nsplit = std::max<int64_t>(1, std::min<int64_t>(nsplit, 512));
    }
    int64_t kchunk = K > 0 ? (K + nsplit - 1) / nsplit : 1;
    kchunk = (kchunk + 31) / 32 * 32;
    nsplit = K > 0 ? (K + kchunk - 1) / kchunk : 1;
    double* P = nsplit > 1 ? c.alloc<double>(nsplit * m * n) : nullptr;
    if (!c.exec || m == 0 || n == 0) return;
    unsigned* ctr = nsplit > 1 ? c.take_counters((int)tiles) : nullptr;
    dim3 grid((unsigned)((m + 15) / 16), (unsigned)((n + 15) / 16), (unsigned)nsplit);
    {
        ProfScope ps(c, df ? "gemm_df" : "gemm_f64",
                     8.0 * (double)(m * ((n + 15) / 16) + n * ((m + 15) / 16)) * K + 8.0 * m * n * nsplit,
                     2.0 * m * n * K);
        if (mode == 1)
            gemm_tile16_kernel<1>
                <<<grid, 256, 0, c.stream>>>(m, n, K, kchunk, A, B, alpha, beta, C, ldc, P, ctr, skip);
        else if (mode == 2)
            gemm_tile16_kernel<2>
                <<<grid, 256, 0, c.stream>>>(m, n, K, kchunk, A, B, alpha, beta, C, ldc, P, ctr, skip);
        else
            gemm_tile16_kernel<0>
                <<<grid, 256, 0, c.stream>>>(m, n, K, kchunk, A, B, alpha, beta, C, ldc, P, ctr, skip);
        c.counted();
        c.check_launch();
    }
    if (nsplit > 1 && !ctr) {
        const int64_t tot = m * n;
        ProfScope ps(c, "gemm_f64", 8.0 * m * n * (nsplit + 1), (double)m * n * nsplit);
        gemm_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, c.stream>>>(m, n, (int)nsplit, P, alpha, beta, C,
                                                                                  ldc, skip);
        c.counted();
        c.check_launch();
    }
}

// ------------------------------------------------------------------ block reductions

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over the block (blockDim.x multiple of 32, <= 1024); every thread gets the result.
__device__ double block_sum(double v, double* scratch /* >= 33 */) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    if (wid == 0) {
        double t = lane < nw ? scratch[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) scratch[32] = t;
    }
    __syncthreads();
    return scratch[32];
}

// ------------------------------------------------------------------ Cholesky + inverse

// Cholesky W = R^T R with R^{-1} formed in the same column loop.  With
// L = R^T, step j computes row j of R (r_jj = sqrt(pivot), r_jl = a_jl / r_jj),
// applies the rank-1 trailing update, and advances a Gauss-Jordan forward
// elimination M <- L^{-1} started from M = I: row j of M is scaled by 1/r_jj and
// M(i, 0..j) -= r_ji M(j, 0..j) for i > j.  Both updates are enumerated as one
// packed index space, so every FP64 lane does useful work (the FP64 pipe is the
// bottleneck of this kernel).  The pivot's 1/sqrt is an FP32 seed refined by
// two FP64 Newton steps (error below one FP64 ulp-scale), and it is taken one
// column ahead by the thread that updates the next diagonal entry, which leaves
// two barriers per column.  R^{-1} = M^T.
__device__ __forceinline__ double chol_rsqrt(double a) {
    double y = (double)rsqrtf((float)a);
    const double h = 0.5 * a;
    y = y * fma(-h * y, y, 1.5);
    y = y * fma(-h * y, y, 1.5);
    return y;
}

constexpr int CHOL_THREADS = 256;

__global__ void __launch_bounds__(CHOL_THREADS) chol_inv_kernel(KDims kd, int kmax, const double* W, double* Rinv,
                                                                int* bad, double tol) {
    extern __shared__ double sm[];  // A: k x k (upper part becomes R), M: k x k lower (L^{-1})
    __shared__ double dg[256];
    __shared__ double s_y;
    __shared__ int s_bad;
    const int b = blockIdx.x;
    if (bad[b]) return;
    const int k = kd.k[b];
    double* A = sm;
    double* M = sm + (size_t)k * k;
    const double* Wb = W + (int64_t)b * kmax * kmax;
    double* Rb = Rinv + (int64_t)b * kmax * kmax;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < k * k; e += nt) {
        const int i = e % k, l = e / k;
        A[e] = Wb[i + (int64_t)kmax * l];
        M[e] = (i == l) ? 1.0 : 0.0;
    }
    for (int i = tid; i < k; i += nt) dg[i] = Wb[i + (int64_t)kmax * i];
    __syncthreads();
    if (tid == 0) {
        const double piv = A[0];
        s_bad = !(piv > tol * dg[0]) || !(piv > 0.0);
        s_y = s_bad ? 0.0 : chol_rsqrt(piv);
    }
    __syncthreads();
    for (int j = 0; j < k; ++j) {
        if (s_bad) break;  // uniform: written before the last barrier
        const double y = s_y;
        // row j of R and row j of M, one packed loop over the k columns
        for (int l = tid; l < k; l += nt) {
            if (l < j)
                M[j + k * l] *= y;
            else if (l == j) {
                M[j + k * j] *= y;
                A[j + k * j] *= y;  // pivot * (1/sqrt(pivot)) = r_jj
            } else
                A[j + k * l] *= y;
        }
        __syncthreads();
        // trailing update (j < i <= l) followed by the inverse update (i > j, l <= j)
        const int w = k - j - 1;
        const int ntri = w * (w + 1) / 2;
        const int ntot = ntri + w * (j + 1);
        for (int e = tid; e < ntot; e += nt) {
            if (e < ntri) {
                // column-packed triangle: l' = floor((sqrt(8e+1)-1)/2), i' = e - l'(l'+1)/2
                int lp = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
                while (lp * (lp + 1) / 2 > e) --lp;
                while ((lp + 1) * (lp + 2) / 2 <= e) ++lp;
                const int ip = e - lp * (lp + 1) / 2;
                const int i = j + 1 + ip, l = j + 1 + lp;
                const double v = A[i + k * l] - A[j + k * i] * A[j + k * l];
                A[i + k * l] = v;
                if (e == 0) {  // the next pivot: this thread updated A(j+1, j+1)
                    const bool fail = !(v > tol * dg[j + 1]) || !(v > 0.0);
                    s_bad = fail;
                    s_y = fail ? 0.0 : chol_rsqrt(v);
                }
            } else {
                const int e2 = e - ntri;
                const int i = j + 1 + e2 % w, l = e2 / w;
                M[i + k * l] -= A[j + k * i] * M[j + k * l];
            }
        }
        __syncthreads();
    }
    if (s_bad) {
        if (tid == 0) bad[b] = 1;
        return;
    }
    for (int e = tid; e < k * k; e += nt) {
        const int i = e % k, l = e / k;
        Rb[i + (int64_t)kmax * l] = (i <= l) ? M[l + k * i] : 0.0;
    }
}

// ------------------------------------------------------------------ Cholesky + inverse, double-float

// The same factorisation for Gram matrices of FP32-class data, carried out in
// double-float arithmetic (value = hi + lo, two FP32 numbers, ~48 significant
// bits) on the FP32 pipe, which is 64 times wider than the FP64 pipe here.
// W is scaled by 4^-e (2^{2e} near its largest diagonal entry) so that every
// entry is below ~4 in magnitude (|w_il| <= sqrt(w_ii w_ll)), far inside the
// FP32 exponent range; R_W^{-1} = 2^-e R_A^{-1} undoes it exactly.
//
// The column loop is the LDL^T form: with p_j the j-th pivot and l_ij =
// a_ji / p_j, step j updates the trailing upper triangle a_il -= l_ij a_jl
// (j < i <= l) and the unit lower M = L^{-1} by M(i, 0..j) -= l_ij M(j, 0..j);
// then R = D^{1/2} L^T and R^{-1} = M^T D^{-1/2}, i.e. R^{-1}(a, b) =
// M(b, a) / sqrt(p_b).  Row j is never rescaled, so warps can own whole rows
// (row-major storage, lanes along the row).

__device__ __forceinline__ float2 df_norm(float s, float t) {  // fast two-sum, |s| >= |t|
    const float h = __fadd_rn(s, t);
    return make_float2(h, __fsub_rn(t, __fsub_rn(h, s)));
}

__device__ __forceinline__ float2 df_mul2(float2 a, float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    return df_norm(p, e);
}

// a - f b
__device__ __forceinline__ float2 df_fnms2(float2 a, float2 f, float2 b) {
    const float p = __fmul_rn(f.x, b.x);
    float e = fmaf(f.x, b.x, -p);
    e = fmaf(f.x, b.y, e);
    e = fmaf(f.y, b.x, e);
    const float s = __fsub_rn(a.x, p);  // two-sum of a.x and -p
    const float v = __fsub_rn(s, a.x);
    const float t = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, v)), __fsub_rn(-p, v));
    return df_norm(s, __fadd_rn(t, __fsub_rn(a.y, e)));
}

// 1/p and 1/sqrt(p) of a positive double-float p: an FP32 seed (the fast
// approximate reciprocal and square root, a few ulp) and one Newton step
// evaluated in double-float, which squares the seed's relative error
// (~2^-44, then limited by the double-float format).
__device__ __forceinline__ void df_rcp_rsqrt(float2 p, float2& inv, float2& ys) {
    const float q0 = __fdividef(1.0f, p.x);
    float t = fmaf(-p.x, q0, 1.0f);
    t = fmaf(-p.y, q0, t);
    inv = df_norm(q0, __fmul_rn(q0, t));
    const float y0 = rsqrtf(p.x);
    const float a = __fmul_rn(y0, y0);
    const float2 y2 = make_float2(a, fmaf(y0, y0, -a));  // y0^2 exactly
    const float2 py = df_mul2(p, y2);
    const float d = __fsub_rn(__fsub_rn(1.0f, py.x), py.y);  // 1 - p y0^2 (~2^-22)
    ys = df_norm(y0, __fmul_rn(__fmul_rn(0.5f, y0), d));
}

constexpr int CHDF_THREADS = 768;
constexpr int CHDF_PANEL = 8;  // columns per panel (warps 0 .. CHDF_PANEL-1 own its rows)

// Blocked over panels of CHDF_PANEL columns.  Within a panel, warp w owns row
// j0 + w: at step j every warp whose row lies below j reads the pivot p_j
// (final: row j was last updated at step j - 1), forms 1/p_j itself, its
// multiplier l_ij and updates its row of A and of M; the panel's warps meet at
// a named barrier per column.  The rows below the panel then take the panel's
// updates in one pass, a_il -= sum_j l_ij a_jl and M(i, .) -= sum_j l_ij M(j, .),
// in the same order of j as the column-by-column form, so every entry sees the
// same operations on the same values (the result is that form's, bit for
// bit) with two CTA barriers per panel instead of one per column.
__global__ void __launch_bounds__(CHDF_THREADS) chol_inv_df_kernel(KDims kd, int kmax, const double* W,
                                                                   double* Rinv, int* bad, double tol) {
    extern __shared__ float2 sf[];  // A: k x k row-major (upper part), M: k x k row-major (lower part)
    __shared__ float2 s_ys[112];    // 1 / sqrt(p_j)
    __shared__ float2 s_inv[CHDF_PANEL];         // 1 / p_j of the panel's columns
    __shared__ float2 s_l[CHDF_PANEL][112];      // l_ij of the panel's columns for the rows below the panel
    __shared__ float s_dg[112];     // scaled original diagonal (breakdown test)
    __shared__ int s_fail;
    __shared__ int s_e;
    const int b = blockIdx.x;
    if (bad[b]) return;
    const int k = kd.k[b];
    float2* A = sf;
    float2* M = sf + (size_t)k * k;
    const double* Wb = W + (int64_t)b * kmax * kmax;
    double* Rb = Rinv + (int64_t)b * kmax * kmax;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    if (warp == 0) {
        double m = 0.0;
        for (int i = lane; i < k; i += 32) m = fmax(m, Wb[i + (int64_t)kmax * i]);
        for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) {
            int e = 0;
            if (m > 0.0 && m < 1e300) {
                const int be = (int)((__double_as_longlong(m) >> 52) & 0x7FF) - 1023;  // floor(log2 m), m normal
                e = (be >= 0 ? be : be - 1) / 2;
            }
            s_e = e;
            s_fail = 0;
        }
    }
    __syncthreads();
    const int e = s_e;
    for (int idx = tid; idx < k * k; idx += nt) {
        const int i = idx / k, l = idx - i * k;
        A[idx] = l >= i ? df_from_f64(Wb[i + (int64_t)kmax * l], 2 * e) : make_float2(0.f, 0.f);
        M[idx] = make_float2(i == l ? 1.f : 0.f, 0.f);
    }
    for (int i = tid; i < k; i += nt) s_dg[i] = df_from_f64(Wb[i + (int64_t)kmax * i], 2 * e).x;
    __syncthreads();
    for (int j0 = 0; j0 < k; j0 += CHDF_PANEL) {
        const int jb = min(CHDF_PANEL, k - j0);
        if (warp < CHDF_PANEL) {
            const int i = j0 + warp;  // this warp's row (none when warp >= jb)
            for (int jj = 0; jj < jb; ++jj) {
                const int j = j0 + jj;
                const float2 p = A[(size_t)j * k + j];
                if (!(p.x > (float)tol * s_dg[j] && p.x > 0.f)) {  // the same test in every warp
                    if (warp == 0 && lane == 0) s_fail = 1;
                    break;
                }
                float2 inv, ys;
                df_rcp_rsqrt(p, inv, ys);
                if (warp == jj && lane == 0) {
                    s_inv[jj] = inv;
                    s_ys[j] = ys;
                }
                if (warp < jb && i > j) {
                    const float2* Aj = A + (size_t)j * k;
                    const float2* Mj = M + (size_t)j * k;
                    const float2 f = df_mul2(Aj[i], inv);  // l_ij
                    float2* Ai = A + (size_t)i * k;
                    float2* Mi = M + (size_t)i * k;
                    for (int l = i + lane; l < k; l += 32) Ai[l] = df_fnms2(Ai[l], f, Aj[l]);
                    for (int cc = lane; cc <= j; cc += 32) Mi[cc] = df_fnms2(Mi[cc], f, Mj[cc]);
                }
                asm volatile("bar.sync 1, %0;" ::"n"(32 * CHDF_PANEL) : "memory");
            }
        }
        __syncthreads();
        if (s_fail) break;  // uniform: written before the barrier
        const int t0 = j0 + jb, nr = k - t0;
        if (nr <= 0) break;
        // the panel's multipliers for the rows below it
        for (int x = tid; x < jb * nr; x += nt) {
            const int jj = x / nr, i = t0 + x % nr;
            s_l[jj][i] = df_mul2(A[(size_t)(j0 + jj) * k + i], s_inv[jj]);
        }
        __syncthreads();
        for (int x = tid; x < nr * nr; x += nt) {  // A(i, l), t0 <= i <= l < k
            const int i = t0 + x / nr, l = t0 + x % nr;
            if (l < i) continue;
            float2 v = A[(size_t)i * k + l];
            for (int jj = 0; jj < jb; ++jj) v = df_fnms2(v, s_l[jj][i], A[(size_t)(j0 + jj) * k + l]);
            A[(size_t)i * k + l] = v;
        }
        for (int x = tid; x < nr * t0; x += nt) {  // M(i, c), t0 <= i < k, c < t0 (M(j, c) = 0 for c > j)
            const int i = t0 + x / t0, c = x % t0;
            float2 v = M[(size_t)i * k + c];
            for (int jj = 0; jj < jb; ++jj)
                if (c <= j0 + jj) v = df_fnms2(v, s_l[jj][i], M[(size_t)(j0 + jj) * k + c]);
            M[(size_t)i * k + c] = v;
        }
        __syncthreads();
    }
    if (s_fail) {  // a rejected pivot
        if (tid == 0) bad[b] = 1;
        return;
    }
    const double sc = __longlong_as_double((long long)(1023 - e) << 52);  // 2^-e
    for (int idx = tid; idx < k * k; idx += nt) {
        const int a = idx % k, c = idx / k;  // R^{-1}(a, c), column-major out
        double v = 0.0;
        if (a <= c) {
            const float2 r = df_mul2(M[(size_t)c * k + a], s_ys[c]);
            v = ((double)r.x + (double)r.y) * sc;
        }
        Rb[a + (int64_t)kmax * c] = v;
    }
}

void launch_chol_inv(const Ctx& c, int batch, const KDims& kd, int kmax, const double* W, double* Rinv, int* bad,
                     double tol, bool df) {
    if (!c.exec) return;
    TK_REQUIRE(kmax <= 112, TK_ERR_SHAPE, "chol_inv: at most 112 columns");
    if (df) {
        const size_t smem = 2 * sizeof(float2) * kmax * kmax;
        if (smem > 48 * 1024)
            TK_CUDA(cudaFuncSetAttribute(chol_inv_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        ProfScope ps(c, "chol_inv", 16.0 * batch * kmax * kmax, (2.0 / 3.0) * batch * kmax * kmax * kmax);
        chol_inv_df_kernel<<<batch, CHDF_THREADS, smem, c.stream>>>(kd, kmax, W, Rinv, bad, tol);
        c.counted();
        c.check_launch();
        return;
    }
    size_t smem = 2 * sizeof(double) * kmax * kmax;
    if (smem > 48 * 1024)
        TK_CUDA(cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ProfScope ps(c, "chol_inv", 16.0 * batch * kmax * kmax, (2.0 / 3.0) * batch * kmax * kmax * kmax);
    chol_inv_kernel<<<batch, CHOL_THREADS, smem, c.stream>>>(kd, kmax, W, Rinv, bad, tol);
    c.counted();
    c.check_launch();
}

// ------------------------------------------------------------------ Q = Y R^{-1}

__global__ void __launch_bounds__(256) apply_rinv_kernel(int64_t n, int64_t k, int rpc, View2 Y, const double* Rinv,
                                                         int64_t ldr, double* Q, const int* skip) {
    extern __shared__ double ys[];  // rpc x k
    if (skip && *skip) return;
    const int64_t i0 = (int64_t)blockIdx.x * rpc;
    for (int64_t e = threadIdx.x; e < rpc * k; e += blockDim.x) {
        int64_t ii = e % rpc, cc = e / rpc;
        ys[e] = (i0 + ii < n) ? v2ld(Y, i0 + ii, cc) : 0.0;
    }
    __syncthreads();
    for (int64_t e = threadIdx.x; e < rpc * k; e += blockDim.x) {
        int64_t ii = e % rpc, col = e / rpc;
        if (i0 + ii >= n) continue;
        double s = 0.0;
        for (int64_t cp = 0; cp <= col; ++cp) s = fma(ys[ii + rpc * cp], __ldg(Rinv + cp + ldr * col), s);
        Q[(i0 + ii) + n * col] = s;
    }
}

void launch_apply_rinv(const Ctx& c, int64_t n, int64_t k, const View2& Y, const double* Rinv, int64_t ldr, double* Q,
                       const int* skip) {
    if (!c.exec) return;
    // rows per CTA: enough CTAs to cover the SMs (the FP64 pipe of one SM is narrow), at most 8
    const int rpc = (int)std::min<int64_t>(8, std::max<int64_t>(1, (n + 151) / 152));
    size_t smem = sizeof(double) * rpc * k;
    if (smem > 48 * 1024)
        TK_CUDA(cudaFuncSetAttribute(apply_rinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ProfScope ps(c, "apply_rinv", 16.0 * n * k + 8.0 * k * k, (double)n * k * k);
    apply_rinv_kernel<<<(unsigned)((n + rpc - 1) / rpc), 256, smem, c.stream>>>(n, k, rpc, Y, Rinv, ldr, Q, skip);
    c.counted();
    c.check_launch();
}

// The same product for several matrices in one launch, in double-float
// arithmetic on the FP32 pipe: Y (FP32 or FP64) and R^{-1} (FP64) are split
// into hi + lo pairs and each output is a Dot2 sum (exact two-product of the
// high parts, the cross terms and both rounding errors in the correction),
// ~48 significant bits.  CTA (x, b): rows 32x .. 32x+31 of matrix b, a lane
// per row; warps take the column pairs (c, k-1-c) in turn, so that every
// warp sums about the same number of terms.
struct ApplyBatch {
    View2 Y[TK_MAX_D];
    const double* R[TK_MAX_D];
    double* Q[TK_MAX_D];
    const int* skip[TK_MAX_D];
    int64_t n[TK_MAX_D];
    int k[TK_MAX_D];
    int64_t ldr;
};

constexpr int APDF_THREADS = 256;
constexpr int APDF_U = 8;  // global loads in flight per thread while staging

__global__ void __launch_bounds__(APDF_THREADS) apply_rinv_df_kernel(ApplyBatch ab) {
    extern __shared__ float2 sa[];  // R^{-1}: k x k column-major, then Y rows: k x 32 ([col][row])
    const int b = blockIdx.y;
    if (ab.skip[b] && *ab.skip[b]) return;
    const int64_t n = ab.n[b];
    const int k = ab.k[b];
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    if (r0 >= n) return;
    float2* rs = sa;
    float2* ys = sa + (size_t)k * k;
    const double* R = ab.R[b];
    const View2 Y = ab.Y[b];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    // staging: every thread issues its global loads in groups of APDF_U before using any of
    // them (one round of L2 latency per group instead of one per element)
    const int nt = blockDim.x;
    for (int e0 = tid; e0 < k * k; e0 += APDF_U * nt) {
        double v[APDF_U];
#pragma unroll
        for (int u = 0; u < APDF_U; ++u) {
            const int e = e0 + u * nt, a = e % k, c = e / k;
            v[u] = (e < k * k && a <= c) ? R[a + ab.ldr * c] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < APDF_U; ++u)
            if (e0 + u * nt < k * k) rs[e0 + u * nt] = df_from_f64(v[u], 0);
    }
    if (Y.dt == TK_F64) {
        for (int e0 = tid; e0 < 32 * k; e0 += APDF_U * nt) {
            double v[APDF_U];
#pragma unroll
            for (int u = 0; u < APDF_U; ++u) {
                const int e = e0 + u * nt, rr = e & 31, c = e >> 5;
                v[u] = (e < 32 * k && r0 + rr < n) ? static_cast<const double*>(Y.p)[v2off(Y, r0 + rr, c)] : 0.0;
            }
#pragma unroll
            for (int u = 0; u < APDF_U; ++u)
                if (e0 + u * nt < 32 * k) ys[e0 + u * nt] = df_from_f64(v[u], 0);
        }
    } else {
        for (int e0 = tid; e0 < 32 * k; e0 += APDF_U * nt) {
            float v[APDF_U];
#pragma unroll
            for (int u = 0; u < APDF_U; ++u) {
                const int e = e0 + u * nt, rr = e & 31, c = e >> 5;
                v[u] = (e < 32 * k && r0 + rr < n) ? static_cast<const float*>(Y.p)[v2off(Y, r0 + rr, c)] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < APDF_U; ++u)
                if (e0 + u * nt < 32 * k) ys[e0 + u * nt] = make_float2(v[u], 0.f);
        }
    }
    __syncthreads();
    const int64_t row = r0 + lane;
    double* Q = ab.Q[b];
    for (int pc = warp; pc < (k + 1) / 2; pc += nw) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int col = h ? k - 1 - pc : pc;
            if (h && col == pc) break;
            float sh = 0.f, sl = 0.f;
            const float2* rc = rs + (size_t)k * col;
            for (int cp = 0; cp <= col; ++cp) {
                const float2 a = ys[cp * 32 + lane], r = rc[cp];
                const float p = __fmul_rn(a.x, r.x);
                float e = fmaf(a.x, r.x, -p);
                e = fmaf(a.x, r.y, e);
                e = fmaf(a.y, r.x, e);
                const float t = __fadd_rn(sh, p);
                const float z = __fsub_rn(t, sh);
                const float q = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, z)), __fsub_rn(p, z));
                sh = t;
                sl = __fadd_rn(sl, __fadd_rn(q, e));
            }
            if (row < n) Q[row + n * col] = (double)sh + (double)sl;
        }
    }
}

void launch_apply_rinv_df(const Ctx& c, int batch, const View2* Y, const int64_t* n, const int64_t* k,
                          const double* Rinv, int64_t kmax, double* const* Q, const int* bad) {
    if (!c.exec) return;
    ApplyBatch ab;
    int64_t nmax = 1;
    for (int b = 0; b < batch; ++b) {
        ab.Y[b] = Y[b];
        ab.R[b] = Rinv + b * kmax * kmax;
        ab.Q[b] = Q[b];
        ab.skip[b] = bad + b;
        ab.n[b] = n[b];
        ab.k[b] = (int)k[b];
        nmax = std::max(nmax, n[b]);
    }
    ab.ldr = kmax;
    const size_t smem = sizeof(float2) * (kmax * kmax + 32 * kmax);
    if (smem > 48 * 1024)
        TK_CUDA(cudaFuncSetAttribute(apply_rinv_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    double bytes = 0.0, flops = 0.0;
    for (int b = 0; b < batch; ++b) {
        bytes += 16.0 * n[b] * k[b] + 8.0 * k[b] * k[b];
        flops += (double)n[b] * k[b] * k[b];
    }
    ProfScope ps(c, "apply_rinv", bytes, flops);
    dim3 grid((unsigned)((nmax + 31) / 32), (unsigned)batch);
    apply_rinv_df_kernel<<<grid, APDF_THREADS, smem, c.stream>>>(ab);
    c.counted();
    c.check_launch();
}

// ------------------------------------------------------------------ Householder QR (fallback)

__global__ void __launch_bounds__(256) householder_kernel(int64_t n, int64_t k, View2 Y, double* A, double* Q,
                                                          double* tau, const int* run, int* slot, int slot_value) {
    __shared__ double red[33];
    __shared__ double v0s[256];
    const int tid = threadIdx.x, nt = blockDim.x;
    const bool go = !run || *run;
    if (slot && tid == 0) *slot = go ? slot_value : 0;  // the QR method this matrix took
    if (!go) return;
    for (int64_t idx = tid; idx < n * k; idx += nt) A[idx] = v2ld(Y, idx % n, idx / n);  // FP64 copy of Y
    __syncthreads();
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
    for (int64_t j = 0; j < k; ++j) {
        double* aj = A + n * j;
        double part = 0.0;
        for (int64_t i = j + 1 + tid; i < n; i += nt) part += aj[i] * aj[i];
        double sigma = block_sum(part, red);
        double x0 = aj[j];
        double nrm = sqrt(x0 * x0 + sigma);
        double beta = 0.0, v0 = 0.0, alpha = 0.0;
        if (nrm > 0.0) {
            alpha = x0 >= 0.0 ? -nrm : nrm;
            v0 = x0 - alpha;
            beta = 2.0 / (v0 * v0 + sigma);
        }
        __syncthreads();  // every thread has read aj[j]
        if (tid == 0) {
            if (nrm > 0.0) aj[j] = alpha;  // R_jj
            tau[j] = beta;
            v0s[j] = v0;
        }
        __syncthreads();
        if (beta != 0.0) {
            for (int64_t l = j + 1 + wid; l < k; l += nw) {
                double* al = A + n * l;
                const double alj = al[j];
                double w = 0.0;
                for (int64_t i = j + 1 + lane; i < n; i += 32) w += aj[i] * al[i];
                w = warp_sum(w);  // also orders every lane's read of al[j] before lane 0 writes it
                w += v0 * alj;
                if (lane == 0) al[j] -= beta * v0 * w;
                for (int64_t i = j + 1 + lane; i < n; i += 32) al[i] -= beta * aj[i] * w;
            }
        }
        __syncthreads();
    }
    // Q = H_0 ... H_{k-1} [I; 0]
    for (int64_t e = tid; e < n * k; e += nt) {
        int64_t i = e % n, col = e / n;
        Q[e] = (i == col) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int64_t j = k - 1; j >= 0; --j) {
        double beta = tau[j], v0 = v0s[j];
        const double* aj = A + n * j;
        if (beta != 0.0) {
            for (int64_t col = wid; col < k; col += nw) {
                double* qc = Q + n * col;
                const double qcj = qc[j];
                double w = 0.0;
                for (int64_t i = j + 1 + lane; i < n; i += 32) w += aj[i] * qc[i];
                w = warp_sum(w);
                w += v0 * qcj;
                if (lane == 0) qc[j] -= beta * v0 * w;
                for (int64_t i = j + 1 + lane; i < n; i += 32) qc[i] -= beta * aj[i] * w;
            }
        }
        __syncthreads();
    }
    // make diag(R) >= 0
    for (int64_t col = wid; col < k; col += nw) {
        double rjj = A[col + n * col];
        if (rjj < 0.0)
            for (int64_t i = lane; i < n; i += 32) Q[i + n * col] = -Q[i + n * col];
    }
}

void launch_householder(const Ctx& c, int64_t n, int64_t k, const View2& Y, double* A, double* Q, double* tau,
                        const int* run, int* slot, int slot_value) {
    if (!c.exec) return;
    TK_REQUIRE(k <= 256, TK_ERR_SHAPE, "householder: at most 256 columns");
    ProfScope ps(c, "householder", 16.0 * n * k, 8.0 * n * k * k);
    householder_kernel<<<1, 256, 0, c.stream>>>(n, k, Y, A, Q, tau, run, slot, slot_value);
    c.counted();
    c.check_launch();
}

// ------------------------------------------------------------------ Jacobi eigensolver

// 1 / sqrt(a) and 1 / a for a positive double inside FP32's range: an FP32
// seed (~2^-22) and two Newton steps in FP64 (quadratic: ~2^-88, i.e. FP64
// rounding), FMAs only.
__device__ __forceinline__ double jac_rsqrt(double a) {
    double y = (double)rsqrtf((float)a);
    const double h = 0.5 * a;
    y = y * fma(-h * y, y, 1.5);
    return y * fma(-h * y, y, 1.5);
}
__device__ __forceinline__ double jac_rcp(double a) {
    double y = (double)__frcp_rn((float)a);
    y = fma(y, fma(-a, y, 1.0), y);
    return fma(y, fma(-a, y, 1.0), y);
}

__global__ void __launch_bounds__(256) jacobi_kernel(int k, double* Ag, double* w, double* Vout, int max_sweeps,
                                                     int use_smem, double* gV, unsigned* flags) {
    extern __shared__ double sm[];
    __shared__ double cs[128], sn[128];
    __shared__ int P[128], Qp[128];
    const int tid = threadIdx.x, nt = blockDim.x;
    double* A = use_smem ? sm : Ag;
    double* V = use_smem ? sm + k * k : gV;
    if (use_smem)
        for (int e = tid; e < k * k; e += nt) A[e] = Ag[e];
    for (int e = tid; e < k * k; e += nt) V[e] = (e % k == e / k) ? 1.0 : 0.0;
    __syncthreads();
    const int kp = k + (k & 1);
    const int half = kp / 2;
    const double eps = 2.220446049250313e-16;
    __shared__ double red[33];
    double part = 0.0;
    for (int e = tid; e < k * k; e += nt) part += A[e] * A[e];
    const double fro = sqrt(block_sum(part, red));
    // scale by a power of two to ||A||_F in [0.5, 1) (exact), so that the rotation's reciprocal and
    // reciprocal square roots can start from FP32 seeds (the eigenvalues are scaled back at the end)
    int ex = 0;
    if (fro > 0.0 && fro < 1e300) frexp(fro, &ex);
    const double dsc = ldexp(1.0, -ex), usc = ldexp(1.0, ex);
    for (int e = tid; e < k * k; e += nt) A[e] *= dsc;
    __syncthreads();
    const double athr = 4.0 * eps * fro * dsc;  // absolute off-diagonal threshold
    bool converged = (k <= 1);
    for (int sweep = 0; sweep < max_sweeps && !converged; ++sweep) {
        int off = 0;
        for (int e = tid; e < k * k; e += nt) {
            int p = e % k, q = e / k;
            if (p < q) {
                double apq = fabs(A[p + k * q]);
                if (apq > athr) off = 1;
            }
        }
        if (!__syncthreads_or(off)) {
            converged = true;
            break;
        }
        for (int step = 0; step < kp - 1; ++step) {
            for (int t = tid; t < half; t += nt) {
                int p, q;
                if (t == 0) {
                    p = step % (kp - 1);
                    q = kp - 1;
                } else {
                    p = (step + t) % (kp - 1);
                    q = (step - t + (kp - 1)) % (kp - 1);
                }
                if (p > q) { int tmp = p; p = q; q = tmp; }
                double c = 1.0, s = 0.0;
                if (q < k) {
                    double app = A[p + k * p], aqq = A[q + k * q], apq = A[p + k * q];
                    if (fabs(apq) > athr) {
                        // t = sgn(phi) psi / (|phi| + rho), phi = a_qq - a_pp, psi = 2 a_pq,
                        // rho = sqrt(phi^2 + psi^2): the smaller root of t^2 + 2 t phi / psi - 1 = 0;
                        // c = 1 / sqrt(1 + t^2), s = t c.  Reciprocal and reciprocal square roots from
                        // FP32 seeds and FP64 Newton steps (FMAs only; entries are O(1) after scaling
                        // and rotated pairs have psi > 4 eps ||A||, so the seeds stay in FP32 range).
                        const double phi = aqq - app, psi = 2.0 * apq;
                        const double r2 = fma(phi, phi, psi * psi);
                        const double u = jac_rsqrt(r2);                  // 1 / rho
                        const double t1 = (phi >= 0.0 ? psi : -psi) * jac_rcp(fabs(phi) + r2 * u);
                        c = jac_rsqrt(fma(t1, t1, 1.0));
                        s = t1 * c;
                    }
                } else {
                    q = -1;
                }
                P[t] = p; Qp[t] = q; cs[t] = c; sn[t] = s;
            }
            __syncthreads();
            // rows: A <- J^T A
            for (int e = tid; e < half * k; e += nt) {
                int t = e / k, col = e % k;
                int p = P[t], q = Qp[t];
                if (q < 0 || sn[t] == 0.0) continue;
                double c = cs[t], s = sn[t];
                double a = A[p + k * col], b = A[q + k * col];
                A[p + k * col] = c * a - s * b;
                A[q + k * col] = s * a + c * b;
            }
            __syncthreads();
            // columns: A <- A J, V <- V J
            for (int e = tid; e < half * k; e += nt) {
                int t = e / k, row = e % k;
                int p = P[t], q = Qp[t];
                if (q < 0 || sn[t] == 0.0) continue;
                double c = cs[t], s = sn[t];
                double a = A[row + k * p], b = A[row + k * q];
                A[row + k * p] = c * a - s * b;
                A[row + k * q] = s * a + c * b;
                a = V[row + k * p]; b = V[row + k * q];
                V[row + k * p] = c * a - s * b;
                V[row + k * q] = s * a + c * b;
            }
            __syncthreads();
        }
    }
    if (!converged) {
        // one last check after the final sweep
        int off = 0;
        for (int e = tid; e < k * k; e += nt) {
            int p = e % k, q = e / k;
            if (p < q) {
                double apq = fabs(A[p + k * q]);
                if (apq > athr) off = 1;
            }
        }
        converged = !__syncthreads_or(off);
        if (!converged && tid == 0) atomicOr(flags, FLAG_NOT_CONVERGED);
    }
    // sort descending (stable by index)
    for (int i = tid; i < k; i += nt) {
        double wi = A[i + k * i];
        int rank = 0;
        for (int j2 = 0; j2 < k; ++j2) {
            double wj = A[j2 + k * j2];
            rank += (wj > wi) || (wj == wi && j2 < i);
        }
        w[rank] = wi * usc;
        for (int row = 0; row < k; ++row) Vout[row + k * rank] = V[row + k * i];
    }
}

void launch_jacobi(const Ctx& c, int64_t k, double* A, double* w, double* V, int max_sweeps, double* gV) {
    if (!c.exec) return;
    TK_REQUIRE(k <= 256, TK_ERR_SHAPE, "jacobi: at most 256 rows");
    int use_smem = k <= 112;
    size_t smem = use_smem ? 2 * sizeof(double) * k * k : 0;
    TK_REQUIRE(use_smem || gV, TK_ERR_SHAPE, "jacobi: above 112 rows the global-memory variant needs k x k scratch");
    if (smem > 48 * 1024)
        TK_CUDA(cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ProfScope ps(c, "jacobi", 24.0 * k * k, 9.0 * k * k * k * 8);
    jacobi_kernel<<<1, 256, smem, c.stream>>>((int)k, A, w, V, max_sweeps, use_smem, use_smem ? nullptr : gV,
                                              c.dflags);
    c.counted();
    c.check_launch();
}

// ------------------------------------------------------------------ mixed-precision Jacobi
// Two-sided cyclic Jacobi on a symmetric matrix held as a diagonal D and an
// FP32 off-diagonal F (zero diagonal), accumulating the rotations in an FP32
// matrix J.  Rotation angles use the diagonal difference; the pair's own 2 x 2
// block is updated in closed form (a_pp -= t a_pq, a_qq += t a_pq, a_pq = 0).
// When F is small in absolute terms (a matrix already close to diagonal), FP32
// storage of F carries FP64-level absolute accuracy, provided D accumulates the
// tiny updates t a_pq without loss: the resolving stage keeps D as an unevaluated
// sum of two floats (hi + lo, about 48 significant bits) updated with an exact
// two-product and two-sum (Dekker; Knuth), so no FP64 instruction (1/64 of the
// FP32 rate on this GPU) sits on the per-round critical path.
// Pairs follow the circle method on kp = k rounded up to even (an odd k gets
// a zero row and column that never rotates).  The indices sit in kp slots;
// slot pair t = (2t, 2t + 1) is rotated at every step, after which every entry
// moves by one fixed slot permutation pi (slot 0 stays, the other kp - 1 slots
// advance one place around a cycle), so over kp - 1 consecutive steps every
// pair of indices meets once.  Because the pairing is fixed in slot
// coordinates, a thread updates the same 2 x 2 block (pair t, pair u >= t) of
// F' = R^T F R at every step and writes it straight to the permuted positions
// of the next step: every shared-memory address is computed once, before the
// sweeps.  F keeps its upper triangle only (it stays exactly symmetric) and is
// double-buffered.  Warp 0 computes the rotations: at each step, lane t forms
// the next step's pivot of pair t itself (one entry of the block update, from
// the same inputs) and its rotation, and carries the pair's diagonal entries
// and index labels to their new slots, while the other warps update F; one
// barrier per step.  Rotations (c, s per pair and step) are logged to global
// memory and J = R_1 R_2 ... is formed by a second kernel that replays the log
// on every row of J independently (one warp per row, several CTAs) with the
// same permutation, so J's work is off the per-step critical path.  The matrix
// is scaled by a power of two to about unit Frobenius norm on entry (exact),
// which keeps its FP32 entries and the rotation arithmetic clear of overflow
// and underflow.  Converged: a sweep boundary at which no off-diagonal entry
// exceeds the threshold (absolute for the resolving stage, relative to the
// pair's diagonal entries for the seeding stage), or kp - 1 consecutive steps
// without a rotation.

constexpr int JM_MAX_THREADS = 1024;
constexpr int JM_BPT = 2;  // blocks per update thread: h (h + 1) / 2 <= 2 * 992 for h <= 56

// The slot an entry at slot x moves to after a step (h = kp / 2 pairs).
__device__ __forceinline__ int jm_pi(int x, int h) {
    if (h == 1 || x == 0) return x;
    if (x == 1) return 2;
    if (x & 1) return x - 2;
    return x == 2 * h - 2 ? 2 * h - 1 : x + 2;
}

// The slot whose entry moves to slot y.
__device__ __forceinline__ int jm_pi_inv(int y, int h) {
    if (h == 1 || y == 0) return y;
    if (y == 2) return 1;
    if (y & 1) return y == 2 * h - 1 ? 2 * h - 2 : y + 2;
    return y - 2;
}

__device__ __forceinline__ int jm_tri(int i, int j, int ld) { return i < j ? i * ld + j : j * ld + i; }

// Rotation annihilating the (p, q) entry f against the diagonal (p: hp + lp,
// q: hq + lq), with phi = a_qq - a_pp, psi = 2 a_pq, rho = sqrt(phi^2 +
// psi^2): the tangent is the smaller root t = sgn(phi) psi / (|phi| + rho) of
// t^2 + 2 t phi / psi - 1 = 0 and the diagonal moves by -+ t f; (c, s) come
// from the half angle, cos 2a = |phi| / rho, c = sqrt((1 + cos 2a) / 2),
// s = sin 2a / (2 c) = sgn(phi) f / (rho c), so that t and (c, s) each sit two
// special-function latencies after rho instead of c waiting on t.  Fast FP32
// reciprocals and square roots suffice (the off-diagonal is zeroed explicitly
// and convergence is measured).  Returns whether it rotates.
// Whether the off-diagonal entry f of the pair with diagonal entries hp, hq
// still needs a rotation: f^2 > max(trel2 |hp hq|, fthr2), a relative test
// (trel2 = tol^2) with an absolute floor (fthr2); trel2 = 0 gives the plain
// absolute test |f| > fthr.
__device__ __forceinline__ bool jm_big(float f, float hp, float hq, float trel2, float fthr2) {
    return f * f > fmaxf(trel2 * fabsf(hp * hq), fthr2);
}

template <bool DF>
__device__ __forceinline__ int jm_rotate(float f, float trel2, float fthr2, bool allow, float& hp, float& lp,
                                         float& hq, float& lq, float2& cs) {
    cs = make_float2(1.f, 0.f);
    if (!(allow && jm_big(f, hp, hq, trel2, fthr2))) return 0;
    float phi = hq - hp;
    if (DF) phi += lq - lp;
    const float psi = 2.f * f;
    const float r2 = fmaxf(fmaf(phi, phi, psi * psi), 1e-37f);
    const float u = rsqrtf(r2);  // 1 / rho
    const float aphi = fabsf(phi);
    const float t = __fdividef(phi >= 0.f ? psi : -psi, aphi + r2 * u);
    const float x = fmaf(0.5f * aphi, u, 0.5f);  // (1 + cos 2a) / 2, in [1/2, 1]
    const float w = rsqrtf(x);
    cs = make_float2(x * w, (phi >= 0.f ? f : -f) * u * w);
    if (DF) {
        const float ph = __fmul_rn(t, f);
        const float pl = fmaf(t, f, -ph);  // t f = ph + pl exactly
        df_add(hp, lp, -ph, -pl);
        df_add(hq, lq, ph, pl);
    } else {
        const float dt = t * f;
        hp -= dt;
        hq += dt;
    }
    return 1;
}

// What warp 0's lane needs to form the next-step pivot of one pair: the
// source block's read base and pairs, which of its four outputs, the source
// slots of the pair's two entries.
struct JmPivot {
    int rd, t, u, sp, sq;
    bool diag, row1, col1;
};

__device__ __forceinline__ JmPivot jm_pivot_source(int tp, int h, int ld) {
    JmPivot pv;
    pv.sp = jm_pi_inv(2 * tp, h);
    pv.sq = jm_pi_inv(2 * tp + 1, h);
    const int ta = pv.sp >> 1, tb = pv.sq >> 1;
    pv.diag = (ta == tb);  // only with a single pair
    pv.t = min(ta, tb);
    pv.u = max(ta, tb);
    const int rs = (ta <= tb) ? pv.sp : pv.sq, cs = (ta <= tb) ? pv.sq : pv.sp;  // row slot in pair t, column slot in u
    pv.row1 = rs & 1;
    pv.col1 = cs & 1;
    pv.rd = pv.diag ? (2 * pv.t) * ld + 2 * pv.t + 1 : (2 * pv.t) * ld + 2 * pv.u;
    return pv;
}

// The next-step pivot of a pair: one output of its source block's update.
__device__ __forceinline__ float jm_pivot_value(const JmPivot& pv, const float* F, const float2* mc, int ld) {
    const float2 rt = mc[pv.t];
    if (pv.diag) return rt.y != 0.f ? 0.f : F[pv.rd];
    const float2 ru = mc[pv.u];
    const float a = F[pv.rd], b = F[pv.rd + 1], c = F[pv.rd + ld], d = F[pv.rd + ld + 1];
    const float al = pv.row1 ? rt.y : rt.x, be = pv.row1 ? rt.x : -rt.y;  // row (2t or 2t + 1) of R_t^T
    const float x0 = fmaf(al, a, be * c), x1 = fmaf(al, b, be * d);
    const float ga = pv.col1 ? ru.y : ru.x, de = pv.col1 ? ru.x : -ru.y;  // column (2u or 2u + 1) of R_u
    return fmaf(ga, x0, de * x1);
}

// DF: the diagonal is a double-float pair (the stage that resolves the
// eigenvalues); otherwise a plain float (the first stage, which only seeds the
// second).  rlog: (max_sweeps * (kp - 1) + 1) * (kp / 2) entries; ginfo:
// 1 + kp ints (steps taken, then the final slot -> index labels).
template <bool DF>
__global__ void __launch_bounds__(JM_MAX_THREADS) jacobi_sweep_kernel(int k, const double* __restrict__ A,
                                                                      double* Dout, double tol, int max_sweeps,
                                                                      float2* __restrict__ rlog,
                                                                      int* __restrict__ ginfo, unsigned* flags) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int kp = k + (k & 1), h = kp / 2, m = kp - 1;
    const int ld = kp + 1;  // odd stride: walks along either index are bank-conflict free
    float* Fc = reinterpret_cast<float*>(smraw);  // upper triangle in slot coordinates: F(a, b) = Fc[a * ld + b], a < b
    float* Fx = Fc + (size_t)kp * ld;             // the next step's
    float* Hc = Fx + (size_t)kp * ld;             // diagonal (high part) per slot
    float* Hx = Hc + kp;
    float* Lc = Hx + kp;                          // diagonal (low part) per slot
    float* Lx = Lc + kp;
    int* lab = reinterpret_cast<int*>(Lx + kp);   // final index label per slot (after the sweeps)
    __shared__ float2 meta[2][64];  // (c, s) per pair of the current / next step
    __shared__ int ired[33];
    __shared__ float fred[33];
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    const bool rwarp = tid < 32;
    // Scale 2^-sh with ||A||_F 2^-sh in [0.5, 1), found with integer and FP32 operations only
    // (FP64 runs at 1/64 of the FP32 rate here): the largest exponent of the entries, then the
    // norm of the entries scaled below 1 in FP32, which places ||A|| within its binade.
    int emax = -100000;
    for (int e = tid; e < k * k; e += nt) {
        const int ex = (int)((__double_as_longlong(A[e]) >> 52) & 0x7FF);
        if (ex) emax = max(emax, ex - 1023);
    }
    for (int o = 16; o; o >>= 1) emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
    if (lane == 0) ired[tid >> 5] = emax;
    __syncthreads();
    if (tid < 32) {
        int v = tid < (nt >> 5) ? ired[tid] : -100000;
        for (int o = 16; o; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (tid == 0) ired[32] = v;
    }
    __syncthreads();
    emax = ired[32];
    float part = 0.f;
    if (emax > -100000)
        for (int e = tid; e < k * k; e += nt) {
            const float2 v = df_from_f64(A[e], emax + 1);
            part = fmaf(v.x, v.x, part);
        }
    for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) fred[tid >> 5] = part;
    __syncthreads();
    if (tid < 32) {
        float v = tid < (nt >> 5) ? fred[tid] : 0.f;
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (tid == 0) fred[32] = v;
    }
    __syncthreads();
    int ex2 = 0;
    const float nsc = (fred[32] > 0.f) ? frexpf(sqrtf(fred[32]), &ex2) : 0.f;  // ||A|| 2^-sh in [0.5, 1)
    const int sh = (fred[32] > 0.f) ? emax + 1 + ex2 : 0;
    for (int e = tid; e < kp * kp; e += nt) {
        const int i = e % kp, j = e / kp;
        if (i < j) {
            float f = 0.f;
            if (j < k) {
                const float2 v = df_from_f64(A[i + (int64_t)k * j], sh);
                f = __fadd_rn(v.x, v.y);
            }
            Fc[i * ld + j] = f;
        } else if (i == j) {
            float2 v = make_float2(0.f, 0.f);
            if (i < k) v = df_from_f64(A[i + (int64_t)k * i], sh);
            const float hv = __fadd_rn(v.x, v.y);  // nearest FP32 value (hi + lo renormalised)
            Hc[i] = hv;
            Lc[i] = DF ? __fsub_rn(v.y, __fsub_rn(hv, v.x)) : 0.f;
        }
    }
    // DF (the resolving stage): absolute threshold tol ||A||.  Otherwise (the
    // seeding stage) relative: |a_pq| <= tol sqrt(|a_pp a_qq|), with a floor of
    // 1e-13 ||A|| below which FP32 entries carry no information (an exactly
    // rank-deficient tail would otherwise keep rotating on rounding noise).
    // Resolving each pair against its own diagonal entries leaves the
    // small-eigenvalue tail coupled only at ~1e-7 of its own scale, so the
    // resolving stage then needs one or two sweeps instead of four to six.
    const float trel2 = DF ? 0.f : (float)(tol * tol);
    const float fthr = (DF ? (float)tol : 1e-13f) * nsc;
    const float fthr2 = fthr * fthr;
    // update threads (warps 1..): their blocks' read bases and write addresses
    const int nblk = h * (h + 1) / 2, nu = nt - 32, ut = tid - 32;
    int bt[JM_BPT], rd[JM_BPT], w0[JM_BPT], w1[JM_BPT], w2[JM_BPT], w3[JM_BPT];
#pragma unroll
    for (int b = 0; b < JM_BPT; ++b) {
        bt[b] = -1;
        rd[b] = w0[b] = w1[b] = w2[b] = w3[b] = 0;
        const int e = ut + b * nu;
        if (rwarp || e >= nblk) continue;
        int t = 0, rem = e;
        while (rem >= h - t) {
            rem -= h - t;
            ++t;
        }
        const int u = t + rem;
        bt[b] = t | (u << 8);
        if (t == u) {
            rd[b] = 2 * t * ld + 2 * t + 1;
            w0[b] = jm_tri(jm_pi(2 * t, h), jm_pi(2 * t + 1, h), ld);
        } else {
            rd[b] = 2 * t * ld + 2 * u;
            const int pr0 = jm_pi(2 * t, h), pr1 = jm_pi(2 * t + 1, h), pc0 = jm_pi(2 * u, h), pc1 = jm_pi(2 * u + 1, h);
            w0[b] = jm_tri(pr0, pc0, ld);
            w1[b] = jm_tri(pr0, pc1, ld);
            w2[b] = jm_tri(pr1, pc0, ld);
            w3[b] = jm_tri(pr1, pc1, ld);
        }
    }
    // warp 0: the pairs lane and lane + 32
    const bool has0 = rwarp && lane < h, has1 = rwarp && lane + 32 < h;
    JmPivot pv0 = jm_pivot_source(has0 ? lane : 0, h, ld), pv1 = jm_pivot_source(has1 ? lane + 32 : 0, h, ld);
    __syncthreads();
    const int total = max_sweeps * m;  // steps allowed (the launcher bounds it)
    int any = 0;
    if (total > 0 && rwarp) {  // the first step's rotations, in place
#pragma unroll
        for (int o = 0; o < 2; ++o) {
            const int tp = lane + 32 * o;
            if (tp >= h) continue;
            const int p = 2 * tp, q = p + 1;
            float hp = Hc[p], lp = Lc[p], hq = Hc[q], lq = Lc[q];
            float2 cs;
            any |= jm_rotate<DF>(Fc[p * ld + q], trel2, fthr2, true, hp, lp, hq, lq, cs);
            Hc[p] = hp;
            Lc[p] = lp;
            Hc[q] = hq;
            Lc[q] = lq;
            meta[0][tp] = cs;
            rlog[tp] = cs;
        }
    }
    int active = __syncthreads_or(any);  // whether the current step rotates anything
    int cur = 0, steps = 0, s = 0, idle = 0;
    bool converged = false;
    float2* lg = rlog + h;  // the next step's log slot
    for (int g = 0; g < total; ++g, lg += h) {
        if (s == 0) {
            int off = 0;
            for (int a = tid >> 5; a < kp; a += nt >> 5)
                for (int b = a + 1 + lane; b < kp; b += 32) off |= jm_big(Fc[a * ld + b], Hc[a], Hc[b], trel2, fthr2);
            if (!__syncthreads_or(off)) {
                converged = true;
                break;
            }
        }
        idle = active ? 0 : idle + 1;
        if (idle >= m) {
            converged = true;
            break;
        }
        const float2* mc = meta[cur];
        any = 0;
        if (rwarp) {
            const bool want = g + 1 < total;
            float2* mn = meta[cur ^ 1];
#pragma unroll
            for (int o = 0; o < 2; ++o) {
                if (!(o ? has1 : has0)) continue;
                const JmPivot& pv = o ? pv1 : pv0;
                const int tp = lane + 32 * o;
                float hp = Hc[pv.sp], hq = Hc[pv.sq], lp = 0.f, lq = 0.f;
                if (DF) {
                    lp = Lc[pv.sp];
                    lq = Lc[pv.sq];
                }
                const float f = jm_pivot_value(pv, Fc, mc, ld);
                float2 cs;
                any |= jm_rotate<DF>(f, trel2, fthr2, want, hp, lp, hq, lq, cs);
                Hx[2 * tp] = hp;
                Hx[2 * tp + 1] = hq;
                if (DF) {
                    Lx[2 * tp] = lp;
                    Lx[2 * tp + 1] = lq;
                }
                mn[tp] = cs;
                lg[tp] = cs;
            }
        } else {
#pragma unroll
            for (int b = 0; b < JM_BPT; ++b) {
                if (bt[b] < 0) continue;
                const int t = bt[b] & 255, u = bt[b] >> 8;
                const float2 rt = mc[t];
                if (t == u) {  // the pair's own entry: annihilated when it rotates
                    Fx[w0[b]] = rt.y != 0.f ? 0.f : Fc[rd[b]];
                    continue;
                }
                const float2 ru = mc[u];
                const int r = rd[b];
                const float a = Fc[r], bb = Fc[r + 1], cc = Fc[r + ld], dd = Fc[r + ld + 1];
                const float r00 = fmaf(rt.x, a, -rt.y * cc), r01 = fmaf(rt.x, bb, -rt.y * dd);
                const float r10 = fmaf(rt.y, a, rt.x * cc), r11 = fmaf(rt.y, bb, rt.x * dd);
                Fx[w0[b]] = fmaf(ru.x, r00, -ru.y * r01);
                Fx[w1[b]] = fmaf(ru.y, r00, ru.x * r01);
                Fx[w2[b]] = fmaf(ru.x, r10, -ru.y * r11);
                Fx[w3[b]] = fmaf(ru.y, r10, ru.x * r11);
            }
        }
        const int nxt = __syncthreads_or(any);
        float* x;
        x = Fc; Fc = Fx; Fx = x;
        x = Hc; Hc = Hx; Hx = x;
        x = Lc; Lc = Lx; Lx = x;
        cur ^= 1;
        ++steps;
        s = (s + 1 == m) ? 0 : s + 1;
        active = nxt;
    }
    if (!converged) {  // the allowed sweeps ran out: measure once more
        int off = 0;
        for (int a = tid >> 5; a < kp; a += nt >> 5)
            for (int b = a + 1 + lane; b < kp; b += 32) off |= jm_big(Fc[a * ld + b], Hc[a], Hc[b], trel2, fthr2);
        converged = !__syncthreads_or(off);
    }
    if (!converged && tid == 0) atomicOr(flags, FLAG_NOT_CONVERGED);
    // index labels: after `steps` moves slot x holds the index that started in
    // slot pi^{-steps}(x); slots 1..kp-1 form one cycle of pi, walked once
    // (the cycle in closed form: position j holds slot 1 for j = 0, slot 2j for 1 <= j < h, slot
    // 2h - 1 - 2(j - h) for j >= h; so slot x sits at 0, x / 2 or h + (2h - 1 - x) / 2)
    if (tid < kp) {
        int lb = 0;
        if (tid > 0 && m > 0) {
            const int pos = tid == 1 ? 0 : ((tid & 1) ? h + (2 * h - 1 - tid) / 2 : tid / 2);
            int j = pos - steps % m;
            if (j < 0) j += m;
            lb = j == 0 ? 1 : (j < h ? 2 * j : 2 * h - 1 - 2 * (j - h));
        }
        lab[tid] = lb;
    }
    __syncthreads();
    // 2^sh as two representable factors (sh may reach past the FP64 exponent range by one)
    const double up1 = __longlong_as_double((long long)(1023 + sh / 2) << 52);
    const double up2 = __longlong_as_double((long long)(1023 + sh - sh / 2) << 52);
    for (int x = tid; x < kp; x += nt) {
        const int i = lab[x];
        if (i < k) Dout[i] = (((double)Hc[x] + (DF ? (double)Lc[x] : 0.0)) * up1) * up2;
        ginfo[1 + x] = i;
    }
    if (tid == 0) ginfo[0] = steps;
}

// J = R_1 R_2 ... R_steps from the log, one warp per row of J: lane t holds
// pair t (and t + 32), rotates it and writes it to the permuted slots of the
// next step; the final slot labels say which column each slot is.  The log is
// staged through shared memory in chunks, the next chunk fetched into
// registers while the current one is applied.
constexpr int JR_WARPS = 4;
constexpr int JR_STAGE = 8;  // log entries a thread carries while staging

// Order key of a double (an int64 that compares as the value does; -0.0 as +0.0).
__device__ __forceinline__ long long jr_key(double d) {
    if (d == 0.0) return 0;
    const long long u = __double_as_longlong(d);
    return u >= 0 ? u : (u ^ 0x7FFFFFFFFFFFFFFFll);
}

// With V1 (k x k, FP64, ld k) the rows replayed are those of V1 instead of the
// identity, i.e. the kernel forms V = V1 J without J, and writes the columns
// of V of the r largest D (ties: lower index first) into Vt and Vr (k x r,
// ld k), ordered by rank.
__global__ void __launch_bounds__(JR_WARPS * 32) jacobi_replay_kernel(int k, const float2* __restrict__ rlog,
                                                                      const int* __restrict__ ginfo, float* Jout,
                                                                      double* J64a, double* J64b,
                                                                      const double* __restrict__ V1,
                                                                      const double* __restrict__ D, int r,
                                                                      double* Vt, double* Vr) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int kp = k + (k & 1), h = kp / 2;
    const int nt = JR_WARPS * 32, cr = JR_STAGE * nt / h;  // steps per chunk
    float2* stage = reinterpret_cast<float2*>(smraw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float* ra = reinterpret_cast<float*>(stage + (size_t)cr * h) + (size_t)warp * 2 * kp;  // this warp's row
    float* rb = ra + kp;
    long long* keys = reinterpret_cast<long long*>(ra - (size_t)warp * 2 * kp + (size_t)JR_WARPS * 2 * kp);
    const int i = blockIdx.x * JR_WARPS + warp;
    const int steps = ginfo[0];
    if (V1) {
        for (int x = lane; x < kp; x += 32) ra[x] = (i < k && x < k) ? (float)V1[i + (int64_t)k * x] : 0.f;
        for (int x = tid; x < k; x += nt) keys[x] = jr_key(D[x]);
    } else {
        for (int x = lane; x < kp; x += 32) ra[x] = (x == i) ? 1.f : 0.f;
    }
    __syncthreads();  // the keys are read by every warp at the end (also when no step was taken)
    const int t0 = lane, t1 = lane + 32;
    const int d00 = jm_pi(2 * t0, h), d01 = jm_pi(2 * t0 + 1, h);
    const int d10 = jm_pi(2 * t1, h), d11 = jm_pi(2 * t1 + 1, h);
    float2 pre[JR_STAGE];
    int cn = min(cr, steps);
#pragma unroll
    for (int w = 0; w < JR_STAGE; ++w) {
        const int e = tid + w * nt;
        if (e < cn * h) pre[w] = rlog[e];
    }
    for (int c0 = 0; c0 < steps;) {
        __syncthreads();  // the previous chunk is no longer read
#pragma unroll
        for (int w = 0; w < JR_STAGE; ++w) {
            const int e = tid + w * nt;
            if (e < cn * h) stage[e] = pre[w];
        }
        __syncthreads();
        const int c1 = c0 + cn, nn = min(cr, steps - c1);
#pragma unroll
        for (int w = 0; w < JR_STAGE; ++w) {
            const int e = tid + w * nt;
            if (e < nn * h) pre[w] = rlog[(int64_t)c1 * h + e];
        }
        if (i < k) {
            for (int rr = 0; rr < cn; ++rr) {
                const float2* cs = stage + rr * h;
                if (t0 < h) {
                    const float2 q = cs[t0];
                    const float a = ra[2 * t0], b = ra[2 * t0 + 1];
                    rb[d00] = fmaf(q.x, a, -q.y * b);
                    rb[d01] = fmaf(q.y, a, q.x * b);
                }
                if (t1 < h) {
                    const float2 q = cs[t1];
                    const float a = ra[2 * t1], b = ra[2 * t1 + 1];
                    rb[d10] = fmaf(q.x, a, -q.y * b);
                    rb[d11] = fmaf(q.y, a, q.x * b);
                }
                __syncwarp();  // the next step reads slots other lanes wrote
                float* x = ra;
                ra = rb;
                rb = x;
            }
        }
        c0 = c1;
        cn = nn;
    }
    __syncwarp();
    if (i >= k) return;
    for (int x = lane; x < kp; x += 32) {
        const int j = ginfo[1 + x];
        if (j >= k) continue;
        const float v = ra[x];
        if (V1) {
            const long long kj = keys[j];
            int rank = 0;
            for (int l = 0; l < k; ++l) {
                const long long kl = keys[l];
                rank += (kl > kj) || (kl == kj && l < j);
            }
            if (rank < r) {
                Vt[i + (int64_t)k * rank] = (double)v;
                Vr[i + (int64_t)k * rank] = (double)v;
            }
            continue;
        }
        if (Jout) Jout[i + (int64_t)k * j] = v;
        if (J64a) J64a[i + (int64_t)k * j] = (double)v;
        if (J64b) J64b[i + (int64_t)k * j] = (double)v;
    }
}

void launch_jacobi_mixed(Ctx& c, int64_t k, const double* A, double* D, float* J, double* J64a, double* J64b,
                         double tol, int max_sweeps, bool fp64_diag, const double* V1, int64_t r, double* Vt,
                         double* Vr) {
    TK_REQUIRE(k >= 1 && k <= 112, TK_ERR_SHAPE, "jacobi_mixed: 1 <= k <= 112");
    TK_REQUIRE(max_sweeps >= 0 && (int64_t)max_sweeps * (k + 1) < (1 << 30), TK_ERR_ARG,
               "jacobi_mixed: 0 <= max_sweeps and max_sweeps * k below 2^30");
    const int64_t kp = k + (k & 1), h = kp / 2, nblk = h * (h + 1) / 2;
    float2* rlog = c.alloc<float2>(((int64_t)max_sweeps * (kp - 1) + 1) * h);
    int* ginfo = c.alloc<int>(1 + kp);
    if (!c.exec) return;
    const size_t smem = sizeof(float) * (2 * kp * (kp + 1) + 4 * kp) + sizeof(int) * 2 * kp;
    // warp 0 computes rotations; the rest update blocks (at most JM_BPT each)
    const int64_t nu = std::min<int64_t>(JM_MAX_THREADS - 32, (nblk + 31) / 32 * 32);
    const int nt = (int)(32 + nu);
    {
        ProfScope ps(c, "jacobi", 8.0 * k * k + 8.0 * k, 12.0 * k * k * k * max_sweeps);
        if (fp64_diag) {
            if (smem > 48 * 1024)
                TK_CUDA(cudaFuncSetAttribute(jacobi_sweep_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem));
            jacobi_sweep_kernel<true>
                <<<1, nt, smem, c.stream>>>((int)k, A, D, tol, max_sweeps, rlog, ginfo, c.dflags);
        } else {
            if (smem > 48 * 1024)
                TK_CUDA(cudaFuncSetAttribute(jacobi_sweep_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem));
            jacobi_sweep_kernel<false>
                <<<1, nt, smem, c.stream>>>((int)k, A, D, tol, max_sweeps, rlog, ginfo, c.dflags);
        }
        c.counted();
        c.check_launch();
    }
    if (!J && !J64a && !J64b && !V1) return;
    TK_REQUIRE(!V1 || (Vt && Vr && r >= 1 && r <= k), TK_ERR_ARG, "jacobi_mixed: V1 needs Vt, Vr and 1 <= r <= k");
    const int cr = JR_STAGE * JR_WARPS * 32 / (int)h;
    const size_t rsmem = sizeof(float2) * cr * h + sizeof(float) * JR_WARPS * 2 * kp + sizeof(long long) * kp;
    ProfScope ps(c, "jacobi", 8.0 * h * (max_sweeps * (kp - 1) + 1) + 8.0 * k * k, 6.0 * k * k * k * max_sweeps);
    jacobi_replay_kernel<<<(unsigned)((k + JR_WARPS - 1) / JR_WARPS), JR_WARPS * 32, rsmem, c.stream>>>(
        (int)k, rlog, ginfo, J, J64a, J64b, V1, D, (int)r, Vt, Vr);
    c.counted();
    c.check_launch();
}

// Vr[:, rank] = V[:, i] for the r largest D (ties: lower index first).
__global__ void select_top_kernel(int64_t k, int64_t r, const double* D, const double* V, double* Vr, double* Vr2) {
    for (int64_t i = blockIdx.x; i < k; i += gridDim.x) {
        double di = D[i];
        int64_t rank = 0;
        for (int64_t j = 0; j < k; ++j) {
            double dj = D[j];
            rank += (dj > di) || (dj == di && j < i);
        }
        if (rank >= r) continue;
        for (int64_t row = threadIdx.x; row < k; row += blockDim.x) {
            const double v = V[row + k * i];
            Vr[row + k * rank] = v;
            if (Vr2) Vr2[row + k * rank] = v;
        }
    }
}

void launch_select_top(const Ctx& c, int64_t k, int64_t r, const double* D, const double* V, double* Vr,
                       double* Vr2) {
    if (!c.exec || k == 0 || r == 0) return;
    ProfScope ps(c, "elementwise", 16.0 * k * r, 0.0);
    select_top_kernel<<<(unsigned)k, 64, 0, c.stream>>>(k, r, D, V, Vr, Vr2);
    c.counted();
    c.check_launch();
}

// ------------------------------------------------------------------ element-wise helpers

__global__ void convert_kernel(const void* src, tk_dtype sdt, int64_t rows, int64_t cols, int64_t lds, void* dst,
                               tk_dtype ddt, int64_t ldd, float inv) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    int64_t i = idx % rows, j = idx / rows;
    st_any(dst, ddt, i + ldd * j, ld_any(src, sdt, i + lds * j, inv));
}

void launch_convert(const Ctx& c, const void* src, tk_dtype sdt, int64_t rows, int64_t cols, int64_t lds, void* dst,
                    tk_dtype ddt, int64_t ldd, float src_scale) {
    if (!c.exec || rows * cols == 0) return;
    float inv = (sdt == TK_FP8_E4M3) ? 1.f / src_scale : 1.f;
    int64_t tot = rows * cols;
    ProfScope ps(c, "elementwise", (double)tot * (dtype_size(sdt) + dtype_size(ddt)), 0.0);
    convert_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, c.stream>>>(src, sdt, rows, cols, lds, dst, ddt, ldd,
                                                                         inv);
    c.counted();
    c.check_launch();
}

__global__ void fill_identity_kernel(double* Q, int64_t n) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    Q[idx] = (idx % n == idx / n) ? 1.0 : 0.0;
}

void launch_fill_identity(const Ctx& c, double* Q, int64_t n) {
    if (!c.exec || n == 0) return;
    ProfScope ps(c, "elementwise", 8.0 * n * n, 0.0);
    fill_identity_kernel<<<(unsigned)((n * n + 255) / 256), 256, 0, c.stream>>>(Q, n);
    c.counted();
    c.check_launch();
}

__global__ void copy_unfold_kernel(View2 Y, int64_t n, int64_t k, double* A, const int* run) {
    if (run && !*run) return;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * k) return;
    A[idx] = v2ld(Y, idx % n, idx / n);
}

void launch_copy_unfold_to_matrix(const Ctx& c, const View2& Y, int64_t n, int64_t k, double* A, const int* run) {
    if (!c.exec || n * k == 0) return;
    ProfScope ps(c, "elementwise", 16.0 * n * k, 0.0);
    copy_unfold_kernel<<<(unsigned)((n * k + 255) / 256), 256, 0, c.stream>>>(Y, n, k, A, run);
    c.counted();
    c.check_launch();
}

__global__ void fill_int_kernel(int* p, int count, int v) {
    for (int i = threadIdx.x; i < count; i += blockDim.x) p[i] = v;
}
void launch_fill_int(const Ctx& c, int* p, int count, int value) {
    if (!c.exec || count <= 0) return;
    ProfScope ps(c, "elementwise", 4.0 * count, 0.0);
    fill_int_kernel<<<1, 32, 0, c.stream>>>(p, count, value);
    c.counted();
    c.check_launch();
}

__global__ void qr_info_kernel(int* slot, const int* bad, int bad_value) { *slot = *bad ? bad_value : 0; }
void launch_qr_info(const Ctx& c, int* slot, const int* bad, int bad_value) {
    if (!c.exec) return;
    ProfScope ps(c, "elementwise", 8.0, 0.0);
    qr_info_kernel<<<1, 1, 0, c.stream>>>(slot, bad, bad_value);
    c.counted();
    c.check_launch();
}

__global__ void __launch_bounds__(256) sign_fix_kernel(double* U, int64_t n, double* sign, void* out, tk_dtype odt,
                                                       int64_t ldo) {
    __shared__ double bv[256];
    __shared__ int64_t bi[256];
    const int64_t col = blockIdx.x;
    double* u = U + n * col;
    double best = -1.0;
    int64_t besti = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        double a = fabs(u[i]);
        if (a > best) { best = a; besti = i; }
    }
    bv[threadIdx.x] = best;
    bi[threadIdx.x] = besti;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            double o = bv[threadIdx.x + s];
            int64_t oi = bi[threadIdx.x + s];
            if (o > bv[threadIdx.x] || (o == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
                bv[threadIdx.x] = o;
                bi[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    double sg = u[bi[0]] < 0.0 ? -1.0 : 1.0;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const double v = u[i] * sg;
        u[i] = v;
        if (out) st_any(out, odt, i + ldo * col, v);
    }
    if (threadIdx.x == 0) sign[col] = sg;
}

void launch_sign_fix(const Ctx& c, double* U, int64_t n, int64_t r, double* sign, void* out, tk_dtype odt,
                     int64_t ldo) {
    if (!c.exec || r == 0) return;
    ProfScope ps(c, "elementwise", 16.0 * n * r, 0.0);
    sign_fix_kernel<<<(unsigned)r, 256, 0, c.stream>>>(U, n, sign, out, odt, ldo);
    c.counted();
    c.check_launch();
}

struct SignPtrs {
    const double* s[TK_MAX_D];
    int64_t n[TK_MAX_D];
    int d;
};

__global__ void apply_signs_kernel(double* G, int64_t tot, SignPtrs sp, void* out, tk_dtype odt) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= tot) return;
    int64_t rem = idx;
    double f = 1.0;
    for (int j = 0; j < sp.d; ++j) {
        int64_t ij = rem % sp.n[j];
        rem /= sp.n[j];
        if (sp.s[j]) f *= sp.s[j][ij];  // no sign array: the mode keeps its signs
    }
    const double v = G[idx] * f;
    G[idx] = v;
    if (out) st_any(out, odt, idx, v);
}

void launch_apply_signs(const Ctx& c, double* G, const Tens& shape, double* const* signs, void* out, tk_dtype odt) {
    if (!c.exec) return;
    SignPtrs sp;
    sp.d = shape.d;
    for (int j = 0; j < shape.d; ++j) {
        sp.s[j] = signs[j];
        sp.n[j] = shape.n[j];
    }
    int64_t tot = shape.numel();
    if (tot == 0) return;
    ProfScope ps(c, "elementwise", 16.0 * tot, (double)tot * shape.d);
    apply_signs_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, c.stream>>>(G, tot, sp, out, odt);
    c.counted();
    c.check_launch();
}

// partial sums of (x - y)^2 and x^2; FP32 runs of 32 elements folded into FP64.
template <typename Tx, typename Ty>
__global__ void __launch_bounds__(256) residual_partial_kernel(const Tx* X, const Ty* Y, int64_t tot, float xinv,
                                                               double* part) {
    __shared__ double red[33];
    double sr = 0.0, sx = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    while (i < tot) {
        float fr = 0.f, fx = 0.f;
        double dr = 0.0, dx = 0.0;
        for (int t = 0; t < 32 && i < tot; ++t, i += stride) {
            if constexpr (sizeof(Tx) == 8) {
                double x = (double)X[i], y = (double)Y[i];
                dr += (x - y) * (x - y);
                dx += x * x;
            } else {
                float x = ldx(X, i, xinv), y = (float)Y[i];
                float dd = x - y;
                fr = fmaf(dd, dd, fr);
                fx = fmaf(x, x, fx);
            }
        }
        sr += dr + (double)fr;
        sx += dx + (double)fx;
    }
    sr = block_sum(sr, red);
    sx = block_sum(sx, red);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sr;
        part[2 * blockIdx.x + 1] = sx;
    }
}

// Sum of nb (a, b) pairs: fixed strided per-thread sums, then warp and block
// trees in a fixed order (deterministic for a given nb).
__global__ void __launch_bounds__(256) residual_final_kernel(const double* part, int nb, double* out2) {
    __shared__ double sa[8], sb[8];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        a += part[2 * i];
        b += part[2 * i + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sa[w] = a;
        sb[w] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ta = 0.0, tb = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
            ta += sa[i];
            tb += sb[i];
        }
        out2[0] = ta;
        out2[1] = tb;
    }
}

void launch_sum_pairs(const Ctx& c, const double* part, int nb, double* out2) {
    if (!c.exec) return;
    ProfScope ps(c, "elementwise", 16.0 * nb, 2.0 * nb);
    residual_final_kernel<<<1, 256, 0, c.stream>>>(part, nb, out2);
    c.counted();
    c.check_launch();
}

void launch_residual_norms(Ctx& c, const Tens& X, const void* Y, tk_dtype ydt, double* out2) {
    const int nb = 152 * 8;
    double* part = c.alloc<double>(2 * nb);
    if (!c.exec) return;
    int64_t tot = X.numel();
    float inv = X.dt == TK_FP8_E4M3 ? 1.f / X.scale : 1.f;
    ProfScope ps(c, "residual", (double)tot * (dtype_size(X.dt) + dtype_size(ydt)), 4.0 * tot);
    if (X.dt == TK_F64) {
        TK_REQUIRE(ydt == TK_F64, TK_ERR_DTYPE, "residual: F64 data needs F64 reconstruction");
        residual_partial_kernel<double, double><<<nb, 256, 0, c.stream>>>((const double*)X.p, (const double*)Y, tot,
                                                                          1.f, part);
    } else {
        TK_REQUIRE(ydt == TK_F32, TK_ERR_DTYPE, "residual: reconstruction must be F32");
        switch (X.dt) {
            case TK_F32:
                residual_partial_kernel<float, float><<<nb, 256, 0, c.stream>>>((const float*)X.p, (const float*)Y,
                                                                                tot, inv, part);
                break;
            case TK_BF16:
                residual_partial_kernel<__nv_bfloat16, float><<<nb, 256, 0, c.stream>>>(
                    (const __nv_bfloat16*)X.p, (const float*)Y, tot, inv, part);
                break;
            default:
                residual_partial_kernel<__nv_fp8_e4m3, float><<<nb, 256, 0, c.stream>>>(
                    (const __nv_fp8_e4m3*)X.p, (const float*)Y, tot, inv, part);
                break;
        }
    }
    c.counted();
    c.check_launch();
    residual_final_kernel<<<1, 32, 0, c.stream>>>(part, nb, out2);
    c.counted();
    c.check_launch();
}

__global__ void axpby_residual_kernel(const void* X, tk_dtype xdt, float xinv, const void* Y, tk_dtype ydt,
                                      int64_t tot, double alpha, void* dst, tk_dtype ddt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= tot) return;
    if (xdt == TK_F64 || ydt == TK_F64) {  // difference formed in FP64 when either side carries it
        st_any(dst, ddt, i, alpha * (ld_any(X, xdt, i, xinv) - ld_any(Y, ydt, i)));
    } else {
        float x = (float)ld_any(X, xdt, i, xinv), y = (float)ld_any(Y, ydt, i);
        st_any(dst, ddt, i, (double)((float)alpha * (x - y)));
    }
}

void launch_axpby_residual(const Ctx& c, const Tens& X, const void* Y, tk_dtype ydt, double alpha, void* dst,
                           tk_dtype ddt) {
    if (!c.exec) return;
    int64_t tot = X.numel();
    if (tot == 0) return;
    float inv = X.dt == TK_FP8_E4M3 ? 1.f / X.scale : 1.f;
    ProfScope ps(c, "residual", (double)tot * (dtype_size(X.dt) + dtype_size(ydt) + dtype_size(ddt)), 2.0 * tot);
    axpby_residual_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, c.stream>>>(X.p, X.dt, inv, Y, ydt, tot, alpha, dst,
                                                                                ddt);
    c.counted();
    c.check_launch();
}

__global__ void scale_copy_kernel(const void* src, tk_dtype sdt, int64_t n, double alpha, void* dst, tk_dtype ddt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    st_any(dst, ddt, i, alpha * ld_any(src, sdt, i));
}

void launch_scale_copy(const Ctx& c, const void* src, tk_dtype sdt, int64_t n, double alpha, void* dst,
                       tk_dtype ddt) {
    if (!c.exec || n == 0) return;
    ProfScope ps(c, "elementwise", (double)n * (dtype_size(sdt) + dtype_size(ddt)), (double)n);
    scale_copy_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c.stream>>>(src, sdt, n, alpha, dst, ddt);
    c.counted();
    c.check_launch();
}

}  // namespace tk
