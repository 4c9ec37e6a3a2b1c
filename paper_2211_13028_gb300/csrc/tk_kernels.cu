// SIMT kernels of libtucker: generic mode-j TTM, FP64 small dense linear
// algebra (Gram / GEMM, Cholesky + triangular inverse, Householder QR, Jacobi
// eigensolver) and element-wise helpers.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <math.h>

#include "tk_internal.cuh"

namespace tk {

void Ctx::check_launch() const {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) fail(TK_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
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

template <typename Tx, typename Ta>
static void ttm_dispatch(const Ctx& c, const Tx* X, int64_t L, int64_t nj, int64_t R, const Ta* M, int64_t ldm,
                         bool mtrans, int64_t m, Ta* out, Ta xinv) {
    int64_t rows = L * R;
    if (rows * m <= (1 << 21) && nj <= 512) {
        const char* name = (const void*)X == c.xdata ? "ttm_x" : "ttm";
        ProfScope ps(c, name, (double)rows * nj * sizeof(Tx) + (double)rows * m * sizeof(Ta), 2.0 * rows * nj * m);
        ttm_direct_kernel<Tx, Ta><<<(unsigned)((rows * m + 255) / 256), 256, 0, c.stream>>>(X, L, nj, R, M, ldm,
                                                                                           mtrans, m, out, xinv);
        c.counted();
        c.check_launch();
        return;
    }
    const char* name = (const void*)X == c.xdata ? "ttm_x" : (rows * m == c.xnumel ? "ttm_full" : "ttm");
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

// ------------------------------------------------------------------ FP64 GEMM (NT) with split-K

__global__ void __launch_bounds__(256) gemm_nt_partial_kernel(int64_t m, int64_t n, int64_t K, int64_t kchunk,
                                                              View2 A, View2 B, double* P, const int* skip) {
    if (skip && *skip) return;
    __shared__ double As[16][33];
    __shared__ double Bs[16][33];
    const int tid = threadIdx.x;
    const int tx = tid % 16, ty = tid / 16;
    const int64_t a0 = (int64_t)blockIdx.x * 32, b0 = (int64_t)blockIdx.y * 32;
    const int64_t kb = (int64_t)blockIdx.z * kchunk;
    const int64_t ke = min(K, kb + kchunk);
    double acc[2][2] = {{0, 0}, {0, 0}};
    // each thread loads rows rr0, rr0 + 16 at column offset kk (fixed): precompute row offsets
    const int kk = tid % 16, rr0 = tid / 16;
    int64_t oa[2], ob[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        int64_t ra = a0 + rr0 + 16 * q, rb = b0 + rr0 + 16 * q;
        oa[q] = ra < m ? ((A.A1 == INT64_MAX) ? ra * A.sa1 : (ra % A.A1) * A.sa1 + (ra / A.A1) * A.sa2) : -1;
        ob[q] = rb < n ? ((B.A1 == INT64_MAX) ? rb * B.sa1 : (rb % B.A1) * B.sa1 + (rb / B.A1) * B.sa2) : -1;
    }
    for (int64_t k0 = kb; k0 < ke; k0 += 16) {
        int64_t k = k0 + kk;
        int64_t ta = -1, tb = -1;
        if (k < ke) {
            ta = (A.T1 == INT64_MAX) ? k * A.st1 : (k % A.T1) * A.st1 + (k / A.T1) * A.st2;
            tb = (B.T1 == INT64_MAX) ? k * B.st1 : (k % B.T1) * B.st1 + (k / B.T1) * B.st2;
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            double va = 0.0, vb = 0.0;
            if (ta >= 0 && oa[q] >= 0) {
                int64_t o = oa[q] + ta;
                va = A.dt == TK_F64 ? static_cast<const double*>(A.p)[o] : (double)static_cast<const float*>(A.p)[o];
            }
            if (tb >= 0 && ob[q] >= 0) {
                int64_t o = ob[q] + tb;
                vb = B.dt == TK_F64 ? static_cast<const double*>(B.p)[o] : (double)static_cast<const float*>(B.p)[o];
            }
            As[kk][rr0 + 16 * q] = va;
            Bs[kk][rr0 + 16 * q] = vb;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double av[2] = {As[kk][tx], As[kk][tx + 16]};
            double bv[2] = {Bs[kk][ty], Bs[kk][ty + 16]};
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
    double* Pz = P + (int64_t)blockIdx.z * m * n;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            int64_t a = a0 + tx + 16 * i, b = b0 + ty + 16 * j;
            if (a < m && b < n) Pz[a + m * b] = acc[i][j];
        }
}

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

// Small outputs: one warp per output element, the K terms split over the lanes
// (a short dependent chain per lane) and combined by shuffles.
struct V2Lane {  // walk t = lane, lane + 32, ... of row a of a View2
    const View2& v;
    int64_t base, lo, hi;
    __device__ V2Lane(const View2& vv, int64_t a, int64_t t0) : v(vv) {
        base = (v.A1 == INT64_MAX) ? a * v.sa1 : (a % v.A1) * v.sa1 + (a / v.A1) * v.sa2;
        if (v.T1 == INT64_MAX) {
            lo = t0;
            hi = 0;
        } else {
            lo = t0 % v.T1;
            hi = t0 / v.T1;
        }
    }
    __device__ __forceinline__ double load() const {
        int64_t o = base + lo * v.st1 + hi * v.st2;
        return v.dt == TK_F64 ? static_cast<const double*>(v.p)[o] : (double)static_cast<const float*>(v.p)[o];
    }
    __device__ __forceinline__ void next32() {
        lo += 32;
        if (v.T1 != INT64_MAX && lo >= v.T1) {
            hi += lo / v.T1;
            lo %= v.T1;
        }
    }
};

__global__ void __launch_bounds__(256) gemm_nt_warp_kernel(int64_t m, int64_t n, int64_t K, View2 A, View2 B,
                                                           double alpha, double beta, double* C, int64_t ldc,
                                                           const int* skip) {
    if (skip && *skip) return;
    const int lane = threadIdx.x & 31;
    const int64_t o = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (o >= m * n) return;
    const int64_t a = o % m, b = o / m;
    double s = 0.0;
    if (lane < K) {
        V2Lane wa(A, a, lane), wb(B, b, lane);
        for (int64_t t = lane; t < K; t += 32) {
            s = fma(wa.load(), wb.load(), s);
            wa.next32();
            wb.next32();
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) {
        double* dst = C + a + ldc * b;
        *dst = beta == 0.0 ? alpha * s : alpha * s + beta * *dst;
    }
}

void gemm_nt_f64(Ctx& c, int64_t m, int64_t n, int64_t K, const View2& A, const View2& B, double alpha, double beta,
                 double* C, int64_t ldc, const int* skip) {
    if (m * n <= (1 << 17) && K > 0) {
        if (!c.exec || m == 0 || n == 0) return;
        ProfScope ps(c, "gemm_f64", 8.0 * (double)(m + n) * K + 8.0 * m * n, 2.0 * m * n * K);
        gemm_nt_warp_kernel<<<(unsigned)((m * n + 7) / 8), 256, 0, c.stream>>>(m, n, K, A, B, alpha, beta, C, ldc,
                                                                                skip);
        c.counted();
        c.check_launch();
        return;
    }
    int64_t tiles = ((m + 31) / 32) * ((n + 31) / 32);
    int64_t nsplit = (304 + tiles - 1) / tiles;
    int64_t maxsplit = (K + 63) / 64;
    if (nsplit > maxsplit) nsplit = maxsplit;
    if (nsplit < 1) nsplit = 1;
    if (nsplit > 1024) nsplit = 1024;
    int64_t kchunk = (K + nsplit - 1) / nsplit;
    kchunk = (kchunk + 15) / 16 * 16;
    nsplit = K > 0 ? (K + kchunk - 1) / kchunk : 1;
    double* P = c.alloc<double>(nsplit * m * n);
    if (!c.exec || m == 0 || n == 0) return;
    if (K == 0) {
        cudaMemsetAsync(P, 0, sizeof(double) * m * n, c.stream);
    } else {
        dim3 grid((unsigned)((m + 31) / 32), (unsigned)((n + 31) / 32), (unsigned)nsplit);
        ProfScope ps(c, "gemm_f64", 8.0 * (double)(m + n) * K + 8.0 * m * n * nsplit, 2.0 * m * n * K);
        gemm_nt_partial_kernel<<<grid, 256, 0, c.stream>>>(m, n, K, kchunk, A, B, P, skip);
        c.counted();
        c.check_launch();
    }
    int64_t tot = m * n;
    ProfScope ps(c, "gemm_f64", 8.0 * m * n * (nsplit + 1), (double)m * n * nsplit);
    gemm_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, c.stream>>>(m, n, (int)nsplit, P, alpha, beta, C,
                                                                              ldc, skip);
    c.counted();
    c.check_launch();
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

__global__ void __launch_bounds__(512) chol_inv_kernel(KDims kd, int kmax, const double* W, double* Rinv, int* bad,
                                                       double tol) {
    extern __shared__ double A[];  // k x k, A(i, l) = A[i + k*l]
    __shared__ double dg[256];
    __shared__ int s_bad;
    const int b = blockIdx.x;
    if (bad[b]) return;
    const int k = kd.k[b];
    const double* Wb = W + (int64_t)b * kmax * kmax;
    double* Rb = Rinv + (int64_t)b * kmax * kmax;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < k * k; e += nt) {
        int i = e % k, l = e / k;
        A[e] = Wb[i + (int64_t)kmax * l];
    }
    for (int i = tid; i < k; i += nt) dg[i] = Wb[i + (int64_t)kmax * i];
    if (tid == 0) s_bad = 0;
    __syncthreads();
    __shared__ double s_rinv;
    for (int j = 0; j < k; ++j) {
        // one thread takes the FP64 square root and reciprocal (FP64 throughput is scarce)
        if (tid == 0) {
            const double piv = A[j + k * j];
            if (!(piv > tol * dg[j]) || !(piv > 0.0)) {
                s_bad = 1;
            } else {
                const double rjj = sqrt(piv);
                A[j + k * j] = rjj;
                s_rinv = 1.0 / rjj;
            }
        }
        __syncthreads();
        if (s_bad) break;  // uniform
        const double rinv = s_rinv;
        for (int l = j + 1 + tid; l < k; l += nt) A[j + k * l] *= rinv;
        __syncthreads();
        const int w = k - j - 1;
        for (int e = tid; e < w * w; e += nt) {
            const int i = j + 1 + e % w, l = j + 1 + e / w;
            if (i <= l) A[i + k * l] -= A[j + k * i] * A[j + k * l];
        }
        __syncthreads();
    }
    __syncthreads();
    if (s_bad) {
        if (tid == 0) bad[b] = 1;
        return;
    }
    // R^{-1} by back substitution, one warp per column: x_col = 1 / r_cc and
    // x_i = -(sum_{l=i+1..col} r_il x_l) / r_ii, the sum split over the lanes.
    for (int i = tid; i < k; i += nt) dg[i] = 1.0 / A[i + k * i];
    __syncthreads();
    const int lane = tid & 31, nw = nt >> 5;
    for (int col = tid >> 5; col < k; col += nw) {
        double* X = Rb + (int64_t)kmax * col;
        for (int i = col + 1 + lane; i < k; i += 32) X[i] = 0.0;
        if (lane == 0) X[col] = dg[col];
        __syncwarp();
        for (int i = col - 1; i >= 0; --i) {
            double s = 0.0;
            for (int l = i + 1 + lane; l <= col; l += 32) s = fma(A[i + k * l], X[l], s);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (lane == 0) X[i] = -s * dg[i];
            __syncwarp();
        }
    }
}

void launch_chol_inv(const Ctx& c, int batch, const KDims& kd, int kmax, const double* W, double* Rinv, int* bad,
                     double tol) {
    if (!c.exec) return;
    TK_REQUIRE(kmax <= 112, TK_ERR_SHAPE, "chol_inv: at most 112 columns");
    size_t smem = sizeof(double) * kmax * kmax;
    if (smem > 48 * 1024)
        TK_CUDA(cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ProfScope ps(c, "chol_inv", 16.0 * batch * kmax * kmax, (2.0 / 3.0) * batch * kmax * kmax * kmax);
    chol_inv_kernel<<<batch, 512, smem, c.stream>>>(kd, kmax, W, Rinv, bad, tol);
    c.counted();
    c.check_launch();
}

// ------------------------------------------------------------------ Q = Y R^{-1}

__global__ void __launch_bounds__(256) apply_rinv_kernel(int64_t n, int64_t k, View2 Y, const double* Rinv,
                                                         int64_t ldr, double* Q, const int* skip) {
    extern __shared__ double ys[];  // 8 x k
    if (skip && *skip) return;
    const int64_t i0 = (int64_t)blockIdx.x * 8;
    for (int64_t e = threadIdx.x; e < 8 * k; e += blockDim.x) {
        int64_t ii = e % 8, cc = e / 8;
        ys[e] = (i0 + ii < n) ? v2ld(Y, i0 + ii, cc) : 0.0;
    }
    __syncthreads();
    for (int64_t e = threadIdx.x; e < 8 * k; e += blockDim.x) {
        int64_t ii = e % 8, col = e / 8;
        if (i0 + ii >= n) continue;
        double s = 0.0;
        for (int64_t cp = 0; cp <= col; ++cp) s = fma(ys[ii + 8 * cp], Rinv[cp + ldr * col], s);
        Q[(i0 + ii) + n * col] = s;
    }
}

void launch_apply_rinv(const Ctx& c, int64_t n, int64_t k, const View2& Y, const double* Rinv, int64_t ldr, double* Q,
                       const int* skip) {
    if (!c.exec) return;
    size_t smem = sizeof(double) * 8 * k;
    if (smem > 48 * 1024)
        TK_CUDA(cudaFuncSetAttribute(apply_rinv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ProfScope ps(c, "apply_rinv", 16.0 * n * k + 8.0 * k * k, (double)n * k * k);
    apply_rinv_kernel<<<(unsigned)((n + 7) / 8), 256, smem, c.stream>>>(n, k, Y, Rinv, ldr, Q, skip);
    c.counted();
    c.check_launch();
}

// ------------------------------------------------------------------ Householder QR (fallback)

__global__ void __launch_bounds__(256) householder_kernel(int64_t n, int64_t k, double* A, double* Q, double* tau,
                                                          const int* run) {
    __shared__ double red[33];
    __shared__ double v0s[256];
    if (run && !*run) return;
    const int tid = threadIdx.x, nt = blockDim.x;
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

void launch_householder(const Ctx& c, int64_t n, int64_t k, double* A, double* Q, double* tau, const int* run) {
    if (!c.exec) return;
    TK_REQUIRE(k <= 256, TK_ERR_SHAPE, "householder: at most 256 columns");
    ProfScope ps(c, "householder", 16.0 * n * k, 8.0 * n * k * k);
    householder_kernel<<<1, 256, 0, c.stream>>>(n, k, A, Q, tau, run);
    c.counted();
    c.check_launch();
}

// ------------------------------------------------------------------ Jacobi eigensolver

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
    const double athr = 4.0 * eps * sqrt(block_sum(part, red));  // absolute off-diagonal threshold
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
                        double tau = (aqq - app) / (2.0 * apq);
                        double t1 = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + hypot(1.0, tau));
                        c = 1.0 / hypot(1.0, t1);
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
        w[rank] = wi;
        for (int row = 0; row < k; ++row) Vout[row + k * rank] = V[row + k * i];
    }
}

void launch_jacobi(const Ctx& c, int64_t k, double* A, double* w, double* V, int max_sweeps) {
    if (!c.exec) return;
    TK_REQUIRE(k <= 256, TK_ERR_SHAPE, "jacobi: at most 256 rows");
    int use_smem = k <= 112;
    size_t smem = use_smem ? 2 * sizeof(double) * k * k : 0;
    TK_REQUIRE(use_smem, TK_ERR_SHAPE, "jacobi: core mode above 112 needs the global-memory variant");
    if (smem > 48 * 1024)
        TK_CUDA(cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    ProfScope ps(c, "jacobi", 24.0 * k * k, 9.0 * k * k * k * 8);
    jacobi_kernel<<<1, 256, smem, c.stream>>>((int)k, A, w, V, max_sweeps, use_smem, nullptr, c.dflags);
    c.counted();
    c.check_launch();
}

// ------------------------------------------------------------------ mixed-precision Jacobi
// Two-sided cyclic Jacobi on a symmetric matrix held as an FP64 diagonal D and
// an FP32 off-diagonal F (zero diagonal), accumulating the rotations in an
// FP32 matrix J.  Rotation angles use the FP64 diagonal difference; the pair's
// own 2 x 2 block is updated in closed form (a_pp -= t a_pq, a_qq += t a_pq,
// a_pq = 0).  When F is small in absolute terms (a matrix already close to
// diagonal), FP32 storage of F carries FP64-level absolute accuracy.
// Pairs follow a round-robin tournament; each thread rotates whole 2 x 2
// blocks (rows of one pair x columns of another) in one read-modify-write.
// One CTA; F, J and D live in shared memory (k <= 112).

constexpr int JM_THREADS = 512;
constexpr int JM_FB = 4;  // F blocks per thread: half(half+1)/2 <= 1596 for k <= 112
constexpr int JM_JB = 7;  // J blocks per thread: ceil(k/2) * half <= 3136

// TD: type of the diagonal.  float for the first stage (whose result only
// seeds the second), double for the stage that resolves the eigenvalues.
template <typename TD>
__global__ void __launch_bounds__(JM_THREADS) jacobi_mixed_kernel(int k, const double* __restrict__ A, double* Dout,
                                                                  float* Jout, double tol, int max_sweeps,
                                                                  unsigned* flags) {
    extern __shared__ unsigned char smraw[];
    const int ldf = k + 1;  // odd row stride: column walks are bank-conflict free
    TD* D = reinterpret_cast<TD*>(smraw);
    float* F = reinterpret_cast<float*>(reinterpret_cast<double*>(smraw) + k);
    float* J = F + (size_t)k * ldf;
    __shared__ float cs[64], sn[64];
    __shared__ int P[64], Qp[64];
    __shared__ double red[33];
    const int tid = threadIdx.x, nt = blockDim.x;
    double part = 0.0;
    for (int e = tid; e < k * k; e += nt) {
        int i = e % k, j = e / k;
        double v = A[i + (int64_t)k * j];
        part += v * v;
        if (i == j) {
            D[i] = (TD)v;
            F[i * ldf + j] = 0.f;
        } else {
            F[i * ldf + j] = (float)v;
        }
        J[i * ldf + j] = (i == j) ? 1.f : 0.f;
    }
    const double thr = tol * sqrt(block_sum(part, red));
    const float fthr = (float)thr;
    const int kp = k + (k & 1), half = kp / 2, nrp = (k + 1) / 2;
    // per-thread work lists, fixed for the whole solve
    int fb[JM_FB], jb[JM_JB];
    const int nfb = half * (half + 1) / 2;
#pragma unroll
    for (int i = 0; i < JM_FB; ++i) {
        int e = tid + nt * i;
        fb[i] = -1;
        if (e < nfb) {
            int u = (int)((sqrtf(8.f * e + 1.f) - 1.f) * 0.5f);
            while (u * (u + 1) / 2 > e) --u;
            while ((u + 1) * (u + 2) / 2 <= e) ++u;
            int t = e - u * (u + 1) / 2;
            fb[i] = t | (u << 8);
        }
    }
#pragma unroll
    for (int i = 0; i < JM_JB; ++i) {
        int e = tid + nt * i;
        jb[i] = e < nrp * half ? ((e % nrp) | ((e / nrp) << 8)) : -1;
    }
    bool converged = false;
    for (int sweep = 0; sweep <= max_sweeps; ++sweep) {
        int off = 0;
        for (int e = tid; e < k * k; e += nt) {
            int i = e % k, j = e / k;
            if (i < j && fabsf(F[i * ldf + j]) > fthr) off = 1;
        }
        if (!__syncthreads_or(off)) {
            converged = true;
            break;
        }
        if (sweep == max_sweeps) break;
        for (int step = 0; step < kp - 1; ++step) {
            if (tid < half) {
                const int t = tid;
                int p, q;
                if (t == 0) {
                    p = step;
                    q = kp - 1;
                } else {
                    p = step + t;
                    if (p >= kp - 1) p -= kp - 1;
                    q = step - t;
                    if (q < 0) q += kp - 1;
                }
                if (p > q) { int tmp = p; p = q; q = tmp; }
                float c = 1.f, sv = 0.f;
                if (q < k) {
                    float fpq = F[p * ldf + q];
                    if (fabsf(fpq) > fthr) {
                        // rotation angle from the diagonal difference; fast FP32 reciprocals suffice
                        // (the off-diagonal is zeroed explicitly and convergence is measured)
                        float tau = __fdividef((float)(D[q] - D[p]), 2.f * fpq);
                        float tt = __fdividef(tau >= 0.f ? 1.f : -1.f, fabsf(tau) + sqrtf(fmaf(tau, tau, 1.f)));
                        c = rsqrtf(fmaf(tt, tt, 1.f));
                        sv = tt * c;
                        const TD dt = (TD)tt * (TD)fpq;
                        D[p] -= dt;
                        D[q] += dt;
                    }
                } else {
                    q = -1;
                }
                P[t] = p; Qp[t] = q; cs[t] = c; sn[t] = sv;
            }
            __syncthreads();
            // F <- R_t^T F R_u on the 2 x 2 block (pair t rows, pair u columns), t <= u,
            // with the (u, t) block written as its mirror: F stays exactly symmetric.
#pragma unroll
            for (int i = 0; i < JM_FB; ++i) {
                if (fb[i] < 0) continue;
                const int t = fb[i] & 0xff, u = fb[i] >> 8;
                const int p = P[t], q = Qp[t], pp = P[u], qq = Qp[u];
                const float s1 = sn[t], s2 = sn[u];
                if (t == u) {
                    if (q >= 0 && s1 != 0.f) F[p * ldf + q] = F[q * ldf + p] = 0.f;
                    continue;
                }
                if (s1 == 0.f && s2 == 0.f) continue;
                const float c1 = cs[t], c2 = cs[u];
                float a = F[p * ldf + pp];
                float b = qq >= 0 ? F[p * ldf + qq] : 0.f;
                float cc = q >= 0 ? F[q * ldf + pp] : 0.f;
                float dd = (q >= 0 && qq >= 0) ? F[q * ldf + qq] : 0.f;
                float r00 = c1 * a - s1 * cc, r01 = c1 * b - s1 * dd;
                float r10 = s1 * a + c1 * cc, r11 = s1 * b + c1 * dd;
                float v00 = c2 * r00 - s2 * r01, v01 = s2 * r00 + c2 * r01;
                float v10 = c2 * r10 - s2 * r11, v11 = s2 * r10 + c2 * r11;
                F[p * ldf + pp] = v00;
                F[pp * ldf + p] = v00;
                if (qq >= 0) {
                    F[p * ldf + qq] = v01;
                    F[qq * ldf + p] = v01;
                }
                if (q >= 0) {
                    F[q * ldf + pp] = v10;
                    F[pp * ldf + q] = v10;
                    if (qq >= 0) {
                        F[q * ldf + qq] = v11;
                        F[qq * ldf + q] = v11;
                    }
                }
            }
            // J <- J R on 2-row x pair blocks
#pragma unroll
            for (int i = 0; i < JM_JB; ++i) {
                if (jb[i] < 0) continue;
                const int rp = jb[i] & 0xff, t = jb[i] >> 8;
                const int p = P[t], q = Qp[t];
                const float s1 = sn[t];
                if (q < 0 || s1 == 0.f) continue;
                const float c1 = cs[t];
                const int r0 = 2 * rp, r1 = 2 * rp + 1;
                float a = J[r0 * ldf + p], b = J[r0 * ldf + q];
                J[r0 * ldf + p] = c1 * a - s1 * b;
                J[r0 * ldf + q] = s1 * a + c1 * b;
                if (r1 < k) {
                    a = J[r1 * ldf + p];
                    b = J[r1 * ldf + q];
                    J[r1 * ldf + p] = c1 * a - s1 * b;
                    J[r1 * ldf + q] = s1 * a + c1 * b;
                }
            }
            __syncthreads();
        }
    }
    if (!converged && tid == 0) atomicOr(flags, FLAG_NOT_CONVERGED);
    for (int i = tid; i < k; i += nt) Dout[i] = (double)D[i];
    for (int e = tid; e < k * k; e += nt) {
        int i = e % k, j = e / k;
        Jout[i + (int64_t)k * j] = J[i * ldf + j];
    }
}

void launch_jacobi_mixed(const Ctx& c, int64_t k, const double* A, double* D, float* J, double tol, int max_sweeps,
                         bool fp64_diag) {
    if (!c.exec) return;
    TK_REQUIRE(k >= 1 && k <= 112, TK_ERR_SHAPE, "jacobi_mixed: 1 <= k <= 112");
    size_t smem = sizeof(double) * k + 2 * sizeof(float) * k * (k + 1);
    ProfScope ps(c, "jacobi", 8.0 * k * k + 8.0 * k * k, 12.0 * k * k * k * max_sweeps);
    if (fp64_diag) {
        if (smem > 48 * 1024)
            TK_CUDA(cudaFuncSetAttribute(jacobi_mixed_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
        jacobi_mixed_kernel<double><<<1, JM_THREADS, smem, c.stream>>>((int)k, A, D, J, tol, max_sweeps, c.dflags);
    } else {
        if (smem > 48 * 1024)
            TK_CUDA(cudaFuncSetAttribute(jacobi_mixed_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
        jacobi_mixed_kernel<float><<<1, JM_THREADS, smem, c.stream>>>((int)k, A, D, J, tol, max_sweeps, c.dflags);
    }
    c.counted();
    c.check_launch();
}

// Vr[:, rank] = V[:, i] for the r largest D (ties: lower index first).
__global__ void select_top_kernel(int64_t k, int64_t r, const double* D, const double* V, double* Vr) {
    for (int64_t i = blockIdx.x; i < k; i += gridDim.x) {
        double di = D[i];
        int64_t rank = 0;
        for (int64_t j = 0; j < k; ++j) {
            double dj = D[j];
            rank += (dj > di) || (dj == di && j < i);
        }
        if (rank >= r) continue;
        for (int64_t row = threadIdx.x; row < k; row += blockDim.x) Vr[row + k * rank] = V[row + k * i];
    }
}

void launch_select_top(const Ctx& c, int64_t k, int64_t r, const double* D, const double* V, double* Vr) {
    if (!c.exec || k == 0 || r == 0) return;
    ProfScope ps(c, "elementwise", 16.0 * k * r, 0.0);
    select_top_kernel<<<(unsigned)k, 64, 0, c.stream>>>(k, r, D, V, Vr);
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

__global__ void __launch_bounds__(256) sign_fix_kernel(double* U, int64_t n, double* sign) {
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
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) u[i] *= sg;
    if (threadIdx.x == 0) sign[col] = sg;
}

void launch_sign_fix(const Ctx& c, double* U, int64_t n, int64_t r, double* sign) {
    if (!c.exec || r == 0) return;
    ProfScope ps(c, "elementwise", 16.0 * n * r, 0.0);
    sign_fix_kernel<<<(unsigned)r, 256, 0, c.stream>>>(U, n, sign);
    c.counted();
    c.check_launch();
}

struct SignPtrs {
    const double* s[TK_MAX_D];
    int64_t n[TK_MAX_D];
    int d;
};

__global__ void apply_signs_kernel(double* G, int64_t tot, SignPtrs sp) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= tot) return;
    int64_t rem = idx;
    double f = 1.0;
    for (int j = 0; j < sp.d; ++j) {
        int64_t ij = rem % sp.n[j];
        rem /= sp.n[j];
        f *= sp.s[j][ij];
    }
    G[idx] *= f;
}

void launch_apply_signs(const Ctx& c, double* G, const Tens& shape, double* const* signs) {
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
    apply_signs_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, c.stream>>>(G, tot, sp);
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

__global__ void residual_final_kernel(const double* part, int nb, double* out2) {
    if (threadIdx.x != 0) return;
    double a = 0.0, b = 0.0;
    for (int i = 0; i < nb; ++i) {
        a += part[2 * i];
        b += part[2 * i + 1];
    }
    out2[0] = a;
    out2[1] = b;
}

void launch_sum_pairs(const Ctx& c, const double* part, int nb, double* out2) {
    if (!c.exec) return;
    ProfScope ps(c, "elementwise", 16.0 * nb, 2.0 * nb);
    residual_final_kernel<<<1, 32, 0, c.stream>>>(part, nb, out2);
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
