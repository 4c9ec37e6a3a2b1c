// Gaussian sketch factors drawn on the device (the draw lines of Algorithms
// rHKron-re and rSTHKron: Phi_j with i.i.d. N(0, 1) entries), from the
// counter-based generator Philox4x32-10 (Salmon, Moraes, Dror and Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11).  Each element is a
// pure function of (seed, stream, index), so a factor of any size is drawn in
// one launch with no generator state, and the same draws can be reproduced
// anywhere from the published definition.
//
// Block i of stream s under seed S: counter (i mod 2^32, i div 2^32, s, 0),
// key (S mod 2^32, S div 2^32).  A factor matrix (column-major, element e =
// row + rows * col) takes output e mod 4 of block e div 4; a block (x0, x1,
// x2, x3) gives two Box-Muller pairs, u = (x0 + 1) 2^-32 in (0, 1], t = x1
// 2^-32, r = sqrt(-2 ln u), (r cos 2 pi t, r sin 2 pi t), and likewise from
// (x2, x3).  The transform is evaluated in FP64 and rounded once to the
// factor's dtype.
#include "tk_internal.cuh"

#include <cuda_bf16.h>

namespace tk {

constexpr int GF_MAX = 64;  // factors per launch

// One Philox4x32 round per iteration: words 0 and 2 multiplied by the round
// constants, their high halves xored with the other words and the key; the
// key advances by the Weyl increments before every round but the first.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int rnd = 0; rnd < 10; ++rnd) {
        if (rnd > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const unsigned lo2 = 0xCD9E8D57u * c.z, hi2 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi2 ^ c.y ^ k.x, lo2, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ uint4 philox_block(unsigned long long seed, unsigned stream, unsigned long long i) {
    return philox4x32_10(make_uint4((unsigned)i, (unsigned)(i >> 32), stream, 0u),
                         make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
}

__global__ void philox_blocks_kernel(unsigned long long seed, unsigned stream, unsigned long long offset,
                                     int64_t nblocks, uint4* out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nblocks; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = philox_block(seed, stream, offset + (unsigned long long)i);
}

__device__ __forceinline__ void gf_store(void* p, tk_dtype dt, int64_t o, double v) {
    if (dt == TK_F64)
        static_cast<double*>(p)[o] = v;
    else if (dt == TK_F32)
        static_cast<float*>(p)[o] = __double2float_rn(v);
    else
        static_cast<__nv_bfloat16*>(p)[o] = __double2bfloat16(v);
}

// One thread per block of four outputs; blockIdx.y selects the factor.
struct GfBatch {
    int64_t rows[GF_MAX], cols[GF_MAX], ld[GF_MAX];
    void* out[GF_MAX];
    unsigned stream[GF_MAX];
    tk_dtype dt[GF_MAX];
};

__global__ void gaussian_factor_kernel(unsigned long long seed, GfBatch gb) {
    const int f = blockIdx.y;
    const int64_t rows = gb.rows[f], cols = gb.cols[f], ld = gb.ld[f];
    const unsigned stream = gb.stream[f];
    const tk_dtype dt = gb.dt[f];
    void* out = gb.out[f];
    const int64_t n = rows * cols, nb = (n + 3) / 4;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
        const uint4 x = philox_block(seed, stream, (unsigned long long)b);
        double z[4];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const unsigned xu = a ? x.z : x.x, xt = a ? x.w : x.y;
            const double u = ((double)xu + 1.0) * 0x1p-32;
            const double r = sqrt(-2.0 * log(u));
            double sn, cs;
            sincospi((double)xt * 0x1p-31, &sn, &cs);  // angle 2 pi t, t = xt 2^-32
            z[2 * a] = r * cs;
            z[2 * a + 1] = r * sn;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t e = 4 * b + q;
            if (e < n) gf_store(out, dt, e % rows + ld * (e / rows), z[q]);
        }
    }
}

void launch_philox_blocks(const Ctx& c, unsigned long long seed, unsigned stream, unsigned long long offset,
                          int64_t nblocks, unsigned* out) {
    if (!c.exec || nblocks == 0) return;
    const unsigned grid = (unsigned)std::min<int64_t>((nblocks + 255) / 256, 152 * 8);
    ProfScope ps(c, "rng", 16.0 * nblocks, 0.0);
    philox_blocks_kernel<<<grid, 256, 0, c.stream>>>(seed, stream, offset, nblocks, reinterpret_cast<uint4*>(out));
    c.counted();
    c.check_launch();
}

void launch_gaussian_factors(const Ctx& c, unsigned long long seed, int count, const unsigned* streams,
                             const Mat* m) {
    if (!c.exec || count == 0) return;
    TK_REQUIRE(count <= GF_MAX, TK_ERR_ARG, "gaussian factors: at most 64 per launch");
    GfBatch gb;
    int64_t nbmax = 0;
    double bytes = 0.0;
    for (int f = 0; f < count; ++f) {
        gb.rows[f] = m[f].rows;
        gb.cols[f] = m[f].cols;
        gb.ld[f] = m[f].ld;
        gb.out[f] = const_cast<void*>(m[f].p);
        gb.stream[f] = streams[f];
        gb.dt[f] = m[f].dt;
        nbmax = std::max(nbmax, (m[f].rows * m[f].cols + 3) / 4);
        bytes += (double)dtype_size(m[f].dt) * m[f].rows * m[f].cols;
    }
    if (nbmax == 0) return;
    const unsigned gx = (unsigned)std::min<int64_t>((nbmax + 127) / 128, 152 * 8);
    ProfScope ps(c, "rng", bytes, 0.0);
    gaussian_factor_kernel<<<dim3(gx, (unsigned)count), 128, 0, c.stream>>>(seed, gb);
    c.counted();
    c.check_launch();
}

}  // namespace tk
