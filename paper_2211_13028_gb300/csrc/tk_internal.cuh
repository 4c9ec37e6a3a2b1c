// Internal declarations shared by the libtucker translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/tucker.h"

namespace tk {

// ------------------------------------------------------------------ errors

struct Error {
    tk_status st;
    std::string msg;
};

[[noreturn]] void fail(tk_status st, const std::string& msg);

#define TK_CUDA(x)                                                                        \
    do {                                                                                  \
        cudaError_t e_ = (x);                                                             \
        if (e_ != cudaSuccess) ::tk::fail(TK_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define TK_REQUIRE(cond, st, msg)            \
    do {                                     \
        if (!(cond)) ::tk::fail((st), (msg)); \
    } while (0)

// device-side condition bits (handle flag word)
enum : unsigned { FLAG_NOT_CONVERGED = 1u, FLAG_TIMEOUT = 2u };

inline size_t dtype_size(tk_dtype t) {
    switch (t) {
        case TK_F64: return 8;
        case TK_F32: return 4;
        case TK_BF16: return 2;
        case TK_FP8_E4M3: return 1;
    }
    return 0;
}

// ------------------------------------------------------------------ views

// Dense column-major tensor.
struct Tens {
    void* p = nullptr;
    tk_dtype dt = TK_F32;
    int d = 0;
    int64_t n[TK_MAX_D] = {0};
    float scale = 1.f;
    int64_t numel() const {
        int64_t s = 1;
        for (int i = 0; i < d; ++i) s *= n[i];
        return s;
    }
    int64_t left(int j) const {  // prod_{k<j} n_k
        int64_t s = 1;
        for (int i = 0; i < j; ++i) s *= n[i];
        return s;
    }
    int64_t right(int j) const {  // prod_{k>j} n_k
        int64_t s = 1;
        for (int i = j + 1; i < d; ++i) s *= n[i];
        return s;
    }
};

// Column-major matrix, element (i, j) at p[i + j*ld].
struct Mat {
    const void* p = nullptr;
    tk_dtype dt = TK_F64;
    int64_t rows = 0, cols = 0, ld = 0;
};

// Strided 2-D view used by the small FP64 kernels: element (a, t) sits at
//   (a % A1)*sa1 + (a / A1)*sa2 + (t % T1)*st1 + (t / T1)*st2.
// It expresses plain column-major matrices, their transposes and tensor
// unfoldings without copies.
struct View2 {
    const void* p = nullptr;
    tk_dtype dt = TK_F64;
    int64_t A1 = INT64_MAX, sa1 = 0, sa2 = 0;
    int64_t T1 = INT64_MAX, st1 = 0, st2 = 0;
};

// (a, t) = (row, col) of a column-major matrix.
inline View2 view_rows(const void* p, tk_dtype dt, int64_t ld) {
    View2 v; v.p = p; v.dt = dt; v.sa1 = 1; v.st1 = ld; return v;
}
// (a, t) = (col, row) of a column-major matrix.
inline View2 view_cols(const void* p, tk_dtype dt, int64_t ld) {
    View2 v; v.p = p; v.dt = dt; v.sa1 = ld; v.st1 = 1; return v;
}
// (a, t) = (row, col) of the mode-j unfolding of a tensor (L, n_j, R).
inline View2 view_unfold_rows(const Tens& T, int j) {
    View2 v; v.p = T.p; v.dt = T.dt;
    int64_t L = T.left(j);
    v.sa1 = L;
    v.T1 = L; v.st1 = 1; v.st2 = L * T.n[j];
    return v;
}
// (a, t) = (col, row) of the mode-j unfolding of a tensor (L, n_j, R).
inline View2 view_unfold_cols(const Tens& T, int j) {
    View2 v; v.p = T.p; v.dt = T.dt;
    int64_t L = T.left(j);
    v.A1 = L; v.sa1 = 1; v.sa2 = L * T.n[j];
    v.st1 = L;
    return v;
}

// ------------------------------------------------------------------ profiler

// Optional per-launch timing: when enabled on the handle, each launcher
// records a CUDA event pair on the launching stream around its kernel and
// tags it with a class name plus the algorithmic bytes and flops of the
// launch.  tk_profile_read() resolves the pairs after a synchronisation.
struct ProfRec {
    const char* name;
    cudaEvent_t a, b;
    double bytes, flops;
    cudaStream_t st;  // the launching stream (the handle's or one of its auxiliary streams)
};
struct Profiler {
    bool on = false;
    std::string only;  // record only classes whose name starts with this ("" = all)
    std::vector<ProfRec> recs;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t get();
};

// ------------------------------------------------------------------ call context

// Bump allocator over the handle's workspace.  Each entry point runs its
// orchestration twice: a planning pass (exec == false) that only sums the
// sizes, then, with the workspace grown to fit, the executing pass.  Both
// passes make the same allocations in the same order.
struct Ctx {
    cudaStream_t stream = nullptr;
    bool exec = false;
    char* base = nullptr;
    size_t used = 0;
    unsigned* dflags = nullptr;  // device condition word
    int* dqr = nullptr;          // device QR method per mode
    int64_t* launches = nullptr;
    int max_sweeps = 40;
    int qr_method = 0;
    int refine = 0;
    Profiler* prof = nullptr;
    const void* xdata = nullptr;   // the caller's data tensor (tags its full passes)
    int64_t xnumel = 0;
    bool use_tc = true;            // tensor-core TTM where eligible
    int grid_sms = 0;              // CTAs of the persistent streaming kernels (0: every SM)
    bool background = false;       // a streaming pass on part of the SMs beside a chain of small kernels
    bool capturing = false;        // the stream is recording a CUDA graph (launches are not run now)
    bool df64 = false;             // FP32-class data: FP64 products may run in double-float arithmetic
    // Factor splits (TF32 hi / lo) made in this pass, reused while split_cache is
    // on: only inside a dimension tree, whose factors are not modified.
    struct Split {
        const void* p;
        int64_t ld, nj, m, npad, rows;
        int dt, mtrans;
        float* hi;
        float* lo;
    };
    std::vector<Split> splits;
    bool split_cache = false;
    // Zeroed arrival counters of the handle for split-K products whose last
    // CTA per tile adds the partial tiles (each use leaves them at zero again);
    // every product of a call takes its own slice, so forked products never
    // share one.  nullptr: the separate reduction kernel is used.
    static constexpr int kCounters = 16384;
    unsigned* ctr = nullptr;
    int ctr_used = 0;
    unsigned* take_counters(int n) {
        if (!ctr || ctr_used + n > kCounters) return nullptr;
        unsigned* p = ctr + ctr_used;
        ctr_used += n;
        return p;
    }
    // Auxiliary streams of the handle: the first kFork for independent
    // per-mode work (fork), the last for a long branch that runs beside the
    // rest of the call (side).
    static constexpr int kFork = 3;
    static constexpr int kAux = kFork + 1;
    cudaStream_t aux[kAux] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[kAux] = {};

    // Runs body(b) for b = 0 .. nb-1, item b on auxiliary stream b mod kAux,
    // each forked from the call's stream by an event and joined back into it
    // before fork returns, so the items overlap one another (latency-bound
    // small kernels) while the call stays one stream-ordered unit (also when
    // it is recorded into a CUDA graph: the fork and join become graph edges).
    // Workspace allocations happen in item order in the planning pass and in
    // the executing pass alike.  Without auxiliary streams, or in the planning
    // pass, the items run in order on the call's stream.
    template <typename F>
    void fork(int nb, F&& body);

    // Runs side_body on the side stream (forked from the call's stream) and
    // then main_body on the call's stream, joining the side stream back
    // before returning: the two overlap, and forks inside main_body never
    // queue behind side_body.  side_body must not fork.  Without auxiliary
    // streams, or in the planning pass, both run in order on the call's stream.
    template <typename M, typename S>
    void side(M&& main_body, S&& side_body);

    template <typename T>
    T* alloc(int64_t count) {
        size_t bytes = (size_t)(count > 0 ? count : 1) * sizeof(T);
        size_t off = (used + 255) & ~(size_t)255;
        used = off + bytes;
        return exec ? reinterpret_cast<T*>(base + off) : reinterpret_cast<T*>((uintptr_t)(off + 256));
    }
    void* alloc_bytes(size_t bytes) { return alloc<char>((int64_t)bytes); }
    void counted(int n = 1) const {
        if (launches) *launches += n;
    }
    void check_launch() const;
};

void ctx_fork_begin(Ctx& c, int used);
void ctx_fork_end(Ctx& c, cudaStream_t main, int used);

template <typename F>
void Ctx::fork(int nb, F&& body) {
    if (!exec || nb <= 1 || !aux[0]) {
        for (int b = 0; b < nb; ++b) body(b);
        return;
    }
    cudaStream_t main = stream;
    const int used = nb < kFork ? nb : kFork;
    ctx_fork_begin(*this, used);
    try {
        for (int b = 0; b < nb; ++b) {
            stream = aux[b % kFork];
            body(b);
        }
    } catch (...) {
        ctx_fork_end(*this, main, used);
        throw;
    }
    ctx_fork_end(*this, main, used);
}

void ctx_side_begin(Ctx& c);
void ctx_side_end(Ctx& c, cudaStream_t main);

template <typename M, typename S>
void Ctx::side(M&& main_body, S&& side_body) {
    if (!exec || !aux[kFork]) {
        side_body();
        main_body();
        return;
    }
    cudaStream_t main = stream;
    ctx_side_begin(*this);  // the side stream waits for the call's stream; the call's stream becomes it
    try {
        side_body();
        stream = main;
        main_body();
    } catch (...) {
        ctx_side_end(*this, main);
        throw;
    }
    ctx_side_end(*this, main);
}

// RAII event pair around one launch (no-op unless profiling is on).
struct ProfScope {
    const Ctx& c;
    ProfRec* rec = nullptr;
    ProfScope(const Ctx& ctx, const char* name, double bytes, double flops);
    ~ProfScope();
};

// ------------------------------------------------------------------ kernel launchers
// Every launcher returns immediately when !c.exec.

// out = X x_j M^T   (out[.., a, ..] = sum_i M(i, a) X[.., i, ..]), M(i, a) = M.p[i + a*ld]
// or, with mtrans, M(i, a) = M.p[a + i*ld].  M must be F64 (F64 data) or F32.
// out is dense column-major, dims of X with n_j -> m, dtype F64 or F32.
void launch_ttm(const Ctx& c, const Tens& X, int j, const Mat& M, bool mtrans, int64_t m, void* out, tk_dtype out_dt);

// Tensor-core (tcgen05, 3xTF32) version of launch_ttm for FP32 data and output,
// m <= 96; ttm_tc_eligible says whether a TTM qualifies (shape, dtype, alignment).
bool ttm_tc_eligible(const Tens& X, int j, int64_t m, tk_dtype out_dt);
// A factor a tensor-core TTM will split (the contracted mode's size nj, output
// width m; residual: the fused-residual blocking).
struct TcSplitReq {
    Mat M;
    bool mtrans;
    int64_t nj, m;
    bool residual;
};
// Makes the splits of several factors in one launch and enters them in the
// call's split cache (which must be on while the TTMs run).
void tc_presplit(Ctx& c, const std::vector<TcSplitReq>& reqs);
void launch_ttm_tc(Ctx& c, const Tens& X, int j, const Mat& M, bool mtrans, int64_t m, float* out);
// BF16 data: tcgen05 kind::f16 with A straight from shared memory and the
// factor split into BF16 hi + lo (FP32 output).
// Rademacher diagonal of the Kronecker-SRHT sketch (tk_rademacher in tucker.h):
// the sign bit (0x80000000 for -1, 0 for +1) of entry c of D_n, with
// u = (uint32)seed + 0x9E3779B9 (n + 1): the MurmurHash3 32-bit finalizer of
// c ^ u, top bit.
__host__ __device__ inline uint32_t tk_rad_key(uint64_t seed, int n) {
    return (uint32_t)seed + 0x9E3779B9u * (uint32_t)(n + 1);
}
__host__ __device__ inline uint32_t tk_rad_bits(uint32_t u, uint32_t c) {
    uint32_t x = c ^ u;
    x ^= x >> 16;
    x *= 0x85EBCA6Bu;
    x ^= x >> 13;
    x *= 0xC2B2AE35u;
    x ^= x >> 16;
    return x & 0x80000000u;
}

// Column index of the mode-n unfolding for the elements a streaming TTM along
// mode j0 (X viewed as L x n_j0 x R) meets: c = C1 (row % P1) + P2 (row / P3)
// + B1 (rr % Q1) + B2 (rr / Q2) + A i for row `row` of the tile layout (l, or
// r when j0 is the leading mode), outer index rr and contracted index i.
struct SignMap {
    uint32_t key = 0;
    int64_t C1 = 0, P1 = 1, P2 = 0, P3 = 1, B1 = 0, Q1 = 1, B2 = 0, Q2 = 1, A = 0;
};
SignMap sign_map(const Tens& X, int n, int j0, uint64_t seed);

// Narrow TTMs (m <= 8 output columns) on large FP32 data: a TMA-fed FP32 FMA
// streaming kernel (the tensor-core kernels' tiling; tk_fma_stream.cu).
bool ttm_narrow_eligible(const Tens& X, int j, int64_t m, tk_dtype out_dt);
// With sm, X's elements are multiplied by the Rademacher signs of SignMap first.
void launch_ttm_narrow(const Ctx& c, const Tens& X, int j, const Mat& M, bool mtrans, int64_t m, float* out,
                       const SignMap* sm = nullptr);
// dst = D_n o X (X's dtype and layout): every element times its SRHT sign.
void launch_sign_copy(const Ctx& c, const Tens& X, int n, uint64_t seed, void* dst);

// Philox4x32-10 blocks offset .. offset + nblocks - 1 of stream `stream`
// (4 uint32 each, out 16-byte aligned); Gaussian factor draws into m.
void launch_philox_blocks(const Ctx& c, unsigned long long seed, unsigned stream, unsigned long long offset,
                          int64_t nblocks, unsigned* out);
void launch_gaussian_factors(const Ctx& c, unsigned long long seed, int count, const unsigned* streams,
                             const Mat* m);
// FP8 (E4M3) data, contraction over the contiguous mode only (L == 1: X is a
// K-major operand): tcgen05 kind::f8f6f4 with X straight from shared memory and
// the factor split into four power-of-two-scaled E4M3 pieces (FP32 output).
bool ttm_fp8_eligible(const Tens& X, int j, int64_t m, tk_dtype out_dt);
void launch_ttm_fp8(Ctx& c, const Tens& X, int j, const Mat& M, bool mtrans, int64_t m, float* out);
bool ttm_bf16_eligible(const Tens& X, int j, int64_t m, tk_dtype out_dt);
void launch_ttm_bf16(Ctx& c, const Tens& X, int j, const Mat& M, bool mtrans, int64_t m, float* out);
// Fused last step of a reconstruction: P = W x_j M^T is formed tile by tile and
// compared with xref (P's dims, F32): per-CTA partial sums of (xref - P)^2 and
// xref^2 go to partials[2 * cta]; with dx != NULL also dx = alpha * (xref - P).
// P itself is never stored.  tc_num_ctas gives the number of partial pairs.
// xref (F32, BF16, or FP8 for the norms only) is read as stored value * xr_scale.
void launch_ttm_tc_residual(Ctx& c, const Tens& W, int j, const Mat& M, bool mtrans, int64_t m, const void* xref,
                            tk_dtype xrdt, void* dx, float alpha, double* partials, float xr_scale = 1.f);
int tc_num_ctas(const Ctx& c, const Tens& X, int j, int64_t m, bool residual);
bool ttm_tc_residual_eligible(const Tens& W, int j, int64_t m);
// One warp waits with the tcgen05 kernels' bounded wait on an mbarrier that
// nothing arrives at (limit_ns), which raises FLAG_TIMEOUT; *waited (device)
// receives how long it waited in ns (-1 had the wait completed).
void launch_wait_selftest(const Ctx& c, uint64_t limit_ns, long long* waited);
// out2 = {sum part[2i], sum part[2i+1]} over nb pairs
void launch_sum_pairs(const Ctx& c, const double* part, int nb, double* out2);

// C = alpha * sum_t A(a, t) B(b, t) + beta * C, FP64, C column-major m x n (ldc).
// A, B: View2 of F64 or F32 data.  Uses split-K partials in the workspace.
// When skip is given and *skip != 0 the kernels return without work.  With
// df_ok and both operands F32, products are accumulated as double-float pairs
// on the FP32 pipe (~48 significant bits) instead of in FP64.
void gemm_nt_f64(Ctx& c, int64_t m, int64_t n, int64_t K, const View2& A, const View2& B, double alpha,
                 double beta, double* C, int64_t ldc, const int* skip = nullptr, bool df_ok = false);

struct KDims {
    int k[TK_MAX_D];
};

// Batched Cholesky W = R^T R and R^{-1} (one CTA per matrix).  W: batch
// matrices k_b x k_b (ld = kmax, stride kmax*kmax), FP64.  Rinv receives
// R^{-1} (upper), FP64.  Matrix b is skipped when bad[b] != 0; a breakdown
// (pivot <= tol * original diagonal) sets bad[b] = 1.  df: the factorisation
// runs in double-float arithmetic (~48 bits) instead of FP64.
void launch_chol_inv(const Ctx& c, int batch, const KDims& kd, int kmax, const double* W, double* Rinv, int* bad,
                     double tol, bool df = false);

// Q(i, c) = sum_{c' <= c} Y(i, c') Rinv(c', c), FP64 out (n x k, ld n).  Skipped when *skip != 0.
void launch_apply_rinv(const Ctx& c, int64_t n, int64_t k, const View2& Y, const double* Rinv, int64_t ldr,
                       double* Q, const int* skip);

// Q_b = Y_b R_b^{-1} for batch matrices in one launch, in double-float
// arithmetic (Y_b FP32 or FP64, n_b x k_b; R_b = Rinv + b kmax^2, ld kmax;
// Q_b FP64, ld n_b).  Matrix b is skipped when bad[b] != 0.
void launch_apply_rinv_df(const Ctx& c, int batch, const View2* Y, const int64_t* n, const int64_t* k,
                          const double* Rinv, int64_t kmax, double* const* Q, const int* bad);

// Householder thin QR of Y (View2, n x k; copied to FP64 scratch A, ld n) producing Q with
// R_ii >= 0, run only when *run != 0 (run may be NULL = always).  One CTA.  tau: k doubles
// scratch.  When slot is given, *slot = slot_value if the QR runs, else 0 (the QR method a
// matrix of a batch took).
void launch_householder(const Ctx& c, int64_t n, int64_t k, const View2& Y, double* A, double* Q, double* tau,
                        const int* run, int* slot = nullptr, int slot_value = 1);

// Jacobi eigensolver (one CTA per matrix): A (k x k FP64 symmetric, destroyed),
// eigenvalues descending in w, eigenvectors as columns of V (ld k).  k <= 112
// works in shared memory; 112 < k <= 256 in global memory, with gV (k x k
// doubles of scratch) required.
void launch_jacobi(const Ctx& c, int64_t k, double* A, double* w, double* V, int max_sweeps, double* gV = nullptr);

// Mixed-precision Jacobi (FP64 diagonal, FP32 off-diagonal and rotations) on the
// symmetric k x k FP64 matrix A (ld k): eigenvalue estimates in D (unsorted),
// accumulated rotations in J (FP32, k x k, ld k; may be NULL) and, when
// non-NULL, as FP64 copies in J64a and J64b.  Converged when every
// off-diagonal |a_pq| <= tol * ||A||_F (fp64_diag: the resolving stage) or
// |a_pq| <= max(tol sqrt(|a_pp a_qq|), 1e-13 ||A||_F) (otherwise: the seeding
// stage); otherwise FLAG_NOT_CONVERGED is raised.
void launch_jacobi_mixed(Ctx& c, int64_t k, const double* A, double* D, float* J, double* J64a, double* J64b,
                         double tol, int max_sweeps, bool fp64_diag, const double* V1 = nullptr, int64_t r = 0,
                         double* Vt = nullptr, double* Vr = nullptr);
// (With V1: the rotations are replayed on the rows of V1, giving V = V1 J
// without forming J, and the columns of V of the r largest eigenvalue
// estimates, in descending order, go to Vt and Vr (k x r, ld k).)
// Vr (k x r, ld k) = the columns of V (k x k) for the r largest entries of D, in descending order.
void launch_select_top(const Ctx& c, int64_t k, int64_t r, const double* D, const double* V, double* Vr,
                       double* Vr2 = nullptr);

// Thin QR of the plain matrix y (rows x cols) into q (rows x min(rows, cols)):
// CholeskyQR2 with the Householder fallback, identity when cols >= rows; the
// method used goes to c.dqr[0].  All scratch comes from c.alloc.
void orth_matrix(Ctx& c, const Mat& y, const Mat& q);
Mat mat_in(const tk_matrix* m, const char* name);

// Element-wise helpers.
void launch_convert(const Ctx& c, const void* src, tk_dtype sdt, int64_t rows, int64_t cols, int64_t lds,
                    void* dst, tk_dtype ddt, int64_t ldd, float src_scale);
void launch_fill_identity(const Ctx& c, double* Q, int64_t n);
// A (n x k, FP64, ld n) = Y; only when *run != 0 (run may be NULL = always).
void launch_copy_unfold_to_matrix(const Ctx& c, const View2& Y, int64_t n, int64_t k, double* A,
                                  const int* run = nullptr);
void launch_fill_int(const Ctx& c, int* p, int count, int value);
// *slot = *bad ? bad_value : 0
void launch_qr_info(const Ctx& c, int* slot, const int* bad, int bad_value);
// Sign gauge: for each column of U (n x r, F64, ld n) make the largest-|.|
// entry positive; sign[c] = +-1.
// out (may be NULL): the signed U also stored there in odt (ld ldo).
void launch_sign_fix(const Ctx& c, double* U, int64_t n, int64_t r, double* sign, void* out = nullptr,
                     tk_dtype odt = TK_F64, int64_t ldo = 0);
// G (a tensor of the given shape, FP64) times the product of the modes' signs
// (a NULL sign array leaves its mode alone); out (may be NULL): also stored
// there in odt, dense.
void launch_apply_signs(const Ctx& c, double* G, const Tens& shape, double* const* signs_dev, void* out = nullptr,
                        tk_dtype odt = TK_F64);
// partial sums of (X - Y)^2 and X^2 over a tensor, reduced into out[0..1] (FP64).
void launch_residual_norms(Ctx& c, const Tens& X, const void* Y, tk_dtype ydt, double* out2);
// dst = alpha * (X - Y) elementwise (dst dtype = X dtype or F32/F64)
void launch_axpby_residual(const Ctx& c, const Tens& X, const void* Y, tk_dtype ydt, double alpha, void* dst,
                           tk_dtype ddt);
void launch_scale_copy(const Ctx& c, const void* src, tk_dtype sdt, int64_t n, double alpha, void* dst,
                       tk_dtype ddt);

}  // namespace tk

// ------------------------------------------------------------------ handle
struct tk_handle {
    cudaStream_t stream = nullptr;
    int device = 0;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    unsigned* dflags = nullptr;
    int* dqr = nullptr;
    std::string last_error;
    int64_t launches = 0;
    tk::Profiler prof;
    bool use_tc = true;  // TUCKER_TTM=simt selects the SIMT TTM kernels instead
    int sm_reserve = 0;  // SMs the persistent streaming kernels leave free (tk_set_sm_reserve)
    // pinned ring for host scalar outputs delivered by stream-ordered callbacks
    static constexpr int kHostSlots = 64;
    struct HostSlot {
        double vals[2];
        double* dst;
        int mode;              // 0: sqrt(a / b) (relative error), 1: a (squared norm)
        volatile int pending;  // set when queued, cleared by the host callback
        int reserved;          // recorded into a CUDA graph: delivered at every replay, never reused
    };
    HostSlot* slots = nullptr;
    int next_slot = 0;
    // CUDA graph recording: the workspace block a graph recorded must outlive it,
    // so a block that was in use while recording is retired, not freed, when
    // the workspace grows (freed by tk_graph_release or tk_destroy)
    bool ws_held = false;
    std::vector<char*> retired;
    unsigned* ctr = nullptr;  // Ctx::kCounters zeroed split-K arrival counters
    // auxiliary streams and fork / join events (Ctx::fork)
    cudaStream_t aux[tk::Ctx::kAux] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[tk::Ctx::kAux] = {};
};
