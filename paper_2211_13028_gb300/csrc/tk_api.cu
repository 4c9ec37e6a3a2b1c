// C-ABI entry points of libtucker and the host-side orchestration of
// Algorithms rHKron-re and rSTHKron (arXiv 2211.13028, Sections 4.2-4.3).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <numeric>

#include "tk_internal.cuh"
#include "tk_tc_common.cuh"

namespace tk {

[[noreturn]] void fail(tk_status st, const std::string& msg) { throw Error{st, msg}; }

cudaEvent_t Profiler::get() {
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    TK_CUDA(cudaEventCreate(&e));
    return e;
}

ProfScope::ProfScope(const Ctx& ctx, const char* name, double bytes, double flops) : c(ctx) {
    if (!c.exec || c.capturing || !c.prof || !c.prof->on) return;
    if (!c.prof->only.empty() && strncmp(name, c.prof->only.c_str(), c.prof->only.size()) != 0) return;
    ProfRec r{name, c.prof->get(), c.prof->get(), bytes, flops, c.stream};
    TK_CUDA(cudaEventRecord(r.a, c.stream));
    c.prof->recs.push_back(r);
    rec = &c.prof->recs.back();
}

ProfScope::~ProfScope() {
    if (rec) cudaEventRecord(c.prof->recs.back().b, c.stream);
}

// ------------------------------------------------------------------ validation

static Tens tens_in(const tk_tensor* t, const char* name, bool allow_empty = true) {
    TK_REQUIRE(t != nullptr, TK_ERR_ARG, std::string(name) + ": null tensor");
    TK_REQUIRE(t->d >= 1 && t->d <= TK_MAX_D, TK_ERR_SHAPE, std::string(name) + ": d out of range");
    TK_REQUIRE(t->dtype >= TK_F64 && t->dtype <= TK_FP8_E4M3, TK_ERR_DTYPE, std::string(name) + ": bad dtype");
    Tens T;
    T.p = t->data;
    T.dt = t->dtype;
    T.d = t->d;
    T.scale = t->scale;
    for (int i = 0; i < t->d; ++i) {
        TK_REQUIRE(t->dims[i] >= 0, TK_ERR_SHAPE, std::string(name) + ": negative dimension");
        TK_REQUIRE(allow_empty || t->dims[i] > 0, TK_ERR_SHAPE, std::string(name) + ": empty dimension");
        T.n[i] = t->dims[i];
    }
    if (T.numel() > 0) {
        TK_REQUIRE(t->data != nullptr, TK_ERR_ARG, std::string(name) + ": null data");
        TK_REQUIRE(((uintptr_t)t->data % 16) == 0, TK_ERR_ALIGN, std::string(name) + ": data not 16-byte aligned");
    }
    if (T.dt == TK_FP8_E4M3)
        TK_REQUIRE(t->scale > 0.f && std::isfinite(t->scale), TK_ERR_ARG, std::string(name) + ": FP8 scale must be > 0");
    return T;
}

Mat mat_in(const tk_matrix* m, const char* name) {
    TK_REQUIRE(m != nullptr, TK_ERR_ARG, std::string(name) + ": null matrix");
    TK_REQUIRE(m->rows >= 0 && m->cols >= 0, TK_ERR_SHAPE, std::string(name) + ": negative size");
    TK_REQUIRE(m->ld >= std::max<int64_t>(1, m->rows), TK_ERR_SHAPE, std::string(name) + ": ld < rows");
    TK_REQUIRE(m->dtype >= TK_F64 && m->dtype <= TK_BF16, TK_ERR_DTYPE, std::string(name) + ": bad dtype");
    if (m->rows * m->cols > 0) {
        TK_REQUIRE(m->data != nullptr, TK_ERR_ARG, std::string(name) + ": null data");
        TK_REQUIRE(((uintptr_t)m->data % dtype_size(m->dtype)) == 0, TK_ERR_ALIGN,
                   std::string(name) + ": data misaligned");
    }
    Mat M;
    M.p = m->data;
    M.dt = m->dtype;
    M.rows = m->rows;
    M.cols = m->cols;
    M.ld = m->ld;
    return M;
}

static tk_dtype acc_of(tk_dtype data) { return data == TK_F64 ? TK_F64 : TK_F32; }

struct Opts {
    std::vector<int> order;
    int qr_method = 0;
    int refine = 0;
    int max_sweeps = 40;
    bool async_outputs = false;
};

static Opts opts_in(const tk_opts* o, int d) {
    Opts r;
    r.order.resize(d);
    std::iota(r.order.begin(), r.order.end(), 0);
    if (!o) return r;
    if (o->mode_order) {
        std::vector<int> seen(d, 0);
        for (int i = 0; i < d; ++i) {
            int m = o->mode_order[i];
            TK_REQUIRE(m >= 0 && m < d && !seen[m], TK_ERR_ARG, "opts.mode_order is not a permutation of 0..d-1");
            seen[m] = 1;
            r.order[i] = m;
        }
    }
    TK_REQUIRE(o->qr_method >= 0 && o->qr_method <= 2, TK_ERR_ARG, "opts.qr_method must be 0, 1 or 2");
    r.qr_method = o->qr_method;
    r.refine = o->refine;
    TK_REQUIRE(o->async_outputs == 0 || o->async_outputs == 1, TK_ERR_ARG, "opts.async_outputs must be 0 or 1");
    r.async_outputs = o->async_outputs != 0;
    if (o->max_jacobi_sweeps > 0) r.max_sweeps = o->max_jacobi_sweeps;
    else if (o->max_jacobi_sweeps == -1) r.max_sweeps = 0;
    else TK_REQUIRE(o->max_jacobi_sweeps == 0, TK_ERR_ARG, "opts.max_jacobi_sweeps must be >= -1");
    return r;
}

// ------------------------------------------------------------------ small helpers

// The matrix in the accumulation dtype, contiguous (ld = rows): the matrix
// itself when it already is, else a converted copy (the factors are read only).
static Mat mat_to(Ctx& c, const Mat& M, tk_dtype dt) {
    if (M.dt == dt && (M.ld == M.rows || M.cols <= 1)) return M;  // already what the consumers read
    Mat o;
    o.dt = dt;
    o.rows = M.rows;
    o.cols = M.cols;
    o.ld = std::max<int64_t>(1, M.rows);
    void* p = c.alloc_bytes(dtype_size(dt) * M.rows * M.cols);
    launch_convert(c, M.p, M.dt, M.rows, M.cols, M.ld, p, dt, o.ld, 1.f);
    o.p = p;
    return o;
}

static Tens tens_to(Ctx& c, const Tens& T, tk_dtype dt) {
    Tens o = T;
    o.dt = dt;
    o.scale = 1.f;
    o.p = c.alloc_bytes(dtype_size(dt) * T.numel());
    launch_convert(c, T.p, T.dt, T.numel(), 1, std::max<int64_t>(1, T.numel()), o.p, dt, std::max<int64_t>(1, T.numel()),
                   T.scale);
    return o;
}

// Y = T x_j M^T with M(i, a) = M[i + ld a] (mtrans = false) or M[a + ld i];
// output allocated in the workspace unless dst is given.
static Tens ttm_to(Ctx& c, const Tens& T, int j, const Mat& M, bool mtrans, tk_dtype acc, void* dst = nullptr) {
    int64_t m = mtrans ? M.rows : M.cols;
    Tens o = T;
    o.n[j] = m;
    o.dt = acc;
    o.scale = 1.f;
    o.p = dst ? dst : c.alloc_bytes(dtype_size(acc) * o.numel());
    const bool aligned = reinterpret_cast<uintptr_t>(o.p) % 16 == 0;
    const bool narrow = c.use_tc && ttm_narrow_eligible(T, j, m, acc) && aligned;
    const bool tc = !narrow && c.use_tc && ttm_tc_eligible(T, j, m, acc);
    const bool bf = !narrow && !tc && c.use_tc && ttm_bf16_eligible(T, j, m, acc);
    const bool f8 = !narrow && !tc && !bf && c.use_tc && ttm_fp8_eligible(T, j, m, acc) && aligned;
    // the tensor-core kernels split an FP64 factor themselves; the narrow and SIMT kernels of FP32-class
    // data read FP32 factors
    const Mat Mu = (M.dt == TK_F64 && acc != TK_F64 && !(tc || bf || f8)) ? mat_to(c, M, acc) : M;
    if (narrow)
        launch_ttm_narrow(c, T, j, Mu, mtrans, m, static_cast<float*>(o.p));
    else if (tc)
        launch_ttm_tc(c, T, j, Mu, mtrans, m, static_cast<float*>(o.p));
    else if (bf)
        launch_ttm_bf16(c, T, j, Mu, mtrans, m, static_cast<float*>(o.p));
    else if (f8)
        launch_ttm_fp8(c, T, j, Mu, mtrans, m, static_cast<float*>(o.p));
    else
        launch_ttm(c, T, j, Mu, mtrans, m, o.p, acc);
    return o;
}

// Whether ttm_to takes a tensor-core kernel that splits the factor (tf32x3)
// for this product (a workspace output, 16-byte aligned).
static bool ttm_uses_tc(const Ctx& c, const Tens& T, int j, int64_t m, tk_dtype acc) {
    return c.use_tc && !ttm_narrow_eligible(T, j, m, acc) && ttm_tc_eligible(T, j, m, acc);
}

// The order multi_ttm applies the factors in: cheapest-shrinking mode first
// (smallest output; ties: the higher mode); FP8 data streams through the
// tensor cores only along its contiguous mode, so that one goes first (the
// later products then read the much smaller FP32 intermediate).
static std::vector<int> mtt_order(const Ctx& c, const Tens& T, std::vector<int> modes, const Mat* M, bool mtrans,
                                  tk_dtype acc) {
    std::vector<int> order;
    Tens cur = T;
    while (!modes.empty()) {
        size_t best = 0;
        double bestr = 1e300;
        for (size_t t = 0; t < modes.size(); ++t) {
            int i = modes[t];
            double m = (double)(mtrans ? M[i].rows : M[i].cols);
            double ratio = m / std::max<double>(1.0, (double)cur.n[i]);
            if (ratio < bestr - 1e-15 || (std::fabs(ratio - bestr) <= 1e-15 && i > modes[best])) {
                bestr = ratio;
                best = t;
            }
        }
        for (size_t t = 0; t < modes.size() && c.use_tc && cur.dt == TK_FP8_E4M3; ++t)
            if (modes[t] == 0 && ttm_fp8_eligible(cur, 0, mtrans ? M[0].rows : M[0].cols, acc)) best = t;
        const int i = modes[best];
        modes.erase(modes.begin() + best);
        order.push_back(i);
        cur.n[i] = mtrans ? M[i].rows : M[i].cols;
        cur.dt = acc;
    }
    return order;
}

// Apply M_i to every mode in `modes` in mtt_order, the last product written to
// dst when given; trace (optional) receives (mode, product so far) per step.
// The factors of the tensor-core steps are split in one launch beforehand.
static Tens multi_ttm(Ctx& c, const Tens& T, std::vector<int> modes, const Mat* M, bool mtrans, tk_dtype acc,
                      void* dst = nullptr, std::vector<std::pair<int, Tens>>* trace = nullptr) {
    const std::vector<int> order = mtt_order(c, T, modes, M, mtrans, acc);
    struct CacheOn {
        Ctx& c;
        bool was;
        CacheOn(Ctx& cc, bool on) : c(cc), was(cc.split_cache) { c.split_cache = was || on; }
        ~CacheOn() { c.split_cache = was; }
    };
    std::vector<TcSplitReq> reqs;
    if (c.use_tc && acc == TK_F32 && order.size() >= 2) {
        Tens sh = T;
        for (int i : order) {
            const int64_t m = mtrans ? M[i].rows : M[i].cols;
            if (ttm_uses_tc(c, sh, i, m, acc)) reqs.push_back({M[i], mtrans, sh.n[i], m, false});
            sh.n[i] = m;
            sh.dt = acc;
            sh.p = reinterpret_cast<void*>(uintptr_t(256));  // a workspace block: 256-byte aligned
        }
        if (reqs.size() >= 2) tc_presplit(c, reqs);
    }
    CacheOn cache_on(c, reqs.size() >= 2);
    Tens cur = T;
    for (size_t s = 0; s < order.size(); ++s) {
        const int i = order[s];
        cur = ttm_to(c, cur, i, M[i], mtrans, acc, s + 1 == order.size() ? dst : nullptr);
        if (trace) trace->push_back({i, cur});  // the mode just applied and the product so far
    }
    return cur;
}

// Dimension tree of Section 4.4 (All-Modes-Multi-TTM): apply the factors of
// `nset`, then split the modes still owed a sketch in halves and recurse.
// Y[j] receives X x_{k != j} M_k for every j in `mset`; dst[j] (optional)
// names the buffer for that leaf.
static void all_modes(Ctx& c, const Tens& T, const std::vector<int>& mset, const std::vector<int>& nset, const Mat* M,
                      tk_dtype acc, std::vector<Tens>& Y, void* const* dst) {
    // the tree applies each factor more than once: keep their tensor-core splits
    struct CacheOn {
        Ctx& c;
        bool was;
        explicit CacheOn(Ctx& cc) : c(cc), was(cc.split_cache) { c.split_cache = true; }
        ~CacheOn() { c.split_cache = was; }
    } cache_on(c);
    void* leaf = (mset.size() == 1 && dst) ? dst[mset[0]] : nullptr;
    Tens cur = nset.empty() ? T : multi_ttm(c, T, nset, M, false, acc, leaf);
    if (mset.size() == 1) {
        if (nset.empty() && leaf) {  // d == 1 never reaches here (d >= 2 enforced)
            launch_convert(c, cur.p, cur.dt, cur.numel(), 1, cur.numel(), leaf, acc, cur.numel(), cur.scale);
            cur.p = leaf;
        }
        Y[mset[0]] = cur;
        return;
    }
    size_t h = mset.size() / 2;
    std::vector<int> m1(mset.begin(), mset.begin() + h), m2(mset.begin() + h, mset.end());
    all_modes(c, cur, m1, m2, M, acc, Y, dst);
    all_modes(c, cur, m2, m1, M, acc, Y, dst);
}

// Thin QR (Algorithm RRF) of several sketch unfoldings.  Y[b] is an n_b x k_b
// view; Q[b] receives the n_b x k_b orthonormal factor in FP64 (ld n_b).
// CholeskyQR2 (FP64 Gram, FP64 Cholesky) with a Householder fallback selected
// on the device (no host synchronisation): a breakdown in either Cholesky
// pass raises bad[b], which skips the remaining CholeskyQR2 kernels and lets
// the Householder kernel run.  slots[b] is the QR-info slot to fill.  When
// every Y is FP32 (sketches of FP32-class data) the first Gram is accumulated
// with Dot2, and both Cholesky factorisations and both products Y R^{-1} run
// in double-float arithmetic (~48 bits, on the FP32 pipe); Q stays FP64.
static void orth_batch(Ctx& c, const std::vector<View2>& Y, const std::vector<int64_t>& n,
                       const std::vector<int64_t>& k, const std::vector<double*>& Q, const std::vector<int>& slots) {
    const int B = (int)Y.size();
    if (B == 0) return;
    TK_REQUIRE(B <= TK_MAX_D, TK_ERR_ARG, "orth: too many matrices in one batch");
    int kmax = 1;
    KDims kd;
    for (int b = 0; b < B; ++b) {
        kmax = std::max<int>(kmax, (int)k[b]);
        kd.k[b] = (int)k[b];
    }
    TK_REQUIRE(kmax <= 256, TK_ERR_SHAPE, "orth: sketch width above 256 is not supported");
    // Beyond 112 columns the one-CTA CholeskyQR2 kernels do not fit: Householder QR (FP64) for the batch.
    const bool wide = kmax > 112;
    const bool house_only = wide || c.qr_method == 1;
    int* bad = c.alloc<int>(2 * B);  // [0, B): any breakdown, [B, 2B): pass-2 breakdown
    double* W = c.alloc<double>((int64_t)B * kmax * kmax);
    double* Rinv = c.alloc<double>((int64_t)B * kmax * kmax);
    std::vector<double*> Q1(B), Hsrc(B), Htau(B);
    for (int b = 0; b < B; ++b) {
        Q1[b] = c.alloc<double>(n[b] * k[b]);
        Hsrc[b] = c.alloc<double>(n[b] * k[b]);
        Htau[b] = c.alloc<double>(k[b]);
    }
    launch_fill_int(c, bad, 2 * B, house_only ? 1 : 0);
    bool df = true;
    for (int b = 0; b < B; ++b) df = df && Y[b].dt == TK_F32;
    if (!house_only) {
        // pass 1: W = Y^T Y, R1^{-1}, Q1 = Y R1^{-1}
        c.fork(B, [&](int b) {
            const View2& A = Y[b];
            View2 At;  // (column, row) indexing of the same data
            At.p = A.p;
            At.dt = A.dt;
            At.A1 = A.T1; At.sa1 = A.st1; At.sa2 = A.st2;
            At.T1 = A.A1; At.st1 = A.sa1; At.st2 = A.sa2;
            gemm_nt_f64(c, k[b], k[b], n[b], At, At, 1.0, 0.0, W + (int64_t)b * kmax * kmax, kmax, bad + b, df);
        });
        launch_chol_inv(c, B, kd, kmax, W, Rinv, bad, 1e-12, df);
        if (df)
            launch_apply_rinv_df(c, B, Y.data(), n.data(), k.data(), Rinv, kmax, Q1.data(), bad);
        else
            for (int b = 0; b < B; ++b)
                launch_apply_rinv(c, n[b], k[b], Y[b], Rinv + (int64_t)b * kmax * kmax, kmax, Q1[b], bad + b);
        // pass 2 on Q1
        c.fork(B, [&](int b) {
            View2 Qt = view_cols(Q1[b], TK_F64, n[b]);
            gemm_nt_f64(c, k[b], k[b], n[b], Qt, Qt, 1.0, 0.0, W + (int64_t)b * kmax * kmax, kmax, bad + b);
        });
        launch_chol_inv(c, B, kd, kmax, W, Rinv, bad, 1e-12, df);
        if (df) {
            std::vector<View2> Qr(B);
            for (int b = 0; b < B; ++b) Qr[b] = view_rows(Q1[b], TK_F64, n[b]);
            launch_apply_rinv_df(c, B, Qr.data(), n.data(), k.data(), Rinv, kmax, Q.data(), bad);
        } else {
            for (int b = 0; b < B; ++b) {
                View2 Qr = view_rows(Q1[b], TK_F64, n[b]);
                launch_apply_rinv(c, n[b], k[b], Qr, Rinv + (int64_t)b * kmax * kmax, kmax, Q[b], bad + b);
            }
        }
    }
    c.fork(B, [&](int b) {
        int* slot = slots[b] >= 0 ? c.dqr + slots[b] : nullptr;
        if (c.qr_method != 2 || wide)  // the fallback copies Y itself and records the method taken
            launch_householder(c, n[b], k[b], Y[b], Hsrc[b], Q[b], Htau[b], bad + b, slot, 1);
        else if (slot)
            launch_qr_info(c, slot, bad + b, 3);
    });
}

static void orth_one(Ctx& c, const View2& Y, int64_t n, int64_t k, double* Q, int slot) {
    orth_batch(c, {Y}, {n}, {k}, {Q}, {slot});
}

// Same steps as tucker_orth's body, for the allocation-free entry point.
void orth_matrix(Ctx& c, const Mat& y, const Mat& q) {
    const int64_t k = std::min(y.rows, y.cols);
    double* Qd = c.alloc<double>(y.rows * k);
    if (y.cols >= y.rows) {
        launch_fill_identity(c, Qd, y.rows);
        launch_fill_int(c, c.dqr, 1, 2);
    } else {
        orth_one(c, view_rows(y.p, y.dt, y.ld), y.rows, k, Qd, 0);
    }
    launch_convert(c, Qd, TK_F64, y.rows, k, y.rows, (void*)q.p, q.dt, q.ld, 1.f);
}

// Leading r eigenvectors of the symmetric k x k FP64 matrix A, as the columns
// of Vr (k x r, ld k), in descending eigenvalue order.
//  * any k above 112 (beyond the shared-memory kernels): cyclic Jacobi
//    entirely in FP64.
//  * FP64 data: stage 1 below, then FP64 Jacobi on V1^T A V1 (eig_top).
//  * otherwise: a two-stage scheme built for a chip whose FP64 rate is a small
//    fraction of its FP32 rate.  Stage 1, mixed Jacobi on A (FP32 accuracy),
//    gives V0; one FP64 Newton-Schulz step V0 <- V0 (3I - V0^T V0) / 2 makes it
//    orthonormal to FP64 rounding; B = V0^T A V0 (FP64) is then diagonal up to
//    ~1e-7 ||A||, so stage 2, mixed Jacobi on B, resolves it to 1e-11 ||A||
//    in absolute terms; V = V0 J, the leading r columns are selected and
//    made orthonormal with one more Newton-Schulz step.  (A is the Gram of a
//    core computed from FP32-class data, whose entries carry relative errors
//    near 1e-7.  On the benchmark's cores the singular-value-weighted error
//    of the leading eigenvectors is ~2e-8 at 1e-11, ~3e-9 at 1e-14 and
//    ~3e-7 at 1e-10; 1e-11 takes 13 stage-2 sweeps over the three modes
//    where 1e-14 takes 17.)
// Stage 1 of the FP32-class eigensolver: FP32 Jacobi on A until every
// |a_pq| <= 1e-6 sqrt(|a_pp a_qq|) (relative to the pair's own diagonal
// entries), then FP64 Newton-Schulz steps V <- V (3I - V^T V) / 2, each of
// which squares the distance from orthonormality (the FP32 rotations leave
// J about 1e-6 off, one step ~1e-12, two FP64 rounding); V1 (k x k, ld k)
// diagonalises A, small eigenvalues included, to ~1e-7 of each entry's own
// scale (on the benchmark's cores: the eigenvectors to a singular-value-
// weighted 1e-6 already, and stage 2 then needs one or two sweeps; an
// absolute 1e-6 ||A|| stop leaves the small-eigenvalue tail unresolved and
// stage 2 with four to six).  One step serves FP32-class data (stage 2 makes
// the final factor orthonormal itself); FP64 data, whose stage 2 works in the
// V1 basis, takes two.
static double* eig_seed(Ctx& c, int64_t k, const double* A, int ns_steps = 1) {
    double* D = c.alloc<double>(k);
    double* V0 = c.alloc<double>(k * k);
    double* V1 = c.alloc<double>(k * k);
    double* W = c.alloc<double>(k * k);
    launch_jacobi_mixed(c, k, A, D, nullptr, V0, V1, 1e-6, c.max_sweeps, false);  // V0 = V1 = J in FP64
    for (int step = 0; step < ns_steps; ++step) {
        if (step > 0) launch_convert(c, V1, TK_F64, k * k, 1, k * k, V0, TK_F64, k * k, 1.f);  // V0 = V1
        gemm_nt_f64(c, k, k, k, view_cols(V0, TK_F64, k), view_cols(V0, TK_F64, k), 1.0, 0.0, W, k);
        gemm_nt_f64(c, k, k, k, view_rows(V0, TK_F64, k), view_cols(W, TK_F64, k), -0.5, 1.5, V1, k);
    }
    return V1;
}

// Stage 2: B = V1^T A V1 (FP64) is resolved by mixed Jacobi with a
// double-float diagonal to 1e-11 ||A|| in absolute terms; V = V1 J, the
// leading r columns are selected (Vr, k x r, ld k) and made orthonormal with
// one more Newton-Schulz step.  V1 only has to diagonalise A approximately:
// stage 2 starts from whatever off-diagonal B has (it is run to the same
// absolute threshold either way).
static void eig_resolve(Ctx& c, int64_t k, const double* A, const double* V1, int64_t r, double* Vr) {
    double* D = c.alloc<double>(k);
    double* Pm = c.alloc<double>(k * k);
    double* B = c.alloc<double>(k * k);
    double* Vt = c.alloc<double>(k * r);
    double* Wr = c.alloc<double>(r * r);
    gemm_nt_f64(c, k, k, k, view_rows(A, TK_F64, k), view_cols(V1, TK_F64, k), 1.0, 0.0, Pm, k);
    gemm_nt_f64(c, k, k, k, view_cols(V1, TK_F64, k), view_cols(Pm, TK_F64, k), 1.0, 0.0, B, k);
    // the rotations replayed on the rows of V1 give V = V1 J, whose top-r columns go to Vt and to Vr
    // (Vr starts as a copy of Vt for the Newton-Schulz step)
    launch_jacobi_mixed(c, k, B, D, nullptr, nullptr, nullptr, 1e-11, c.max_sweeps, true, V1, r, Vt, Vr);
    gemm_nt_f64(c, r, r, k, view_cols(Vt, TK_F64, k), view_cols(Vt, TK_F64, k), 1.0, 0.0, Wr, r);
    gemm_nt_f64(c, k, r, r, view_rows(Vt, TK_F64, k), view_cols(Wr, TK_F64, r), -0.5, 1.5, Vr, k);
}

// Leading r eigenvectors of the symmetric k x k FP64 matrix A, as the columns
// of Vr (k x r, ld k), in descending eigenvalue order.
//  * any k above 112 (beyond the shared-memory kernels): cyclic Jacobi
//    entirely in FP64.
//  * FP64 data: the FP32 seeding stage (eig_seed with two Newton-Schulz
//    steps), then FP64 Jacobi on V1^T A V1.
//  * otherwise: a two-stage scheme built for a chip whose FP64 rate is a small
//    fraction of its FP32 rate (eig_seed, then eig_resolve).  (A is the Gram
//    of a core computed from FP32-class data, whose entries carry relative
//    errors near 1e-7.  On the benchmark's cores the singular-value-weighted
//    error of the leading eigenvectors is ~2e-8 at a 1e-11 stage-2 threshold,
//    ~3e-9 at 1e-14 and ~3e-7 at 1e-10.)
static void eig_top(Ctx& c, int64_t k, const double* A, int64_t r, double* Vr, bool fp64_path) {
    if (fp64_path && k > 112) {  // beyond the shared-memory kernels: FP64 Jacobi in global memory
        double* Ac = c.alloc<double>(k * k);
        double* w = c.alloc<double>(k);
        double* Vf = c.alloc<double>(k * k);
        double* gV = c.alloc<double>(k * k);
        launch_convert(c, A, TK_F64, k * k, 1, k * k, Ac, TK_F64, k * k, 1.f);
        launch_jacobi(c, k, Ac, w, Vf, c.max_sweeps, gV);
        launch_convert(c, Vf, TK_F64, k, r, k, Vr, TK_F64, k, 1.f);
        return;
    }
    if (fp64_path) {
        // FP64 data: the FP32 seeding stage, then FP64 Jacobi on B = V1^T A V1, which is diagonal up to
        // ~1e-7 of each entry's scale, so its quadratic convergence takes two or three sweeps instead
        // of the ten or so from A itself; V = V1 Vb keeps FP64 accuracy (V1 is orthonormal to FP64
        // rounding after two Newton-Schulz steps)
        const double* V1 = eig_seed(c, k, A, 2);
        double* Pm = c.alloc<double>(k * k);
        double* B = c.alloc<double>(k * k);
        double* w = c.alloc<double>(k);
        double* Vb = c.alloc<double>(k * k);
        gemm_nt_f64(c, k, k, k, view_rows(A, TK_F64, k), view_cols(V1, TK_F64, k), 1.0, 0.0, Pm, k);
        gemm_nt_f64(c, k, k, k, view_cols(V1, TK_F64, k), view_cols(Pm, TK_F64, k), 1.0, 0.0, B, k);
        launch_jacobi(c, k, B, w, Vb, c.max_sweeps);  // eigenpairs sorted by descending eigenvalue
        gemm_nt_f64(c, k, r, k, view_rows(V1, TK_F64, k), view_cols(Vb, TK_F64, k), 1.0, 0.0, Vr, k);
        return;
    }
    eig_resolve(c, k, A, eig_seed(c, k, A), r, Vr);
}

// STHOSVD of the core (Algorithm STHOSVD applied to Ghat) with an FP64 Gram
// matrix per mode: leading r_j eigenvectors V_j of Ghat_(j) Ghat_(j)^T, then
// Ghat <- Ghat x_j V_j^T.  Returns the truncated core; V[j] = k_j x r_j (ld k_j).
// FP32-class data: the seeding stage of every mode's eigensolver runs at once,
// on the Grams of the untruncated core (concurrent, off the sequential chain);
// truncating the other modes first changes mode j's Gram only by their
// discarded energy, which the resolving stage, run on the Gram of the core
// as truncated so far, absorbs.  The result is that of the sequential
// algorithm to the resolving stage's threshold.
static void truncate_modes(Ctx& c, const Tens& G0, Tens& G, const int64_t* r, const std::vector<int>& order,
                           std::vector<double*>& V, bool fp64_path, const std::vector<double*>& C0,
                           const std::vector<double*>& V1);

// beside (optional): work for the call's side stream, started once the Grams
// of the seeding stage are queued (so that it does not take their SMs) and
// joined before this returns.
static Tens sthosvd_core(Ctx& c, const Tens& G0, const int64_t* r, const std::vector<int>& order,
                         std::vector<double*>& V, bool fp64_path, const std::function<void()>* beside = nullptr) {
    Tens G = G0;
    const int d = G0.d;
    V.assign(d, nullptr);
    for (int j = 0; j < d; ++j)
        TK_REQUIRE(G0.n[j] <= 256, TK_ERR_SHAPE, "sthosvd: core mode above 256 is not supported");
    std::vector<double*> C0(d, nullptr), V1(d, nullptr);
    if (!fp64_path) {
        c.fork(d, [&](int j) {
            const int64_t kj = G0.n[j];
            if (kj > 112) return;  // solved in FP64 below
            const int64_t K = kj ? G0.numel() / kj : 0;
            C0[j] = c.alloc<double>(kj * kj);
            const View2 A = view_unfold_rows(G0, j);
            gemm_nt_f64(c, kj, kj, K, A, A, 1.0, 0.0, C0[j], kj);
        });
    }
    auto body = [&]() {
        if (!fp64_path) {
            c.fork(d, [&](int j) {
                if (C0[j]) V1[j] = eig_seed(c, G0.n[j], C0[j]);
            });
        }
        truncate_modes(c, G0, G, r, order, V, fp64_path, C0, V1);
    };
    if (beside && *beside) c.side(body, *beside);
    else body();
    return G;
}

// The sequential part of sthosvd_core: mode by mode in `order`, the leading
// eigenvectors of the current core's Gram and the truncation of that mode.
static void truncate_modes(Ctx& c, const Tens& G0, Tens& G, const int64_t* r, const std::vector<int>& order,
                           std::vector<double*>& V, bool fp64_path, const std::vector<double*>& C0,
                           const std::vector<double*>& V1) {
    for (int j : order) {
        int64_t kj = G.n[j];
        int64_t K = kj ? G.numel() / kj : 0;
        double* Vj = c.alloc<double>(kj * r[j]);
        if (fp64_path || kj > 112) {
            double* C = c.alloc<double>(kj * kj);
            View2 A = view_unfold_rows(G, j);
            gemm_nt_f64(c, kj, kj, K, A, A, 1.0, 0.0, C, kj);
            eig_top(c, kj, C, r[j], Vj, true);
        } else {
            double* C = C0[j];
            if (G.p != G0.p) {  // some mode is truncated already: the Gram of the current core
                C = c.alloc<double>(kj * kj);
                View2 A = view_unfold_rows(G, j);
                gemm_nt_f64(c, kj, kj, K, A, A, 1.0, 0.0, C, kj);
            }
            eig_resolve(c, kj, C, V1[j], r[j], Vj);
        }
        V[j] = Vj;
        Mat Vm;
        Vm.p = Vj;
        Vm.dt = TK_F64;
        Vm.rows = kj;
        Vm.cols = r[j];
        Vm.ld = kj;
        G = ttm_to(c, G, j, Vm, false, TK_F64);
    }
}

// ||X - G x_1 U_1 ... x_d U_d||^2 and ||X||^2 into err2 (device, 2 doubles); with
// dx != NULL also dx = alpha (X - Xhat).  G and U are in the accumulation
// dtype.  All modes but one are expanded first (smallest growth first); the
// last one is fused with the residual on tensor cores when eligible, so Xhat is
// never written; otherwise Xhat is formed and compared by separate kernels.
static void residual_pass(Ctx& c, const Tens& X, const Tens& G, const std::vector<Mat>& U, tk_dtype acc,
                          double* err2, void* dx, tk_dtype dxdt, double alpha) {
    const int d = X.d;
    int f = d - 1;
    std::vector<int> todo, order;
    for (int j = 0; j < d; ++j)
        if (j != f) todo.push_back(j);
    while (!todo.empty()) {
        size_t best = 0;
        double bestr = 1e300;
        for (size_t t = 0; t < todo.size(); ++t) {
            int i = todo[t];
            double ratio = (double)U[i].rows / std::max<double>(1.0, (double)U[i].cols);
            if (ratio < bestr) { bestr = ratio; best = t; }
        }
        order.push_back(todo[best]);
        todo.erase(todo.begin() + best);
    }
    const int64_t m = U[f].rows;
    // BF16 data: the epilogue reads the BF16 X tile (and writes a BF16 dX) itself; FP8 data: the E4M3 X
    // tile, scaled back by 1 / scale (norms only, no dX)
    Tens Ws = G;  // the shape the last product starts from
    for (int i : order) {
        Ws.n[i] = U[i].rows;
        Ws.dt = acc;
        Ws.p = reinterpret_cast<void*>(uintptr_t(256));  // a workspace block: 256-byte aligned
    }
    const bool fused = c.use_tc &&
                       (X.dt == TK_F32 || (X.dt == TK_BF16 && X.left(f) % 8 == 0) ||
                        (X.dt == TK_FP8_E4M3 && X.left(f) % 16 == 0 && !dx)) &&
                       acc == TK_F32 && (!dx || dxdt == X.dt) && ttm_tc_residual_eligible(Ws, f, m);
    // the factors of the tensor-core products split in one launch
    std::vector<TcSplitReq> reqs;
    if (c.use_tc && acc == TK_F32) {
        Tens sh = G;
        for (int i : order) {
            if (ttm_uses_tc(c, sh, i, U[i].rows, acc)) reqs.push_back({U[i], true, sh.n[i], U[i].rows, false});
            sh.n[i] = U[i].rows;
            sh.dt = acc;
            sh.p = reinterpret_cast<void*>(uintptr_t(256));
        }
        if (fused) reqs.push_back({U[f], true, Ws.n[f], m, true});
        if (reqs.size() >= 2) tc_presplit(c, reqs);
    }
    struct CacheOn {
        Ctx& c;
        bool was;
        CacheOn(Ctx& cc, bool on) : c(cc), was(cc.split_cache) { c.split_cache = was || on; }
        ~CacheOn() { c.split_cache = was; }
    } cache_on(c, reqs.size() >= 2);
    Tens W = G;
    for (int i : order) W = ttm_to(c, W, i, U[i], true, acc);
    if (fused) {
        const int nb = tc_num_ctas(c, W, f, m, true);
        double* part = c.alloc<double>(2 * nb);
        launch_ttm_tc_residual(c, W, f, U[f], true, m, X.p, X.dt, dx, (float)alpha, part,
                               X.dt == TK_FP8_E4M3 ? 1.f / X.scale : 1.f);
        launch_sum_pairs(c, part, nb, err2);
        return;
    }
    Tens Xh = ttm_to(c, W, f, U[f], true, acc);
    if (dx) launch_axpby_residual(c, X, Xh.p, acc, alpha, dx, dxdt);
    launch_residual_norms(c, X, Xh.p, acc, err2);
}

// Final steps shared by both algorithms: U_j = Q_j V_j, sign gauge, casts
// into the caller's G and U, optional relative error.
static void finish(Ctx& c, const Tens& X, const std::vector<double*>& Qd, const std::vector<int64_t>& kdim,
                   Tens Gt, const std::vector<double*>& V, const int64_t* r, const Tens& Gout,
                   const std::vector<Mat>& Uout, double* err_dev, std::vector<double*>* signs = nullptr) {
    const int d = X.d;
    std::vector<double*> U(d), sg(d);
    c.fork(d, [&](int j) {
        U[j] = c.alloc<double>(X.n[j] * r[j]);
        sg[j] = c.alloc<double>(r[j]);
        gemm_nt_f64(c, X.n[j], r[j], kdim[j], view_rows(Qd[j], TK_F64, X.n[j]), view_cols(V[j], TK_F64, kdim[j]), 1.0,
                    0.0, U[j], X.n[j]);
        launch_sign_fix(c, U[j], X.n[j], r[j], sg[j], (void*)Uout[j].p, Uout[j].dt, Uout[j].ld);
    });
    launch_apply_signs(c, (double*)Gt.p, Gt, sg.data(), Gout.p, Gout.dt);
    if (signs) *signs = sg;
    if (!err_dev) return;
    // ||X - G x_j U_j|| from the returned G and U, in the accumulation dtype.
    tk_dtype acc = acc_of(X.dt);
    Tens Ga = tens_to(c, Gout, acc);
    std::vector<Mat> Ua(d);
    for (int j = 0; j < d; ++j) Ua[j] = mat_to(c, Uout[j], acc);
    residual_pass(c, X, Ga, Ua, acc, err_dev, nullptr, TK_F32, 0.0);
}

struct Plan {
    std::vector<int64_t> s, k;
};

}  // namespace tk

using namespace tk;

// ------------------------------------------------------------------ call wrapper

template <typename F>
static tk_status run_call(tk_handle* h, F&& body) {
    if (!h) return TK_ERR_ARG;
    h->last_error.clear();
    try {
        int cur = 0;
        TK_CUDA(cudaGetDevice(&cur));
        TK_REQUIRE(cur == h->device, TK_ERR_ARG, "handle was created on another device than the current one");
        cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
        TK_CUDA(cudaStreamIsCapturing(h->stream, &cst));
        const bool capturing = cst != cudaStreamCaptureStatusNone;
        Ctx plan;
        plan.stream = h->stream;
        plan.exec = false;
        plan.use_tc = h->use_tc;
        plan.grid_sms = h->sm_reserve > 0 ? std::max(1, tc::num_sms() - h->sm_reserve) : 0;
        plan.capturing = capturing;
        body(plan);
        size_t need = plan.used + 512;
        if (need > h->ws_bytes) {
            TK_REQUIRE(!capturing, TK_ERR_WORKSPACE,
                       "recording into a CUDA graph needs a large enough workspace: run the call once first");
            TK_CUDA(cudaStreamSynchronize(h->stream));
            if (h->ws) {
                if (h->ws_held)
                    h->retired.push_back(h->ws);
                else
                    TK_CUDA(cudaFree(h->ws));
            }
            h->ws_held = false;
            h->ws = nullptr;
            h->ws_bytes = 0;
            size_t grow = need + need / 4;
            if (cudaMalloc((void**)&h->ws, grow) != cudaSuccess) {
                cudaGetLastError();
                h->ws = nullptr;
                fail(TK_ERR_WORKSPACE, "workspace allocation of " + std::to_string(grow) + " bytes failed");
            }
            h->ws_bytes = grow;
        }
        if (capturing) h->ws_held = true;
        Ctx ex;
        ex.stream = h->stream;
        ex.exec = true;
        ex.capturing = capturing;
        ex.base = h->ws;
        ex.dflags = h->dflags;
        ex.dqr = h->dqr;
        ex.launches = &h->launches;
        ex.prof = &h->prof;
        ex.use_tc = h->use_tc;
        ex.grid_sms = plan.grid_sms;
        for (int i = 0; i < Ctx::kAux; ++i) {
            ex.aux[i] = h->aux[i];
            ex.ev_join[i] = h->ev_join[i];
        }
        ex.ev_fork = h->ev_fork;
        ex.ctr = h->ctr;
        body(ex);
        return TK_OK;
    } catch (const Error& e) {
        h->last_error = e.msg;
        return e.st;
    } catch (const std::exception& e) {
        h->last_error = e.what();
        return TK_ERR_ARG;
    }
}

static void set_opts(Ctx& c, const Opts& o) {
    c.qr_method = o.qr_method;
    c.refine = o.refine;
    c.max_sweeps = o.max_sweeps;
}

static void CUDART_CB deliver_slot(void* arg) {
    auto* sl = static_cast<tk_handle::HostSlot*>(arg);
    if (sl->mode == 1)
        *sl->dst = sl->vals[0];
    else
        *sl->dst = sl->vals[1] > 0 ? std::sqrt(sl->vals[0] / sl->vals[1]) : 0.0;
    __atomic_store_n(&sl->pending, 0, __ATOMIC_RELEASE);
}

// Host scalar from the device pair dev2 = {a, b}: sqrt(a / b) or a.  With
// async, a D2H copy into the handle's pinned ring and a host callback that
// writes *out after the stream reaches it; otherwise a synchronising copy.
static void read_err(tk_handle* h, Ctx& c, const double* dev2, double* out_rel, bool squared_abs,
                     bool async = false) {
    if (!c.exec) return;
    TK_REQUIRE(async || !c.capturing, TK_ERR_ARG, "a host output recorded into a CUDA graph needs async_outputs");
    if (async) {
        // next slot not recorded by a graph; a slot is reused only after its callback has run
        tk_handle::HostSlot* sl = nullptr;
        for (int n = 0; n < tk_handle::kHostSlots && !sl; ++n) {
            tk_handle::HostSlot* x = &h->slots[h->next_slot];
            h->next_slot = (h->next_slot + 1) % tk_handle::kHostSlots;
            if (!x->reserved && !(c.capturing && __atomic_load_n(&x->pending, __ATOMIC_ACQUIRE))) sl = x;
        }
        TK_REQUIRE(sl, TK_ERR_ARG, "every host-output slot is held by a recorded CUDA graph (tk_graph_release)");
        if (c.capturing) {
            sl->reserved = 1;  // delivered at every replay of the graph
        } else {
            if (__atomic_load_n(&sl->pending, __ATOMIC_ACQUIRE)) TK_CUDA(cudaStreamSynchronize(c.stream));
            sl->pending = 1;
        }
        sl->dst = out_rel;
        sl->mode = squared_abs ? 1 : 0;
        TK_CUDA(cudaMemcpyAsync(sl->vals, dev2, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
        TK_CUDA(cudaLaunchHostFunc(c.stream, deliver_slot, sl));
        return;
    }
    double host[2] = {0, 0};
    TK_CUDA(cudaMemcpyAsync(host, dev2, sizeof(host), cudaMemcpyDeviceToHost, c.stream));
    TK_CUDA(cudaStreamSynchronize(c.stream));
    if (squared_abs)
        *out_rel = host[0];
    else
        *out_rel = host[1] > 0 ? std::sqrt(host[0] / host[1]) : 0.0;
    (void)h;
}

// ------------------------------------------------------------------ handle API

extern "C" {

tk_status tk_create(tk_handle** h, void* stream) {
    if (!h) return TK_ERR_ARG;
    *h = nullptr;
    tk_handle* x = new (std::nothrow) tk_handle();
    if (!x) return TK_ERR_WORKSPACE;
    x->stream = (cudaStream_t)stream;
    const char* ttm_env = getenv("TUCKER_TTM");
    x->use_tc = !(ttm_env && strcmp(ttm_env, "simt") == 0);
    if (cudaGetDevice(&x->device) != cudaSuccess || cudaMalloc((void**)&x->dflags, 64) != cudaSuccess) {
        cudaGetLastError();
        delete x;
        return TK_ERR_CUDA;
    }
    x->dqr = (int*)((char*)x->dflags + 16);
    if (cudaHostAlloc((void**)&x->slots, sizeof(tk_handle::HostSlot) * tk_handle::kHostSlots, cudaHostAllocDefault) !=
        cudaSuccess) {
        cudaGetLastError();
        cudaFree(x->dflags);
        delete x;
        return TK_ERR_CUDA;
    }
    std::memset((void*)x->slots, 0, sizeof(tk_handle::HostSlot) * tk_handle::kHostSlots);
    if (cudaMemset(x->dflags, 0, 64) != cudaSuccess) {
        cudaFree(x->dflags);
        delete x;
        return TK_ERR_CUDA;
    }
    bool ok = cudaMalloc((void**)&x->ctr, sizeof(unsigned) * tk::Ctx::kCounters) == cudaSuccess &&
              cudaMemset(x->ctr, 0, sizeof(unsigned) * tk::Ctx::kCounters) == cudaSuccess &&
              cudaEventCreateWithFlags(&x->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    // the auxiliary streams take the priority of the handle's stream, so that a caller can rank the
    // whole of a call (its forked work included) against work on other streams
    int prio = 0;
    if (cudaStreamGetPriority(x->stream, &prio) != cudaSuccess) {
        cudaGetLastError();
        prio = 0;
    }
    for (int i = 0; i < tk::Ctx::kAux && ok; ++i)
        ok = cudaStreamCreateWithPriority(&x->aux[i], cudaStreamNonBlocking, prio) == cudaSuccess &&
             cudaEventCreateWithFlags(&x->ev_join[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        tk_destroy(x);
        return TK_ERR_CUDA;
    }
    *h = x;
    return TK_OK;
}

tk_status tk_destroy(tk_handle* h) {
    if (!h) return TK_ERR_ARG;
    cudaStreamSynchronize(h->stream);
    if (h->ws) cudaFree(h->ws);
    for (char* p : h->retired) cudaFree(p);
    if (h->dflags) cudaFree(h->dflags);
    if (h->slots) cudaFreeHost(h->slots);
    for (auto& r : h->prof.recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : h->prof.pool) cudaEventDestroy(e);
    for (int i = 0; i < tk::Ctx::kAux; ++i) {
        if (h->aux[i]) {
            cudaStreamSynchronize(h->aux[i]);
            cudaStreamDestroy(h->aux[i]);
        }
        if (h->ev_join[i]) cudaEventDestroy(h->ev_join[i]);
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ctr) cudaFree(h->ctr);
    delete h;
    return TK_OK;
}

tk_status tk_graph_release(tk_handle* h) {
    if (!h) return TK_ERR_ARG;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
        h->last_error = "tk_graph_release: stream synchronisation failed";
        return TK_ERR_CUDA;
    }
    for (char* p : h->retired) cudaFree(p);
    h->retired.clear();
    h->ws_held = false;
    for (int i = 0; i < tk_handle::kHostSlots; ++i) h->slots[i].reserved = 0;
    return TK_OK;
}

tk_status tk_set_stream(tk_handle* h, void* stream) {
    if (!h) return TK_ERR_ARG;
    h->stream = (cudaStream_t)stream;
    return TK_OK;
}

tk_status tk_set_sm_reserve(tk_handle* h, int sms) {
    if (!h) return TK_ERR_ARG;
    if (sms < 0 || sms >= tk::tc::num_sms()) {
        h->last_error = "tk_set_sm_reserve: need 0 <= sms < the SM count";
        return TK_ERR_ARG;
    }
    h->sm_reserve = sms;
    return TK_OK;
}

const char* tk_last_error(const tk_handle* h) { return h ? h->last_error.c_str() : "null handle"; }

tk_status tk_sync_status(tk_handle* h, int* qr_info) {
    if (!h) return TK_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        h->last_error = cudaGetErrorString(e);
        return TK_ERR_CUDA;
    }
    unsigned flags = 0;
    int qr[TK_MAX_D];
    if (cudaMemcpy(&flags, h->dflags, sizeof(flags), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(qr, h->dqr, sizeof(qr), cudaMemcpyDeviceToHost) != cudaSuccess) {
        h->last_error = "reading device status failed";
        return TK_ERR_CUDA;
    }
    cudaMemset(h->dflags, 0, sizeof(unsigned));
    if (qr_info) memcpy(qr_info, qr, sizeof(qr));
    if (flags & FLAG_TIMEOUT) {
        h->last_error = "a bounded device wait gave up";
        return TK_ERR_TIMEOUT;
    }
    if (flags & FLAG_NOT_CONVERGED) {
        h->last_error = "Jacobi eigensolver reached its sweep limit";
        return TK_ERR_NOT_CONVERGED;
    }
    return TK_OK;
}

tk_status tk_selftest_bounded_wait(tk_handle* h, int64_t limit_ns, int64_t* waited_ns) {
    if (limit_ns < 1000 || limit_ns > 2000000000) {
        if (h) h->last_error = "selftest: limit_ns must lie in [1e3, 2e9]";
        return TK_ERR_ARG;
    }
    long long* dev = nullptr;
    tk_status st = run_call(h, [&](Ctx& c) {
        dev = c.alloc<long long>(1);
        launch_wait_selftest(c, (uint64_t)limit_ns, dev);
    });
    if (st != TK_OK || !waited_ns) return st;
    long long v = 0;
    if (cudaMemcpyAsync(&v, dev, sizeof(v), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
        h->last_error = "selftest: reading the waited time failed";
        return TK_ERR_CUDA;
    }
    *waited_ns = v;
    return TK_OK;
}

static std::mutex g_origin_mu;
static std::map<int, cudaEvent_t> g_origin;  // per device: recorded by the latest tk_profile(h, 1)

tk_status tk_profile(tk_handle* h, int enable) {
    if (!h) return TK_ERR_ARG;
    if (enable) {
        for (auto& r : h->prof.recs) {
            h->prof.pool.push_back(r.a);
            h->prof.pool.push_back(r.b);
        }
        h->prof.recs.clear();
        // Create the events now: cudaEventCreate inside the profiled region would cost the
        // host far more than the launches being timed.
        h->prof.recs.reserve(4096);
        while (h->prof.pool.size() < 8192) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                break;
            }
            h->prof.pool.push_back(e);
        }
    }
    h->prof.on = enable != 0;
    if (enable) {  // the time origin of tk_profile_trace, shared by the device's handles
        std::lock_guard<std::mutex> lk(g_origin_mu);
        cudaEvent_t& o = g_origin[h->device];
        if (!o && cudaEventCreate(&o) != cudaSuccess) {
            cudaGetLastError();
            o = nullptr;
        }
        if (o) cudaEventRecord(o, h->stream);
    }
    return TK_OK;
}

tk_status tk_profile_only(tk_handle* h, const char* prefix) {
    if (!h) return TK_ERR_ARG;
    h->prof.only = prefix ? prefix : "";
    return TK_OK;
}

int tk_profile_read(tk_handle* h, tk_prof_entry* out, int max) {
    if (!h) return -1;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return -1;
    std::vector<tk_prof_entry> acc;
    for (auto& r : h->prof.recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) ms = 0.f;
        size_t i = 0;
        for (; i < acc.size(); ++i)
            if (strncmp(acc[i].name, r.name, sizeof(acc[i].name)) == 0) break;
        if (i == acc.size()) {
            tk_prof_entry e;
            memset(&e, 0, sizeof(e));
            strncpy(e.name, r.name, sizeof(e.name) - 1);
            acc.push_back(e);
        }
        acc[i].launches += 1;
        acc[i].ms += ms;
        acc[i].bytes += r.bytes;
        acc[i].flops += r.flops;
        h->prof.pool.push_back(r.a);
        h->prof.pool.push_back(r.b);
    }
    h->prof.recs.clear();
    int n = (int)std::min<size_t>(acc.size(), (size_t)std::max(0, max));
    for (int i = 0; i < n; ++i) out[i] = acc[i];
    return (int)acc.size();
}

int tk_profile_trace(tk_handle* h, tk_trace_entry* out, int max) {
    if (!h) return -1;
    if (!out) return (int)h->prof.recs.size();  // count only; the records stay
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return -1;
    for (auto s : h->aux)
        if (s && cudaStreamSynchronize(s) != cudaSuccess) return -1;
    cudaEvent_t o = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_origin_mu);
        auto it = g_origin.find(h->device);
        if (it != g_origin.end()) o = it->second;
    }
    int n = 0;
    for (auto& r : h->prof.recs) {
        if (n < max) {
            tk_trace_entry e;
            memset(&e, 0, sizeof(e));
            strncpy(e.name, r.name, sizeof(e.name) - 1);
            e.stream = -1;
            if (r.st == h->stream) e.stream = 0;
            for (int i = 0; i < tk::Ctx::kAux; ++i)
                if (r.st == h->aux[i]) e.stream = 1 + i;
            float a = 0.f, b = 0.f;
            if (!o || cudaEventElapsedTime(&a, o, r.a) != cudaSuccess) a = 0.f;
            if (!o || cudaEventElapsedTime(&b, o, r.b) != cudaSuccess) b = a;
            cudaGetLastError();
            e.start_us = 1e3 * (double)a;
            e.end_us = 1e3 * (double)b;
            e.bytes = r.bytes;
            e.flops = r.flops;
            out[n] = e;
        }
        ++n;
        h->prof.pool.push_back(r.a);
        h->prof.pool.push_back(r.b);
    }
    h->prof.recs.clear();
    return n;
}

int64_t tk_workspace_bytes(const tk_handle* h) { return h ? (int64_t)h->ws_bytes : 0; }
int64_t tk_launch_count(const tk_handle* h) { return h ? h->launches : 0; }

// ------------------------------------------------------------------ subranks (host only)

static __int128 sat_mul(__int128 a, __int128 b) {
    const __int128 cap = ((__int128)1) << 100;
    if (a == 0 || b == 0) return 0;
    if (a > cap / b) return cap;
    return a * b;
}

static __int128 sat_pow(__int128 a, int e) {
    __int128 r = 1;
    for (int i = 0; i < e; ++i) r = sat_mul(r, a);
    return r;
}

tk_status tucker_subranks_reuse(int d, const int64_t* r, int p, int64_t* s_out, int64_t* width_out) {
    if (d < 2 || d > TK_MAX_D || !r || !s_out || p < 0) return TK_ERR_ARG;
    std::vector<int64_t> ell(d), s(d);
    __int128 P = 1;
    for (int j = 0; j < d; ++j) {
        if (r[j] < 1) return TK_ERR_ARG;
        ell[j] = r[j] + p;
        P = sat_mul(P, ell[j]);
    }
    for (int i = 0; i < d; ++i) {
        // smallest s with (s * l_i)^(d-1) >= P
        double guess = std::pow((double)P, 1.0 / (d - 1)) / (double)ell[i];
        int64_t v = std::max<int64_t>(1, (int64_t)guess);
        while (v > 1 && sat_pow((__int128)(v - 1) * ell[i], d - 1) >= P) --v;
        while (sat_pow((__int128)v * ell[i], d - 1) < P) ++v;
        s[i] = v;
    }
    std::vector<int> idx(d);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return s[a] > s[b]; });
    for (int i : idx) {
        int64_t need = 1;
        for (int j = 0; j < d; ++j) {
            if (j == i) continue;
            __int128 rest = 1;
            for (int k = 0; k < d; ++k)
                if (k != i && k != j) rest = sat_mul(rest, s[k]);
            int64_t q = (int64_t)((ell[j] + rest - 1) / rest);
            need = std::max(need, q);
        }
        s[i] = std::min(s[i], need);
    }
    for (int j = 0; j < d; ++j) {
        s_out[j] = s[j];
        if (width_out) {
            __int128 w = 1;
            for (int k = 0; k < d; ++k)
                if (k != j) w = sat_mul(w, s[k]);
            width_out[j] = (int64_t)std::min<__int128>(w, (__int128)INT64_MAX);
        }
    }
    return TK_OK;
}

// Most balanced factorisation of L into m factors >= 2 (sorted descending,
// lexicographically smallest); returns false when none exists.
static void factor_rec(int64_t n, int m, int64_t lo, std::vector<int64_t>& cur, std::vector<int64_t>& best,
                       bool& found) {
    if (m == 1) {
        if (n >= lo) {
            cur.push_back(n);
            std::vector<int64_t> key(cur.rbegin(), cur.rend());  // ascending build -> descending key
            if (!found || key < best) {
                best = key;
                found = true;
            }
            cur.pop_back();
        }
        return;
    }
    for (int64_t f = lo; ; ++f) {
        // f^m <= n
        __int128 pw = 1;
        for (int t = 0; t < m; ++t) pw *= f;
        if (pw > n) break;
        if (n % f == 0) {
            cur.push_back(f);
            factor_rec(n / f, m - 1, f, cur, best, found);
            cur.pop_back();
        }
    }
}

tk_status tucker_subranks_matrix(int d, const int64_t* r, int p, const int* order, int64_t* S_out,
                                 int64_t* width_out) {
    if (d < 2 || d > TK_MAX_D || !r || !S_out || p < 0) return TK_ERR_ARG;
    std::vector<int> ord(d);
    std::iota(ord.begin(), ord.end(), 0);
    if (order) {
        std::vector<int> seen(d, 0);
        for (int i = 0; i < d; ++i) {
            if (order[i] < 0 || order[i] >= d || seen[order[i]]) return TK_ERR_ARG;
            seen[order[i]] = 1;
            ord[i] = order[i];
        }
    }
    const int m = d - 1;
    for (int j = 0; j < d; ++j) {
        if (r[j] < 1) return TK_ERR_ARG;
        int64_t L = std::max<int64_t>(r[j] + p, (int64_t)1 << m);
        std::vector<int64_t> best, cur;
        bool found = false;
        for (;; ++L) {
            factor_rec(L, m, 2, cur, best, found);
            if (found) break;
        }
        for (int k = 0; k < d; ++k) S_out[j * d + k] = 1;
        int t = 0;
        for (int k : ord) {
            if (k == j) continue;
            S_out[j * d + k] = best[t++];
        }
        if (width_out) width_out[j] = L;
    }
    return TK_OK;
}

// ------------------------------------------------------------------ building blocks

}  // extern "C"

extern "C" {  // defined further down, inside the C-ABI block
static void check_outputs(const Tens& X, const int64_t* r, const tk_tensor* G, const tk_matrix* U, Tens& Gt,
                          std::vector<Mat>& Um);
static void check_tucker(const Tens& Gt, const tk_matrix* U, std::vector<Mat>& Um, std::vector<int64_t>& n);
}

// Rows r0 .. r0 + nr - 1 of a column-major matrix (same ld).
static Mat rows_of(const Mat& M, int64_t r0, int64_t nr) {
    Mat v = M;
    v.p = static_cast<const char*>(M.p) + (size_t)r0 * dtype_size(M.dt);
    v.rows = nr;
    return v;
}

// The last mode of X is the slab [off, off + X.n[d-1]) of a mode of length nd
// (nd = X.n[d-1], off = 0 for a whole tensor); a factor of that mode with nd
// rows is used through its slab rows.
static Mat slab_factor(const Mat& M, const Tens& X, int j, int64_t off, int64_t nd, const char* what) {
    const int d = X.d;
    if (j != d - 1 || (off == 0 && nd == X.n[j])) {
        TK_REQUIRE(M.rows == X.n[j], TK_ERR_SHAPE, std::string(what) + ": factor j must have n_j rows");
        return M;
    }
    TK_REQUIRE(M.rows == nd, TK_ERR_SHAPE, std::string(what) + ": the last factor must have the full mode's rows");
    return rows_of(M, off, X.n[j]);
}

static void check_slab(const Tens& X, int64_t off, int64_t nd, const char* what) {
    TK_REQUIRE(X.d >= 2, TK_ERR_SHAPE, std::string(what) + ": d must be >= 2");
    TK_REQUIRE(off >= 0 && nd >= 1 && X.n[X.d - 1] >= 1 && off + X.n[X.d - 1] <= nd, TK_ERR_SHAPE,
               std::string(what) + ": the slab must lie inside the last mode (0 <= offset, offset + rows <= n_d)");
}

// Kronecker sketches of X (Section 4.2) whose last mode is the slab
// [off, off + n) of a mode of length nd: Y[n] for n < d-1 are the slab's
// partial sums of the full sketches (every slab adds to them), Y[d-1] holds
// the slab's rows of the full Y_d.
static void sketch_body(Ctx& c, const tk_tensor* X, int64_t off, int64_t nd, const tk_matrix* Omega, tk_tensor* Y,
                        bool slab) {
    Tens Xt = tens_in(X, "X");
    c.xdata = Xt.p;
    c.df64 = Xt.dt != TK_F64;
    c.xnumel = Xt.numel();
    const int d = Xt.d;
    TK_REQUIRE(d >= 2, TK_ERR_SHAPE, "sketch: d must be >= 2");
    TK_REQUIRE(Omega && Y, TK_ERR_ARG, "sketch: null Omega or Y");
    if (slab) check_slab(Xt, off, nd, "sketch_slab");
    else nd = Xt.n[d - 1];
    tk_dtype acc = acc_of(Xt.dt);
    std::vector<Mat> Om(d);
    std::vector<void*> dst(d);
    for (int j = 0; j < d; ++j) {
        Mat o = slab_factor(mat_in(&Omega[j], "Omega"), Xt, j, off, nd, "sketch");
        TK_REQUIRE(acc == TK_F64 ? o.dt == TK_F64 : o.dt != TK_F64, TK_ERR_DTYPE,
                   "sketch: Omega must be F64 for F64 data, else F32/BF16");
        Om[j] = mat_to(c, o, acc);
    }
    for (int n = 0; n < d; ++n) {
        Tens y = tens_in(&Y[n], "Y");
        TK_REQUIRE(y.d == d && y.dt == acc, TK_ERR_DTYPE, "sketch: Y must have the data's d and F64/F32 dtype");
        for (int j = 0; j < d; ++j)
            TK_REQUIRE(y.n[j] == (j == n ? Xt.n[j] : Om[j].cols), TK_ERR_SHAPE, "sketch: Y[n] has wrong dims");
        dst[n] = y.p;
    }
    std::vector<Tens> Ys(d);
    std::vector<int> all(d);
    std::iota(all.begin(), all.end(), 0);
    all_modes(c, Xt, all, {}, Om.data(), acc, Ys, dst.data());
}

// Core multi-TTM of X whose last mode is the slab [off, off + n) of a mode of
// length nd: the slab's partial sum X_slab x_{j<d} Q_j^T x_d Q_d[slab rows]^T.
static void core_body(Ctx& c, const tk_tensor* X, int64_t off, int64_t nd, const tk_matrix* Q, tk_tensor* G,
                      bool slab) {
    Tens Xt = tens_in(X, "X");
    c.xdata = Xt.p;
    c.df64 = Xt.dt != TK_F64;
    c.xnumel = Xt.numel();
    Tens Gt = tens_in(G, "G");
    const int d = Xt.d;
    TK_REQUIRE(Q != nullptr, TK_ERR_ARG, "core: null Q");
    if (slab) check_slab(Xt, off, nd, "core_slab");
    else nd = Xt.n[d - 1];
    tk_dtype acc = acc_of(Xt.dt);
    TK_REQUIRE(Gt.d == d && (Gt.dt == TK_F64 || Gt.dt == TK_F32), TK_ERR_DTYPE, "core: G must be F64/F32, same d");
    std::vector<Mat> Qm(d);
    std::vector<int> modes(d);
    for (int j = 0; j < d; ++j) {
        Mat q = slab_factor(mat_in(&Q[j], "Q"), Xt, j, off, nd, "core");
        TK_REQUIRE(q.cols == Gt.n[j], TK_ERR_SHAPE, "core: Q_j must be n_j x k_j");
        Qm[j] = mat_to(c, q, acc);
        modes[j] = j;
    }
    bool direct = Gt.dt == acc;
    Tens out = multi_ttm(c, Xt, modes, Qm.data(), false, acc, direct ? Gt.p : nullptr);
    if (!direct) launch_convert(c, out.p, acc, out.numel(), 1, out.numel(), Gt.p, Gt.dt, out.numel(), 1.f);
}

extern "C" {

tk_status tucker_sketch(tk_handle* h, const tk_tensor* X, const tk_matrix* Omega, tk_tensor* Y) {
    return run_call(h, [&](Ctx& c) { sketch_body(c, X, 0, 0, Omega, Y, false); });
}

tk_status tucker_sketch_slab(tk_handle* h, const tk_tensor* X_slab, int64_t offset, int64_t n_last,
                             const tk_matrix* Omega, tk_tensor* Y) {
    return run_call(h, [&](Ctx& c) { sketch_body(c, X_slab, offset, n_last, Omega, Y, true); });
}

tk_status tucker_orth(tk_handle* h, const tk_matrix* Y, tk_matrix* Q, int* info, const tk_opts* opts) {
    tk_status st = run_call(h, [&](Ctx& c) {
        Mat y = mat_in(Y, "Y");
        Mat q = mat_in(Q, "Q");
        Opts o = opts_in(opts, 1);
        set_opts(c, o);
        TK_REQUIRE(y.dt == TK_F64 || y.dt == TK_F32, TK_ERR_DTYPE, "orth: Y must be F64 or F32");
        TK_REQUIRE(q.dt == TK_F64 || q.dt == TK_F32, TK_ERR_DTYPE, "orth: Q must be F64 or F32");
        int64_t k = std::min(y.rows, y.cols);
        TK_REQUIRE(q.rows == y.rows && q.cols == k, TK_ERR_SHAPE, "orth: Q must be rows x min(rows, cols)");
        double* Qd = c.alloc<double>(y.rows * k);
        if (y.cols >= y.rows) {
            launch_fill_identity(c, Qd, y.rows);
            launch_fill_int(c, c.dqr, 1, 2);
        } else {
            orth_one(c, view_rows(y.p, y.dt, y.ld), y.rows, k, Qd, 0);
        }
        launch_convert(c, Qd, TK_F64, y.rows, k, y.rows, (void*)q.p, q.dt, q.ld, 1.f);
    });
    if (st == TK_OK && info) {
        int qr[TK_MAX_D];
        st = tk_sync_status(h, qr);
        *info = qr[0];
    }
    return st;
}

tk_status tk_philox4x32(tk_handle* h, uint64_t seed, uint32_t stream, uint64_t offset, int64_t nblocks,
                        uint32_t* out) {
    return run_call(h, [&](Ctx& c) {
        TK_REQUIRE(nblocks >= 0, TK_ERR_SHAPE, "philox: negative block count");
        TK_REQUIRE(nblocks == 0 || out != nullptr, TK_ERR_ARG, "philox: null output");
        TK_REQUIRE(((uintptr_t)out % 16) == 0, TK_ERR_ALIGN, "philox: output not 16-byte aligned");
        launch_philox_blocks(c, seed, stream, offset, nblocks, out);
    });
}

tk_status tucker_gaussian_factor(tk_handle* h, uint64_t seed, uint32_t stream, tk_matrix* M) {
    return run_call(h, [&](Ctx& c) {
        Mat m = mat_in(M, "M");
        unsigned s = stream;
        launch_gaussian_factors(c, seed, 1, &s, &m);
    });
}

tk_status tucker_gaussian_factors(tk_handle* h, uint64_t seed, int count, const uint32_t* streams, tk_matrix* M) {
    return run_call(h, [&](Ctx& c) {
        TK_REQUIRE(count >= 0 && count <= 64, TK_ERR_ARG, "gaussian factors: 0 <= count <= 64");
        TK_REQUIRE(count == 0 || (streams && M), TK_ERR_ARG, "gaussian factors: null streams or M");
        std::vector<Mat> m(count);
        std::vector<unsigned> st(count);
        for (int f = 0; f < count; ++f) {
            m[f] = mat_in(&M[f], "M");
            st[f] = streams[f];
        }
        launch_gaussian_factors(c, seed, count, st.data(), m.data());
    });
}

tk_status tucker_core(tk_handle* h, const tk_tensor* X, const tk_matrix* Q, tk_tensor* G) {
    return run_call(h, [&](Ctx& c) { core_body(c, X, 0, 0, Q, G, false); });
}

tk_status tucker_core_slab(tk_handle* h, const tk_tensor* X_slab, int64_t offset, int64_t n_last, const tk_matrix* Q,
                           tk_tensor* G) {
    return run_call(h, [&](Ctx& c) { core_body(c, X_slab, offset, n_last, Q, G, true); });
}

tk_status tucker_orth_sketches(tk_handle* h, int d, const tk_tensor* Y, tk_matrix* Q) {
    return run_call(h, [&](Ctx& c) {
        TK_REQUIRE(d >= 1 && d <= TK_MAX_D, TK_ERR_ARG, "orth_sketches: 1 <= d <= TK_MAX_D");
        TK_REQUIRE(Y && Q, TK_ERR_ARG, "orth_sketches: null Y or Q");
        std::vector<Tens> Yt(d);
        std::vector<Mat> Qm(d);
        std::vector<double*> Qd(d);
        std::vector<View2> Yv;
        std::vector<int64_t> nb, kb;
        std::vector<double*> qb;
        std::vector<int> slots;
        bool f32 = true;
        for (int n = 0; n < d; ++n) {
            Yt[n] = tens_in(&Y[n], "Y");
            TK_REQUIRE(Yt[n].d == d, TK_ERR_SHAPE, "orth_sketches: every Y has order d");
            TK_REQUIRE(Yt[n].dt == TK_F64 || Yt[n].dt == TK_F32, TK_ERR_DTYPE, "orth_sketches: Y must be F64/F32");
            f32 = f32 && Yt[n].dt == TK_F32;
        }
        c.df64 = f32;
        launch_fill_int(c, c.dqr, TK_MAX_D, 2);
        for (int n = 0; n < d; ++n) {
            const int64_t nn = Yt[n].n[n], cols = nn ? Yt[n].numel() / nn : 0, k = std::min(nn, cols);
            TK_REQUIRE(nn >= 1 && cols >= 1, TK_ERR_SHAPE, "orth_sketches: empty sketch");
            TK_REQUIRE(k <= 256, TK_ERR_SHAPE, "orth_sketches: sketch width above 256 is not supported");
            Qm[n] = mat_in(&Q[n], "Q");
            TK_REQUIRE(Qm[n].rows == nn && Qm[n].cols == k, TK_ERR_SHAPE, "orth_sketches: Q[n] must be n_n x k_n");
            TK_REQUIRE(Qm[n].dt == TK_F64 || Qm[n].dt == TK_F32, TK_ERR_DTYPE, "orth_sketches: Q must be F64/F32");
            Qd[n] = c.alloc<double>(nn * k);
            if (k < nn) {
                Yv.push_back(view_unfold_rows(Yt[n], n));
                nb.push_back(nn);
                kb.push_back(k);
                qb.push_back(Qd[n]);
                slots.push_back(n);
            } else {
                launch_fill_identity(c, Qd[n], nn);
            }
        }
        orth_batch(c, Yv, nb, kb, qb, slots);
        for (int n = 0; n < d; ++n)
            launch_convert(c, Qd[n], TK_F64, Qm[n].rows, Qm[n].cols, Qm[n].rows, (void*)Qm[n].p, Qm[n].dt, Qm[n].ld,
                           1.f);
    });
}

tk_status tucker_sthosvd(tk_handle* h, const tk_tensor* Ghat, const tk_matrix* Q, const int64_t* r,
                         const tk_opts* opts, tk_tensor* G, tk_matrix* U) {
    return run_call(h, [&](Ctx& c) {
        Tens Gh = tens_in(Ghat, "Ghat", false);
        const int d = Gh.d;
        TK_REQUIRE(Gh.dt == TK_F64 || Gh.dt == TK_F32, TK_ERR_DTYPE, "sthosvd: Ghat must be F64/F32");
        TK_REQUIRE(Q && r && G && U, TK_ERR_ARG, "sthosvd: null argument");
        Opts o = opts_in(opts, d);
        set_opts(c, o);
        c.df64 = Gh.dt != TK_F64;
        Tens dims;  // the tensor's dims, from the factors' rows
        dims.d = d;
        std::vector<double*> Qd(d);
        std::vector<int64_t> k(d);
        for (int j = 0; j < d; ++j) {
            Mat q = mat_in(&Q[j], "Q");
            TK_REQUIRE(q.cols == Gh.n[j] && q.rows >= 1, TK_ERR_SHAPE, "sthosvd: Q_j must be n_j x k_j");
            TK_REQUIRE(r[j] >= 1 && r[j] <= Gh.n[j], TK_ERR_SHAPE, "sthosvd: need 1 <= r_j <= k_j");
            dims.n[j] = q.rows;
            k[j] = q.cols;
            Qd[j] = (double*)mat_to(c, q, TK_F64).p;
        }
        Tens Gt;
        std::vector<Mat> Um;
        check_outputs(dims, r, G, U, Gt, Um);
        Tens G64 = Gh.dt == TK_F64 ? Gh : tens_to(c, Gh, TK_F64);
        std::vector<double*> V;
        Tens Gt64 = sthosvd_core(c, G64, r, o.order, V, Gh.dt == TK_F64);
        finish(c, dims, Qd, k, Gt64, V, r, Gt, Um, nullptr);
    });
}

tk_status tucker_loss_slab(tk_handle* h, const tk_tensor* X_slab, int64_t offset, int64_t n_last, const tk_tensor* G,
                           const tk_matrix* U, double* norms2) {
    double* dev = nullptr;
    tk_status st = run_call(h, [&](Ctx& c) {
        Tens Xt = tens_in(X_slab, "X");
        c.xdata = Xt.p;
        c.df64 = Xt.dt != TK_F64;
        c.xnumel = Xt.numel();
        check_slab(Xt, offset, n_last, "loss_slab");
        Tens Gt = tens_in(G, "G");
        TK_REQUIRE(norms2 != nullptr, TK_ERR_ARG, "loss_slab: null output");
        std::vector<Mat> Um;
        std::vector<int64_t> n;
        check_tucker(Gt, U, Um, n);
        const int d = Xt.d;
        TK_REQUIRE(Gt.d == d, TK_ERR_SHAPE, "loss_slab: X and G must have the same d");
        tk_dtype acc = acc_of(Xt.dt);
        Tens Ga = Gt.dt == acc ? Gt : tens_to(c, Gt, acc);
        std::vector<Mat> Ua(d);
        for (int j = 0; j < d; ++j) Ua[j] = mat_to(c, slab_factor(Um[j], Xt, j, offset, n_last, "loss_slab"), acc);
        dev = c.alloc<double>(2);
        residual_pass(c, Xt, Ga, Ua, acc, dev, nullptr, TK_F32, 0.0);
    });
    if (st != TK_OK) return st;
    if (cudaMemcpyAsync(norms2, dev, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
        h->last_error = "loss_slab: reading the norms failed";
        return TK_ERR_CUDA;
    }
    return TK_OK;
}

// ------------------------------------------------------------------ algorithms

static void check_outputs(const Tens& X, const int64_t* r, const tk_tensor* G, const tk_matrix* U, Tens& Gt,
                          std::vector<Mat>& Um) {
    const int d = X.d;
    Gt = tens_in(G, "G");
    TK_REQUIRE(Gt.d == d && (Gt.dt == TK_F64 || Gt.dt == TK_F32), TK_ERR_DTYPE, "G must be F64/F32 with the data's d");
    TK_REQUIRE(U != nullptr, TK_ERR_ARG, "null U");
    Um.resize(d);
    for (int j = 0; j < d; ++j) {
        TK_REQUIRE(Gt.n[j] == r[j], TK_ERR_SHAPE, "G dims must equal the target ranks");
        Um[j] = mat_in(&U[j], "U");
        TK_REQUIRE(Um[j].rows == X.n[j] && Um[j].cols == r[j], TK_ERR_SHAPE, "U_j must be n_j x r_j");
        TK_REQUIRE(Um[j].dt == TK_F64 || Um[j].dt == TK_F32, TK_ERR_DTYPE, "U must be F64/F32");
    }
}

}  // extern "C"

// Steps 2-4 of Alg. rHKron-re (and of the appendix Alg. rHKron, which differs
// only in its sketches): thin QR of each sketch unfolding (Q = I where the
// sketch is at least as wide as the mode), the core Ghat = X x_j Q_j^T, the FP64
// STHOSVD of the core, U_j = Q_j V_j, and the relative error into errd.
// What the gradient of the loss at the result can reuse: the core's chain of
// products (chain[t] = X x_{modes[0..t]} Q^T, in the order applied), the
// factors V_j (k_j x r_j, FP64, ld k_j) and the column signs of U_j.
// With want_T the call also forms T = X x_{j != m_1} Q_j^T (m_1: the chain's
// first mode, the one product of the gradient the chain does not hold) on the
// side stream while the core is truncated, on a fraction of the SMs; Tapplied
// marks the modes T has applied.
struct CoreTrace {
    std::vector<std::pair<int, Tens>> chain;
    std::vector<double*> V, sg;
    bool want_T = false;
    Tens T;
    std::vector<char> Tapplied;
};

// SMs for a streaming pass that runs beside a latency-bound chain of small
// kernels and has that chain's length to finish in: two thirds of the call's
// (measured on the 512^3 benchmark step: a third starves the pass, all of them
// starve the chain).
static int background_grid(const Ctx& c) {
    const int full = c.grid_sms > 0 ? c.grid_sms : tc::num_sms();
    return std::max(8, 2 * full / 3);
}

static void rhkron_from_sketches(Ctx& c, const Tens& Xt, std::vector<Tens>& Y, const std::vector<int64_t>& k,
                                 const int64_t* r, const Opts& o, const Tens& Gt, const std::vector<Mat>& Um,
                                 double* errd, CoreTrace* tr = nullptr) {
    const int d = Xt.d;
    const tk_dtype acc = acc_of(Xt.dt);
    // 2. thin QR of each sketch unfolding
    std::vector<double*> Qd(d);
    std::vector<View2> Yv;
    std::vector<int64_t> nb, kb;
    std::vector<double*> qb;
    std::vector<int> slots;
    for (int n = 0; n < d; ++n) {
        Qd[n] = c.alloc<double>(Xt.n[n] * k[n]);
        if (k[n] < Xt.n[n]) {
            View2 v = view_unfold_rows(Y[n], n);
            Yv.push_back(v);
            nb.push_back(Xt.n[n]);
            kb.push_back(k[n]);
            qb.push_back(Qd[n]);
            slots.push_back(n);
        } else {
            launch_fill_identity(c, Qd[n], Xt.n[n]);
        }
    }
    launch_fill_int(c, c.dqr, TK_MAX_D, 2);
    orth_batch(c, Yv, nb, kb, qb, slots);
    // 3. core Ghat = X x_j Q_j^T (modes with Q = I are skipped)
    std::vector<Mat> Qa(d);
    std::vector<int> cm;
    for (int j = 0; j < d; ++j) {  // FP64: the TTMs take the factor in the form they read (ttm_to)
        Qa[j].p = Qd[j];
        Qa[j].dt = TK_F64;
        Qa[j].rows = Xt.n[j];
        Qa[j].cols = k[j];
        Qa[j].ld = Xt.n[j];
    }
    for (int j = 0; j < d; ++j)
        if (k[j] < Xt.n[j]) cm.push_back(j);
    Tens Gh = cm.empty() ? Xt : multi_ttm(c, Xt, cm, Qa.data(), false, acc, nullptr, tr ? &tr->chain : nullptr);
    // 4. STHOSVD of the core in FP64, U_j = Q_j V_j, gauge, casts, error
    std::vector<double*> V;
    std::vector<int> tm;
    if (tr && tr->want_T && !tr->chain.empty())
        for (int j : cm)
            if (j != tr->chain[0].first) tm.push_back(j);
    std::function<void()> tpass;
    if (!tm.empty()) {
        tpass = [&]() {
            // the side stream's pass leaves most SMs to the truncation's kernels; the splits it makes
            // are its own (the main stream must not find them in the cache)
            const int keep = c.grid_sms;
            const size_t ns = c.splits.size();
            c.grid_sms = background_grid(c);
            c.background = true;
            tr->T = multi_ttm(c, Xt, tm, Qa.data(), false, acc);
            c.background = false;
            c.grid_sms = keep;
            c.splits.resize(ns);
            tr->Tapplied.assign(d, 0);
            for (int j : tm) tr->Tapplied[j] = 1;
        };
    }
    Tens G64 = (Gh.dt == TK_F64 && Gh.p != Xt.p) ? Gh : tens_to(c, Gh, TK_F64);
    Tens Gt64 = sthosvd_core(c, G64, r, o.order, V, Xt.dt == TK_F64, tpass ? &tpass : nullptr);
    finish(c, Xt, Qd, k, Gt64, V, r, Gt, Um, errd, tr ? &tr->sg : nullptr);
    if (tr) tr->V = V;
}

extern "C" {

tk_status tucker_rhkron(tk_handle* h, const tk_tensor* X, const int64_t* r, int p, const tk_matrix* Omega,
                        const tk_opts* opts, tk_tensor* G, tk_matrix* U, double* rel_err) {
    double* errd = nullptr;
    return run_call(h, [&](Ctx& c) {
        Tens Xt = tens_in(X, "X", false);
        c.xdata = Xt.p;
        c.df64 = Xt.dt != TK_F64;
        c.xnumel = Xt.numel();
        const int d = Xt.d;
        TK_REQUIRE(d >= 2, TK_ERR_SHAPE, "rhkron: d must be >= 2");
        TK_REQUIRE(r && Omega, TK_ERR_ARG, "rhkron: null r or Omega");
        TK_REQUIRE(p >= 0, TK_ERR_ARG, "rhkron: p must be >= 0");
        Opts o = opts_in(opts, d);
        set_opts(c, o);
        tk_dtype acc = acc_of(Xt.dt);
        Tens Gt;
        std::vector<Mat> Um;
        check_outputs(Xt, r, G, U, Gt, Um);
        std::vector<Mat> Om(d);
        std::vector<int64_t> s(d), k(d);
        for (int j = 0; j < d; ++j) {
            Mat om = mat_in(&Omega[j], "Omega");
            TK_REQUIRE(om.rows == Xt.n[j] && om.cols >= 1, TK_ERR_SHAPE, "rhkron: Omega_j must be n_j x s_j");
            TK_REQUIRE(acc == TK_F64 ? om.dt == TK_F64 : om.dt != TK_F64, TK_ERR_DTYPE,
                       "rhkron: Omega must be F64 for F64 data, else F32/BF16");
            s[j] = om.cols;
            Om[j] = mat_to(c, om, acc);
        }
        std::vector<int> need;
        for (int n = 0; n < d; ++n) {
            double w = 1;
            for (int j = 0; j < d; ++j)
                if (j != n) w *= (double)s[j];
            TK_REQUIRE(w >= (double)(r[n] + p), TK_ERR_SHAPE, "rhkron: prod_{j!=n} s_j must be >= r_n + p");
            k[n] = (int64_t)std::min<double>((double)Xt.n[n], w);
            TK_REQUIRE(r[n] >= 1 && r[n] <= k[n], TK_ERR_SHAPE, "rhkron: need 1 <= r_n <= sketch width");
            if (k[n] < Xt.n[n]) need.push_back(n);
        }
        // 1. sketches (dimension tree) for the modes that need a QR
        std::vector<Tens> Y(d);
        if (!need.empty()) {
            std::vector<int> rest;
            for (int j = 0; j < d; ++j)
                if (std::find(need.begin(), need.end(), j) == need.end()) rest.push_back(j);
            all_modes(c, Xt, need, rest, Om.data(), acc, Y, nullptr);
        }
        if (rel_err) errd = c.alloc<double>(2);
        rhkron_from_sketches(c, Xt, Y, k, r, o, Gt, Um, errd);
        if (rel_err) read_err(h, c, errd, rel_err, false, o.async_outputs);
    });
}

tk_status tucker_rhkron_srht(tk_handle* h, const tk_tensor* X, const int64_t* r, int p, const tk_matrix* Omega,
                             uint64_t seed, const tk_opts* opts, tk_tensor* G, tk_matrix* U, double* rel_err) {
    double* errd = nullptr;
    return run_call(h, [&](Ctx& c) {
        Tens Xt = tens_in(X, "X", false);
        c.xdata = Xt.p;
        c.df64 = Xt.dt != TK_F64;
        c.xnumel = Xt.numel();
        const int d = Xt.d;
        TK_REQUIRE(d >= 2, TK_ERR_SHAPE, "rhkron_srht: d must be >= 2");
        TK_REQUIRE(r && Omega, TK_ERR_ARG, "rhkron_srht: null r or Omega");
        TK_REQUIRE(p >= 0, TK_ERR_ARG, "rhkron_srht: p must be >= 0");
        Opts o = opts_in(opts, d);
        set_opts(c, o);
        tk_dtype acc = acc_of(Xt.dt);
        Tens Gt;
        std::vector<Mat> Um;
        check_outputs(Xt, r, G, U, Gt, Um);
        std::vector<Mat> Om(d);
        std::vector<int64_t> s(d), k(d);
        for (int j = 0; j < d; ++j) {
            Mat om = mat_in(&Omega[j], "Omega");
            TK_REQUIRE(om.rows == Xt.n[j] && om.cols >= 1, TK_ERR_SHAPE, "rhkron_srht: Omega_j must be n_j x s_j");
            TK_REQUIRE(acc == TK_F64 ? om.dt == TK_F64 : om.dt != TK_F64, TK_ERR_DTYPE,
                       "rhkron_srht: Omega must be F64 for F64 data, else F32/BF16");
            s[j] = om.cols;
            Om[j] = mat_to(c, om, acc);
        }
        std::vector<int> need;
        for (int n = 0; n < d; ++n) {
            double w = 1;
            for (int j = 0; j < d; ++j)
                if (j != n) w *= (double)s[j];
            TK_REQUIRE(w >= (double)(r[n] + p), TK_ERR_SHAPE, "rhkron_srht: prod_{j!=n} s_j must be >= r_n + p");
            TK_REQUIRE(Xt.numel() / std::max<int64_t>(1, Xt.n[n]) < ((int64_t)1 << 32), TK_ERR_SHAPE,
                       "rhkron_srht: the mode-n unfolding needs fewer than 2^32 columns");
            k[n] = (int64_t)std::min<double>((double)Xt.n[n], w);
            TK_REQUIRE(r[n] >= 1 && r[n] <= k[n], TK_ERR_SHAPE, "rhkron_srht: need 1 <= r_n <= sketch width");
            if (k[n] < Xt.n[n]) need.push_back(n);
        }
        // 1. Y_n = X_(n) D_n (kron_{j != n} H_j): D_n is applied to X as it is streamed by the first
        // product (the narrow FP32 kernel), else to a sign-flipped copy of X
        std::vector<Tens> Y(d);
        void* flipped = nullptr;
        for (int n : need) {
            int j0 = -1;
            double best = 1e300;
            for (int j = 0; j < d; ++j) {
                if (j == n) continue;
                const double ratio = (double)s[j] / std::max<double>(1.0, (double)Xt.n[j]);
                if (ratio < best - 1e-15 || (std::fabs(ratio - best) <= 1e-15 && j > j0)) {
                    best = ratio;
                    j0 = j;
                }
            }
            Tens T1;
            if (c.use_tc && ttm_narrow_eligible(Xt, j0, s[j0], acc)) {
                T1 = Xt;
                T1.n[j0] = s[j0];
                T1.dt = acc;
                T1.scale = 1.f;
                T1.p = c.alloc_bytes(dtype_size(acc) * T1.numel());
                const SignMap sm = sign_map(Xt, n, j0, seed);
                launch_ttm_narrow(c, Xt, j0, Om[j0], false, s[j0], static_cast<float*>(T1.p), &sm);
            } else {
                if (!flipped) flipped = c.alloc_bytes(dtype_size(Xt.dt) * Xt.numel());
                launch_sign_copy(c, Xt, n, seed, flipped);
                Tens Xs = Xt;
                Xs.p = flipped;
                T1 = ttm_to(c, Xs, j0, Om[j0], false, acc);
            }
            std::vector<int> rest;
            for (int j = 0; j < d; ++j)
                if (j != n && j != j0) rest.push_back(j);
            Y[n] = rest.empty() ? T1 : multi_ttm(c, T1, rest, Om.data(), false, acc);
        }
        if (rel_err) errd = c.alloc<double>(2);
        rhkron_from_sketches(c, Xt, Y, k, r, o, Gt, Um, errd);
        if (rel_err) read_err(h, c, errd, rel_err, false, o.async_outputs);
    });
}

tk_status tucker_rhkron_noreuse(tk_handle* h, const tk_tensor* X, const int64_t* r, int p, const tk_matrix* Omega,
                                const tk_opts* opts, tk_tensor* G, tk_matrix* U, double* rel_err) {
    double* errd = nullptr;
    return run_call(h, [&](Ctx& c) {
        Tens Xt = tens_in(X, "X", false);
        c.xdata = Xt.p;
        c.df64 = Xt.dt != TK_F64;
        c.xnumel = Xt.numel();
        const int d = Xt.d;
        TK_REQUIRE(d >= 2, TK_ERR_SHAPE, "rhkron_noreuse: d must be >= 2");
        TK_REQUIRE(r && Omega, TK_ERR_ARG, "rhkron_noreuse: null r or Omega");
        TK_REQUIRE(p >= 0, TK_ERR_ARG, "rhkron_noreuse: p must be >= 0");
        Opts o = opts_in(opts, d);
        set_opts(c, o);
        tk_dtype acc = acc_of(Xt.dt);
        Tens Gt;
        std::vector<Mat> Um;
        check_outputs(Xt, r, G, U, Gt, Um);
        std::vector<int64_t> k(d);
        std::vector<Tens> Y(d);
        for (int n = 0; n < d; ++n) {
            // Y_n = X x_{j != n} Phi_{n,j} with fresh factors per mode (no shared tree)
            std::vector<Mat> Om(d);
            std::vector<int> modes;
            double w = 1;
            for (int j = 0; j < d; ++j) {
                if (j == n) continue;
                Mat om = mat_in(&Omega[n * d + j], "Omega");
                TK_REQUIRE(om.rows == Xt.n[j] && om.cols >= 1, TK_ERR_SHAPE,
                           "rhkron_noreuse: Omega_{n,j} must be n_j x s_{n,j}");
                TK_REQUIRE(acc == TK_F64 ? om.dt == TK_F64 : om.dt != TK_F64, TK_ERR_DTYPE,
                           "rhkron_noreuse: Omega must be F64 for F64 data, else F32/BF16");
                w *= (double)om.cols;
                Om[j] = mat_to(c, om, acc);
                modes.push_back(j);
            }
            TK_REQUIRE(w >= (double)(r[n] + p), TK_ERR_SHAPE,
                       "rhkron_noreuse: prod_{j!=n} s_{n,j} must be >= r_n + p");
            k[n] = (int64_t)std::min<double>((double)Xt.n[n], w);
            TK_REQUIRE(r[n] >= 1 && r[n] <= k[n], TK_ERR_SHAPE, "rhkron_noreuse: need 1 <= r_n <= sketch width");
            if (k[n] < Xt.n[n]) Y[n] = multi_ttm(c, Xt, modes, Om.data(), false, acc);
        }
        if (rel_err) errd = c.alloc<double>(2);
        rhkron_from_sketches(c, Xt, Y, k, r, o, Gt, Um, errd);
        if (rel_err) read_err(h, c, errd, rel_err, false, o.async_outputs);
    });
}

tk_status tucker_rsthkron(tk_handle* h, const tk_tensor* X, const int64_t* r, int p, const tk_matrix* Omega,
                          const tk_opts* opts, tk_tensor* G, tk_matrix* U, double* rel_err) {
    double* errd = nullptr;
    return run_call(h, [&](Ctx& c) {
        Tens Xt = tens_in(X, "X", false);
        c.xdata = Xt.p;
        c.df64 = Xt.dt != TK_F64;
        c.xnumel = Xt.numel();
        const int d = Xt.d;
        TK_REQUIRE(d >= 2, TK_ERR_SHAPE, "rsthkron: d must be >= 2");
        TK_REQUIRE(r && Omega, TK_ERR_ARG, "rsthkron: null r or Omega");
        TK_REQUIRE(p >= 0, TK_ERR_ARG, "rsthkron: p must be >= 0");
        Opts o = opts_in(opts, d);
        set_opts(c, o);
        tk_dtype acc = acc_of(Xt.dt);
        Tens Gt;
        std::vector<Mat> Um;
        check_outputs(Xt, r, G, U, Gt, Um);
        launch_fill_int(c, c.dqr, TK_MAX_D, 2);
        Tens Gh = Xt;
        std::vector<int64_t> cur(Xt.n, Xt.n + d), k(d);
        std::vector<double*> Qd(d);
        for (int j : o.order) {
            std::vector<Mat> Om(d);
            std::vector<int> modes;
            double w = 1;
            for (int kk = 0; kk < d; ++kk) {
                if (kk == j) continue;
                Mat om = mat_in(&Omega[j * d + kk], "Omega");
                TK_REQUIRE(om.rows == cur[kk] && om.cols >= 1, TK_ERR_SHAPE,
                           "rsthkron: Omega[j*d+k] must be (current size of mode k) x s_{j,k}");
                TK_REQUIRE(acc == TK_F64 ? om.dt == TK_F64 : om.dt != TK_F64, TK_ERR_DTYPE,
                           "rsthkron: Omega must be F64 for F64 data, else F32/BF16");
                Om[kk] = mat_to(c, om, acc);
                modes.push_back(kk);
                w *= (double)om.cols;
            }
            TK_REQUIRE(w >= (double)(r[j] + p), TK_ERR_SHAPE, "rsthkron: prod_k s_{j,k} must be >= r_j + p");
            k[j] = (int64_t)std::min<double>((double)Xt.n[j], w);
            TK_REQUIRE(r[j] >= 1 && r[j] <= k[j], TK_ERR_SHAPE, "rsthkron: need 1 <= r_j <= sketch width");
            Qd[j] = c.alloc<double>(Xt.n[j] * k[j]);
            if (k[j] < Xt.n[j]) {
                Tens Y = multi_ttm(c, Gh, modes, Om.data(), false, acc);
                orth_one(c, view_unfold_rows(Y, j), Xt.n[j], k[j], Qd[j], j);
                Mat qm;
                qm.p = Qd[j];
                qm.dt = TK_F64;
                qm.rows = Xt.n[j];
                qm.cols = k[j];
                qm.ld = Xt.n[j];
                // the tensor-core TTM splits an FP64 factor into TF32 parts itself: no FP32 copy needed
                const bool tc64 = c.use_tc && !ttm_narrow_eligible(Gh, j, k[j], acc) && ttm_tc_eligible(Gh, j, k[j], acc);
                Mat qa = (acc == TK_F64 || tc64) ? qm : mat_to(c, qm, acc);
                Gh = ttm_to(c, Gh, j, qa, false, acc);
            } else {
                launch_fill_identity(c, Qd[j], Xt.n[j]);
            }
            cur[j] = k[j];
        }
        Tens G64 = (Gh.dt == TK_F64 && Gh.p != Xt.p) ? Gh : tens_to(c, Gh, TK_F64);
        std::vector<double*> V;
        Tens Gt64 = sthosvd_core(c, G64, r, o.order, V, Xt.dt == TK_F64);
        if (rel_err) errd = c.alloc<double>(2);
        finish(c, Xt, Qd, k, Gt64, V, r, Gt, Um, rel_err ? errd : nullptr);
        if (rel_err) read_err(h, c, errd, rel_err, false, o.async_outputs);
    });
}

// ------------------------------------------------------------------ reconstruction, loss, gradient

static Tens reconstruct_acc(Ctx& c, const Tens& Gt, const std::vector<Mat>& Um, tk_dtype acc, void* dst) {
    const int d = Gt.d;
    Tens Ga = Gt.dt == acc ? Gt : tens_to(c, Gt, acc);
    std::vector<Mat> Ua(d);
    for (int j = 0; j < d; ++j) Ua[j] = Um[j].dt == acc ? Um[j] : mat_to(c, Um[j], acc);
    std::vector<int> todo(d);
    std::iota(todo.begin(), todo.end(), 0);
    Tens cur = Ga;
    while (!todo.empty()) {
        size_t best = 0;
        double bestr = 1e300;
        for (size_t t = 0; t < todo.size(); ++t) {
            int i = todo[t];
            double ratio = (double)Ua[i].rows / std::max<double>(1.0, (double)Ua[i].cols);
            if (ratio < bestr) { bestr = ratio; best = t; }
        }
        int i = todo[best];
        todo.erase(todo.begin() + best);
        cur = ttm_to(c, cur, i, Ua[i], true, acc, todo.empty() ? dst : nullptr);
    }
    return cur;
}

static void check_tucker(const Tens& Gt, const tk_matrix* U, std::vector<Mat>& Um, std::vector<int64_t>& n) {
    const int d = Gt.d;
    TK_REQUIRE(Gt.dt == TK_F64 || Gt.dt == TK_F32, TK_ERR_DTYPE, "G must be F64/F32");
    TK_REQUIRE(U != nullptr, TK_ERR_ARG, "null U");
    Um.resize(d);
    n.resize(d);
    for (int j = 0; j < d; ++j) {
        Um[j] = mat_in(&U[j], "U");
        TK_REQUIRE(Um[j].cols == Gt.n[j], TK_ERR_SHAPE, "U_j must have r_j columns");
        TK_REQUIRE(Um[j].dt == TK_F64 || Um[j].dt == TK_F32, TK_ERR_DTYPE, "U must be F64/F32");
        n[j] = Um[j].rows;
    }
}

tk_status tucker_reconstruct(tk_handle* h, const tk_tensor* G, const tk_matrix* U, tk_tensor* Xhat) {
    return run_call(h, [&](Ctx& c) {
        Tens Gt = tens_in(G, "G");
        Tens Xh = tens_in(Xhat, "Xhat");
        std::vector<Mat> Um;
        std::vector<int64_t> n;
        check_tucker(Gt, U, Um, n);
        TK_REQUIRE(Xh.d == Gt.d, TK_ERR_SHAPE, "reconstruct: Xhat must have G's d");
        TK_REQUIRE(Xh.dt == TK_F64 || Xh.dt == TK_F32, TK_ERR_DTYPE, "reconstruct: Xhat must be F64/F32");
        for (int j = 0; j < Gt.d; ++j) TK_REQUIRE(Xh.n[j] == n[j], TK_ERR_SHAPE, "reconstruct: Xhat dims != U rows");
        reconstruct_acc(c, Gt, Um, Xh.dt, Xh.p);
    });
}

tk_status tucker_loss(tk_handle* h, const tk_tensor* X, const tk_tensor* G, const tk_matrix* U, double* loss) {
    double* dev = nullptr;
    return run_call(h, [&](Ctx& c) {
        Tens Xt = tens_in(X, "X");
        c.xdata = Xt.p;
        c.df64 = Xt.dt != TK_F64;
        c.xnumel = Xt.numel();
        Tens Gt = tens_in(G, "G");
        TK_REQUIRE(loss != nullptr, TK_ERR_ARG, "loss: null output");
        std::vector<Mat> Um;
        std::vector<int64_t> n;
        check_tucker(Gt, U, Um, n);
        TK_REQUIRE(Xt.d == Gt.d, TK_ERR_SHAPE, "loss: X and G must have the same d");
        for (int j = 0; j < Xt.d; ++j) TK_REQUIRE(Xt.n[j] == n[j], TK_ERR_SHAPE, "loss: X dims != U rows");
        tk_dtype acc = acc_of(Xt.dt);
        Tens Ga = Gt.dt == acc ? Gt : tens_to(c, Gt, acc);
        std::vector<Mat> Ua(Xt.d);
        for (int j = 0; j < Xt.d; ++j) Ua[j] = Um[j].dt == acc ? Um[j] : mat_to(c, Um[j], acc);
        dev = c.alloc<double>(2);
        residual_pass(c, Xt, Ga, Ua, acc, dev, nullptr, TK_F32, 0.0);
        read_err(h, c, dev, loss, true);
    });
}

}  // extern "C"

// ------------------------------------------------------------------ gradient of the loss
// The gradient outputs, checked against X (dims n) and G.
struct GradOut {
    Tens dG, dX;
    std::vector<Mat> dU;
};

static GradOut grad_outputs_in(const Tens& Xt, const Tens& Gt, const std::vector<int64_t>& n, tk_tensor* dG,
                               tk_matrix* dU, tk_tensor* dX) {
    const int d = Xt.d;
    GradOut g;
    if (dG) {
        g.dG = tens_in(dG, "dG");
        TK_REQUIRE(g.dG.d == d && (g.dG.dt == TK_F64 || g.dG.dt == TK_F32), TK_ERR_DTYPE,
                   "backward: dG must be F64/F32");
        for (int j = 0; j < d; ++j) TK_REQUIRE(g.dG.n[j] == Gt.n[j], TK_ERR_SHAPE, "backward: dG dims != G dims");
    }
    g.dU.resize(d);
    if (dU) {
        for (int j = 0; j < d; ++j) {
            g.dU[j] = mat_in(&dU[j], "dU");
            TK_REQUIRE(g.dU[j].rows == n[j] && g.dU[j].cols == Gt.n[j], TK_ERR_SHAPE,
                       "backward: dU_j must be n_j x r_j");
            TK_REQUIRE(g.dU[j].dt == TK_F64 || g.dU[j].dt == TK_F32, TK_ERR_DTYPE, "backward: dU must be F64/F32");
        }
    }
    if (dX) {
        g.dX = tens_in(dX, "dX");
        TK_REQUIRE(g.dX.d == d && g.dX.dt == Xt.dt, TK_ERR_DTYPE, "backward: dX must have X's dims and dtype");
        for (int j = 0; j < d; ++j) TK_REQUIRE(g.dX.n[j] == Xt.n[j], TK_ERR_SHAPE, "backward: dX dims != X dims");
    }
    return g;
}

// dG and dU from S_n = X x_{j!=n} U_j^T (n = 0..d-1).  With R = X - G x_j U_j
// and C_j = U_j^T U_j:
//   R x_{j!=n} U_j^T = S_n - G x_n U_n x_{j!=n} C_j,
// so every product with the residual comes from the S_n plus small core-sized
// corrections in FP64.  Gt / Um: G and U as given (F64/F32); Ua: U in the
// accumulation dtype.
static void grad_from_sketches(Ctx& c, const Tens& Gt, const std::vector<Mat>& Um, const std::vector<Mat>& Ua,
                               const std::vector<int64_t>& n, std::vector<Tens>& S, tk_dtype acc, double grad_scale,
                               bool want_dG, bool want_dU, GradOut& g) {
    const int d = Gt.d;
    const double s2 = -2.0 * grad_scale;
    Tens G64 = Gt.dt == TK_F64 ? Gt : tens_to(c, Gt, TK_F64);
    std::vector<double*> U64(d);
    std::vector<Mat> Cm(d);
    c.fork(d, [&](int j) {
        const int64_t nj = n[j], rj = Gt.n[j];
        U64[j] = c.alloc<double>(nj * rj);
        launch_convert(c, Um[j].p, Um[j].dt, nj, rj, Um[j].ld, U64[j], TK_F64, nj, 1.f);
        double* Cj = c.alloc<double>(rj * rj);
        gemm_nt_f64(c, rj, rj, nj, view_cols(U64[j], TK_F64, nj), view_cols(U64[j], TK_F64, nj), 1.0, 0.0, Cj, rj);
        Cm[j].p = Cj;
        Cm[j].dt = TK_F64;
        Cm[j].rows = rj;
        Cm[j].cols = rj;
        Cm[j].ld = rj;
    });
    std::vector<Tens> Pm(d);  // P_n = G x_{j != n} C_j: one short chain per mode, side by side
    c.fork(d, [&](int n) {
        std::vector<int> modes;
        for (int j = 0; j < d; ++j)
            if (j != n) modes.push_back(j);
        Pm[n] = multi_ttm(c, G64, modes, Cm.data(), false, TK_F64);
    });
    // dU_n per mode and dG are independent: item j < d is dU_j, item d is dG
    const int ndu = want_dU ? d : 0;
    c.fork(ndu + (want_dG ? 1 : 0), [&](int j) {
        if (j == ndu) {
            // dG = -2s (X x_j U_j^T - G x_j C_j) = -2s (S_0 x_0 U_0^T - P_0 x_0 C_0)
            Tens E = ttm_to(c, S[0], 0, Ua[0], false, acc);
            Tens F = ttm_to(c, Pm[0], 0, Cm[0], false, TK_F64);
            launch_axpby_residual(c, E, F.p, TK_F64, s2, g.dG.p, g.dG.dt);
            return;
        }
        const int64_t nj = n[j], rj = Gt.n[j];
        int64_t K = 1;
        for (int i = 0; i < d; ++i)
            if (i != j) K *= Gt.n[i];
        double* A1 = c.alloc<double>(nj * rj);
        double* B1 = c.alloc<double>(rj * rj);
        // S_n carries the FP32 rounding of the sketch pass, far above double-float accumulation error,
        // so for FP32 data this product (the largest of the gradient) runs on the FP32 pipe
        gemm_nt_f64(c, nj, rj, K, view_unfold_rows(S[j], j), view_unfold_rows(Gt.dt == TK_F32 ? Gt : G64, j), s2,
                    0.0, A1, nj, nullptr, true);
        gemm_nt_f64(c, rj, rj, K, view_unfold_rows(Pm[j], j), view_unfold_rows(G64, j), 1.0, 0.0, B1, rj);
        gemm_nt_f64(c, nj, rj, rj, view_rows(U64[j], TK_F64, nj), view_cols(B1, TK_F64, rj), -s2, 1.0, A1, nj);
        launch_convert(c, A1, TK_F64, nj, rj, nj, (void*)g.dU[j].p, g.dU[j].dt, g.dU[j].ld, 1.f);
    });
}

extern "C" {

tk_status tucker_reconstruct_backward(tk_handle* h, const tk_tensor* X, const tk_tensor* G, const tk_matrix* U,
                                      double grad_scale, tk_tensor* dG, tk_matrix* dU, tk_tensor* dX,
                                      double* norms2) {
    return run_call(h, [&](Ctx& c) {
        Tens Xt = tens_in(X, "X");
        c.xdata = Xt.p;
        c.df64 = Xt.dt != TK_F64;
        c.xnumel = Xt.numel();
        Tens Gt = tens_in(G, "G");
        const int d = Xt.d;
        std::vector<Mat> Um;
        std::vector<int64_t> n;
        check_tucker(Gt, U, Um, n);
        TK_REQUIRE(Xt.d == Gt.d && d >= 2, TK_ERR_SHAPE, "backward: X and G must have the same d >= 2");
        for (int j = 0; j < d; ++j) TK_REQUIRE(Xt.n[j] == n[j], TK_ERR_SHAPE, "backward: X dims != U rows");
        TK_REQUIRE(dG || dU || dX || norms2, TK_ERR_ARG, "backward: no output requested");
        TK_REQUIRE(((uintptr_t)norms2 & 7) == 0, TK_ERR_ARG, "backward: norms2 must be 8-byte aligned");
        GradOut g = grad_outputs_in(Xt, Gt, n, dG, dU, dX);
        tk_dtype acc = acc_of(Xt.dt);
        std::vector<Mat> Ua(d);
        for (int j = 0; j < d; ++j) Ua[j] = Um[j].dt == acc ? Um[j] : mat_to(c, Um[j], acc);
        if (dG || dU) {
            // the S_n by the dimension tree (recomputed, never stored across calls)
            std::vector<Tens> S(d);
            std::vector<int> all(d);
            std::iota(all.begin(), all.end(), 0);
            all_modes(c, Xt, all, {}, Ua.data(), acc, S, nullptr);
            grad_from_sketches(c, Gt, Um, Ua, n, S, acc, grad_scale, dG != nullptr, dU != nullptr, g);
        }
        if (dX || norms2) {
            // dX and the norms from one fused residual pass (the residual is only formed, tile by tile,
            // for them)
            Tens Ga = Gt.dt == acc ? Gt : tens_to(c, Gt, acc);
            double* nrm = norms2 ? norms2 : c.alloc<double>(2);
            residual_pass(c, Xt, Ga, Ua, acc, nrm, dX ? g.dX.p : nullptr, dX ? g.dX.dt : TK_F32, 2.0 * grad_scale);
        }
    });
}

tk_status tucker_rhkron_grad(tk_handle* h, const tk_tensor* X, const int64_t* r, int p, const tk_matrix* Omega,
                             const tk_opts* opts, tk_tensor* G, tk_matrix* U, double* rel_err, double grad_scale,
                             tk_tensor* dG, tk_matrix* dU, tk_tensor* dX) {
    double* errd = nullptr;
    return run_call(h, [&](Ctx& c) {
        Tens Xt = tens_in(X, "X", false);
        c.xdata = Xt.p;
        c.df64 = Xt.dt != TK_F64;
        c.xnumel = Xt.numel();
        const int d = Xt.d;
        TK_REQUIRE(d >= 2, TK_ERR_SHAPE, "rhkron_grad: d must be >= 2");
        TK_REQUIRE(r && Omega, TK_ERR_ARG, "rhkron_grad: null r or Omega");
        TK_REQUIRE(p >= 0, TK_ERR_ARG, "rhkron_grad: p must be >= 0");
        Opts o = opts_in(opts, d);
        set_opts(c, o);
        tk_dtype acc = acc_of(Xt.dt);
        Tens Gt;
        std::vector<Mat> Um;
        check_outputs(Xt, r, G, U, Gt, Um);
        std::vector<int64_t> n(Xt.n, Xt.n + d);
        GradOut g = grad_outputs_in(Xt, Gt, n, dG, dU, dX);
        std::vector<Mat> Om(d);
        std::vector<int64_t> s(d), k(d);
        for (int j = 0; j < d; ++j) {
            Mat om = mat_in(&Omega[j], "Omega");
            TK_REQUIRE(om.rows == Xt.n[j] && om.cols >= 1, TK_ERR_SHAPE, "rhkron_grad: Omega_j must be n_j x s_j");
            TK_REQUIRE(acc == TK_F64 ? om.dt == TK_F64 : om.dt != TK_F64, TK_ERR_DTYPE,
                       "rhkron_grad: Omega must be F64 for F64 data, else F32/BF16");
            s[j] = om.cols;
            Om[j] = mat_to(c, om, acc);
        }
        std::vector<int> need;
        for (int m = 0; m < d; ++m) {
            double w = 1;
            for (int j = 0; j < d; ++j)
                if (j != m) w *= (double)s[j];
            TK_REQUIRE(w >= (double)(r[m] + p), TK_ERR_SHAPE, "rhkron_grad: prod_{j!=n} s_j must be >= r_n + p");
            k[m] = (int64_t)std::min<double>((double)Xt.n[m], w);
            TK_REQUIRE(r[m] >= 1 && r[m] <= k[m], TK_ERR_SHAPE, "rhkron_grad: need 1 <= r_n <= sketch width");
            if (k[m] < Xt.n[m]) need.push_back(m);
        }
        // 1-4. rHKron-re (sketches, QR, core, STHOSVD), keeping the core's chain of products
        std::vector<Tens> Y(d);
        if (!need.empty()) {
            std::vector<int> rest;
            for (int j = 0; j < d; ++j)
                if (std::find(need.begin(), need.end(), j) == need.end()) rest.push_back(j);
            all_modes(c, Xt, need, rest, Om.data(), acc, Y, nullptr);
        }
        CoreTrace tr;
        tr.want_T = dG || dU;
        rhkron_from_sketches(c, Xt, Y, k, r, o, Gt, Um, nullptr, &tr);
        // 5. the gradient at the result (G, U).  U_j = Q_j V_j' (V_j' = V_j with U_j's column signs), so
        // for the core's chain C_t = X x_{m_1..m_t} Q^T (m_1, m_2, .. the modes in the order applied)
        //   S_n = X x_{j!=n} U_j^T = C_t x_{j in m_1..m_t} V_j'^T x_{other j != n} U_j^T,
        // C_t the last product in which mode n is still whole.  S_{m_1} = T x_{j != m_1} V_j'^T with
        // T = X x_{j != m_1} Q_j^T, the one further pass over X, made beside the truncation (it needs
        // only the Q_j); the other S_n read the much smaller products of the chain.  The residual pass
        // (dX, and the norms of the relative error) runs beside them on the side stream.
        std::vector<Mat> Ua(d);
        for (int j = 0; j < d; ++j) Ua[j] = Um[j].dt == acc ? Um[j] : mat_to(c, Um[j], acc);
        Tens Ga = Gt.dt == acc ? Gt : tens_to(c, Gt, acc);
        const bool want_res = dX || rel_err;
        if (want_res) errd = c.alloc<double>(2);
        std::vector<Mat> Va(d);
        if (dG || dU) {
            c.fork(d, [&](int j) {
                double* sgn[2] = {nullptr, tr.sg[j]};
                Tens sh;
                sh.d = 2;
                sh.n[0] = k[j];
                sh.n[1] = r[j];
                launch_apply_signs(c, tr.V[j], sh, sgn);
                Va[j].p = tr.V[j];  // FP64: the TTMs take the factor in the form they read (ttm_to)
                Va[j].dt = TK_F64;
                Va[j].rows = k[j];
                Va[j].cols = r[j];
                Va[j].ld = k[j];
            });
        }
        c.side(
            [&]() {
                if (!dG && !dU) return;
                std::vector<Tens> S(d);
                c.fork(d, [&](int m) {
                    Tens C = Xt;
                    std::vector<char> applied(d, 0);
                    if (tr.T.p && m == tr.chain[0].first) {  // formed beside the truncation
                        C = tr.T;
                        applied = tr.Tapplied;
                    } else {
                        for (const auto& st : tr.chain) {
                            if (st.first == m) break;
                            C = st.second;
                            applied[st.first] = 1;
                        }
                    }
                    std::vector<Mat> M(d);
                    std::vector<int> modes;
                    for (int j = 0; j < d; ++j) {
                        if (j == m) continue;
                        M[j] = applied[j] ? Va[j] : Ua[j];
                        modes.push_back(j);
                    }
                    S[m] = multi_ttm(c, C, modes, M.data(), false, acc);
                });
                grad_from_sketches(c, Gt, Um, Ua, n, S, acc, grad_scale, dG != nullptr, dU != nullptr, g);
            },
            [&]() {
                if (!want_res) return;
                // the pass has the gradient's chain of small kernels to finish in: it leaves them SMs
                const int keep = c.grid_sms;
                if (dG || dU) {
                    c.grid_sms = background_grid(c);
                    c.background = true;
                }
                residual_pass(c, Xt, Ga, Ua, acc, errd, dX ? g.dX.p : nullptr, dX ? g.dX.dt : TK_F32,
                              2.0 * grad_scale);
                c.background = false;
                c.grid_sms = keep;
            });
        if (rel_err) read_err(h, c, errd, rel_err, false, o.async_outputs);
    });
}

}  // extern "C"
