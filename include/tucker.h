/*
 * tucker.h -- C ABI of libtucker, a GB300 (sm_103a) implementation of the
 * randomized Tucker decompositions of "Parallel Randomized Tucker
 * Decomposition Algorithms" (arXiv 2211.13028): rHKron-re (Section 4.3,
 * Algorithm rHKron-re) and rSTHKron (Section 4.2, Algorithm rSTHKron), their
 * building blocks (Kronecker sketch multi-TTM, thin QR of a sketch, core
 * multi-TTM, core truncation) and the reconstruction loss with its gradient.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Tensors are dense and column-major: mode 1 varies fastest, element
 *    (i1,...,id) sits at i1 + n1*(i2 + n2*(i3 + ...)).  The mode-j unfolding
 *    X_(j) is n_j x prod_{k!=j} n_k with the remaining modes in the same
 *    order (Section 2.1).
 *  - Matrices are column-major with leading dimension ld >= rows.
 *  - Every data pointer in tk_tensor / tk_matrix is a DEVICE pointer owned by
 *    the caller; the library never frees it.  Outputs must not alias inputs.
 *  - Scalar results (rel_err, loss, info) are written to HOST memory; an entry
 *    point with a host result synchronises the handle's stream before it
 *    returns.  All other work is queued asynchronously on that stream.
 *  - Sketch factors are inputs: Omega_j = Phi_j^T (n_j x s_j), drawn by the
 *    caller, so any generator (and the tests' FP64 oracle) sees the same values.
 *  - A call validates shapes, dtypes, strides and alignment before it queues
 *    any work and returns a non-zero tk_status on the first violation, with a
 *    message available from tk_last_error().  No C++ exception crosses the ABI.
 *  - Numerical conditions found on the device (a Cholesky breakdown that sent a
 *    QR to the Householder fallback, a Jacobi solve that hit its sweep limit)
 *    are recorded in the handle and reported by tk_sync_status().
 *  - The handle owns a device workspace that grows on demand (cudaMalloc).
 *    A handle must not be used from two host threads at once.
 */
#ifndef TUCKER_H
#define TUCKER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TK_MAX_D 8

#if defined(__GNUC__)
#define TK_API __attribute__((visibility("default")))
#else
#define TK_API
#endif

typedef enum {
    TK_OK = 0,
    TK_ERR_ARG = 1,           /* null pointer, bad option or count            */
    TK_ERR_SHAPE = 2,         /* inconsistent or unsupported sizes            */
    TK_ERR_DTYPE = 3,         /* dtype combination not supported              */
    TK_ERR_ALIGN = 4,         /* pointer or leading dimension misaligned      */
    TK_ERR_WORKSPACE = 5,     /* workspace allocation failed                  */
    TK_ERR_CUDA = 6,          /* a CUDA runtime call failed                   */
    TK_ERR_NOT_CONVERGED = 7, /* Jacobi eigensolver hit its sweep limit        */
    TK_ERR_TIMEOUT = 8        /* a bounded device wait gave up                */
} tk_status;

typedef enum { TK_F64 = 0, TK_F32 = 1, TK_BF16 = 2, TK_FP8_E4M3 = 3 } tk_dtype;

/* Dense column-major tensor on the device.  For TK_FP8_E4M3 the stored value
 * q represents q / scale (scale > 0); scale is ignored for other dtypes. */
typedef struct {
    int d;
    int64_t dims[TK_MAX_D];
    tk_dtype dtype;
    void* data;
    float scale;
} tk_tensor;

/* Column-major matrix on the device, element (i, j) at data[i + j*ld]. */
typedef struct {
    int64_t rows, cols, ld;
    tk_dtype dtype;
    void* data;
} tk_matrix;

/* Options; a zero-initialised struct selects the defaults.
 *  mode_order        processing order of the modes (0-based, d entries) for
 *                    rSTHKron and for the final STHOSVD of the core; NULL = 0..d-1.
 *  qr_method         0 = CholeskyQR2 with Householder fallback on breakdown,
 *                    1 = always Householder, 2 = CholeskyQR2 only.
 *  refine            bulk TTMs on BF16/FP8 data: 0 = apply Q as a BF16 hi+lo
 *                    pair (refinement pass), -1 = BF16 Q only.
 *  max_jacobi_sweeps 0 = default (40); > 0 = limit; -1 = zero sweeps (makes the
 *                    solver report non-convergence, for testing).
 *  async_outputs     0 = a host scalar output (rel_err) is written before the
 *                    call returns (the call synchronises its stream);
 *                    1 = it is written by a stream-ordered host callback, so
 *                    the call returns without synchronising and several
 *                    decompositions can be in flight on different streams;
 *                    read it only after synchronising the stream (or an
 *                    event recorded after the call).  The output pointer
 *                    must stay valid until then.  A handle keeps 64 pending
 *                    outputs at most; the 65th call waits for the stream.   */
typedef struct {
    const int* mode_order;
    int qr_method;
    int refine;
    int max_jacobi_sweeps;
    int async_outputs;
    int reserved[4];
} tk_opts;

typedef struct tk_handle tk_handle;

/* CUDA graphs.  The decompositions, the reconstruction and its gradient can
 * be recorded into a CUDA graph by stream capture of the handle's stream
 * (cudaStreamBeginCapture, or any framework built on it) and replayed many
 * times; nothing in them synchronises.  Rules while recording:
 *  - each recorded call must have run once on the handle with the same sizes
 *    beforehand, so that the workspace is large enough (TK_ERR_WORKSPACE
 *    otherwise); all calls recorded from one handle share its workspace, so
 *    replay them on that handle's stream (or in stream order with it);
 *  - a host scalar output (rel_err) needs async_outputs = 1 (TK_ERR_ARG
 *    otherwise); it is written to the pointer given when recording, at every
 *    replay, once the stream reaches it;
 *  - the profiler records nothing.
 * The workspace block and the host-output slots that a graph recorded stay
 * reserved (a later workspace growth retires the block instead of freeing it)
 * until tk_graph_release, which the caller may call only when no graph
 * recorded from this handle will run again, or tk_destroy.  Neither the
 * handle nor the recorded tensors may be freed while a graph can still run. */
TK_API tk_status tk_graph_release(tk_handle* h);

/* Create a handle bound to a CUDA stream (cudaStream_t passed as void*, NULL =
 * legacy default stream) on the current device.  *h receives the handle.
 * The handle's auxiliary streams (independent per-mode work is forked onto
 * them and joined back within each call) are created with the priority of
 * that stream, so a stream's priority ranks all of a call's work. */
TK_API tk_status tk_create(tk_handle** h, void* cuda_stream);
/* Destroy a handle and free its workspace (synchronises its stream). */
TK_API tk_status tk_destroy(tk_handle* h);
/* Rebind the handle to another stream. */
TK_API tk_status tk_set_stream(tk_handle* h, void* cuda_stream);
/* The persistent streaming kernels of this handle's calls (the passes over X
 * and the other tensor-core and narrow TTMs, one CTA per SM) leave `sms` SMs
 * free, so that kernels queued on other streams (another decomposition's
 * chains of small, latency-bound kernels) find SMs while a pass runs instead
 * of waiting for its end.  0 (default): every SM.  TK_ERR_ARG unless
 * 0 <= sms < the SM count.  Results do not depend on it. */
TK_API tk_status tk_set_sm_reserve(tk_handle* h, int sms);
/* Message of the last failing call on this handle ("" if none).  The string
 * is owned by the handle and valid until the next call. */
TK_API const char* tk_last_error(const tk_handle* h);
/* Synchronise the handle's stream, then report device-side conditions
 * recorded since the previous tk_sync_status: TK_ERR_NOT_CONVERGED if a
 * Jacobi solve hit its sweep limit, TK_ERR_TIMEOUT if a bounded wait gave up,
 * TK_ERR_CUDA for an asynchronous CUDA error, else TK_OK.  If qr_info is not
 * NULL it receives, for the last QR of each mode (up to TK_MAX_D entries),
 * 0 = CholeskyQR2, 1 = Householder, 2 = identity (full-width sketch). */
TK_API tk_status tk_sync_status(tk_handle* h, int* qr_info);
/* Self-test of failure detection (the paper has no counterpart): one warp
 * waits, through the same bounded mbarrier wait every tcgen05 / TMA kernel of
 * the library uses, on an mbarrier that nothing ever arrives at.  The wait
 * gives up after limit_ns (1e3 <= limit_ns <= 2e9, else TK_ERR_ARG; the
 * kernels themselves use 2e9), records the timeout in the handle and returns,
 * leaving the context usable: the next tk_sync_status reports
 * TK_ERR_TIMEOUT (and clears it).  waited_ns (host, may be NULL; non-NULL
 * synchronises): how long the wait lasted on the device clock. */
TK_API tk_status tk_selftest_bounded_wait(tk_handle* h, int64_t limit_ns, int64_t* waited_ns);
/* Bytes of device workspace the handle currently holds. */
TK_API int64_t tk_workspace_bytes(const tk_handle* h);
/* Number of kernel launches queued through this handle since creation. */
TK_API int64_t tk_launch_count(const tk_handle* h);

/* Per-kernel-class timing.  tk_profile(h, 1) clears and starts recording a
 * CUDA event pair on the handle's stream around every kernel the handle
 * launches; tk_profile(h, 0) stops.  tk_profile_read synchronises the stream
 * and fills up to max entries (one per class, in first-seen order) with the
 * launch count, summed device milliseconds and summed algorithmic bytes
 * (inputs read once + outputs written once) and flops; it returns the number
 * of classes (or -1 on error) and clears the records.  Each recorded launch
 * costs two cudaEventRecord calls on the host, so tk_profile_only restricts
 * recording to the classes whose name starts with `prefix` (NULL or "" = all
 * classes; the filter persists until changed).  Class names ("xpass_*": a
 * pass over the whole data tensor): "xpass_tc", "xpass_tc_bg" (a tensor-core
 * pass on part of the SMs, beside a chain of small kernels of the same call),
 * "xpass_narrow", "xpass_simt", "ttm_tc", "ttm_narrow", "ttm_simt",
 * "gemm_f64", "gemm_df", "chol_inv", "apply_rinv", "householder", "jacobi",
 * "residual", "elementwise", "rng". */
typedef struct {
    char name[32];
    int64_t launches;
    double ms;
    double bytes;
    double flops;
} tk_prof_entry;
TK_API tk_status tk_profile(tk_handle* h, int enable);
TK_API tk_status tk_profile_only(tk_handle* h, const char* prefix);
TK_API int tk_profile_read(tk_handle* h, tk_prof_entry* out, int max);
/* The same records one by one, in the order they were queued: class name,
 * launching stream (0: the handle's stream, 1..4: its auxiliary streams),
 * start and end in microseconds after the latest tk_profile(., 1) on the
 * device (any handle; the origin event is recorded on that handle's stream),
 * algorithmic bytes and flops.  Synchronises the handle's streams, fills up
 * to max entries, returns the number of records (-1 on error) and clears
 * them, like tk_profile_read; with out == NULL it only returns the number of
 * records and keeps them. */
typedef struct {
    char name[32];
    int stream;
    int reserved;
    double start_us;
    double end_us;
    double bytes;
    double flops;
} tk_trace_entry;
TK_API int tk_profile_trace(tk_handle* h, tk_trace_entry* out, int max);

/* ---- host-side integer planning (no device work; h may be NULL) -------- */

/* Subrank vector of Algorithm rHKron-re (Section 4.3, the formula
 * s_i = ceil((prod_j l_j)^(1/(d-1)) / l_i) with l_j = r_j + p), followed by a
 * reduction: entries taken largest first (ties: lowest mode) are each lowered
 * to the smallest value that keeps prod_{k!=j} s_k >= l_j for every mode j.
 * r: d target ranks.  s_out: d subranks.  width_out (may be NULL): d sketch
 * column counts prod_{k!=j} s_k.  Errors: TK_ERR_ARG for d < 2, d > TK_MAX_D,
 * r_j < 1 or p < 0. */
TK_API tk_status tucker_subranks_reuse(int d, const int64_t* r, int p, int64_t* s_out, int64_t* width_out);

/* Subrank matrix of Algorithm rSTHKron (Section 4.2, "Choosing subranks"):
 * row j holds d-1 integer factors >= 2 of the smallest l_j' >= r_j + p that
 * has such a factorisation, the most balanced one (smallest largest factor).
 * The factors are given in descending order to the other modes taken in
 * processing order (order: d entries, NULL = 0..d-1).  S_out: d*d, row-major,
 * S_out[j*d+k] = s_{j,k}, diagonal 1.  width_out (may be NULL): l_j'.  */
TK_API tk_status tucker_subranks_matrix(int d, const int64_t* r, int p, const int* order,
                                 int64_t* S_out, int64_t* width_out);

/* ---- building blocks ---------------------------------------------------- */

/* Gaussian sketch factors drawn on the device (the draw lines of Algorithms
 * rHKron-re and rSTHKron: Phi_j with i.i.d. N(0, 1) entries) from the
 * counter-based generator Philox4x32-10 (Salmon, Moraes, Dror and Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11), so that every draw
 * is a pure function of (seed, stream, index) and reproducible anywhere.
 *
 * tk_philox4x32: blocks offset .. offset + nblocks - 1 of stream `stream`;
 * block i is Philox4x32-10 of the counter (i mod 2^32, i div 2^32, stream, 0)
 * under the key (seed mod 2^32, seed div 2^32).  out: 4 * nblocks uint32 on
 * the device, 16-byte aligned, block-major.  Errors: TK_ERR_SHAPE for
 * nblocks < 0, TK_ERR_ARG for a null out, TK_ERR_ALIGN.
 *
 * tucker_gaussian_factor: fills the device matrix M (F64, F32 or BF16;
 * element e = i + rows * j of the column-major order) with N(0, 1) draws of
 * stream `stream`: element e is output e mod 4 of block e div 4 (offset 0),
 * where block (x0, x1, x2, x3) yields the Box-Muller pairs u = (x0 + 1) 2^-32,
 * t = x1 2^-32, (r cos 2 pi t, r sin 2 pi t) with r = sqrt(-2 ln u), and the
 * same from (x2, x3); evaluated in FP64 and rounded once to M's dtype.
 * Asynchronous on the handle's stream.  Distinct streams give independent
 * factors (the Python binding draws Phi_j of mode j from stream j). */
TK_API tk_status tk_philox4x32(tk_handle* h, uint64_t seed, uint32_t stream, uint64_t offset, int64_t nblocks,
                               uint32_t* out);
TK_API tk_status tucker_gaussian_factor(tk_handle* h, uint64_t seed, uint32_t stream, tk_matrix* M);

/* count factors (0 <= count <= 64) in one launch: M[f] gets the draws of
 * stream streams[f], exactly as tucker_gaussian_factor would write them.
 * Errors: TK_ERR_ARG for a bad count or null arrays, then as above. */
TK_API tk_status tucker_gaussian_factors(tk_handle* h, uint64_t seed, int count, const uint32_t* streams,
                                         tk_matrix* M);

/* Kronecker-structured sketches of Algorithm rHKron-re (sketch line):
 * for every mode n, Y_n = X x_1 Phi_1 ... x_{n-1} Phi_{n-1} x_{n+1} Phi_{n+1} ... x_d Phi_d,
 * equivalently Y_n(n) = X_(n) (Phi_d kron ... kron Phi_1, skipping n)^T
 * (Section 4.2), computed with the dimension tree of Section 4.4 and never
 * forming the Kronecker product.
 * X: d-way tensor (F64, F32, BF16 or FP8_E4M3).  Omega: d matrices
 * Omega_j = Phi_j^T, n_j x s_j, dtype F64 for F64 data else F32 or BF16.
 * Y: d tensors; Y[n] has dims (s_1,..,s_{n-1}, n_n, s_{n+1},..,s_d) and dtype
 * F64 (F64 data) or F32 (otherwise). */
TK_API tk_status tucker_sketch(tk_handle* h, const tk_tensor* X, const tk_matrix* Omega, tk_tensor* Y);

/* Thin QR of a tall sketch, Y = Q R with R_ii > 0 (Algorithm RRF):
 * CholeskyQR2 with an FP64 Gram matrix and FP64 Cholesky for F64 Y; for F32 Y
 * the first Gram accumulates with Dot2 (compensated FP32) and both Cholesky
 * factorisations and products Y R^{-1} run in double-float arithmetic (about
 * 48 significant bits, on the FP32 pipe); Householder QR in
 * FP64 when the Cholesky factorisation breaks down or a pivot falls below
 * 1e-12 of its column's squared norm; Q = I when Y has at least as many
 * columns as rows.  Y: rows x cols (F64 or F32).  Q: rows x min(rows, cols),
 * F64 or F32.  info (host, may be NULL): 0 CholeskyQR2, 1 Householder,
 * 2 identity; a non-NULL info synchronises. */
TK_API tk_status tucker_orth(tk_handle* h, const tk_matrix* Y, tk_matrix* Q, int* info, const tk_opts* opts);

/* Thin QR that allocates nothing (the paper has no counterpart; it is a
 * service for callers that cannot allocate device memory where they need the
 * factorisation: applications whose device memory belongs to a pool or arena
 * (a framework's caching allocator holding the free memory, a deployment that
 * forbids allocation after start-up), and latency-critical paths that must not
 * risk the device-wide synchronisation cudaMalloc / cudaFree can cause).  Same
 * result as tucker_orth with default options (CholeskyQR2, Householder
 * fallback, identity for cols >= rows), but it takes no handle: work is queued
 * on cuda_stream (void* cudaStream_t of the current device, NULL = legacy
 * default stream) and its scratch is a fixed 8 MiB device array inside the
 * library, present on every GPU that loads it until the process exits.  It
 * calls no cudaMalloc, cudaFree or allocating library routine.
 * Limits: rows <= 4096 and min(rows, cols) <= 64, else TK_ERR_SHAPE.
 * The first call on a device looks up that array's device address (once per
 * device, with that device current), so make the first call before any stream
 * capture on that device.  Every call shares the array and finds the previous
 * call's contents in it (each call sets what it reads first): calls that
 * overlap on the GPU (different streams, or several threads) race and must be
 * serialised by the caller.  Y: rows x cols, F64 or F32; Q: rows x
 * min(rows, cols), F64 or F32, both device pointers on the current device.
 * info (host, may be NULL; non-NULL synchronises the stream): 0 CholeskyQR2,
 * 1 Householder, 2 identity.  Other errors: TK_ERR_ARG (also a stream of
 * another device, and a non-NULL info on a stream that is recording a CUDA
 * graph: nothing is queued then), TK_ERR_DTYPE, TK_ERR_ALIGN, TK_ERR_CUDA. */
TK_API tk_status tucker_orth_noalloc(void* cuda_stream, const tk_matrix* Y, tk_matrix* Q, int* info);

/* Core multi-TTM Ghat = X x_1 Q_1^T x_2 Q_2^T ... x_d Q_d^T (Algorithm
 * rHKron-re, core line).  Q: d matrices n_j x k_j (F64 for F64 data, else F32).
 * G: tensor (k_1,...,k_d), F64 or F32. */
TK_API tk_status tucker_core(tk_handle* h, const tk_tensor* X, const tk_matrix* Q, tk_tensor* G);

/* ---- the sharded form: X split along its last mode into slabs ------------ */

/* The data-parallel form of Algorithm rHKron-re (Section 6.3, parallel
 * rHKron-re; Section 6.1, all-at-once multi-TTM): X is split along its last
 * mode d into contiguous slabs (column-major storage makes each slab one
 * contiguous block), one per rank, and every rank holds the full (small)
 * factors.  Each slab call works on its slab only; the partial results are
 * exchanged as stated (a SUM all-reduce or an all-gather over the ranks,
 * outside the library), and the small steps in between run redundantly on
 * every rank.  A slab is rows [offset, offset + X_slab.dims[d-1]) of the
 * last mode, whose full length is n_last (0 <= offset, offset + rows <=
 * n_last, else TK_ERR_SHAPE).
 *
 * tucker_sketch_slab: the Kronecker sketches of the slab, with Omega as in
 * tucker_sketch (Omega[d-1] is the full n_last x s_d factor; its slab rows are
 * used).  Y[n] for n < d-1 (dims as tucker_sketch's) receives the slab's
 * partial sum of Y_n: SUM-reduce them over the slabs.  Y[d-1] (dims
 * s_1..s_{d-1} x slab rows) receives the slab's rows of Y_d: gather them
 * along the last mode.
 *
 * tucker_orth_sketches: thin QR Q_n of the mode-n unfolding of each of d
 * sketch tensors Y[n] (k_n = min(n_n, prod_{j!=n} dims), Q = I when the sketch
 * is at least as wide as the mode), as inside tucker_rhkron; Q[n]: n_n x k_n,
 * F64 or F32.  The QR info goes to tk_sync_status.
 *
 * tucker_core_slab: the slab's partial core X_slab x_{j<d} Q_j^T x_d
 * Q_d[slab rows]^T (Q[d-1] is the full n_last x k_d factor): SUM-reduce over
 * the slabs to get Ghat.  G: (k_1..k_d), F64 or F32.
 *
 * tucker_sthosvd: steps 4-5 of Algorithm rHKron-re on a given core: STHOSVD
 * of Ghat (k_1..k_d, F64: FP64 Jacobi; F32: the two-stage mixed eigensolver)
 * to ranks r in opts->mode_order, U_j = Q_j V_j (Q[j]: n_j x k_j), each U_j
 * column signed so that its largest-magnitude entry is positive, G's slices
 * following.  G: (r_1..r_d), U: n_j x r_j, F64 or F32.
 *
 * tucker_loss_slab: norms2 (host, 2 doubles; synchronises) receives
 * ||X_slab - G x_{j<d} U_j x_d U_d[slab rows]||^2 and ||X_slab||^2 (U[d-1] is
 * the full n_last x r_d factor); SUM them over the slabs: the relative error
 * is sqrt(sum first / sum second). */
TK_API tk_status tucker_sketch_slab(tk_handle* h, const tk_tensor* X_slab, int64_t offset, int64_t n_last,
                                    const tk_matrix* Omega, tk_tensor* Y);
TK_API tk_status tucker_orth_sketches(tk_handle* h, int d, const tk_tensor* Y, tk_matrix* Q);
TK_API tk_status tucker_core_slab(tk_handle* h, const tk_tensor* X_slab, int64_t offset, int64_t n_last,
                                  const tk_matrix* Q, tk_tensor* G);
TK_API tk_status tucker_sthosvd(tk_handle* h, const tk_tensor* Ghat, const tk_matrix* Q, const int64_t* r,
                                const tk_opts* opts, tk_tensor* G, tk_matrix* U);
TK_API tk_status tucker_loss_slab(tk_handle* h, const tk_tensor* X_slab, int64_t offset, int64_t n_last,
                                  const tk_tensor* G, const tk_matrix* U, double* norms2);

/* ---- the two algorithms -------------------------------------------------- */

/* Algorithm rHKron-re: sketches with the d reused factors Omega_j = Phi_j^T
 * (n_j x s_j), thin QR of each sketch unfolding into Q_n (n_n x k_n,
 * k_n = min(n_n, prod_{j!=n} s_j)), core Ghat = X x_j Q_j^T, STHOSVD of Ghat to
 * ranks r (Gram matrix + Jacobi eigensolver per mode: FP64 for F64 data; for
 * the other dtypes double-float products and a two-stage mixed-precision
 * Jacobi resolving the Gram to 1e-11 of its norm), U_j = Q_j V_j
 * (Section 4, holistic truncation).  Each column of U_j is signed so that its
 * largest-magnitude entry is positive; G's slices follow.
 * X: F64, F32, BF16 or FP8_E4M3.  r: d host ranks, 1 <= r_j <= k_j.
 * p: oversampling, only checked against the Omega widths (prod_{j!=n} s_j >= r_n + p).
 * G: (r_1..r_d) F64 or F32.  U: d matrices n_j x r_j, F64 or F32.
 * rel_err (host, may be NULL): ||X - G x_j U_j|| / ||X||, which synchronises.
 * Sizes: every sketch width k_n (and so every core mode) must be <= 256, else
 * TK_ERR_SHAPE.  Widths up to 112 take the fast one-CTA kernels above; widths
 * 113-256 fall back to the FP64 Householder QR and the FP64 Jacobi eigensolver
 * in global memory (correct, but one CTA does O(k^3) FP64 work per mode, i.e.
 * milliseconds at k ~ 150).  The same limits hold for the other
 * decompositions, tucker_orth, tucker_orth_sketches and tucker_sthosvd. */
TK_API tk_status tucker_rhkron(tk_handle* h, const tk_tensor* X, const int64_t* r, int p, const tk_matrix* Omega,
                        const tk_opts* opts, tk_tensor* G, tk_matrix* U, double* rel_err);

/* Appendix Alg. rHKron (without factor reuse): like tucker_rhkron, but each
 * mode n has its own sketch factors, Y_n = X x_{j!=n} Phi_{n,j}, so the
 * sketches share no products.  Omega: d*d matrices, Omega[n*d + j] =
 * Phi_{n,j}^T (n_j x s_{n,j}); the diagonal entries are not read.  Needs
 * prod_{j!=n} s_{n,j} >= r_n + p for every n.  Other arguments as
 * tucker_rhkron. */
TK_API tk_status tucker_rhkron_noreuse(tk_handle* h, const tk_tensor* X, const int64_t* r, int p,
                                       const tk_matrix* Omega, const tk_opts* opts, tk_tensor* G, tk_matrix* U,
                                       double* rel_err);

/* rHKron-re with the Kronecker-SRHT sketch of Section 5 (Eq. srht_kron):
 * Y_n = X_(n) D_n (H_1 kron ... kron H_d without H_n), where Omega[j] = H_j is
 * n_j x s_j (in the paper s_j sampled columns of the n_j x n_j Walsh-Hadamard
 * matrix scaled by 1/sqrt(n_j); any matrix is accepted) and D_n is a
 * Rademacher diagonal over the columns of the mode-n unfolding that is not a
 * Kronecker product: entry c of D_n is tk_rademacher(seed, n, c) below.  The
 * sketches share no products (each applies its own D_n to X), so X is
 * streamed once per mode that needs a QR.  Other arguments and outputs as
 * tucker_rhkron.  X: F64, F32, BF16 or FP8; the unfolding column count
 * prod_{j!=n} n_j must be below 2^32.
 *
 * tk_rademacher(seed, n, c) = +1 or -1: with u = (uint32)seed +
 * 0x9E3779B9 * (n + 1) (mod 2^32) and x = (uint32)c ^ u, take the MurmurHash3
 * 32-bit finalizer h = fmix32(x) (x ^= x >> 16; x *= 0x85EBCA6B;
 * x ^= x >> 13; x *= 0xC2B2AE35; x ^= x >> 16) and return -1 when the top bit
 * of h is set.  c is the column index of X_(n) in column-major order (the
 * other modes' indices, mode 1 fastest). */
TK_API tk_status tucker_rhkron_srht(tk_handle* h, const tk_tensor* X, const int64_t* r, int p,
                                    const tk_matrix* Omega, uint64_t seed, const tk_opts* opts, tk_tensor* G,
                                    tk_matrix* U, double* rel_err);

/* Algorithm rSTHKron: modes processed in opts->mode_order; for mode j the
 * sketch Y = Ghat x_{k!=j} Phi_{j,k}, its thin QR Q_j, and Ghat <- Ghat x_j Q_j^T;
 * then STHOSVD(Ghat, r) in the same order and U_j = Q_j V_j.
 * Omega: d*d matrices, Omega[j*d+k] = Phi_{j,k}^T of size (current size of mode
 * k when j is processed) x s_{j,k}, i.e. k_k rows for modes processed before j
 * and n_k rows otherwise; diagonal entries are ignored.
 * Other arguments as tucker_rhkron. */
TK_API tk_status tucker_rsthkron(tk_handle* h, const tk_tensor* X, const int64_t* r, int p, const tk_matrix* Omega,
                          const tk_opts* opts, tk_tensor* G, tk_matrix* U, double* rel_err);

/* ---- reconstruction, loss and its gradient ------------------------------- */

/* Xhat = G x_1 U_1 ... x_d U_d (Section 2.2).  G: (r_1..r_d) F64/F32;
 * U: n_j x r_j F64/F32; Xhat: (n_1..n_d) F64/F32. */
TK_API tk_status tucker_reconstruct(tk_handle* h, const tk_tensor* G, const tk_matrix* U, tk_tensor* Xhat);

/* loss = ||X - G x_1 U_1 ... x_d U_d||^2 with the residual formed explicitly
 * and summed in FP64.  loss: host, synchronises. */
TK_API tk_status tucker_loss(tk_handle* h, const tk_tensor* X, const tk_tensor* G, const tk_matrix* U, double* loss);

/* Gradient of grad_scale * ||X - G x_j U_j||^2 (R = X - G x_j U_j, derived from
 * the unfolding identity of Section 2.1):
 *   dX   = 2 grad_scale R
 *   dG   = -2 grad_scale R x_1 U_1^T ... x_d U_d^T
 *   dU_n = -2 grad_scale (R x_{j!=n} U_j^T)_(n) G_(n)^T
 * The products R x_{j!=n} U_j^T for all n reuse the sketch dimension tree.
 * dG: like G; dU: d matrices like U; dX: like X.  Each output may be NULL
 * (not computed; dU is all d matrices or NULL), so the dX pass and the dG / dU
 * part can be queued separately, e.g. on two streams.
 * norms2: DEVICE pointer to 2 doubles (8-byte aligned), or NULL: receives
 * ||R||^2 and ||X||^2, summed in FP64 from the same residual tiles that dX is
 * formed from (one pass over X serves both), written in stream order with no
 * synchronisation; sqrt(norms2[0] / norms2[1]) is the relative error of
 * (G, U), the value tucker_rhkron returns for its own outputs.  With norms2
 * and no dX the residual pass runs for the norms alone.
 * At least one output must be given (TK_ERR_ARG otherwise). */
TK_API tk_status tucker_reconstruct_backward(tk_handle* h, const tk_tensor* X, const tk_tensor* G, const tk_matrix* U,
                                      double grad_scale, tk_tensor* dG, tk_matrix* dU, tk_tensor* dX,
                                      double* norms2);

/* Algorithm rHKron-re followed by the gradient of grad_scale * ||X - G x_j U_j||^2
 * at its result, in one call that shares the passes over X (no counterpart in
 * the paper, which has no loss gradient; the same values as tucker_rhkron
 * followed by tucker_reconstruct_backward).  The core
 * Ghat = X x_{m_1} Q_{m_1}^T x_{m_2} Q_{m_2}^T .. is formed one mode at a time;
 * with U_j = Q_j V_j, each product R x_{j!=n} U_j^T of the gradient is read
 * from the last product of that chain in which mode n is still whole (so only
 * the mode applied first streams X again), and the relative error comes from
 * the norms of the pass that forms dX.  Arguments as tucker_rhkron and
 * tucker_reconstruct_backward; G and U receive the decomposition, rel_err
 * (host, may be NULL) its relative error, dG, dU, dX (each may be NULL) the
 * gradient at (G, U) as given to the caller. */
TK_API tk_status tucker_rhkron_grad(tk_handle* h, const tk_tensor* X, const int64_t* r, int p,
                                    const tk_matrix* Omega, const tk_opts* opts, tk_tensor* G, tk_matrix* U,
                                    double* rel_err, double grad_scale, tk_tensor* dG, tk_matrix* dU,
                                    tk_tensor* dX);

#ifdef __cplusplus
}
#endif

#endif /* TUCKER_H */
