"""GPU parity: every entry point of the C ABI against the FP64 oracle on the
same seeded inputs, element by element.  Tolerances: 1e-12 (F64 path) and
1e-5 (F32 path, and BF16/FP8 storage whose values the oracle consumes
exactly), relative Frobenius norm unless stated."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2211_13028_gb300 import synth
from paper_2211_13028_gb300 import tucker as T
from tests.gpu_helpers import TOL, align, make_X, mats, rel, require_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return require_gpu()


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


# ------------------------------------------------------------------ sketch (multi-TTM)

@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16", "fp8"])
@pytest.mark.parametrize("dims,s", [((37, 29, 41), (3, 4, 2)), ((130, 7, 66), (5, 2, 3)), ((13, 9, 11, 7), (2, 3, 2, 2))])
def test_sketch_parity(dev, dtype, dims, s):
    g = _rng(1)
    X, xv, sc = make_X(g.standard_normal(dims), dtype, dev)
    odt = "f64" if dtype == "f64" else ("bf16" if dtype == "bf16" else "f32")
    oms = synth.sketch_factors_reuse(dims, s, seed=2, dtype=odt)
    Y = T.tucker_sketch(X, mats(oms, odt, dev), scale=sc)
    d = len(dims)
    for n in range(d):
        ref = O.multi_ttm(xv, [(j, oms[j].T) for j in range(d) if j != n])
        assert tuple(Y[n].shape) == ref.shape
        assert rel(to_np(Y[n]), ref) <= TOL[dtype]


@pytest.mark.parametrize("dims,s", [((192, 160, 200), (6, 7, 8)), ((190, 171, 160), (5, 8, 3)), ((256, 64, 300), (1, 8, 7))])
def test_sketch_parity_streaming_fp32(dev, dims, s):
    # FP32 tensors above 4M elements with sketch widths <= 8: the FP32 streaming kernels
    # (strided contracted mode with L % 4 == 0, or contiguous); dims (190, ...) also take the
    # tensor-core path where L % 4 != 0.  Each sampled entry against the FP64 oracle.
    g = _rng(11)
    X, xv, sc = make_X(g.standard_normal(dims), "f32", dev)
    oms = synth.sketch_factors_reuse(dims, s, seed=12, dtype="f32")
    Y = T.tucker_sketch(X, mats(oms, "f32", dev), scale=sc)
    d = len(dims)
    for n in range(d):
        ref = O.multi_ttm(xv, [(j, oms[j].T) for j in range(d) if j != n])
        assert tuple(Y[n].shape) == ref.shape
        assert rel(to_np(Y[n]), ref) <= TOL["f32"]


def test_sketch_matches_explicit_kronecker(dev):
    # Y_n(n) = X_(n) Omega_n with the Kronecker product formed explicitly (Section 4.2 identity).
    g = _rng(3)
    dims, s = (9, 8, 7), (2, 3, 2)
    x = g.standard_normal(dims)
    oms = synth.sketch_factors_reuse(dims, s, seed=4)
    Y = T.tucker_sketch(synth.fortran(x, "f64", dev), mats(oms, "f64", dev))
    phis = [o.T for o in oms]
    for n in range(3):
        assert rel(O.unfold(to_np(Y[n]), n), O.unfold(x, n) @ O.kron_omega(phis, n)) <= 1e-12


# ------------------------------------------------------------------ thin QR

@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n,k", [(512, 49), (97, 13), (300, 112), (64, 1), (33, 2)])
def test_orth_cholqr2_parity(dev, dtype, n, k):
    y = synth.round_to(_rng(5).standard_normal((n, k)), dtype)
    Q, info = T.tucker_orth(synth.fmat(y, dtype, dev), out_dtype=torch.float64)
    assert info == 0
    ref = O.thin_qr(y)
    assert np.max(np.abs(to_np(Q) - ref)) <= 1e-12


def test_orth_householder_forced_parity(dev):
    y = _rng(6).standard_normal((200, 30))
    Q, info = T.tucker_orth(synth.fmat(y, "f64", dev), qr_method=1)
    assert info == 1
    assert np.max(np.abs(to_np(Q) - O.thin_qr(y))) <= 1e-12


def test_orth_rank_deficient_falls_back(dev):
    g = _rng(7)
    y = g.standard_normal((150, 4)) @ g.standard_normal((4, 12))  # rank 4, 12 columns
    Q, info = T.tucker_orth(synth.fmat(y, "f64", dev))
    assert info == 1
    q = to_np(Q)
    assert np.max(np.abs(q.T @ q - np.eye(12))) <= 1e-13
    assert np.linalg.norm(q @ (q.T @ y) - y) <= 1e-12 * np.linalg.norm(y)


def test_orth_rank_deficient_f32_falls_back(dev):
    # FP32 sketches take the double-float CholeskyQR2; a numerically rank-deficient one must
    # still be caught by the pivot test and handed to Householder
    g = _rng(17)
    y = synth.round_to(g.standard_normal((300, 5)) @ g.standard_normal((5, 20)), "f32")
    Q, info = T.tucker_orth(synth.fmat(y, "f32", dev), out_dtype=torch.float64)
    assert info == 1
    q = to_np(Q)
    assert np.max(np.abs(q.T @ q - np.eye(20))) <= 1e-13
    assert np.linalg.norm(q @ (q.T @ y) - y) <= 1e-12 * np.linalg.norm(y)


def test_orth_wide_is_identity(dev):
    y = _rng(8).standard_normal((20, 25))
    Q, info = T.tucker_orth(synth.fmat(y, "f64", dev))
    assert info == 2
    np.testing.assert_array_equal(to_np(Q), np.eye(20))


# ------------------------------------------------------------------ core multi-TTM

@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_core_parity(dev, dtype):
    g = _rng(9)
    dims, k = (70, 33, 45), (11, 9, 13)
    X, xv, _ = make_X(g.standard_normal(dims), dtype, dev)
    qs = [O.thin_qr(g.standard_normal((n, kk))) for n, kk in zip(dims, k)]
    acc = "f64" if dtype == "f64" else "f32"
    qs = [synth.round_to(q, acc) for q in qs]
    G = T.tucker_core(X, mats(qs, acc, dev))
    ref = O.multi_ttm(xv, [(j, qs[j].T) for j in range(3)])
    assert rel(to_np(G), ref) <= TOL[dtype]


# ------------------------------------------------------------------ rHKron-re end to end

def _check_decomp(G, U, err, ref, xv, tol):
    """rel_err (absolute difference), core G (relative Frobenius, after fixing
    the sign gauge), reconstruction, and each U_j weighted by the singular
    values of G_(j): a column whose singular value is s_i is only determined
    to (rounding) * s_1 / gap_i, and its effect on the reconstruction scales
    with s_i, so || (U_j - U_j^ref) diag(s) || / || s || is the meaningful
    per-factor error."""
    ref_err = O.rel_err(xv, ref["G"], ref["U"])
    assert abs(err - ref_err) <= tol, (err, ref_err)
    g, u = align(to_np(G), [to_np(x) for x in U], ref["U"])
    assert rel(g, ref["G"]) <= tol
    for j in range(len(u)):
        sv = np.linalg.svd(O.unfold(ref["G"], j), compute_uv=False)
        werr = np.linalg.norm((u[j] - ref["U"][j]) * sv[None, :]) / np.linalg.norm(sv)
        assert werr <= tol, (j, werr)
        assert np.max(np.abs(u[j].T @ u[j] - np.eye(u[j].shape[1]))) <= max(tol, 1e-6)
    assert rel(O.reconstruct(g, u), O.reconstruct(ref["G"], ref["U"])) <= tol


@pytest.mark.parametrize("literal", [False, True])
def test_rhkron_f64_tucker64(dev, literal):
    # 64^3 FP64: Tucker core 8^3 N(0,1), orthonormal factors, 1e-3 noise; r = 8, p = 4.
    dims, r, p = (64, 64, 64), (8, 8, 8), 4
    x = synth.tucker_tensor(dims, (8, 8, 8), seed=0, noise_rel=1e-3)
    s = (12, 12, 12) if literal else tuple(O.subranks_reuse(r, p)[0])
    oms = synth.sketch_factors_reuse(dims, s, seed=1)
    G, U, err = T.tucker_rhkron(synth.fortran(x, "f64", dev), r, p, mats(oms, "f64", dev))
    ref = O.rhkron(x, r, oms)
    _check_decomp(G, U, err, ref, x, 1e-12)
    if literal:  # full-width sketches: rHKron-re reduces to STHOSVD of X
        Gs, Us, _ = O.sthosvd(x, r)
        assert abs(err - O.rel_err(x, Gs, Us)) <= 1e-12
    st, info = T.tk_sync_status(dev)
    assert st == 0 and info[:3] == ([2, 2, 2] if literal else [0, 0, 0])


@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
def test_rhkron_narrow_storage(dev, dtype):
    # Core entries decay by 0.5 per index so that consecutive singular values of
    # the unfoldings are well separated: the factors are then determined to
    # the FP32 rounding level and can be compared column by column.  FP8
    # quantisation noise (~2% of ||X||) hides all but the leading directions,
    # so the FP8 case uses rank 4.
    dims, r, p = (96, 80, 72), ((4, 4, 4) if dtype == "fp8" else (10, 12, 8)), 6
    core = synth.decaying_core((16, 16, 16), 0.5, seed=11)
    x = synth.tucker_tensor(dims, (16, 16, 16), seed=12, noise_rel=1e-4, core=core)
    X, xv, sc = make_X(x, dtype, dev)
    s = O.subranks_reuse(r, p)[0]
    odt = "bf16" if dtype == "bf16" else "f32"
    oms = synth.sketch_factors_reuse(dims, s, seed=13, dtype=odt)
    G, U, err = T.tucker_rhkron(X, r, p, mats(oms, odt, dev), scale=sc)
    st, info = T.tk_sync_status(dev)
    assert st == 0 and info[:3] == [0, 0, 0]  # eigensolvers converged, CholeskyQR2 held
    ref = O.rhkron(xv, r, oms)
    _check_decomp(G, U, err, ref, xv, 1e-5)


def test_rhkron_exact_low_rank_f64(dev):
    dims, rk = (48, 40, 36), (4, 5, 3)
    x = synth.tucker_tensor(dims, rk, seed=21, noise_rel=0.0)
    r, p = rk, 6
    s = O.subranks_reuse(r, p)[0]
    oms = synth.sketch_factors_reuse(dims, s, seed=22)
    G, U, err = T.tucker_rhkron(synth.fortran(x, "f64", dev), r, p, mats(oms, "f64", dev))
    assert err <= 1e-12
    st, info = T.tk_sync_status(dev)
    assert st == 0 and 1 in info[:3]  # rank-deficient sketches took the Householder path
    ref = O.rhkron(x, r, oms)
    xh = O.reconstruct(to_np(G), [to_np(u) for u in U])
    assert rel(xh, O.reconstruct(ref["G"], ref["U"])) <= 1e-12


# ------------------------------------------------------------------ rSTHKron end to end

def test_rsthkron_f64_d3(dev):
    dims, r, p = (50, 44, 38), (6, 5, 7), 4
    x = synth.tucker_tensor(dims, (9, 9, 9), seed=31, noise_rel=1e-3)
    order = [0, 1, 2]
    S, w = O.subranks_matrix(r, p, order)
    k = [min(n, ww) for n, ww in zip(dims, w)]
    oms = synth.sketch_factors_matrix(dims, S, k, order, seed=32)
    Om = {key: synth.fmat(v, "f64", dev) for key, v in oms.items()}
    G, U, err = T.tucker_rsthkron(synth.fortran(x, "f64", dev), r, p, Om, order=order)
    _check_decomp(G, U, err, O.rsthkron(x, r, oms, order), x, 1e-12)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_rsthkron_d4_uneven_reverse_order(dev, dtype):
    # 4-way, uneven ranks, modes processed 4 -> 1 (the shape of the 4-way workload, scaled down).
    dims, r, p = (24, 22, 20, 26), (3, 4, 5, 6), 3
    core = synth.decaying_core((8, 8, 8, 8), 0.7, seed=41)
    x = synth.tucker_tensor(dims, (8, 8, 8, 8), seed=42, noise_rel=1e-3, core=core)
    X, xv, _ = make_X(x, dtype, dev)
    order = [3, 2, 1, 0]
    S, w = O.subranks_matrix(r, p, order)
    k = [min(n, ww) for n, ww in zip(dims, w)]
    oms = synth.sketch_factors_matrix(dims, S, k, order, seed=43, dtype=dtype)
    Om = {key: synth.fmat(v, dtype, dev) for key, v in oms.items()}
    G, U, err = T.tucker_rsthkron(X, r, p, Om, order=order)
    _check_decomp(G, U, err, O.rsthkron(xv, r, oms, order), xv, TOL[dtype])


# ------------------------------------------------------------------ reconstruction, loss, gradient

@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_reconstruct_loss_backward(dev, dtype):
    g = _rng(51)
    dims, rk = (20, 18, 16), (4, 3, 5)
    x = synth.round_to(g.standard_normal(dims), dtype)
    G = synth.round_to(g.standard_normal(rk), dtype)
    U = [synth.round_to(g.standard_normal((n, k)), dtype) for n, k in zip(dims, rk)]
    Xd, Gd, Ud = synth.fortran(x, dtype, dev), synth.fortran(G, dtype, dev), mats(U, dtype, dev)
    tol = TOL[dtype]
    assert rel(to_np(T.tucker_reconstruct(Gd, Ud)), O.reconstruct(G, U)) <= tol
    ref_loss = O.loss(x, G, U)
    assert abs(T.tucker_loss(Xd, Gd, Ud) - ref_loss) <= tol * ref_loss
    dG, dU, dX = T.tucker_reconstruct_backward(Xd, Gd, Ud, grad_scale=0.5)
    ref = O.loss_grads(x, G, U)
    assert rel(to_np(dG), 0.5 * ref["dG"]) <= 10 * tol
    for j in range(3):
        assert rel(to_np(dU[j]), 0.5 * ref["dU"][j]) <= 10 * tol
    assert rel(to_np(dX), 0.5 * ref["dX"]) <= tol


def test_autograd_function_matches_oracle(dev):
    g = _rng(52)
    dims, rk = (12, 10, 9), (3, 2, 4)
    x = g.standard_normal(dims)
    G0 = g.standard_normal(rk)
    U0 = [g.standard_normal((n, k)) for n, k in zip(dims, rk)]
    X = synth.fortran(x, "f64", dev).requires_grad_(True)
    G = synth.fortran(G0, "f64", dev).requires_grad_(True)
    U = [synth.fmat(u, "f64", dev).requires_grad_(True) for u in U0]
    loss = T.TuckerLoss.apply(X, G, *U)
    (3.0 * loss).backward()
    ref = O.loss_grads(x, G0, U0)
    assert abs(loss.item() - O.loss(x, G0, U0)) <= 1e-12 * O.loss(x, G0, U0)
    assert rel(to_np(G.grad), 3.0 * ref["dG"]) <= 1e-12
    assert rel(to_np(X.grad), 3.0 * ref["dX"]) <= 1e-12
    for j in range(3):
        assert rel(U[j].grad.cpu().numpy(), 3.0 * ref["dU"][j]) <= 1e-12


def test_gradient_matches_fp64_finite_differences(dev):
    # Central differences (h = 1e-6) of the GPU loss itself on a 24^3 FP64 problem, along
    # random directions in (X, G, U) and at 20 individual entries, against the GPU gradient.
    g = _rng(53)
    dims, rk = (24, 24, 24), (4, 3, 5)
    G0 = g.standard_normal(rk)
    U0 = [g.standard_normal((n, k)) / np.sqrt(n) for n, k in zip(dims, rk)]
    # X near the model keeps the loss O(1), so the differences are not lost to cancellation
    x = O.reconstruct(G0, U0) + 0.05 * g.standard_normal(dims)
    X = synth.fortran(x, "f64", dev).requires_grad_(True)
    G = synth.fortran(G0, "f64", dev).requires_grad_(True)
    U = [synth.fmat(u, "f64", dev).requires_grad_(True) for u in U0]
    params = [X, G] + U
    T.TuckerLoss.apply(*params).backward()
    grads = [p.grad.detach().clone() for p in params]

    def loss_at(shift):
        with torch.no_grad():
            return T.tucker_loss(X + shift[0], G + shift[1], [u + d for u, d in zip(U, shift[2:])])

    h = 1e-6
    for trial in range(6):
        dirs = [torch.randn(p.shape, dtype=torch.float64, device=dev, generator=torch.Generator(dev).manual_seed(trial))
                for p in params]
        fd = (loss_at([h * d for d in dirs]) - loss_at([-h * d for d in dirs])) / (2 * h)
        an = sum(float((gr * d).sum()) for gr, d in zip(grads, dirs))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), trial
    for e in range(20):
        which = e % len(params)
        idx = tuple(int(i) for i in np.unravel_index(int(g.integers(params[which].numel())), params[which].shape))
        shift = [torch.zeros_like(p) for p in params]
        shift[which][idx] = h
        fd = (loss_at(shift) - loss_at([-s for s in shift])) / (2 * h)
        an = float(grads[which][idx])
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (which, idx)


# ------------------------------------------------------------------ error paths

def test_bad_shapes_are_rejected(dev):
    x = synth.fortran(np.zeros((8, 7, 6)), "f64", dev)
    oms = mats(synth.sketch_factors_reuse((8, 7, 6), (2, 2, 2), seed=0), "f64", dev)
    with pytest.raises(T.TuckerError) as e:
        T.tucker_rhkron(x, (3, 3, 3), 1, oms[:2] + [oms[0]])  # Omega_3 has the wrong row count
    assert e.value.status == 2
    with pytest.raises(T.TuckerError) as e:
        T.tucker_rhkron(x, (9, 3, 3), 0, oms)  # rank above the sketch width
    assert e.value.status == 2
    with pytest.raises(T.TuckerError) as e:
        T.tucker_sketch(torch.zeros((8, 7, 6), dtype=torch.float64, device=dev), oms)  # row-major
    assert e.value.status == 4


def test_jacobi_sweep_limit_is_reported(dev):
    x = synth.tucker_tensor((30, 28, 26), (5, 5, 5), seed=61, noise_rel=1e-2)
    r, p = (3, 3, 3), 2
    oms = synth.sketch_factors_reuse(x.shape, O.subranks_reuse(r, p)[0], seed=62)
    T.tucker_rhkron(synth.fortran(x, "f64", dev), r, p, mats(oms, "f64", dev), max_jacobi_sweeps=-1, rel_err=False)
    st, _ = T.tk_sync_status(dev)
    assert st == 7
    T.tucker_rhkron(synth.fortran(x, "f64", dev), r, p, mats(oms, "f64", dev), rel_err=False)
    st, _ = T.tk_sync_status(dev)
    assert st == 0


# ------------------------------------------------------------------ appendix rHKron (no reuse), 4-way, edge cases

@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_rhkron_noreuse_parity(dev, dtype):
    # appendix Algorithm rHKron: fresh factors per mode (rows of the subrank matrix)
    dims, r, p = (40, 36, 32), (5, 4, 6), 5
    core = synth.decaying_core((10, 10, 10), 0.6, seed=71)
    x = synth.tucker_tensor(dims, (10, 10, 10), seed=72, noise_rel=1e-3, core=core)
    X, xv, _ = make_X(x, dtype, dev)
    S, _ = O.subranks_matrix(r, p)
    oms = synth.sketch_factors_noreuse(dims, S, seed=73, dtype=dtype)
    Om = {key: synth.fmat(v, dtype, dev) for key, v in oms.items()}
    G, U, err = T.tucker_rhkron_noreuse(X, r, p, Om)
    _check_decomp(G, U, err, O.rhkron_noreuse(xv, r, oms), xv, TOL[dtype])


def test_rhkron_noreuse_exact_low_rank(dev):
    dims, rk = (24, 20, 18, 16), (3, 2, 4, 2)
    x = synth.tucker_tensor(dims, rk, seed=74, noise_rel=0.0)
    S, _ = O.subranks_matrix(rk, 2)
    oms = synth.sketch_factors_noreuse(dims, S, seed=75)
    Om = {key: synth.fmat(v, "f64", dev) for key, v in oms.items()}
    _, _, err = T.tucker_rhkron_noreuse(synth.fortran(x, "f64", dev), rk, 2, Om)
    assert err <= 1e-12


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_rhkron_four_way(dev, dtype):
    # rHKron-re on a 4-way tensor: the dimension tree over four modes (Sec. 4.4)
    dims, r, p = (20, 18, 16, 22), (3, 4, 2, 5), 3
    core = synth.decaying_core((6, 6, 6, 6), 0.6, seed=76)
    x = synth.tucker_tensor(dims, (6, 6, 6, 6), seed=77, noise_rel=1e-3, core=core)
    X, xv, _ = make_X(x, dtype, dev)
    s = O.subranks_reuse(r, p)[0]
    oms = synth.sketch_factors_reuse(dims, s, seed=78, dtype=dtype)
    G, U, err = T.tucker_rhkron(X, r, p, mats(oms, dtype, dev))
    _check_decomp(G, U, err, O.rhkron(xv, r, oms), xv, TOL[dtype])


def test_rhkron_full_rank_and_no_oversampling(dev):
    # r = n on one mode (its factor is a rotation of the whole space) and p = 0
    dims = (12, 30, 26)
    x = synth.round_to(np.random.Generator(np.random.PCG64(79)).standard_normal(dims), "f64")
    r, p = (12, 5, 4), 0
    s = O.subranks_reuse(r, p)[0]
    oms = synth.sketch_factors_reuse(dims, s, seed=80)
    G, U, err = T.tucker_rhkron(synth.fortran(x, "f64", dev), r, p, mats(oms, "f64", dev))
    ref = O.rhkron(x, r, oms)
    assert abs(err - O.rel_err(x, ref["G"], ref["U"])) <= 1e-12
    assert rel(O.reconstruct(*align(to_np(G), [to_np(u) for u in U], ref["U"])), O.reconstruct(ref["G"], ref["U"])) <= 1e-12


def test_core_truncation_at_the_maximum_width(dev):
    # sketch widths of 112 (the largest the core eigensolver and Cholesky take) on FP32 data
    dims, r, p = (200, 150, 130), (104, 56, 104), 8
    core = synth.decaying_core((112, 112, 112), 0.97, seed=81)
    x = synth.tucker_tensor(dims, (112, 112, 112), seed=82, noise_rel=1e-3, core=core)
    X, xv, _ = make_X(x, "f32", dev)
    s = (8, 14, 8)  # sketch widths prod_{j!=n} s_j = 112, 64, 112
    oms = synth.sketch_factors_reuse(dims, s, seed=83, dtype="f32")
    G, U, err = T.tucker_rhkron(X, r, p, mats(oms, "f32", dev))
    ref = O.rhkron(xv, r, oms)
    assert abs(err - O.rel_err(xv, ref["G"], ref["U"])) <= 1e-5
    st, _ = T.tk_sync_status(dev)
    assert st == 0


def test_empty_dimension_is_rejected_before_launch(dev):
    x = torch.zeros((0, 4, 5), dtype=torch.float64, device=dev).permute(2, 1, 0).contiguous().permute(2, 1, 0)
    oms = [torch.zeros((0, 2), dtype=torch.float64, device=dev).t().contiguous().t(),
           synth.fmat(np.ones((4, 2)), "f64", dev), synth.fmat(np.ones((5, 2)), "f64", dev)]
    l0 = T.tk_launch_count(dev)
    with pytest.raises(T.TuckerError):
        T.tucker_rhkron(x, (1, 1, 1), 1, oms)
    assert T.tk_launch_count(dev) == l0


# ------------------------------------------------------------------ sketch widths above the one-CTA kernels

@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_rhkron_sketch_widths_above_112(dev, dtype):
    # widths 156, 143 and 132: the Householder QR and the FP64 Jacobi in global memory take over
    dims, r, p = (200, 180, 170), (10, 9, 8), 5
    x = synth.tucker_tensor(dims, (12, 12, 12), seed=41, noise_rel=1e-3)
    X, xv, sc = make_X(x, dtype, dev)
    oms = synth.sketch_factors_reuse(dims, (11, 12, 13), seed=42, dtype="f64" if dtype == "f64" else "f32")
    G, U, err = T.tucker_rhkron(X, r, p, mats(oms, "f64" if dtype == "f64" else "f32", dev), scale=sc)
    st, info = T.tk_sync_status(dev)
    assert st == 0 and info[:3] == [1, 1, 1]  # Householder QR for the wide sketches
    ref = O.rhkron(xv, r, oms)
    _check_decomp(G, U, err, ref, xv, TOL[dtype])
