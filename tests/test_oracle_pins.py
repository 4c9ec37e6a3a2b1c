"""Pins for the FP64 oracle: brute force, closed forms, printed values, invariants.

Each check here is independent of the oracle's own formula: a plausible slip
(dropped term, transposed operand, wrong unfolding order, wrong sign) fails at
least one of them.
"""
import itertools
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2211_13028_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


# ------------------------------------------------------------------ Section 2.1

def test_unfold_column_order_by_loops():
    g = _rng(1)
    X = g.standard_normal((3, 4, 5, 2))
    for j in range(4):
        M = O.unfold(X, j)
        rest = [k for k in range(4) if k != j]
        for idx in itertools.product(*[range(s) for s in X.shape]):
            col, stride = 0, 1
            for k in rest:  # lowest remaining mode fastest
                col += idx[k] * stride
                stride *= X.shape[k]
            assert M[idx[j], col] == X[idx]
        np.testing.assert_array_equal(O.fold(M, j, X.shape), X)


@pytest.mark.parametrize("shape", [(4, 3, 5), (3, 2, 4, 3), (1, 5, 2)])
def test_ttm_matches_elementwise_loops(shape):
    g = _rng(2)
    X = g.standard_normal(shape)
    for j in range(len(shape)):
        A = g.standard_normal((3, shape[j]))
        np.testing.assert_allclose(O.ttm(X, A, j), O.ttm_loops(X, A, j), rtol=1e-13, atol=1e-13)


def test_multi_ttm_kronecker_unfolding_identity():
    # Section 2.1: (X x_1 A_1 ... x_d A_d)_(j) = A_j X_(j) (A_d kron .. A_{j+1} kron A_{j-1} .. A_1)^T,
    # with the left side computed by brute-force loops.
    g = _rng(3)
    X = g.standard_normal((3, 4, 2, 3))
    A = [g.standard_normal((2, 3)), g.standard_normal((3, 4)), g.standard_normal((2, 2)), g.standard_normal((4, 3))]
    Y = X
    for k in range(4):
        Y = O.ttm_loops(Y, A[k], k)
    for j in range(4):
        np.testing.assert_allclose(O.unfold(Y, j), O.kron_unfolded_multi_ttm(X, A, j), rtol=1e-12, atol=1e-12)


def test_kronecker_sketch_identity():
    # X_(n) Omega_n = (X x_{j != n} Phi_j)_(n) with Omega_n the explicit Kronecker product (Section 4.2).
    g = _rng(4)
    X = g.standard_normal((5, 4, 6))
    phis = [g.standard_normal((2, 5)), g.standard_normal((3, 4)), g.standard_normal((2, 6))]
    for n in range(3):
        Y = X
        for j in range(3):
            if j != n:
                Y = O.ttm_loops(Y, phis[j], j)
        np.testing.assert_allclose(O.unfold(X, n) @ O.kron_omega(phis, n), O.unfold(Y, n), rtol=1e-12, atol=1e-12)


def test_multi_ttm_order_is_free():
    g = _rng(5)
    X = g.standard_normal((4, 5, 3))
    mats = [(0, g.standard_normal((2, 4))), (1, g.standard_normal((3, 5))), (2, g.standard_normal((2, 3)))]
    ref = O.multi_ttm(X, mats)
    for perm in itertools.permutations(mats):
        np.testing.assert_allclose(O.multi_ttm(X, list(perm)), ref, rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------ QR

def _gram_schmidt(Y):
    m, k = Y.shape
    Q = np.zeros((m, k))
    for c in range(k):
        v = Y[:, c].copy()
        for t in range(c):
            v -= (Q[:, t] @ Y[:, c]) * Q[:, t]
        Q[:, c] = v / np.sqrt(v @ v)
    return Q


def test_thin_qr_characterisation():
    g = _rng(6)
    Y = g.standard_normal((9, 4))
    Q = O.thin_qr(Y)
    R = Q.T @ Y
    np.testing.assert_allclose(Q.T @ Q, np.eye(4), atol=1e-14)
    np.testing.assert_allclose(np.tril(R, -1), 0, atol=1e-13)
    assert np.all(np.diag(R) > 0)
    np.testing.assert_allclose(Q @ R, Y, atol=1e-13)
    np.testing.assert_allclose(Q, _gram_schmidt(Y), atol=1e-12)


def test_thin_qr_full_width_is_identity():
    g = _rng(7)
    np.testing.assert_array_equal(O.thin_qr(g.standard_normal((5, 7))), np.eye(5))
    np.testing.assert_array_equal(O.thin_qr(g.standard_normal((5, 5))), np.eye(5))


# ------------------------------------------------------------------ STHOSVD

def test_sthosvd_closed_form_on_section61_tensor():
    # Superdiagonal core 0.4^(i-1): truncating to rank 10 leaves error exactly 0.4^10 (Section 7.1).
    X = synth.e1_tensor(40, 0.4, seed=0)
    G, U, _ = O.sthosvd(X, (10, 10, 10))
    err = O.rel_err(X, G, U)
    assert abs(err - 0.4 ** 10) <= 1e-12
    golden = json.load(open(os.path.join(GOLDEN, "e1_accuracy.json")))
    assert abs(err - golden["sthosvd_rel_err"]) / golden["sthosvd_rel_err"] < 1e-5


def test_sthosvd_error_identity():
    # ||X - T||^2 equals the sum of the squared singular values discarded at each step.
    g = _rng(8)
    X = g.standard_normal((7, 6, 5))
    for order in ([0, 1, 2], [2, 0, 1]):
        G, U, disc = O.sthosvd(X, (3, 2, 4), order)
        assert abs(O.loss(X, G, U) - sum(disc)) <= 1e-10 * np.sum(X * X)
        for u in U:
            np.testing.assert_allclose(u.T @ u, np.eye(u.shape[1]), atol=1e-13)


def test_sthosvd_full_rank_reproduces():
    g = _rng(9)
    X = g.standard_normal((4, 3, 5))
    G, U, _ = O.sthosvd(X, (4, 3, 5))
    np.testing.assert_allclose(O.reconstruct(G, U), X, atol=1e-12)


# ------------------------------------------------------------------ subranks

def _row_multiset(row, j):
    return sorted(int(v) for k, v in enumerate(row) if k != j)


@pytest.mark.parametrize("name", ["miranda", "sp"])
def test_subranks_reproduce_printed_values(name):
    gd = json.load(open(os.path.join(GOLDEN, "paper_subranks.json")))[name]
    s, _ = O.subranks_reuse(gd["r"], gd["p"])
    assert s == gd["s"]
    S, widths = O.subranks_matrix(gd["r"], gd["p"])
    d = len(gd["r"])
    for j in range(d):
        assert _row_multiset(S[j], j) == _row_multiset(gd["S"][j], j)
        assert int(np.prod([S[j][k] for k in range(d) if k != j])) == widths[j] >= gd["r"][j] + gd["p"]


def test_subranks_constraints_random():
    g = _rng(10)
    for _ in range(200):
        d = int(g.integers(3, 6))
        r = [int(x) for x in g.integers(1, 60, d)]
        p = int(g.integers(0, 10))
        s, w = O.subranks_reuse(r, p)
        for j in range(d):
            assert w[j] >= r[j] + p
            # minimality of each entry given the others
            if s[j] > 1:
                t = list(s)
                t[j] -= 1
                ok = all(np.prod([t[k] for k in range(d) if k != i]) >= r[i] + p for i in range(d))
                assert not ok
        S, w2 = O.subranks_matrix(r, p)
        for j in range(d):
            row = [int(S[j][k]) for k in range(d) if k != j]
            assert min(row) >= 2 and int(np.prod(row)) == w2[j] >= r[j] + p
            for L in range(r[j] + p, w2[j]):  # nothing smaller has d-1 factors >= 2
                assert O.balanced_factors(L, d - 1)[0] != L


def test_subranks_for_the_workloads():
    # Values the readings give for the benchmark and parity workloads.
    assert O.subranks_reuse((8, 8, 8), 4)[0] == [3, 4, 4]
    assert O.subranks_reuse((32, 32, 32), 8)[0] == [6, 7, 7]
    assert O.subranks_reuse((64, 64, 64), 16)[0] == [9, 9, 9]
    assert O.subranks_reuse((16, 16, 16), 8)[0] == [5, 5, 5]
    S, w = O.subranks_matrix((10, 20, 30, 40), 6, order=[3, 2, 1, 0])
    assert w == [16, 27, 36, 48]
    assert [_row_multiset(S[j], j) for j in range(4)] == [[2, 2, 4], [3, 3, 3], [3, 3, 4], [3, 4, 4]]
    S, w = O.subranks_matrix((32, 32, 32), 8)
    assert w == [40, 40, 40] and _row_multiset(S[0], 0) == [5, 8]


# ------------------------------------------------------------------ the randomized algorithms

def _low_rank(shape, ranks, seed):
    return synth.tucker_tensor(shape, ranks, seed, 0.0)


def _reuse_factors(shape, r, p, seed):
    s, _ = O.subranks_reuse(r, p)
    return synth.sketch_factors_reuse(shape, s, seed)


def _matrix_factors(shape, r, p, order, seed):
    S, w = O.subranks_matrix(r, p, order)
    k = [min(n, x) for n, x in zip(shape, w)]
    return synth.sketch_factors_matrix(shape, S, k, order, seed)


@pytest.mark.parametrize("shape,r,p", [((12, 10, 9), (3, 4, 2), 2), ((9, 8, 7, 6), (2, 3, 2, 2), 1), ((16, 16, 16), (3, 3, 3), 6)])
def test_exact_recovery_of_low_rank(shape, r, p):
    X = _low_rank(shape, r, seed=11)
    d = len(shape)
    out = O.rhkron(X, r, _reuse_factors(shape, r, p, 12))
    assert O.rel_err(X, out["G"], out["U"]) <= 1e-12
    order = list(range(d))[::-1]
    out = O.rsthkron(X, r, _matrix_factors(shape, r, p, order, 13), order)
    assert O.rel_err(X, out["G"], out["U"]) <= 1e-12
    S, _ = O.subranks_matrix(r, p)
    out = O.rhkron_noreuse(X, r, synth.sketch_factors_noreuse(shape, S, 14))
    assert O.rel_err(X, out["G"], out["U"]) <= 1e-12


def test_outputs_orthonormal_and_consistent():
    X = synth.tucker_tensor((14, 12, 10), (4, 4, 4), 15, 1e-2)
    r, p = (3, 3, 3), 3
    out = O.rhkron(X, r, _reuse_factors(X.shape, r, p, 16))
    for u in out["U"]:
        np.testing.assert_allclose(u.T @ u, np.eye(u.shape[1]), atol=1e-13)
    # G = X x_j U_j^T for the final orthonormal factors.
    np.testing.assert_allclose(O.multi_ttm(X, [(j, out["U"][j].T) for j in range(3)]), out["G"], atol=1e-12)


def test_section5_invariants():
    X = synth.tucker_tensor((16, 14, 12), (6, 6, 6), 17, 5e-2)
    r, p = (3, 4, 2), 3
    out = O.rhkron(X, r, _reuse_factors(X.shape, r, p, 18))
    Q, Ghat = out["Q"], out["Ghat"]
    for j in range(3):
        sx = np.linalg.svd(O.unfold(X, j), compute_uv=False)
        sg = np.linalg.svd(O.unfold(Ghat, j), compute_uv=False)
        assert np.all(sg <= sx[: len(sg)] * (1 + 1e-12) + 1e-13)  # Lemma core_svals
    That = O.multi_ttm(Ghat, [(j, Q[j]) for j in range(3)])
    e_rand2 = np.sum((X - That) ** 2)
    assert abs(e_rand2 - (np.sum(X * X) - np.sum(Ghat * Ghat))) <= 1e-12 * np.sum(X * X)  # orthonormal Q
    T = O.reconstruct(out["G"], out["U"])
    e_core2 = np.sum((That - T) ** 2)
    bound = 0.0
    for j in range(3):
        sx = np.linalg.svd(O.unfold(X, j), compute_uv=False)
        bound += np.sum(sx[r[j]:Q[j].shape[1]] ** 2)
    assert e_core2 <= bound * (1 + 1e-10)  # Eq. core_svals
    assert np.sqrt(np.sum((X - T) ** 2)) <= np.sqrt(e_rand2) + np.sqrt(e_core2) + 1e-12


def test_section61_medians_statistical():
    # 100 trials on a 64^3 copy of the Section 7.1 tensor: medians within 1% of 0.4^10 and upper
    # quartiles within 2% (the printed quartiles reach 1.65%).
    golden = json.load(open(os.path.join(GOLDEN, "e1_accuracy.json")))
    X = synth.e1_tensor(64, golden["ratio"], seed=0)
    r, p = (golden["r"],) * 3, golden["p"]
    target = golden["ratio"] ** golden["r"]
    errs = {"rHKron-re": [], "rSTHKron": []}
    for t in range(100):
        out = O.rhkron(X, r, _reuse_factors(X.shape, r, p, 1000 + t))
        errs["rHKron-re"].append(O.rel_err(X, out["G"], out["U"]))
        out = O.rsthkron(X, r, _matrix_factors(X.shape, r, p, [0, 1, 2], 2000 + t))
        errs["rSTHKron"].append(O.rel_err(X, out["G"], out["U"]))
    for name, e in errs.items():
        e = np.array(e)
        assert np.all(e >= target * (1 - 1e-9))
        assert abs(np.median(e) - target) / target <= golden["median_tolerance"], name
        assert np.quantile(e, 0.75) <= target * (1 + golden["upper_quartile_tolerance"]), name


# ------------------------------------------------------------------ gradients

def test_loss_grads_match_finite_differences():
    g = _rng(19)
    X = g.standard_normal((5, 4, 3))
    G = g.standard_normal((2, 3, 2))
    U = [g.standard_normal((5, 2)), g.standard_normal((4, 3)), g.standard_normal((3, 2))]
    gr = O.loss_grads(X, G, U)
    h = 1e-6
    for trial in range(5):
        vX = g.standard_normal(X.shape)
        vG = g.standard_normal(G.shape)
        vU = [g.standard_normal(u.shape) for u in U]
        lp = O.loss(X + h * vX, G + h * vG, [u + h * v for u, v in zip(U, vU)])
        lm = O.loss(X - h * vX, G - h * vG, [u - h * v for u, v in zip(U, vU)])
        fd = (lp - lm) / (2 * h)
        an = np.sum(gr["dX"] * vX) + np.sum(gr["dG"] * vG) + sum(np.sum(a * b) for a, b in zip(gr["dU"], vU))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))
    # single entries
    for (j, i, c) in [(0, 4, 1), (1, 0, 2), (2, 2, 0)]:
        E = np.zeros_like(U[j]); E[i, c] = 1.0
        Up = [u + (h * E if k == j else 0) for k, u in enumerate(U)]
        Um = [u - (h * E if k == j else 0) for k, u in enumerate(U)]
        fd = (O.loss(X, G, Up) - O.loss(X, G, Um)) / (2 * h)
        assert abs(fd - gr["dU"][j][i, c]) <= 1e-6 * max(1.0, abs(fd))
