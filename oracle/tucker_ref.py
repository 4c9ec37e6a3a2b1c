"""Plain FP64 statement of the randomized Tucker methods of "Parallel
Randomized Tucker Decomposition Algorithms" (arXiv 2211.13028).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
the CPU-baseline leg of bench.py, never by the product path.  It shares no code
with the CUDA path.

Every step is written in the paper's order and notation with NumPy (float64,
LAPACK for QR and SVD as single library steps) and without any blocking,
fusion or reordering beyond what the definitions state.  Tensors are numpy
arrays indexed ``X[i1, ..., id]`` with zero-based modes 0..d-1 standing for the
paper's modes 1..d.

Pins (tests/test_oracle_*.py):
  * unfold / ttm / multi_ttm: elementwise brute-force loops, the multi-TTM
    Kronecker unfolding identity of Section 2.1, round trips.
  * thin_qr: Q^T Q = I, Q R = Y, R upper triangular with positive diagonal
    (which fixes Q uniquely), classical Gram-Schmidt on tiny inputs.
  * sthosvd: closed-form error 0.4^r on the Section 7.1 tensor, the STHOSVD
    error identity (sum of discarded squared singular values).
  * fmix32 / rademacher_signs / rhkron_srht: the published MurmurHash3_x86_32
    results for the empty input (= fmix32 of the seed); each sign is the top
    bit of fmix32; the Kronecker-SRHT sketch Y_(n) = X_(n) D_n (kron H_j)
    checked against the explicitly formed matrix on tiny inputs, balanced
    signs, exact recovery of exactly low-rank tensors.
  * rhkron / rsthkron / rhkron_noreuse: exact recovery of exactly low-rank
    tensors, the Section 5 invariants (core singular values bounded by those
    of X, the core error bound Eq. core_svals, Pythagoras for orthonormal
    factors), the Section 7.1 medians (statistical).
  * subranks_reuse / subranks_matrix: the vectors and matrices printed for
    the Miranda and SP runs (Sections 7.5-7.6).
  * loss_grads: central finite differences in FP64.
  * philox4x32_10 / gaussian_factor: the known-answer vectors published with
    the Philox generator; uniformity and independence of the 32-bit words;
    the Box-Muller draws against the normal distribution (moments and a
    Kolmogorov-Smirnov test).
"""
from __future__ import annotations

import itertools
from typing import Dict, List, Sequence, Tuple

import numpy as np

__all__ = [
    "unfold", "fold", "ttm", "ttm_loops", "multi_ttm", "kron_unfolded_multi_ttm", "kron_omega",
    "thin_qr", "leading_left_singular_vectors", "sthosvd", "canonical_signs",
    "subranks_reuse", "subranks_matrix", "balanced_factors",
    "rhkron", "rsthkron", "rhkron_noreuse", "fmix32", "rademacher_signs", "srht_sign_tensor", "rhkron_srht",
    "philox4x32_10", "philox_blocks", "gaussian_factor",
    "reconstruct", "rel_err", "loss", "loss_grads",
]


# ---------------------------------------------------------------- Section 2.1

def unfold(X: np.ndarray, j: int) -> np.ndarray:
    """Mode-j unfolding X_(j) (Section 2.1).

    n_j x prod_{k != j} n_k; its columns are the mode-j fibres, ordered with the
    lowest remaining mode varying fastest.
    """
    return np.reshape(np.moveaxis(X, j, 0), (X.shape[j], -1), order="F")


def fold(M: np.ndarray, j: int, shape: Sequence[int]) -> np.ndarray:
    """Inverse of ``unfold`` for a tensor of the given shape."""
    rest = [int(shape[k]) for k in range(len(shape)) if k != j]
    return np.moveaxis(np.reshape(M, [int(shape[j])] + rest, order="F"), 0, j)


def ttm(X: np.ndarray, A: np.ndarray, j: int) -> np.ndarray:
    """Tensor-times-matrix Y = X x_j A, defined by Y_(j) = A X_(j) (Section 2.1).

    A is m x n_j; Y has mode j of size m.
    """
    if A.shape[1] != X.shape[j]:
        raise ValueError("ttm: A has %d columns, mode %d has size %d" % (A.shape[1], j, X.shape[j]))
    shape = list(X.shape)
    shape[j] = A.shape[0]
    return fold(A @ unfold(X, j), j, shape)


def ttm_loops(X: np.ndarray, A: np.ndarray, j: int) -> np.ndarray:
    """Elementwise TTM: Y[..., a, ...] = sum_i A[a, i] X[..., i, ...] (pure Python loops)."""
    shape = list(X.shape)
    shape[j] = A.shape[0]
    Y = np.zeros(shape)
    for idx in itertools.product(*[range(s) for s in shape]):
        acc = 0.0
        for i in range(X.shape[j]):
            src = list(idx)
            src[j] = i
            acc += A[idx[j], i] * X[tuple(src)]
        Y[idx] = acc
    return Y


def multi_ttm(X: np.ndarray, mats: Sequence[Tuple[int, np.ndarray]]) -> np.ndarray:
    """Multi-TTM X x_{j1} A_{j1} x_{j2} A_{j2} ... applied in the listed order (Section 2.1)."""
    Y = X
    for j, A in mats:
        Y = ttm(Y, A, j)
    return Y


def kron_unfolded_multi_ttm(X: np.ndarray, A: Sequence[np.ndarray], j: int) -> np.ndarray:
    """Mode-j unfolding of X x_1 A_1 ... x_d A_d by the Kronecker formula of Section 2.1.

    A_j X_(j) (A_d kron ... kron A_{j+1} kron A_{j-1} kron ... kron A_1)^T, with the
    Kronecker product formed explicitly (test-sized inputs only).
    """
    d = X.ndim
    K = np.ones((1, 1))
    for k in range(d - 1, -1, -1):
        if k != j:
            K = np.kron(K, A[k])
    return A[j] @ unfold(X, j) @ K.T


def kron_omega(phis: Sequence[np.ndarray], j: int) -> np.ndarray:
    """Omega_j = (Phi_d kron ... kron Phi_{j+1} kron Phi_{j-1} kron ... kron Phi_1)^T (Section 4.2)."""
    K = np.ones((1, 1))
    for k in range(len(phis) - 1, -1, -1):
        if k != j:
            K = np.kron(K, phis[k])
    return K.T


# ------------------------------------------------------- Algorithms RRF, STHOSVD

def thin_qr(Y: np.ndarray) -> np.ndarray:
    """Q of the thin QR Y = Q R with diag(R) >= 0 (Algorithm RRF, second step).

    Reading: when Y has at least as many columns as rows its columns already
    span the whole space and Q is the identity (the sketch width is
    min(n_j, number of sketch columns)).
    """
    m, k = Y.shape
    if k >= m:
        return np.eye(m)
    Q, R = np.linalg.qr(Y, mode="reduced")
    return Q * np.where(np.diag(R) < 0.0, -1.0, 1.0)[None, :]


def leading_left_singular_vectors(M: np.ndarray, r: int) -> np.ndarray:
    """First r left singular vectors of M (LAPACK SVD)."""
    u, _, _ = np.linalg.svd(M, full_matrices=False)
    return u[:, :r]


def sthosvd(X: np.ndarray, r: Sequence[int], order: Sequence[int] | None = None):
    """Algorithm STHOSVD: for each mode in ``order``, U_j = first r_j left singular
    vectors of the current G_(j), then G <- G x_j U_j^T.

    Returns (G, [U_j], discarded) where discarded[t] is the sum of the squared
    singular values dropped at step t.
    """
    d = X.ndim
    order = list(range(d)) if order is None else list(order)
    G = X
    U: List[np.ndarray] = [None] * d  # type: ignore
    discarded = []
    for j in order:
        u, sv, _ = np.linalg.svd(unfold(G, j), full_matrices=False)
        U[j] = u[:, : r[j]]
        discarded.append(float(np.sum(sv[r[j]:] ** 2)))
        G = ttm(G, U[j].T, j)
    return G, U, discarded


def canonical_signs(G: np.ndarray, U: Sequence[np.ndarray]):
    """Fix the sign gauge: each column of U_j has its largest-magnitude entry
    (lowest row on ties) positive; the matching slice of G flips with it."""
    G = G.copy()
    U = [u.copy() for u in U]
    for j, u in enumerate(U):
        for c in range(u.shape[1]):
            i = int(np.argmax(np.abs(u[:, c])))
            if u[i, c] < 0:
                u[:, c] = -u[:, c]
                sl = [slice(None)] * G.ndim
                sl[j] = c
                G[tuple(sl)] = -G[tuple(sl)]
    return G, U


# --------------------------------------------------------------- subranks

def _ceil_root_ratio(P: int, ell: int, d: int) -> int:
    """Smallest integer s with s >= P^(1/(d-1)) / ell, i.e. (s*ell)^(d-1) >= P."""
    s = max(1, int((P ** (1.0 / (d - 1))) / ell))
    while s > 1 and ((s - 1) * ell) ** (d - 1) >= P:
        s -= 1
    while (s * ell) ** (d - 1) < P:
        s += 1
    return s


def subranks_reuse(r: Sequence[int], p: int):
    """Subrank vector of Algorithm rHKron-re (Section 4.3).

    The paper's formula s_i = ceil((prod_j l_j)^(1/(d-1)) / l_i), then (reading)
    each entry, largest first (ties: lowest mode), is lowered to the smallest
    value that keeps prod_{k != j} s_k >= l_j for every mode j.
    Returns (s, widths) with widths[j] = prod_{k != j} s_k.
    """
    d = len(r)
    ell = [int(x) + int(p) for x in r]
    P = 1
    for x in ell:
        P *= x
    s = [_ceil_root_ratio(P, ell[i], d) for i in range(d)]
    for i in sorted(range(d), key=lambda t: (-s[t], t)):
        need = 1
        for j in range(d):
            if j == i:
                continue
            rest = 1
            for k in range(d):
                if k != i and k != j:
                    rest *= s[k]
            need = max(need, -(-ell[j] // rest))
        s[i] = min(s[i], need)
    widths = []
    for j in range(d):
        w = 1
        for k in range(d):
            if k != j:
                w *= s[k]
        widths.append(w)
    return s, widths


def balanced_factors(ell: int, m: int):
    """Smallest L >= ell that is a product of m integers >= 2, and its most balanced
    such factorisation (smallest largest factor, compared as sorted-descending
    tuples).  Reading of Section 4.2's subrank heuristic."""
    def facts(n, m, lo):
        if m == 1:
            if n >= lo:
                yield (n,)
            return
        f = lo
        while f ** m <= n:
            if n % f == 0:
                for rest in facts(n // f, m - 1, f):
                    yield (f,) + rest
            f += 1

    L = max(int(ell), 2 ** m)
    while True:
        best = None
        for fs in facts(L, m, 2):
            key = tuple(sorted(fs, reverse=True))
            if best is None or key < best:
                best = key
        if best is not None:
            return L, list(best)
        L += 1


def subranks_matrix(r: Sequence[int], p: int, order: Sequence[int] | None = None):
    """Subrank matrix S of Algorithm rSTHKron (Section 4.2).

    Row j holds d-1 integer factors (each >= 2) of l_j' >= l_j = r_j + p, l_j' the
    smallest such value, most balanced factorisation.  Reading: the factors
    go in descending order to the other modes taken in processing order.  The
    diagonal is 1.  Returns (S, widths) with widths[j] = l_j'.
    """
    d = len(r)
    order = list(range(d)) if order is None else list(order)
    S = np.ones((d, d), dtype=np.int64)
    widths = []
    for j in range(d):
        L, fs = balanced_factors(int(r[j]) + int(p), d - 1)
        others = [k for k in order if k != j]
        for k, f in zip(others, fs):
            S[j, k] = f
        widths.append(L)
    return S, widths


# ------------------------------------------------------ Algorithms rHKron-re, rSTHKron

def rhkron(X: np.ndarray, r: Sequence[int], omegas: Sequence[np.ndarray], order: Sequence[int] | None = None):
    """Algorithm rHKron-re (randomized HOSVD, Kronecker sketch, reused factors).

    omegas[j] = Phi_j^T (n_j x s_j).  For each mode n: Y = X x_{j != n} Phi_j,
    Q_n from the thin QR of Y_(n); then Ghat = X x_1 Q_1^T ... x_d Q_d^T,
    [G, {V_j}] = STHOSVD(Ghat, r) and U_j = Q_j V_j.
    """
    d = X.ndim
    order = list(range(d)) if order is None else list(order)
    Q, Ys = [], []
    for n in range(d):
        Y = multi_ttm(X, [(j, omegas[j].T) for j in range(d) if j != n])
        Ys.append(Y)
        Q.append(thin_qr(unfold(Y, n)))
    Ghat = multi_ttm(X, [(j, Q[j].T) for j in range(d)])
    G, V, _ = sthosvd(Ghat, r, order)
    U = [Q[j] @ V[j] for j in range(d)]
    G, U = canonical_signs(G, U)
    return dict(G=G, U=U, Q=Q, Y=Ys, Ghat=Ghat)


# ---------------------------------------------------------------- Gaussian sketch factors (Alg. rHKron-re draw lines)

_M32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """Philox4x32 with 10 rounds (Salmon, Moraes, Dror and Shaw, "Parallel
    random numbers: as easy as 1, 2, 3", SC'11), for arrays of counter blocks.

    ctr: (N, 4) and key: (N, 2) arrays of 32-bit words.  A round multiplies
    words 0 and 2 by 0xD2511F53 and 0xCD9E8D57 (64-bit products split into
    high and low halves) and returns (hi_2 ^ c_1 ^ k_0, lo_2, hi_0 ^ c_3 ^ k_1,
    lo_0); before every round but the first the key advances by the Weyl
    increments (0x9E3779B9, 0xBB67AE85).  Returns (N, 4) uint64 words.
    """
    c = np.asarray(ctr, dtype=np.uint64) & _M32
    k = np.asarray(key, dtype=np.uint64) & _M32
    c0, c1, c2, c3 = (c[:, i].copy() for i in range(4))
    k0, k1 = k[:, 0].copy(), k[:, 1].copy()
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + np.uint64(0x9E3779B9)) & _M32
            k1 = (k1 + np.uint64(0xBB67AE85)) & _M32
        p0 = np.uint64(0xD2511F53) * c0
        p2 = np.uint64(0xCD9E8D57) * c2
        c0, c1, c2, c3 = ((p2 >> np.uint64(32)) ^ c1 ^ k0, p2 & _M32,
                          (p0 >> np.uint64(32)) ^ c3 ^ k1, p0 & _M32)
    return np.stack([c0, c1, c2, c3], axis=1)


def philox_blocks(seed: int, stream: int, offset: int, nblocks: int) -> np.ndarray:
    """Blocks offset .. offset + nblocks - 1 of the sketch-factor stream: counter
    (i mod 2^32, i div 2^32, stream, 0), key (seed mod 2^32, seed div 2^32).
    Returns (nblocks, 4) uint64 words (each below 2^32)."""
    i = np.arange(offset, offset + nblocks, dtype=np.uint64)
    ctr = np.stack([i & _M32, i >> np.uint64(32), np.full_like(i, stream & 0xFFFFFFFF),
                    np.zeros_like(i)], axis=1)
    key = np.tile(np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64), (nblocks, 1))
    return philox4x32_10(ctr, key)


def gaussian_factor(rows: int, cols: int, seed: int, stream: int) -> np.ndarray:
    """A rows x cols matrix of N(0, 1) draws (the paper's Gaussian sketch
    factors), FP64.  Element e = row + rows * col (column-major) is output
    e mod 4 of block e div 4 of ``philox_blocks(seed, stream, 0, .)``; a block
    (x0, x1, x2, x3) gives two Box-Muller pairs: with u = (x0 + 1) 2^-32 in
    (0, 1] and t = x1 2^-32, r = sqrt(-2 ln u) and (r cos 2 pi t, r sin 2 pi t);
    likewise from (x2, x3)."""
    n = rows * cols
    nb = (n + 3) // 4
    x = philox_blocks(seed, stream, 0, nb).astype(np.float64)
    out = np.empty((nb, 4))
    for a in (0, 2):
        u = (x[:, a] + 1.0) * 2.0 ** -32
        t = x[:, a + 1] * 2.0 ** -32
        r = np.sqrt(-2.0 * np.log(u))
        out[:, a] = r * np.cos(2.0 * np.pi * t)
        out[:, a + 1] = r * np.sin(2.0 * np.pi * t)
    return out.reshape(-1)[:n].reshape((rows, cols), order="F")


# ---------------------------------------------------------------- Section 5, Eq. srht_kron

def fmix32(x: np.ndarray) -> np.ndarray:
    """The 32-bit finalizer of MurmurHash3 (Appleby): x ^= x >> 16, x *= 0x85EBCA6B,
    x ^= x >> 13, x *= 0xC2B2AE35, x ^= x >> 16, all mod 2^32.  On its own it is
    MurmurHash3_x86_32 of the empty input with seed x."""
    M32 = np.uint64(0xFFFFFFFF)
    x = np.asarray(x, dtype=np.uint64) & M32
    x = x ^ (x >> np.uint64(16))
    x = (x * np.uint64(0x85EBCA6B)) & M32
    x = x ^ (x >> np.uint64(13))
    x = (x * np.uint64(0xC2B2AE35)) & M32
    return x ^ (x >> np.uint64(16))


def rademacher_signs(seed: int, n: int, c: np.ndarray) -> np.ndarray:
    """Entries c of the Rademacher diagonal D_n of the Kronecker-SRHT sketch.

    The paper draws D i.i.d. uniformly from {+1, -1} over the columns of the
    unfolding, not as a Kronecker product; here the draw is the counter-based
    generator the C header defines (tk_rademacher): u = seed + 0x9E3779B9 (n + 1)
    mod 2^32, x = c XOR u, the MurmurHash3 32-bit finalizer of x, and -1 when
    its top bit is set.
    """
    M32 = np.uint64(0xFFFFFFFF)
    u = (np.uint64(seed) + np.uint64(0x9E3779B9) * np.uint64(n + 1)) & M32
    x = fmix32((np.asarray(c, dtype=np.uint64) & M32) ^ u)
    return np.where((x >> np.uint64(31)) & np.uint64(1), -1.0, 1.0)


def srht_sign_tensor(shape: Sequence[int], n: int, seed: int) -> np.ndarray:
    """D_n laid out over X's index space: entry (i_1..i_d) is the sign of the
    column of X_(n) that holds it (the other modes' indices, mode 1 fastest)."""
    d = len(shape)
    c = np.zeros(shape, dtype=np.int64)
    stride = 1
    for j in range(d):
        if j == n:
            continue
        idx = np.arange(shape[j], dtype=np.int64).reshape([-1 if k == j else 1 for k in range(d)])
        c = c + idx * stride
        stride *= shape[j]
    return rademacher_signs(seed, n, c)


def rhkron_srht(X: np.ndarray, r: Sequence[int], H: Sequence[np.ndarray], seed: int,
                order: Sequence[int] | None = None):
    """rHKron-re with the Kronecker-SRHT sketch of Section 5.

    H[j] is the n_j x s_j factor (sampled columns of the scaled Walsh-Hadamard
    matrix); for each mode n, Y_(n) = X_(n) D_n (kron of the H_j, j != n), i.e.
    Y_n = (D_n o X) x_{j != n} H_j^T, then the steps of rHKron-re: Q_n from the
    thin QR, Ghat = X x_j Q_j^T, STHOSVD(Ghat, r), U_j = Q_j V_j.
    """
    d = X.ndim
    order = list(range(d)) if order is None else list(order)
    Q, Ys = [], []
    for n in range(d):
        Xs = X * srht_sign_tensor(X.shape, n, seed)
        Y = multi_ttm(Xs, [(j, H[j].T) for j in range(d) if j != n])
        Ys.append(Y)
        Q.append(thin_qr(unfold(Y, n)))
    Ghat = multi_ttm(X, [(j, Q[j].T) for j in range(d)])
    G, V, _ = sthosvd(Ghat, r, order)
    U = [Q[j] @ V[j] for j in range(d)]
    G, U = canonical_signs(G, U)
    return dict(G=G, U=U, Q=Q, Y=Ys, Ghat=Ghat)


def rsthkron(X: np.ndarray, r: Sequence[int], omegas: Dict[Tuple[int, int], np.ndarray],
             order: Sequence[int] | None = None):
    """Algorithm rSTHKron (randomized STHOSVD with a Kronecker sketch).

    Modes are processed in ``order``.  For mode j: Y = Ghat x_{k != j} Phi_{j,k}
    with omegas[(j, k)] = Phi_{j,k}^T sized to the current mode k of Ghat;
    Q_j from the thin QR of Y_(j); Ghat <- Ghat x_j Q_j^T.  Then
    [G, {V_j}] = STHOSVD(Ghat, r) in the same order and U_j = Q_j V_j.
    """
    d = X.ndim
    order = list(range(d)) if order is None else list(order)
    Ghat = X
    Q: List[np.ndarray] = [None] * d  # type: ignore
    Ys = {}
    for j in order:
        Y = multi_ttm(Ghat, [(k, omegas[(j, k)].T) for k in range(d) if k != j])
        Ys[j] = Y
        Q[j] = thin_qr(unfold(Y, j))
        Ghat = ttm(Ghat, Q[j].T, j)
    G, V, _ = sthosvd(Ghat, r, order)
    U = [Q[j] @ V[j] for j in range(d)]
    G, U = canonical_signs(G, U)
    return dict(G=G, U=U, Q=Q, Y=Ys, Ghat=Ghat)


def rhkron_noreuse(X: np.ndarray, r: Sequence[int], omegas: Dict[Tuple[int, int], np.ndarray],
                   order: Sequence[int] | None = None):
    """Appendix Algorithm rHKron: like rHKron-re but with fresh factors per mode,
    omegas[(j, k)] = Phi_{j,k}^T (n_k x s_{j,k})."""
    d = X.ndim
    order = list(range(d)) if order is None else list(order)
    Q = []
    for n in range(d):
        Y = multi_ttm(X, [(k, omegas[(n, k)].T) for k in range(d) if k != n])
        Q.append(thin_qr(unfold(Y, n)))
    Ghat = multi_ttm(X, [(j, Q[j].T) for j in range(d)])
    G, V, _ = sthosvd(Ghat, r, order)
    U = [Q[j] @ V[j] for j in range(d)]
    G, U = canonical_signs(G, U)
    return dict(G=G, U=U, Q=Q, Ghat=Ghat)


# ------------------------------------------------ reconstruction, error, loss

def reconstruct(G: np.ndarray, U: Sequence[np.ndarray]) -> np.ndarray:
    """T = G x_1 U_1 ... x_d U_d (Section 2.2)."""
    return multi_ttm(G, [(j, U[j]) for j in range(G.ndim)])


def rel_err(X: np.ndarray, G: np.ndarray, U: Sequence[np.ndarray]) -> float:
    """||X - G x_1 U_1 ... x_d U_d|| / ||X|| with the residual formed explicitly."""
    return float(np.linalg.norm(X - reconstruct(G, U)) / np.linalg.norm(X))


def loss(X: np.ndarray, G: np.ndarray, U: Sequence[np.ndarray]) -> float:
    """||X - G x_1 U_1 ... x_d U_d||^2."""
    R = X - reconstruct(G, U)
    return float(np.sum(R * R))


def loss_grads(X: np.ndarray, G: np.ndarray, U: Sequence[np.ndarray]):
    """Gradients of ||X - G x_j U_j||^2 with R = X - G x_j U_j:
    dX = 2R, dG = -2 R x_1 U_1^T ... x_d U_d^T,
    dU_n = -2 (R x_{j != n} U_j^T)_(n) G_(n)^T  (from the unfolding identity of Section 2.1).
    """
    d = X.ndim
    R = X - reconstruct(G, U)
    dG = -2.0 * multi_ttm(R, [(j, U[j].T) for j in range(d)])
    dU = []
    for n in range(d):
        Z = multi_ttm(R, [(j, U[j].T) for j in range(d) if j != n])
        dU.append(-2.0 * unfold(Z, n) @ unfold(G, n).T)
    return dict(dX=2.0 * R, dG=dG, dU=dU)
