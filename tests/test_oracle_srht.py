"""Oracle pins for the Kronecker-SRHT sketch (Section 5, Eq. srht_kron)."""
import json
import os

import numpy as np

import oracle as O
from paper_2211_13028_gb300 import synth


def test_hadamard_columns_orthonormal():
    H = synth.hadamard_columns(64, 10, seed=3)
    assert H.shape == (64, 10)
    assert np.allclose(np.abs(H), 1.0 / 8.0)
    assert np.max(np.abs(H.T @ H - np.eye(10))) <= 1e-14
    full = synth.hadamard_columns(16, 16, seed=4)  # all columns: the orthonormal Walsh-Hadamard matrix
    assert np.max(np.abs(full @ full.T - np.eye(16))) <= 1e-14
    # Sylvester recursion: H_2n = [[H_n, H_n], [H_n, -H_n]] (columns sorted, so all 16 = the matrix)
    h8 = synth.hadamard_columns(8, 8, seed=5) * np.sqrt(8.0)
    h16 = full * 4.0
    assert np.array_equal(h16, np.block([[h8, h8], [h8, -h8]]))


def test_fmix32_known_answers():
    # the published MurmurHash3_x86_32 results for the empty input are fmix32(seed)
    with open(os.path.join(os.path.dirname(__file__), "golden", "murmur3_x86_32_empty_kat.json")) as f:
        kat = json.load(f)
    seeds = np.array([int(v["seed"], 16) for v in kat["vectors"]], dtype=np.uint64)
    want = [int(v["hash"], 16) for v in kat["vectors"]]
    assert [int(h) for h in O.fmix32(seeds)] == want


def test_rademacher_sign_is_the_top_bit_of_fmix32():
    # with the per-mode offset u = seed + 0x9E3779B9 (n + 1) cancelled (seed = -u0 mod 2^32), entry c
    # of D_n is -1 exactly when fmix32(c) has its top bit set
    c = np.arange(4096, dtype=np.uint64) * np.uint64(2654435761) & np.uint64(0xFFFFFFFF)
    for n in (0, 2):
        seed = (-(0x9E3779B9 * (n + 1))) % (1 << 32)
        sg = O.rademacher_signs(seed, n, c)
        top = (O.fmix32(c) >> np.uint64(31)).astype(bool)
        assert np.array_equal(sg == -1.0, top)
    assert int(O.fmix32(np.uint64(1))) >> 31 == 0 and O.rademacher_signs(-0x9E3779B9 % (1 << 32), 0, [1])[0] == 1.0


def test_rademacher_signs_balanced():
    c = np.arange(1 << 16)
    for seed, n in ((0, 0), (12345, 1), (2**31 + 7, 2)):
        sg = O.rademacher_signs(seed, n, c)
        assert set(np.unique(sg)) == {-1.0, 1.0}
        assert abs(sg.mean()) < 0.02
        assert abs(np.mean(sg[1:] == sg[:-1]) - 0.5) < 0.02  # no run structure between neighbours
    # different modes draw different diagonals
    assert np.mean(O.rademacher_signs(9, 0, c) == O.rademacher_signs(9, 1, c)) < 0.55


def test_srht_sketch_is_the_explicit_matrix_product():
    # Y_(n) = X_(n) D_n (kron of the H_j): D_n indexed by the column of the unfolding
    g = np.random.Generator(np.random.PCG64(6))
    dims, s, seed = (4, 2, 8), (2, 2, 3), 77
    x = g.standard_normal(dims)
    H = synth.sketch_factors_srht(dims, s, seed=8)
    ref = O.rhkron_srht(x, (1, 1, 1), H, seed)
    for n in range(3):
        ncols = int(np.prod([dims[j] for j in range(3) if j != n]))
        D = np.diag(O.rademacher_signs(seed, n, np.arange(ncols)))
        Om = D @ O.kron_omega([h.T for h in H], n)
        assert np.allclose(O.unfold(ref["Y"][n], n), O.unfold(x, n) @ Om, atol=1e-13)


def test_rhkron_srht_recovers_exact_low_rank():
    dims, rk = (32, 16, 32), (4, 5, 3)
    x = synth.tucker_tensor(dims, rk, seed=21, noise_rel=0.0)
    s = O.subranks_reuse(rk, 6)[0]
    H = synth.sketch_factors_srht(dims, s, seed=22)
    ref = O.rhkron_srht(x, rk, H, seed=5)
    assert O.rel_err(x, ref["G"], ref["U"]) <= 1e-12
