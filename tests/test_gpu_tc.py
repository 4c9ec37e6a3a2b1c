"""GPU parity of the tensor-core (tcgen05, 3xTF32) TTM path against the FP64 oracle.

Shapes are chosen so that the tensor-core kernel is the one that runs (FP32
data, 16-byte strides, contracted mode >= 32): contraction over the contiguous
mode (K-major), over the last mode and over a middle mode (MN-major), every
supported output width (16..96 columns after padding), several 128-row tiles
with ragged row and K tails.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2211_13028_gb300 import synth
from paper_2211_13028_gb300 import tucker as T
from tests.gpu_helpers import make_X, mats, rel, require_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return require_gpu()


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


@pytest.mark.parametrize("s", [(5, 3), (17, 16), (49, 42), (96, 81), (33, 64)])
def test_tc_two_way_both_majors(dev, s):
    # 100 x 1665: mode 1 -> K-major (K = 100, 13 tiles + 1 ragged row), mode 2 -> MN-major (L = 100 < 128).
    g = _rng(1)
    dims = (100, 1665)
    X, xv, _ = make_X(g.standard_normal(dims), "f32", dev)
    oms = synth.sketch_factors_reuse(dims, s, seed=2, dtype="f32")
    Y = T.tucker_sketch(X, mats(oms, "f32", dev))
    assert rel(to_np(Y[0]), O.ttm(xv, oms[1].T, 1)) <= 1e-5
    assert rel(to_np(Y[1]), O.ttm(xv, oms[0].T, 0)) <= 1e-5


@pytest.mark.parametrize("dims", [(64, 70, 9), (36, 20, 300), (128, 33, 40)])
def test_tc_three_way_middle_and_last(dev, dims):
    g = _rng(3)
    X, xv, _ = make_X(g.standard_normal(dims), "f32", dev)
    s = (7, 6, 5)
    oms = synth.sketch_factors_reuse(dims, s, seed=4, dtype="f32")
    Y = T.tucker_sketch(X, mats(oms, "f32", dev))
    for n in range(3):
        ref = O.multi_ttm(xv, [(j, oms[j].T) for j in range(3) if j != n])
        assert rel(to_np(Y[n]), ref) <= 1e-5


def test_tc_core_wide_factors(dev):
    # the core multi-TTM with k_j near the largest supported width
    g = _rng(5)
    dims, k = (160, 96, 200), (96, 81, 49)
    X, xv, _ = make_X(g.standard_normal(dims), "f32", dev)
    qs = [synth.round_to(O.thin_qr(g.standard_normal((n, kk))), "f32") for n, kk in zip(dims, k)]
    G = T.tucker_core(X, mats(qs, "f32", dev))
    assert rel(to_np(G), O.multi_ttm(xv, [(j, qs[j].T) for j in range(3)])) <= 1e-5


def test_tc_full_size_bench_tensor(dev):
    # the 512^3 FP32 field of the benchmark: mode-1 and mode-3 contractions as the bench runs them
    X = synth.gaussian_bumps(512, 3, 200, 0, 1e-4, dev, "f32")
    xv = synth.from_fortran(X)
    s = (6, 7, 7)
    oms = synth.sketch_factors_reuse(X.shape, s, seed=1, dtype="f32")
    Y = T.tucker_sketch(X, mats(oms, "f32", dev))
    for n in range(3):
        ref = O.multi_ttm(xv, [(j, oms[j].T) for j in range(3) if j != n])
        assert rel(to_np(Y[n]), ref) <= 1e-5
    st, _ = T.tk_sync_status(dev)
    assert st == 0


@pytest.mark.parametrize("need_dx", [False, True])
def test_tc_fused_residual_loss_and_gradient(dev, need_dx):
    # last reconstruction step fused with the residual on tensor cores (r_3 >= 32), gradients from
    # sketches of X plus FP64 core corrections
    g = _rng(7)
    dims, rk = (96, 80, 72), (12, 10, 36)
    x = synth.round_to(g.standard_normal(dims), "f32")
    G = synth.round_to(g.standard_normal(rk), "f32")
    U = [synth.round_to(g.standard_normal((nn, k)) / np.sqrt(nn), "f32") for nn, k in zip(dims, rk)]
    Xd, Gd, Ud = synth.fortran(x, "f32", dev), synth.fortran(G, "f32", dev), mats(U, "f32", dev)
    ref_loss = O.loss(x, G, U)
    assert abs(T.tucker_loss(Xd, Gd, Ud) - ref_loss) <= 1e-5 * ref_loss
    dG, dU, dX = T.tucker_reconstruct_backward(Xd, Gd, Ud, grad_scale=0.25, need_dX=need_dx)
    ref = O.loss_grads(x, G, U)
    assert rel(to_np(dG), 0.25 * ref["dG"]) <= 1e-4
    for j in range(3):
        assert rel(to_np(dU[j]), 0.25 * ref["dU"][j]) <= 1e-4
    if need_dx:
        assert rel(to_np(dX), 0.25 * ref["dX"]) <= 1e-5
    st, _ = T.tk_sync_status(dev)
    assert st == 0


def test_tc_rel_err_fused_matches_oracle(dev):
    # rHKron-re with r_3 = 32 so the relative error uses the fused tensor-core residual
    dims, r, p = (128, 96, 112), (20, 24, 32), 6
    core = synth.decaying_core((40, 40, 40), 0.8, seed=31)
    x = synth.tucker_tensor(dims, (40, 40, 40), seed=32, noise_rel=1e-3, core=core)
    X, xv, _ = make_X(x, "f32", dev)
    s = O.subranks_reuse(r, p)[0]
    oms = synth.sketch_factors_reuse(dims, s, seed=33, dtype="f32")
    G, U, err = T.tucker_rhkron(X, r, p, mats(oms, "f32", dev))
    ref = O.rhkron(xv, r, oms)
    assert abs(err - O.rel_err(xv, ref["G"], ref["U"])) <= 1e-5
    # the error the GPU reports is the error of the factors it returned
    assert abs(err - O.rel_err(xv, to_np(G), [to_np(u) for u in U])) <= 1e-6


@pytest.mark.parametrize("dims,k", [((40, 96, 77), (40, 20, 77)), ((32, 130, 65), (32, 48, 65)),
                                    ((60, 64, 50), (60, 16, 50)), ((44, 512, 9), (44, 64, 9))])
def test_tc_short_rows_packed_tiles(dev, dims, k):
    # the first product contracts mode 2 with only L = dims[0] (32..60) rows before it: the tensor-core
    # kernel packs floor(128 / L) consecutive slabs into each 128-row tile (the last one partial)
    g = _rng(11)
    X, xv, _ = make_X(g.standard_normal(dims), "f32", dev)
    qs = [synth.round_to(O.thin_qr(g.standard_normal((n, kk))), "f32") for n, kk in zip(dims, k)]
    T.tk_profile(True, dev)
    G = T.tucker_core(X, mats(qs, "f32", dev))
    prof = T.tk_profile_read(dev)
    T.tk_profile(False, dev)
    assert "xpass_tc" in prof  # X was streamed by the tensor-core kernel
    ref = O.multi_ttm(xv, [(j, qs[j].T) for j in range(3)])
    assert rel(to_np(G), ref) <= 1e-5


@pytest.mark.parametrize("dims,k", [((500, 40, 40), (48, 40, 40)), ((40, 40, 500), (40, 40, 44)),
                                    ((48, 44, 1000), (48, 44, 64))])
def test_tc_few_tiles_split_k(dev, dims, k):
    # the first product has a long contraction (500-1000) and only 13-17 row tiles: its K chunks are
    # split over several CTAs and the partial products summed in order afterwards
    g = _rng(12)
    X, xv, _ = make_X(g.standard_normal(dims), "f32", dev)
    qs = [synth.round_to(O.thin_qr(g.standard_normal((n, kk))), "f32") for n, kk in zip(dims, k)]
    T.tk_profile(True, dev)
    G = T.tucker_core(X, mats(qs, "f32", dev))
    prof = T.tk_profile_read(dev)
    T.tk_profile(False, dev)
    assert "xpass_tc" in prof
    ref = O.multi_ttm(xv, [(j, qs[j].T) for j in range(3)])
    assert rel(to_np(G), ref) <= 1e-5
    G2 = T.tucker_core(X, mats(qs, "f32", dev))
    assert torch.equal(G, G2)  # the partial sums are added in a fixed order
