"""GPU parity of the BF16 tensor-core TTM (tcgen05 kind::f16, factor split into
BF16 hi + lo) against the FP64 oracle applied to the BF16-rounded tensor.

The factor split leaves a relative error of about 2^-18 per factor entry and
products of BF16 values are exact in the FP32 accumulator, so the products
agree with the oracle to ~1e-5.  The shapes put every contraction layout on
the kernel: mode 1 (contiguous: K-major tiles), a middle mode and the last mode
(MN-major tiles), with ragged row tiles (rows not a multiple of 128), ragged
K chunks (contracted dimension not a multiple of 64) and output widths that
take one column block (<= 96) or several blocks of 64.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2211_13028_gb300 import synth
from paper_2211_13028_gb300 import tucker as T
from tests.gpu_helpers import align, make_X, mats, rel, require_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return require_gpu()


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


@pytest.mark.parametrize("dims,k", [((136, 72, 40), (7, 16, 33)), ((200, 64, 24), (96, 50, 17)),
                                    ((64, 40, 136), (130, 40, 80))])
def test_bf16_core_each_layout(dev, dims, k):
    g = _rng(1)
    X, xv, _ = make_X(g.standard_normal(dims), "bf16", dev)
    qs = [O.thin_qr(g.standard_normal((n, kk))) if kk <= n else g.standard_normal((n, kk)) / np.sqrt(n)
          for n, kk in zip(dims, k)]
    for j in range(3):  # one mode at a time: the first TTM of each streams the BF16 tensor
        M = [synth.fmat(np.eye(n), "f32", dev) for n in dims]
        M[j] = synth.fmat(qs[j], "f32", dev)
        G = T.tucker_core(X, M)
        ref = O.ttm(xv, synth.round_to(qs[j], "f32").T, j)
        assert rel(to_np(G), ref) <= 2e-5, j
    st, _ = T.tk_sync_status(dev)
    assert st == 0


@pytest.mark.parametrize("dims,s", [((136, 72, 40), (5, 6, 4)), ((256, 128, 96), (9, 9, 9))])
def test_bf16_sketch(dev, dims, s):
    g = _rng(2)
    X, xv, _ = make_X(g.standard_normal(dims), "bf16", dev)
    oms = synth.sketch_factors_reuse(dims, s, seed=3, dtype="bf16")
    Y = T.tucker_sketch(X, mats(oms, "bf16", dev))
    for n in range(3):
        ref = O.multi_ttm(xv, [(j, oms[j].T) for j in range(3) if j != n])
        assert rel(to_np(Y[n]), ref) <= 2e-5


def test_bf16_refinement_pass_matters(dev):
    # rHKron-re on BF16 data: with the Q hi + lo pass (refine = 0) the core matches the
    # oracle's to ~1e-5; with Q rounded once to BF16 (refine = -1) the core carries the
    # BF16 rounding of Q (~1e-3).  Core entries decay by 0.5 per index, so the factors
    # are well determined and the comparison after the sign gauge is meaningful.
    dims, r, p = (128, 96, 80), (8, 8, 8), 6
    core = synth.decaying_core((12, 12, 12), 0.5, seed=5)
    x = synth.tucker_tensor(dims, (12, 12, 12), seed=6, noise_rel=1e-4, core=core)
    X, xv, _ = make_X(x, "bf16", dev)
    s = O.subranks_reuse(r, p)[0]
    oms = synth.sketch_factors_reuse(dims, s, seed=7, dtype="bf16")
    ref = O.rhkron(xv, r, oms)

    def core_err(**kw):
        G, U, _ = T.tucker_rhkron(X, r, p, mats(oms, "bf16", dev), **kw)
        Ga, _ = align(to_np(G), [to_np(u) for u in U], ref["U"])
        return rel(Ga, ref["G"])

    e_refined, e_single = core_err(), core_err(refine=-1)
    assert e_refined <= 2e-5
    assert e_single >= 10 * e_refined


def test_bf16_fused_residual_loss_and_gradient(dev):
    # the last reconstruction TTM fused with the residual against the BF16 tensor (no
    # FP32 Xhat); dX is returned in X's dtype, so it carries one BF16 rounding
    g = _rng(8)
    dims, rk = (96, 80, 72), (12, 10, 36)
    x = synth.round_to(g.standard_normal(dims), "bf16")
    G = synth.round_to(g.standard_normal(rk), "f32")
    U = [synth.round_to(g.standard_normal((nn, k)) / np.sqrt(nn), "f32") for nn, k in zip(dims, rk)]
    Xd, Gd, Ud = synth.fortran(x, "bf16", dev), synth.fortran(G, "f32", dev), mats(U, "f32", dev)
    ref_loss = O.loss(x, G, U)
    assert abs(T.tucker_loss(Xd, Gd, Ud) - ref_loss) <= 1e-5 * ref_loss
    dG, dU, dX = T.tucker_reconstruct_backward(Xd, Gd, Ud, grad_scale=0.25, need_dX=True)
    ref = O.loss_grads(x, G, U)
    assert dX.dtype == torch.bfloat16
    assert rel(to_np(dG), 0.25 * ref["dG"]) <= 1e-4
    for j in range(3):
        assert rel(to_np(dU[j]), 0.25 * ref["dU"][j]) <= 1e-4
    assert rel(to_np(dX), 0.25 * ref["dX"]) <= 4e-3
    st, _ = T.tk_sync_status(dev)
    assert st == 0
