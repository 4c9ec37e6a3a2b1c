"""rHKron-re and the gradient of its reconstruction loss in one call (tucker_rhkron_grad).

The fused call reads the products R x_{j!=n} U_j^T of the gradient from the core's chain
X x_{m_1} Q^T x_{m_2} Q^T .. (U_j = Q_j V_j) instead of streaming X again, and takes the
relative error from the pass that forms dX.  Its decomposition must be the one tucker_rhkron
returns, its dX the one tucker_reconstruct_backward forms, and dG, dU the oracle's loss
gradient at the returned (G, U).  dG vanishes at an orthonormal Tucker projection and dU_n
is the difference of two nearly equal terms, so the gradients are compared on the scale of
those terms (||G||, ||X|| ||G||) rather than relative to their own size."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2211_13028_gb300 import synth
from paper_2211_13028_gb300 import tucker as T
from tests.gpu_helpers import make_X, mats, require_gpu, to_np

pytestmark = pytest.mark.gpu

# error of the gradient terms on their own scale: FP64 data; FP32 data (tensor-core passes,
# ~1e-6 relative per product); BF16 data (FP32 products of BF16 values)
TOL = {"f64": 1e-11, "f32": 3e-5, "bf16": 1e-4}


@pytest.fixture(scope="module")
def dev():
    return require_gpu()


def _case(dims, r, p, dtype, dev, seed, noise=1e-2, d_core=None):
    core = synth.decaying_core(d_core or tuple(min(n, 2 * k) for n, k in zip(dims, r)), 0.7, seed=seed)
    x = synth.tucker_tensor(dims, core.shape, seed=seed + 1, noise_rel=noise, core=core)
    X, xv, sc = make_X(x, dtype, dev)
    s = O.subranks_reuse(r, p)[0]
    fdt = "f64" if dtype == "f64" else "f32"
    om = mats(synth.sketch_factors_reuse(dims, s, seed=seed + 2, dtype=fdt), fdt, dev)
    return X, xv, om


def _check_grads(xv, G, U, dG, dU, dX, gs, tol, dx_tol=None):
    g, u = to_np(G), [to_np(a) for a in U]
    ref = O.loss_grads(xv, g, u)
    gn, xn = np.linalg.norm(g), np.linalg.norm(xv)
    assert np.linalg.norm(to_np(dG) - gs * ref["dG"]) <= tol * 2 * gs * gn
    for j in range(len(U)):
        assert np.linalg.norm(to_np(dU[j]) - gs * ref["dU"][j]) <= tol * 2 * gs * xn * gn, j
    if dx_tol is None:
        assert np.max(np.abs(to_np(dX) - gs * ref["dX"])) <= tol * 2 * gs * np.max(np.abs(xv))
    else:  # dX stored in X's BF16: one rounding of the residual
        assert np.max(np.abs(to_np(dX) - gs * ref["dX"])) <= dx_tol * gs * np.max(np.abs(ref["dX"]))


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_fused_call_matches_separate_calls_and_oracle(dev, dtype):
    dims, r, p = (96, 80, 72), (12, 10, 9), 5
    X, xv, om = _case(dims, r, p, dtype, dev, 70)
    gs = 0.5
    G, U, err, dG, dU, dX = T.tucker_rhkron_grad(X, r, p, om, gs)
    G1, U1, err1 = T.tucker_rhkron(X, r, p, om)
    assert torch.equal(G, G1) and all(torch.equal(a, b) for a, b in zip(U, U1))
    assert abs(err - err1) <= 1e-12 * err1
    assert abs(err - O.rel_err(xv, to_np(G), [to_np(u) for u in U])) <= (1e-12 if dtype == "f64" else 1e-6)
    dG2, dU2, dX2 = T.tucker_reconstruct_backward(X, G1, U1, gs)
    assert torch.equal(dX, dX2)  # the same residual pass
    tol = TOL[dtype]
    gn, xn = np.linalg.norm(to_np(G)), np.linalg.norm(xv)
    assert np.linalg.norm(to_np(dG) - to_np(dG2)) <= tol * 2 * gs * gn
    for a, b in zip(dU, dU2):
        assert np.linalg.norm(to_np(a) - to_np(b)) <= tol * 2 * gs * xn * gn
    _check_grads(xv, G, U, dG, dU, dX, gs, tol, dx_tol=4e-3 if dtype == "bf16" else None)
    assert T.tk_sync_status(dev)[0] == 0


def test_fused_call_mode_without_qr_and_partial_outputs(dev):
    # mode 3 (6 rows) is narrower than its sketch: Q_3 = I is never applied in the core's chain
    dims, r, p = (40, 36, 6), (5, 4, 3), 3
    for dtype in ("f64", "f32"):
        X, xv, om = _case(dims, r, p, dtype, dev, 80, d_core=(10, 8, 6))
        G, U, err, dG, dU, dX = T.tucker_rhkron_grad(X, r, p, om, 1.5)
        _check_grads(xv, G, U, dG, dU, dX, 1.5, TOL[dtype])
        # each output on its own gives the same values
        _, _, e_only, n1, n2, n3 = T.tucker_rhkron_grad(X, r, p, om, 1.5, need_dG=False, need_dU=False,
                                                        need_dX=False)
        assert n1 is None and n2 is None and n3 is None and abs(e_only - err) <= 1e-12 * err
        _, _, none, dG2, dU2, dX2 = T.tucker_rhkron_grad(X, r, p, om, 1.5, rel_err=False, need_dX=False)
        assert none is None and dX2 is None and torch.equal(dG, dG2)
        assert all(torch.equal(a, b) for a, b in zip(dU, dU2))
        _, _, _, dG3, dU3, dX3 = T.tucker_rhkron_grad(X, r, p, om, 1.5, need_dG=False, need_dU=False)
        assert dG3 is None and dU3 is None and torch.equal(dX, dX3)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_fused_call_four_way(dev, dtype):
    dims, r, p = (24, 20, 18, 16), (4, 3, 4, 3), 3
    X, xv, om = _case(dims, r, p, dtype, dev, 90, d_core=(8, 6, 8, 6))
    G, U, err, dG, dU, dX = T.tucker_rhkron_grad(X, r, p, om, 1.0)
    _check_grads(xv, G, U, dG, dU, dX, 1.0, TOL[dtype])
    G1, U1, err1 = T.tucker_rhkron(X, r, p, om)
    assert torch.equal(G, G1) and abs(err - err1) <= 1e-12 * err1


def test_fused_call_rejects_bad_outputs(dev):
    dims, r, p = (40, 36, 32), (5, 4, 3), 3
    X, xv, om = _case(dims, r, p, "f64", dev, 95)
    with pytest.raises(T.TuckerError):  # p too large for the sketch widths
        T.tucker_rhkron_grad(X, r, 400, om)
    lib = T.load()
    G = T.empty_f(list(r), torch.float64, dev)
    U = [T._colmajor_matrix(n, k, torch.float64, dev) for n, k in zip(dims, r)]
    dG_bad = T.empty_f([r[0] + 1, r[1], r[2]], torch.float64, dev)
    rr = (T.ctypes.c_int64 * 3)(*r)
    o, keep = T._opts(None, 0, 0, 0, False)
    h = T._handle(dev)
    st = lib.tucker_rhkron_grad(h, T.ctypes.byref(T._tensor(X)), rr, p, T._mats(om), T.ctypes.byref(o),
                                T.ctypes.byref(T._tensor(G)), T._mats(U), None, 1.0,
                                T.ctypes.byref(T._tensor(dG_bad)), None, None)
    with pytest.raises(T.TuckerError) as e:
        T._check(st, h)
    assert e.value.status == 2  # TK_ERR_SHAPE: dG must have G's dims
