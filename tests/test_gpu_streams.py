"""Concurrent decompositions on two streams with stream-ordered host outputs.

rHKron-re on one stream and rSTHKron on another, both reading the same X, must
give exactly what the same calls give one after the other on one stream (each
stream has its own handle and workspace, and every kernel is deterministic for
a given shape).  More pending outputs than the handle's callback slots must
still all be delivered.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2211_13028_gb300 import synth
from paper_2211_13028_gb300 import tucker as T
from tests.gpu_helpers import make_X, mats, require_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return require_gpu()


def _setup(dev):
    dims, r, p = (96, 80, 72), (12, 10, 9), 5
    core = synth.decaying_core((20, 20, 20), 0.7, seed=41)
    x = synth.tucker_tensor(dims, (20, 20, 20), seed=42, noise_rel=1e-3, core=core)
    X, xv, _ = make_X(x, "f32", dev)
    s, _ = O.subranks_reuse(r, p)
    om = mats(synth.sketch_factors_reuse(dims, s, seed=43, dtype="f32"), "f32", dev)
    S, w = O.subranks_matrix(r, p)
    k = [min(n, ww) for n, ww in zip(dims, w)]
    oms = {key: synth.fmat(v, "f32", dev)
           for key, v in synth.sketch_factors_matrix(dims, S, k, [0, 1, 2], 44, "f32").items()}
    return X, r, p, om, oms


def test_two_streams_match_one_stream(dev):
    X, r, p, om, oms = _setup(dev)
    G1, U1, e1 = T.tucker_rhkron(X, r, p, om)
    G2, U2, e2 = T.tucker_rsthkron(X, r, p, oms)
    torch.cuda.synchronize()
    sa, sb = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    sa.wait_stream(torch.cuda.current_stream(dev))
    sb.wait_stream(torch.cuda.current_stream(dev))
    res = []
    for _ in range(3):
        with torch.cuda.stream(sa):
            a = T.tucker_rhkron(X, r, p, om, async_outputs=True)
        with torch.cuda.stream(sb):
            b = T.tucker_rsthkron(X, r, p, oms, async_outputs=True)
        res.append((a, b))
    torch.cuda.synchronize()
    for (Ga, Ua, ea), (Gb, Ub, eb) in res:
        assert torch.equal(Ga, G1) and torch.equal(Gb, G2)
        assert all(torch.equal(u, v) for u, v in zip(Ua, U1))
        assert all(torch.equal(u, v) for u, v in zip(Ub, U2))
        assert ea.value == e1 and eb.value == e2
    assert T.tk_sync_status(dev)[0] == 0


def test_more_pending_outputs_than_slots(dev):
    X, r, p, om, _ = _setup(dev)
    _, _, e_ref = T.tucker_rhkron(X, r, p, om)
    s = torch.cuda.Stream(dev)
    s.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(s):
        outs = [T.tucker_rhkron(X, r, p, om, async_outputs=True)[2] for _ in range(70)]
    s.synchronize()
    vals = np.array([o.value for o in outs])
    assert np.all(vals == e_ref)


def test_backward_outputs_can_be_requested_separately(dev):
    # dX alone (one fused residual pass) and (dG, dU) alone give what one call gives
    g = np.random.Generator(np.random.PCG64(61))
    dims, rk = (96, 80, 72), (12, 10, 36)
    x = synth.round_to(g.standard_normal(dims), "f32")
    G = synth.round_to(g.standard_normal(rk), "f32")
    U = [synth.round_to(g.standard_normal((nn, k)) / np.sqrt(nn), "f32") for nn, k in zip(dims, rk)]
    Xd, Gd, Ud = synth.fortran(x, "f32", dev), synth.fortran(G, "f32", dev), mats(U, "f32", dev)
    dG, dU, dX = T.tucker_reconstruct_backward(Xd, Gd, Ud, 0.5)
    _, _, dX2 = T.tucker_reconstruct_backward(Xd, Gd, Ud, 0.5, need_dG=False, need_dU=False)
    dG2, dU2, none = T.tucker_reconstruct_backward(Xd, Gd, Ud, 0.5, need_dX=False)
    dG3, none2, none3 = T.tucker_reconstruct_backward(Xd, Gd, Ud, 0.5, need_dX=False, need_dU=False)
    assert none is None and none2 is None and none3 is None
    assert torch.equal(dX, dX2) and torch.equal(dG, dG2) and torch.equal(dG, dG3)
    assert all(torch.equal(a, b) for a, b in zip(dU, dU2))
    with pytest.raises(T.TuckerError):
        T.tucker_reconstruct_backward(Xd, Gd, Ud, 0.5, need_dX=False, need_dG=False, need_dU=False)


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_backward_norms_give_the_decompositions_relative_error(dev, dtype):
    # the residual pass that forms dX also returns ||X - Xhat||^2 and ||X||^2: with the G, U that rHKron-re
    # returns, their ratio is the relative error the decomposition reports for itself (same residual pass),
    # and the oracle's for the same G, U
    dims, r, p = (96, 80, 72), (12, 10, 9), 5
    core = synth.decaying_core((20, 20, 20), 0.7, seed=43)
    x = synth.tucker_tensor(dims, (20, 20, 20), seed=44, noise_rel=1e-3, core=core)
    X, xv, _ = make_X(x, dtype, dev)
    s = O.subranks_reuse(r, p)[0]
    om = mats(synth.sketch_factors_reuse(dims, s, seed=45, dtype=dtype), dtype, dev)
    G, U, err = T.tucker_rhkron(X, r, p, om)
    G2, U2, none = T.tucker_rhkron(X, r, p, om, rel_err=False)
    assert none is None and torch.equal(G, G2) and all(torch.equal(a, b) for a, b in zip(U, U2))
    ref = O.rel_err(xv, to_np(G), [to_np(u) for u in U])
    tol = 1e-12 if dtype == "f64" else 1e-6
    outs = {}
    for need_dx, need_dgu in ((True, False), (False, False), (True, True), (False, True)):
        n2 = torch.full((2,), float("nan"), dtype=torch.float64, device=dev)
        dG, dU, dX = T.tucker_reconstruct_backward(X, G, U, 0.5, need_dX=need_dx, need_dG=need_dgu,
                                                   need_dU=need_dgu, norms2=n2)
        a, b = n2.cpu().tolist()
        # FP32 data: the fused pass sums short runs of squares in FP32 before adding them in FP64
        assert abs(b - np.sum(xv ** 2)) <= tol * np.sum(xv ** 2)
        e = np.sqrt(a / b)
        assert abs(e - ref) <= tol * max(ref, 1.0), (need_dx, need_dgu, e, ref)
        outs[(need_dx, need_dgu)] = e
        if need_dx:
            r_ref = O.reconstruct(to_np(G), [to_np(u) for u in U]) - xv
            assert np.max(np.abs(to_np(dX) + r_ref)) <= tol * np.max(np.abs(xv)) * 10
    # one residual pass whichever other outputs are requested (the sums' order may differ between the
    # fused kernel's norm-only and dX-writing forms)
    vals = list(outs.values()) + [err]
    assert max(vals) - min(vals) <= 1e-12 * max(vals)
    with pytest.raises(T.TuckerError):  # wrong dtype
        T.tucker_reconstruct_backward(X, G, U, 0.5, norms2=torch.zeros(2, dtype=torch.float32, device=dev))


def test_sm_reserve_leaves_results_unchanged(dev):
    # the streaming kernels on fewer CTAs (SMs left to other streams): the same products element by
    # element; only the order of the residual's per-CTA partial sums changes
    dims, r, p = (128, 96, 160), (12, 10, 9), 5
    core = synth.decaying_core((20, 20, 20), 0.7, seed=47)
    x = synth.tucker_tensor(dims, (20, 20, 20), seed=48, noise_rel=1e-3, core=core)
    X, xv, _ = make_X(x, "f32", dev)
    s = O.subranks_reuse(r, p)[0]
    om = mats(synth.sketch_factors_reuse(dims, s, seed=49, dtype="f32"), "f32", dev)
    G0, U0, e0 = T.tucker_rhkron(X, r, p, om)
    try:
        for sms in (1, 24, 100):
            T.tk_set_sm_reserve(sms, dev)
            G1, U1, e1 = T.tucker_rhkron(X, r, p, om)
            assert torch.equal(G0, G1) and all(torch.equal(a, b) for a, b in zip(U0, U1)), sms
            assert abs(e1 - e0) <= 1e-12 * e0, sms
        with pytest.raises(T.TuckerError):
            T.tk_set_sm_reserve(-1, dev)
        with pytest.raises(T.TuckerError):
            T.tk_set_sm_reserve(100000, dev)
    finally:
        T.tk_set_sm_reserve(0, dev)
    assert T.tk_sync_status(dev)[0] == 0


def test_profile_trace_lists_every_recorded_launch(dev):
    # the per-launch records of two concurrent calls: one per launch the class totals count, each with
    # its stream, ordered intervals after the common origin
    X, r, p, om, oms = _setup(dev)
    sa, sb = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    for _ in range(2):  # the second round is recorded
        torch.cuda.synchronize()
        with torch.cuda.stream(sa):
            T.tk_profile(True, dev)
        with torch.cuda.stream(sb):
            T.tk_profile(True, dev)
        sa.wait_stream(torch.cuda.current_stream(dev))
        sb.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(sa):
            T.tucker_rhkron(X, r, p, om, async_outputs=True)
        with torch.cuda.stream(sb):
            T.tucker_rsthkron(X, r, p, oms, async_outputs=True)
        torch.cuda.synchronize()
    n = [T.load().tk_profile_trace(h, None, 0) for h in T._device_handles(dev)]  # counts, records kept
    assert min(n) >= 0
    tr = T.tk_profile_trace(dev)
    assert len(tr) == sum(n) > 20
    assert T.tk_profile_trace(dev) == []  # consumed
    assert [e["start_us"] for e in tr] == sorted(e["start_us"] for e in tr)
    assert all(0.0 <= e["start_us"] <= e["end_us"] for e in tr)
    assert all(-1 <= e["stream"] <= 4 for e in tr) and any(e["stream"] > 0 for e in tr)  # forked chains
    cls = {e["cls"] for e in tr}
    assert "jacobi" in cls and any(c.startswith("xpass") for c in cls)
    for h in T._device_handles(dev):
        T.load().tk_profile(h, 0)
