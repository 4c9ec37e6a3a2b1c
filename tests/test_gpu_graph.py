"""Decompositions recorded into CUDA graphs and replayed.

A recorded call must give at every replay exactly what the same call gives
eagerly (every kernel is deterministic for a given shape), including its
stream-ordered host output; recording needs a sized workspace and async host
outputs; a workspace block a graph recorded survives a later growth.
"""
import numpy as np
import pytest
import torch

from paper_2211_13028_gb300 import synth
from paper_2211_13028_gb300 import tucker as T
from tests.gpu_helpers import make_X, mats, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return require_gpu()


def _problem(dev, dims=(96, 80, 72), seed=41):
    import oracle as O
    r, p = (12, 10, 9), 5
    core = synth.decaying_core((20, 20, 20), 0.7, seed=seed)
    x = synth.tucker_tensor(dims, (20, 20, 20), seed=seed + 1, noise_rel=1e-3, core=core)
    X, _, _ = make_X(x, "f32", dev)
    s, _ = O.subranks_reuse(r, p)
    om = mats(synth.sketch_factors_reuse(dims, s, seed=seed + 2, dtype="f32"), "f32", dev)
    S, w = O.subranks_matrix(r, p)
    k = [min(n, ww) for n, ww in zip(dims, w)]
    oms = {key: synth.fmat(v, "f32", dev)
           for key, v in synth.sketch_factors_matrix(dims, S, k, [0, 1, 2], seed + 3, "f32").items()}
    return X, r, p, om, oms


def _same(a, b):
    Ga, Ua, ea = a
    Gb, Ub, eb = b
    assert torch.equal(Ga, Gb)
    assert all(torch.equal(u, v) for u, v in zip(Ua, Ub))
    assert ea == eb


def test_recorded_rhkron_replays_bitwise(dev):
    X, r, p, om, _ = _problem(dev)
    ref = T.tucker_rhkron(X, r, p, om)
    g = T.TuckerGraph(lambda: T.tucker_rhkron(X, r, p, om, async_outputs=True))
    for _ in range(3):
        g.outputs[0].zero_()
        for u in g.outputs[1]:
            u.zero_()
        g.replay()
        torch.cuda.synchronize()
        G, U, e = g.outputs
        _same((G, U, e.value), ref)
    assert T.tk_sync_status(dev)[0] == 0


def test_recorded_two_stream_step(dev):
    # rHKron-re and its gradient on one stream, rSTHKron on another, forked from the recording stream
    X, r, p, om, oms = _problem(dev)
    sa, sb = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def step():
        main = torch.cuda.current_stream(dev)
        sa.wait_stream(main)
        sb.wait_stream(main)
        with torch.cuda.stream(sa):
            a = T.tucker_rhkron(X, r, p, om, async_outputs=True)
            dG, dU, _ = T.tucker_reconstruct_backward(X, a[0], a[1], 0.5, need_dX=False)
        with torch.cuda.stream(sb):
            b = T.tucker_rsthkron(X, r, p, oms, async_outputs=True)
        main.wait_stream(sa)
        main.wait_stream(sb)
        return a, b, dG, dU

    a_ref, b_ref, dG_ref, dU_ref = step()
    torch.cuda.synchronize()
    a_ref = (a_ref[0], a_ref[1], a_ref[2].value)
    b_ref = (b_ref[0], b_ref[1], b_ref[2].value)
    g = T.TuckerGraph(step)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        a, b, dG, dU = g.outputs
        _same((a[0], a[1], a[2].value), a_ref)
        _same((b[0], b[1], b[2].value), b_ref)
        assert torch.equal(dG, dG_ref) and all(torch.equal(u, v) for u, v in zip(dU, dU_ref))


def test_recording_needs_sized_workspace_and_async_outputs(dev):
    X, r, p, om, _ = _problem(dev, dims=(64, 56, 48), seed=51)
    s = torch.cuda.Stream(dev)
    with torch.cuda.stream(s):
        T.tk_sync_status(dev)  # creates this stream's handle (outside the recording), no workspace yet
    g = torch.cuda.CUDAGraph()
    with pytest.raises(T.TuckerError) as ei:
        with torch.cuda.graph(g, stream=s):
            T.tucker_rhkron(X, r, p, om, async_outputs=True)
    assert ei.value.status == 5  # TK_ERR_WORKSPACE
    with torch.cuda.stream(s):
        T.tucker_rhkron(X, r, p, om)  # sizes the workspace
    torch.cuda.synchronize()
    g2 = torch.cuda.CUDAGraph()
    with pytest.raises(T.TuckerError) as ei:
        with torch.cuda.graph(g2, stream=s):
            T.tucker_rhkron(X, r, p, om)  # a synchronous host output cannot be recorded
    assert ei.value.status == 1  # TK_ERR_ARG


def test_recorded_workspace_survives_growth(dev):
    X, r, p, om, _ = _problem(dev, dims=(64, 56, 48), seed=61)
    ref = T.tucker_rhkron(X, r, p, om)
    g = T.TuckerGraph(lambda: T.tucker_rhkron(X, r, p, om, async_outputs=True))
    # a larger call on the same stream grows that handle's workspace
    Xb, rb, pb, omb, _ = _problem(dev, dims=(160, 150, 140), seed=71)
    with torch.cuda.stream(g.stream):
        T.tucker_rhkron(Xb, rb, pb, omb)
    g.outputs[0].zero_()
    g.replay()
    torch.cuda.synchronize()
    _same((g.outputs[0], g.outputs[1], g.outputs[2].value), ref)
    del g
    torch.cuda.synchronize()
    T.tk_graph_release(dev)
