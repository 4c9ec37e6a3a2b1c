"""The allocation-free thin QR entry point, checked through the C ABI against
tucker_orth on two calls in a row.  Some callers cannot allocate device
memory where they need the factorisation (memory owned by a pool or arena;
paths that must not take the implicit synchronisation of cudaMalloc), so
tucker_orth_noalloc works in a fixed scratch array inside the library.  The
file is collected last because that array is shared by every call and keeps
the previous call's contents."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2211_13028_gb300 import synth
from paper_2211_13028_gb300 import tucker as T
from tests.gpu_helpers import require_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return require_gpu()


def _inputs(seed):
    g = np.random.Generator(np.random.PCG64(seed))
    full = g.standard_normal((512, 49))
    deficient = g.standard_normal((300, 5)) @ g.standard_normal((5, 20))  # rank 5: Householder path
    limit = g.standard_normal((4096, 64))  # the largest accepted size
    return full, deficient, limit


def _check_same(y, Q, info, Q_ref, info_ref):
    assert info == info_ref
    if info == 0:  # CholeskyQR2: unique thin QR factor
        assert np.max(np.abs(to_np(Q) - to_np(Q_ref))) <= 1e-12
    else:  # rank-deficient: compare orthonormality and the projector onto range(Y)
        q, qr = to_np(Q), to_np(Q_ref)
        assert np.max(np.abs(q.T @ q - np.eye(q.shape[1]))) <= 1e-12
        assert np.max(np.abs(q @ (q.T @ y) - qr @ (qr.T @ y))) <= 1e-10 * np.abs(y).max()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_matches_tucker_orth_twice(dev, dtype):
    for y64 in _inputs(11):
        y = synth.round_to(y64, dtype)
        Y = synth.fmat(y, dtype, dev)
        Q_ref, info_ref = T.tucker_orth(Y, out_dtype=torch.float64)
        for _ in range(2):  # the scratch keeps the previous call's contents
            Q, info = T.tucker_orth_noalloc(Y, out_dtype=torch.float64)
            _check_same(y, Q, info, Q_ref, info_ref)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_at_its_size_limit_matches_oracle(dev, dtype):
    y = synth.round_to(_inputs(12)[2], dtype)
    Y = synth.fmat(y, dtype, dev)
    Q, info = T.tucker_orth_noalloc(Y, out_dtype=torch.float64)
    assert info == 0
    assert np.max(np.abs(to_np(Q) - O.thin_qr(y))) <= 1e-12


def test_noalloc_rejects_oversized(dev):
    Y = synth.fmat(np.zeros((5000, 8)), "f64", dev)
    with pytest.raises(T.TuckerError) as e:
        T.tucker_orth_noalloc(Y)
    assert e.value.status == 2
    Y = synth.fmat(np.zeros((200, 65)), "f64", dev)
    with pytest.raises(T.TuckerError) as e:
        T.tucker_orth_noalloc(Y)
    assert e.value.status == 2


def test_noalloc_without_reading_info(dev):
    # info = NULL: the call only queues work; Q equals the synchronising call's
    y = synth.round_to(_inputs(13)[0], "f64")
    Y = synth.fmat(y, "f64", dev)
    Q_ref, _ = T.tucker_orth_noalloc(Y, out_dtype=torch.float64)
    Q, info = T.tucker_orth_noalloc(Y, out_dtype=torch.float64, read_info=False)
    torch.cuda.synchronize()
    assert info is None and torch.equal(Q, Q_ref)
