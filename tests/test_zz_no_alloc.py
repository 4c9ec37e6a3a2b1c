"""The allocation-free thin QR entry point, checked through the C ABI against
tucker_orth on two calls in a row.  Kept in a file of its own that is
collected last, because the entry point's scratch is a fixed device array
shared by every call."""
import numpy as np
import pytest
import torch

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
    return full, deficient


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_matches_tucker_orth_twice(dev, dtype):
    full, deficient = _inputs(11)
    for y64 in (full, deficient):
        y = synth.round_to(y64, dtype)
        Y = synth.fmat(y, dtype, dev)
        Q_ref, info_ref = T.tucker_orth(Y, out_dtype=torch.float64)
        for _ in range(2):  # the scratch keeps the previous call's contents
            Q, info = T.tucker_orth_noalloc(Y, out_dtype=torch.float64)
            assert info == info_ref
            if info == 0:  # CholeskyQR2: unique thin QR factor
                assert np.max(np.abs(to_np(Q) - to_np(Q_ref))) <= 1e-12
            else:  # rank-deficient: compare orthonormality and the projector onto range(Y)
                q, qr = to_np(Q), to_np(Q_ref)
                assert np.max(np.abs(q.T @ q - np.eye(q.shape[1]))) <= 1e-12
                assert np.max(np.abs(q @ (q.T @ y) - qr @ (qr.T @ y))) <= 1e-10 * np.abs(y).max()


def test_noalloc_rejects_oversized(dev):
    Y = synth.fmat(np.zeros((5000, 8)), "f64", dev)
    with pytest.raises(T.TuckerError) as e:
        T.tucker_orth_noalloc(Y)
    assert e.value.status == 2
    Y = synth.fmat(np.zeros((200, 65)), "f64", dev)
    with pytest.raises(T.TuckerError) as e:
        T.tucker_orth_noalloc(Y)
    assert e.value.status == 2
