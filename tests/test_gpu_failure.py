"""Failure detection on the GPU without a GPU fault: a bounded device wait that
runs out.  The self-test entry point makes one warp wait, through the same
bounded mbarrier wait the tcgen05 / TMA kernels use, on an mbarrier that
nothing arrives at; the wait gives up after the limit given from the host,
the handle reports TK_ERR_TIMEOUT at the next status check (once), and the
context stays usable: a decomposition afterwards still matches the oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2211_13028_gb300 import synth
from paper_2211_13028_gb300 import tucker as T
from tests.gpu_helpers import require_gpu

pytestmark = pytest.mark.gpu

TK_ERR_ARG, TK_ERR_TIMEOUT = 1, 8


@pytest.fixture(scope="module")
def dev():
    return require_gpu()


def test_bounded_wait_runs_out_and_reports_timeout(dev):
    assert T.tk_sync_status(dev)[0] == 0
    limit = 20_000_000  # 20 ms
    waited = T.tk_selftest_bounded_wait(limit, dev)
    assert limit <= waited < 1_000_000_000, waited
    assert T.tk_sync_status(dev)[0] == TK_ERR_TIMEOUT
    assert T.tk_sync_status(dev)[0] == 0  # reported once, then cleared


def test_context_usable_after_timeout(dev):
    T.tk_selftest_bounded_wait(5_000_000, dev)
    assert T.tk_sync_status(dev)[0] == TK_ERR_TIMEOUT
    dims, r, p = (40, 36, 32), (6, 5, 4), 4
    x = synth.tucker_tensor(dims, r, seed=3, noise_rel=1e-3)
    s, _ = T.tucker_subranks_reuse(r, p)
    om = synth.sketch_factors_reuse(dims, s, seed=4)
    _, _, err = T.tucker_rhkron(synth.fortran(x, "f64", dev), r, p, [synth.fmat(o, "f64", dev) for o in om])
    ref = O.rhkron(x, r, om)
    assert abs(err - O.rel_err(x, ref["G"], ref["U"])) <= 1e-12
    assert T.tk_sync_status(dev)[0] == 0


def test_limit_out_of_range_is_rejected(dev):
    for bad in (0, 999, 3_000_000_000):
        with pytest.raises(T.TuckerError) as e:
            T.tk_selftest_bounded_wait(bad, dev)
        assert e.value.status == TK_ERR_ARG
    assert np.isfinite(T.tk_sync_status(dev)[0])
