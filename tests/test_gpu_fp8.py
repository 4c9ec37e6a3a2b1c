"""The FP8 (E4M3) tensor-core TTM: contractions over the contiguous mode of FP8 data run on
tcgen05 kind::f8f6f4 with the factor carried as five power-of-two-scaled E4M3 pieces.  The
product is checked against the FP64 oracle on the FP8-rounded values (the tolerance the other
storage forms meet, 1e-5 relative), with ragged K chunks, ragged row tiles and factors wider than
one block; the profiler confirms that the tensor-core kernel ran."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("dims,m", [((256, 40, 36), 3), ((272, 33, 17), 20), ((384, 24, 30), 48),
                                    ((160, 50, 9), 70), ((512, 21, 13), 130)])
def test_fp8_mode1_ttm_against_oracle(dev, dims, m):
    g = _rng(31)
    X, xv, sc = make_X(g.standard_normal(dims), "fp8", dev)
    q0 = np.linalg.qr(g.standard_normal((dims[0], max(m, 1))))[0][:, :m] if m <= dims[0] else None
    qs = [q0, np.eye(dims[1]), np.eye(dims[2])]  # identities: the product is X x_1 Q_0^T alone
    T.tk_profile(True, dev)
    G = T.tucker_core(X, mats(qs, "f32", dev), scale=sc)
    prof = T.tk_profile_read(dev)
    T.tk_profile(False, dev)
    ref = O.ttm(xv, q0.T, 0)
    assert rel(to_np(G), ref) <= 1e-5
    assert np.max(np.abs(to_np(G) - ref)) <= 1e-5 * np.max(np.abs(ref))
    assert "xpass_tc" in prof and "xpass_simt" not in prof  # X was streamed by the tensor-core kernel


def test_fp8_gaussian_factor_narrow(dev):
    # a sketch-width factor of N(0, 1) draws (entries well above 1): the pieces' scale adapts
    g = _rng(32)
    dims = (128, 64, 40)
    X, xv, sc = make_X(g.standard_normal(dims) * 1e3, "fp8", dev)
    om = g.standard_normal((dims[0], 7))
    G = T.tucker_core(X, mats([om, np.eye(dims[1]), np.eye(dims[2])], "f32", dev), scale=sc)
    ref = O.ttm(xv, om.T, 0)
    assert rel(to_np(G), ref) <= 1e-5


def test_fp8_rhkron_uses_tensor_cores_and_matches_oracle(dev):
    dims, r, p = (128, 96, 80), (6, 5, 4), 4
    core = synth.decaying_core((12, 12, 12), 0.5, seed=33)
    x = synth.tucker_tensor(dims, (12, 12, 12), seed=34, noise_rel=1e-4, core=core)
    X, xv, sc = make_X(x, "fp8", dev)
    s = O.subranks_reuse(r, p)[0]
    oms = synth.sketch_factors_reuse(dims, s, seed=35, dtype="f32")
    T.tk_profile(True, dev)
    G, U, err = T.tucker_rhkron(X, r, p, mats(oms, "f32", dev), scale=sc)
    prof = T.tk_profile_read(dev)
    T.tk_profile(False, dev)
    assert T.tk_sync_status(dev)[0] == 0
    ref = O.rhkron(xv, r, oms)
    assert abs(err - O.rel_err(xv, ref["G"], ref["U"])) <= 1e-5
    assert prof["xpass_tc"]["launches"] >= 2  # the core pass and the mode-1 sketch pass
