"""GPU parity of rHKron-re with the Kronecker-SRHT sketch against the FP64 oracle.

Small tensors take the sign-flipped-copy path; FP32 tensors of at least 4M
elements with sketch widths <= 8 take the streaming kernel that applies the
Rademacher signs as it loads X.  The shapes make the first product of the
sketches contract the leading mode (rows along r) and strided modes on both
sides of the sketched mode, the three index maps of the signs.
"""
import numpy as np
import pytest

import oracle as O
from paper_2211_13028_gb300 import synth
from paper_2211_13028_gb300 import tucker as T
from tests.gpu_helpers import align, make_X, mats, rel, require_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return require_gpu()


def _check(G, U, err, ref, xv, tol):
    ref_err = O.rel_err(xv, ref["G"], ref["U"])
    assert abs(err - ref_err) <= tol, (err, ref_err)
    g, u = align(to_np(G), [to_np(x) for x in U], ref["U"])
    assert rel(g, ref["G"]) <= tol
    for j in range(len(u)):
        sv = np.linalg.svd(O.unfold(ref["G"], j), compute_uv=False)
        werr = np.linalg.norm((u[j] - ref["U"][j]) * sv[None, :]) / np.linalg.norm(sv)
        assert werr <= tol, (j, werr)
    assert rel(O.reconstruct(g, u), O.reconstruct(ref["G"], ref["U"])) <= tol


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
def test_srht_small(dev, dtype):
    dims, r, p = (64, 32, 64), (8, 6, 8), 4
    core = synth.decaying_core((16, 16, 16), 0.5, seed=31)
    x = synth.tucker_tensor(dims, (16, 16, 16), seed=32, noise_rel=1e-4, core=core)
    X, xv, sc = make_X(x, dtype, dev)
    s = O.subranks_reuse(r, p)[0]
    odt = "f64" if dtype == "f64" else "f32"
    H = synth.sketch_factors_srht(dims, s, seed=33, dtype=odt)
    G, U, err = T.tucker_rhkron_srht(X, r, p, mats(H, odt, dev), seed=12345, scale=sc)
    assert T.tk_sync_status(dev)[0] == 0
    ref = O.rhkron_srht(xv, r, H, 12345)
    _check(G, U, err, ref, xv, 1e-12 if dtype == "f64" else 1e-5)


@pytest.mark.parametrize("dims,s", [((256, 128, 128), (4, 6, 6)), ((128, 128, 256), (6, 4, 6))])
def test_srht_streaming_fp32(dev, dims, s):
    r, p = (8, 8, 8), 8
    core = synth.decaying_core((16, 16, 16), 0.5, seed=41)
    x = synth.tucker_tensor(dims, (16, 16, 16), seed=42, noise_rel=1e-4, core=core)
    X, xv, _ = make_X(x, "f32", dev)
    H = synth.sketch_factors_srht(dims, s, seed=43, dtype="f32")
    G, U, err = T.tucker_rhkron_srht(X, r, p, mats(H, "f32", dev), seed=2**40 + 99)
    assert T.tk_sync_status(dev)[0] == 0
    ref = O.rhkron_srht(xv, r, H, 2**40 + 99)
    _check(G, U, err, ref, xv, 1e-5)
