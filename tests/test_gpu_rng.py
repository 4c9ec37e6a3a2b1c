"""GPU parity of the device generator of Gaussian sketch factors against the oracle's statement
of the same published generator (Philox4x32-10 and Box-Muller), and rHKron-re run with factors
drawn on the device against the FP64 oracle run with the oracle's own draws."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2211_13028_gb300 import synth
from paper_2211_13028_gb300 import tucker as T
from tests.gpu_helpers import align, make_X, rel, require_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    return require_gpu()


@pytest.mark.parametrize("seed,stream,offset,nblocks", [
    (0, 0, 0, 1), (12345, 3, 0, 1000), (0xFEDCBA9876543210, 7, (1 << 32) - 300, 700), (1, 0, 0, 0)])
def test_philox_blocks_bit_exact(dev, seed, stream, offset, nblocks):
    got = T.tk_philox4x32(seed, stream, offset, nblocks, dev).cpu().numpy().view(np.uint32).astype(np.uint64)
    ref = O.philox_blocks(seed, stream, offset, nblocks)
    assert got.shape == ref.shape and np.array_equal(got, ref)


@pytest.mark.parametrize("rows,cols", [(512, 7), (97, 13), (3, 1), (0, 5), (1, 1)])
def test_gaussian_factor_f64(dev, rows, cols):
    got = to_np(T.tucker_gaussian_factor(rows, cols, 99, 2, torch.float64, dev))
    ref = O.gaussian_factor(rows, cols, 99, 2)
    assert got.shape == ref.shape
    # FP64 log / sincospi on the device against NumPy's log / sin / cos: a few ulps
    assert np.max(np.abs(got - ref), initial=0.0) <= 1e-14 * max(1.0, np.max(np.abs(ref), initial=0.0))


@pytest.mark.parametrize("dtype,ulp", [(torch.float32, 2.0 ** -23), (torch.bfloat16, 2.0 ** -7)])
def test_gaussian_factor_rounded(dev, dtype, ulp):
    rows, cols = 333, 9
    got = to_np(T.tucker_gaussian_factor(rows, cols, 5, 1, dtype, dev))
    ref = O.gaussian_factor(rows, cols, 5, 1)
    # rounded once from FP64: within one unit in the last place (either side of a tie)
    assert np.all(np.abs(got - ref) <= ulp * np.maximum(np.abs(ref), 2.0 ** -126))
    exact = synth.round_to(ref, "f32" if dtype == torch.float32 else "bf16")
    assert np.mean(got == exact) > 0.999


def test_gaussian_factor_strided(dev):
    # a factor written into a column-major matrix with ld > rows leaves the rows past `rows` untouched
    buf = torch.full((5, 12), 7.0, dtype=torch.float64, device=dev)  # 5 columns of ld 12
    m = buf.t()[:10]  # 10 x 5, strides (1, 12)
    h = T._handle(m.device)
    T._check(T.load().tucker_gaussian_factor(h, 3, 4, T.ctypes.byref(T._matrix(m))), h)
    full = buf.t().cpu().numpy()
    assert np.array_equal(full[10:], np.full((2, 5), 7.0))
    assert np.max(np.abs(full[:10] - O.gaussian_factor(10, 5, 3, 4))) <= 1e-13


def test_rhkron_with_device_factors(dev):
    # the factors drawn on the device by the binding (mode j from stream j) equal the oracle's own
    # draws (up to a rounding tie), so the decomposition matches the oracle's rHKron-re on its draws
    dims, r, p = (96, 80, 72), (10, 12, 8), 6
    core = synth.decaying_core((16, 16, 16), 0.5, seed=41)
    x = synth.tucker_tensor(dims, (16, 16, 16), seed=42, noise_rel=1e-4, core=core)
    X, xv, sc = make_X(x, "f32", dev)
    s = O.subranks_reuse(r, p)[0]
    om_dev = T.gaussian_factors(dims, s, 2024, torch.float32, dev)
    om_ref = [synth.round_to(O.gaussian_factor(n, k, 2024, j), "f32") for j, (n, k) in enumerate(zip(dims, s))]
    for a, b in zip(om_dev, om_ref):
        assert np.mean(to_np(a) == b) > 0.999
    G, U, err = T.tucker_rhkron(X, r, p, om_dev)
    ref = O.rhkron(xv, r, om_ref)
    tol = 1e-5
    assert abs(err - O.rel_err(xv, ref["G"], ref["U"])) <= tol
    g, u = align(to_np(G), [to_np(v) for v in U], ref["U"])
    assert rel(g, ref["G"]) <= tol
    assert rel(O.reconstruct(g, u), O.reconstruct(ref["G"], ref["U"])) <= tol


def test_gaussian_factors_batched_equals_single(dev):
    # one launch for several factors writes what one call per factor writes
    shapes, streams = [(64, 5), (33, 7), (0, 3), (9, 1)], [0, 9, 2, 17]
    many = T.tucker_gaussian_factors(shapes, 77, streams, torch.float64, dev)
    for (r, c), s, m in zip(shapes, streams, many):
        one = T.tucker_gaussian_factor(r, c, 77, s, torch.float64, dev)
        assert torch.equal(m, one)
        assert np.max(np.abs(to_np(m) - O.gaussian_factor(r, c, 77, s)), initial=0.0) <= 1e-13
