"""Parity at the benchmark's full size: the 512^3 FP32 Gaussian-bump field, rHKron-re and rSTHKron
at r = (32, 32, 32), p = 8, with the Gaussian sketch factors drawn on the device (Philox4x32-10), the
way bench.py runs a step, against the FP64 oracle run on the same field with its own statement of
the same generator (about ten seconds of host time per algorithm)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2211_13028_gb300 import synth
from paper_2211_13028_gb300 import tucker as T
from tests.gpu_helpers import align, rel, require_gpu, to_np

pytestmark = pytest.mark.gpu

N, R, P, SEED = 512, (32, 32, 32), 8, 0


@pytest.fixture(scope="module")
def dev():
    return require_gpu()


@pytest.fixture(scope="module")
def field(dev):
    X = synth.gaussian_bumps(N, 3, 200, SEED, 1e-4, dev, "f32")
    return X, synth.from_fortran(X)


def _check(G, U, err, ref, xv, tol):
    ref_err = O.rel_err(xv, ref["G"], ref["U"])
    assert abs(err - ref_err) <= tol, (err, ref_err)
    g, u = align(to_np(G), [to_np(x) for x in U], ref["U"])
    assert rel(g, ref["G"]) <= tol
    for j in range(len(u)):
        sv = np.linalg.svd(O.unfold(ref["G"], j), compute_uv=False)
        werr = np.linalg.norm((u[j] - ref["U"][j]) * sv[None, :]) / np.linalg.norm(sv)
        assert werr <= tol, (j, werr)


def _same_draws(dev_factor, ref):
    # the device's FP64 Box-Muller and the oracle's differ by a few FP64 ulps, so the FP32 values agree
    # to the last bit except where a value straddles a rounding boundary: at most one FP32 ulp apart
    a = to_np(dev_factor)
    assert np.mean(a == ref) > 0.999
    assert np.all(np.abs(a - ref) <= 2.0 ** -23 * np.maximum(np.abs(ref), 2.0 ** -126))


def test_rhkron_full_size_device_factors(dev, field):
    X, xv = field
    s = O.subranks_reuse(R, P)[0]
    om_dev = T.gaussian_factors(X.shape, s, SEED + 1, torch.float32, dev)
    om_ref = [synth.round_to(O.gaussian_factor(N, s[j], SEED + 1, j), "f32") for j in range(3)]
    for a, b in zip(om_dev, om_ref):
        _same_draws(a, b)
    G, U, err = T.tucker_rhkron(X, R, P, om_dev)
    ref = O.rhkron(xv, R, om_ref)
    _check(G, U, err, ref, xv, 1e-5)
    assert T.tk_sync_status(dev)[0] == 0


def test_rsthkron_full_size_device_factors(dev, field):
    X, xv = field
    S, w = O.subranks_matrix(R, P)
    k = [min(N, ww) for ww in w]
    oms_dev = T.gaussian_factors_matrix(X.shape, S, k, [0, 1, 2], SEED + 2, torch.float32, dev)
    oms_ref, done = {}, set()
    for j in range(3):
        for kk in range(3):
            if kk != j:
                cur = k[kk] if kk in done else N
                oms_ref[(j, kk)] = synth.round_to(O.gaussian_factor(cur, int(S[j][kk]), SEED + 2, 8 * j + kk), "f32")
        done.add(j)
    for key, a in oms_dev.items():
        _same_draws(a, oms_ref[key])
    G, U, err = T.tucker_rsthkron(X, R, P, oms_dev)
    ref = O.rsthkron(xv, R, oms_ref)
    _check(G, U, err, ref, xv, 1e-5)
    assert T.tk_sync_status(dev)[0] == 0
