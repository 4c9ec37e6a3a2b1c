"""Oracle pins for the Gaussian sketch-factor generator (Philox4x32-10 and Box-Muller)."""
import json
import os

import numpy as np
import pytest

import oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))


def _kat():
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.json")) as f:
        return json.load(f)["vectors"]


def test_philox_known_answers():
    for v in _kat():
        ctr = np.array([[int(w, 16) for w in v["counter"]]], dtype=np.uint64)
        key = np.array([[int(w, 16) for w in v["key"]]], dtype=np.uint64)
        got = O.philox4x32_10(ctr, key)[0]
        assert [int(g) for g in got] == [int(w, 16) for w in v["out"]]


def test_philox_blocks_layout():
    # block i of (seed, stream): counter (i lo, i hi, stream, 0), key (seed lo, seed hi)
    seed, stream = (0x0123456789ABCDEF, 5)
    off = (1 << 32) - 3  # crosses the carry into the counter's second word
    b = O.philox_blocks(seed, stream, off, 6)
    for t in range(6):
        i = off + t
        ctr = np.array([[i & 0xFFFFFFFF, i >> 32, stream, 0]], dtype=np.uint64)
        key = np.array([[seed & 0xFFFFFFFF, seed >> 32]], dtype=np.uint64)
        assert np.array_equal(b[t], O.philox4x32_10(ctr, key)[0])
    assert np.all(b < (1 << 32))


def test_philox_words_uniform_and_independent():
    w = O.philox_blocks(7, 0, 0, 1 << 15)
    top = (w >> np.uint64(24)).astype(np.int64).ravel()  # top byte of every word: 256 bins
    cnt = np.bincount(top, minlength=256)
    exp = top.size / 256.0
    chi2 = float(np.sum((cnt - exp) ** 2 / exp))
    assert chi2 < 255 + 6 * np.sqrt(2 * 255)  # chi-square, 255 degrees of freedom, > 6 sigma fails
    u = w.astype(np.float64) / 2.0 ** 32
    c = np.corrcoef(u.T)
    assert np.max(np.abs(c - np.eye(4))) < 5.0 / np.sqrt(u.shape[0])  # the four words of a block
    v = O.philox_blocks(7, 1, 0, 1 << 15).astype(np.float64) / 2.0 ** 32  # another stream
    assert abs(np.corrcoef(u.ravel(), v.ravel())[0, 1]) < 5.0 / np.sqrt(u.size)


def test_gaussian_factor_is_standard_normal():
    stats = pytest.importorskip("scipy.stats")
    z = O.gaussian_factor(1 << 14, 8, seed=11, stream=2)
    assert z.shape == (1 << 14, 8)
    x = z.ravel(order="F")
    n = x.size
    assert abs(x.mean()) < 5.0 / np.sqrt(n)
    assert abs(x.var() - 1.0) < 5.0 * np.sqrt(2.0 / n)
    assert stats.kstest(x, "norm").pvalue > 1e-4
    # the two members of a Box-Muller pair are uncorrelated, and so are the pairs of a block
    q = x[: (n // 4) * 4].reshape(-1, 4)
    c = np.corrcoef(q.T)
    assert np.max(np.abs(c - np.eye(4))) < 5.0 / np.sqrt(q.shape[0])
    # the radius r^2 = z0^2 + z1^2 of a pair is exponential with mean 2 (chi-square, 2 dof)
    r2 = q[:, 0] ** 2 + q[:, 1] ** 2
    assert stats.kstest(r2, "expon", args=(0, 2)).pvalue > 1e-4


def test_gaussian_factor_layout():
    # element e of the column-major order is draw e of the stream, whatever the shape
    a = O.gaussian_factor(5, 3, seed=4, stream=1)
    b = O.gaussian_factor(15, 1, seed=4, stream=1)
    c = O.gaussian_factor(1, 17, seed=4, stream=1)
    assert np.array_equal(a.ravel(order="F"), b.ravel())
    assert np.array_equal(c.ravel()[:15], b.ravel())
    assert O.gaussian_factor(0, 4, seed=4, stream=1).shape == (0, 4)
    assert not np.array_equal(O.gaussian_factor(8, 2, 4, 1), O.gaussian_factor(8, 2, 4, 2))
