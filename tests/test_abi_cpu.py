"""Host-side checks of the C ABI (no GPU): the library loads, exports every
entry point declared in include/tucker.h, and its integer planners agree with
the oracle and with the subranks printed in the paper."""
import ctypes
import json
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_2211_13028_gb300 import build as B
from paper_2211_13028_gb300 import synth
from paper_2211_13028_gb300 import tucker as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLDEN = os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return T.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "tucker.h")).read()
    return re.findall(r"^TK_API\s+[\w\s\*]+?\b(\w+)\s*\(", src, flags=re.M)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), n


def test_build_targets_sm103a():
    assert "arch=compute_103a,code=sm_103a" in B.ARCH


def _row_multiset(row, j):
    return sorted(int(v) for k, v in enumerate(row) if k != j)


@pytest.mark.parametrize("name", ["miranda", "sp"])
def test_c_planners_reproduce_paper(lib, name):
    gd = json.load(open(os.path.join(GOLDEN, "paper_subranks.json")))[name]
    s, _ = T.tucker_subranks_reuse(gd["r"], gd["p"])
    assert s == gd["s"]
    S, w = T.tucker_subranks_matrix(gd["r"], gd["p"])
    for j in range(len(gd["r"])):
        assert _row_multiset(S[j], j) == _row_multiset(gd["S"][j], j)


def test_c_planners_match_oracle_random(lib):
    g = np.random.Generator(np.random.PCG64(0))
    for _ in range(300):
        d = int(g.integers(2, 7))
        r = [int(x) for x in g.integers(1, 80, d)]
        p = int(g.integers(0, 12))
        order = [int(x) for x in g.permutation(d)]
        s_c, w_c = T.tucker_subranks_reuse(r, p)
        s_o, w_o = O.subranks_reuse(r, p)
        assert s_c == s_o and w_c == w_o
        S_c, w_c = T.tucker_subranks_matrix(r, p, order)
        S_o, w_o = O.subranks_matrix(r, p, order)
        assert w_c == list(w_o)
        assert S_c == [[int(v) for v in row] for row in S_o]


def test_c_planners_reject_bad_args(lib):
    with pytest.raises(T.TuckerError):
        T.tucker_subranks_reuse([5], 2)
    with pytest.raises(T.TuckerError):
        T.tucker_subranks_reuse([5, 0, 3], 2)
    with pytest.raises(T.TuckerError):
        T.tucker_subranks_matrix([5, 4, 3], -1)
    with pytest.raises(T.TuckerError):
        T.tucker_subranks_matrix([5, 4, 3], 1, [0, 0, 1])


def test_null_handle_is_rejected(lib):
    assert lib.tk_destroy(None) == 1
    assert lib.tk_sync_status(None, None) == 1
    assert lib.tucker_rhkron(None, None, None, 0, None, None, None, None, None) == 1


def test_binding_rejects_row_major_tensor():
    import torch
    t = torch.zeros((3, 4, 5))
    assert not T.is_colmajor(t)
    assert T.is_colmajor(t.permute(2, 1, 0).contiguous().permute(2, 1, 0))


def test_rsthkron_factor_plan_matches_host_draw_shapes(lib):
    # the device-draw plan of rSTHKron's factors has the shapes of the host generator's factors
    # (the oracle's inputs) and one distinct stream per factor
    for r, p, order in [((32, 32, 32), 8, [0, 1, 2]), ((10, 20, 30, 40), 6, [3, 2, 1, 0])]:
        d = len(r)
        dims = tuple(64 + 16 * j for j in range(d))
        S, w = T.tucker_subranks_matrix(r, p, order)
        k = [min(n, ww) for n, ww in zip(dims, w)]
        keys, shapes, streams = T.rsthkron_factor_plan(dims, S, k, order)
        host = synth.sketch_factors_matrix(dims, np.array(S), k, order, seed=0, dtype="f32")
        assert set(keys) == set(host.keys())
        for key, shp in zip(keys, shapes):
            assert shp == host[key].shape
        assert len(set(streams)) == len(streams)
        assert streams == [8 * j + kk for j, kk in keys]
