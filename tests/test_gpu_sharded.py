"""The sharded form of rHKron-re (X split along its last mode) on one GPU.

The slab calls run on every slab of one device tensor (sharded.rhkron_slabs: the SUM exchanges
become sums on the device, the gather a copy into place) and must reproduce the whole-tensor
decomposition and the FP64 oracle.  Each slab call is also checked against the oracle's
statement of what a slab contributes.  Finally two gloo ranks on the CPU run the library's
exchange helpers (the ones sharded.rhkron_sharded calls) on the slab calls' own outputs."""
import os
import socket
import sys
import tempfile

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle as O
from paper_2211_13028_gb300 import sharded, synth
from paper_2211_13028_gb300 import tucker as T
from tests.gpu_helpers import align, mats, rel, require_gpu, to_np

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dev():
    return require_gpu()


def _check(G, U, err, ref, xv, tol):
    ref_err = O.rel_err(xv, ref["G"], ref["U"])
    assert abs(err - ref_err) <= tol, (err, ref_err)
    g, u = align(to_np(G), [to_np(x) for x in U], ref["U"])
    assert rel(g, ref["G"]) <= tol
    assert rel(O.reconstruct(g, u), O.reconstruct(ref["G"], ref["U"])) <= tol


@pytest.mark.parametrize("nslabs", [1, 2, 3])
def test_slabs_reproduce_rhkron_f64(dev, nslabs):
    dims, r, p = (40, 36, 31), (6, 5, 4), 4  # 31 rows: uneven slabs
    x = synth.tucker_tensor(dims, r, seed=3, noise_rel=1e-3)
    s = O.subranks_reuse(r, p)[0]
    oms = synth.sketch_factors_reuse(dims, s, seed=4)
    X = synth.fortran(x, "f64", dev)
    G, U, err = sharded.rhkron_slabs(X, nslabs, r, p, mats(oms, "f64", dev))
    ref = O.rhkron(x, r, oms)
    _check(G, U, err, ref, x, 1e-12)
    G1, U1, err1 = T.tucker_rhkron(X, r, p, mats(oms, "f64", dev))
    assert abs(err - err1) <= 1e-13


def test_slabs_reproduce_rhkron_f32_bumps(dev):
    n, r, p = 96, (12, 12, 12), 6
    X = synth.gaussian_bumps(n, 3, 200, 0, 1e-4, dev, "f32")
    xv = synth.from_fortran(X)
    s = O.subranks_reuse(r, p)[0]
    oms = synth.sketch_factors_reuse(X.shape, s, seed=5, dtype="f32")
    G, U, err = sharded.rhkron_slabs(X, 4, r, p, mats(oms, "f32", dev))
    ref = O.rhkron(xv, r, oms)
    _check(G, U, err, ref, xv, 1e-5)


def test_each_slab_call_against_the_oracle(dev):
    dims, s = (24, 20, 18), (4, 3, 5)
    g = np.random.Generator(np.random.PCG64(9))
    x = g.standard_normal(dims)
    oms = [g.standard_normal((nn, ss)) for nn, ss in zip(dims, s)]
    qs = [np.linalg.qr(g.standard_normal((nn, k)))[0] for nn, k in zip(dims, (7, 6, 5))]
    X = synth.fortran(x, "f64", dev)
    off, rows = 5, 9
    Xs = X[..., off:off + rows]
    xs = x[..., off:off + rows]
    Y = T.tucker_sketch_slab(Xs, off, dims[-1], mats(oms, "f64", dev))
    om_s = oms[:-1] + [oms[-1][off:off + rows]]
    for nn in range(2):
        ref = O.multi_ttm(xs, [(j, om_s[j].T) for j in range(3) if j != nn])
        assert rel(to_np(Y[nn]), ref) <= 1e-13
    assert rel(to_np(Y[2]), O.multi_ttm(xs, [(j, oms[j].T) for j in range(2)])) <= 1e-13
    Gp = T.tucker_core_slab(Xs, off, dims[-1], mats(qs, "f64", dev))
    ref = O.multi_ttm(xs, [(0, qs[0].T), (1, qs[1].T), (2, qs[2][off:off + rows].T)])
    assert rel(to_np(Gp), ref) <= 1e-13
    Gr = g.standard_normal((3, 2, 4))
    Ur = [np.linalg.qr(g.standard_normal((nn, k)))[0] for nn, k in zip(dims, (3, 2, 4))]
    a, b = T.tucker_loss_slab(Xs, off, dims[-1], synth.fortran(Gr, "f64", dev), mats(Ur, "f64", dev))
    xh = O.reconstruct(Gr, Ur)[..., off:off + rows]
    assert abs(a - np.sum((xs - xh) ** 2)) <= 1e-12 * np.sum(xs ** 2)
    assert abs(b - np.sum(xs ** 2)) <= 1e-12 * np.sum(xs ** 2)
    with pytest.raises(T.TuckerError):  # a slab reaching past the mode
        T.tucker_sketch_slab(Xs, dims[-1] - rows + 1, dims[-1], mats(oms, "f64", dev))


def test_sthosvd_of_the_core_matches_rhkron(dev):
    dims, r, p = (40, 36, 32), (6, 5, 4), 4
    x = synth.tucker_tensor(dims, r, seed=13, noise_rel=1e-3)
    s = O.subranks_reuse(r, p)[0]
    oms = synth.sketch_factors_reuse(dims, s, seed=14)
    X = synth.fortran(x, "f64", dev)
    Q = T.tucker_orth_sketches(T.tucker_sketch(X, mats(oms, "f64", dev)))
    G, U = T.tucker_sthosvd(T.tucker_core(X, Q), Q, r)
    ref = O.rhkron(x, r, oms)
    g, u = align(to_np(G), [to_np(q) for q in U], ref["U"])
    assert rel(g, ref["G"]) <= 1e-12


# ------------------------------------------------------------------ two gloo ranks on the slab calls' outputs

def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, folder, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch as th
    import torch.distributed as dist

    from paper_2211_13028_gb300 import sharded as sh

    dist.init_process_group("gloo", rank=rank, world_size=world)
    z = np.load(os.path.join(folder, "rank%d.npz" % rank))
    full = np.load(os.path.join(folder, "full.npz"))
    n_last, off = int(z["n_last"]), int(z["off"])

    def fortran(a):
        return th.from_numpy(np.ascontiguousarray(a.transpose())).permute(*reversed(range(a.ndim)))

    def back(t):
        return t.permute(*reversed(range(t.dim()))).numpy().transpose()

    errs = []
    for nn in range(2):
        errs.append(rel(back(sh.allreduce_sum(fortran(z["y%d" % nn]))), full["y%d" % nn]))
    errs.append(rel(back(sh.gather_last_mode(fortran(z["y2"]), off, n_last)), full["y2"]))
    errs.append(rel(back(sh.allreduce_sum(fortran(z["g"]))), full["g"]))
    dist.destroy_process_group()
    q.put((rank, max(errs)))


def test_two_gloo_ranks_exchange_the_slab_calls_outputs(dev):
    dims, s = (30, 28, 25), (4, 3, 5)
    g = np.random.Generator(np.random.PCG64(21))
    x = g.standard_normal(dims)
    oms = [g.standard_normal((nn, ss)) for nn, ss in zip(dims, s)]
    X = synth.fortran(x, "f64", dev)
    Yf = T.tucker_sketch(X, mats(oms, "f64", dev))
    Q = T.tucker_orth_sketches(Yf)
    Gf = T.tucker_core(X, Q)
    with tempfile.TemporaryDirectory() as folder:
        np.savez(os.path.join(folder, "full.npz"), y0=to_np(Yf[0]), y1=to_np(Yf[1]), y2=to_np(Yf[2]), g=to_np(Gf))
        for rank in range(2):
            off, rows = sharded.slab_bounds(dims[-1], 2, rank)
            Xs = X[..., off:off + rows]
            Y = T.tucker_sketch_slab(Xs, off, dims[-1], mats(oms, "f64", dev))
            Gp = T.tucker_core_slab(Xs, off, dims[-1], Q)
            np.savez(os.path.join(folder, "rank%d.npz" % rank), y0=to_np(Y[0]), y1=to_np(Y[1]), y2=to_np(Y[2]),
                     g=to_np(Gp), n_last=dims[-1], off=off)
        ctx = mp.get_context("spawn")
        q = ctx.Queue()
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, folder, q)) for r in range(2)]
        for p in procs:
            p.start()
        out = sorted(q.get(timeout=180) for _ in procs)
        for p in procs:
            p.join(timeout=60)
            assert p.exitcode == 0
    for rank, err in out:
        assert err <= 1e-13, (rank, err)
