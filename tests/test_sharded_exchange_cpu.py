"""The exchange of the sharded rHKron-re (CPU).

With X split into slabs along its last mode d (rank q holds X[..., rows_q]), every quantity of
rHKron-re that contracts mode d is a sum of per-slab partials, and the sketch of mode d itself is
a row-wise concatenation (one exchange per phase): Y_n for n != d is the sum over slabs of
X_q x_{j!=n} Phi_j with Phi_d restricted to the slab's rows, Y_d stacks the slabs' Y_d rows, and
Ghat is the sum of X_q x_{j<d} Q_j^T x_d Q_d[rows_q]^T.  The first two tests pin these identities
on the FP64 oracle alone; the gloo test runs the library's exchange helpers (sharded.allreduce_sum
and sharded.gather_last_mode, the ones sharded.rhkron_sharded uses) across two ranks on the
oracle's slab partials.  tests/test_gpu_sharded.py feeds the library's own slab calls into them.
"""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DIMS, S = (9, 8, 13), (3, 2, 4)  # 13 rows: two ranks get uneven slabs (7 and 6)


def _problem(seed=5):
    g = np.random.Generator(np.random.PCG64(seed))
    x = g.standard_normal(DIMS)
    oms = [g.standard_normal((n, s)) for n, s in zip(DIMS, S)]  # Omega_j = Phi_j^T
    return x, oms


def _slab_partials(x, oms, rows):
    """Rank-local sketches of the slab X[..., rows]: Y_n (n != d) partials and the slab's Y_d rows."""
    d = x.ndim
    xs = x[..., rows]
    om_s = list(oms[:-1]) + [oms[-1][rows, :]]
    part = [O.multi_ttm(xs, [(j, om_s[j].T) for j in range(d) if j != n]) for n in range(d - 1)]
    yd = O.multi_ttm(xs, [(j, oms[j].T) for j in range(d - 1)])
    return part, yd


def test_slab_sketches_sum_and_stack_to_the_full_sketch():
    x, oms = _problem()
    d = x.ndim
    full = [O.multi_ttm(x, [(j, oms[j].T) for j in range(d) if j != n]) for n in range(d)]
    slabs = [np.arange(0, 5), np.arange(5, 9), np.arange(9, 13)]  # uneven slabs
    parts = [_slab_partials(x, oms, rows) for rows in slabs]
    for n in range(d - 1):
        assert np.max(np.abs(sum(p[0][n] for p in parts) - full[n])) <= 1e-12 * np.max(np.abs(full[n]))
    assert np.array_equal(np.concatenate([p[1] for p in parts], axis=d - 1), full[d - 1])


def test_slab_cores_sum_to_the_full_core():
    x, oms = _problem(7)
    d = x.ndim
    qs = [O.thin_qr(O.unfold(O.multi_ttm(x, [(j, oms[j].T) for j in range(d) if j != n]), n)) for n in range(d)]
    full = O.multi_ttm(x, [(j, qs[j].T) for j in range(d)])
    slabs = [np.arange(0, 7), np.arange(7, 13)]
    parts = [O.multi_ttm(x[..., rows], [(j, qs[j].T) for j in range(d - 1)] + [(d - 1, qs[d - 1][rows, :].T)])
             for rows in slabs]
    assert np.max(np.abs(sum(parts) - full)) <= 1e-12 * np.max(np.abs(full))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _fortran(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a.transpose())).permute(*reversed(range(a.ndim)))


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import oracle as Ox
    from paper_2211_13028_gb300 import sharded

    dist.init_process_group("gloo", rank=rank, world_size=world)
    x, oms = _problem(11)
    off, nrows = sharded.slab_bounds(DIMS[-1], world, rank)
    rows = np.arange(off, off + nrows)
    part, yd = _slab_partials(x, oms, rows)
    reduced = [sharded.allreduce_sum(_fortran(y)).permute(*reversed(range(x.ndim))).numpy().transpose()
               for y in part]  # the all-reduce of the sketches of the modes other than d
    full_d = sharded.gather_last_mode(_fortran(yd), off, DIMS[-1])  # the gather of the mode-d rows
    dist.destroy_process_group()
    d = x.ndim
    full = [Ox.multi_ttm(x, [(j, oms[j].T) for j in range(d) if j != n]) for n in range(d)]
    err = max(float(np.max(np.abs(reduced[n] - full[n]))) for n in range(d - 1))
    stacked = full_d.permute(*reversed(range(d))).numpy().transpose()
    q.put((rank, err, bool(np.array_equal(stacked, full[d - 1]))))


def test_slab_bounds_cover_the_mode():
    sys.path.insert(0, ROOT)
    from paper_2211_13028_gb300 import sharded

    for n, parts in ((12, 2), (13, 3), (512, 8), (5, 5), (7, 1)):
        spans = [sharded.slab_bounds(n, parts, i) for i in range(parts)]
        assert spans[0][0] == 0 and sum(r for _, r in spans) == n
        assert all(a + r == b for (a, r), (b, _) in zip(spans, spans[1:]))
        assert max(r for _, r in spans) - min(r for _, r in spans) <= 1


def test_two_gloo_ranks_exchange_the_slab_sketches():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, err, stacked_ok in out:
        assert err <= 1e-12 and stacked_ok, (rank, err)
