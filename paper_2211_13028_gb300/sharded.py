"""The sharded (data-parallel) form of Algorithm rHKron-re (Section 6.3, parallel
rHKron-re; Section 6.1, the all-at-once multi-TTM): X is split along its last
mode into contiguous slabs, one per rank, and every rank holds the full small
factors.

Each rank runs the library's slab calls on its own slab; the ranks exchange
  * the partial sketches Y_n, n < d-1 (SUM all-reduce) and the rows of Y_d
    (gathered along the last mode),
  * the partial cores (SUM all-reduce),
  * the two squared norms of the relative error (SUM all-reduce),
and the thin QR of the sketches and the STHOSVD of the core run redundantly on
every rank.  The exchanges use torch.distributed's collectives on whatever
group is initialised (device tensors are staged through host memory for a
backend without device support, such as gloo); with no group, or one rank,
they are no-ops.  ``rhkron_slabs`` runs the same steps for several slabs
inside one process (the exchanges become sums and copies on the device), so
one GPU can check the partitioning against the whole-tensor call.

This module only orchestrates: every step of the method runs in the library's
kernels (tucker.py's calls)."""
from __future__ import annotations

import math
from typing import List, Sequence, Tuple

import torch

from . import tucker as T

__all__ = ["allreduce_sum", "gather_last_mode", "rhkron_sharded", "rhkron_slabs", "slab_bounds"]


def _group_info(group):
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return None, 1, 0
    return dist, dist.get_world_size(group), dist.get_rank(group)


def _needs_host(t: torch.Tensor, dist, group) -> bool:
    return t.is_cuda and dist.get_backend(group) != "nccl"


def allreduce_sum(t: torch.Tensor, group=None) -> torch.Tensor:
    """In-place SUM over the ranks of ``group`` (a no-op for one rank); returns t."""
    dist, world, _ = _group_info(group)
    if world == 1:
        return t
    if _needs_host(t, dist, group):
        h = t.detach().cpu()
        dist.all_reduce(h, op=dist.ReduceOp.SUM, group=group)
        t.copy_(h)
    else:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t


def _flat(t: torch.Tensor) -> torch.Tensor:
    """The storage-order flat view of a column-major (mode-1 fastest) tensor."""
    return t.permute(*reversed(range(t.dim()))).reshape(-1)


def gather_last_mode(block: torch.Tensor, offset: int, n_last: int, group=None) -> torch.Tensor:
    """The full column-major tensor along the last mode (length n_last) from every rank's block of rows
    [offset, offset + block.shape[-1]).  Column-major storage puts a block of last-mode rows in one
    contiguous run, so the gather moves whole runs."""
    dist, world, _ = _group_info(group)
    shape = list(block.shape)
    rows = shape[-1]
    inner = block.numel() // max(1, rows)
    shape[-1] = n_last
    full = T.empty_f(shape, block.dtype, block.device)
    ff = _flat(full)
    if world == 1:
        ff[offset * inner:(offset + rows) * inner] = _flat(block)
        return full
    host = _needs_host(block, dist, group)
    meta = torch.tensor([offset, rows], dtype=torch.int64, device="cpu" if host or not block.is_cuda else block.device)
    metas = [torch.empty_like(meta) for _ in range(world)]
    dist.all_gather(metas, meta, group=group)
    spans = [(int(m[0]), int(m[1])) for m in metas]
    maxr = max(r for _, r in spans)
    pad = torch.zeros(maxr * inner, dtype=block.dtype, device=meta.device)
    pad[:rows * inner] = _flat(block).to(meta.device)
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    for (off, r), part in zip(spans, parts):
        ff[off * inner:(off + r) * inner] = part[:r * inner].to(ff.device)
    return full


def slab_bounds(n_last: int, parts: int, index: int) -> Tuple[int, int]:
    """(offset, rows) of slab ``index`` when n_last rows are split into ``parts`` near-equal slabs."""
    base, extra = divmod(n_last, parts)
    off = index * base + min(index, extra)
    return off, base + (1 if index < extra else 0)


def _check_widths(dims: Sequence[int], r: Sequence[int], p: int, Omega: Sequence[torch.Tensor]) -> None:
    s = [int(o.shape[1]) for o in Omega]
    for n in range(len(dims)):
        w = math.prod(s[j] for j in range(len(dims)) if j != n)
        if w < r[n] + p:
            raise T.TuckerError(2, "prod_{j!=n} s_j must be >= r_n + p")


def rhkron_sharded(X_slab: torch.Tensor, offset: int, n_last: int, r: Sequence[int], p: int,
                   Omega: Sequence[torch.Tensor], order=None, group=None):
    """Algorithm rHKron-re with X split along its last mode: this rank holds rows [offset, offset +
    X_slab.shape[-1]) of a last mode of length n_last, and the full factors Omega_j = Phi_j^T (Omega[-1]
    is n_last x s_d).  Returns (G, [U_j], rel_err), the same on every rank."""
    d = X_slab.dim()
    dims = list(X_slab.shape[:-1]) + [n_last]
    _check_widths(dims, r, p, Omega)
    Y = T.tucker_sketch_slab(X_slab, offset, n_last, Omega)
    for n in range(d - 1):
        allreduce_sum(Y[n], group)
    Y[d - 1] = gather_last_mode(Y[d - 1], offset, n_last, group)
    Q = T.tucker_orth_sketches(Y)
    G_hat = allreduce_sum(T.tucker_core_slab(X_slab, offset, n_last, Q), group)
    G, U = T.tucker_sthosvd(G_hat, Q, r, order)
    res2, x2 = T.tucker_loss_slab(X_slab, offset, n_last, G, U)
    norms = allreduce_sum(torch.tensor([res2, x2], dtype=torch.float64, device=X_slab.device), group)
    res2, x2 = float(norms[0]), float(norms[1])
    return G, U, (math.sqrt(res2 / x2) if x2 > 0 else 0.0)


def rhkron_slabs(X: torch.Tensor, nslabs: int, r: Sequence[int], p: int, Omega: Sequence[torch.Tensor],
                 order=None) -> Tuple[torch.Tensor, List[torch.Tensor], float]:
    """The sharded steps for ``nslabs`` slabs of one device tensor X (column-major) inside one process:
    the SUM exchanges become sums on the device and the gather a copy into place."""
    d = X.dim()
    n_last = int(X.shape[-1])
    _check_widths(list(X.shape), r, p, Omega)
    slabs = [slab_bounds(n_last, nslabs, i) for i in range(nslabs)]
    Y = None
    Yd = None
    for off, rows in slabs:
        part = T.tucker_sketch_slab(X[..., off:off + rows], off, n_last, Omega)
        if Y is None:
            Y = part[:d - 1]
            shape = list(part[d - 1].shape)
            shape[-1] = n_last
            Yd = T.empty_f(shape, part[d - 1].dtype, X.device)
        else:
            for n in range(d - 1):
                Y[n] += part[n]
        Yd[..., off:off + rows] = part[d - 1]
    Q = T.tucker_orth_sketches(Y + [Yd])
    G_hat = None
    for off, rows in slabs:
        g = T.tucker_core_slab(X[..., off:off + rows], off, n_last, Q)
        G_hat = g if G_hat is None else G_hat.add_(g)
    G, U = T.tucker_sthosvd(G_hat, Q, r, order)
    res2 = x2 = 0.0
    for off, rows in slabs:
        a, b = T.tucker_loss_slab(X[..., off:off + rows], off, n_last, G, U)
        res2 += a
        x2 += b
    return G, U, (math.sqrt(res2 / x2) if x2 > 0 else 0.0)
