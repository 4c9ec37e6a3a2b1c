"""Seeded synthetic inputs for the randomized Tucker path.

This module draws random numbers and assembles test tensors; it performs no
step of the decomposition (no sketch, no QR of a sketch, no core multi-TTM, no
truncation).  The tests, the benchmark and the oracle's expected-value
scripts all take their inputs from here, so the CUDA path and the FP64 oracle
consume identical values.

Conventions
-----------
* Tensors are returned as numpy float64 arrays indexed ``X[i1, ..., id]``
  (values already rounded to the working dtype when one is given) or as torch
  tensors in column-major layout (mode 1 fastest, strides ascending), which is
  the layout the C-ABI expects.
* Sketch factors follow Section 4.2: Phi_j is s_j x n_j with i.i.d. N(0,1)
  entries.  They are handed around as Omega_j = Phi_j^T (n_j x s_j), the
  orientation the C-ABI takes.
* ``dtype`` names are the C-ABI's: "f64", "f32", "bf16", "fp8".  A value drawn
  for a narrower dtype is rounded once (round to nearest even) so that both
  sides see exactly representable numbers.
"""
from __future__ import annotations

import math
from typing import Dict, List, Sequence, Tuple

import numpy as np
import torch

__all__ = [
    "round_to",
    "fortran",
    "from_fortran",
    "fmat",
    "sketch_factors_reuse",
    "sketch_factors_matrix",
    "sketch_factors_noreuse",
    "tucker_tensor",
    "decaying_core",
    "gaussian_bumps",
    "e1_tensor",
    "tucker4_device",
]

_TORCH_DT = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}


def round_to(x: np.ndarray, dtype: str) -> np.ndarray:
    """Round float64 values to the nearest value representable in ``dtype``.

    Returns float64 so the oracle can consume the rounded values directly.
    """
    x = np.asarray(x, dtype=np.float64)
    if dtype == "f64":
        return x.copy()
    if dtype == "f32":
        return x.astype(np.float32).astype(np.float64)
    if dtype == "bf16":
        t = torch.from_numpy(np.ascontiguousarray(x)).to(torch.bfloat16)
        return t.to(torch.float64).numpy().reshape(x.shape)
    raise ValueError(f"unknown dtype {dtype!r}")


def fortran(x: np.ndarray | torch.Tensor, dtype: str = "f32", device="cpu") -> torch.Tensor:
    """Column-major (mode-1 fastest) torch tensor with the values of ``x``.

    The result has shape (n1, ..., nd) and strides (1, n1, n1*n2, ...).
    """
    if isinstance(x, np.ndarray):
        t = torch.from_numpy(np.ascontiguousarray(x.transpose()))
    else:
        t = x.permute(*reversed(range(x.dim()))).contiguous()
    t = t.to(device=device, dtype=_TORCH_DT[dtype])
    return t.permute(*reversed(range(t.dim())))


def fmat(a: np.ndarray, dtype: str = "f32", device="cpu") -> torch.Tensor:
    """Column-major (stride(0) == 1) torch matrix with the values of the 2-D array ``a``."""
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.float64).T))
    return t.to(device=device, dtype=_TORCH_DT[dtype]).t()


def from_fortran(t: torch.Tensor) -> np.ndarray:
    """float64 numpy array ``X[i1, ..., id]`` from a column-major torch tensor."""
    return t.detach().to("cpu", torch.float64).numpy().copy()


def _gen(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def sketch_factors_reuse(dims: Sequence[int], s: Sequence[int], seed: int, dtype: str = "f64") -> List[np.ndarray]:
    """Omega_j = Phi_j^T, Phi_j in R^{s_j x n_j} i.i.d. N(0,1) (Algorithm rHKron-re).

    One set of d factors, shared by every mode's sketch.
    """
    g = _gen(seed)
    out = []
    for n, sj in zip(dims, s):
        phi = g.standard_normal((int(sj), int(n)))
        out.append(round_to(phi.T, dtype))
    return out


def hadamard_columns(n: int, s: int, seed: int, dtype: str = "f64") -> np.ndarray:
    """H_j of the Kronecker-SRHT sketch: s distinct columns, drawn uniformly
    without replacement, of the n x n Walsh-Hadamard matrix (Sylvester order,
    entry (i, k) = (-1)^popcount(i & k)) scaled by 1/sqrt(n).  n must be a
    power of two."""
    if n < 1 or n & (n - 1):
        raise ValueError("hadamard_columns: n must be a power of two")
    cols = np.sort(_gen(seed).choice(n, size=int(s), replace=False))
    i = np.arange(n, dtype=np.int64)[:, None]
    bits = np.bitwise_and(i, cols[None, :].astype(np.int64))
    par = np.zeros_like(bits)
    while np.any(bits):
        par ^= bits & 1
        bits >>= 1
    return round_to(np.where(par == 1, -1.0, 1.0) / np.sqrt(n), dtype)


def sketch_factors_srht(dims: Sequence[int], s: Sequence[int], seed: int, dtype: str = "f64") -> List[np.ndarray]:
    """One Walsh-Hadamard factor per mode, independent draws (Section 5)."""
    return [hadamard_columns(int(n), int(sj), seed + 7919 * j, dtype) for j, (n, sj) in enumerate(zip(dims, s))]


def sketch_factors_noreuse(dims: Sequence[int], S: np.ndarray, seed: int, dtype: str = "f64") -> Dict[Tuple[int, int], np.ndarray]:
    """Omega_{j,k} = Phi_{j,k}^T with Phi_{j,k} in R^{s_{j,k} x n_k} (appendix Algorithm rHKron)."""
    g = _gen(seed)
    d = len(dims)
    out = {}
    for j in range(d):
        for k in range(d):
            if k == j:
                continue
            phi = g.standard_normal((int(S[j][k]), int(dims[k])))
            out[(j, k)] = round_to(phi.T, dtype)
    return out


def sketch_factors_matrix(dims: Sequence[int], S: np.ndarray, kdims: Sequence[int], order: Sequence[int],
                          seed: int, dtype: str = "f64") -> Dict[Tuple[int, int], np.ndarray]:
    """Factors for Algorithm rSTHKron, drawn in processing order.

    For the mode j processed at position t, Phi_{j,k} is s_{j,k} x (current
    size of mode k): k_k for modes processed earlier, n_k otherwise.
    Returned as Omega_{j,k} = Phi_{j,k}^T keyed by (j, k).
    """
    g = _gen(seed)
    d = len(dims)
    out = {}
    done = set()
    for j in order:
        for k in range(d):
            if k == j:
                continue
            cur = int(kdims[k]) if k in done else int(dims[k])
            phi = g.standard_normal((int(S[j][k]), cur))
            out[(j, k)] = round_to(phi.T, dtype)
        done.add(j)
    return out


def _orthonormal(g: np.random.Generator, n: int, r: int) -> np.ndarray:
    q, rr = np.linalg.qr(g.standard_normal((n, r)))
    return q * np.where(np.diag(rr) < 0, -1.0, 1.0)


def decaying_core(core_dims: Sequence[int], ratio: float, seed: int) -> np.ndarray:
    """Core with entries N(0,1) * ratio^(sum of zero-based indices)."""
    g = _gen(seed)
    c = g.standard_normal(tuple(core_dims))
    idx = np.indices(tuple(core_dims)).sum(axis=0)
    return c * ratio ** idx


def tucker_tensor(dims: Sequence[int], core_dims: Sequence[int], seed: int, noise_rel: float = 0.0,
                  core: np.ndarray | None = None) -> np.ndarray:
    """core x_1 U_1 ... x_d U_d with random orthonormal U_j, plus Gaussian noise.

    The noise E ~ N(0,1) is scaled so that ||E|| = noise_rel * ||X0||.
    ``core`` defaults to i.i.d. N(0,1) entries.  Assembled with einsum
    contractions on the host (input synthesis only).
    """
    g = _gen(seed)
    d = len(dims)
    if core is None:
        core = g.standard_normal(tuple(core_dims))
    us = [_orthonormal(g, int(n), int(r)) for n, r in zip(dims, core_dims)]
    x = core
    for j in range(d):
        x = np.moveaxis(np.tensordot(us[j], x, axes=([1], [j])), 0, j)
    if noise_rel > 0:
        e = g.standard_normal(x.shape)
        x = x + e * (noise_rel * np.linalg.norm(x) / np.linalg.norm(e))
    return x


def e1_tensor(n: int, ratio: float = 0.4, seed: int = 0, d: int = 3) -> np.ndarray:
    """Section 7.1 test tensor: superdiagonal core ratio^(i-1), random orthogonal factors."""
    g = _gen(seed)
    core = np.zeros((n,) * d)
    for i in range(n):
        core[(i,) * d] = ratio ** i
    x = core
    for j in range(d):
        q = _orthonormal(g, n, n)
        x = np.moveaxis(np.tensordot(q, x, axes=([1], [j])), 0, j)
    return x


def gaussian_bumps(n: int, d: int = 3, nbumps: int = 200, seed: int = 0, noise_rel: float = 1e-4,
                   device="cpu", out_dtype: str = "f32") -> torch.Tensor:
    """Smooth field: sum of axis-aligned anisotropic Gaussian bumps plus noise.

    X[i] = sum_b a_b prod_k exp(-(i_k - c_bk)^2 / (2 sigma_bk^2)) on the unit
    grid i_k = 0..n-1, with a ~ U(0.5, 1.5), c ~ U(0, n), sigma ~ U(n/64, n/8),
    plus Gaussian noise scaled to noise_rel * ||X0||.  The bump parameters are
    drawn with numpy PCG64(seed); the field is assembled (one GEMM of the
    mode-1 factor against the Khatri-Rao product of the others, float64) and the
    noise drawn with a seeded torch generator on ``device``.  Returned
    column-major in ``out_dtype``.
    """
    g = _gen(seed)
    a = g.uniform(0.5, 1.5, nbumps)
    c = g.uniform(0.0, n, (d, nbumps))
    sg = g.uniform(n / 64.0, n / 8.0, (d, nbumps))
    grid = np.arange(n, dtype=np.float64)[:, None]
    facs = [np.exp(-((grid - c[k][None, :]) ** 2) / (2.0 * sg[k][None, :] ** 2)) for k in range(d)]
    dev = torch.device(device)
    f = [torch.from_numpy(fk).to(dev) for fk in facs]
    # Khatri-Rao product of modes d..2 (mode 2 fastest in the column index).
    kr = f[1]
    for k in range(2, d):
        kr = (f[k][:, None, :] * kr[None, :, :]).reshape(-1, nbumps)
    a_t = torch.from_numpy(a).to(dev)
    x1 = (f[0] * a_t[None, :]) @ kr.T  # X_(1), n x n^(d-1), float64
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed + 1)
    e = torch.randn(x1.shape, generator=gen, device=dev, dtype=torch.float64)
    x1 += e * (noise_rel * torch.linalg.vector_norm(x1) / torch.linalg.vector_norm(e))
    del e
    # X_(1) column-major n x n^(d-1) is exactly the column-major tensor layout.
    flat = x1.T.contiguous().to(_TORCH_DT[out_dtype])  # (n^(d-1), n) row-major == X col-major
    t = flat.reshape((n,) * d)  # reversed-dims C order
    return t.permute(*reversed(range(d)))


def tucker4_device(n: int, core_n: int, ratio: float, noise_rel: float, seed: int, device, out_dtype="f32") -> torch.Tensor:
    """4-way core x U (random orthonormal factors) + noise, assembled on ``device``.

    Core entries N(0,1) * ratio^(index sum); factors and core drawn with
    numpy PCG64(seed); the noise with a seeded torch generator on ``device``.
    """
    g = _gen(seed)
    core = g.standard_normal((core_n,) * 4) * ratio ** np.indices((core_n,) * 4).sum(axis=0)
    us = [_orthonormal(g, n, core_n) for _ in range(4)]
    dev = torch.device(device)
    x = torch.from_numpy(core).to(dev)
    for j in range(4):
        u = torch.from_numpy(us[j]).to(dev)
        x = torch.movedim(torch.tensordot(u, x, dims=([1], [j])), 0, j)
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed + 1)
    e = torch.randn(x.shape, generator=gen, device=dev, dtype=torch.float64)
    x += e * (noise_rel * torch.linalg.vector_norm(x) / torch.linalg.vector_norm(e))
    del e
    t = x.permute(3, 2, 1, 0).contiguous().to(_TORCH_DT[out_dtype])
    return t.permute(3, 2, 1, 0)
