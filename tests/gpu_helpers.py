"""Shared helpers for the GPU parity tests (no test functions here)."""
import numpy as np
import pytest
import torch

from paper_2211_13028_gb300 import synth

TOL = {"f64": 1e-12, "f32": 1e-5, "bf16": 1e-5, "fp8": 1e-5}


def require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2211_13028_gb300 import build as B
    from paper_2211_13028_gb300 import tucker as T
    B.build()
    T.load()
    return torch.device("cuda", 0)


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def to_np(t):
    if t.dim() == 2:
        return t.detach().double().cpu().numpy()
    return synth.from_fortran(t)


def align(G, U, Uref):
    """Flip the columns of U (and G's matching slices) to the reference's sign gauge."""
    G = G.copy()
    U = [u.copy() for u in U]
    for j, (u, ur) in enumerate(zip(U, Uref)):
        sg = np.sign(np.sum(u * ur, axis=0))
        sg[sg == 0] = 1.0
        U[j] = u * sg
        G = np.moveaxis(np.moveaxis(G, j, -1) * sg, -1, j)
    return G, U


def make_X(x64, dtype, dev, fp8_scale=None):
    """Device tensor in ``dtype`` plus the float64 values the oracle must see."""
    if dtype == "fp8":
        amax = np.max(np.abs(x64))
        scale = 448.0 / amax if fp8_scale is None else fp8_scale
        t = torch.from_numpy(np.ascontiguousarray((x64 * scale).transpose())).to(dev, torch.float32)
        t8 = t.to(torch.float8_e4m3fn)
        vals = t8.to(torch.float64).cpu().numpy().transpose() / scale
        X = t8.permute(*reversed(range(t8.dim())))
        return X, vals, float(scale)
    vals = synth.round_to(x64, dtype)
    return synth.fortran(vals, dtype, dev), vals, 1.0


def mats(oms, dtype, dev):
    return [synth.fmat(o, dtype, dev) for o in oms]
