"""ctypes binding of libtucker (include/tucker.h), one Python function per C
entry point with the same name.  Argument marshalling only: every step of the
computation runs in the library's CUDA kernels.  Torch supplies device memory
and the current stream.

Tensors are torch tensors on a CUDA device in column-major layout (mode 1
fastest, strides ascending; see ``empty_f`` / ``synth.fortran``); a tensor in
any other layout is rejected, never copied silently.  Matrices are 2-D torch
tensors with stride(0) == 1 (column-major, leading dimension stride(1)).

Loading fails loudly (``TuckerError``) when libtucker.so has not been built;
there is no fallback path.
"""
from __future__ import annotations

import collections
import ctypes
import os
import threading
from typing import Dict, List, Optional, Sequence, Tuple

import torch

__all__ = [
    "TuckerError", "load", "empty_f", "is_colmajor",
    "tucker_subranks_reuse", "tucker_subranks_matrix",
    "tucker_sketch", "tucker_orth", "tucker_orth_noalloc", "tucker_core", "tucker_rhkron", "tucker_rsthkron",
    "tucker_reconstruct", "tucker_loss", "tucker_reconstruct_backward", "tucker_rhkron_grad",
    "tk_sync_status", "tk_selftest_bounded_wait", "tk_set_sm_reserve", "tk_launch_count", "tk_workspace_bytes", "tk_profile", "tk_profile_read", "tk_profile_trace", "TuckerLoss",
    "library_path", "PendingScalar", "tucker_rhkron_noreuse", "tucker_rhkron_srht", "tk_graph_release",
    "tk_philox4x32", "tucker_gaussian_factor", "tucker_gaussian_factors", "gaussian_factors",
    "gaussian_factors_matrix", "rsthkron_factor_plan",
    "TuckerGraph", "tucker_sketch_slab", "tucker_orth_sketches", "tucker_core_slab", "tucker_sthosvd",
    "tucker_loss_slab",
]

TK_MAX_D = 8
TK_F64, TK_F32, TK_BF16, TK_FP8 = 0, 1, 2, 3
_STATUS = {0: "TK_OK", 1: "TK_ERR_ARG", 2: "TK_ERR_SHAPE", 3: "TK_ERR_DTYPE", 4: "TK_ERR_ALIGN",
           5: "TK_ERR_WORKSPACE", 6: "TK_ERR_CUDA", 7: "TK_ERR_NOT_CONVERGED", 8: "TK_ERR_TIMEOUT"}
_DT = {torch.float64: TK_F64, torch.float32: TK_F32, torch.bfloat16: TK_BF16}
if hasattr(torch, "float8_e4m3fn"):
    _DT[torch.float8_e4m3fn] = TK_FP8


class TuckerError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class TkTensor(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("dims", ctypes.c_int64 * TK_MAX_D), ("dtype", ctypes.c_int),
                ("data", ctypes.c_void_p), ("scale", ctypes.c_float)]


class TkMatrix(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("ld", ctypes.c_int64),
                ("dtype", ctypes.c_int), ("data", ctypes.c_void_p)]


class TkProfEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


class TkTraceEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("stream", ctypes.c_int), ("reserved", ctypes.c_int),
                ("start_us", ctypes.c_double), ("end_us", ctypes.c_double), ("bytes", ctypes.c_double),
                ("flops", ctypes.c_double)]


class TkOpts(ctypes.Structure):
    _fields_ = [("mode_order", ctypes.POINTER(ctypes.c_int)), ("qr_method", ctypes.c_int), ("refine", ctypes.c_int),
                ("max_jacobi_sweeps", ctypes.c_int), ("async_outputs", ctypes.c_int), ("reserved", ctypes.c_int * 4)]


_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None
_lock = threading.Lock()
_handles: Dict[Tuple[int, int], ctypes.c_void_p] = {}  # one handle (and workspace) per (device, stream)
# Host doubles that a handle's stream-ordered callbacks may still write: the library reuses one of
# its 64 callback slots only after that slot's callback ran, so the 64 most recent stay referenced.
_pending: Dict[int, "collections.deque"] = {}


def library_path() -> str:
    return os.environ.get("TUCKER_LIB", os.path.join(_HERE, "_build", "libtucker.so"))


def load():
    """Load libtucker.so (built by paper_2211_13028_gb300.build); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise TuckerError(6, f"libtucker.so not found at {path}; build it with "
                                 "`python -m paper_2211_13028_gb300.build`")
        lib = ctypes.CDLL(path)
        P = ctypes.POINTER
        vp, i64p = ctypes.c_void_p, P(ctypes.c_int64)
        sig = {
            "tk_create": ([P(vp), vp], ctypes.c_int),
            "tk_destroy": ([vp], ctypes.c_int),
            "tk_set_stream": ([vp, vp], ctypes.c_int),
            "tk_last_error": ([vp], ctypes.c_char_p),
            "tk_sync_status": ([vp, P(ctypes.c_int)], ctypes.c_int),
            "tk_selftest_bounded_wait": ([vp, ctypes.c_int64, P(ctypes.c_int64)], ctypes.c_int),
            "tk_workspace_bytes": ([vp], ctypes.c_int64),
            "tk_launch_count": ([vp], ctypes.c_int64),
            "tk_profile": ([vp, ctypes.c_int], ctypes.c_int),
            "tk_profile_only": ([vp, ctypes.c_char_p], ctypes.c_int),
            "tk_profile_read": ([vp, P(TkProfEntry), ctypes.c_int], ctypes.c_int),
            "tk_profile_trace": ([vp, P(TkTraceEntry), ctypes.c_int], ctypes.c_int),
            "tk_graph_release": ([vp], ctypes.c_int),
            "tk_philox4x32": ([vp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64, vp],
                              ctypes.c_int),
            "tucker_gaussian_factor": ([vp, ctypes.c_uint64, ctypes.c_uint32, P(TkMatrix)], ctypes.c_int),
            "tucker_gaussian_factors": ([vp, ctypes.c_uint64, ctypes.c_int, P(ctypes.c_uint32), P(TkMatrix)],
                                        ctypes.c_int),
            "tucker_subranks_reuse": ([ctypes.c_int, i64p, ctypes.c_int, i64p, i64p], ctypes.c_int),
            "tucker_subranks_matrix": ([ctypes.c_int, i64p, ctypes.c_int, P(ctypes.c_int), i64p, i64p], ctypes.c_int),
            "tucker_sketch": ([vp, P(TkTensor), P(TkMatrix), P(TkTensor)], ctypes.c_int),
            "tucker_orth": ([vp, P(TkMatrix), P(TkMatrix), P(ctypes.c_int), P(TkOpts)], ctypes.c_int),
            "tucker_core": ([vp, P(TkTensor), P(TkMatrix), P(TkTensor)], ctypes.c_int),
            "tucker_orth_noalloc": ([vp, P(TkMatrix), P(TkMatrix), P(ctypes.c_int)], ctypes.c_int),
            "tucker_rhkron": ([vp, P(TkTensor), i64p, ctypes.c_int, P(TkMatrix), P(TkOpts), P(TkTensor), P(TkMatrix),
                               P(ctypes.c_double)], ctypes.c_int),
            "tk_set_sm_reserve": ([vp, ctypes.c_int], ctypes.c_int),
            "tucker_rhkron_grad": ([vp, P(TkTensor), i64p, ctypes.c_int, P(TkMatrix), P(TkOpts), P(TkTensor),
                                    P(TkMatrix), P(ctypes.c_double), ctypes.c_double, P(TkTensor), P(TkMatrix),
                                    P(TkTensor)], ctypes.c_int),
            "tucker_rsthkron": ([vp, P(TkTensor), i64p, ctypes.c_int, P(TkMatrix), P(TkOpts), P(TkTensor),
                                 P(TkMatrix), P(ctypes.c_double)], ctypes.c_int),
            "tucker_rhkron_noreuse": ([vp, P(TkTensor), i64p, ctypes.c_int, P(TkMatrix), P(TkOpts), P(TkTensor),
                                 P(TkMatrix), P(ctypes.c_double)], ctypes.c_int),
            "tucker_rhkron_srht": ([vp, P(TkTensor), i64p, ctypes.c_int, P(TkMatrix), ctypes.c_uint64, P(TkOpts),
                                    P(TkTensor), P(TkMatrix), P(ctypes.c_double)], ctypes.c_int),
            "tucker_reconstruct": ([vp, P(TkTensor), P(TkMatrix), P(TkTensor)], ctypes.c_int),
            "tucker_sketch_slab": ([vp, P(TkTensor), ctypes.c_int64, ctypes.c_int64, P(TkMatrix), P(TkTensor)],
                                   ctypes.c_int),
            "tucker_orth_sketches": ([vp, ctypes.c_int, P(TkTensor), P(TkMatrix)], ctypes.c_int),
            "tucker_core_slab": ([vp, P(TkTensor), ctypes.c_int64, ctypes.c_int64, P(TkMatrix), P(TkTensor)],
                                 ctypes.c_int),
            "tucker_sthosvd": ([vp, P(TkTensor), P(TkMatrix), i64p, P(TkOpts), P(TkTensor), P(TkMatrix)],
                               ctypes.c_int),
            "tucker_loss_slab": ([vp, P(TkTensor), ctypes.c_int64, ctypes.c_int64, P(TkTensor), P(TkMatrix),
                                  P(ctypes.c_double)], ctypes.c_int),
            "tucker_loss": ([vp, P(TkTensor), P(TkTensor), P(TkMatrix), P(ctypes.c_double)], ctypes.c_int),
            "tucker_reconstruct_backward": ([vp, P(TkTensor), P(TkTensor), P(TkMatrix), ctypes.c_double, P(TkTensor),
                                             P(TkMatrix), P(TkTensor), vp], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


# ------------------------------------------------------------------ marshalling

def empty_f(dims: Sequence[int], dtype=torch.float32, device="cuda") -> torch.Tensor:
    """Uninitialised column-major tensor of shape ``dims``."""
    t = torch.empty(tuple(int(x) for x in reversed(dims)), dtype=dtype, device=device)
    return t.permute(*reversed(range(len(dims))))


def is_colmajor(t: torch.Tensor) -> bool:
    expect = 1
    for n, s in zip(t.shape, t.stride()):
        if n != 1 and s != expect:
            return False
        expect *= n
    return True


def _dt(t: torch.Tensor) -> int:
    if t.dtype not in _DT:
        raise TuckerError(3, f"unsupported dtype {t.dtype}")
    return _DT[t.dtype]


def _tensor(t: torch.Tensor, scale: float = 1.0) -> TkTensor:
    if not t.is_cuda:
        raise TuckerError(1, "tensor must be on a CUDA device")
    if t.dim() < 1 or t.dim() > TK_MAX_D:
        raise TuckerError(2, "tensor order out of range")
    if not is_colmajor(t):
        raise TuckerError(4, "tensor must be column-major (mode 1 fastest); use empty_f / synth.fortran")
    s = TkTensor()
    s.d = t.dim()
    for i, n in enumerate(t.shape):
        s.dims[i] = int(n)
    s.dtype = _dt(t)
    s.data = t.data_ptr() if t.numel() else None
    s.scale = float(scale)
    return s


def _matrix(m: torch.Tensor) -> TkMatrix:
    if not m.is_cuda:
        raise TuckerError(1, "matrix must be on a CUDA device")
    if m.dim() != 2:
        raise TuckerError(2, "matrix must be 2-D")
    rows, cols = m.shape
    if rows > 1 and cols > 0 and m.stride(0) != 1:
        raise TuckerError(4, "matrix must be column-major (stride(0) == 1)")
    ld = m.stride(1) if cols > 1 else max(1, rows)
    s = TkMatrix()
    s.rows, s.cols, s.ld = int(rows), int(cols), int(max(ld, rows, 1))
    s.dtype = _dt(m)
    s.data = m.data_ptr() if m.numel() else None
    return s


def _mats(ms: Sequence[torch.Tensor]):
    arr = (TkMatrix * len(ms))()
    for i, m in enumerate(ms):
        arr[i] = _matrix(m)
    return arr


def _colmajor_matrix(rows: int, cols: int, dtype, device) -> torch.Tensor:
    return torch.empty((cols, rows), dtype=dtype, device=device).t()


def _handle(device: torch.device) -> ctypes.c_void_p:
    """Handle bound to the current torch stream of ``device``.  Streams never
    share a handle, so calls queued on different streams never share workspace."""
    lib = load()
    idx = device.index if device.index is not None else torch.cuda.current_device()
    stream = torch.cuda.current_stream(idx).cuda_stream
    h = _handles.get((idx, stream))
    if h is None:
        with torch.cuda.device(idx):
            h = ctypes.c_void_p()
            st = lib.tk_create(ctypes.byref(h), ctypes.c_void_p(stream))
            if st != 0:
                raise TuckerError(st, "tk_create failed")
        _handles[(idx, stream)] = h
    return h


def _check(st: int, h) -> None:
    if st != 0:
        msg = load().tk_last_error(h) if h is not None else b""
        raise TuckerError(st, (msg or b"").decode())


def _opts(order=None, qr_method=0, refine=0, max_jacobi_sweeps=0, async_outputs=False):
    o = TkOpts()
    o.async_outputs = 1 if async_outputs else 0
    keep = None
    if order is not None:
        keep = (ctypes.c_int * len(order))(*[int(x) for x in order])
        o.mode_order = ctypes.cast(keep, ctypes.POINTER(ctypes.c_int))
    o.qr_method, o.refine, o.max_jacobi_sweeps = int(qr_method), int(refine), int(max_jacobi_sweeps)
    return o, keep


def _acc_dtype(X: torch.Tensor):
    return torch.float64 if X.dtype == torch.float64 else torch.float32


# ------------------------------------------------------------------ host planning

def tucker_subranks_reuse(r: Sequence[int], p: int) -> Tuple[List[int], List[int]]:
    d = len(r)
    rr = (ctypes.c_int64 * d)(*r)
    s = (ctypes.c_int64 * d)()
    w = (ctypes.c_int64 * d)()
    _check(load().tucker_subranks_reuse(d, rr, int(p), s, w), None)
    return list(s), list(w)


def tucker_subranks_matrix(r: Sequence[int], p: int, order: Optional[Sequence[int]] = None):
    d = len(r)
    rr = (ctypes.c_int64 * d)(*r)
    S = (ctypes.c_int64 * (d * d))()
    w = (ctypes.c_int64 * d)()
    ordp = (ctypes.c_int * d)(*order) if order is not None else None
    _check(load().tucker_subranks_matrix(d, rr, int(p), ordp, S, w), None)
    return [[S[j * d + k] for k in range(d)] for j in range(d)], list(w)


# ------------------------------------------------------------------ device entry points

def tk_sync_status(device=None) -> Tuple[int, List[int]]:
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    h = _handle(dev)
    info = (ctypes.c_int * TK_MAX_D)()
    st = load().tk_sync_status(h, info)
    return st, list(info)


def tk_selftest_bounded_wait(limit_ns: int, device=None) -> int:
    """Run the library's bounded-wait self-test on the handle of ``device``'s current stream: a warp
    waits, with the tcgen05 kernels' bounded wait, on an mbarrier nothing arrives at, and gives up
    after ``limit_ns``.  Returns the nanoseconds the wait lasted; the timeout is then reported by
    the next tk_sync_status (TK_ERR_TIMEOUT)."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    h = _handle(dev)
    out = ctypes.c_int64(0)
    st = load().tk_selftest_bounded_wait(h, int(limit_ns), ctypes.byref(out))
    if st != 0:
        raise TuckerError(st, load().tk_last_error(h).decode())
    return int(out.value)


def tk_launch_count(device=None) -> int:
    """Kernel launches queued through every handle of the device."""
    return int(sum(load().tk_launch_count(h) for h in _device_handles(device)))


def _device_handles(device):
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    _handle(dev)
    idx = dev.index if dev.index is not None else torch.cuda.current_device()
    return [h for (i, _), h in _handles.items() if i == idx]


def tk_graph_release(device=None) -> None:
    """Free the workspace blocks and host-output slots that CUDA graphs recorded from this device's
    handles; call it only when none of those graphs will be replayed again."""
    for h in _device_handles(device):
        _check(load().tk_graph_release(h), h)


class TuckerGraph:
    """``fn`` (a sequence of this module's calls, on the current stream or streams forked from it)
    recorded once into a CUDA graph and replayed.  ``fn`` runs ``warmup`` times first on a private
    stream, which sizes the workspaces of the handles it uses; its return value from the recording
    run is ``outputs`` (tensors and PendingScalar objects that every replay rewrites).  Host scalars
    need ``async_outputs=True``.  ``replay()`` queues the graph on the current stream."""

    def __init__(self, fn, warmup: int = 1):
        self.stream = torch.cuda.Stream()
        self.stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(self.stream):
            for _ in range(max(1, warmup)):
                fn()
        self.stream.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            self.outputs = fn()

    def replay(self) -> None:
        self.graph.replay()


def tk_set_sm_reserve(sms: int, device=None) -> None:
    """The streaming kernels of calls queued on the current stream of ``device`` leave ``sms`` SMs free
    for kernels of other streams (0: every SM); results do not depend on it."""
    dev = device if device is not None else torch.device("cuda", torch.cuda.current_device())
    h = _handle(dev)
    _check(load().tk_set_sm_reserve(h, int(sms)), h)


def tk_profile(enable: bool, device=None, only: Optional[str] = None) -> None:
    """Start (clearing old records) or stop per-kernel-class event timing on every handle of the device;
    ``only`` restricts the recording to classes whose name starts with it (each timed launch costs
    the host two event records)."""
    for h in _device_handles(device):
        if enable:
            _check(load().tk_profile_only(h, (only or "").encode()), h)
        _check(load().tk_profile(h, 1 if enable else 0), h)


def tk_profile_read(device=None) -> Dict[str, dict]:
    """Synchronise and return {class: {launches, ms, bytes, flops}} since tk_profile(True), summed over handles."""
    out: Dict[str, dict] = {}
    for h in _device_handles(device):
        buf = (TkProfEntry * 64)()
        n = load().tk_profile_read(h, buf, 64)
        if n < 0:
            raise TuckerError(6, "tk_profile_read failed")
        for i in range(min(n, 64)):
            e = out.setdefault(buf[i].name.decode(), dict(launches=0, ms=0.0, bytes=0.0, flops=0.0))
            e["launches"] += buf[i].launches
            e["ms"] += buf[i].ms
            e["bytes"] += buf[i].bytes
            e["flops"] += buf[i].flops
    return out


def tk_profile_trace(device=None) -> List[dict]:
    """Synchronise and return every launch recorded since tk_profile(True), one dict per launch
    (handle, stream, cls, start_us, end_us, bytes, flops), times after the latest tk_profile(True)
    on the device, sorted by start time."""
    out: List[dict] = []
    for hi, h in enumerate(_device_handles(device)):
        n = load().tk_profile_trace(h, None, 0)
        if n < 0:
            raise TuckerError(6, "tk_profile_trace failed")
        buf = (TkTraceEntry * max(n, 1))()
        n = load().tk_profile_trace(h, buf, n)
        if n < 0:
            raise TuckerError(6, "tk_profile_trace failed")
        out.extend(dict(handle=hi, stream=e.stream, cls=e.name.decode(), start_us=e.start_us, end_us=e.end_us,
                        bytes=e.bytes, flops=e.flops) for e in buf[:n])
    out.sort(key=lambda e: e["start_us"])
    return out


def tk_workspace_bytes(device=None) -> int:
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    return int(load().tk_workspace_bytes(_handle(dev)))


def tucker_sketch(X: torch.Tensor, Omega: Sequence[torch.Tensor], scale: float = 1.0) -> List[torch.Tensor]:
    """Y_n = X x_{j != n} Phi_j for every n (Omega_j = Phi_j^T, n_j x s_j)."""
    d = X.dim()
    s = [int(o.shape[1]) for o in Omega]
    acc = _acc_dtype(X)
    Y = [empty_f([X.shape[j] if j == n else s[j] for j in range(d)], acc, X.device) for n in range(d)]
    ys = (TkTensor * d)(*[_tensor(y) for y in Y])
    h = _handle(X.device)
    _check(load().tucker_sketch(h, ctypes.byref(_tensor(X, scale)), _mats(Omega), ys), h)
    return Y


def tucker_sketch_slab(X_slab: torch.Tensor, offset: int, n_last: int, Omega: Sequence[torch.Tensor],
                       scale: float = 1.0) -> List[torch.Tensor]:
    """Sketches of a slab of X along its last mode (rows offset .. offset + X_slab.shape[-1] - 1 of a mode of
    length n_last; Omega[-1] is the full n_last x s_d factor).  Y[n], n < d-1: the slab's partial sums of
    Y_n (SUM them over the slabs); Y[d-1]: the slab's rows of Y_d (gather them along the last mode)."""
    d = X_slab.dim()
    s = [int(o.shape[1]) for o in Omega]
    acc = _acc_dtype(X_slab)
    Y = [empty_f([X_slab.shape[j] if j == n else s[j] for j in range(d)], acc, X_slab.device) for n in range(d)]
    ys = (TkTensor * d)(*[_tensor(y) for y in Y])
    h = _handle(X_slab.device)
    _check(load().tucker_sketch_slab(h, ctypes.byref(_tensor(X_slab, scale)), int(offset), int(n_last),
                                     _mats(Omega), ys), h)
    return Y


def tucker_orth_sketches(Y: Sequence[torch.Tensor], out_dtype=torch.float64) -> List[torch.Tensor]:
    """Thin QR factor Q_n (n_n x k_n) of the mode-n unfolding of each sketch tensor Y[n] (Q = I when the sketch
    is at least as wide as the mode), as inside tucker_rhkron."""
    d = len(Y)
    Q = []
    for n, y in enumerate(Y):
        nn = int(y.shape[n])
        cols = y.numel() // max(1, nn)
        Q.append(_colmajor_matrix(nn, min(nn, cols), out_dtype, y.device))
    ys = (TkTensor * d)(*[_tensor(y) for y in Y])
    h = _handle(Y[0].device)
    _check(load().tucker_orth_sketches(h, d, ys, _mats(Q)), h)
    return Q


def tucker_core_slab(X_slab: torch.Tensor, offset: int, n_last: int, Q: Sequence[torch.Tensor], out_dtype=None,
                     scale: float = 1.0) -> torch.Tensor:
    """The slab's partial core X_slab x_{j<d} Q_j^T x_d Q_d[slab rows]^T (Q[-1] is the full n_last x k_d
    factor); SUM it over the slabs."""
    G = empty_f([int(q.shape[1]) for q in Q], out_dtype or _acc_dtype(X_slab), X_slab.device)
    h = _handle(X_slab.device)
    _check(load().tucker_core_slab(h, ctypes.byref(_tensor(X_slab, scale)), int(offset), int(n_last), _mats(Q),
                                   ctypes.byref(_tensor(G))), h)
    return G


def tucker_sthosvd(Ghat: torch.Tensor, Q: Sequence[torch.Tensor], r: Sequence[int], order=None, out_dtype=None):
    """STHOSVD of a given core to ranks r and U_j = Q_j V_j (steps 4-5 of Algorithm rHKron-re): (G, [U_j])."""
    d = Ghat.dim()
    dt = out_dtype or Ghat.dtype
    G = empty_f(list(r), dt, Ghat.device)
    U = [_colmajor_matrix(int(Q[j].shape[0]), int(r[j]), dt, Ghat.device) for j in range(d)]
    rr = (ctypes.c_int64 * d)(*[int(x) for x in r])
    o, keep = _opts(order)
    h = _handle(Ghat.device)
    _check(load().tucker_sthosvd(h, ctypes.byref(_tensor(Ghat)), _mats(Q), rr, ctypes.byref(o),
                                 ctypes.byref(_tensor(G)), _mats(U)), h)
    return G, U


def tucker_loss_slab(X_slab: torch.Tensor, offset: int, n_last: int, G: torch.Tensor, U: Sequence[torch.Tensor],
                     scale: float = 1.0) -> Tuple[float, float]:
    """(||X_slab - G x_{j<d} U_j x_d U_d[slab rows]||^2, ||X_slab||^2) (U[-1] is the full n_last x r_d factor);
    SUM both over the slabs."""
    out = (ctypes.c_double * 2)()
    h = _handle(X_slab.device)
    _check(load().tucker_loss_slab(h, ctypes.byref(_tensor(X_slab, scale)), int(offset), int(n_last),
                                   ctypes.byref(_tensor(G)), _mats(U), out), h)
    return float(out[0]), float(out[1])


def tucker_orth(Y: torch.Tensor, qr_method: int = 0, out_dtype=None) -> Tuple[torch.Tensor, int]:
    """Thin QR factor Q of a tall matrix Y (Q = I when cols >= rows); returns (Q, info)."""
    rows, cols = Y.shape
    k = min(rows, cols)
    Q = _colmajor_matrix(rows, k, out_dtype or Y.dtype, Y.device)
    info = ctypes.c_int(-1)
    o, keep = _opts(qr_method=qr_method)
    h = _handle(Y.device)
    _check(load().tucker_orth(h, ctypes.byref(_matrix(Y)), ctypes.byref(_matrix(Q)), ctypes.byref(info),
                              ctypes.byref(o)), h)
    return Q, info.value


def tucker_orth_noalloc(Y: torch.Tensor, out_dtype=None, Q: torch.Tensor | None = None,
                        read_info: bool = True) -> Tuple[torch.Tensor, Optional[int]]:
    """Thin QR like tucker_orth, computed without any device allocation by the
    library (a fixed internal scratch array; rows <= 4096, min(rows, cols) <= 64).
    For callers that cannot allocate device memory at the call site: memory
    owned by a pool or arena, or paths that must not take the implicit
    synchronisation of cudaMalloc / cudaFree.  Q (column-major, rows x
    min(rows, cols)) may be passed in so that nothing is allocated here either.
    Calls must not overlap on the GPU (they share the scratch).  Returns
    (Q, info); with read_info the method taken is read back, which synchronises
    the stream, else info is None and the call only queues work."""
    rows, cols = Y.shape
    if Q is None:
        Q = _colmajor_matrix(rows, min(rows, cols), out_dtype or Y.dtype, Y.device)
    info = ctypes.c_int(-1)
    with torch.cuda.device(Y.device):
        st = load().tucker_orth_noalloc(ctypes.c_void_p(torch.cuda.current_stream(Y.device).cuda_stream),
                                        ctypes.byref(_matrix(Y)), ctypes.byref(_matrix(Q)),
                                        ctypes.byref(info) if read_info else None)
    if st != 0:
        raise TuckerError(st, "tucker_orth_noalloc failed")
    return Q, (info.value if read_info else None)


def tucker_core(X: torch.Tensor, Q: Sequence[torch.Tensor], out_dtype=None, scale: float = 1.0) -> torch.Tensor:
    """Ghat = X x_1 Q_1^T ... x_d Q_d^T."""
    G = empty_f([int(q.shape[1]) for q in Q], out_dtype or _acc_dtype(X), X.device)
    h = _handle(X.device)
    _check(load().tucker_core(h, ctypes.byref(_tensor(X, scale)), _mats(Q), ctypes.byref(_tensor(G))), h)
    return G


class PendingScalar:
    """Host scalar written by a stream-ordered callback (``async_outputs=True``);
    ``value`` is valid once the stream has been synchronised."""

    def __init__(self):
        self._c = ctypes.c_double(float("nan"))

    @property
    def value(self) -> float:
        return self._c.value


def _decomp(fn, X, r, p, Omega_list, order, qr_method, refine, max_jacobi_sweeps, rel_err, out_dtype, scale,
            async_outputs=False):
    d = X.dim()
    dt = out_dtype or _acc_dtype(X)
    G = empty_f(list(r), dt, X.device)
    U = [_colmajor_matrix(int(X.shape[j]), int(r[j]), dt, X.device) for j in range(d)]
    rr = (ctypes.c_int64 * d)(*[int(x) for x in r])
    o, keep = _opts(order, qr_method, refine, max_jacobi_sweeps, async_outputs)
    pend = PendingScalar()
    h = _handle(X.device)
    st = fn(h, ctypes.byref(_tensor(X, scale)), rr, int(p), _mats(Omega_list), ctypes.byref(o),
            ctypes.byref(_tensor(G)), _mats(U), ctypes.byref(pend._c) if rel_err else None)
    _check(st, h)
    if not rel_err:
        return G, U, None
    if async_outputs:
        _pending.setdefault(h.value, collections.deque(maxlen=64)).append(pend)
        return G, U, pend
    return G, U, pend.value


def tucker_rhkron(X: torch.Tensor, r: Sequence[int], p: int, Omega: Sequence[torch.Tensor], *, order=None,
                  qr_method: int = 0, refine: int = 0, max_jacobi_sweeps: int = 0, rel_err: bool = True,
                  out_dtype=None, scale: float = 1.0, async_outputs: bool = False):
    """Algorithm rHKron-re.  Omega[j] = Phi_j^T (n_j x s_j).  Returns (G, [U_j], rel_err or None);
    with async_outputs the relative error is a PendingScalar and the call does not synchronise."""
    return _decomp(load().tucker_rhkron, X, r, p, list(Omega), order, qr_method, refine, max_jacobi_sweeps, rel_err,
                   out_dtype, scale, async_outputs)


def tucker_rhkron_grad(X: torch.Tensor, r: Sequence[int], p: int, Omega: Sequence[torch.Tensor],
                       grad_scale: float = 1.0, *, need_dG: bool = True, need_dU: bool = True, need_dX: bool = True,
                       order=None, qr_method: int = 0, refine: int = 0, max_jacobi_sweeps: int = 0,
                       rel_err: bool = True, out_dtype=None, scale: float = 1.0, async_outputs: bool = False):
    """Algorithm rHKron-re and the gradient of grad_scale * ||X - G x_j U_j||^2 at its result in one call
    (the passes over X shared).  Returns (G, [U_j], rel_err or None, dG, [dU_j], dX), gradients None when
    not requested; rel_err as tucker_rhkron."""
    d = X.dim()
    dt = out_dtype or _acc_dtype(X)
    G = empty_f(list(r), dt, X.device)
    U = [_colmajor_matrix(int(X.shape[j]), int(r[j]), dt, X.device) for j in range(d)]
    dG = empty_f(list(r), dt, X.device) if need_dG else None
    dU = [_colmajor_matrix(int(X.shape[j]), int(r[j]), dt, X.device) for j in range(d)] if need_dU else None
    dX = empty_f(list(X.shape), X.dtype, X.device) if need_dX else None
    rr = (ctypes.c_int64 * d)(*[int(x) for x in r])
    o, keep = _opts(order, qr_method, refine, max_jacobi_sweeps, async_outputs)
    pend = PendingScalar()
    h = _handle(X.device)
    st = load().tucker_rhkron_grad(h, ctypes.byref(_tensor(X, scale)), rr, int(p), _mats(list(Omega)),
                                   ctypes.byref(o), ctypes.byref(_tensor(G)), _mats(U),
                                   ctypes.byref(pend._c) if rel_err else None, float(grad_scale),
                                   ctypes.byref(_tensor(dG)) if need_dG else None, _mats(dU) if need_dU else None,
                                   ctypes.byref(_tensor(dX)) if need_dX else None)
    _check(st, h)
    if not rel_err:
        err = None
    elif async_outputs:
        _pending.setdefault(h.value, collections.deque(maxlen=64)).append(pend)
        err = pend
    else:
        err = pend.value
    return G, U, err, dG, dU, dX


def tucker_rsthkron(X: torch.Tensor, r: Sequence[int], p: int, Omega: Dict[Tuple[int, int], torch.Tensor], *,
                    order=None, qr_method: int = 0, refine: int = 0, max_jacobi_sweeps: int = 0,
                    rel_err: bool = True, out_dtype=None, scale: float = 1.0, async_outputs: bool = False):
    """Algorithm rSTHKron.  Omega[(j, k)] = Phi_{j,k}^T sized to mode k's current size."""
    d = X.dim()
    dummy = torch.zeros((1, 1), dtype=next(iter(Omega.values())).dtype, device=X.device)
    lst = [Omega.get((j, k), dummy) if j != k else dummy for j in range(d) for k in range(d)]
    return _decomp(load().tucker_rsthkron, X, r, p, lst, order, qr_method, refine, max_jacobi_sweeps, rel_err,
                   out_dtype, scale, async_outputs)


def tucker_rhkron_srht(X: torch.Tensor, r: Sequence[int], p: int, H: Sequence[torch.Tensor], seed: int, *,
                       order=None, qr_method: int = 0, refine: int = 0, max_jacobi_sweeps: int = 0,
                       rel_err: bool = True, out_dtype=None, scale: float = 1.0, async_outputs: bool = False):
    """rHKron-re with the Kronecker-SRHT sketch (Section 5): H[j] = n_j x s_j sampled, scaled
    Walsh-Hadamard columns; the Rademacher diagonals D_n come from the counter-based generator
    tk_rademacher(seed, n, c) of the C header."""
    lib = load()
    sd = ctypes.c_uint64(int(seed) & 0xFFFFFFFFFFFFFFFF)

    def fn(h, x, rr, pp, om, o, g, u, e):
        return lib.tucker_rhkron_srht(h, x, rr, pp, om, sd, o, g, u, e)

    return _decomp(fn, X, r, p, list(H), order, qr_method, refine, max_jacobi_sweeps, rel_err, out_dtype, scale,
                   async_outputs)


def tk_philox4x32(seed: int, stream: int, offset: int, nblocks: int, device) -> torch.Tensor:
    """Philox4x32-10 blocks offset .. offset + nblocks - 1 of ``stream`` (the C header's counter and key
    layout) as an (nblocks, 4) int32 tensor holding the uint32 words' bits."""
    out = torch.empty((int(nblocks), 4), dtype=torch.int32, device=device)
    h = _handle(out.device)
    _check(load().tk_philox4x32(h, ctypes.c_uint64(int(seed) & 0xFFFFFFFFFFFFFFFF), ctypes.c_uint32(int(stream)),
                                ctypes.c_uint64(int(offset)), int(nblocks), out.data_ptr() if nblocks else None), h)
    return out


def tucker_gaussian_factor(rows: int, cols: int, seed: int, stream: int, dtype=torch.float32,
                           device="cuda") -> torch.Tensor:
    """A rows x cols column-major matrix of N(0, 1) draws from the device generator (Philox4x32-10 and
    Box-Muller; the C header defines the element-to-draw map)."""
    m = _colmajor_matrix(int(rows), int(cols), dtype, torch.device(device))
    h = _handle(m.device)
    _check(load().tucker_gaussian_factor(h, ctypes.c_uint64(int(seed) & 0xFFFFFFFFFFFFFFFF),
                                         ctypes.c_uint32(int(stream)), ctypes.byref(_matrix(m))), h)
    return m


def _draw_factors(shapes, streams, seed: int, dtype, device) -> List[torch.Tensor]:
    """One launch drawing a factor of each shape (rows, cols) from the given streams."""
    dev = torch.device(device)
    ms = [_colmajor_matrix(int(r), int(c), dtype, dev) for r, c in shapes]
    if not ms:
        return ms
    st = (ctypes.c_uint32 * len(ms))(*[int(x) for x in streams])
    h = _handle(ms[0].device)
    _check(load().tucker_gaussian_factors(h, ctypes.c_uint64(int(seed) & 0xFFFFFFFFFFFFFFFF), len(ms), st,
                                          _mats(ms)), h)
    return ms


def gaussian_factors(dims: Sequence[int], s: Sequence[int], seed: int, dtype=torch.float32, device="cuda"):
    """The sketch factors Omega_j = Phi_j^T (n_j x s_j) of Algorithm rHKron-re, drawn on the device in one
    launch: mode j from stream j."""
    return _draw_factors(list(zip(dims, s)), range(len(dims)), seed, dtype, device)


def tucker_gaussian_factors(shapes: Sequence[Tuple[int, int]], seed: int, streams: Sequence[int],
                            dtype=torch.float32, device="cuda") -> List[torch.Tensor]:
    """Several column-major factors of N(0, 1) draws in one launch; factor f has shape shapes[f] and
    the draws of stream streams[f] (the same values tucker_gaussian_factor gives)."""
    if len(shapes) != len(streams):
        raise TuckerError(1, "one stream per factor")
    return _draw_factors(list(shapes), list(streams), seed, dtype, device)


def rsthkron_factor_plan(dims: Sequence[int], S, kdims: Sequence[int], order: Sequence[int]):
    """Host-side plan of Algorithm rSTHKron's factors: for the mode j processed at position t,
    Omega_{j,k} is (current size of mode k) x s_{j,k} (k_k for modes processed earlier, n_k
    otherwise), drawn from stream 8 j + k.  Returns (keys (j, k), shapes, streams) in draw order."""
    d = len(dims)
    keys, shapes, streams, done = [], [], [], set()
    for j in order:
        for k in range(d):
            if k == j:
                continue
            keys.append((j, k))
            shapes.append((int(kdims[k]) if k in done else int(dims[k]), int(S[j][k])))
            streams.append(8 * j + k)
        done.add(j)
    return keys, shapes, streams


def gaussian_factors_matrix(dims: Sequence[int], S, kdims: Sequence[int], order: Sequence[int], seed: int,
                            dtype=torch.float32, device="cuda") -> Dict[Tuple[int, int], torch.Tensor]:
    """The sketch factors Omega_{j,k} = Phi_{j,k}^T of Algorithm rSTHKron, drawn on the device from stream
    8 j + k: for the mode j processed at position t, Phi_{j,k} is s_{j,k} x (current size of mode k),
    k_k for modes processed earlier and n_k otherwise.  S: d x d subranks (row j), as
    tucker_subranks_matrix returns them."""
    keys, shapes, streams = rsthkron_factor_plan(dims, S, kdims, order)
    ms = _draw_factors(shapes, streams, seed, dtype, device)
    return dict(zip(keys, ms))


def tucker_rhkron_noreuse(X: torch.Tensor, r: Sequence[int], p: int, Omega: Dict[Tuple[int, int], torch.Tensor], *,
                          order=None, qr_method: int = 0, refine: int = 0, max_jacobi_sweeps: int = 0,
                          rel_err: bool = True, out_dtype=None, scale: float = 1.0, async_outputs: bool = False):
    """Appendix Algorithm rHKron (no factor reuse).  Omega[(n, j)] = Phi_{n,j}^T (n_j x s_{n,j})."""
    d = X.dim()
    dummy = torch.zeros((1, 1), dtype=next(iter(Omega.values())).dtype, device=X.device)
    lst = [Omega.get((n, j), dummy) if n != j else dummy for n in range(d) for j in range(d)]
    return _decomp(load().tucker_rhkron_noreuse, X, r, p, lst, order, qr_method, refine, max_jacobi_sweeps, rel_err,
                   out_dtype, scale, async_outputs)


def tucker_reconstruct(G: torch.Tensor, U: Sequence[torch.Tensor], out_dtype=None) -> torch.Tensor:
    """Xhat = G x_1 U_1 ... x_d U_d."""
    Xh = empty_f([int(u.shape[0]) for u in U], out_dtype or G.dtype, G.device)
    h = _handle(G.device)
    _check(load().tucker_reconstruct(h, ctypes.byref(_tensor(G)), _mats(U), ctypes.byref(_tensor(Xh))), h)
    return Xh


def tucker_loss(X: torch.Tensor, G: torch.Tensor, U: Sequence[torch.Tensor], scale: float = 1.0) -> float:
    """||X - G x_j U_j||^2 (host float; synchronises)."""
    out = ctypes.c_double()
    h = _handle(X.device)
    _check(load().tucker_loss(h, ctypes.byref(_tensor(X, scale)), ctypes.byref(_tensor(G)), _mats(U),
                              ctypes.byref(out)), h)
    return out.value


def tucker_reconstruct_backward(X: torch.Tensor, G: torch.Tensor, U: Sequence[torch.Tensor], grad_scale: float = 1.0,
                                need_dX: bool = True, scale: float = 1.0, need_dG: bool = True, need_dU: bool = True,
                                norms2: Optional[torch.Tensor] = None):
    """Gradients of grad_scale * ||X - G x_j U_j||^2: returns (dG, [dU_j], dX), each None when not requested.
    ``norms2``: an optional float64 device tensor of 2 elements that receives ||X - G x_j U_j||^2 and ||X||^2
    from the residual pass (stream-ordered, no synchronisation)."""
    dG = empty_f(list(G.shape), G.dtype, G.device) if need_dG else None
    dU = [_colmajor_matrix(int(u.shape[0]), int(u.shape[1]), u.dtype, u.device) for u in U] if need_dU else None
    dX = empty_f(list(X.shape), X.dtype, X.device) if need_dX else None
    if norms2 is not None and (norms2.dtype != torch.float64 or norms2.numel() < 2 or not norms2.is_contiguous()
                               or norms2.device != X.device):
        raise TuckerError(1, "norms2 must be a contiguous float64 tensor of 2 elements on X's device")
    h = _handle(X.device)
    _check(load().tucker_reconstruct_backward(h, ctypes.byref(_tensor(X, scale)), ctypes.byref(_tensor(G)), _mats(U),
                                              float(grad_scale), ctypes.byref(_tensor(dG)) if need_dG else None,
                                              _mats(dU) if need_dU else None,
                                              ctypes.byref(_tensor(dX)) if need_dX else None,
                                              norms2.data_ptr() if norms2 is not None else None), h)
    return dG, dU, dX


class TuckerLoss(torch.autograd.Function):
    """loss = ||X - G x_1 U_1 ... x_d U_d||^2 with the library's adjoint multi-TTM backward.

    ``TuckerLoss.apply(X, G, U_1, ..., U_d)``.  Nothing is saved besides the
    inputs: the backward recomputes the residual and its sketches.
    """

    @staticmethod
    def forward(ctx, X, G, *U):
        ctx.save_for_backward(X, G, *U)
        return torch.tensor(tucker_loss(X, G, list(U)), dtype=torch.float64, device=X.device)

    @staticmethod
    def backward(ctx, gout):
        X, G, *U = ctx.saved_tensors
        scale = float(gout.item())
        need_u = any(ctx.needs_input_grad[2:])
        dG, dU, dX = tucker_reconstruct_backward(X, G, U, scale, need_dX=ctx.needs_input_grad[0],
                                                 need_dG=ctx.needs_input_grad[1], need_dU=need_u)
        return (dX, dG, *(dU if dU is not None else [None] * len(U)))
