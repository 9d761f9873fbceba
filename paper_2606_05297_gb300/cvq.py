"""Python binding of libcvq.so (include/cvq.h): argument marshalling only.

Every computation runs in the CUDA kernels behind the C ABI.  PyTorch provides
device memory (complex128 state tensors, workspaces) and streams.  There is no
fallback: if the native library is missing or fails to load, importing the
first function raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from .workloads import Model, Op

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcvq.so")

OP_CODES = {"hop": 0, "sq2": 1, "sq1": 2, "pairhop": 3, "kerr": 4, "nn1": 5, "rot": 6, "xkerr": 7}
KIND_CODES = {"bh": 0, "bkc": 1}


class CvqError(RuntimeError):
    pass


class _Model(C.Structure):
    _fields_ = [("kind", C.c_int), ("L", C.c_int), ("N", C.c_int), ("d", C.c_int), ("parity", C.c_int),
                ("periodic", C.c_int), ("hop", C.POINTER(C.c_double)), ("pair", C.POINTER(C.c_double)),
                ("onsite_nn1", C.POINTER(C.c_double)), ("onsite_n2", C.POINTER(C.c_double)),
                ("onsite_n", C.POINTER(C.c_double))]


class _Op(C.Structure):
    _fields_ = [("type", C.c_int), ("i", C.c_int), ("j", C.c_int), ("phase", C.c_int)]


_lib = None


def lib():
    """Load libcvq.so (built in-tree by paper_2606_05297_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise CvqError(f"native library {LIB_PATH} is missing: run paper_2606_05297_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, sz, i64 = C.c_void_p, C.c_size_t, C.c_int64
        L.cvq_last_error.restype = C.c_char_p
        L.cvq_init_sector.argtypes = [C.POINTER(_Model), C.POINTER(vp)]
        L.cvq_sector_dim.argtypes = [vp, C.POINTER(i64)]
        L.cvq_sector_index.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(i64)]
        L.cvq_destroy_sector.argtypes = [vp]
        L.cvq_destroy_sector.restype = None
        L.cvq_set_pool.argtypes = [vp, C.POINTER(_Op), C.c_int, C.POINTER(vp)]
        L.cvq_destroy_pool.argtypes = [vp]
        L.cvq_destroy_pool.restype = None
        L.cvq_workspace_bytes.argtypes = [vp, vp, C.c_int, C.POINTER(sz)]
        L.cvq_apply_H.argtypes = [vp, vp, vp, vp, vp, sz, vp]
        L.cvq_screen_pool.argtypes = [vp, vp, vp, C.POINTER(C.c_int), C.c_int, vp, vp, sz, vp]
        L.cvq_apply_ansatz.argtypes = [vp, vp, C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_int, vp, vp, vp, sz, vp]
        L.cvq_energy_and_grad.argtypes = [vp, vp, C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_int, vp, vp, vp, vp,
                                          sz, vp]
        L.cvq_lanczos_step.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
        L.cvq_screen_subset_noalloc.argtypes = [vp, vp, vp, C.POINTER(C.c_int), C.c_int, vp, vp]
        dp = C.POINTER(C.c_double)
        L.cvq_op_cost.argtypes = [vp, vp, C.c_int, dp, dp, dp, dp]
        _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != 0:
        msg = lib().cvq_last_error().decode(errors="replace")
        raise CvqError(f"{what} failed (code {rc}): {msg}")


def _dbl(vals, n):
    a = np.zeros(max(n, 1), dtype=np.float64)
    if vals:
        a[:len(vals)] = vals
    return a


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t) -> C.c_void_p:
    return C.c_void_p(t.data_ptr())


_DTYPE_NAMES = {"c128": "complex128", "f64": "float64", "f32": "float32", "i32": "int32", "u8": "uint8"}


def _dev(t, kind: str, n: int, what: str) -> C.c_void_p:
    """Device pointer of tensor t after checking that the kernels may use it:
    a contiguous CUDA tensor of dtype `kind` holding at least n elements.
    Anything else would let a kernel read or write past the buffer."""
    import torch
    want = getattr(torch, _DTYPE_NAMES[kind])
    if not isinstance(t, torch.Tensor):
        raise ValueError(f"{what}: expected a torch tensor, got {type(t).__name__}")
    if t.dtype != want:
        raise ValueError(f"{what}: dtype {t.dtype}, expected {want}")
    if not t.is_contiguous():
        raise ValueError(f"{what}: must be contiguous")
    if t.numel() < n:
        raise ValueError(f"{what}: {t.numel()} elements, need at least {n}")
    if not t.is_cuda:
        raise ValueError(f"{what}: must be a CUDA tensor")
    return C.c_void_p(t.data_ptr())


class Sector:
    """cvq_sector: the symmetry sector of a lattice model on the current device."""

    def __init__(self, model: Model):
        self.model = model
        nb = model.L if model.periodic else model.L - 1
        self._arrs = [_dbl(model.hop, nb), _dbl(model.pair, nb), _dbl(model.nn1, model.L), _dbl(model.n2, model.L),
                      _dbl(model.n1, model.L)]
        P = [a.ctypes.data_as(C.POINTER(C.c_double)) for a in self._arrs]
        m = _Model(KIND_CODES[model.kind], model.L, model.N, model.d, model.parity, int(bool(model.periodic)), *P)
        h = C.c_void_p()
        _check(lib().cvq_init_sector(C.byref(m), C.byref(h)), "cvq_init_sector")
        self.h = h
        dim = C.c_int64()
        _check(lib().cvq_sector_dim(h, C.byref(dim)), "cvq_sector_dim")
        self.dim = int(dim.value)
        self.L = model.L

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.cvq_destroy_sector(self.h)
            self.h = None

    def index(self, occ: Sequence[int]) -> int:
        a = (C.c_int * self.L)(*[int(v) for v in occ])
        out = C.c_int64()
        _check(lib().cvq_sector_index(self.h, a, C.byref(out)), "cvq_sector_index")
        return int(out.value)

    def basis_state(self, occ: Sequence[int], device="cuda"):
        import torch
        v = torch.zeros(self.dim, dtype=torch.complex128, device=device)
        v[self.index(occ)] = 1.0
        return v

    def workspace(self, pool: Optional["Pool"] = None, n_max: int = 0):
        import torch
        b = C.c_size_t()
        _check(lib().cvq_workspace_bytes(self.h, pool.h if pool is not None else None, int(n_max), C.byref(b)),
               "cvq_workspace_bytes")
        return torch.empty(int(b.value), dtype=torch.uint8, device="cuda")


class Pool:
    """cvq_pool: operator pool generators with their block eigendecompositions."""

    def __init__(self, sector: Sector, ops: Sequence[Op]):
        self.sector = sector
        self.ops = list(ops)
        K = len(self.ops)
        arr = (_Op * max(K, 1))(*[_Op(OP_CODES[o.type], o.i, o.j if o.j is not None else -1, o.phase)
                                  for o in self.ops])
        h = C.c_void_p()
        _check(lib().cvq_set_pool(sector.h, arr, K, C.byref(h)), "cvq_set_pool")
        self.h = h
        self.K = K

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.cvq_destroy_pool(self.h)
            self.h = None


def _ws(sector, pool, n, ws):
    if ws is None:
        ws = sector.workspace(pool, n)
    return ws, C.c_size_t(ws.numel())


def apply_H(sector: Sector, psi, sigma=None, energy=None, ws=None, stream=None):
    """sigma = H psi; energy (optional 1-element float64 device tensor) = Re <psi|H|psi>."""
    import torch
    if sigma is None:
        sigma = torch.empty_like(psi)
    ws, wsb = _ws(sector, None, 0, ws)
    d = sector.dim
    _check(lib().cvq_apply_H(sector.h, _dev(psi, "c128", d, "psi"), _dev(sigma, "c128", d, "sigma"),
                             _dev(energy, "f64", 1, "energy") if energy is not None else None,
                             _dev(ws, "u8", 0, "workspace"), wsb, _stream(stream)), "cvq_apply_H")
    return sigma


def screen_pool(sector: Sector, pool: Pool, psi, subset=None, out=None, ws=None, stream=None):
    """Eq. (grad) gradients of the pool (or of the pool indices in subset)."""
    import torch
    n = pool.K if subset is None else len(subset)
    if out is None:
        out = torch.empty(max(n, 1), dtype=torch.float64, device=psi.device)
    ws, wsb = _ws(sector, pool, 0, ws)
    if subset is None:
        sp, ns = None, 0
    else:
        sa = (C.c_int * max(n, 1))(*[int(k) for k in subset])
        sp, ns = sa, n
    _check(lib().cvq_screen_pool(sector.h, pool.h, _dev(psi, "c128", sector.dim, "psi"), sp, ns,
                                 _dev(out, "f64", n, "out"), _dev(ws, "u8", 0, "workspace"), wsb, _stream(stream)),
           "cvq_screen_pool")
    return out[:n]


def _ids_theta(op_ids, theta):
    n = len(op_ids)
    ids = (C.c_int * max(n, 1))(*[int(k) for k in op_ids])
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(-1))
    if th.size != n:
        raise ValueError("op_ids and theta differ in length")
    return n, ids, th


def apply_ansatz(sector: Sector, pool: Pool, op_ids, theta, psi0, out=None, ws=None, stream=None):
    """psi_out = prod_k exp(theta_k A_{op_ids[k]}) psi0."""
    import torch
    n, ids, th = _ids_theta(op_ids, theta)
    if out is None:
        out = torch.empty_like(psi0)
    ws, wsb = _ws(sector, pool, n, ws)
    d = sector.dim
    _check(lib().cvq_apply_ansatz(sector.h, pool.h, ids, th.ctypes.data_as(C.POINTER(C.c_double)), n,
                                  _dev(psi0, "c128", d, "psi0"), _dev(out, "c128", d, "out"),
                                  _dev(ws, "u8", 0, "workspace"), wsb, _stream(stream)), "cvq_apply_ansatz")
    return out


def energy_and_grad(sector: Sector, pool: Pool, op_ids, theta, psi0, E=None, grad=None, ws=None, stream=None):
    """Energy and adjoint gradient of the ansatz; returns device tensors (E[1], grad[n])."""
    import torch
    n, ids, th = _ids_theta(op_ids, theta)
    if E is None:
        E = torch.empty(1, dtype=torch.float64, device=psi0.device)
    if grad is None:
        grad = torch.empty(max(n, 1), dtype=torch.float64, device=psi0.device)
    ws, wsb = _ws(sector, pool, n, ws)
    _check(lib().cvq_energy_and_grad(sector.h, pool.h, ids, th.ctypes.data_as(C.POINTER(C.c_double)), n,
                                     _dev(psi0, "c128", sector.dim, "psi0"), _dev(E, "f64", 1, "E"),
                                     _dev(grad, "f64", n, "grad"), _dev(ws, "u8", 0, "workspace"), wsb,
                                     _stream(stream)), "cvq_energy_and_grad")
    return E, grad[:n]


def lanczos_step(sector: Sector, v_prev, v, w, v_next, alpha, beta_prev, beta, ws=None, stream=None):
    """w <- w - alpha v - beta_prev v_prev; beta = ||w||; v_next = w / beta (all on the device)."""
    ws, wsb = _ws(sector, None, 0, ws)
    d = sector.dim
    _check(lib().cvq_lanczos_step(sector.h, _dev(v_prev, "c128", d, "v_prev"), _dev(v, "c128", d, "v"),
                                  _dev(w, "c128", d, "w"), _dev(v_next, "c128", d, "v_next"),
                                  _dev(alpha, "f64", 1, "alpha"), _dev(beta_prev, "f64", 1, "beta_prev"),
                                  _dev(beta, "f64", 1, "beta"), _dev(ws, "u8", 0, "workspace"), wsb,
                                  _stream(stream)), "cvq_lanczos_step")


def op_cost(sector: Sector, pool: Pool, op: int):
    """Algorithmic (fwd_bytes, fwd_flops, adj_bytes, adj_flops) of one pool element's gate."""
    v = [C.c_double() for _ in range(4)]
    _check(lib().cvq_op_cost(sector.h, pool.h, int(op), *[C.byref(x) for x in v]), "cvq_op_cost")
    return tuple(x.value for x in v)


class _KStat(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("ms", C.c_double), ("bytes", C.c_double),
                ("flops", C.c_double)]


def profile_sample(every: int):
    L = lib()
    L.cvq_profile_sample.argtypes = [C.c_int]
    _check(L.cvq_profile_sample(int(every)), "cvq_profile_sample")


def profile_start(capacity: int = 1 << 20):
    """Time every later launch of this library with CUDA events on its stream."""
    L = lib()
    L.cvq_profile_start.argtypes = [C.c_int]
    _check(L.cvq_profile_start(int(capacity)), "cvq_profile_start")


def profile_stop():
    """Stop timing; returns {kernel: dict(launches, ms, bytes, flops)}."""
    L = lib()
    L.cvq_profile_stop.argtypes = [C.POINTER(_KStat), C.c_int, C.POINTER(C.c_int)]
    out = (_KStat * 32)()
    n = C.c_int()
    _check(L.cvq_profile_stop(out, 32, C.byref(n)), "cvq_profile_stop")
    return {out[k].name.decode(): dict(launches=int(out[k].launches), ms=out[k].ms, bytes=out[k].bytes,
                                       flops=out[k].flops) for k in range(n.value)}


def screen_subset_noalloc(sector: Sector, pool: Pool, psi, subset, out=None, stream=None):
    """Eq. (grad) gradients of at most 64 pool elements without any workspace
    or device allocation inside the call (cvq_screen_subset_noalloc): for
    callers that cannot allocate at that point (latency-critical loops, hosts
    whose allocator owns all device memory).  Such callers pass a preallocated
    `out`; calls that overlap on the GPU race on the library's shared array."""
    import torch
    n = len(subset)
    if out is None:
        out = torch.empty(max(n, 1), dtype=torch.float64, device=psi.device)
    sa = (C.c_int * max(n, 1))(*[int(k) for k in subset])
    _check(lib().cvq_screen_subset_noalloc(sector.h, pool.h, _dev(psi, "c128", sector.dim, "psi"), sa, n,
                                           _dev(out, "f64", n, "out"), _stream(stream)),
           "cvq_screen_subset_noalloc")
    return out[:n]


def features(sector: Sector, psi, pairs=(), out=None, stream=None):
    """<n_r>, <n_r^2> per mode and Re/Im <a_i^dag a_j> per (i, j) in pairs (device float64 vector
    of length 2L + 2 len(pairs))."""
    import torch
    L = sector.L
    npairs = len(pairs)
    lib().cvq_features_workspace_bytes.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_size_t)]
    lib().cvq_features.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_int,
                                   C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p]
    b = C.c_size_t()
    _check(lib().cvq_features_workspace_bytes(sector.h, npairs, C.byref(b)), "cvq_features_workspace_bytes")
    ws = torch.empty(int(b.value), dtype=torch.uint8, device=psi.device)
    if out is None:
        out = torch.empty(2 * L + 2 * npairs, dtype=torch.float64, device=psi.device)
    pi = (C.c_int * max(npairs, 1))(*[int(p[0]) for p in pairs])
    pj = (C.c_int * max(npairs, 1))(*[int(p[1]) for p in pairs])
    _check(lib().cvq_features(sector.h, _dev(psi, "c128", sector.dim, "psi"), pi, pj, npairs,
                              _dev(out, "f64", 2 * L + 2 * npairs, "out"), _ptr(ws), C.c_size_t(ws.numel()),
                              _stream(stream)), "cvq_features")
    return out


MLP_IN, MLP_HIDDEN, MLP_NPARAM = 32, 256, 74497


def _mlp_sigs(L):
    vp, f32p = C.c_void_p, C.POINTER(C.c_float)
    L.cvq_mlp_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_uint64, C.POINTER(vp)]
    L.cvq_mlp_destroy.argtypes = [vp]
    L.cvq_mlp_destroy.restype = None
    L.cvq_mlp_forward.argtypes = [vp, vp, C.c_int, vp, vp]
    L.cvq_mlp_backward.argtypes = [vp, vp, C.c_int, vp, vp]
    L.cvq_mlp_listwise_loss.argtypes = [vp, vp, vp, C.c_int, vp, vp, vp]
    L.cvq_mlp_adam_step.argtypes = [vp, C.c_float, C.c_int, vp]
    L.cvq_mlp_get.argtypes = [vp, C.c_int, f32p, C.c_size_t]
    L.cvq_mlp_set.argtypes = [vp, f32p, C.c_size_t]
    return L


class Scorer:
    """The proposal scorer (32 -> 256 -> 256 -> 1, bf16 weights, fp32 sums) on the current device.
    Inputs and outputs are device float32 tensors."""

    def __init__(self, max_rows: int, seed: int = 0):
        L = _mlp_sigs(lib())
        h = C.c_void_p()
        _check(L.cvq_mlp_create(MLP_IN, MLP_HIDDEN, int(max_rows), int(seed) & (2 ** 64 - 1), C.byref(h)),
               "cvq_mlp_create")
        self.h, self.max_rows, self.t = h, int(max_rows), 0

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.cvq_mlp_destroy(self.h)
            self.h = None

    def forward(self, X, out=None, stream=None):
        import torch
        if X.dim() != 2 or X.shape[-1] != MLP_IN:
            raise ValueError(f"X: expected shape (rows, {MLP_IN}), got {tuple(X.shape)}")
        rows = int(X.shape[0])
        if out is None:
            out = torch.empty(rows, dtype=torch.float32, device=X.device)
        _check(lib().cvq_mlp_forward(self.h, _dev(X, "f32", rows * MLP_IN, "X"), rows, _dev(out, "f32", rows, "out"),
                                     _stream(stream)), "cvq_mlp_forward")
        return out

    def backward(self, X, dscores, stream=None):
        if X.dim() != 2 or X.shape[-1] != MLP_IN:
            raise ValueError(f"X: expected shape (rows, {MLP_IN}), got {tuple(X.shape)}")
        rows = int(X.shape[0])
        _check(lib().cvq_mlp_backward(self.h, _dev(X, "f32", rows * MLP_IN, "X"), rows,
                                      _dev(dscores, "f32", rows, "dscores"), _stream(stream)), "cvq_mlp_backward")

    def adam_step(self, lr: float, stream=None):
        self.t += 1
        _check(lib().cvq_mlp_adam_step(self.h, C.c_float(lr), self.t, _stream(stream)), "cvq_mlp_adam_step")

    def get(self, which: int = 0):
        buf = np.empty(MLP_NPARAM, dtype=np.float32)
        _check(lib().cvq_mlp_get(self.h, which, buf.ctypes.data_as(C.POINTER(C.c_float)), buf.size), "cvq_mlp_get")
        return buf

    def set(self, params):
        buf = np.ascontiguousarray(params, dtype=np.float32)
        _check(lib().cvq_mlp_set(self.h, buf.ctypes.data_as(C.POINTER(C.c_float)), buf.size), "cvq_mlp_set")
        self.t = 0


def listwise_loss(scores, targets, list_off, dscores=None, loss=None, stream=None):
    """Per-list softmax cross-entropy and d loss / d scores; list_off is a device int32 tensor of nlists + 1
    offsets."""
    import torch
    L = _mlp_sigs(lib())
    n = int(list_off.numel()) - 1
    if dscores is None:
        dscores = torch.empty_like(scores)
    if loss is None:
        loss = torch.empty(max(n, 0), dtype=torch.float32, device=scores.device)
    rows = int(scores.numel())
    _check(L.cvq_mlp_listwise_loss(_dev(scores, "f32", rows, "scores"), _dev(targets, "f32", rows, "targets"),
                                   _dev(list_off, "i32", n + 1, "list_off"), n, _dev(dscores, "f32", rows, "dscores"),
                                   _dev(loss, "f32", max(n, 0), "loss"), _stream(stream)), "cvq_mlp_listwise_loss")
    return loss, dscores


def _batch_sigs(L):
    vp, ip = C.c_void_p, C.POINTER(C.c_int)
    L.cvq_batch_create.argtypes = [C.POINTER(vp), C.POINTER(vp), C.c_int, C.c_int, C.POINTER(vp)]
    L.cvq_batch_destroy.argtypes = [vp]
    L.cvq_batch_destroy.restype = None
    L.cvq_batch_set_ansatz.argtypes = [vp, ip, ip, C.POINTER(vp)]
    L.cvq_batch_set_schedule.argtypes = [vp, C.c_int64, C.c_int]
    L.cvq_batch_energy_and_grad.argtypes = [vp, vp, vp, vp, vp]
    L.cvq_batch_info.argtypes = [vp, ip, ip, ip, C.POINTER(C.c_int64)]
    L.cvq_batch_set_active.argtypes = [vp, ip, vp]
    L.cvq_batch_screen.argtypes = [vp, vp, ip, ip, vp, vp]
    return L


class Batch:
    """Batched energy and adjoint gradient of many instances (cvq_batch_*).
    The sectors, pools and reference states must stay alive with the batch."""

    def __init__(self, sectors: Sequence[Sector], pools: Sequence[Pool], n_max: int):
        import torch
        L = _batch_sigs(lib())
        n = len(sectors)
        self._keep = (list(sectors), list(pools))
        sa = (C.c_void_p * n)(*[s.h.value if isinstance(s.h, C.c_void_p) else s.h for s in sectors])
        pa = (C.c_void_p * n)(*[p.h.value if isinstance(p.h, C.c_void_p) else p.h for p in pools])
        h = C.c_void_p()
        _check(L.cvq_batch_create(sa, pa, n, int(n_max), C.byref(h)), "cvq_batch_create")
        self.h, self.n, self.n_max = h, n, int(n_max)
        self.E = torch.empty(n, dtype=torch.float64, device="cuda")
        self.theta = torch.zeros(max(1, n * self.n_max), dtype=torch.float64, device="cuda")
        self.grad = torch.zeros_like(self.theta)
        self.n_ops = [-1] * n
        self.offsets = [0] * (n + 1)

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.cvq_batch_destroy(self.h)
            self.h = None

    def set_ansatz(self, op_ids: Sequence[Optional[Sequence[int]]], psi0: Sequence):
        """op_ids[i] is the ansatz of instance i (None leaves it out); psi0[i] its reference state."""
        n_ops = [(-1 if ids is None else len(ids)) for ids in op_ids]
        flat = [int(k) for ids in op_ids if ids is not None for k in ids]
        na = (C.c_int * self.n)(*n_ops)
        ia = (C.c_int * max(1, len(flat)))(*flat)
        pa = (C.c_void_p * self.n)(*[(_dev(p, "c128", s.dim, f"psi0[{i}]").value if p is not None else 0)
                                     for i, (p, s) in enumerate(zip(psi0, self._keep[0]))])
        self._psi0 = list(psi0)
        _check(lib().cvq_batch_set_ansatz(self.h, na, ia, pa), "cvq_batch_set_ansatz")
        self.n_ops = n_ops
        off = [0]
        for k in n_ops:
            off.append(off[-1] + max(k, 0))
        self.offsets = off

    def set_active(self, active: Sequence[bool], stream=None):
        a = (C.c_int * self.n)(*[int(bool(v)) for v in active])
        _check(lib().cvq_batch_set_active(self.h, a, _stream(stream)), "cvq_batch_set_active")

    def set_schedule(self, tile: int, ctas_per_sm: int):
        _check(lib().cvq_batch_set_schedule(self.h, int(tile), int(ctas_per_sm)), "cvq_batch_set_schedule")

    def energy_and_grad(self, theta=None, stream=None):
        """theta: device float64 vector packed like the op ids (None: use self.theta as filled by the caller).
        Returns the device tensors (E[n], grad[packed])."""
        if theta is not None:
            self.theta[: theta.numel()].copy_(theta)
        _check(lib().cvq_batch_energy_and_grad(self.h, _dev(self.theta, "f64", self.offsets[-1], "theta"),
                                               _dev(self.E, "f64", self.n, "E"),
                                               _dev(self.grad, "f64", self.offsets[-1], "grad"), _stream(stream)),
               "cvq_batch_energy_and_grad")
        return self.E, self.grad[: self.offsets[-1]]

    def screen(self, subsets=None, out=None, stream=None):
        """Eq. (grad) on the current state U(theta) psi0 of every active instance
        (theta as last loaded into self.theta), for every pool element
        (subsets None) or for subsets[i] (a list of pool indices per instance).
        Returns the packed device tensor and the per-instance output offsets."""
        import torch
        K = [p.K for p in self._keep[1]]
        counts = [0 if self.n_ops[i] < 0 else (K[i] if subsets is None else len(subsets[i])) for i in range(self.n)]
        off = [0]
        for c in counts:
            off.append(off[-1] + c)
        if out is None:
            out = torch.empty(max(off[-1], 1), dtype=torch.float64, device="cuda")
        if subsets is None:
            so, sa = None, None
        else:
            so = (C.c_int * (self.n + 1))(*[0] + [sum(len(subsets[q]) for q in range(i + 1)) for i in range(self.n)])
            flat = [int(k) for sub in subsets for k in sub]
            sa = (C.c_int * max(1, len(flat)))(*flat)
        _check(lib().cvq_batch_screen(self.h, _dev(self.theta, "f64", self.offsets[-1], "theta"), so, sa,
                                      _dev(out, "f64", off[-1], "out"), _stream(stream)), "cvq_batch_screen")
        return out, off

    def info(self):
        k, it, ly = C.c_int(), C.c_int(), C.c_int()
        npar = C.c_int64()
        _check(lib().cvq_batch_info(self.h, C.byref(k), C.byref(it), C.byref(ly), C.byref(npar)), "cvq_batch_info")
        return dict(kernels_per_eval=k.value, items=it.value, layers=ly.value, params=npar.value)


def energy_and_grad_ckpt(sector: Sector, pool: Pool, op_ids, theta, psi0, every: int, E=None, grad=None, ws=None,
                         ckpt=None, stream=None):
    """cvq_energy_and_grad with forward states checkpointed every `every` gates (see the header)."""
    import torch
    L = lib()
    L.cvq_checkpoint_bytes.argtypes = [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_size_t)]
    L.cvq_energy_and_grad_ckpt.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double),
                                           C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                           C.c_size_t, C.c_void_p, C.c_size_t, C.c_void_p]
    n, ids, th = _ids_theta(op_ids, theta)
    if E is None:
        E = torch.empty(1, dtype=torch.float64, device=psi0.device)
    if grad is None:
        grad = torch.empty(max(n, 1), dtype=torch.float64, device=psi0.device)
    ws, wsb = _ws(sector, pool, n, ws)
    need = C.c_size_t()
    _check(L.cvq_checkpoint_bytes(sector.h, n, int(every), C.byref(need)), "cvq_checkpoint_bytes")
    if ckpt is None:
        ckpt = torch.empty(max(int(need.value), 1), dtype=torch.uint8, device=psi0.device)
    _check(L.cvq_energy_and_grad_ckpt(sector.h, pool.h, ids, th.ctypes.data_as(C.POINTER(C.c_double)), n,
                                      _dev(psi0, "c128", sector.dim, "psi0"), _dev(E, "f64", 1, "E"),
                                      _dev(grad, "f64", n, "grad"), int(every), _dev(ckpt, "u8", 0, "ckpt"),
                                      ckpt.numel(), _dev(ws, "u8", 0, "workspace"), wsb, _stream(stream)),
           "cvq_energy_and_grad_ckpt")
    return E, grad[:n]


def stored_states_bytes(sector: Sector, pool: Pool, op_ids) -> int:
    """Device bytes of the stored forward states of this ansatz (cvq_stored_states_bytes)."""
    L = lib()
    L.cvq_stored_states_bytes.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(C.c_int), C.c_int,
                                          C.POINTER(C.c_size_t)]
    n = len(op_ids)
    ids = (C.c_int * max(n, 1))(*[int(k) for k in op_ids])
    need = C.c_size_t()
    _check(L.cvq_stored_states_bytes(sector.h, pool.h, ids, n, C.byref(need)), "cvq_stored_states_bytes")
    return int(need.value)


def energy_and_grad_stored(sector: Sector, pool: Pool, op_ids, theta, psi0, states=None, E=None, grad=None, ws=None,
                           stream=None):
    """cvq_energy_and_grad with the forward states kept for the reverse sweep
    (see the header); states: a uint8 device buffer of at least
    stored_states_bytes(...) bytes, allocated here when None."""
    import torch
    L = lib()
    L.cvq_energy_and_grad_stored.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double),
                                             C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_size_t,
                                             C.c_void_p, C.c_size_t, C.c_void_p]
    n, ids, th = _ids_theta(op_ids, theta)
    if E is None:
        E = torch.empty(1, dtype=torch.float64, device=psi0.device)
    if grad is None:
        grad = torch.empty(max(n, 1), dtype=torch.float64, device=psi0.device)
    ws, wsb = _ws(sector, pool, n, ws)
    need = stored_states_bytes(sector, pool, op_ids)
    if states is None:
        states = torch.empty(max(need, 1), dtype=torch.uint8, device=psi0.device)
    _check(L.cvq_energy_and_grad_stored(sector.h, pool.h, ids, th.ctypes.data_as(C.POINTER(C.c_double)), n,
                                        _dev(psi0, "c128", sector.dim, "psi0"), _dev(E, "f64", 1, "E"),
                                        _dev(grad, "f64", n, "grad"), _dev(states, "u8", need, "states"),
                                        states.numel(), _dev(ws, "u8", 0, "workspace"), wsb, _stream(stream)),
           "cvq_energy_and_grad_stored")
    return E, grad[:n]


def _proj_sigs(L):
    vp, ip, dp = C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)
    L.cvq_set_pool_projected.argtypes = [vp, C.POINTER(_Op), C.c_int, C.c_int, C.POINTER(vp)]
    L.cvq_projected_states_bytes.argtypes = [vp, vp, ip, C.c_int, C.POINTER(C.c_size_t)]
    L.cvq_apply_ansatz_projected.argtypes = [vp, vp, ip, dp, C.c_int, vp, vp, vp, C.c_size_t, vp, C.c_size_t, vp]
    L.cvq_energy_and_grad_projected.argtypes = [vp, vp, ip, dp, C.c_int, vp, vp, vp, vp, C.c_size_t, vp, C.c_size_t,
                                                vp]
    return L


class ProjectedPool(Pool):
    """A pool whose gates are the untruncated gates projected onto the cutoff (Sec. V.A)."""

    def __init__(self, sector: Sector, ops: Sequence[Op], inner_cutoff: int):
        L = _proj_sigs(lib())
        self.sector = sector
        self.ops = list(ops)
        K = len(self.ops)
        arr = (_Op * max(K, 1))(*[_Op(OP_CODES[o.type], o.i, o.j if o.j is not None else -1, o.phase)
                                  for o in self.ops])
        h = C.c_void_p()
        _check(L.cvq_set_pool_projected(sector.h, arr, K, int(inner_cutoff), C.byref(h)), "cvq_set_pool_projected")
        self.h = h
        self.K = K
        self.inner_cutoff = int(inner_cutoff)


def _proj_states(sector, pool, ids, n, states, device):
    import torch
    b = C.c_size_t()
    _check(lib().cvq_projected_states_bytes(sector.h, pool.h, ids, n, C.byref(b)), "cvq_projected_states_bytes")
    if states is None or states.numel() < b.value:
        states = torch.empty(int(b.value), dtype=torch.uint8, device=device)
    return states


def apply_ansatz_projected(sector: Sector, pool: ProjectedPool, op_ids, theta, psi0, out=None, ws=None, states=None,
                           stream=None):
    import torch
    _proj_sigs(lib())
    n, ids, th = _ids_theta(op_ids, theta)
    if out is None:
        out = torch.empty_like(psi0)
    ws, wsb = _ws(sector, pool, n, ws)
    states = _proj_states(sector, pool, ids, n, states, psi0.device)
    d = sector.dim
    _check(lib().cvq_apply_ansatz_projected(sector.h, pool.h, ids, th.ctypes.data_as(C.POINTER(C.c_double)), n,
                                            _dev(psi0, "c128", d, "psi0"), _dev(out, "c128", d, "out"),
                                            _dev(states, "u8", 0, "states"), states.numel(),
                                            _dev(ws, "u8", 0, "workspace"), wsb, _stream(stream)),
           "cvq_apply_ansatz_projected")
    return out


def energy_and_grad_projected(sector: Sector, pool: ProjectedPool, op_ids, theta, psi0, E=None, grad=None, ws=None,
                              states=None, stream=None):
    import torch
    _proj_sigs(lib())
    n, ids, th = _ids_theta(op_ids, theta)
    if E is None:
        E = torch.empty(1, dtype=torch.float64, device=psi0.device)
    if grad is None:
        grad = torch.empty(max(n, 1), dtype=torch.float64, device=psi0.device)
    ws, wsb = _ws(sector, pool, n, ws)
    states = _proj_states(sector, pool, ids, n, states, psi0.device)
    _check(lib().cvq_energy_and_grad_projected(sector.h, pool.h, ids, th.ctypes.data_as(C.POINTER(C.c_double)), n,
                                               _dev(psi0, "c128", sector.dim, "psi0"), _dev(E, "f64", 1, "E"),
                                               _dev(grad, "f64", n, "grad"), _dev(states, "u8", 0, "states"),
                                               states.numel(), _dev(ws, "u8", 0, "workspace"), wsb,
                                               _stream(stream)), "cvq_energy_and_grad_projected")
    return E, grad[:n]
