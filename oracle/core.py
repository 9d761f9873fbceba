"""ctypes binding of the C oracle (cvq_oracle.c).  Test infrastructure only.

Sector states are numpy complex128 vectors indexed in lexicographic order of
the occupation tuples (mode 0 most significant).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Sequence

import numpy as np

from . import build as _build
from .operators import generator_strings, hamiltonian_strings, MAXF

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp, i64, dp, ip = C.c_void_p, C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_int)
        L.orc_sector_new.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(vp), C.POINTER(i64)]
        L.orc_sector_free.argtypes = [vp]
        L.orc_sector_index.argtypes = [vp, ip]
        L.orc_sector_index.restype = i64
        L.orc_sector_tuples.argtypes = [vp, ip]
        L.orc_op_new.argtypes = [C.c_int, dp, ip, C.POINTER(vp)]
        L.orc_op_free.argtypes = [vp]
        L.orc_apply.argtypes = [vp, vp, vp, vp]
        L.orc_apply_rows.argtypes = [vp, vp, vp, C.POINTER(i64), i64, vp]
        L.orc_norm_bound.argtypes = [vp, vp]
        L.orc_norm_bound.restype = C.c_double
        L.orc_expm_apply.argtypes = [vp, vp, C.c_double, vp, vp]
        L.orc_energy.argtypes = [vp, vp, vp, dp, dp]
        L.orc_screen.argtypes = [vp, vp, C.c_int, C.POINTER(vp), vp, dp, dp]
        L.orc_apply_ansatz.argtypes = [vp, C.c_int, C.POINTER(vp), dp, vp, vp]
        L.orc_energy_and_grad.argtypes = [vp, vp, C.c_int, C.POINTER(vp), dp, vp, dp, dp]
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_set_threads.restype = None
        L.orc_max_threads.restype = C.c_int
        _lib = L
    return _lib


def set_threads(n: int) -> None:
    """Threads of the oracle's parallel loops (OpenMP)."""
    lib().orc_set_threads(int(n))


def max_threads() -> int:
    return int(lib().orc_max_threads())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


class Operator:
    """Sum of ladder strings, owned by the C oracle."""

    def __init__(self, strings):
        ns = len(strings)
        coef = np.zeros(2 * max(ns, 1), dtype=np.float64)
        fac = -np.ones((max(ns, 1), MAXF, 2), dtype=np.int32)
        for t, (c, factors) in enumerate(strings):
            coef[2 * t] = complex(c).real
            coef[2 * t + 1] = complex(c).imag
            assert len(factors) <= MAXF
            for f, (mode, dag) in enumerate(factors):
                fac[t, f, 0] = mode
                fac[t, f, 1] = dag
        self._coef, self._fac = coef, fac
        h = C.c_void_p()
        _check(lib().orc_op_new(ns, coef.ctypes.data_as(C.POINTER(C.c_double)),
                                fac.ctypes.data_as(C.POINTER(C.c_int)), C.byref(h)), "op_new")
        self.h = h
        self.strings = strings

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.orc_op_free(self.h)
            self.h = None


class Sector:
    """Symmetry sector of a model (Sec. III): fixed N (BH) or parity (BKC)."""

    def __init__(self, model):
        self.model = model
        kind = 0 if model.kind == "bh" else 1
        h = C.c_void_p()
        dim = C.c_int64()
        _check(lib().orc_sector_new(kind, model.L, model.N, model.d, model.parity, C.byref(h), C.byref(dim)),
               "sector_new")
        self.h = h
        self.dim = int(dim.value)
        self.L = model.L
        self.D = model.N + 1 if model.kind == "bh" else model.d
        self.H = Operator(hamiltonian_strings(model))
        self._ops = {}

    def __del__(self):
        if getattr(self, "h", None) is not None and _lib is not None:
            _lib.orc_sector_free(self.h)
            self.h = None

    # --- basis
    def tuples(self) -> np.ndarray:
        out = np.zeros((self.dim, self.L), dtype=np.int32)
        lib().orc_sector_tuples(self.h, out.ctypes.data_as(C.POINTER(C.c_int)))
        return out

    def index(self, occ: Sequence[int]) -> int:
        a = np.asarray(occ, dtype=np.int32)
        return int(lib().orc_sector_index(self.h, a.ctypes.data_as(C.POINTER(C.c_int))))

    def basis_state(self, occ: Sequence[int]) -> np.ndarray:
        v = np.zeros(self.dim, dtype=np.complex128)
        x = self.index(occ)
        if x < 0:
            raise ValueError(f"occupation {occ} not in the sector")
        v[x] = 1.0
        return v

    # --- operators
    def op(self, o) -> Operator:
        key = tuple(o)
        if key not in self._ops:
            self._ops[key] = Operator(generator_strings(o))
        return self._ops[key]

    def apply(self, operator: Operator, v: np.ndarray) -> np.ndarray:
        v = np.ascontiguousarray(v, dtype=np.complex128)
        out = np.empty_like(v)
        _check(lib().orc_apply(self.h, operator.h, _ptr(v), _ptr(out)), "apply")
        return out

    def apply_H(self, v: np.ndarray) -> np.ndarray:
        return self.apply(self.H, v)

    def apply_rows(self, operator: Operator, v: np.ndarray, rows: Sequence[int]) -> np.ndarray:
        v = np.ascontiguousarray(v, dtype=np.complex128)
        r = np.ascontiguousarray(rows, dtype=np.int64)
        out = np.empty(len(r), dtype=np.complex128)
        _check(lib().orc_apply_rows(self.h, operator.h, _ptr(v), r.ctypes.data_as(C.POINTER(C.c_int64)),
                                    len(r), _ptr(out)), "apply_rows")
        return out

    def matrix(self, operator: Operator) -> np.ndarray:
        """Dense matrix of an operator in the sector (column x = O|x>); small sectors only."""
        M = np.zeros((self.dim, self.dim), dtype=np.complex128)
        e = np.zeros(self.dim, dtype=np.complex128)
        for x in range(self.dim):
            e[:] = 0
            e[x] = 1
            M[:, x] = self.apply(operator, e)
        return M

    def norm_bound(self, operator: Operator) -> float:
        return float(lib().orc_norm_bound(self.h, operator.h))

    def expm_apply(self, o, theta: float, v: np.ndarray) -> np.ndarray:
        v = np.ascontiguousarray(v, dtype=np.complex128)
        out = np.empty_like(v)
        _check(lib().orc_expm_apply(self.h, self.op(o).h, float(theta), _ptr(v), _ptr(out)), "expm_apply")
        return out

    def energy(self, v: np.ndarray):
        v = np.ascontiguousarray(v, dtype=np.complex128)
        E, n2 = C.c_double(), C.c_double()
        _check(lib().orc_energy(self.h, self.H.h, _ptr(v), C.byref(E), C.byref(n2)), "energy")
        return E.value, n2.value

    def screen(self, ops: Sequence, v: np.ndarray, return_imag: bool = False):
        v = np.ascontiguousarray(v, dtype=np.complex128)
        K = len(ops)
        handles = (C.c_void_p * K)(*[self.op(o).h for o in ops])
        g = np.zeros(K)
        gi = np.zeros(K)
        _check(lib().orc_screen(self.h, self.H.h, K, handles, _ptr(v), g.ctypes.data_as(C.POINTER(C.c_double)),
                                gi.ctypes.data_as(C.POINTER(C.c_double))), "screen")
        return (g, gi) if return_imag else g

    def apply_ansatz(self, ops: Sequence, theta: Sequence[float], psi0: np.ndarray) -> np.ndarray:
        psi0 = np.ascontiguousarray(psi0, dtype=np.complex128)
        n = len(ops)
        th = np.ascontiguousarray(theta, dtype=np.float64)
        handles = (C.c_void_p * max(n, 1))(*[self.op(o).h for o in ops])
        out = np.empty_like(psi0)
        _check(lib().orc_apply_ansatz(self.h, n, handles, th.ctypes.data_as(C.POINTER(C.c_double)), _ptr(psi0),
                                      _ptr(out)), "apply_ansatz")
        return out

    def energy_and_grad(self, ops: Sequence, theta: Sequence[float], psi0: np.ndarray):
        psi0 = np.ascontiguousarray(psi0, dtype=np.complex128)
        n = len(ops)
        th = np.ascontiguousarray(theta, dtype=np.float64)
        handles = (C.c_void_p * max(n, 1))(*[self.op(o).h for o in ops])
        E = C.c_double()
        g = np.zeros(n)
        _check(lib().orc_energy_and_grad(self.h, self.H.h, n, handles, th.ctypes.data_as(C.POINTER(C.c_double)),
                                         _ptr(psi0), C.byref(E), g.ctypes.data_as(C.POINTER(C.c_double))),
               "energy_and_grad")
        return E.value, g
