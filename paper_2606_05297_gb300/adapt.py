"""CV-ADAPT-VQE host driver on top of libcvq.so (Sec. IV.B).

Per ADAPT iteration: screen the pool with the Eq. (grad) gradients on the
current state, append the operator of largest |g| as exp(theta A) with
theta = 0, then re-minimise E(theta) over every parameter with BFGS whose
energy and gradient come from cvq_energy_and_grad.  Only scalars and vectors
of length n or K cross the host/device boundary.

Readings of the paper used here, where it is silent:
  * warm start: one HVA layer with angles U[-0.05, 0.05] is optimised first
    (L-inf gradient tolerance 1e-9) and stays in the ansatz, re-optimised with
    every ADAPT parameter (Sec. IV.B, App. C, App. D);
  * selection ties: lowest pool index among |g_k| >= max|g| (1 - 1e-9);
  * BFGS per ADAPT step: at most 1000 iterations, L-inf gradient tolerance
    min(1e-6, |g_init| 1e-5) (Sec. IV.A); textbook BFGS with a strong-Wolfe
    line search (c1 = 1e-4, c2 = 0.9), initial inverse Hessian = identity;
  * stopping: max|g| < grad_tol, max_ops ADAPT operators (~160 in Sec. IV.B),
    or |E - E0| < energy_tol when E0 is known.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Callable, List, Optional, Sequence

import numpy as np

from . import cvq
from .workloads import Model, Op

TIE_REL = 1e-9


# ---------------------------------------------------------------- BFGS

@dataclasses.dataclass
class OptResult:
    x: np.ndarray
    f: float
    g: np.ndarray
    nit: int
    nfev: int
    Hinv: np.ndarray
    status: str


class BFGS:
    """Quasi-Newton minimiser: inverse-Hessian BFGS update with a line search
    satisfying the strong Wolfe conditions (bracketing, then zoom with a
    safeguarded cubic step)."""

    def __init__(self, fg: Callable[[np.ndarray], tuple], c1: float = 1e-4, c2: float = 0.9, max_ls: int = 30,
                 step_max: float = 50.0):
        self.fg = fg
        self.c1, self.c2, self.max_ls, self.step_max = c1, c2, max_ls, step_max
        self.nfev = 0

    def _eval(self, x):
        # one evaluation, asked of whoever drives the generator
        self.nfev += 1
        f, g = yield x
        return float(f), np.asarray(g, dtype=np.float64)

    @staticmethod
    def _cubic(a, fa, da, b, fb, db):
        # minimiser of the Hermite cubic through (a, fa, da) and (b, fb, db);
        # a zero-width bracket has none (the caller bisects)
        if a == b:
            return None
        t1 = da + db - 3.0 * (fa - fb) / (a - b)
        sq = t1 * t1 - da * db
        if sq < 0.0:
            return None
        t2 = np.copysign(np.sqrt(sq), b - a)
        den = db - da + 2.0 * t2
        if den == 0.0:
            return None
        return b - (b - a) * (db + t2 - t1) / den

    def _search(self, x, f0, g0, p):
        d0 = float(g0 @ p)
        memo = {0.0: (f0, g0, d0)}

        def phi(a):
            if a not in memo:
                f, g = yield from self._eval(x + a * p)
                memo[a] = (f, g, float(g @ p))
            return memo[a]

        def zoom(lo, hi):
            for _ in range(self.max_ls):
                flo, _, dlo = yield from phi(lo)
                fhi, _, dhi = yield from phi(hi)
                w = abs(hi - lo)
                a = self._cubic(lo, flo, dlo, hi, fhi, dhi)
                if a is None or not (min(lo, hi) + 0.1 * w <= a <= max(lo, hi) - 0.1 * w):
                    a = 0.5 * (lo + hi)
                fa, _, da = yield from phi(a)
                if fa > f0 + self.c1 * a * d0 or fa >= flo:
                    hi = a
                else:
                    if abs(da) <= -self.c2 * d0:
                        return a
                    if da * (hi - lo) >= 0.0:
                        hi = lo
                    lo = a
                if abs(hi - lo) < 1e-16 * max(1.0, abs(lo)):
                    break
            flo = (yield from phi(lo))[0]
            return lo if (lo > 0.0 and flo < f0) else None

        prev, a, fprev = 0.0, 1.0, f0
        found = None
        for it in range(self.max_ls):
            fa, _, da = yield from phi(a)
            if fa > f0 + self.c1 * a * d0 or (it > 0 and fa >= fprev):
                found = yield from zoom(prev, a)
                break
            if abs(da) <= -self.c2 * d0:
                found = a
                break
            if da >= 0.0:
                found = yield from zoom(a, prev)
                break
            prev, fprev = a, fa
            a = min(2.0 * a, self.step_max)
        if found is None:
            return None, f0, g0
        f, g, _ = yield from phi(found)
        return found, f, g

    def steps(self, x0, gtol: float, max_iter: int = 1000, Hinv0=None):
        """The minimisation as a generator: it yields each point to evaluate,
        takes (f, g) back through send(), and returns the OptResult.  Several
        minimisations can then share one batched evaluation per round."""
        self.nfev = 0
        x = np.array(x0, dtype=np.float64)
        n = x.size
        f, g = yield from self._eval(x)
        Hi = np.eye(n) if Hinv0 is None else np.array(Hinv0, dtype=np.float64)
        status, it = "max_iter", 0
        while it < max_iter:
            if np.max(np.abs(g), initial=0.0) < gtol:
                status = "gtol"
                break
            p = -(Hi @ g)
            if float(g @ p) >= 0.0:
                Hi = np.eye(n)
                p = -g
            a, fn, gn = yield from self._search(x, f, g, p)
            if a is None:
                status = "line_search"
                break
            s = a * p
            y = gn - g
            x, f, g = x + s, fn, gn
            sy = float(s @ y)
            if sy > 0.0:
                r = 1.0 / sy
                Hy = Hi @ y
                # (I - r s y^T) Hi (I - r y s^T) + r s s^T, expanded
                Hi = Hi - r * (np.outer(s, Hy) + np.outer(Hy, s)) + (r * r * float(y @ Hy) + r) * np.outer(s, s)
            it += 1
        if np.max(np.abs(g), initial=0.0) < gtol:
            status = "gtol"
        return OptResult(x, f, g, it, self.nfev, Hi, status)

    def minimize(self, x0, gtol: float, max_iter: int = 1000, Hinv0=None) -> OptResult:
        gen = self.steps(x0, gtol, max_iter, Hinv0)
        try:
            x = next(gen)
            while True:
                x = gen.send(self.fg(x))
        except StopIteration as stop:
            return stop.value


# ---------------------------------------------------------------- selection

def select(g: np.ndarray):
    a = np.abs(np.asarray(g))
    m = float(a.max())
    return int(np.nonzero(a >= m * (1.0 - TIE_REL))[0][0]), m


# ---------------------------------------------------------------- driver

class Adapt:
    """One CV-ADAPT-VQE run on one Hamiltonian instance."""

    def __init__(self, model: Model, pool_ops: Sequence[Op], init_occ: Sequence[int], warm_ops: Sequence[Op] = (),
                 warm_theta: Sequence[float] = (), n_max: int = 256, stream=None, hessian_recycling: bool = False,
                 fix_warm: bool = False, stored_states: Optional[bool] = None):
        import torch
        self.torch = torch
        self.model = model
        self.K = len(pool_ops)
        self.pool_ops = list(pool_ops)
        self.sector = cvq.Sector(model)
        self.pool = cvq.Pool(self.sector, list(pool_ops) + list(warm_ops))
        self.psi0 = self.sector.basis_state(init_occ)
        self.n_max = n_max
        self.ws = self.sector.workspace(self.pool, n_max)
        self.stream = stream
        self.ids: List[int] = list(range(self.K, self.K + len(warm_ops)))
        self.theta = np.array(warm_theta, dtype=np.float64)
        self.trace = []
        self.Hinv = None
        # App. D variants: BFGS starts from the previous iteration's inverse
        # Hessian (extended by an identity row and column for the new
        # parameter); the warm-up layer keeps its initial parameters
        self.hessian_recycling = hessian_recycling
        self.fix_warm = fix_warm
        self._out = torch.empty(n_max + 1, dtype=torch.float64, device="cuda")
        self._host = torch.empty(n_max + 1, dtype=torch.float64, pin_memory=True)
        self._g = torch.empty(self.K, dtype=torch.float64, device="cuda")
        self._subset = list(range(self.K))
        self.nfev_total = 0
        # The reverse sweep reads the forward states kept in device memory
        # (cvq_energy_and_grad_stored) instead of recomputing them, when asked
        # to, or by default on sectors of at least 2^20 amplitudes (below that
        # the launches, not the arithmetic, bound an evaluation, and the extra
        # copies cost more than they save) whose worst case (one full state per
        # gate) fits in a quarter of the free device memory.
        if stored_states is None:
            free, _ = torch.cuda.mem_get_info()
            stored_states = self.sector.dim >= (1 << 20) and n_max * self.sector.dim * 16 <= free // 4
        self.stored_states = bool(stored_states)
        self._states = None
        self._states_key = None

    # energy and gradient of the current ansatz structure at theta (host vectors)
    def fg(self, theta):
        n = len(self.ids)
        if self.stored_states:
            key = tuple(self.ids)
            if self._states_key != key:  # the ansatz changed: size the stored states for it
                need = cvq.stored_states_bytes(self.sector, self.pool, self.ids)
                if self._states is None or self._states.numel() < need:
                    self._states = self.torch.empty(max(need, 1), dtype=self.torch.uint8, device="cuda")
                self._states_key = key
            E, g = cvq.energy_and_grad_stored(self.sector, self.pool, self.ids, theta, self.psi0, states=self._states,
                                              E=self._out[0:1], grad=self._out[1:n + 1] if n else self._out[1:2],
                                              ws=self.ws, stream=self.stream)
        else:
            E, g = cvq.energy_and_grad(self.sector, self.pool, self.ids, theta, self.psi0, E=self._out[0:1],
                                       grad=self._out[1:n + 1] if n else self._out[1:2], ws=self.ws,
                                       stream=self.stream)
        h = self._host[: n + 1]
        h.copy_(self._out[: n + 1], non_blocking=True)
        (self.stream or self.torch.cuda.current_stream()).synchronize()
        v = h.numpy()
        self.nfev_total += 1
        return float(v[0]), v[1:n + 1].copy()

    def state(self):
        return cvq.apply_ansatz(self.sector, self.pool, self.ids, self.theta, self.psi0, ws=self.ws,
                                stream=self.stream)

    def energy(self):
        return self.fg(self.theta)[0] if self.ids else self._energy_of(self.psi0)

    def _energy_of(self, psi):
        E = self._out[0:1]
        cvq.apply_H(self.sector, psi, energy=E, stream=self.stream)
        return float(E.item())

    def screen(self, psi=None, subset=None):
        psi = self.state() if psi is None else psi
        sub = self._subset if subset is None else list(subset)
        g = cvq.screen_pool(self.sector, self.pool, psi, subset=sub, out=self._g, ws=self.ws, stream=self.stream)
        return g[: len(sub)].cpu().numpy()

    def optimise_warm_start(self, gtol=1e-9, max_iter=1000):
        if not self.ids:
            return None
        r = BFGS(self.fg).minimize(self.theta, gtol=gtol, max_iter=max_iter)
        self.theta = r.x
        self.Hinv = r.Hinv
        self.trace.append(dict(kind="warm", E=r.f, nfev=r.nfev, nit=r.nit, status=r.status))
        if self.fix_warm:  # the warm-up state becomes the reference of the adaptive ansatz
            self.psi0 = self.state().clone()
            self.ids, self.theta, self.Hinv = [], np.zeros(0), None
        return r

    def step(self, grad_tol=1e-6, max_iter=1000, g=None):
        """One ADAPT iteration.  Returns the trace record, or None if converged."""
        t0 = time.perf_counter()
        g = self.screen() if g is None else g
        k, gmax = select(g)
        if gmax < grad_tol:
            return None
        return self._grow(k, gmax, max_iter, t0)

    def _grow(self, k, gmax, max_iter, t0):
        """Append pool operator k with theta = 0 and re-minimise every parameter."""
        if len(self.ids) + 1 > self.n_max:
            raise RuntimeError("ansatz length exceeds the workspace")
        self.ids.append(k)
        self.theta = np.append(self.theta, 0.0)
        H0 = None
        if self.hessian_recycling and self.Hinv is not None:
            H0 = np.eye(self.theta.size)
            H0[:-1, :-1] = self.Hinv
        r = BFGS(self.fg).minimize(self.theta, gtol=min(1e-6, gmax * 1e-5), max_iter=max_iter, Hinv0=H0)
        self.theta = r.x
        self.Hinv = r.Hinv
        rec = dict(kind="adapt", op=k, gmax=gmax, E=r.f, nfev=r.nfev, nit=r.nit, status=r.status, n=len(self.ids),
                   seconds=time.perf_counter() - t0)
        self.trace.append(rec)
        return rec

    def run(self, max_ops=160, grad_tol=1e-6, E0=None, energy_tol=None, max_iter=1000):
        n_adapt = 0
        stop = "max_ops"
        while n_adapt < max_ops:
            if E0 is not None and energy_tol is not None and self.ids and abs(self.energy() - E0) < energy_tol:
                stop = "energy_tol"
                break
            rec = self.step(grad_tol=grad_tol, max_iter=max_iter)
            if rec is None:
                stop = "grad_tol"
                break
            n_adapt += 1
        return dict(stop=stop, n_adapt=n_adapt, E=self.energy(), trace=self.trace)


# ---------------------------------------------------------------- E0

def ground_energy(sector: cvq.Sector, max_iter: int = 400, tol: float = 1e-13, seed: int = 0, check_every: int = 10,
                  stream=None) -> float:
    """Lowest eigenvalue of H in the sector by the Lanczos recurrence on the
    device (no re-orthogonalisation: the lowest Ritz value converges to E0)."""
    import torch
    from .workloads import random_state
    dim = sector.dim
    if dim == 1:
        E = torch.zeros(1, dtype=torch.float64, device="cuda")
        cvq.apply_H(sector, torch.ones(1, dtype=torch.complex128, device="cuda"), energy=E, stream=stream)
        return float(E.item())
    v = torch.from_numpy(random_state(dim, seed)).cuda()
    vp = torch.zeros_like(v)
    w = torch.empty_like(v)
    m = min(max_iter, dim)
    alpha = torch.zeros(m, dtype=torch.float64, device="cuda")
    beta = torch.zeros(m + 1, dtype=torch.float64, device="cuda")
    ws = sector.workspace(None, 0)
    last = None
    for j in range(m):
        cvq.apply_H(sector, v, sigma=w, energy=alpha[j:j + 1], ws=ws, stream=stream)
        cvq.lanczos_step(sector, vp, v, w, vp, alpha[j:j + 1], beta[j:j + 1], beta[j + 1:j + 2], ws=ws, stream=stream)
        v, vp = vp, v
        if (j + 1) % check_every == 0 or j == m - 1:
            a = alpha[: j + 1].cpu().numpy()
            b = beta[: j + 2].cpu().numpy()  # b[1..j] couple the j+1 Lanczos vectors, b[j+1] is the next norm
            T = np.diag(a) + np.diag(b[1:j + 1], 1) + np.diag(b[1:j + 1], -1)
            e = float(np.linalg.eigvalsh(T)[0])
            if (last is not None and abs(e - last) <= tol * max(1.0, abs(e))) or b[j + 1] < 1e-14:
                return e
            last = e
    return last
