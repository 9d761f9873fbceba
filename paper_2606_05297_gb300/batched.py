"""Batched ADAPT over many Hamiltonian instances (a U/J sweep) on one GPU.

Every instance runs the plain method of Sec. IV.B (screen, select the largest
|g|, append, re-minimise with BFGS), but the energy-and-gradient evaluations
of all instances share one batched graph launch per round: each instance's
BFGS is a generator that yields the point it wants evaluated, and one round
evaluates every pending point at once (cvq_batch_energy_and_grad).
Instances whose minimisation has finished are paused in the batch, so the
graph is captured once per ansatz structure.

The work-item size and CTAs per SM of the batched launches are chosen by
`autotune`, which times every candidate schedule on the batch itself.
"""
from __future__ import annotations

import json
import os
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import cvq
from .adapt import BFGS, OptResult, select
from .workloads import Model, Op

TILES = (4096, 16384, 65536, 262144)
CTAS = (1, 2)
_TUNED: Dict[tuple, tuple] = {}
# Schedules found by autotune, kept across processes: one JSON object per
# GPU model and set of sector sizes (the build folder is never committed).
TUNE_CACHE = os.environ.get("CVQ_TUNE_CACHE",
                            os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "batch_tune.json"))


def _tune_key(sectors) -> str:
    import torch
    return torch.cuda.get_device_name() + "|" + ",".join(str(d) for d in sorted(s.dim for s in sectors))


def _load_tuned() -> Dict[str, list]:
    try:
        with open(TUNE_CACHE) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def _store_tuned(key: str, tile: int, ctas: int) -> None:
    d = _load_tuned()
    d[key] = [int(tile), int(ctas)]
    try:
        os.makedirs(os.path.dirname(TUNE_CACHE), exist_ok=True)
        tmp = f"{TUNE_CACHE}.{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(d, f)
        os.replace(tmp, TUNE_CACHE)
    except OSError:
        pass  # an unwritable cache only costs a re-tune in the next process


def time_eval(batch: "cvq.Batch", reps: int = 3) -> float:
    """Mean milliseconds of one batched evaluation (CUDA events, after one warm-up)."""
    import torch
    batch.energy_and_grad()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        batch.energy_and_grad()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def autotune(batch: "cvq.Batch", sectors, tiles=TILES, ctas=CTAS, reps: int = 3, cache: bool = True) -> dict:
    """Time every (tile, CTAs per SM) schedule on the batch's current ansatz
    and keep the fastest.  Results are cached per GPU model and set of sector
    sizes, in memory and in TUNE_CACHE."""
    key = _tune_key(sectors)
    if cache and key not in _TUNED:
        hit = _load_tuned().get(key)
        if hit and len(hit) == 2:
            _TUNED[key] = (int(hit[0]), int(hit[1]))
    if cache and key in _TUNED:
        tile, c = _TUNED[key]
        batch.set_schedule(tile, c)
        return dict(tile=tile, ctas_per_sm=c, cached=True)
    best, table = None, []
    for tile in tiles:
        for c in ctas:
            batch.set_schedule(tile, c)
            ms = time_eval(batch, reps)
            table.append((tile, c, ms))
            if best is None or ms < best[2]:
                best = (tile, c, ms)
    batch.set_schedule(best[0], best[1])
    _TUNED[key] = (best[0], best[1])
    if cache:
        _store_tuned(key, best[0], best[1])
    return dict(tile=best[0], ctas_per_sm=best[1], ms=best[2], table=table, cached=False)


class BatchedAdapt:
    """Lockstep CV-ADAPT-VQE on n instances with one shared batched engine."""

    def __init__(self, models: Sequence[Model], pool_ops: Sequence[Sequence[Op]], init_occ: Sequence[Sequence[int]],
                 warm_ops: Sequence[Sequence[Op]] = None, warm_theta: Sequence[Sequence[float]] = None,
                 n_max: int = 160, tune: bool = True, hessian_recycling: bool = False):
        import torch
        self.torch = torch
        n = len(models)
        warm_ops = warm_ops or [[] for _ in range(n)]
        warm_theta = warm_theta or [[] for _ in range(n)]
        self.models = list(models)
        self.K = [len(p) for p in pool_ops]
        self.sectors = [cvq.Sector(m) for m in models]
        self.pools = [cvq.Pool(s, list(p) + list(w)) for s, p, w in zip(self.sectors, pool_ops, warm_ops)]
        self.psi0 = [s.basis_state(o) for s, o in zip(self.sectors, init_occ)]
        self.ids: List[List[int]] = [list(range(K, K + len(w))) for K, w in zip(self.K, warm_ops)]
        self.theta = [np.array(t, dtype=np.float64) for t in warm_theta]
        self.n_max = n_max
        self.batch = cvq.Batch(self.sectors, self.pools, n_max)
        self.done = [False] * n
        self.trace: List[list] = [[] for _ in range(n)]
        self.rounds = 0
        self.evals = 0
        self.tune = tune
        self.tuned = None
        self._host = torch.empty(n * n_max + n, dtype=torch.float64, pin_memory=True)
        self.batch_ready = False
        self.screens = 0
        self._gout = None
        # App. D: each BFGS starts from the instance's previous inverse Hessian,
        # extended by an identity row and column for the new parameter
        self.hessian_recycling = hessian_recycling
        self.Hinv: List[Optional[np.ndarray]] = [None] * n

    # ---------------------------------------------------------------- evaluations

    def _structure(self):
        self.batch.set_ansatz([None if self.done[i] else self.ids[i] for i in range(len(self.ids))], self.psi0)
        self.batch_ready = True
        if self.tune and self.tuned is None:
            self._load_theta({i: self.theta[i] for i in range(len(self.ids)) if not self.done[i]})
            self.tuned = autotune(self.batch, self.sectors)

    def _load_theta(self, xs: Dict[int, np.ndarray]):
        off = self.batch.offsets
        h = self._host[: off[-1]].numpy()
        for i, x in xs.items():
            h[off[i]:off[i + 1]] = x
        self.batch.theta[: off[-1]].copy_(self._host[: off[-1]], non_blocking=True)

    def lockstep(self, gens: Dict[int, object]) -> Dict[int, OptResult]:
        """Drive several BFGS generators; every round evaluates all pending
        points with one batched launch."""
        torch = self.torch
        xs = {}
        res = {}
        for i, g in gens.items():
            xs[i] = next(g)
        n = len(self.ids)
        off = self.batch.offsets
        while xs:
            self.batch.set_active([i in xs for i in range(n)])
            self._load_theta(xs)
            E, G = self.batch.energy_and_grad()
            hE = E.cpu().numpy()
            hG = G.cpu().numpy()
            self.rounds += 1
            self.evals += len(xs)
            for i in list(xs):
                try:
                    xs[i] = gens[i].send((float(hE[i]), hG[off[i]:off[i + 1]].copy()))
                except StopIteration as stop:
                    res[i] = stop.value
                    del xs[i]
        return res

    def optimise_warm_start(self, gtol: float = 1e-9, max_iter: int = 1000):
        self._structure()
        gens = {i: BFGS(None).steps(self.theta[i], gtol=gtol, max_iter=max_iter)
                for i in range(len(self.ids)) if len(self.ids[i])}
        for i, r in self.lockstep(gens).items():
            self.theta[i] = r.x
            self.Hinv[i] = r.Hinv
            self.trace[i].append(dict(kind="warm", E=r.f, nfev=r.nfev, nit=r.nit, status=r.status))

    def screen_all(self, subsets=None, which=None):
        """Eq. (grad) on the current state of the instances in `which` (default:
        every instance that has not converged), all in one batched launch
        (cvq_batch_screen): the pool operators of subsets[i] (default: the
        whole pool without the warm-start gates).  Returns {instance: host
        gradient vector}."""
        n = len(self.ids)
        if not self.batch_ready:
            self._structure()
        live = [i for i in range(n) if not self.done[i] and (which is None or i in which)]
        on = set(live)
        self.batch.set_active([i in on for i in range(n)])
        self._load_theta({i: self.theta[i] for i in live})
        subs = [(list(range(self.K[i])) if subsets is None else list(subsets[i])) if i in on else []
                for i in range(n)]
        need = sum(len(q) for q in subs)
        if self._gout is None or self._gout.numel() < max(need, 1):
            self._gout = self.torch.empty(max(sum(self.K), 1), dtype=self.torch.float64, device="cuda")
        out, off = self.batch.screen(subs, out=self._gout)
        h = out[: max(off[-1], 1)].cpu().numpy()
        self.screens += 1
        return {i: h[off[i]:off[i + 1]].copy() for i in live}

    def choose(self, grad_tol: float, which=None):
        """The operator each live instance (of `which`, default all) appends:
        {instance: (pool index, |g|)} (plain rule: largest exact gradient of a
        full screen).  Instances whose largest |g| is below grad_tol are marked
        done."""
        chosen = {}
        gs = self.screen_all(which=which)
        for i, g in gs.items():
            k, gmax = select(g)
            if gmax < grad_tol or len(self.ids[i]) + 1 > self.n_max:
                self.done[i] = True
                continue
            chosen[i] = (k, gmax)
        return chosen

    def step(self, grad_tol: float = 1e-6, max_iter: int = 1000, stop=None):
        """One ADAPT iteration on every instance that has not converged (nor
        been stopped: stop[i] True leaves instance i out for good).
        Returns the number of instances that grew."""
        if stop is not None:
            for i, st in enumerate(stop):
                if st:
                    self.done[i] = True
        grown = self.choose(grad_tol)
        for i, (k, _) in grown.items():
            self.ids[i].append(k)
            self.theta[i] = np.append(self.theta[i], 0.0)
        if not grown:
            return 0
        self._structure()
        gens = {}
        for i, (_, gm) in grown.items():
            H0 = None
            if self.hessian_recycling and self.Hinv[i] is not None:
                H0 = np.eye(self.theta[i].size)
                H0[:-1, :-1] = self.Hinv[i]
            gens[i] = BFGS(None).steps(self.theta[i], gtol=min(1e-6, gm * 1e-5), max_iter=max_iter, Hinv0=H0)
        for i, r in self.lockstep(gens).items():
            self.theta[i] = r.x
            self.Hinv[i] = r.Hinv
            self.trace[i].append(dict(kind="adapt", op=grown[i][0], gmax=grown[i][1], E=r.f, nfev=r.nfev, nit=r.nit,
                                      status=r.status, n=len(self.ids[i])))
        self.after_step(grown)
        return len(grown)

    def run(self, max_ops: int = 160, grad_tol: float = 1e-6, max_iter: int = 1000, stop_after=None,
            on_iteration=None):
        """ADAPT on every instance with asynchronous rounds: each round screens
        (one batched screen) and grows every instance whose last minimisation
        has finished, then evaluates every pending BFGS point with one batched
        launch, so no instance waits for the slowest one's BFGS.  An instance
        ends on max|g| < grad_tol, after max_ops operators, or when
        stop_after(i, record) returns True.  on_iteration(i, record) sees
        every finished iteration."""
        n = len(self.ids)
        if not self.batch_ready:
            self._structure()
        count = [0] * n
        gens, xs, grown = {}, {}, {}
        ready = [i for i in range(n) if not self.done[i]]
        while True:
            ready = [i for i in ready if not self.done[i]]
            if ready:
                chosen = self.choose(grad_tol, which=set(ready))
                for i, (k, gm) in chosen.items():
                    self.ids[i].append(k)
                    self.theta[i] = np.append(self.theta[i], 0.0)
                    H0 = None
                    if self.hessian_recycling and self.Hinv[i] is not None:
                        H0 = np.eye(self.theta[i].size)
                        H0[:-1, :-1] = self.Hinv[i]
                    gens[i] = BFGS(None).steps(self.theta[i], gtol=min(1e-6, gm * 1e-5), max_iter=max_iter, Hinv0=H0)
                    grown[i] = (k, gm)
                if chosen:
                    self._structure()
                    for i in chosen:
                        xs[i] = next(gens[i])
                ready = []
            if not xs:
                break
            self.batch.set_active([i in xs for i in range(n)])
            self._load_theta(xs)
            E, G = self.batch.energy_and_grad()
            hE = E.cpu().numpy()
            hG = G.cpu().numpy()
            off = self.batch.offsets
            self.rounds += 1
            self.evals += len(xs)
            for i in list(xs):
                try:
                    xs[i] = gens[i].send((float(hE[i]), hG[off[i]:off[i + 1]].copy()))
                except StopIteration as st:
                    r = st.value
                    del xs[i], gens[i]
                    self.theta[i] = r.x
                    self.Hinv[i] = r.Hinv
                    k, gm = grown.pop(i)
                    rec = dict(kind="adapt", op=k, gmax=gm, E=r.f, nfev=r.nfev, nit=r.nit, status=r.status,
                               n=len(self.ids[i]))
                    self.trace[i].append(rec)
                    self.after_step({i: (k, gm)})
                    count[i] += 1
                    if on_iteration is not None:
                        on_iteration(i, rec)
                    if count[i] >= max_ops or (stop_after is not None and stop_after(i, rec)):
                        self.done[i] = True
                    else:
                        ready.append(i)
        return dict(iterations=count, rounds=self.rounds, evals=self.evals)

    def after_step(self, grown):
        """Hook for drivers that keep per-iteration state (the learned proposal)."""


def c4_batch_inputs(seed: int = 0, count: int = 64, extra_ops: int = 8):
    """The 64-instance sweep with an HVA warm-start layer plus `extra_ops`
    seeded pool operators per instance, for throughput measurements."""
    from . import workloads as W
    insts = W.c4_instances(seed, count)
    rng = np.random.default_rng(seed + 1)
    out = []
    for m in insts:
        pool = W.bh_allpairs_pool(m.L)
        warm = W.hva_layer(m)
        ids = list(range(len(pool), len(pool) + len(warm))) + [int(k) for k in rng.integers(0, len(pool), extra_ops)]
        th = np.concatenate([W.warm_start_thetas(len(warm), 0), rng.uniform(-0.2, 0.2, extra_ops)])
        out.append((m, pool + warm, ids, th))
    return out


def shard(dims: Sequence[int], rank: int, world: int) -> List[int]:
    """Instances of one rank when a sweep is split over `world` GPUs:
    longest-first assignment to the least-loaded rank by sector dimension
    (ties to the lower rank), so every rank computes the same split without
    communicating.  Returns the sorted instance indices of `rank`."""
    load = [0] * world
    owner = [0] * len(dims)
    for i in sorted(range(len(dims)), key=lambda k: (-dims[k], k)):
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += dims[i]
    return [i for i in range(len(dims)) if owner[i] == rank]


def measure_c4(reps: int = 5, seed: int = 0, count: int = 64, extra_ops: int = 8, sequential: bool = True,
               rank: int = 0, world: int = 1) -> dict:
    """Throughput of energy-and-gradient evaluations over the 64-instance sweep:
    one batched graph launch per evaluation of every instance, against the
    same evaluations issued instance by instance through cvq_energy_and_grad.
    Device-resident inputs; CUDA events on the launching stream.  With
    world > 1 this rank measures its own shard of the instances."""
    import torch
    data = c4_batch_inputs(seed, count, extra_ops)
    if world > 1:
        from math import comb
        dims = [comb(m.N + m.L - 1, m.L - 1) for m, _, _, _ in data]
        data = [data[i] for i in shard(dims, rank, world)]
        count = len(data)
    sectors = [cvq.Sector(m) for m, _, _, _ in data]
    pools = [cvq.Pool(s, ops) for s, (_, ops, _, _) in zip(sectors, data)]
    psi0 = [s.basis_state(_mott(m)) for s, (m, _, _, _) in zip(sectors, data)]
    n_max = max(len(ids) for _, _, ids, _ in data)
    b = cvq.Batch(sectors, pools, n_max)
    b.set_ansatz([ids for _, _, ids, _ in data], psi0)
    flat = np.concatenate([th for _, _, _, th in data])
    b.theta[: flat.size].copy_(torch.from_numpy(flat))
    tuned = autotune(b, sectors, cache=False)
    ms_batch = time_eval(b, reps)
    info = b.info()
    amps = sum(s.dim for s in sectors)
    gates = sum(len(ids) for _, _, ids, _ in data)
    out = dict(instances=count, amplitudes=amps, params=int(flat.size), ms_per_eval_batched=ms_batch,
               evals_per_s_batched=count * 1e3 / ms_batch, schedule=dict(tile=tuned["tile"],
                                                                           ctas_per_sm=tuned["ctas_per_sm"]),
               kernels_per_eval=info["kernels_per_eval"], items=info["items"], layers=info["layers"],
               gate_amplitudes_per_s_batched=sum(s.dim * len(ids) for s, (_, _, ids, _) in zip(sectors, data)) * 2e3
               / ms_batch, total_gates=gates)
    if sequential:
        E = torch.empty(count, dtype=torch.float64, device="cuda")
        G = torch.empty(flat.size, dtype=torch.float64, device="cuda")
        wss = [s.workspace(p, len(ids)) for s, p, (_, _, ids, _) in zip(sectors, pools, data)]
        offs = np.concatenate([[0], np.cumsum([len(ids) for _, _, ids, _ in data])])

        def loop():
            for i, (s, p, (m, _, ids, th)) in enumerate(zip(sectors, pools, data)):
                cvq.energy_and_grad(s, p, ids, th, psi0[i], E=E[i:i + 1], grad=G[offs[i]:offs[i + 1]], ws=wss[i])

        loop()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            loop()
        e1.record()
        e1.synchronize()
        ms_seq = e0.elapsed_time(e1) / reps
        Eb, Gb = b.energy_and_grad()
        out.update(ms_per_eval_sequential=ms_seq, evals_per_s_sequential=count * 1e3 / ms_seq,
                   speedup=ms_seq / ms_batch,
                   max_abs_diff_E=float((Eb - E).abs().max()), max_abs_diff_grad=float((Gb - G).abs().max()))
    return out


def _mott(m):
    from .workloads import mott_occupation
    return mott_occupation(m.L, m.N)
