"""Learned operator proposal for ADAPT (an extension of the selection step of
Sec. IV.B, whose rule is the largest exact pool gradient, Eq. 12).

Per ADAPT iteration the proposal builds one 32-float input row per pool
operator from cheap state features (<n_r>, <n_r^2> and <a_i^dag a_j>,
computed on the device by cvq_features) and from the operator's history of
exact gradients, scores the rows with the scorer MLP (cvq_mlp_*), screens only
the top_k best-scored operators exactly and appends the largest of those.
Every full_every-th iteration (and whenever the top-k gradients all fall below
the convergence threshold) the whole pool is screened instead: that full
screen is the fallback, measures the proposal's selection error, and adds one
training list to the data on which the scorer keeps training (Adam on the
device, listwise softmax cross-entropy towards the ranking of |g|).

Everything else (warm start, BFGS, stopping rules) is the plain driver's.
"""
from __future__ import annotations

import dataclasses
import math
import time
from typing import List, Optional, Sequence

import numpy as np

from . import cvq
from .adapt import Adapt, BFGS, TIE_REL, select
from .batched import BatchedAdapt
from .workloads import OP_TYPES, Model, Op

NFEAT = 32
HIST = 3
TARGET_POWER = 4.0  # target p_k proportional to (|g_k| / max|g|)^TARGET_POWER


def target_distribution(g) -> np.ndarray:
    a = np.abs(np.asarray(g, dtype=np.float64))
    m = a.max(initial=0.0)
    if m <= 0.0:
        return np.full(a.size, 1.0 / max(a.size, 1))
    p = (a / m) ** TARGET_POWER
    return p / p.sum()


def _log_scaled(v: float) -> float:
    return min(max((math.log10(max(v, 1e-16)) + 16.0) / 16.0, 0.0), 1.5)


class FeatureBuilder:
    """Input rows of the scorer for one pool on one sector."""

    def __init__(self, model: Model, pool_ops: Sequence[Op]):
        self.model = model
        self.ops = list(pool_ops)
        self.K = len(self.ops)
        self.D = float(model.N + 1 if model.kind == "bh" else model.d)
        pairs = sorted({(o.i, o.j) for o in self.ops if o.j >= 0})
        self.pairs = pairs
        self.pair_index = {p: k for k, p in enumerate(pairs)}
        L = model.L
        self.static = np.zeros((self.K, NFEAT), dtype=np.float32)
        for k, o in enumerate(self.ops):
            self.static[k, OP_TYPES.index(o.type)] = 1.0
            self.static[k, 8] = o.phase / 3.0
            self.static[k, 9] = 1.0 if o.j < 0 else 0.0
            if o.j >= 0:
                d = abs(o.i - o.j)
                if model.periodic:
                    d = min(d, L - d)
                self.static[k, 19] = d / L

    def rows(self, feats: np.ndarray, hist: "History", it_frac: float) -> np.ndarray:
        L, D = self.model.L, self.D
        n1 = feats[:L]
        n2 = feats[L:2 * L]
        var = np.sqrt(np.maximum(n2 - n1 * n1, 0.0))
        cor = feats[2 * L:].reshape(-1, 2)
        X = self.static.copy()
        for k, o in enumerate(self.ops):
            X[k, 10] = n1[o.i] / D
            X[k, 12] = var[o.i] / D
            X[k, 14] = n2[o.i] / (D * D)
            if o.j >= 0:
                X[k, 11] = n1[o.j] / D
                X[k, 13] = var[o.j] / D
                X[k, 15] = n2[o.j] / (D * D)
                c = cor[self.pair_index[(o.i, o.j)]]
                X[k, 16] = c[0] / D
                X[k, 17] = c[1] / D
                X[k, 18] = math.hypot(c[0], c[1]) / D
        X[:, 20:26] = hist.block()
        X[:, 26] = it_frac
        X[:, 27] = np.minimum(hist.selected / 5.0, 2.0)
        X[:, 28] = 0.0
        if hist.last_op is not None:
            X[hist.last_op, 28] = 1.0
        X[:, 29] = _log_scaled(hist.last_gmax)
        X[:, 30] = _log_scaled(hist.last_dE)
        X[:, 31] = np.minimum(hist.age / 5.0, 2.0)
        return X


class History:
    """Per-operator record of the last HIST exact |g| values."""

    def __init__(self, K: int):
        self.g = np.zeros((K, HIST))
        self.mask = np.zeros((K, HIST))
        self.age = np.full(K, 10.0)
        self.selected = np.zeros(K)
        self.last_op: Optional[int] = None
        self.last_gmax = 0.0
        self.last_dE = 0.0

    def tick(self):
        self.age += 1.0

    def record(self, idx, g):
        idx = np.asarray(idx, dtype=np.int64)
        self.g[idx, 1:] = self.g[idx, :-1]
        self.mask[idx, 1:] = self.mask[idx, :-1]
        self.g[idx, 0] = np.abs(g)
        self.mask[idx, 0] = 1.0
        self.age[idx] = 0.0

    def block(self) -> np.ndarray:
        out = np.zeros((self.g.shape[0], 2 * HIST), dtype=np.float32)
        lg = (np.log10(np.maximum(self.g, 1e-16)) + 16.0) / 16.0
        out[:, :HIST] = np.clip(lg, 0.0, 1.5) * self.mask
        out[:, HIST:] = self.mask
        return out


class Trainer:
    """Listwise training of a cvq.Scorer on device-resident lists."""

    def __init__(self, scorer: "cvq.Scorer", lr: float = 1e-3):
        self.scorer = scorer
        self.lr = lr
        self.X: List[np.ndarray] = []
        self.P: List[np.ndarray] = []
        self.G: List[np.ndarray] = []

    def add(self, X: np.ndarray, g) -> None:
        self.X.append(np.asarray(X, dtype=np.float32))
        self.P.append(target_distribution(g).astype(np.float32))
        self.G.append(np.abs(np.asarray(g, dtype=np.float64)))

    def rows(self) -> int:
        return sum(x.shape[0] for x in self.X)

    def train(self, steps: int, max_rows: Optional[int] = None) -> List[float]:
        """Full-batch Adam steps over every stored list (newest lists kept when
        the rows exceed the scorer's capacity).  Returns the mean loss per step."""
        import torch
        if not self.X or steps <= 0:
            return []
        cap = self.scorer.max_rows if max_rows is None else min(max_rows, self.scorer.max_rows)
        keep, tot = [], 0
        for k in range(len(self.X) - 1, -1, -1):
            if tot + self.X[k].shape[0] > cap:
                break
            keep.append(k)
            tot += self.X[k].shape[0]
        keep.reverse()
        X = torch.from_numpy(np.concatenate([self.X[k] for k in keep])).cuda()
        P = torch.from_numpy(np.concatenate([self.P[k] for k in keep])).cuda()
        off = np.concatenate([[0], np.cumsum([self.X[k].shape[0] for k in keep])]).astype(np.int32)
        off_d = torch.from_numpy(off).cuda()
        losses = torch.empty(steps, dtype=torch.float32, device="cuda")
        for s in range(steps):
            scores = self.scorer.forward(X)
            loss, ds = cvq.listwise_loss(scores, P, off_d)
            losses[s] = loss.mean()
            ds.div_(len(keep))
            self.scorer.backward(X, ds)
            self.scorer.adam_step(self.lr)
        return losses.cpu().tolist()


@dataclasses.dataclass
class ProposalStats:
    full_screens: int = 0
    subset_screens: int = 0
    exact_gradients: int = 0
    judged: int = 0              # full screens at which the proposal's choice could be judged
    hits: int = 0                # ... and the true argmax was among its top_k
    regret: List[float] = dataclasses.field(default_factory=list)  # 1 - |g(choice)| / max|g|


class LearnedAdapt(Adapt):
    """ADAPT whose operator choice comes from the scorer's top_k, with a full
    screen every full_every iterations."""

    def __init__(self, model: Model, pool_ops: Sequence[Op], init_occ: Sequence[int], scorer: "cvq.Scorer",
                 trainer: Optional[Trainer] = None, top_k: int = 8, full_every: int = 5, train_steps: int = 20,
                 max_ops_hint: int = 160, **kw):
        super().__init__(model, pool_ops, init_occ, **kw)
        self.scorer = scorer
        self.trainer = trainer
        self.top_k = top_k
        self.full_every = full_every
        self.train_steps = train_steps
        self.max_ops_hint = max_ops_hint
        self.fb = FeatureBuilder(model, pool_ops)
        self.hist = History(self.K)
        self.stats = ProposalStats()
        self.n_adapt = 0
        self._X = None
        import torch
        self._Xd = torch.empty((self.K, NFEAT), dtype=torch.float32, device="cuda")

    def _features(self, psi) -> np.ndarray:
        f = cvq.features(self.sector, psi, self.fb.pairs, stream=self.stream)
        return f.cpu().numpy()

    def _scores(self, X) -> np.ndarray:
        self._Xd.copy_(self.torch.from_numpy(X))
        return self.scorer.forward(self._Xd, stream=self.stream).cpu().numpy()

    def propose(self, psi):
        X = self.fb.rows(self._features(psi), self.hist, self.n_adapt / self.max_ops_hint)
        s = self._scores(X)
        order = np.lexsort((np.arange(self.K), -s))  # best score first, lowest index on ties
        return X, order[: self.top_k]

    def _full(self, psi, X, top):
        g = self.screen(psi)
        self.stats.full_screens += 1
        self.stats.exact_gradients += self.K
        self.hist.record(np.arange(self.K), g)
        k, gmax = select(g)
        if top is not None and gmax > 0.0:
            self.stats.judged += 1
            self.stats.hits += int(k in set(int(t) for t in top))
            sub = np.abs(g[top])
            self.stats.regret.append(1.0 - float(sub.max()) / gmax)
        if self.trainer is not None:
            self.trainer.add(X, g)
            self.trainer.train(self.train_steps)
        return k, gmax

    def step(self, grad_tol=1e-6, max_iter=1000, g=None):
        t0 = time.perf_counter()
        psi = self.state()
        X, top = self.propose(psi)
        if self.n_adapt % self.full_every == 0:
            k, gmax = self._full(psi, X, top)
        else:
            sub = [int(t) for t in top]
            gs = self.screen(psi, subset=sub)
            self.stats.subset_screens += 1
            self.stats.exact_gradients += len(sub)
            self.hist.record(sub, gs)
            a = np.abs(gs)
            m = float(a.max())
            cand = [sub[j] for j in np.nonzero(a >= m * (1.0 - TIE_REL))[0]]
            k, gmax = min(cand), m
            if gmax < grad_tol:  # the proposal sees nothing left: confirm with the whole pool
                k, gmax = self._full(psi, X, None)
        self.hist.tick()
        if gmax < grad_tol:
            return None
        E_before = self.trace[-1]["E"] if self.trace else None
        rec = self._grow(k, gmax, max_iter, t0)
        self.hist.selected[k] += 1
        self.hist.last_op = k
        self.hist.last_gmax = gmax
        self.hist.last_dE = abs(rec["E"] - E_before) if E_before is not None else 0.0
        self.n_adapt += 1
        return rec


def collect_traces(model: Model, pool_ops: Sequence[Op], init_occ: Sequence[int], trainer: Trainer,
                   warm_ops: Sequence[Op] = (), warm_theta: Sequence[float] = (), max_ops: int = 30,
                   grad_tol: float = 1e-6, top_k: int = 8, full_every: int = 5, max_ops_hint: int = 160,
                   bfgs_max_iter: int = 1000) -> dict:
    """Run plain full-screen ADAPT on one instance and store one training list
    per iteration: the scorer's input rows (with the operator history the
    learned driver would have, i.e. refreshed for the whole pool every
    full_every-th iteration and for the top_k largest |g| otherwise) and the
    exact |g| of the full screen."""
    ad = Adapt(model, pool_ops, init_occ, warm_ops=warm_ops, warm_theta=warm_theta)
    ad.optimise_warm_start()
    fb = FeatureBuilder(model, pool_ops)
    hist = History(ad.K)
    lists = 0
    E_prev = ad.trace[-1]["E"] if ad.trace else None
    for it in range(max_ops):
        psi = ad.state()
        feats = cvq.features(ad.sector, psi, fb.pairs).cpu().numpy()
        X = fb.rows(feats, hist, it / max_ops_hint)
        g = ad.screen(psi)
        trainer.add(X, g)
        lists += 1
        k, gmax = select(g)
        if gmax < grad_tol:
            break
        if it % full_every == 0:
            hist.record(np.arange(ad.K), g)
        else:
            top = np.lexsort((np.arange(ad.K), -np.abs(g)))[:top_k]
            hist.record(top, g[top])
        hist.tick()
        rec = ad._grow(k, gmax, bfgs_max_iter, time.perf_counter())
        hist.selected[k] += 1
        hist.last_op, hist.last_gmax = k, gmax
        hist.last_dE = abs(rec["E"] - E_prev) if E_prev is not None else 0.0
        E_prev = rec["E"]
    return dict(lists=lists, E=ad.energy(), n=len(ad.ids))


def hit_rate(scorer: "cvq.Scorer", Xs: Sequence[np.ndarray], gs: Sequence[np.ndarray], top_k: int = 8) -> float:
    """Fraction of lists whose exact argmax |g| is among the scorer's top_k."""
    import torch
    hits = 0
    for X, g in zip(Xs, gs):
        s = scorer.forward(torch.from_numpy(np.asarray(X, dtype=np.float32)).cuda()).cpu().numpy()
        top = np.lexsort((np.arange(len(s)), -s))[:top_k]
        hits += int(select(g)[0] in set(int(t) for t in top))
    return hits / max(len(Xs), 1)


class LearnedBatchedAdapt(BatchedAdapt):
    """Learned proposal on the batched engine: lockstep ADAPT over many
    instances (a U/J sweep) in which every iteration makes one scorer forward
    over the pool rows of every live instance, one batched exact screen of
    each instance's top_k (its whole pool every full_every-th iteration of
    that instance, and whenever its top_k gradients all fall below the
    threshold), and one lockstep BFGS whose evaluations share batched graph
    launches.  The scorer keeps training on every full screen."""

    def __init__(self, models: Sequence[Model], pool_ops: Sequence[Sequence[Op]], init_occ, scorer: "cvq.Scorer",
                 trainer: Optional[Trainer] = None, top_k: int = 8, full_every: int = 5, train_steps: int = 20,
                 max_ops_hint: int = 160, **kw):
        import torch
        super().__init__(models, pool_ops, init_occ, **kw)
        self.scorer = scorer
        self.trainer = trainer
        self.top_k = top_k
        self.full_every = full_every
        self.train_steps = train_steps
        self.max_ops_hint = max_ops_hint
        self.fbs = [FeatureBuilder(m, p) for m, p in zip(models, pool_ops)]
        self.hists = [History(K) for K in self.K]
        self.n_adapt = [0] * len(models)
        self.stats = ProposalStats()
        self.state_ws = [s.workspace(p, self.n_max) for s, p in zip(self.sectors, self.pools)]
        self._Xd = torch.empty((max(sum(self.K), 1), NFEAT), dtype=torch.float32, device="cuda")

    def _rows(self, live):
        rows = {}
        for i in live:
            psi = cvq.apply_ansatz(self.sectors[i], self.pools[i], self.ids[i], self.theta[i], self.psi0[i],
                                   ws=self.state_ws[i])
            f = cvq.features(self.sectors[i], psi, self.fbs[i].pairs).cpu().numpy()
            rows[i] = self.fbs[i].rows(f, self.hists[i], self.n_adapt[i] / self.max_ops_hint)
        return rows

    def _full_screen(self, i, X, g, top):
        self.stats.full_screens += 1
        self.stats.exact_gradients += self.K[i]
        self.hists[i].record(np.arange(self.K[i]), g)
        k, gmax = select(g)
        if top is not None and gmax > 0.0:
            self.stats.judged += 1
            self.stats.hits += int(k in set(int(t) for t in top))
            self.stats.regret.append(1.0 - float(np.abs(g[top]).max()) / gmax)
        if self.trainer is not None:
            self.trainer.add(X, g)
        return k, gmax

    def choose(self, grad_tol: float, which=None):
        torch = self.torch
        n = len(self.ids)
        live = [i for i in range(n) if not self.done[i] and (which is None or i in which)]
        if not live:
            return {}
        rows = self._rows(live)
        Xcat = np.concatenate([rows[i] for i in live]).astype(np.float32)
        self._Xd[: Xcat.shape[0]].copy_(torch.from_numpy(Xcat))
        s_all = self.scorer.forward(self._Xd[: Xcat.shape[0]]).cpu().numpy()
        top, o = {}, 0
        for i in live:
            s = s_all[o:o + self.K[i]]
            o += self.K[i]
            top[i] = np.lexsort((np.arange(self.K[i]), -s))[: self.top_k]
        full = {i: self.n_adapt[i] % self.full_every == 0 for i in live}
        subs = [[] for _ in range(n)]
        for i in live:
            subs[i] = list(range(self.K[i])) if full[i] else [int(t) for t in top[i]]
        gs = self.screen_all(subs, which=set(live))
        chosen, confirm, trained = {}, [], False
        for i in live:
            g = gs[i]
            if full[i]:
                chosen[i] = self._full_screen(i, rows[i], g, top[i])
                trained = True
                continue
            sub = subs[i]
            self.stats.subset_screens += 1
            self.stats.exact_gradients += len(sub)
            self.hists[i].record(sub, g)
            a = np.abs(g)
            m = float(a.max())
            if m < grad_tol:  # the proposal sees nothing left: confirm with the whole pool
                confirm.append(i)
                continue
            chosen[i] = (min(sub[j] for j in np.nonzero(a >= m * (1.0 - TIE_REL))[0]), m)
        if confirm:
            subs2 = [list(range(self.K[i])) if i in confirm else [] for i in range(n)]
            gs2 = self.screen_all(subs2, which=set(confirm))
            for i in confirm:
                chosen[i] = self._full_screen(i, rows[i], gs2[i], None)
                trained = True
        if trained and self.trainer is not None:
            self.trainer.train(self.train_steps)
        for i in live:
            self.hists[i].tick()
        for i in list(chosen):
            if chosen[i][1] < grad_tol or len(self.ids[i]) + 1 > self.n_max:
                self.done[i] = True
                del chosen[i]
        return chosen

    def after_step(self, grown):
        for i, (k, gmax) in grown.items():
            tr = [r for r in self.trace[i]]
            E_before = tr[-2]["E"] if len(tr) >= 2 else None
            h = self.hists[i]
            h.selected[k] += 1
            h.last_op = k
            h.last_gmax = gmax
            h.last_dE = abs(tr[-1]["E"] - E_before) if E_before is not None else 0.0
            self.n_adapt[i] += 1
