"""Learned-proposal ADAPT against plain full-screen ADAPT on the same GPU.

    python -m paper_2606_05297_gb300.race [--L 10 --d 6] [--max-ops 40]
    python -m paper_2606_05297_gb300.race --target bh --L 8 --U 3.4 --max-ops 150

1. Trace collection: plain ADAPT runs on the Bose-Hubbard L=4 chain (Mott
   start), the L=12 periodic chain at U/J = 3.4 and the Kitaev chain with
   Kerr at L=8, d=8 (vacuum start) store one training list per iteration;
   the scorer is trained on them with the project's own kernels.
2. E0 of the target instance by Lanczos on the device: the Kitaev chain
   with Kerr (t=1, Delta=0.6, K=0.3, open chain; default), or with
   `--target bh` a periodic Bose-Hubbard chain at N = L and the given U/J
   (a chain length the traces do not contain), all-pairs pool, Mott start.
3. Both arms from the same warm start: plain full-screen ADAPT, and learned
   ADAPT (exact screen of the scorer's top k, full screen every
   `full_every` iterations, online training on every full screen).  Each
   arm records wall time and |E - E0| after every iteration and the time at
   which |E - E0| first drops below 1e-1, 1e-2, ..., 1e-6.

Prints one JSON object.  Trace sizes can be reduced with --trace-ops and the
source instances with --small-traces.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

THRESHOLDS = (1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6)


def trace_sources(small: bool):
    from . import workloads as W
    c1 = W.c1_model()
    c2 = W.bose_hubbard(6, 6, J=1.0, U=3.4, periodic=True) if small else W.c2_model(3.4)
    c3 = W.kitaev_kerr(5, 4, t=1.0, Delta=0.5, K=0.1) if small else W.c3_model(0, K=0.1)
    out = []
    for m, warm in ((c1, True), (c2, True), (c3, False)):
        ops = W.hva_layer(m) if warm else []
        out.append((m, W.pool_for(m), W.initial_occupation(m), ops, W.warm_start_thetas(len(ops), 0)))
    return out


def run_arm(make, E0, max_ops, grad_tol=1e-6):
    a = make()
    t0 = time.perf_counter()
    a.optimise_warm_start()
    hist = []
    reached = {}
    for it in range(max_ops):
        rec = a.step(grad_tol=grad_tol)
        t = time.perf_counter() - t0
        if rec is None:
            break
        dE = abs(rec["E"] - E0)
        hist.append(dict(it=it + 1, t=t, dE=dE, op=rec["op"], nfev=rec["nfev"]))
        for th in THRESHOLDS:
            if dE < th and str(th) not in reached:
                reached[str(th)] = dict(seconds=t, iterations=it + 1)
        if dE < THRESHOLDS[-1]:
            break
    return a, hist, reached, time.perf_counter() - t0


def sweep_instances(count: int, seed: int, Ls=(4,), U_range=(1.0, 4.0)):
    """A U/J sweep of small open Bose-Hubbard chains (N = L, Eq. BoseHubbard in
    its literal sign), all-pairs pool, Mott start plus the HVA warm start:
    instances on which ADAPT reaches |E - E0| < 1e-6 within the paper's budget
    of about 160 operators."""
    from . import workloads as W
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        L = int(Ls[q % len(Ls)])
        U = float(np.exp(rng.uniform(np.log(U_range[0]), np.log(U_range[1]))))
        m = W.bose_hubbard(L, L, J=1.0, U=U, periodic=False, name=f"bh_open_L{L}_U{U:.3f}")
        warm = W.hva_layer(m)
        out.append((m, W.bh_allpairs_pool(L), W.mott_occupation(L, L), warm, W.warm_start_thetas(len(warm), seed + q)))
    return out


def _reach(reached, dE, t, it):
    for th in THRESHOLDS:
        if dE < th and str(th) not in reached:
            reached[str(th)] = dict(seconds=t, iterations=it)


def _summary(per, t_total, n):
    """Time at which every instance had reached each threshold (None if some never did)."""
    out = {}
    for th in THRESHOLDS:
        ts = [p["reached"].get(str(th), {}).get("seconds") for p in per]
        out[str(th)] = None if any(t is None for t in ts) else max(ts)
    return dict(seconds=t_total, all_reached=out, instances_reaching_tol=sum(str(THRESHOLDS[-1]) in p["reached"] for p in per),
                instances=n, dE_final=[p["dE"] for p in per], iterations=[p["iterations"] for p in per])


def race_sweep(insts, E0s, scorer, trainer, max_ops=160, hessian_recycling=True, top_k=8, full_every=5,
               tol=1e-6):
    """Wall time to |E - E0| < tol on every instance of a sweep: plain
    full-screen ADAPT run instance after instance, the same method on the
    batched engine (asynchronous rounds: every pending BFGS point of every
    instance in one batched launch, batched screens), and the learned proposal
    on the batched engine."""
    from . import adapt, batched, learned
    n = len(insts)
    arms = {}
    # plain, one instance after another
    t0 = time.perf_counter()
    per = []
    for (m, pool, occ, warm, wth), E0 in zip(insts, E0s):
        A = adapt.Adapt(m, pool, occ, warm, wth, n_max=max_ops + len(warm) + 1, hessian_recycling=hessian_recycling)
        A.optimise_warm_start()
        reached, dE, it = {}, abs(A.trace[-1]["E"] - E0), 0
        _reach(reached, dE, time.perf_counter() - t0, 0)
        while it < max_ops and dE >= tol:
            rec = A.step()
            if rec is None:
                break
            it += 1
            dE = abs(rec["E"] - E0)
            _reach(reached, dE, time.perf_counter() - t0, it)
        per.append(dict(dE=dE, iterations=it, reached=reached))
    arms["plain_sequential"] = _summary(per, time.perf_counter() - t0, n)

    def run_batched(make):
        t0 = time.perf_counter()
        B = make()
        B.optimise_warm_start()
        reached = [dict() for _ in range(n)]
        dE = [abs(B.trace[i][-1]["E"] - E0s[i]) for i in range(n)]
        its = [0] * n
        for i in range(n):
            _reach(reached[i], dE[i], time.perf_counter() - t0, 0)
            if dE[i] < tol:
                B.done[i] = True

        def on_it(i, rec):
            its[i] += 1
            dE[i] = abs(rec["E"] - E0s[i])
            _reach(reached[i], dE[i], time.perf_counter() - t0, its[i])

        B.run(max_ops=max_ops, stop_after=lambda i, rec: abs(rec["E"] - E0s[i]) < tol, on_iteration=on_it)
        per = [dict(dE=dE[i], iterations=its[i], reached=reached[i]) for i in range(n)]
        return B, _summary(per, time.perf_counter() - t0, n)

    models = [x[0] for x in insts]
    pools = [x[1] for x in insts]
    occs = [x[2] for x in insts]
    warms = [x[3] for x in insts]
    wths = [x[4] for x in insts]
    nm = max_ops + max(len(w) for w in warms) + 1
    _, arms["plain_batched"] = run_batched(lambda: batched.BatchedAdapt(
        models, pools, occs, warms, wths, n_max=nm, hessian_recycling=hessian_recycling))
    B, arms["learned_batched"] = run_batched(lambda: learned.LearnedBatchedAdapt(
        models, pools, occs, scorer, trainer=trainer, top_k=top_k, full_every=full_every, warm_ops=warms,
        warm_theta=wths, n_max=nm, hessian_recycling=hessian_recycling))
    st = B.stats
    arms["learned_batched"].update(exact_gradients=st.exact_gradients, full_screens=st.full_screens,
                                   subset_screens=st.subset_screens, judged=st.judged, hits=st.hits)
    return arms


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--target", choices=["kitaev", "bh", "sweep"], default="kitaev")
    ap.add_argument("--count", type=int, default=8, help="instances of the sweep target")
    ap.add_argument("--Ls", type=int, nargs="+", default=[4], help="chain lengths of the sweep target (N = L)")
    ap.add_argument("--U-range", type=float, nargs=2, default=[1.0, 4.0],
                    help="U/J of the sweep target, log-uniform in this range")
    ap.add_argument("--L", type=int, default=10)
    ap.add_argument("--U", type=float, default=3.4, help="U/J of the Bose-Hubbard target")
    ap.add_argument("--d", type=int, default=6)
    ap.add_argument("--max-ops", type=int, default=40)
    ap.add_argument("--trace-ops", type=int, default=20)
    ap.add_argument("--small-traces", action="store_true")
    ap.add_argument("--top-k", type=int, default=8)
    ap.add_argument("--full-every", type=int, default=5)
    ap.add_argument("--train-steps", type=int, default=300)
    ap.add_argument("--hessian-recycling", action="store_true", help="both arms recycle the BFGS inverse Hessian (App. D)")
    a = ap.parse_args(argv)

    import torch
    from . import adapt, cvq, learned
    from . import workloads as W

    t0 = time.perf_counter()
    scorer = cvq.Scorer(65536, seed=1)
    tr = learned.Trainer(scorer, lr=1e-3)
    for (m, pool, occ, wops, wth) in trace_sources(a.small_traces):
        learned.collect_traces(m, pool, occ, tr, warm_ops=wops, warm_theta=wth, max_ops=a.trace_ops, top_k=a.top_k)
    losses = tr.train(a.train_steps)
    t_train = time.perf_counter() - t0

    if a.target == "sweep":
        insts = sweep_instances(a.count, 100, Ls=tuple(a.Ls), U_range=tuple(a.U_range))
        E0s = []
        for (m, *_rest) in insts:
            E0s.append(adapt.ground_energy(cvq.Sector(m)))
        arms = race_sweep(insts, E0s, scorer, tr, max_ops=a.max_ops, hessian_recycling=a.hessian_recycling,
                          top_k=a.top_k, full_every=a.full_every)
        out = dict(target=dict(model=f"open Bose-Hubbard chains L = N in {list(a.Ls)}, U/J log-uniform "
                                     f"[{a.U_range[0]}, {a.U_range[1]}]", max_ops=a.max_ops,
                               instances=[x[0].name for x in insts], E0=E0s, pool="all pairs",
                               tolerance=1e-6),
                   training=dict(lists=len(tr.X), rows=tr.rows(), seconds=t_train,
                                 loss_first=losses[0] if losses else None, loss_last=losses[-1] if losses else None),
                   arms=arms, top_k=a.top_k, full_every=a.full_every, hessian_recycling=a.hessian_recycling)
        print(json.dumps(out), flush=True)
        return out
    if a.target == "bh":
        m = W.bose_hubbard(a.L, a.L, J=1.0, U=a.U, periodic=True)
        pool = W.bh_allpairs_pool(a.L)
        occ = W.mott_occupation(a.L, a.L)
        label = f"bose_hubbard periodic L={a.L} N={a.L} J=1 U={a.U}"
    else:
        m = W.kitaev_kerr(a.L, a.d, t=1.0, Delta=0.6, K=0.3, periodic=False)
        pool = W.bkc_kerr_pool(a.L)
        occ = W.vacuum_occupation(a.L)
        label = f"kitaev_kerr open L={a.L} d={a.d} t=1 Delta=0.6 K=0.3"
    warm = W.hva_layer(m)
    wth = W.warm_start_thetas(len(warm), 0)
    sec = cvq.Sector(m)
    E0 = adapt.ground_energy(sec)
    del sec
    torch.cuda.empty_cache()

    plain, h_plain, r_plain, t_plain = run_arm(
        lambda: adapt.Adapt(m, pool, occ, warm, wth, n_max=a.max_ops + len(warm) + 1,
                            hessian_recycling=a.hessian_recycling), E0, a.max_ops)
    del plain
    torch.cuda.empty_cache()
    la, h_learn, r_learn, t_learn = run_arm(
        lambda: learned.LearnedAdapt(m, pool, occ, scorer, trainer=tr, top_k=a.top_k, full_every=a.full_every,
                                     train_steps=20, warm_ops=warm, warm_theta=wth,
                                     n_max=a.max_ops + len(warm) + 1, hessian_recycling=a.hessian_recycling),
        E0, a.max_ops)
    st = la.stats
    out = dict(
        target=dict(model=label, dim=int(la.sector.dim),
                    pool=len(pool), E0=E0, warm_start_gates=len(warm)),
        training=dict(lists=len(tr.X), rows=tr.rows(), loss_first=losses[0] if losses else None,
                      loss_last=losses[-1] if losses else None, seconds=t_train,
                      sources="Bose-Hubbard L=4 (Mott), " + ("L=6" if a.small_traces else "L=12") +
                              " PBC U/J=3.4, Kitaev+Kerr " + ("L=5 d=4" if a.small_traces else "L=8 d=8")),
        plain=dict(seconds=t_plain, iterations=len(h_plain), dE_final=h_plain[-1]["dE"] if h_plain else None,
                   reached=r_plain, exact_gradients=len(h_plain) * len(pool), history=h_plain),
        learned=dict(seconds=t_learn, iterations=len(h_learn), dE_final=h_learn[-1]["dE"] if h_learn else None,
                     reached=r_learn, exact_gradients=st.exact_gradients, full_screens=st.full_screens,
                     subset_screens=st.subset_screens, judged=st.judged, hits=st.hits,
                     mean_regret=float(np.mean(st.regret)) if st.regret else None, history=h_learn),
        top_k=a.top_k, full_every=a.full_every, hessian_recycling=a.hessian_recycling)
    print(json.dumps(out), flush=True)
    return out


if __name__ == "__main__":
    main()
