"""A fixed, kernel-focused case for profilers: repeated energy-and-gradient
evaluations of a random ansatz on one workload.

    python -m paper_2606_05297_gb300.profile_case --workload bh12 --depth 40 --reps 3 [--warm 5] [--stored]
        [--op hop:6:7:1]

Workloads: bh12 (Bose-Hubbard L=12, N=12 periodic, 1,352,078 amplitudes),
bkc8 (Kitaev chain + Kerr L=8, d=8, 8,388,608 amplitudes), bkc10 (L=10, d=6,
30,233,088 amplitudes).  Each repetition runs one cvq_energy_and_grad call
(depth forward gates, one H psi, depth reverse steps) and one pool screen.
mlp: each repetition runs one forward and one backward of the proposal
scorer on a 210-row pool (the L=10 Kitaev pool's size).  c4: each repetition
is one batched energy-and-gradient evaluation of the 64-instance Bose-Hubbard
sweep (one graph launch).
"""
from __future__ import annotations

import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def make(workload: str):
    from paper_2606_05297_gb300 import workloads as W
    if workload == "bh12":
        m = W.c2_model(3.4)
        return m, W.bh_allpairs_pool(m.L)
    if workload == "bkc8":
        m = W.c3_model(0, K=0.1)
        return m, W.bkc_kerr_pool(m.L)
    if workload == "bkc10":
        m = W.c5_model()
        return m, W.bkc_kerr_pool(m.L)
    raise ValueError(workload)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="bh12", choices=["bh12", "bkc8", "bkc10", "mlp", "c4"])
    ap.add_argument("--depth", type=int, default=40)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--warm", type=int, default=0, help="unprofiled repetitions before cudaProfilerStart")
    ap.add_argument("--kernels", action="store_true", help="print per-kernel event timings of the profiled range")
    ap.add_argument("--op", default=None,
                    help="one pool element, type:i:j:phase (e.g. hop:6:7:1), repeated --depth times instead of a "
                         "random ansatz")
    ap.add_argument("--stored", action="store_true",
                    help="keep the forward states for the reverse sweep (cvq_energy_and_grad_stored)")
    ap.add_argument("--projected", type=int, default=0,
                    help="Kitaev workloads: projected gates with this inner cutoff (Sec. V.A) instead of truncated ones")
    a = ap.parse_args()
    import torch
    from paper_2606_05297_gb300 import build, cvq
    from paper_2606_05297_gb300 import workloads as W
    build.build()
    if a.workload == "c4":  # the 64-instance sweep: batched evaluations (tile 4096, 2 CTAs per SM)
        import numpy as np
        from paper_2606_05297_gb300 import batched
        data = batched.c4_batch_inputs(a.seed, 64, 8)
        sectors = [cvq.Sector(m) for m, _, _, _ in data]
        pools = [cvq.Pool(s, ops) for s, (_, ops, _, _) in zip(sectors, data)]
        psi0 = [s.basis_state(W.mott_occupation(m.L, m.N)) for s, (m, _, _, _) in zip(sectors, data)]
        b = cvq.Batch(sectors, pools, max(len(ids) for _, _, ids, _ in data))
        b.set_ansatz([ids for _, _, ids, _ in data], psi0)
        flat = np.concatenate([th for _, _, _, th in data])
        b.theta[: flat.size].copy_(torch.from_numpy(flat))
        b.set_schedule(4096, 2)
        for _ in range(max(a.warm, 1)):
            b.energy_and_grad()
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        t0 = time.perf_counter()
        for _ in range(a.reps):
            E, _g = b.energy_and_grad()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        torch.cuda.profiler.stop()
        print(f"c4: instances=64 amplitudes={sum(s.dim for s in sectors)} {b.info()} E[0]={E[0].item():.12f} "
              f"{dt / a.reps * 1e3:.2f} ms/eval")
        return
    if a.workload == "mlp":
        sc = cvq.Scorer(210, seed=a.seed)
        X = torch.from_numpy(W.scorer_inputs(210, a.seed + 1)).cuda()
        ds = torch.ones(210, dtype=torch.float32, device="cuda")
        for _ in range(a.warm):
            sc.forward(X)
            sc.backward(X, ds)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        t0 = time.perf_counter()
        for _ in range(a.reps):
            out = sc.forward(X)
            sc.backward(X, ds)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(f"mlp: rows=210 reps={a.reps} score[0]={out[0].item():.6f} "
              f"{(time.perf_counter() - t0) / a.reps * 1e6:.1f} us/rep (forward + backward)")
        return
    m, pool = make(a.workload)
    s = cvq.Sector(m)
    p = cvq.ProjectedPool(s, pool, a.projected) if a.projected else cvq.Pool(s, pool)
    ids, th = W.random_ansatz(len(pool), a.depth, a.seed, scale=0.2)
    if a.op is not None:
        t, i, j, ph = a.op.split(":")
        want = (t, int(i), int(j) if j else -1, int(ph))
        k = [q for q, o in enumerate(pool) if (o.type, o.i, o.j, o.phase) == want]
        if not k:
            raise SystemExit(f"no pool element {a.op}")
        ids = [k[0]] * a.depth
    psi0 = torch.from_numpy(W.random_state(s.dim, a.seed + 1)).cuda()
    ws = s.workspace(p, a.depth)
    if a.projected:
        eg = cvq.energy_and_grad_projected
    elif a.stored:
        states = torch.empty(max(cvq.stored_states_bytes(s, p, ids), 1), dtype=torch.uint8, device="cuda")

        def eg(s_, p_, ids_, th_, psi0_, ws=None):
            return cvq.energy_and_grad_stored(s_, p_, ids_, th_, psi0_, states=states, ws=ws)
    else:
        eg = cvq.energy_and_grad
    for _ in range(a.warm):
        eg(s, p, ids, th, psi0, ws=ws)
        cvq.screen_pool(s, p, psi0, ws=ws)
    torch.cuda.synchronize()
    torch.cuda.profiler.start()  # profiled range, for profilers started with --profile-from-start off
    if a.kernels:
        cvq.profile_start(1 << 16)
    t0 = time.perf_counter()
    for _ in range(a.reps):
        E, g = eg(s, p, ids, th, psi0, ws=ws)
        cvq.screen_pool(s, p, psi0, ws=ws)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    torch.cuda.profiler.stop()
    if a.kernels:
        for name, st in sorted(cvq.profile_stop().items(), key=lambda kv: -kv[1]["ms"]):
            us = st["ms"] * 1e3 / st["launches"]
            print(f"  {name:16s} {st['launches']:6d} launches {us:9.1f} us/launch "
                  f"{st['bytes'] / st['ms'] / 1e6:8.1f} GB/s {st['flops'] / st['ms'] / 1e9:7.2f} TFLOP/s")
    print(f"{a.workload}: dim={s.dim} depth={a.depth} reps={a.reps} E={E.item():.12f} "
          f"|g|={g.abs().max().item():.6e} {dt / a.reps * 1e3:.2f} ms/rep")


if __name__ == "__main__":
    main()
