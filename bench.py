#!/usr/bin/env python
"""Benchmark: ADAPT iterations/s of plain full-screen CV-ADAPT-VQE on GB300.

Workload (default): Bose-Hubbard periodic chain L=12, N=12 (fixed-N sector of
1,352,078 complex128 amplitudes), J=1, U/J in {1, 3.4, 10} (Eq. BoseHubbard,
literal -U/2 sign), all-pairs number-conserving pool of 210 generators,
start |1^12> plus one HVA warm-start layer (36 gates).  One step = one ADAPT
iteration (screen of the whole pool, selection, BFGS re-optimisation of every
parameter) on each of the three instances.  Warm-up steps are the first W
ADAPT iterations; the next K are timed.  The sector state (21.6 MB) fits in
L2, so a 256 MB buffer is written between timed steps.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ADAPT iters/s (plain full-screen CV-ADAPT-VQE)"
UNIT = "ADAPT iterations/s"
U_VALUES = (1.0, 3.4, 10.0)
WORKLOAD = "bose_hubbard_pbc_L12_N12_dim1352078_UJ1,3.4,10_pool210_plain_adapt"
# FP64 pipe of a GB300: 2 DFMA per clock per SM (nominal 1.25 TFLOP/s at the
# 2070 MHz maximum clock over 152 SMs); see the design notes.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-c4", action="store_true", help="skip the batched 64-instance sweep measurement")
    ap.add_argument("--instances", type=int, default=len(U_VALUES),
                    help="use the first n of the U/J instances (profiling runs)")
    a = ap.parse_args()
    if not 1 <= a.instances <= len(U_VALUES):
        ap.error(f"--instances must be in [1, {len(U_VALUES)}]")
    if a.warmup < 3:
        ap.error("--warmup must be >= 3")
    return a


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.rows = []
        self.proc = None
        self.index = index

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if len(r) >= 8 and r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if len(r) >= 8 and r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows if len(r) >= 8 for k in range(4) if r[4 + k] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def dist_init(args):
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return rank, ws, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(x, ws, op):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"  # gloo reduces host tensors
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x, ws):
    import torch.distributed as dist
    return _reduce(x, ws, dist.ReduceOp.MAX)


def sum_over_ranks(x, ws):
    import torch.distributed as dist
    return _reduce(x, ws, dist.ReduceOp.SUM)


# Sources each measured kernel is compiled from: a committed traffic figure
# stands only while these are unchanged.
KERNEL_SOURCES = {
    "adjoint_block": ["k_gate_impl.cuh", "k_gate_bh_adj.cu", "k_gate_bkc_adj.cu", "cvq_internal.cuh", "df.cuh"],
}


def csrc_hash(files=None):
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2606_05297_gb300", "csrc")
    for f in sorted(files if files is not None else os.listdir(d)):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was captured on the kernel's current sources."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(p) as f:
            d = json.load(f)
        e = d["kernels"].get(kernel)
        if e is None or e.get("sources_hash") != csrc_hash(KERNEL_SOURCES.get(kernel)):
            return None
        return float(e["dram_bytes_per_launch_full_size"])
    except Exception:
        return None


# ------------------------------------------------------------ oracle timing

def oracle_sample(n_gates: int, nfev: float, K: int = 210, U=3.4):
    """Time the FP64 oracle on a bounded sample of the workload: one H psi and
    one beam-splitter gate exp(theta A) psi on the full L=12, N=12 state, then
    scale to one ADAPT iteration: a full screen (K applications of H inside
    the Eq. (grad) commutators dominate) plus nfev energy-and-gradient
    evaluations, each about 2 n gate applications and one H psi."""
    import numpy as np
    from oracle.core import Sector as OS
    from paper_2606_05297_gb300 import workloads as W
    m = W.c2_model(U)
    s = OS(m)
    psi = W.random_state(s.dim, 5)
    t0 = time.perf_counter()
    s.apply_H(psi)
    tH = time.perf_counter() - t0
    t0 = time.perf_counter()
    s.expm_apply(W.Op("hop", 0, 1, 0), 0.1, psi)
    tg = time.perf_counter() - t0
    t_iter = K * tH + nfev * (2 * n_gates * tg + tH)
    return dict(t_H=tH, t_gate=tg, t_iter=t_iter, sample_seconds=tH + tg)


# ------------------------------------------------------------ our arm

def run_ours(args):
    import numpy as np
    import torch
    from paper_2606_05297_gb300 import cvq
    from paper_2606_05297_gb300 import workloads as W
    from paper_2606_05297_gb300.adapt import Adapt, ground_energy

    rank, ws, local = dist_init(args)
    stream = torch.cuda.current_stream()
    insts = []
    for u in U_VALUES[: args.instances]:
        m = W.c2_model(u)
        pool = W.bh_allpairs_pool(m.L)
        warm = W.hva_layer(m)
        th = W.warm_start_thetas(len(warm), 1000 * rank + int(10 * u))
        A = Adapt(m, pool, W.mott_occupation(m.L, m.N), warm, th, n_max=160)
        A.optimise_warm_start()
        A.E0 = ground_energy(A.sector)
        insts.append(A)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def one_step():
        recs = []
        for A in insts:
            r = A.step()
            recs.append(r)
        return recs

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()

    # the e2e leg below repeats exactly these iterations from this state
    snap = [(list(A.ids), A.theta.copy(), len(A.trace), A.Hinv) for A in insts]

    # ---- timed, device-resident
    sampler = ClockSampler(local)
    barrier(ws)
    torch.cuda.synchronize()
    sampler.start()
    torch.cuda.profiler.start()  # the timed region, for profilers started with --profile-from-start off
    cvq.profile_sample(16)  # one event pair per 16 launches of a kind keeps the launch path short
    cvq.profile_start(400000)
    total_ms = 0.0
    iters = 0
    nfev, ngates = [], []
    for k in range(args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        recs = one_step()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        for r in recs:
            if r is not None:
                iters += 1
                nfev.append(r["nfev"])
                ngates.append(r["n"])
    stats = cvq.profile_stop()
    torch.cuda.profiler.stop()
    clocks = sampler.stop()
    torch.cuda.synchronize()
    barrier(ws)
    t_max = max_over_ranks(total_ms / 1e3, ws)
    iters_all = sum_over_ranks(float(iters), ws)
    value = iters_all / t_max

    # ---- e2e: same metric through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        for A, (ids, th, nt, Hi) in zip(insts, snap):
            A.ids, A.theta, A.Hinv = list(ids), th.copy(), Hi
            del A.trace[nt:]
        host_psi = [A.psi0.cpu().pin_memory() for A in insts]
        host_out = torch.empty(len(insts) * 161, dtype=torch.float64, pin_memory=True)
        bi = sum(h.numel() * 16 for h in host_psi)
        e_ms, e_it, bo = 0.0, 0, 0
        for k in range(args.steps):
            flush.fill_(float(k))
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            bo = 0
            for A, hp in zip(insts, host_psi):
                A.psi0.copy_(hp, non_blocking=True)
                r = A.step()
                n = len(A.ids)
                host_out[bo // 8: bo // 8 + n + 1].copy_(A._out[: n + 1], non_blocking=True)
                bo += 8 * (n + 1)
                e_it += r is not None
            e1.record(stream)
            e1.synchronize()
            e_ms += e0.elapsed_time(e1)
        e_t = max_over_ranks(e_ms / 1e3, ws)
        e2e = {"value": sum_over_ranks(float(e_it), ws) / e_t, "unit": UNIT, "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bo, "iterations": "the timed iterations again, from the same state"}

    # ---- roofline of the dominant kernel
    dom = max(stats.items(), key=lambda kv: kv[1]["ms"])
    name, st = dom
    hbm, src = peaks()
    intensity = st["flops"] / max(st["bytes"], 1.0)
    ridge = FP64_PEAK_TFLOPS * 1e12 / (hbm * 1e9)
    per_launch_s = st["ms"] / 1e3 / st["launches"]
    if intensity > ridge:
        achieved = st["flops"] / st["launches"] / per_launch_s / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "pipe": "fp64 (DFMA)",
                "peak_source": "derived: 2 DFMA/clk/SM x 152 SMs x 2070 MHz"}
    else:
        achieved = st["bytes"] / st["launches"] / per_launch_s / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "peak_source": f"{src} MEASURED_PEAKS.json hbm_gbs"}
    roof["kernel"] = name
    roof["traffic"] = measured_traffic(name)
    roof["algorithmic_bytes_per_launch"] = st["bytes"] / st["launches"]
    roof["algorithmic_flops_per_launch"] = st["flops"] / st["launches"]
    roof["avg_launch_us"] = per_launch_s * 1e6
    launches = int(sum(v["launches"] for v in stats.values()))

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        smp = oracle_sample(int(np.mean(ngates)), float(np.mean(nfev)))
        cpu = {"value": 1.0 / smp["t_iter"], "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": (f"one H psi ({smp['t_H']:.2f} s) and one beam-splitter exp(theta A) psi "
                          f"({smp['t_gate']:.2f} s) of the FP64 oracle on the full U/J=3.4 state, scaled to an "
                          f"ADAPT iteration as 210 H applications (screen) + nfev={np.mean(nfev):.1f} x "
                          f"(2 x n={np.mean(ngates):.1f} gates + 1 H)")}

    # ---- batched engine on the 64-instance sweep (outside the timed ADAPT region)
    c4 = None
    if not args.no_c4:
        # every rank evaluates its own shard of the 64 instances (no collective on the data path)
        from paper_2606_05297_gb300 import batched
        c4 = batched.measure_c4(reps=3, sequential=(ws == 1), rank=rank, world=ws)
        barrier(ws)
        t_eval = max_over_ranks(c4["ms_per_eval_batched"], ws)
        c4["instances_per_rank"] = c4.pop("instances")
        c4["ms_per_eval_batched"] = t_eval
        c4["evals_per_s_batched"] = 64 * 1e3 / t_eval
        c4["scaling"] = "strong (64 instances split over the ranks)"
        c4["workload"] = ("64 Bose-Hubbard instances, L ~ U{8..12}, N = L, U/J log-uniform [0.5, 20], PBC, "
                          "all-pairs pool, HVA layer + 8 pool operators each; energy and adjoint gradient of every "
                          "instance per evaluation")

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64 (complex128 states)", "data": "synthetic",
            "config": {"workload": WORKLOAD if len(insts) == len(U_VALUES) else
                       WORKLOAD.replace("UJ1,3.4,10", "UJ" + ",".join(f"{u:g}" for u in U_VALUES[: len(insts)])),
                       "instances_per_rank": len(insts), "dim": insts[0].sector.dim,
                       "pool": insts[0].K, "warm_start_gates": 36, "l2": "256 MB buffer written between steps",
                       "ansatz_len_mean": float(np.mean(ngates)), "bfgs_evals_per_iter_mean": float(np.mean(nfev)),
                       "dE_last": [abs(A.trace[-1]["E"] - A.E0) for A in insts], "parallelism": f"replicas x{ws}"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
            "c4_batched": c4,
            "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 3)} for k, v in stats.items()},
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------------ reference arm

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    n_gates, nfev = 40, 60.0
    for _ in range(args.warmup):
        pass  # the oracle has no warm-up state; warm-up steps are not repeated work
    t = 0.0
    samp = None
    for _ in range(args.steps):
        samp = oracle_sample(n_gates, nfev)
        t += samp["t_iter"]
    value = args.steps / t
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD, "ansatz_len": n_gates, "bfgs_evals_per_iter": nfev},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "per step: one H psi and one beam-splitter gate of the FP64 oracle on the full "
                                   "L=12, N=12 state, scaled to one ADAPT iteration (210 H applications for the "
                                   f"screen + {nfev:.0f} evaluations x (2 x {n_gates} gates + 1 H))"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
