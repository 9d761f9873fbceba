"""Write the stored expected values of the full-size parity tests (test
infrastructure).

Every value comes from the FP64 oracle in this directory; inputs come from
the seeded generators of paper_2606_05297_gb300.workloads, which hold none of
the method's arithmetic.  The GPU tests rebuild the same inputs from the same
seeds and compare their results with these files, so the slow oracle runs
(minutes to an hour at the full sector sizes) happen once, here, and not on
every test run.

    python -m oracle.make_golden [name ...]     (default: every target)

Targets (files under tests/golden/):
  c1_adapt      Bose-Hubbard open chain L=4, N=4, U=2 from |1111> with the HVA
                warm start, ADAPT to max|g| < 1e-6 (Sec. IV.B), with the
                dense exact-diagonalisation E0 (Sec. IV.B stopping rule) and
                the parameters of the state each operator was chosen on.
  c2_screen     Bose-Hubbard periodic L=12, N=12, U/J=3.4: Eq. (grad) for all
                210 pool elements on a random state.
  c2_depth40    the same sector: E and dE/dtheta (Sec. IV.A/B) of a random
                40-gate ansatz applied to a random state.
  c3_depth40    Kitaev chain with Kerr term, open L=8, d=8: E and dE/dtheta of
                a random 40-gate ansatz from the vacuum.
  c5_depth10    Kitaev chain with Kerr term, open L=10, d=6: E and dE/dtheta of
                a random 10-gate ansatz from the vacuum, and Eq. (grad) for 16
                pool elements on a random state.
  bkck_depth160 Kitaev chain with Kerr term, open L=6, d=6: E and dE/dtheta of
                a random 160-gate ansatz (the paper's gate budget of about 160,
                Sec. IV.B) from a random state.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import adapt as oadapt  # noqa: E402
from oracle.core import Sector  # noqa: E402
from paper_2606_05297_gb300 import workloads as W  # noqa: E402

GOLDEN = os.path.join(ROOT, "tests", "golden")

# Seeds and sizes of every target; the GPU tests read them from the files.
SPEC = {
    "c2_screen": dict(U=3.4, state_seed=12),
    "c2_depth40": dict(U=3.4, depth=40, ansatz_seed=15, scale=0.2, state_seed=14),
    "c3_depth40": dict(model_seed=0, K=0.1, depth=40, ansatz_seed=13, scale=0.2),
    "c5_depth10": dict(depth=10, ansatz_seed=21, scale=0.2, screen_seed=22, screen_count=16, state_seed=23),
    "bkck_depth160": dict(L=6, d=6, Delta=0.6, K=0.3, depth=160, ansatz_seed=31, scale=0.2, state_seed=32),
}


def _write(name, payload):
    os.makedirs(GOLDEN, exist_ok=True)
    payload = dict(payload)
    payload["written_by"] = "oracle/make_golden.py (FP64 oracle only)"
    with open(os.path.join(GOLDEN, f"{name}.json"), "w") as f:
        json.dump(payload, f, indent=1)
        f.write("\n")


def c1_adapt():
    m = W.c1_model()
    pool = W.bh_nn_pool(m)
    warm = W.hva_layer(m)
    th0 = W.warm_start_thetas(len(warm), 0)
    occ = W.mott_occupation(4, 4)
    s = Sector(m)
    E0 = float(np.linalg.eigvalsh(s.matrix(s.H))[0])
    res = oadapt.run(s, pool, s.basis_state(occ), warm, th0, max_ops=160, grad_tol=1e-6)
    steps = [t for t in res["trace"] if t["kind"] == "adapt"]
    _write("c1_adapt", dict(
        what="plain ADAPT (Sec. IV.B) on the Bose-Hubbard open chain L=4, N=4, J=1, U=2, nearest-neighbour pool, "
             "Mott start with the HVA warm start (warm_start_thetas seed 0), to max|g| < 1e-6",
        E0_dense=E0, stop=res["stop"], n_adapt=res["n_adapt"], E_final=float(res["E"]),
        E_warm=float(res["trace"][0]["E"]), ops=[int(t["op"]) for t in steps],
        gmax=[float(t["gmax"]) for t in steps], E=[float(t["E"]) for t in steps],
        theta_sel=[[float(v) for v in t["theta_sel"]] for t in steps]))


def c2_screen():
    p = SPEC["c2_screen"]
    m = W.c2_model(p["U"])
    pool = W.bh_allpairs_pool(m.L)
    s = Sector(m)
    psi = W.random_state(s.dim, p["state_seed"])
    g = s.screen(pool, psi)
    E, _ = s.energy(psi)
    _write("c2_screen", dict(what="Eq. (grad) for the whole 210-element pool on random_state(dim, state_seed)",
                             spec=p, dim=s.dim, E=float(E), grad=[float(v) for v in g]))


def _eg(name, m, pool, psi0, spec, what):
    s = Sector(m)
    ids, th = W.random_ansatz(len(pool), spec["depth"], spec["ansatz_seed"], scale=spec["scale"])
    E, g = s.energy_and_grad([pool[k] for k in ids], th, psi0(s))
    return s, dict(what=what, spec=spec, dim=s.dim, ids=ids, E=float(E), grad=[float(v) for v in g])


def c2_depth40():
    p = SPEC["c2_depth40"]
    m = W.c2_model(p["U"])
    _, out = _eg("c2_depth40", m, W.bh_allpairs_pool(m.L), lambda s: W.random_state(s.dim, p["state_seed"]), p,
                 "E and dE/dtheta of random_ansatz(210, depth, ansatz_seed, scale) on random_state(dim, state_seed)")
    _write("c2_depth40", out)


def c3_depth40():
    p = SPEC["c3_depth40"]
    m = W.c3_model(p["model_seed"], K=p["K"])
    _, out = _eg("c3_depth40", m, W.bkc_kerr_pool(m.L), lambda s: s.basis_state(W.initial_occupation(m)), p,
                 "E and dE/dtheta of random_ansatz(136, depth, ansatz_seed, scale) from the vacuum")
    _write("c3_depth40", out)


def c5_depth10():
    p = SPEC["c5_depth10"]
    m = W.c5_model()
    pool = W.bkc_kerr_pool(m.L)
    s, out = _eg("c5_depth10", m, pool, lambda s: s.basis_state(W.initial_occupation(m)), p,
                 "E and dE/dtheta of random_ansatz(210, depth, ansatz_seed, scale) from the vacuum; Eq. (grad) "
                 "for screen_count pool elements drawn by default_rng(screen_seed) on random_state(dim, state_seed)")
    sub = [int(k) for k in np.random.default_rng(p["screen_seed"]).choice(len(pool), p["screen_count"],
                                                                        replace=False)]
    psi = W.random_state(s.dim, p["state_seed"])
    out["screen_subset"] = sub
    out["screen_grad"] = [float(v) for v in s.screen([pool[k] for k in sub], psi)]
    _write("c5_depth10", out)


def bkck_depth160():
    p = SPEC["bkck_depth160"]
    m = W.kitaev_kerr(p["L"], p["d"], t=1.0, Delta=p["Delta"], K=p["K"], periodic=False)
    _, out = _eg("bkck_depth160", m, W.bkc_kerr_pool(m.L), lambda s: W.random_state(s.dim, p["state_seed"]), p,
                 "E and dE/dtheta of a random 160-gate ansatz (the gate budget of Sec. IV.B) on a random state")
    _write("bkck_depth160", out)


TARGETS = dict(c1_adapt=c1_adapt, c2_screen=c2_screen, c2_depth40=c2_depth40, c3_depth40=c3_depth40,
               c5_depth10=c5_depth10, bkck_depth160=bkck_depth160)


def main(names):
    for n in names or list(TARGETS):
        t0 = time.perf_counter()
        TARGETS[n]()
        print(f"{n}: {time.perf_counter() - t0:.1f} s", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
