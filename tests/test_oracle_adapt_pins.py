"""Pins of two oracle functions that the GPU comparisons rest on (CPU only).

orc_apply_rows, the gather form of an operator that the full-size matvec
checks use, against orc_apply, the scatter form pinned to the dense Kronecker
operators in test_oracle_pins.py: every row, for H and every generator type,
on every model of that file.

oracle.adapt.run (the ADAPT loop of Sec. IV.B) against facts that hold
independently of it: the variational principle (no energy below the exact
ground energy, and non-increasing energies since each BFGS starts from the
previous optimum with the new parameter at zero), convergence to the dense
exact-diagonalisation ground energy on a small chain, the closed-form first
gradient on a Fock state, the immediate stop on the Mott state (Sec. IV.B:
every pool gradient vanishes there), and the energy stopping rule.
"""
import json
import os

import numpy as np
import pytest

from oracle import adapt as oadapt
from oracle.core import Sector
from paper_2606_05297_gb300 import workloads as W
from test_oracle_pins import MODELS

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _all_generators(m):
    L = m.L
    ops = []
    for i in range(L):
        for j in range(L):
            if i == j:
                continue
            ops += [W.Op("hop", i, j, p) for p in (0, 1)]
            ops += [W.Op("pairhop", i, j, p) for p in (0, 1)]
            if m.kind == "bkc" and i < j:
                ops += [W.Op("sq2", i, j, p) for p in (0, 1)]
            if i < j:
                ops.append(W.Op("xkerr", i, j))
        ops += [W.Op("kerr", i), W.Op("nn1", i), W.Op("rot", i)]
        if m.kind == "bkc":
            ops += [W.Op("sq1", i, -1, p) for p in (0, 1)]
    return ops


@pytest.mark.parametrize("k", range(len(MODELS)))
def test_apply_rows_equals_apply_on_every_row(k):
    m = MODELS[k]
    s = Sector(m)
    psi = W.random_state(s.dim, 40 + k)
    rows = np.arange(s.dim)
    for name, op in [("H", s.H)] + [(str(o), s.op(o)) for o in _all_generators(m)]:
        full = s.apply(op, psi)
        got = s.apply_rows(op, psi, rows)
        assert np.max(np.abs(got - full)) <= 1e-14 * max(1.0, np.max(np.abs(full))), name
        # first and last index alone, and rows out of order
        pick = np.array([s.dim - 1, 0, s.dim // 2])
        assert np.max(np.abs(s.apply_rows(op, psi, pick) - full[pick])) <= 1e-14 * max(1.0, np.max(np.abs(full)))


def _ed(s):
    return float(np.linalg.eigvalsh(s.matrix(s.H))[0])


def test_adapt_converges_to_exact_ground_energy():
    """Periodic Bose-Hubbard L=3, N=3, U=2 (10 amplitudes) with the HVA warm
    start: energies never increase, none lies below the exact E0, and the run
    stops on max|g| < 1e-6 at E0 within 1e-6."""
    m = W.bose_hubbard(3, 3, J=1.0, U=2.0, periodic=True)
    s = Sector(m)
    E0 = _ed(s)
    pool = W.bh_nn_pool(m)
    warm = W.hva_layer(m)
    occ = W.mott_occupation(3, 3)
    res = oadapt.run(s, pool, s.basis_state(occ), warm, W.warm_start_thetas(len(warm), 0), max_ops=160)
    Es = [t["E"] for t in res["trace"]]
    assert all(b <= a + 1e-12 for a, b in zip(Es, Es[1:]))
    assert min(Es) >= E0 - 1e-12
    assert res["stop"] == "grad_tol"
    assert abs(res["E"] - E0) <= 1e-6
    # the last screen found every gradient below the threshold
    psi = s.apply_ansatz(res["ops"], res["theta"], s.basis_state(occ))
    assert np.max(np.abs(s.screen(pool, psi))) < 1e-6


def test_adapt_stops_at_once_on_the_mott_state():
    """Sec. IV.B: on a Fock state with equal occupations every pool gradient is
    zero (real hops give 2J(n_i - n_j) = 0, imaginary and diagonal ones 0), so
    without a warm start ADAPT ends before its first operator."""
    m = W.c1_model()
    s = Sector(m)
    res = oadapt.run(s, W.bh_nn_pool(m), s.basis_state(W.mott_occupation(4, 4)), max_ops=5)
    assert res["stop"] == "grad_tol" and res["n_adapt"] == 0 and res["ops"] == []


def test_adapt_first_choice_on_a_fock_state():
    """On |2,0,1,1> the real-hop gradients are 2J(n_i - n_j) = 4, 2, 0 on the
    bonds (0,1), (1,2), (2,3), so the first operator is the real hop on (0,1)
    with |g| = 4 exactly, and its optimisation lowers the energy below the
    Fock state's."""
    m = W.c1_model()
    s = Sector(m)
    pool = W.bh_nn_pool(m)
    psi0 = s.basis_state([2, 0, 1, 1])
    res = oadapt.run(s, pool, psi0, max_ops=1)
    t = res["trace"][0]
    assert pool[t["op"]] == W.Op("hop", 0, 1, 0)
    assert abs(t["gmax"] - 4.0) < 1e-12
    assert t["E"] < s.energy(psi0)[0] - 1e-3


def test_adapt_energy_stopping_rule():
    """With E0 and a tolerance given, the loop stops as soon as |E - E0| is
    below it (Sec. IV.B), earlier than the gradient rule."""
    m = W.bose_hubbard(3, 3, J=1.0, U=2.0, periodic=True)
    s = Sector(m)
    E0 = _ed(s)
    pool = W.bh_nn_pool(m)
    warm = W.hva_layer(m)
    occ = W.mott_occupation(3, 3)
    th = W.warm_start_thetas(len(warm), 0)
    res = oadapt.run(s, pool, s.basis_state(occ), warm, th, max_ops=160, E0=E0, energy_tol=1e-2)
    full = oadapt.run(s, pool, s.basis_state(occ), warm, th, max_ops=160)
    assert res["stop"] == "energy_tol" and abs(res["E"] - E0) < 1e-2
    assert res["n_adapt"] < full["n_adapt"]
    assert res["ops"] == full["ops"][: len(res["ops"])]  # warm-start gates, then the same choices


def test_stored_c1_trace_satisfies_the_pins():
    """The stored L=4 trace (written by oracle/make_golden.py) obeys the same
    facts: energies non-increasing and never below the dense E0, the run ends
    on the gradient rule at E0 within 1e-6."""
    path = os.path.join(GOLDEN, "c1_adapt.json")
    if not os.path.exists(path):
        pytest.skip("tests/golden/c1_adapt.json not written yet")
    d = json.load(open(path))
    s = Sector(W.c1_model())
    assert abs(d["E0_dense"] - _ed(s)) < 1e-12
    Es = [d["E_warm"]] + d["E"]
    assert all(b <= a + 1e-12 for a, b in zip(Es, Es[1:]))
    assert min(Es) >= d["E0_dense"] - 1e-12
    assert d["stop"] == "grad_tol" and abs(d["E_final"] - d["E0_dense"]) <= 1e-6
    assert len(d["ops"]) == d["n_adapt"] == len(d["E"])
