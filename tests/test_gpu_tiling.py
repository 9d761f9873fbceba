"""Operator tiling (App. B) through the CUDA driver: patterns learned by GPU
ADAPT on the L=3 Kitaev chain (d=6, Delta=0.5, mu=-3.1) include those of the
oracle's selections there, and GPU ADAPT at L=5 makes the same choices with
the tiled pool as with the full one (same operators, energies to 1e-10)."""
import pytest

from paper_2606_05297_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_gpu_tiling_matches_full_pool():
    from oracle import adapt as oa
    from oracle.core import Sector as OS
    from paper_2606_05297_gb300 import adapt, build, tiling
    build.build()
    m3 = W.kitaev_paper(3, 6, J=1.0, Delta=0.5, mu=-3.1, periodic=False)
    small = W.bkc_table_pool(3)
    pats = tiling.learn_patterns(m3, small, [0, 0, 0], max_ops=10)
    os3 = OS(m3)
    r3 = oa.run(os3, small, os3.basis_state([0, 0, 0]), max_ops=10)
    assert {tiling.pattern_of(small[t["op"]]) for t in r3["trace"] if t["kind"] == "adapt"} <= pats
    m5 = W.kitaev_paper(5, 6, J=1.0, Delta=0.5, mu=-3.1, periodic=False)
    full = W.bkc_table_pool(5)
    tiled = tiling.tiled_pool(full, pats)
    assert len(tiled) < len(full)
    runs = []
    for pool in (full, tiled):
        A = adapt.Adapt(m5, pool, [0] * 5, n_max=16)
        for _ in range(6):
            A.step()
        runs.append(([pool[r["op"]] for r in A.trace], [r["E"] for r in A.trace]))
    assert len(runs[0][0]) == 6 and runs[0][0] == runs[1][0]
    assert all(abs(a - b) <= 1e-10 * max(1.0, abs(a)) for a, b in zip(runs[0][1], runs[1][1]))
