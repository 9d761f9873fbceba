"""Operator tiling (App. B) on the oracle: patterns learned by the oracle's
ADAPT loop on the L=3 Kitaev chain (d=6, Delta=0.5, mu=-3.1, the paper's
tiling example at a smaller size) give an L=5 pool far smaller than the full
one on which ADAPT makes the same choices with the same energies."""
from paper_2606_05297_gb300 import tiling
from paper_2606_05297_gb300 import workloads as W


def _oracle_run(L, pool, n):
    from oracle import adapt as oa
    from oracle.core import Sector
    m = W.kitaev_paper(L, 6, J=1.0, Delta=0.5, mu=-3.1, periodic=False)
    s = Sector(m)
    return oa.run(s, pool, s.basis_state([0] * L), max_ops=n)


def test_pattern_and_pool_filter():
    ops = [W.Op("hop", 0, 2, 1), W.Op("sq1", 3, -1, 0), W.Op("hop", 2, 0, 1)]
    assert [tiling.pattern_of(o) for o in ops] == [("hop", 1, 2), ("sq1", 0, None), ("hop", 1, -2)]
    full = W.bkc_table_pool(5)
    pool = tiling.tiled_pool(full, {("hop", 1, 2), ("sq1", 0, None)})
    assert pool == [W.Op("hop", 0, 2, 1), W.Op("hop", 1, 3, 1), W.Op("hop", 2, 4, 1)] + \
        [W.Op("sq1", r, -1, 0) for r in range(5)]
    assert tiling.degenerate_patterns(full[:3], [0.5, -0.5 * (1 - 1e-9), 0.1]) == {("hop", 0, 1), ("hop", 1, 1)}


def test_tiled_pool_reproduces_full_pool_trajectory():
    small = W.bkc_table_pool(3)
    r3 = _oracle_run(3, small, 10)
    pats = {tiling.pattern_of(small[t["op"]]) for t in r3["trace"] if t["kind"] == "adapt"}
    full = W.bkc_table_pool(5)
    tiled = tiling.tiled_pool(full, pats)
    assert len(tiled) < len(full) / 2
    n = 6
    rf, rt = _oracle_run(5, full, n), _oracle_run(5, tiled, n)
    sel_f = [full[t["op"]] for t in rf["trace"] if t["kind"] == "adapt"]
    sel_t = [tiled[t["op"]] for t in rt["trace"] if t["kind"] == "adapt"]
    assert len(sel_f) == n and sel_f == sel_t
    assert [t["E"] for t in rf["trace"]] == [t["E"] for t in rt["trace"]]
