"""Host-side logic of the product driver (CPU only): BFGS and selection."""
import numpy as np

from paper_2606_05297_gb300.adapt import BFGS, select


def test_bfgs_on_quadratic_and_rosenbrock():
    """Textbook checks: Rosenbrock from (-1.2, 1) reaches (1, 1); a strictly
    convex quadratic reaches A^-1 b."""
    def rosen(x):
        f = 100 * (x[1] - x[0] ** 2) ** 2 + (1 - x[0]) ** 2
        g = np.array([-400 * x[0] * (x[1] - x[0] ** 2) - 2 * (1 - x[0]), 200 * (x[1] - x[0] ** 2)])
        return f, g
    r = BFGS(rosen).minimize([-1.2, 1.0], gtol=1e-10, max_iter=500)
    assert np.max(np.abs(r.x - 1.0)) < 1e-8 and r.status == "gtol"
    rng = np.random.default_rng(0)
    M = rng.standard_normal((6, 6))
    A = M @ M.T + 6 * np.eye(6)
    b = rng.standard_normal(6)
    r = BFGS(lambda x: (0.5 * x @ A @ x - b @ x, A @ x - b)).minimize(np.zeros(6), gtol=1e-12)
    assert np.max(np.abs(r.x - np.linalg.solve(A, b))) < 1e-10


def test_bfgs_matches_oracle_iterates():
    """The product BFGS and the oracle's follow the same textbook rules, so on
    a smooth test function they produce the same iterates up to rounding."""
    from oracle import bfgs as ob
    rng = np.random.default_rng(3)
    M = rng.standard_normal((5, 5))
    A = M @ M.T + np.eye(5)

    def f(x):
        return float(x @ A @ x / 2 + np.sum(np.cos(x))), A @ x - np.sin(x)
    x0 = rng.standard_normal(5)
    r1 = BFGS(f).minimize(x0, gtol=1e-10)
    r2 = ob.minimize(f, x0, gtol=1e-10)
    assert r1.nfev == r2["nfev"] and r1.nit == r2["nit"]
    assert np.max(np.abs(r1.x - r2["x"])) < 1e-12


def test_selection_tie_rule():
    assert select([0.1, -2.0, 2.0, 1.0])[0] == 1
    assert select([0.1, 2.0 * (1 - 5e-10), -2.0])[0] == 1
    assert select([0.1, 2.0 * (1 - 5e-9), -2.0])[0] == 2


def test_bfgs_line_search_at_the_step_cap():
    """A far minimum makes the bracketing phase reach the largest step twice
    (a zero-width bracket); both minimisers must bisect instead of dividing by
    the bracket width, and still agree iterate for iterate."""
    from oracle import bfgs as ob

    def fg(x):
        d = x - 1e4
        return float(1e-6 * d @ d), 2e-6 * d

    r = BFGS(fg).minimize(np.zeros(2), gtol=1e-9, max_iter=200)
    o = ob.minimize(fg, np.zeros(2), gtol=1e-9, max_iter=200)
    assert np.isfinite(r.f) and r.f < fg(np.zeros(2))[0]
    assert np.array_equal(r.x, o["x"]) and r.nit == o["nit"]


def test_oracle_hessian_recycling_reduces_evaluations():
    """App. D: recycling the inverse Hessian between ADAPT iterations lowers the
    optimiser's work; on the L=4 chain the first selections coincide with the
    plain loop's and the evaluations drop by more than a third."""
    from oracle import adapt as oa
    from oracle.core import Sector
    from paper_2606_05297_gb300 import workloads as W
    m = W.c1_model()
    s = Sector(m)
    pool, warm = W.pool_for(m), W.hva_layer(m)
    th = W.warm_start_thetas(len(warm), 3)
    psi0 = s.basis_state(W.initial_occupation(m))
    plain = oa.run(s, pool, psi0, warm, th, max_ops=8)
    hr = oa.run(s, pool, psi0, warm, th, max_ops=8, hessian_recycling=True)
    ops = lambda r: [t["op"] for t in r["trace"] if t["kind"] == "adapt"]
    nfev = lambda r: sum(t["nfev"] for t in r["trace"] if t["kind"] == "adapt")
    assert ops(plain)[:4] == ops(hr)[:4]
    assert nfev(hr) < (2 / 3) * nfev(plain)


def test_autotune_cache_round_trip(tmp_path, monkeypatch):
    """The batched engine's schedule cache survives a new process: entries
    written by one store are read back, merged with later ones, and a
    corrupt file reads as empty."""
    from paper_2606_05297_gb300 import batched
    path = tmp_path / "tune.json"
    monkeypatch.setattr(batched, "TUNE_CACHE", str(path))
    assert batched._load_tuned() == {}
    batched._store_tuned("GB300|6435,24310", 16384, 2)
    batched._store_tuned("GB300|35", 4096, 1)
    assert batched._load_tuned() == {"GB300|6435,24310": [16384, 2], "GB300|35": [4096, 1]}
    path.write_text("{not json")
    assert batched._load_tuned() == {}
