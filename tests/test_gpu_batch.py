"""Batched engine (cvq_batch_*) against the FP64 oracle: several instances of
uneven sector size, each with its own pool and random ansatz (block gates and
runs of diagonal gates, cross-Kerr included), evaluated in one graph launch.
Tolerances as for the single-instance calls: energies 1e-10 relative,
gradients 1e-9 absolute."""
import numpy as np
import pytest

from paper_2606_05297_gb300 import workloads as W

pytestmark = pytest.mark.gpu

E_REL, G_ABS = 1e-10, 1e-9


def _bh_pool(L):
    ops = []
    for i in range(L):
        for j in range(L):
            if i != j:
                ops += [W.Op("hop", i, j, p) for p in (0, 1)]
                ops.append(W.Op("pairhop", i, j, 1))
                if i < j:
                    ops.append(W.Op("xkerr", i, j))
    ops += [W.Op(t, r) for r in range(L) for t in ("kerr", "nn1", "rot")]
    return ops


def _bkc_pool(L):
    return W.bkc_kerr_pool(L) + [W.Op("rot", r) for r in range(L)] + [W.Op("xkerr", 0, L - 1)]


def _ansatz(K, depth, seed):
    rng = np.random.default_rng(seed)
    ids = list(rng.integers(0, K, depth))
    # force a long diagonal run and a cross-Kerr inside it
    return [int(k) for k in ids], rng.uniform(-0.6, 0.6, depth)


def _setup(models, pools, depths, seed):
    import torch
    from oracle.core import Sector as OS
    from paper_2606_05297_gb300 import build, cvq
    build.build()
    secs = [cvq.Sector(m) for m in models]
    pls = [cvq.Pool(s, p) for s, p in zip(secs, pools)]
    psi0 = [torch.from_numpy(W.random_state(s.dim, seed + 7 * i)).cuda() for i, s in enumerate(secs)]
    ans = []
    for i, (p, d) in enumerate(zip(pools, depths)):
        if d is None:
            ans.append((None, None))
            continue
        ids, th = _ansatz(len(p), d, seed + 11 * i)
        ans.append((ids, th))
    b = cvq.Batch(secs, pls, max(d or 0 for d in depths) + 1)
    b.set_ansatz([a[0] for a in ans], psi0)
    oss = [OS(m) for m in models]
    return b, secs, pls, psi0, ans, oss


def _theta_vec(ans):
    import torch
    flat = np.concatenate([a[1] for a in ans if a[0] is not None and len(a[0])] or [np.zeros(0)])
    return torch.from_numpy(flat).cuda()


def _check(b, ans, pools, psi0, oss):
    E, g = b.energy_and_grad(_theta_vec(ans))
    E, g = E.cpu().numpy(), g.cpu().numpy()
    for i, (ids, th) in enumerate(ans):
        if ids is None:
            continue
        o = b.offsets[i]
        ops = [pools[i][k] for k in ids]
        Er, gr = oss[i].energy_and_grad(ops, th, psi0[i].cpu().numpy())
        assert abs(E[i] - Er) <= E_REL * max(1.0, abs(Er)), (i, E[i], Er)
        if ids:
            assert np.max(np.abs(g[o:o + len(ids)] - gr)) <= G_ABS, (i, np.max(np.abs(g[o:o + len(ids)] - gr)))


def test_batch_bose_hubbard_matches_oracle():
    models = [W.c1_model(), W.bose_hubbard(5, 5, J=1.0, U=3.0, periodic=True),
              W.bose_hubbard(3, 7, J=0.7, U=-1.5, periodic=True), W.bose_hubbard(6, 4, J=1.0, U=10.0, periodic=True),
              W.bose_hubbard(4, 2, J=1.0, U=1.0, periodic=False)]
    pools = [_bh_pool(m.L) for m in models]
    depths = [12, 30, 0, 25, None]  # uneven depths, an empty ansatz, an instance left out
    b, secs, pls, psi0, ans, oss = _setup(models, pools, depths, 100)
    _check(b, ans, pools, psi0, oss)
    info = b.info()
    assert info["layers"] >= 3 and info["kernels_per_eval"] <= info["layers"] + 2


def test_batch_kitaev_matches_oracle():
    models = [W.kitaev_kerr(4, 4, t=1.0, Delta=0.6, K=0.3), W.kitaev_kerr(3, 6, t=1.0, Delta=0.2, K=0.5),
              W.kitaev_paper(3, 4, J=1.0, Delta=0.5, mu=-2.7, U=-1.0, periodic=True, parity=1)]
    pools = [_bkc_pool(m.L) for m in models]
    b, secs, pls, psi0, ans, oss = _setup(models, pools, [20, 14, 9], 200)
    _check(b, ans, pools, psi0, oss)


def test_batch_graph_replay_and_schedules():
    """New theta through the captured graph, every schedule, and bitwise
    repeatability of one schedule."""
    models = [W.bose_hubbard(5, 5, J=1.0, U=3.0, periodic=True), W.bose_hubbard(4, 6, J=1.0, U=0.5, periodic=True)]
    pools = [_bh_pool(m.L) for m in models]
    b, secs, pls, psi0, ans, oss = _setup(models, pools, [18, 22], 300)
    _check(b, ans, pools, psi0, oss)
    rng = np.random.default_rng(5)
    ans2 = [(ids, rng.uniform(-1, 1, len(ids))) for ids, _ in ans]
    _check(b, ans2, pools, psi0, oss)
    for tile, ctas in ((256, 1), (4096, 2), (1 << 20, 2)):
        b.set_schedule(tile, ctas)
        _check(b, ans2, pools, psi0, oss)
    E1, g1 = [t.clone() for t in b.energy_and_grad(_theta_vec(ans2))]
    E2, g2 = b.energy_and_grad(_theta_vec(ans2))
    assert np.array_equal(E1.cpu().numpy(), E2.cpu().numpy()) and np.array_equal(g1.cpu().numpy(), g2.cpu().numpy())


def test_batch_c4_instances_sampled():
    """Every instance shape of the 64-instance sweep (L = 8..12, N = L, all-pairs
    pool, HVA warm start plus random pool operators) in one batch: the batched
    result equals the single-instance call on each instance to far below the
    tolerance, and the smallest instances match the oracle."""
    import torch
    from oracle.core import Sector as OS
    from paper_2606_05297_gb300 import build, cvq
    build.build()
    insts = W.c4_instances(0, 64)
    pick = []
    for L in range(8, 13):
        pick += [m for m in insts if m.L == L][:2]
    secs = [cvq.Sector(m) for m in pick]
    pools = [W.bh_allpairs_pool(m.L) + W.hva_layer(m) for m in pick]
    pls = [cvq.Pool(s, p) for s, p in zip(secs, pools)]
    rng = np.random.default_rng(9)
    ans = []
    for m, p in zip(pick, pools):
        K0 = len(W.bh_allpairs_pool(m.L))
        ids = list(range(K0, len(p))) + [int(k) for k in rng.integers(0, K0, 8)]
        ans.append((ids, rng.uniform(-0.3, 0.3, len(ids))))
    psi0 = [s.basis_state(W.mott_occupation(m.L, m.N)) for s, m in zip(secs, pick)]
    b = cvq.Batch(secs, pls, max(len(a[0]) for a in ans))
    b.set_ansatz([a[0] for a in ans], psi0)
    E, g = b.energy_and_grad(_theta_vec(ans))
    E, g = E.cpu().numpy(), g.cpu().numpy()
    for i, (ids, th) in enumerate(ans):
        ws = secs[i].workspace(pls[i], len(ids))
        Es, gs = cvq.energy_and_grad(secs[i], pls[i], ids, th, psi0[i], ws=ws)
        Es, gs = float(Es.item()), gs.cpu().numpy()
        o = b.offsets[i]
        assert abs(E[i] - Es) <= 1e-12 * max(1.0, abs(Es))
        assert np.max(np.abs(g[o:o + len(ids)] - gs)) <= 1e-11
    for i in range(2):  # L = 8, dim 6435: the oracle is quick here
        ids, th = ans[i]
        Er, gr = OS(pick[i]).energy_and_grad([pools[i][k] for k in ids], th, psi0[i].cpu().numpy())
        o = b.offsets[i]
        assert abs(E[i] - Er) <= E_REL * max(1.0, abs(Er))
        assert np.max(np.abs(g[o:o + len(ids)] - gr)) <= G_ABS


def _screen_check(b, ans, pools, psi0, oss, subsets, out, off, skip=()):
    out = out.cpu().numpy()
    for i, (ids, th) in enumerate(ans):
        if ids is None or i in skip:
            continue
        sub = list(range(len(pools[i]))) if subsets is None else subsets[i]
        assert off[i + 1] - off[i] == len(sub)
        if not sub:
            continue
        psi = oss[i].apply_ansatz([pools[i][k] for k in ids], th, psi0[i].cpu().numpy())
        gref = oss[i].screen([pools[i][k] for k in sub], psi)
        got = out[off[i]:off[i + 1]]
        assert np.max(np.abs(got - gref)) < G_ABS, (i, np.max(np.abs(got - gref)))


@pytest.mark.parametrize("kind", ["bh", "bkc"])
def test_batch_screen_matches_oracle(kind):
    """cvq_batch_screen: Eq. (grad) of every instance's whole pool, then of
    per-instance subsets (one of them empty), on U(theta) psi0 of each
    instance's ansatz, against the oracle's screen of the oracle's forward
    state; an instance left out has no outputs, and a paused instance's
    outputs are not written.  Repeated calls are bit-identical."""
    import torch
    if kind == "bh":
        models = [W.c1_model(), W.bose_hubbard(5, 5, J=1.0, U=3.0, periodic=True),
                  W.bose_hubbard(3, 7, J=0.7, U=-1.5, periodic=True), W.bose_hubbard(4, 2, J=1.0, U=1.0, periodic=False)]
        pools = [_bh_pool(m.L) for m in models]
        depths = [12, 20, 0, None]
    else:
        models = [W.kitaev_kerr(4, 4, t=1.0, Delta=0.6, K=0.3), W.kitaev_kerr(3, 6, t=1.0, Delta=0.2, K=0.5),
                  W.kitaev_paper(3, 4, J=1.0, Delta=0.5, mu=-2.7, U=-1.0, periodic=True, parity=1)]
        pools = [_bkc_pool(m.L) for m in models]
        depths = [16, 9, 5]
    b, secs, pls, psi0, ans, oss = _setup(models, pools, depths, 400)
    th = _theta_vec(ans)
    b.theta[: th.numel()].copy_(th)
    out, off = b.screen()
    _screen_check(b, ans, pools, psi0, oss, None, out, off)
    out2, _ = b.screen()
    assert np.array_equal(out.cpu().numpy(), out2.cpu().numpy())
    rng = np.random.default_rng(1)
    subsets = [sorted({int(k) for k in rng.integers(0, len(p), 6)} | {len(p) - 1}) for p in pools]
    subsets[1] = []
    out, off = b.screen(subsets)
    _screen_check(b, ans, pools, psi0, oss, subsets, out, off)
    # pause instance 0: its outputs keep what the buffer held
    b.set_active([i != 0 and ans[i][0] is not None for i in range(len(ans))])
    out.fill_(float("nan"))
    out, off = b.screen(subsets, out=out)
    assert np.all(np.isnan(out.cpu().numpy()[off[0]:off[1]]))
    _screen_check(b, ans, pools, psi0, oss, subsets, out, off, skip=(0,))
