"""Energy and gradient with the forward states kept (the reverse sweep reads
psi_k instead of recomputing it): against the oracle at the usual tolerances
and against the recomputing sweep to rounding, on Bose-Hubbard and Kitaev
chains with block gates and long diagonal runs."""
import numpy as np
import pytest

from paper_2606_05297_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m", [W.bose_hubbard(5, 4, J=1.0, U=2.0, periodic=True),
                               W.kitaev_kerr(4, 6, t=1.0, Delta=0.6, K=0.3),
                               W.c1_model()])
def test_kept_matches_oracle_and_plain(m):
    import torch
    from oracle.core import Sector as OS
    from paper_2606_05297_gb300 import build, cvq
    build.build()
    base = W.bh_allpairs_pool(m.L) if m.kind == "bh" else W.bkc_kerr_pool(m.L)
    pool = base + [W.Op("rot", r) for r in range(m.L)] + [W.Op("xkerr", 0, m.L - 1)]
    s = cvq.Sector(m)
    p = cvq.Pool(s, pool)
    rng = np.random.default_rng(21)
    ids = [int(k) for k in rng.integers(0, len(pool), 30)] + list(range(len(base), len(pool)))  # ends in a long run
    th = rng.uniform(-0.5, 0.5, len(ids))
    psi0 = torch.from_numpy(W.random_state(s.dim, 5)).cuda()
    E, g = cvq.energy_and_grad_kept(s, p, ids, th, psi0)
    Er, gr = OS(m).energy_and_grad([pool[k] for k in ids], th, psi0.cpu().numpy())
    assert abs(E.item() - Er) <= 1e-10 * max(1.0, abs(Er))
    assert np.max(np.abs(g.cpu().numpy() - gr)) <= 1e-9
    E0, g0 = cvq.energy_and_grad(s, p, ids, th, psi0)
    assert abs(E.item() - E0.item()) <= 1e-13 * max(1.0, abs(Er))
    assert np.max(np.abs(g.cpu().numpy() - g0.cpu().numpy())) <= 1e-11
