"""Projected gates (Sec. V.A) on the GPU against the projected-gate oracle:
normalised states, energies (1e-10 relative) and gradients through the
normalisations (1e-9 absolute) on Kitaev chains with and without Kerr,
random ansatze mixing beam splitters, squeezers, Kerr and rotations; the
screen on a projected pool equals the plain one; plain entry points reject a
projected pool."""
import numpy as np
import pytest

from paper_2606_05297_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [
    (W.kitaev_kerr(3, 4, t=1.0, Delta=0.6, K=0.3), 12),
    (W.kitaev_paper(4, 6, J=1.0, Delta=0.5, mu=-3.1, periodic=False), 14),
    (W.kitaev_kerr(4, 4, t=1.0, Delta=0.4, K=0.1, periodic=True), 9),
]


@pytest.mark.parametrize("m,dc", CASES)
def test_projected_matches_oracle(m, dc):
    import torch
    from oracle.core import Sector as OS
    from oracle.projected import Projected
    from paper_2606_05297_gb300 import build, cvq
    build.build()
    pool = W.bkc_table_pool(m.L, kerr=True)
    s = cvq.Sector(m)
    p = cvq.ProjectedPool(s, pool, dc)
    rng = np.random.default_rng(11 + m.L)
    ids = [int(k) for k in rng.integers(0, len(pool), 24)]
    th = rng.uniform(-0.7, 0.7, len(ids))
    psi0 = torch.from_numpy(W.random_state(s.dim, 4)).cuda()
    os_ = OS(m)
    P = Projected(os_, dc)
    ops = [pool[k] for k in ids]
    psi_ref = P.apply_ansatz(ops, th, psi0.cpu().numpy())
    psi = cvq.apply_ansatz_projected(s, p, ids, th, psi0).cpu().numpy()
    assert np.max(np.abs(psi - psi_ref)) < 1e-11
    E, g = cvq.energy_and_grad_projected(s, p, ids, th, psi0)
    Er, gr = P.energy_and_grad(ops, th, psi0.cpu().numpy())
    assert abs(E.item() - Er) <= 1e-10 * max(1.0, abs(Er))
    assert np.max(np.abs(g.cpu().numpy() - gr)) <= 1e-9
    # the screen at theta = 0 does not see the projection
    plain = cvq.Pool(s, pool)
    g1 = cvq.screen_pool(s, p, psi0).cpu().numpy()
    g0 = cvq.screen_pool(s, plain, psi0).cpu().numpy()
    assert np.max(np.abs(g1 - g0)) <= 1e-12
    with pytest.raises(cvq.CvqError):
        cvq.energy_and_grad(s, p, ids, th, psi0)


def test_projected_reduces_to_plain_inside_the_cutoff():
    """States that never reach the cutoff (one boson pair in a wide cutoff and
    beam splitters only) see identical plain and projected gates."""
    import torch
    from paper_2606_05297_gb300 import build, cvq
    build.build()
    m = W.kitaev_paper(3, 8, J=1.0, Delta=0.5, mu=-3.1, periodic=False)
    s = cvq.Sector(m)
    pool = [W.Op("hop", i, j, p) for i in range(3) for j in range(i + 1, 3) for p in (0, 1)]
    psi0 = s.basis_state([1, 1, 0])
    ids = [0, 3, 5, 1, 2, 4]
    th = [0.3, -0.2, 0.5, 0.1, -0.4, 0.25]
    E1, g1 = cvq.energy_and_grad_projected(s, cvq.ProjectedPool(s, pool, 16), ids, th, psi0)
    E0, g0 = cvq.energy_and_grad(s, cvq.Pool(s, pool), ids, th, psi0)
    assert abs(E1.item() - E0.item()) < 1e-13 and torch.max(torch.abs(g1 - g0)).item() < 1e-12
