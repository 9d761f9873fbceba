"""The adjoint gradient behind torch.autograd and with checkpointed forward
states: against the oracle's gradient (1e-9 absolute) and central finite
differences of the energy, on a Kitaev chain with Kerr and a Bose-Hubbard
chain; the checkpointed sweep equals the plain one to rounding."""
import numpy as np
import pytest

from paper_2606_05297_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,pool", [(W.kitaev_kerr(4, 6, t=1.0, Delta=0.6, K=0.3), W.bkc_kerr_pool(4)),
                                    (W.bose_hubbard(5, 5, J=1.0, U=3.4, periodic=True), W.bh_allpairs_pool(5))])
@pytest.mark.parametrize("every", [None, 1, 7])
def test_autograd_matches_oracle_and_fd(m, pool, every):
    import torch
    from oracle.core import Sector as OS
    from paper_2606_05297_gb300 import autograd, build, cvq
    build.build()
    s = cvq.Sector(m)
    p = cvq.Pool(s, pool + [W.Op("kerr", r) for r in range(m.L)])
    rng = np.random.default_rng(4)
    ids = [int(k) for k in rng.integers(0, len(pool) + m.L, 30)]
    th0 = rng.uniform(-0.5, 0.5, len(ids))
    psi0 = torch.from_numpy(W.random_state(s.dim, 8)).cuda()
    theta = torch.tensor(th0, dtype=torch.float64, requires_grad=True)
    E = autograd.ansatz_energy(theta, s, p, ids, psi0, checkpoint_every=every)
    (g,) = torch.autograd.grad(2.0 * E, theta)
    ops = (pool + [W.Op("kerr", r) for r in range(m.L)])
    Er, gr = OS(m).energy_and_grad([ops[k] for k in ids], th0, psi0.cpu().numpy())
    assert abs(E.item() - Er) <= 1e-10 * max(1.0, abs(Er))
    assert np.max(np.abs(g.numpy() - 2.0 * gr)) <= 2e-9
    h = 1e-5
    for k in (0, 13, 29):
        e = np.zeros(len(ids))
        e[k] = h
        Ep = autograd.ansatz_energy(torch.tensor(th0 + e), s, p, ids, psi0, checkpoint_every=every).item()
        Em = autograd.ansatz_energy(torch.tensor(th0 - e), s, p, ids, psi0, checkpoint_every=every).item()
        assert abs((Ep - Em) / (2 * h) - gr[k]) <= 1e-7 * max(1.0, abs(gr[k]))
    if every:
        E2, g2 = cvq.energy_and_grad(s, p, ids, th0, psi0)
        assert abs(E.item() - E2.item()) <= 1e-13 * max(1.0, abs(Er))
        assert np.max(np.abs(g.numpy() / 2.0 - g2.cpu().numpy())) <= 1e-11


def test_checkpoint_buffer_checks():
    import torch
    from paper_2606_05297_gb300 import build, cvq
    build.build()
    m = W.bose_hubbard(4, 4, J=1.0, U=1.0, periodic=True)
    s = cvq.Sector(m)
    p = cvq.Pool(s, W.bh_allpairs_pool(4))
    psi0 = torch.from_numpy(W.random_state(s.dim, 1)).cuda()
    with pytest.raises(cvq.CvqError):
        cvq.energy_and_grad_ckpt(s, p, [0, 1, 2], [0.1, 0.2, 0.3], psi0, every=0)
    with pytest.raises(cvq.CvqError):  # a buffer one byte short of two checkpoints
        cvq.energy_and_grad_ckpt(s, p, [0, 1, 2], [0.1, 0.2, 0.3], psi0, every=1,
                                 ckpt=torch.empty(2 * s.dim * 16 - 1, dtype=torch.uint8, device="cuda"))
    E, g = cvq.energy_and_grad_ckpt(s, p, [0, 1, 2], [0.1, 0.2, 0.3], psi0, every=1,
                                    ckpt=torch.empty(2 * s.dim * 16, dtype=torch.uint8, device="cuda"))
    assert np.isfinite(E.item()) and g.numel() == 3
