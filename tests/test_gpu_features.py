"""Feature kernel (<n_r>, <n_r^2>, <a_i^dag a_j>) against the oracle's plain
definitions, on both sector kinds, with a ragged tail and at full size on
sampled properties."""
import numpy as np
import pytest

from paper_2606_05297_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m", [W.bose_hubbard(6, 5, J=1.0, U=2.0, periodic=True),
                               W.kitaev_kerr(5, 6, t=1.0, Delta=0.4, K=0.3, periodic=False),
                               W.kitaev_paper(3, 4, parity=1, periodic=True),
                               W.bose_hubbard(2, 3, periodic=False)])
def test_features_match_oracle(m):
    import torch
    from oracle import features as ofeat
    from oracle.core import Sector as OS
    from paper_2606_05297_gb300 import build, cvq
    build.build()
    s = cvq.Sector(m)
    os_ = OS(m)
    psi = W.random_state(s.dim, 31)
    pairs = [(i, j) for i in range(m.L) for j in range(m.L) if i != j]
    got = cvq.features(s, torch.from_numpy(psi).cuda(), pairs).cpu().numpy()
    ref = ofeat.features(os_, psi, pairs)
    assert np.max(np.abs(got - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


def test_features_full_size_invariants():
    """L=12, N=12: sum_r <n_r> = N exactly, <a_i^dag a_j> = conj(<a_j^dag a_i>)."""
    import torch
    from paper_2606_05297_gb300 import cvq
    s = cvq.Sector(W.c2_model(3.4))
    psi = torch.from_numpy(W.random_state(s.dim, 32)).cuda()
    f = cvq.features(s, psi, [(0, 5), (5, 0), (3, 4)]).cpu().numpy()
    assert abs(f[:12].sum() - 12.0) < 1e-11
    assert abs(f[24] - f[26]) < 1e-13 and abs(f[25] + f[27]) < 1e-13
