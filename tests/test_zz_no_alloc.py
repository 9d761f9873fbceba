"""cvq_screen_subset_noalloc, the screen for callers that cannot allocate
device memory when they screen: latency-critical loops that cannot pay for the
synchronisation of a cudaMalloc, host applications whose own allocator has
reserved all of the device's memory, and plug-ins handed fixed buffers.  It
must give the Eq. (grad) gradients of the FP64 oracle and the same values as
cvq_screen_pool, call after call, although it keeps its partial sums in one
fixed device array that every call shares instead of a caller workspace.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

from paper_2606_05297_gb300 import workloads as W

pytestmark = pytest.mark.gpu

G_ABS = 1e-9  # the gradient tolerance of the other parity tests


@pytest.mark.parametrize("which", ["bh", "bkc"])
def test_noalloc_screen_matches_oracle_and_workspace_screen_twice(which):
    import torch
    assert torch.cuda.is_available()
    from oracle.core import Sector as OS
    from paper_2606_05297_gb300 import build, cvq
    build.build()
    if which == "bh":
        m = W.bose_hubbard(8, 6, J=1.0, U=-2.5, periodic=True)
        pool = W.bh_allpairs_pool(m.L) + [W.Op("nn1", 0), W.Op("xkerr", 1, 5)]
    else:
        m = W.kitaev_kerr(6, 6, t=1.0, Delta=0.6, K=0.3, periodic=False)
        pool = W.bkc_kerr_pool(m.L) + [W.Op("rot", 2), W.Op("xkerr", 0, 4)]
    s = cvq.Sector(m)
    p = cvq.Pool(s, pool)
    os_ = OS(m)
    rng = np.random.default_rng(3)
    for call in range(2):  # two calls in a row: the shared array keeps the previous call's contents
        psi_h = W.random_state(s.dim, 20 + call)
        psi = torch.from_numpy(psi_h).cuda()
        # 8 elements, then 43 (a ragged last pass of 3), always including the pool's last element
        subset = [int(k) for k in rng.choice(len(pool), size=8 + 35 * call, replace=False)]
        subset[-1] = len(pool) - 1
        got = cvq.screen_subset_noalloc(s, p, psi, subset).cpu().numpy()
        ref = cvq.screen_pool(s, p, psi, subset=subset).cpu().numpy()
        oracle = os_.screen([pool[k] for k in subset], psi_h)
        assert got.shape == ref.shape == oracle.shape
        assert np.max(np.abs(got - oracle)) < G_ABS, (call, np.max(np.abs(got - oracle)))
        assert np.max(np.abs(got - ref)) < G_ABS, (call, np.max(np.abs(got - ref)))
    with pytest.raises(cvq.CvqError, match="n_subset"):
        cvq.screen_subset_noalloc(s, p, psi, list(range(65)))
