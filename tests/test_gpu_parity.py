"""GPU parity: every C-ABI call of libcvq.so against the FP64 oracle on the same
seeded inputs.

Tolerances: energies 1e-10 relative and gradients 1e-9 absolute (the accuracy
target of the method's numerics); normalised state amplitudes 1e-11 absolute,
derived from the kernels' double-float arithmetic (about 2^-48 relative per
operation, at most 16-term block sums, at most ~30 gates deep here:
30 * 16 * 2^-48 ~ 2e-12).  Small sectors are compared element by element; the full-size
workloads on sampled rows the oracle computes one by one and on properties
that hold at any size.
"""
import numpy as np
import pytest

from paper_2606_05297_gb300 import workloads as W

pytestmark = pytest.mark.gpu

E_REL, G_ABS, PSI_ABS = 1e-10, 1e-9, 1e-11


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2606_05297_gb300 import build
    build.build()
    return torch


def _bh(L, N, hop, nn1, periodic, n2=None, n1=None):
    nb = L if periodic else L - 1
    return W.Model("bh", L, N=N, periodic=periodic, hop=list(hop)[:nb], pair=[0.0] * nb, nn1=list(nn1),
                   n2=list(n2 or [0.0] * L), n1=list(n1 or [0.0] * L))


SMALL = {
    "c1": W.c1_model(),
    "bh_pbc_L5_N4": _bh(5, 4, [-1.0, -0.8, -1.2, -0.9, -1.1], [0.4, -0.3, 0.2, 0.0, 0.1], True, n2=[0.1] * 5,
                        n1=[0.05, 0, 0, 0, 0.2]),
    "bh_L2_N3_pbc": _bh(2, 3, [-1.0, -0.6], [0.3, -0.2], True),
    "bh_L3_N1": _bh(3, 1, [-1.0, -0.5], [0.0, 0.0, 0.0], False),
    "bkc_paper_L3_d4_even": W.kitaev_paper(3, 4, J=1.0, Delta=0.5, mu=-2.7, U=-1.0, periodic=True, parity=0),
    "bkc_paper_L3_d4_odd": W.kitaev_paper(3, 4, J=0.8, Delta=0.3, mu=-3.1, periodic=True, parity=1),
    "bkck_L4_d6": W.kitaev_kerr(4, 6, t=1.0, Delta=[0.2, 0.7, 0.4], K=0.5, periodic=False),
    "bkc_L1_d8": W.kitaev_kerr(1, 8, t=1.0, Delta=0.3, K=0.2, periodic=False),
    "bkc_L2_d2": W.kitaev_paper(2, 2, J=1.0, Delta=0.4, mu=-1.0, periodic=False, parity=0),
}


def pool_for_test(m):
    L = m.L
    ops = []
    if m.kind == "bh":
        for i in range(L):
            for j in range(L):
                if i != j:
                    ops += [W.Op("hop", i, j, p) for p in (0, 1, 2, 3)]
                    ops += [W.Op("pairhop", i, j, p) for p in (0, 1)]
                    if i < j:
                        ops.append(W.Op("xkerr", i, j))
        ops += [W.Op(t, r) for r in range(L) for t in ("kerr", "nn1", "rot")]
    else:
        for i in range(L):
            for j in range(L):
                if i != j:
                    ops += [W.Op("hop", i, j, p) for p in (0, 1, 3)]
                    ops += [W.Op("sq2", i, j, p) for p in (0, 1, 2)]
                    ops.append(W.Op("pairhop", i, j, 1))
                    if i < j:
                        ops.append(W.Op("xkerr", i, j))
        ops += [W.Op("sq1", r, -1, p) for r in range(L) for p in (0, 1, 3)]
        ops += [W.Op(t, r) for r in range(L) for t in ("kerr", "nn1", "rot")]
    return ops[:500]


def _np(t):
    return t.detach().cpu().numpy()


def _setup(torch, m, ops=None):
    from oracle.core import Sector as OS
    from paper_2606_05297_gb300 import cvq
    s = cvq.Sector(m)
    os_ = OS(m)
    assert s.dim == os_.dim
    ops = pool_for_test(m) if ops is None else ops
    p = cvq.Pool(s, ops)
    return cvq, s, p, os_, ops


@pytest.mark.parametrize("name", sorted(SMALL))
def test_apply_H_and_energy(torch_cuda, name):
    torch = torch_cuda
    m = SMALL[name]
    cvq, s, p, os_, ops = _setup(torch, m, ops=[])
    psi = W.random_state(s.dim, 1)
    dpsi = torch.from_numpy(psi).cuda()
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    sigma = cvq.apply_H(s, dpsi, energy=E)
    ref = os_.apply_H(psi)
    Eref, _ = os_.energy(psi)
    assert np.max(np.abs(_np(sigma) - ref)) < PSI_ABS * max(1.0, np.max(np.abs(ref)))
    assert abs(E.item() - Eref) <= E_REL * max(1.0, abs(Eref))


@pytest.mark.parametrize("name", sorted(SMALL))
def test_screen_all_generator_types(torch_cuda, name):
    torch = torch_cuda
    m = SMALL[name]
    cvq, s, p, os_, ops = _setup(torch, m)
    psi = W.random_state(s.dim, 2)
    g = _np(cvq.screen_pool(s, p, torch.from_numpy(psi).cuda()))
    ref = os_.screen(ops, psi)
    assert np.max(np.abs(g - ref)) < G_ABS
    sub = [len(ops) - 1, 0, 3, 3]
    gs = _np(cvq.screen_pool(s, p, torch.from_numpy(psi).cuda(), subset=sub))
    assert np.max(np.abs(gs - ref[sub])) < G_ABS


@pytest.mark.parametrize("name", sorted(SMALL))
def test_apply_ansatz(torch_cuda, name):
    torch = torch_cuda
    m = SMALL[name]
    cvq, s, p, os_, ops = _setup(torch, m)
    ids, th = W.random_ansatz(len(ops), 30, 3, scale=0.6)
    psi0 = W.random_state(s.dim, 4)
    out = _np(cvq.apply_ansatz(s, p, ids, th, torch.from_numpy(psi0).cuda()))
    ref = os_.apply_ansatz([ops[i] for i in ids], th, psi0)
    assert np.max(np.abs(out - ref)) < PSI_ABS
    assert abs(np.linalg.norm(out) - 1.0) < 1e-12
    # in place (psi0 and psi_out alias) and the empty ansatz
    d = torch.from_numpy(psi0).cuda()
    cvq.apply_ansatz(s, p, ids, th, d, out=d)
    assert np.max(np.abs(_np(d) - ref)) < PSI_ABS
    out0 = _np(cvq.apply_ansatz(s, p, [], [], torch.from_numpy(psi0).cuda()))
    assert np.max(np.abs(out0 - psi0)) < 1e-15  # complex128 -> df -> complex128 round trip


@pytest.mark.parametrize("name", sorted(SMALL))
def test_energy_and_grad(torch_cuda, name):
    torch = torch_cuda
    m = SMALL[name]
    cvq, s, p, os_, ops = _setup(torch, m)
    ids, th = W.random_ansatz(len(ops), 24, 5, scale=0.5)
    psi0 = W.random_state(s.dim, 6)
    E, g = cvq.energy_and_grad(s, p, ids, th, torch.from_numpy(psi0).cuda())
    Eref, gref = os_.energy_and_grad([ops[i] for i in ids], th, psi0)
    assert abs(E.item() - Eref) <= E_REL * max(1.0, abs(Eref))
    assert np.max(np.abs(_np(g) - gref)) < G_ABS
    E0, g0 = cvq.energy_and_grad(s, p, [], [], torch.from_numpy(psi0).cuda())
    assert abs(E0.item() - os_.energy(psi0)[0]) <= E_REL * max(1.0, abs(Eref))
    # the same with the forward states kept for the reverse sweep
    Es, gs = cvq.energy_and_grad_stored(s, p, ids, th, torch.from_numpy(psi0).cuda())
    assert abs(Es.item() - Eref) <= E_REL * max(1.0, abs(Eref))
    assert np.max(np.abs(_np(gs) - gref)) < G_ABS
    assert cvq.stored_states_bytes(s, p, []) == 0
    Es0, _ = cvq.energy_and_grad_stored(s, p, [], [], torch.from_numpy(psi0).cuda())
    assert abs(Es0.item() - E0.item()) <= 1e-15 * max(1.0, abs(E0.item()))


@pytest.mark.parametrize("name", ["bh_pbc_L5_N4", "bkck_L4_d6"])
def test_long_diagonal_runs(torch_cuda, name):
    """Consecutive diagonal gates are fused into runs of at most 32 gates and
    4 cross-Kerr terms; longer stretches must split without changing results."""
    torch = torch_cuda
    m = SMALL[name]
    L = m.L
    ops = [W.Op(t, r) for r in range(L) for t in ("kerr", "nn1", "rot")]
    ops += [W.Op("xkerr", i, j) for i in range(L) for j in range(i + 1, L)]
    ops.append(W.Op("hop", 0, 1, 1))
    cvq, s, p, os_, ops = _setup(torch, m, ops=ops)
    rng = np.random.default_rng(9)
    ids = [int(k) for k in rng.integers(0, len(ops) - 1, 75)]
    ids[40] = len(ops) - 1
    xk = [k for k, o in enumerate(ops) if o.type == "xkerr"]
    ids[:12] = [xk[q % len(xk)] for q in range(12)]
    th = rng.uniform(-0.7, 0.7, len(ids))
    psi0 = W.random_state(s.dim, 10)
    E, g = cvq.energy_and_grad(s, p, ids, th, torch.from_numpy(psi0).cuda())
    Eref, gref = os_.energy_and_grad([ops[i] for i in ids], th, psi0)
    assert abs(E.item() - Eref) <= E_REL * max(1.0, abs(Eref))
    assert np.max(np.abs(_np(g) - gref)) < G_ABS
    Es, gs = cvq.energy_and_grad_stored(s, p, ids, th, torch.from_numpy(psi0).cuda())
    assert abs(Es.item() - Eref) <= E_REL * max(1.0, abs(Eref))
    assert np.max(np.abs(_np(gs) - gref)) < G_ABS
    out = _np(cvq.apply_ansatz(s, p, ids, th, torch.from_numpy(psi0).cuda()))
    assert np.max(np.abs(out - os_.apply_ansatz([ops[i] for i in ids], th, psi0))) < PSI_ABS


MEDIUM = {
    "bh_pbc_L8_N6": W.bose_hubbard(8, 6, J=1.0, U=-2.5, periodic=True),
    "bh_open_L6_N9": W.bose_hubbard(6, 9, J=0.7, U=1.3, periodic=False),
    "bkck_L6_d6": W.kitaev_kerr(6, 6, t=1.0, Delta=0.6, K=0.3, periodic=False),
    "bkc_L5_d8_odd": W.kitaev_paper(5, 8, J=1.0, Delta=0.5, mu=-3.1, U=-1.0, periodic=True, parity=1),
}


@pytest.mark.parametrize("name", sorted(MEDIUM))
def test_medium_sectors_span_many_tiles(torch_cuda, name):
    """Sectors of 1.7k..16k amplitudes: many CTAs, ragged tails, all calls."""
    torch = torch_cuda
    m = MEDIUM[name]
    ops = W.bh_allpairs_pool(m.L) if m.kind == "bh" else W.bkc_kerr_pool(m.L)
    cvq, s, p, os_, ops = _setup(torch, m, ops=ops)
    psi0 = W.random_state(s.dim, 7)
    d0 = torch.from_numpy(psi0).cuda()
    sig = _np(cvq.apply_H(s, d0))
    assert np.max(np.abs(sig - os_.apply_H(psi0))) < 1e-11 * max(1.0, np.max(np.abs(sig)))
    g = _np(cvq.screen_pool(s, p, d0))
    assert np.max(np.abs(g - os_.screen(ops, psi0))) < G_ABS
    ids, th = W.random_ansatz(len(ops), 12, 8, scale=0.4)
    E, gr = cvq.energy_and_grad(s, p, ids, th, d0)
    Eref, gref = os_.energy_and_grad([ops[i] for i in ids], th, psi0)
    assert abs(E.item() - Eref) <= E_REL * max(1.0, abs(Eref))
    assert np.max(np.abs(_np(gr) - gref)) < G_ABS


# ------------------------------------------------------------- full size

FULL = {
    "c2_bh_pbc_L12_N12": lambda: W.c2_model(3.4),
    "c3_bkck_L8_d8": lambda: W.c3_model(0, K=0.1),
    "c5_bkck_L10_d6": lambda: W.c5_model(),
}


@pytest.mark.parametrize("name", sorted(FULL))
def test_full_size_apply_H_sampled_rows(torch_cuda, name):
    torch = torch_cuda
    m = FULL[name]()
    from oracle.core import Sector as OS
    from paper_2606_05297_gb300 import cvq
    s = cvq.Sector(m)
    os_ = OS(m)
    assert s.dim == os_.dim
    psi = W.random_state(s.dim, 11)
    sig = _np(cvq.apply_H(s, torch.from_numpy(psi).cuda()))
    rng = np.random.default_rng(0)
    rows = np.concatenate([rng.integers(0, s.dim, 3000), [0, 1, s.dim - 2, s.dim - 1]])
    ref = os_.apply_rows(os_.H, psi, rows)
    assert np.max(np.abs(sig[rows] - ref)) < PSI_ABS * max(1.0, np.max(np.abs(ref)))


def test_full_size_c2_energy_screen_and_gate(torch_cuda):
    """Bose-Hubbard L=12, N=12 at full size: energy, three screened pool
    elements and one beam-splitter gate against the oracle."""
    torch = torch_cuda
    m = W.c2_model(3.4)
    ops = W.bh_allpairs_pool(12)
    cvq, s, p, os_, ops = _setup(torch, m, ops=ops)
    psi = W.random_state(s.dim, 12)
    d = torch.from_numpy(psi).cuda()
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    cvq.apply_H(s, d, energy=E)
    Eref, _ = os_.energy(psi)
    assert abs(E.item() - Eref) <= E_REL * max(1.0, abs(Eref))
    sub = [0, 31, 209]
    g = _np(cvq.screen_pool(s, p, d, subset=sub))
    gref = os_.screen([ops[k] for k in sub], psi)
    assert np.max(np.abs(g - gref)) < G_ABS
    out = _np(cvq.apply_ansatz(s, p, [31], [0.3], d))
    ref = os_.expm_apply(ops[31], 0.3, psi)
    assert np.max(np.abs(out - ref)) < PSI_ABS


@pytest.mark.parametrize("name", ["c2_bh_pbc_L12_N12", "c3_bkck_L8_d8"])
def test_full_size_properties(torch_cuda, name):
    """At full size: norm conservation, U(-theta) U(theta) = 1, the adjoint
    gradient equals a central difference, the appended zero-angle gradient
    equals the screen, and repeated calls are bit-identical."""
    torch = torch_cuda
    from paper_2606_05297_gb300 import cvq
    m = FULL[name]()
    ops = W.bh_allpairs_pool(m.L) if m.kind == "bh" else W.bkc_kerr_pool(m.L)
    s = cvq.Sector(m)
    p = cvq.Pool(s, ops)
    depth = 40 if m.kind == "bkc" else 16
    ids, th = W.random_ansatz(len(ops), depth, 13, scale=0.2)
    psi0 = s.basis_state(W.initial_occupation(m)) if m.kind == "bkc" else torch.from_numpy(
        W.random_state(s.dim, 14)).cuda()
    ws = s.workspace(p, depth + 1)
    out = cvq.apply_ansatz(s, p, ids, th, psi0, ws=ws)
    assert abs(torch.linalg.vector_norm(out).item() - 1.0) < 1e-11
    back = cvq.apply_ansatz(s, p, ids[::-1], -th[::-1], out, ws=ws)
    assert torch.max(torch.abs(back - psi0)).item() < 1e-11
    E, g = cvq.energy_and_grad(s, p, ids, th, psi0, ws=ws)
    E2, g2 = cvq.energy_and_grad(s, p, ids, th, psi0, ws=ws)
    assert E.item() == E2.item() and torch.equal(g, g2)
    h = 1e-4
    for k in (0, depth // 2, depth - 1):
        def f(x):
            t = th.copy()
            t[k] += x
            return cvq.energy_and_grad(s, p, ids, t, psi0, ws=ws)[0].item()
        fd = (-f(2 * h) + 8 * f(h) - 8 * f(-h) + f(-2 * h)) / (12 * h)
        assert abs(g[k].item() - fd) < 1e-7 * max(1.0, abs(E.item())), (k, g[k].item(), fd)
    sub = [5, 17]
    gs = _np(cvq.screen_pool(s, p, out, subset=sub, ws=ws))
    for q, k in enumerate(sub):
        _, ga = cvq.energy_and_grad(s, p, ids + [k], np.append(th, 0.0), psi0, ws=ws)
        assert abs(ga[-1].item() - gs[q]) < G_ABS


def test_errors_are_reported(torch_cuda):
    torch = torch_cuda
    from paper_2606_05297_gb300 import cvq
    s = cvq.Sector(W.c1_model())
    with pytest.raises(cvq.CvqError, match="breaks"):
        cvq.Pool(s, [W.Op("sq2", 0, 1, 0)])
    p = cvq.Pool(s, W.bh_nn_pool(W.c1_model()))
    psi = s.basis_state([1, 1, 1, 1])
    with pytest.raises(cvq.CvqError, match="outside the pool"):
        cvq.apply_ansatz(s, p, [99], [0.1], psi)
    small = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(cvq.CvqError, match="workspace"):
        cvq.energy_and_grad(s, p, [0], [0.1], psi, ws=small)
    with pytest.raises(cvq.CvqError):
        cvq.Sector(W.kitaev_paper(3, 5, periodic=True))  # odd cutoff
    with pytest.raises(cvq.CvqError, match="not finite"):
        cvq.apply_ansatz(s, p, [0], [float("nan")], psi)
