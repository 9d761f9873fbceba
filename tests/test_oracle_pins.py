"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics,
not by the oracle itself (CPU only).

Each test names the passage of arXiv 2606.05297 or the textbook result it
checks.  Together they are chosen so that a dropped term, a wrong sign or
index, or a transposed operand in the oracle fails at least one of them.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import adapt as oadapt
from oracle import bfgs as obfgs
from oracle import operators as oops
from oracle.core import Operator, Sector
from oracle.dense import FullSpace
from paper_2606_05297_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _bh(L, N, hop, nn1, periodic, n2=None, n1=None):
    nb = L if periodic else L - 1
    return W.Model("bh", L, N=N, periodic=periodic, hop=list(hop)[:nb], pair=[0.0] * nb, nn1=list(nn1),
                   n2=list(n2 or [0.0] * L), n1=list(n1 or [0.0] * L))


# ------------------------------------------------------------------ sectors

@pytest.mark.parametrize("L,N", [(1, 3), (2, 5), (4, 4), (5, 3), (6, 6), (12, 12)])
def test_bh_sector_dim_is_binomial(L, N):
    """Fixed-N sector (Sec. III.A) = compositions of N into L parts: C(N+L-1, L-1)."""
    s = Sector(W.bose_hubbard(L, N, periodic=False))
    assert s.dim == math.comb(N + L - 1, L - 1)


def test_config_sector_dims():
    """Sector sizes of the workloads: 35, 1,352,078 and 8,388,608 amplitudes."""
    assert Sector(W.c1_model()).dim == 35
    assert Sector(W.c2_model()).dim == 1352078
    assert Sector(W.c3_model()).dim == 8388608


@pytest.mark.parametrize("L,d,p", [(3, 4, 0), (3, 4, 1), (4, 5, 0), (3, 5, 1), (1, 7, 0)])
def test_bkc_sector_dim(L, d, p):
    """Parity sector (Sec. III.B, P = (-1)^N_tot): brute-force count over {0..d-1}^L."""
    cnt = sum(1 for t in itertools.product(range(d), repeat=L) if sum(t) % 2 == p)
    s = Sector(W.kitaev_paper(L, d, parity=p, periodic=False))
    assert s.dim == cnt
    if d % 2 == 0 and L >= 1:
        assert s.dim == d ** L // 2


def test_sector_order_is_lexicographic():
    s = Sector(W.bose_hubbard(4, 5, periodic=False))
    t = s.tuples()
    assert all(tuple(t[i]) < tuple(t[i + 1]) for i in range(len(t) - 1))
    assert np.all(t.sum(axis=1) == 5)
    for x in (0, 7, len(t) - 1):
        assert s.index(t[x]) == x


# ------------------------------------------------- operators vs Kronecker

MODELS = [
    _bh(3, 3, [-1.0, -0.7, -1.3], [0.4, -0.2, 0.1], True),
    _bh(4, 3, [-1.0, -0.5, -1.5], [-1.0, 0.3, 0.0, 0.2], False, n2=[0.1, 0, 0, 0.2], n1=[0.0, 0.5, 0, 0]),
    W.kitaev_paper(3, 4, J=1.0, Delta=0.5, mu=-2.7, U=-1.0, periodic=True, parity=0),
    W.kitaev_paper(3, 4, J=0.8, Delta=0.3, mu=-3.1, periodic=True, parity=1),
    W.kitaev_kerr(4, 3, t=1.0, Delta=[0.2, 0.7, 0.4], K=0.5, periodic=False, parity=0),
]


@pytest.mark.parametrize("m", MODELS)
def test_hamiltonian_matches_dense_kronecker(m):
    """Ladder-string H in the sector == full-space Kronecker H restricted, entrywise
    (Eqs. BoseHubbard, BosonicKitaevChain, BosonicKitaevChain_Kerr)."""
    s = Sector(m)
    fs = FullSpace(m)
    Hs = s.matrix(s.H)
    Hd = fs.restrict(fs.hamiltonian())
    assert s.dim == len(fs.sector_idx)
    np.testing.assert_array_equal(s.tuples(), fs.sector_occ)
    assert np.max(np.abs(Hs - Hd)) < 1e-13
    assert np.max(np.abs(Hs - Hs.conj().T)) < 1e-14
    # the full-space H never couples the sector to its complement (symmetry, Sec. III)
    Hfull = fs.hamiltonian()
    out = np.setdiff1d(np.arange(Hfull.shape[0]), fs.sector_idx)
    assert np.max(np.abs(Hfull[np.ix_(out, fs.sector_idx)]), initial=0.0) == 0.0


ALL_OPS_BKC = [W.Op("hop", 0, 2, 0), W.Op("hop", 2, 1, 1), W.Op("hop", 1, 0, 3), W.Op("sq2", 0, 1, 0),
               W.Op("sq2", 2, 0, 1), W.Op("sq1", 1, -1, 0), W.Op("sq1", 2, -1, 1), W.Op("kerr", 0),
               W.Op("nn1", 1), W.Op("rot", 2), W.Op("xkerr", 0, 2), W.Op("pairhop", 0, 1, 1),
               W.Op("pairhop", 2, 0, 0)]
ALL_OPS_BH = [W.Op("hop", 0, 1, 0), W.Op("hop", 2, 0, 1), W.Op("pairhop", 1, 2, 1), W.Op("pairhop", 0, 2, 0),
              W.Op("kerr", 1), W.Op("nn1", 2), W.Op("rot", 0), W.Op("xkerr", 1, 2)]


@pytest.mark.parametrize("m,ops", [(MODELS[2], ALL_OPS_BKC), (MODELS[3], ALL_OPS_BKC), (MODELS[0], ALL_OPS_BH)])
def test_generators_match_dense_and_are_antihermitian(m, ops):
    """Pool generators (Sec. II.B gates, Sec. IV.B O_r = exp(theta A_r)) are
    anti-Hermitian and preserve the sector."""
    s = Sector(m)
    fs = FullSpace(m)
    out = np.setdiff1d(np.arange(fs.a[0].shape[0]), fs.sector_idx)
    for o in ops:
        A = s.matrix(s.op(o))
        Ad_full = fs.generator(o)
        assert np.max(np.abs(A - fs.restrict(Ad_full))) < 1e-13, o
        assert np.max(np.abs(A + A.conj().T)) < 1e-14, o
        assert np.max(np.abs(Ad_full[np.ix_(out, fs.sector_idx)]), initial=0.0) == 0.0, o


# --------------------------------------------------------- closed forms

@pytest.mark.parametrize("L,N,periodic", [(5, 3, False), (4, 2, False), (5, 3, True), (6, 2, True)])
def test_free_bosons_closed_form(L, N, periodic):
    """U = 0 Bose-Hubbard: all N bosons in the lowest orbital.  D = N + 1 makes
    the truncation exact (Sec. III.A), so E0 = N * eps_0 with eps_0 =
    -2J cos(pi/(L+1)) (open chain) or -2J (periodic)."""
    J = 0.9
    s = Sector(W.bose_hubbard(L, N, J=J, U=0.0, periodic=periodic))
    E0 = np.linalg.eigvalsh(s.matrix(s.H))[0]
    eps0 = -2 * J if periodic else -2 * J * math.cos(math.pi / (L + 1))
    assert abs(E0 - N * eps0) < 1e-12


def test_kitaev_bdg_large_cutoff_limit():
    """App. A: for the stable chain (mu < -2(J + Delta)) the ground energy of the
    quadratic Hamiltonian is (1/2) sum_k (E(k) - xi_k), E(k) = sqrt(xi_k^2 -
    Delta_k^2), xi_k = -2J cos k - mu, Delta_k = 2 Delta cos k.  The truncated
    even sector converges to it exponentially in the cutoff d."""
    L, J, Dl, mu = 3, 1.0, 0.3, -4.0
    k = 2 * np.pi * np.arange(L) / L
    xi = -2 * J * np.cos(k) - mu
    Dk = 2 * Dl * np.cos(k)
    E_bdg = 0.5 * np.sum(np.sqrt(xi ** 2 - Dk ** 2) - xi)
    errs = []
    for d in (4, 6, 8, 12):
        s = Sector(W.kitaev_paper(L, d, J=J, Delta=Dl, mu=mu, periodic=True, parity=0))
        errs.append(np.linalg.eigvalsh(s.matrix(s.H))[0] - E_bdg)
    assert all(e > -1e-14 for e in errs)                   # variational from above
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 2))
    assert abs(errs[-1]) < 1e-13


def test_pair_sign_gauge_invariance():
    """a_j -> i^j a_j flips the sign of the nearest-neighbour pairing on an open
    chain and leaves hopping and n-terms unchanged, so E0(Delta) = E0(-Delta)."""
    m1 = W.kitaev_kerr(4, 4, t=1.0, Delta=0.4, K=0.3, periodic=False)
    m2 = W.kitaev_kerr(4, 4, t=1.0, Delta=-0.4, K=0.3, periodic=False)
    e1 = np.linalg.eigvalsh(Sector(m1).matrix(Sector(m1).H))[0]
    e2 = np.linalg.eigvalsh(Sector(m2).matrix(Sector(m2).H))[0]
    assert abs(e1 - e2) < 1e-12


def _wigner_small_d(j2, mp2, m2, beta):
    f = math.factorial
    j, mp, m = j2 / 2, mp2 / 2, m2 / 2
    out = 0.0
    for s in range(0, j2 + 1):
        args = (j + m - s, s, mp - m + s, j - mp - s)
        if min(args) < -1e-9:
            continue
        a, b, c, e = (int(round(v)) for v in args)
        num = math.sqrt(f(int(round(j + mp))) * f(int(round(j - mp))) * f(int(round(j + m))) * f(int(round(j - m))))
        out += ((-1) ** int(round(mp - m + s)) * num / (f(a) * f(b) * f(c) * f(e))
                * math.cos(beta / 2) ** int(round(2 * j + m - mp - 2 * s))
                * math.sin(beta / 2) ** int(round(mp - m + 2 * s)))
    return out


@pytest.mark.parametrize("m", [1, 2, 3, 6])
def test_beam_splitter_block_is_wigner_d(m):
    """BS(theta, 0) = exp[theta (a_1 a_2^dag - a_1^dag a_2)] (Sec. II.B) on the
    m-boson block is the spin-m/2 rotation exp(-i 2theta J_y) of the Schwinger
    representation J_z = (n_1 - n_2)/2, so its matrix is d^{m/2}(2 theta)."""
    theta = 0.37
    s = Sector(W.bose_hubbard(2, m, periodic=False))
    tup = s.tuples()
    op = W.Op("hop", 0, 1, 0)
    M = np.zeros((s.dim, s.dim), dtype=complex)
    for x in range(s.dim):
        e = np.zeros(s.dim, dtype=complex)
        e[x] = 1
        M[:, x] = s.expm_apply(op, theta, e)
    for y in range(s.dim):
        for x in range(s.dim):
            mz2 = int(tup[x][0] - tup[x][1])
            mzp2 = int(tup[y][0] - tup[y][1])
            assert abs(M[y, x] - _wigner_small_d(m, mzp2, mz2, 2 * theta)) < 1e-13
    if m == 1:  # cos(theta)|1,0> + sin(theta)|0,1>
        v = s.expm_apply(op, theta, s.basis_state([1, 0]))
        assert abs(v[s.index([1, 0])] - math.cos(theta)) < 1e-15
        assert abs(v[s.index([0, 1])] - math.sin(theta)) < 1e-15


def test_single_mode_squeezed_vacuum():
    """S(r, 0)|0> = sech(r)^(1/2) sum_k (-tanh r)^k sqrt((2k)!)/(2^k k!) |2k>
    (textbook, for S = exp[r/2 (a^2 - a^dag^2)] of Sec. II.B), at cutoff 60."""
    r = 0.3
    s = Sector(W.kitaev_paper(1, 60, periodic=False, parity=0))
    v = s.expm_apply(W.Op("sq1", 0, -1, 0), r, s.basis_state([0]))
    for k in range(20):
        ref = (-math.tanh(r)) ** k * math.sqrt(math.factorial(2 * k)) / (2 ** k * math.factorial(k)) / math.sqrt(
            math.cosh(r))
        assert abs(v[s.index([2 * k])] - ref) < 1e-13


def test_two_mode_squeezed_vacuum():
    """S2(r, 0)|00> = sech(r) sum_k (-tanh r)^k |k, k> (textbook, for
    S2 = exp[r (a_1 a_2 - a_1^dag a_2^dag)] of Sec. II.B), at cutoff 30."""
    r = 0.25
    s = Sector(W.kitaev_paper(2, 30, periodic=False, parity=0))
    v = s.expm_apply(W.Op("sq2", 0, 1, 0), r, s.basis_state([0, 0]))
    for k in range(30):
        ref = (-math.tanh(r)) ** k / math.cosh(r)
        assert abs(v[s.index([k, k])] - ref) < 1e-13
    mask = np.ones(s.dim, bool)
    for k in range(30):
        mask[s.index([k, k])] = False
    assert np.max(np.abs(v[mask])) < 1e-16


def test_diagonal_gates_are_phases():
    """R = exp(i theta N), K = exp(i theta N^2), CK = exp(i theta N_1 N_2)
    (Sec. II.B) and exp(i theta N(N-1)) act on Fock states as pure phases."""
    th = 0.41
    s = Sector(W.kitaev_paper(3, 4, periodic=False, parity=1))
    for x, t in enumerate(s.tuples()):
        e = s.basis_state(t)
        for op, f in [(W.Op("rot", 1), t[1]), (W.Op("kerr", 2), t[2] ** 2), (W.Op("nn1", 0), t[0] * (t[0] - 1)),
                      (W.Op("xkerr", 0, 2), t[0] * t[2])]:
            v = s.expm_apply(op, th, e)
            assert abs(v[x] - np.exp(1j * th * f)) < 1e-14
            assert np.sum(np.abs(v)) - abs(v[x]) < 1e-15


def test_gates_unitary_and_symmetric_against_dense_expm():
    """exp(theta A) from the oracle's Taylor series equals the dense
    scipy.linalg.expm in the full space, is norm preserving, and leaves no
    weight outside the symmetry sector (N or parity conservation)."""
    import scipy.linalg
    m = MODELS[2]
    s = Sector(m)
    fs = FullSpace(m)
    psi = W.random_state(s.dim, 5)
    for o, th in zip(ALL_OPS_BKC, np.linspace(-0.6, 0.7, len(ALL_OPS_BKC))):
        v = s.expm_apply(o, th, psi)
        full = scipy.linalg.expm(th * fs.generator(o)) @ fs.embed_state(psi)
        assert np.max(np.abs(full[fs.sector_idx] - v)) < 1e-13, o
        assert abs(np.linalg.norm(full) - np.linalg.norm(full[fs.sector_idx])) < 1e-15
        assert abs(np.linalg.norm(v) - 1.0) < 1e-13
    ids, th = W.random_ansatz(len(ALL_OPS_BKC), 40, 3, scale=0.5)
    v = s.apply_ansatz([ALL_OPS_BKC[i] for i in ids], th, psi)
    assert abs(np.linalg.norm(v) - 1.0) < 1e-13


# ------------------------------------------------------------- gradients

def test_fock_state_gradients_closed_form():
    """Eq. (grad) on a Fock product state |n>: real hopping on a bond with H
    coefficient t gives g = 2 t (n_i - n_j); every other pair, imaginary hopping,
    pair hopping and diagonal generators give 0 (Sec. IV.B: diagonal generators
    vanish on Fock product states)."""
    m = _bh(4, 6, [-1.0, -0.7, -1.3], [0.4, -0.2, 0.1, 0.3], False)
    s = Sector(m)
    occ = [2, 0, 1, 3]
    psi = s.basis_state(occ)
    pool = W.bh_allpairs_pool(4) + [W.Op("nn1", r) for r in range(4)] + [W.Op("xkerr", 0, 3)]
    g, gi = s.screen(pool, psi, return_imag=True)
    bond = {(0, 1): -1.0, (1, 2): -0.7, (2, 3): -1.3}
    for k, o in enumerate(pool):
        if o.type == "hop" and o.phase == 0 and (o.i, o.j) in bond:
            exp = 2 * bond[(o.i, o.j)] * (occ[o.i] - occ[o.j])
        else:
            exp = 0.0
        assert abs(g[k] - exp) < 1e-13, (o, g[k], exp)
    assert np.max(np.abs(gi)) < 1e-13


def _fd4(f, h):
    return (-f(2 * h) + 8 * f(h) - 8 * f(-h) + f(-2 * h)) / (12 * h)


@pytest.mark.parametrize("which", ["bh", "bkc"])
def test_screen_equals_finite_difference(which):
    """g_r = dE/dtheta_r at theta_r = 0 (Eq. grad) against a 4-point central
    difference of E(exp(theta A_r) psi)."""
    if which == "bh":
        m, pool = MODELS[0], W.bh_allpairs_pool(3) + [W.Op("nn1", 1), W.Op("xkerr", 0, 2)]
    else:
        m, pool = MODELS[2], ALL_OPS_BKC
    s = Sector(m)
    psi = W.random_state(s.dim, 11)
    g, gi = s.screen(pool, psi, return_imag=True)
    for k, o in enumerate(pool):
        fd = _fd4(lambda h: s.energy(s.expm_apply(o, h, psi))[0], 1e-3)
        assert abs(g[k] - fd) < 1e-9 * max(1.0, abs(fd)), (o, g[k], fd)
    assert np.max(np.abs(gi)) < 1e-12


@pytest.mark.parametrize("which", ["bh", "bkc"])
def test_ansatz_gradient_equals_finite_difference(which):
    """Adjoint dE/dtheta_k of E = <psi_n|H|psi_n> (Sec. IV.B) against a
    4-point central difference in each theta_k, depth 8."""
    if which == "bh":
        m, pool = MODELS[1], [W.Op("hop", 0, 1, 0), W.Op("hop", 1, 3, 1), W.Op("pairhop", 0, 2, 1),
                              W.Op("kerr", 2), W.Op("nn1", 3), W.Op("rot", 0), W.Op("xkerr", 1, 2)]
    else:
        m, pool = MODELS[4], [W.Op("hop", 0, 1, 0), W.Op("hop", 1, 3, 1), W.Op("sq2", 0, 2, 0),
                              W.Op("sq2", 2, 3, 1), W.Op("sq1", 1, -1, 0), W.Op("sq1", 3, -1, 1), W.Op("kerr", 2)]
    s = Sector(m)
    ids, th = W.random_ansatz(len(pool), 8, 21, scale=0.4)
    ops = [pool[i] for i in ids]
    psi0 = W.random_state(s.dim, 4)
    E, g = s.energy_and_grad(ops, th, psi0)
    Ef = s.energy(s.apply_ansatz(ops, th, psi0))[0]
    assert abs(E - Ef) < 1e-13
    for k in range(len(ops)):
        def f(h):
            t2 = th.copy()
            t2[k] += h
            return s.energy(s.apply_ansatz(ops, t2, psi0))[0]
        fd = _fd4(f, 1e-3)
        assert abs(g[k] - fd) < 1e-8 * max(1.0, abs(E)), (k, g[k], fd)


def test_appended_zero_angle_gradient_equals_screen():
    """Appending O_{n+1} with theta = 0 (Sec. IV.B growth rule) leaves the state
    unchanged, and its adjoint gradient is the Eq. (grad) screen value."""
    m = MODELS[2]
    s = Sector(m)
    ids, th = W.random_ansatz(len(ALL_OPS_BKC), 6, 8, scale=0.4)
    ops = [ALL_OPS_BKC[i] for i in ids]
    psi0 = W.random_state(s.dim, 9)
    psi = s.apply_ansatz(ops, th, psi0)
    g_screen = s.screen(ALL_OPS_BKC, psi)
    for k, o in enumerate(ALL_OPS_BKC):
        _, g = s.energy_and_grad(ops + [o], np.append(th, 0.0), psi0)
        assert abs(g[-1] - g_screen[k]) < 1e-12


def test_phi_derivative_vanishes_at_zero():
    """Sec. IV.B: for the two-parameter gates dE/dphi = 0 at (theta, phi) = 0,
    since exp(theta A(phi)) is the identity at theta = 0 for every phi."""
    m = MODELS[2]
    s = Sector(m)
    psi = W.random_state(s.dim, 13)
    for p in range(4):
        # E(theta=0, phi) does not depend on phi: the gate is the identity
        v = s.expm_apply(W.Op("hop", 0, 1, p), 0.0, psi)
        assert np.max(np.abs(v - psi)) == 0.0


# ------------------------------------------------------------ pool facts

def test_pool_sizes_and_hva_layer_from_paper():
    """App. B: the full Kitaev-chain pool at N_S = 5 has 30 operators (BS and S2
    on all pairs, S and R per site).  Sec. IV.A: an HVA layer has 3 N_S gates
    with periodic boundaries (BH: BS per bond, K and R per site)."""
    with open(os.path.join(GOLDEN, "paper_facts.json")) as f:
        facts = json.load(f)
    assert len(W.paper_bkc_pool_two_param(5)) == facts["bkc_pool_size_NS5"]
    for L in (3, 4, 5):
        assert len(W.hva_layer(W.bose_hubbard(L, L, periodic=True))) == facts["hva_gates_per_layer_per_site"] * L
        mk = W.kitaev_paper(L, 4, U=-1.0, periodic=True)
        assert len(W.hva_layer(mk)) == facts["hva_gates_per_layer_per_site_kerr"] * L
    assert len(W.bh_nn_pool(W.c1_model())) == 10
    assert len(W.bh_allpairs_pool(12)) == 210
    assert len(W.bkc_kerr_pool(8)) == 136
    assert len(W.bkc_kerr_pool(10)) == 210
    # Fig. 2: N_S = 3, D = 6 allows at most N_tot = 3 * 5 = 15
    s = Sector(W.kitaev_paper(3, 6, parity=1, periodic=True))
    assert s.tuples().sum(axis=1).max() == facts["max_Ntot_NS3_D6"]


# --------------------------------------------------------------- optimiser

def test_bfgs_rosenbrock_and_quadratic():
    """BFGS (Nocedal & Wright Alg. 6.1): Rosenbrock from (-1.2, 1) reaches (1, 1);
    a strictly convex quadratic reaches A^-1 b."""
    def rosen(x):
        f = 100 * (x[1] - x[0] ** 2) ** 2 + (1 - x[0]) ** 2
        g = np.array([-400 * x[0] * (x[1] - x[0] ** 2) - 2 * (1 - x[0]), 200 * (x[1] - x[0] ** 2)])
        return f, g
    r = obfgs.minimize(rosen, [-1.2, 1.0], gtol=1e-10, max_iter=500)
    assert np.max(np.abs(r["x"] - 1.0)) < 1e-8
    rng = np.random.default_rng(0)
    M = rng.standard_normal((6, 6))
    A = M @ M.T + 6 * np.eye(6)
    b = rng.standard_normal(6)
    r = obfgs.minimize(lambda x: (0.5 * x @ A @ x - b @ x, A @ x - b), np.zeros(6), gtol=1e-12)
    assert np.max(np.abs(r["x"] - np.linalg.solve(A, b))) < 1e-10


def test_selection_tie_rule():
    """Ties in argmax|g| (Sec. IV.B is silent): lowest pool index within 1e-9 relative."""
    assert oadapt.select([0.1, -2.0, 2.0, 1.0])[0] == 1
    assert oadapt.select([0.1, 2.0 * (1 - 5e-10), -2.0])[0] == 1
    assert oadapt.select([0.1, 2.0 * (1 - 5e-9), -2.0])[0] == 2


def test_mott_start_has_zero_gradients():
    """Sec. IV.B: on the Fock product start |1,1,1,1> every gradient of the
    nearest-neighbour pool vanishes (real hops by n_i = n_j, the rest by the
    Fock-state argument), so a warm start is needed."""
    m = W.c1_model()
    s = Sector(m)
    g = s.screen(W.bh_nn_pool(m), s.basis_state(W.mott_occupation(4, 4)))
    assert np.max(np.abs(g)) == 0.0


# --------------------------------------- planted mistakes must fail the pins

def test_planted_sign_error_in_beam_splitter_fails_wigner_pin(monkeypatch):
    """A wrong relative sign in the BS generator makes it Hermitian; the
    anti-Hermiticity and Wigner-d pins must catch it."""
    orig = oops.generator_strings

    def bad(op):
        st = orig(op)
        if op.type == "hop":
            (c0, f0), (c1, f1) = st
            return [(c0, f0), (-c1, f1)]
        return st
    A = Sector(W.bose_hubbard(2, 2, periodic=False))
    Op = Operator(bad(W.Op("hop", 0, 1, 0)))
    M = A.matrix(Op)
    assert np.max(np.abs(M + M.conj().T)) > 0.5


def test_planted_dropped_pair_term_fails_bdg_pin():
    """Dropping the pairing term of Eq. (BosonicKitaevChain) moves E0 far from
    the App. A value."""
    L, J, Dl, mu = 3, 1.0, 0.3, -4.0
    k = 2 * np.pi * np.arange(L) / L
    xi = -2 * J * np.cos(k) - mu
    E_bdg = 0.5 * np.sum(np.sqrt(xi ** 2 - (2 * Dl * np.cos(k)) ** 2) - xi)
    m = W.kitaev_paper(L, 10, J=J, Delta=Dl, mu=mu, periodic=True)
    m.pair = [0.0] * len(m.pair)
    s = Sector(m)
    assert abs(np.linalg.eigvalsh(s.matrix(s.H))[0] - E_bdg) > 1e-2
