"""Pins of the projected-gate oracle (oracle/projected.py): textbook closed
forms of the untruncated gates, exactness of finite blocks, reduction to the
plain gates where no block is cut, and finite differences of the normalised
energy."""
import math

import numpy as np
import pytest

from oracle.core import Sector
from oracle.projected import Projected, local_generator
from paper_2606_05297_gb300 import workloads as W


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


def test_beam_splitter_elements_beyond_the_cutoff_class():
    """A class M = n1 + n2 above d - 1 is cut by the truncation, but the
    projected gate keeps the untruncated elements: d^{M/2}(2 theta) (spin-M/2
    rotation of the Schwinger representation), exact once dc >= M + 1."""
    d, dc, theta = 4, 7, 0.41
    s = Sector(W.kitaev_paper(2, d, periodic=False, parity=0))
    U, _ = Projected(s, dc).matrices(W.Op("hop", 0, 1, 0), theta)
    for M in range(d, 2 * d - 1):
        for a in range(M - d + 1, d):
            for ap in range(M - d + 1, d):
                ref = _wigner_small_d(M, 2 * ap - M, 2 * a - M, 2 * theta)
                assert abs(U[ap * dc + (M - ap), a * dc + (M - a)] - ref) < 1e-13


def test_squeezed_vacua_closed_forms():
    r = 0.3
    s1 = Sector(W.kitaev_paper(1, 8, periodic=False, parity=0))
    U, _ = Projected(s1, 80).matrices(W.Op("sq1", 0, -1, 0), r)
    for k in range(4):
        ref = (-math.tanh(r)) ** k * math.sqrt(math.factorial(2 * k)) / (2 ** k * math.factorial(k)) / math.sqrt(
            math.cosh(r))
        assert abs(U[2 * k, 0] - ref) < 1e-13
    s2 = Sector(W.kitaev_paper(2, 6, periodic=False, parity=0))
    dc = 40
    U, _ = Projected(s2, dc).matrices(W.Op("sq2", 0, 1, 0), r)
    for k in range(6):
        assert abs(U[k * dc + k, 0] - (-math.tanh(r)) ** k / math.cosh(r)) < 1e-13


def test_generator_is_anti_hermitian_and_derivative():
    for op in (W.Op("hop", 0, 1, 1), W.Op("sq2", 0, 1, 3), W.Op("sq1", 0, -1, 1), W.Op("kerr", 0)):
        A = local_generator(op, 9)
        assert np.allclose(A, -A.conj().T, atol=1e-14)
    s = Sector(W.kitaev_paper(2, 4, periodic=False, parity=0))
    P = Projected(s, 10)
    op, th, h = W.Op("sq2", 0, 1, 1), 0.3, 1e-6
    U, D = P.matrices(op, th)
    Up, _ = P.matrices(op, th + h)
    Um, _ = P.matrices(op, th - h)
    assert np.max(np.abs((Up - Um) / (2 * h) - D)) < 1e-8


def test_reduces_to_plain_gates_when_nothing_is_cut():
    """Bose-Hubbard sectors never leave the cutoff D = N + 1: the projected
    sweep equals the plain one (every norm 1)."""
    m = W.bose_hubbard(4, 3, J=1.0, U=2.0, periodic=True)
    s = Sector(m)
    rng = np.random.default_rng(2)
    pool = W.bh_allpairs_pool(4) + [W.Op("rot", r) for r in range(4)]
    ops = [pool[k] for k in rng.integers(0, len(pool), 12)]
    th = rng.uniform(-0.7, 0.7, 12)
    psi0 = W.random_state(s.dim, 3)
    P = Projected(s, 4)
    states, norms = P.forward(ops, th, psi0)
    assert np.allclose(norms, 1.0, atol=1e-13)
    E, g = P.energy_and_grad(ops, th, psi0)
    Er, gr = s.energy_and_grad(ops, th, psi0)
    assert abs(E - Er) < 1e-12 * max(1, abs(Er)) and np.max(np.abs(g - gr)) < 1e-11


@pytest.mark.parametrize("dc", [8, 12])
def test_gradient_matches_finite_differences(dc):
    m = W.kitaev_kerr(3, 4, t=1.0, Delta=0.6, K=0.3)
    s = Sector(m)
    pool = W.bkc_kerr_pool(3) + [W.Op("rot", r) for r in range(3)]
    rng = np.random.default_rng(7)
    ops = [pool[k] for k in rng.integers(0, len(pool), 14)]
    th = rng.uniform(-0.6, 0.6, 14)
    psi0 = s.basis_state([0, 0, 0])
    P = Projected(s, dc)
    states, norms = P.forward(ops, th, psi0)
    assert min(norms) < 1 - 1e-6  # the cutoff really cuts
    assert all(abs(np.linalg.norm(v) - 1) < 1e-13 for v in states)
    E, g = P.energy_and_grad(ops, th, psi0)
    h = 1e-5
    for k in range(len(ops)):
        e = np.zeros(len(ops))
        e[k] = h
        fd = (P.energy_and_grad(ops, th + e, psi0)[0] - P.energy_and_grad(ops, th - e, psi0)[0]) / (2 * h)
        assert abs(fd - g[k]) < 1e-7 * max(1.0, abs(g[k])), (k, fd, g[k])
