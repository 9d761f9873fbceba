"""Pins of the scorer oracle (oracle/mlp.py) to facts outside itself:
bfloat16 rounding at hand-worked ties and against torch's own conversion, a
network with hand-set weights whose output is known in closed form, central
finite differences of the forward pass, the softmax cross-entropy's closed
forms, and Adam's closed form under a constant gradient."""
import numpy as np
import pytest
import torch
from scipy.special import logsumexp

from oracle import mlp


def test_bf16_round_ties_and_torch():
    one = 1.0
    cases = {
        one: one,
        one + 2.0 ** -8: one,                            # tie between 1 and 1 + 2^-7 -> even (1)
        one + 3 * 2.0 ** -8: one + 2.0 ** -6,            # tie between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
        one + 2.0 ** -8 + 2.0 ** -20: one + 2.0 ** -7,   # just above the tie
        -(one + 2.0 ** -8 + 2.0 ** -20): -(one + 2.0 ** -7),
        0.0: 0.0,
        3.0: 3.0,
    }
    for x, want in cases.items():
        assert mlp.bf16_round(np.float32(x)) == want, x
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-20, 20, 20000))).astype(np.float32)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16_round(x), ref)


def test_forward_hand_set_weights():
    # unit u < 32 copies input u; unit u of layer 2 copies unit u of layer 1;
    # the output sums units 0..3 with weights 1, 2, 0.5, -1 plus 0.25:
    # s = relu(x0) + 2 relu(x1) + 0.5 relu(x2) - relu(x3) + 0.25.
    w = {name: np.zeros(shape) for name, shape in mlp.SHAPES}
    for u in range(mlp.F):
        w["W1"][u, u] = 1.0
    w["W2"][np.arange(mlp.H), np.arange(mlp.H)] = 1.0
    w["w3"][:4] = [1.0, 2.0, 0.5, -1.0]
    w["b3"] = np.array(0.25)
    P = mlp.pack(w)
    X = np.array([[1.5, -2.0, 4.0, 0.75] + [0.0] * 28, [-1.0, 3.0, -0.5, -8.0] + [5.0] * 28])
    s, _ = mlp.forward(P, X)
    assert np.array_equal(s, [1.5 + 2.0 - 0.75 + 0.25, 6.0 + 0.25])


def _smooth_case(seed, rows=6):
    """Random network and inputs with every pre-activation well away from the
    relu kink, so that central differences are valid."""
    rng = np.random.default_rng(seed)
    for _ in range(100):
        P = rng.standard_normal(mlp.NPARAM) * 0.2
        X = rng.standard_normal((rows, mlp.F))
        _, c = mlp.forward(P, X, rounded=False)
        if min(np.abs(c["z1"]).min(), np.abs(c["z2"]).min()) > 1e-3:
            return rng, P, X
    pytest.skip("no smooth case found")


def test_backward_matches_finite_differences():
    rng, P, X = _smooth_case(3)
    ds = rng.standard_normal(X.shape[0])

    def f(Q):
        return float(mlp.forward(Q, X, rounded=False)[0] @ ds)

    g = mlp.backward(mlp.forward(P, X, rounded=False)[1], ds)
    h = 1e-6
    # every parameter group, including b3, by sampled coordinates
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in mlp.SHAPES])
    idx = [int(offs[k] + rng.integers(0, max(1, offs[k + 1] - offs[k]))) for k in range(len(mlp.SHAPES))
           for _ in range(8)]
    for i in idx:
        e = np.zeros(mlp.NPARAM)
        e[i] = h
        fd = (f(P + e) - f(P - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * (1 + abs(g[i])), (i, fd, g[i])
    # and one random direction through all parameters at once
    v = rng.standard_normal(mlp.NPARAM)
    fd = (f(P + h * v) - f(P - h * v)) / (2 * h)
    assert abs(fd - g @ v) <= 1e-6 * (1 + abs(g @ v))


def test_backward_uses_rounded_weights():
    # with rounding on, the gradient equals the unrounded gradient at the rounded point
    rng, P, X = _smooth_case(4)
    ds = rng.standard_normal(X.shape[0])
    g1 = mlp.backward(mlp.forward(P, X)[1], ds)
    g2 = mlp.backward(mlp.forward(mlp.bf16_round(P), X, rounded=False)[1], ds)
    assert np.array_equal(g1, g2)


def test_listwise_loss_closed_forms():
    n = 7
    p = np.zeros(n)
    p[2] = 1.0
    loss, d = mlp.listwise_loss(np.full(n, 0.3), p)
    assert abs(loss - np.log(n)) < 1e-15
    assert np.allclose(d, 1.0 / n - p, atol=1e-16)
    rng = np.random.default_rng(5)
    s = rng.standard_normal(40) * 5
    q = rng.random(40)
    q /= q.sum()
    loss, d = mlp.listwise_loss(s, q)
    assert abs(loss - (logsumexp(s) - q @ s)) < 1e-12
    assert abs(d.sum()) < 1e-14
    loss2, _ = mlp.listwise_loss(s + 123.0, q)              # shift invariance
    assert abs(loss2 - loss) < 1e-11
    h = 1e-6
    for k in (0, 17, 39):
        e = np.zeros(40)
        e[k] = h
        fd = (mlp.listwise_loss(s + e, q)[0] - mlp.listwise_loss(s - e, q)[0]) / (2 * h)
        assert abs(fd - d[k]) < 1e-8
    assert mlp.listwise_loss([], [])[0] == 0.0


def test_adam_constant_gradient_closed_form():
    # with a constant gradient the bias-corrected moments are g and g^2, so
    # every step moves each parameter by lr g / (|g| + eps).
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    P0 = np.array([1.0, 2.0, 3.0, 4.0])
    opt = mlp.Adam(4, lr=0.01)
    P = P0.copy()
    for _ in range(5):
        P = opt.step(P, g)
    want = P0 - 5 * 0.01 * g / (np.abs(g) + 1e-8)
    assert np.allclose(P, want, rtol=0, atol=1e-12)
    assert P[3] == 4.0


def test_features_closed_forms():
    """Feature oracle on hand-worked states: a Fock state gives its own
    occupations and no coherence; psi = alpha|n0+1, n1-1> + beta|n0, n1> gives
    <a_0^dag a_1> = conj(alpha) beta sqrt((n0 + 1) n1) (and its conjugate for
    the reversed pair)."""
    from oracle import features as ofeat
    from oracle.core import Sector
    from paper_2606_05297_gb300 import workloads as W
    s = Sector(W.bose_hubbard(3, 5, periodic=False))
    f = ofeat.features(s, s.basis_state([2, 0, 3]), [(0, 2), (2, 1)])
    assert np.array_equal(f, [2, 0, 3, 4, 0, 9, 0, 0, 0, 0])
    n0, n1 = 1, 3
    alpha, beta = 0.6 * np.exp(0.7j), 0.8 * np.exp(-1.9j)
    psi = alpha * s.basis_state([n0 + 1, n1 - 1, 5 - n0 - n1]) + beta * s.basis_state([n0, n1, 5 - n0 - n1])
    f = ofeat.features(s, psi, [(0, 1), (1, 0), (0, 2)])
    z = np.conj(alpha) * beta * np.sqrt((n0 + 1) * n1)
    assert np.allclose(f[6:], [z.real, z.imag, z.real, -z.imag, 0, 0], atol=1e-15)
    occ0 = abs(alpha) ** 2 * (n0 + 1) + abs(beta) ** 2 * n0
    assert abs(f[0] - occ0) < 1e-15 and abs(f[3] - (abs(alpha) ** 2 * (n0 + 1) ** 2 + abs(beta) ** 2 * n0 ** 2)) < 1e-14
