"""Scorer kernels (forward, backward, listwise softmax cross-entropy, Adam)
against the float64 oracle with bf16-rounded weights.

Tolerances follow from fp32 accumulation (unit roundoff u = 2^-24): a sum of
n terms is off by at most about n u times the sum of the terms' magnitudes, so
every comparison bounds the error by (terms along the longest chain) x u x the
same network evaluated on absolute values.  Rows where a pre-activation lies
within that bound of the relu kink would let the two sides take different
masks; those rows get a zero upstream gradient on both sides, so the masks
they would decide do not enter any compared value."""
import numpy as np
import pytest

from paper_2606_05297_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def _abs_net(P, X):
    from oracle import mlp
    Pa = np.abs(mlp.bf16_round(P))
    s, c = mlp.forward(Pa, np.abs(X), rounded=False)
    return s, c, Pa


def _scorer(max_rows, P):
    from paper_2606_05297_gb300 import build, cvq
    build.build()
    sc = cvq.Scorer(max_rows)
    sc.set(P)
    return sc


@pytest.mark.parametrize("rows", [1, 7, 210, 1003])
def test_forward_matches_oracle(rows):
    import torch
    from oracle import mlp
    P = W.scorer_params(10 + rows)
    X = W.scorer_inputs(rows, 20 + rows)
    sc = _scorer(2048, P)
    got = sc.forward(torch.from_numpy(X).cuda()).cpu().numpy().astype(np.float64)
    ref, _ = mlp.forward(P.astype(np.float64), X)
    sabs, _, _ = _abs_net(P, X)
    tol = (32 + 256 + 256 + 8) * U32 * sabs
    assert np.all(np.abs(got - ref) <= tol), np.max(np.abs(got - ref) / tol)


def test_forward_zero_rows_and_limits():
    import torch
    from paper_2606_05297_gb300 import cvq
    sc = _scorer(16, W.scorer_params(1))
    out = sc.forward(torch.empty((0, 32), dtype=torch.float32, device="cuda"))
    assert out.numel() == 0
    with pytest.raises(cvq.CvqError):
        sc.forward(torch.zeros((17, 32), dtype=torch.float32, device="cuda"))
    X = torch.zeros((5, 32), dtype=torch.float32, device="cuda")
    sc.forward(X)
    with pytest.raises(cvq.CvqError):  # backward must see the rows of the last forward
        sc.backward(X[:4], torch.zeros(4, dtype=torch.float32, device="cuda"))
    P = W.scorer_params(2)
    sc.set(P)
    assert np.array_equal(sc.get(), P)


def _grad_case(rows, seed):
    """Parameters, inputs and an upstream gradient with kink-ambiguous rows
    zeroed.  |dz1| <= 33 u (|W1||x| + |b1|) and |dz2| <= 257 u (|W2||h1| +
    |b2|) + |W2||dz1| bound the fp32 pre-activation errors."""
    from oracle import mlp
    P = W.scorer_params(seed)
    X = W.scorer_inputs(rows, seed + 1)
    ds = np.random.default_rng(seed + 2).standard_normal(rows).astype(np.float32)
    _, c = mlp.forward(P.astype(np.float64), X)
    w = mlp.unpack(np.abs(mlp.bf16_round(P)))
    e1 = 33 * U32 * (np.abs(X) @ w["W1"].T + w["b1"])
    e2 = 257 * U32 * (c["h1"] @ w["W2"].T + w["b2"]) + e1 @ w["W2"].T
    amb = (np.abs(c["z1"]) <= 1.5 * e1).any(axis=1) | (np.abs(c["z2"]) <= 1.5 * e2).any(axis=1)
    ds[amb] = 0.0
    return P, X, ds, int(amb.sum())


def _grad_tol(P, X, ds):
    from oracle import mlp
    _, ca, _ = _abs_net(P, X)
    gabs = mlp.backward(ca, np.abs(ds.astype(np.float64)))
    return (X.shape[0] + 600) * U32 * gabs + 1e-30


@pytest.mark.parametrize("rows", [1, 210, 517])
def test_backward_matches_oracle(rows):
    import torch
    from oracle import mlp
    P, X, ds, namb = _grad_case(rows, 100 + rows)
    assert namb <= rows // 4
    sc = _scorer(1024, P)
    Xd = torch.from_numpy(X).cuda()
    sc.forward(Xd)
    sc.backward(Xd, torch.from_numpy(ds).cuda())
    got = sc.get(1).astype(np.float64)
    ref = mlp.backward(mlp.forward(P.astype(np.float64), X)[1], ds)
    tol = _grad_tol(P, X, ds)
    bad = np.abs(got - ref) > tol
    assert not bad.any(), (np.flatnonzero(bad)[:10], np.max(np.abs(got - ref) / tol))


def test_listwise_loss_matches_oracle():
    import torch
    from oracle import mlp
    from paper_2606_05297_gb300 import cvq
    build_lens = [0, 1, 5, 210, 300, 17, 256, 257]
    rng = np.random.default_rng(7)
    off = np.concatenate([[0], np.cumsum(build_lens)]).astype(np.int32)
    n = int(off[-1])
    s = (rng.standard_normal(n) * 4).astype(np.float32)
    t = np.zeros(n, dtype=np.float32)
    for a, b in zip(off[:-1], off[1:]):
        if b > a:
            q = rng.random(b - a) ** 4
            t[a:b] = q / q.sum()
    _scorer(1, W.scorer_params(0))  # builds and loads the library
    loss, ds = cvq.listwise_loss(torch.from_numpy(s).cuda(), torch.from_numpy(t).cuda(),
                                 torch.from_numpy(off).cuda())
    loss, ds = loss.cpu().numpy(), ds.cpu().numpy()
    for k, (a, b) in enumerate(zip(off[:-1], off[1:])):
        rl, rd = mlp.listwise_loss(s[a:b], t[a:b])
        # fp32 softmax: log-sum-exp and products carry a few ulps of the largest |s|
        assert abs(loss[k] - rl) <= 64 * U32 * (1 + np.abs(s[a:b]).max(initial=0) + abs(rl)), (k, loss[k], rl)
        assert np.all(np.abs(ds[a:b] - rd) <= 64 * U32 * (1 + np.abs(s[a:b]).max(initial=0))), k


def test_adam_step_matches_oracle():
    import torch
    from oracle import mlp
    rows, lr = 210, 1e-3
    P, X, ds, _ = _grad_case(rows, 300)
    sc = _scorer(rows, P)
    Xd = torch.from_numpy(X).cuda()
    sc.forward(Xd)
    sc.backward(Xd, torch.from_numpy(ds).cuda())
    sc.adam_step(lr)
    got = sc.get().astype(np.float64)
    P64 = P.astype(np.float64)
    g = mlp.backward(mlp.forward(P64, X)[1], ds)
    ref = mlp.Adam(mlp.NPARAM, lr=lr).step(P64, g)
    # where |g| is far above its error bound the first step is lr g / (|g| + eps) on both sides; elsewhere
    # the step is still at most lr
    strong = (np.abs(g) > 2 * _grad_tol(P, X, ds)) & (np.abs(g) > 1e-4)
    ulp = np.spacing(np.abs(P)).astype(np.float64)
    assert strong.mean() > 0.3
    assert np.all(np.abs(got - ref)[strong] <= 4 * ulp[strong] + 1e-3 * lr)
    assert np.all(np.abs(got - P64) <= lr * (1 + 1e-6) + 2 * ulp)


def test_adam_moments_carry_over():
    """Step 1 with lr = 0 leaves the weights but fills the moments; step 2 from
    the same weights then depends on both gradients (bias-corrected with t = 2)."""
    import torch
    from oracle import mlp
    rows, lr = 210, 1e-3
    P, X, ds1, _ = _grad_case(rows, 310)
    ds2 = np.random.default_rng(311).standard_normal(rows).astype(np.float32) * (ds1 != 0)
    sc = _scorer(rows, P)
    Xd = torch.from_numpy(X).cuda()
    P64 = P.astype(np.float64)
    opt = mlp.Adam(mlp.NPARAM, lr=0.0)
    grads = []
    for k, (ds, step_lr) in enumerate([(ds1, 0.0), (ds2, lr)]):
        sc.forward(Xd)
        sc.backward(Xd, torch.from_numpy(ds).cuda())
        sc.adam_step(step_lr)
        grads.append(mlp.backward(mlp.forward(P64, X)[1], ds))
        opt.lr = step_lr
        ref = opt.step(P64, grads[-1])
        if k == 0:
            assert np.array_equal(sc.get(), P) and np.array_equal(ref, P64)
    got = sc.get().astype(np.float64)
    # a relative gradient error r moves the step by at most about 4 r lr (both moments enter)
    r = np.maximum(_grad_tol(P, X, ds1) / np.maximum(np.abs(grads[0]), 1e-300),
                   _grad_tol(P, X, ds2) / np.maximum(np.abs(grads[1]), 1e-300))
    strong = r < 1e-2
    ulp = np.spacing(np.abs(P)).astype(np.float64)
    assert strong.mean() > 0.2
    assert np.all(np.abs(got - ref)[strong] <= 4 * ulp[strong] + 5 * r[strong] * lr)
    assert np.all(np.abs(got - P64) <= 2 * lr + 2 * ulp)


def test_training_reduces_listwise_loss():
    """Adam on a fixed ranking task: the targets are a softmax of one input
    column, which the network can represent; 60 steps must cut the loss."""
    import torch
    from paper_2606_05297_gb300 import cvq
    nl, per = 16, 64
    X = W.scorer_inputs(nl * per, 400)
    t = np.zeros(nl * per, dtype=np.float32)
    for l in range(nl):
        z = 2.0 * X[l * per:(l + 1) * per, 20]
        e = np.exp(z - z.max())
        t[l * per:(l + 1) * per] = e / e.sum()
    off = torch.arange(0, nl * per + 1, per, dtype=torch.int32, device="cuda")
    sc = _scorer(nl * per, W.scorer_params(401))
    Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
    losses = []
    for step in range(60):
        s = sc.forward(Xd)
        loss, ds = cvq.listwise_loss(s, td, off)
        losses.append(float(loss.mean()))
        sc.backward(Xd, ds)
        sc.adam_step(1e-3)
    assert np.isfinite(losses).all()
    assert losses[-1] < 0.5 * losses[0] or losses[-1] - np.log(per) < 0.5 * (losses[0] - np.log(per))
