"""CV-ADAPT-VQE loop for the oracle (test infrastructure).

Follows Sec. IV.B: evaluate the Eq. (grad) gradient of every pool operator on
the current state, append the operator with the largest |g| as
exp(theta A) with theta = 0, re-minimise E over all parameters with BFGS.

Readings where the paper is silent:
  * warm start (Sec. IV.B, App. C/D): one HVA layer with angles U[-0.05, 0.05]
    is optimised first (L-inf gradient tolerance 1e-9, 1000 iterations) and is
    re-optimised together with every ADAPT parameter afterwards;
  * selection ties: the lowest pool index among |g_k| >= max|g| (1 - 1e-9);
  * stopping: max|g| < grad_tol, or max_ops ADAPT operators, or |E - E0| <
    energy_tol when an exact E0 is supplied;
  * per-iteration BFGS: at most 1000 iterations, L-inf gradient tolerance
    min(1e-6, |g_init| 1e-5) (Sec. IV.A).
"""
from __future__ import annotations

import numpy as np

from . import bfgs

TIE_REL = 1e-9


def select(g):
    """Index of the selected operator: lowest index within the tie window."""
    a = np.abs(np.asarray(g))
    m = a.max()
    return int(np.nonzero(a >= m * (1.0 - TIE_REL))[0][0]), float(m)


def run(sector, pool, psi_init, warm_ops=(), warm_theta=(), max_ops=160, grad_tol=1e-6, E0=None,
        energy_tol=None, bfgs_max_iter=1000, warm_gtol=1e-9, hessian_recycling=False, fix_warm=False):
    """hessian_recycling (App. D): each BFGS starts from the previous one's
    final inverse Hessian, extended by an identity row and column for the new
    parameter.  fix_warm (App. D): the warm-up layer keeps the parameters of
    its initial optimisation; ADAPT then grows from the warm-up state."""
    ops = list(warm_ops)
    theta = np.array(warm_theta, dtype=np.float64)
    trace = []
    H = None

    def fg(th):
        E, g = sector.energy_and_grad(ops, th, psi_init)
        return E, g

    if len(ops):
        res = bfgs.minimize(fg, theta, gtol=warm_gtol, max_iter=bfgs_max_iter)
        theta = res["x"]
        H = res["H"]
        trace.append(dict(kind="warm", E=res["f"], nfev=res["nfev"], nit=res["nit"]))
        if fix_warm:
            psi_init = sector.apply_ansatz(ops, theta, psi_init)
            ops, theta, H = [], np.zeros(0), None
    n_adapt = 0
    stop = "max_ops"
    while n_adapt < max_ops:
        psi = sector.apply_ansatz(ops, theta, psi_init)
        E, _ = sector.energy(psi)
        if E0 is not None and energy_tol is not None and abs(E - E0) < energy_tol:
            stop = "energy_tol"
            break
        g = sector.screen(pool, psi)
        k, gmax = select(g)
        if gmax < grad_tol:
            stop = "grad_tol"
            break
        theta_sel = theta.tolist()  # the parameters of the state this choice was made on
        ops.append(pool[k])
        theta = np.append(theta, 0.0)
        n_adapt += 1
        tol = min(1e-6, gmax * 1e-5)
        H0 = None
        if hessian_recycling and H is not None:
            H0 = np.eye(theta.size)
            H0[:-1, :-1] = H
        res = bfgs.minimize(fg, theta, gtol=tol, max_iter=bfgs_max_iter, H0=H0)
        theta = res["x"]
        H = res["H"]
        trace.append(dict(kind="adapt", op=k, gmax=gmax, E=res["f"], nfev=res["nfev"], nit=res["nit"],
                          theta_sel=theta_sel))
    E_final = fg(theta)[0] if len(ops) else sector.energy(psi_init)[0]
    return dict(ops=ops, theta=theta, trace=trace, E=E_final, stop=stop, n_adapt=n_adapt)
