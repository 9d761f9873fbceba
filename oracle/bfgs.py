"""BFGS for the oracle (test infrastructure).

The paper minimises E(theta) with BFGS (Sec. IV.A; SciPy).  It states only
the stopping rules: at most 1000 iterations, L-infinity gradient norm below
1e-9 (HVA) or min(1e-6, |g_init| 1e-5) (ADAPT).  The rest follows the
textbook method (Nocedal & Wright, Numerical Optimization, Alg. 6.1 with the
inverse-Hessian update (6.17), initial inverse Hessian = identity, and the
strong-Wolfe line search of Alg. 3.5 / 3.6 with c1 = 1e-4, c2 = 0.9 and a
safeguarded cubic interpolation step in zoom).
"""
from __future__ import annotations

import numpy as np

C1, C2 = 1e-4, 0.9


def _cubic_min(a, fa, ga, b, fb, gb):
    """Minimiser of the cubic interpolating f and f' at a and b (N&W eq. 3.59);
    None for a bracket of zero width, which has no interpolating cubic."""
    if a == b:
        return None
    d1 = ga + gb - 3.0 * (fa - fb) / (a - b)
    disc = d1 * d1 - ga * gb
    if disc < 0:
        return None
    d2 = np.sign(b - a) * np.sqrt(disc)
    den = gb - ga + 2.0 * d2
    if den == 0:
        return None
    return b - (b - a) * (gb + d2 - d1) / den


def line_search(fg, x, f0, g0, p, alpha_max=50.0, max_iter=30):
    """Strong-Wolfe line search.  fg(x) -> (f, g).  Returns (alpha, f, g, nevals)
    or (None, f0, g0, nevals) if no acceptable step was found."""
    d0 = float(g0 @ p)
    nev = 0
    cache = {}

    def phi(a):
        nonlocal nev
        if a not in cache:
            f, g = fg(x + a * p)
            nev += 1
            cache[a] = (f, g, float(g @ p))
        return cache[a]

    def zoom(lo, hi):
        for _ in range(max_iter):
            flo, _, dlo = phi(lo)
            fhi, _, dhi = phi(hi)
            a = _cubic_min(lo, flo, dlo, hi, fhi, dhi)
            width = abs(hi - lo)
            left, right = min(lo, hi), max(lo, hi)
            if a is None or not (left + 0.1 * width <= a <= right - 0.1 * width):
                a = 0.5 * (lo + hi)
            fa, ga, da = phi(a)
            if fa > f0 + C1 * a * d0 or fa >= flo:
                hi = a
            else:
                if abs(da) <= -C2 * d0:
                    return a
                if da * (hi - lo) >= 0:
                    hi = lo
                lo = a
            if abs(hi - lo) < 1e-16 * max(1.0, abs(lo)):
                break
        flo, _, _ = phi(lo)
        return lo if lo > 0 and flo < f0 else None

    cache[0.0] = (f0, g0, d0)
    a_prev, a = 0.0, 1.0
    f_prev = f0
    result = None
    for i in range(max_iter):
        fa, ga, da = phi(a)
        if fa > f0 + C1 * a * d0 or (i > 0 and fa >= f_prev):
            result = zoom(a_prev, a)
            break
        if abs(da) <= -C2 * d0:
            result = a
            break
        if da >= 0:
            result = zoom(a, a_prev)
            break
        a_prev, f_prev = a, fa
        a = min(2.0 * a, alpha_max)
    if result is None:
        return None, f0, g0, nev
    f, g, _ = phi(result)
    return result, f, g, nev


def minimize(fg, x0, gtol=1e-9, max_iter=1000, H0=None):
    """Returns dict(x, f, g, nit, nfev, H, reason)."""
    x = np.array(x0, dtype=np.float64)
    n = x.size
    f, g = fg(x)
    nfev = 1
    H = np.eye(n) if H0 is None else np.array(H0, dtype=np.float64)
    reason = "max_iter"
    it = 0
    for it in range(max_iter):
        if np.max(np.abs(g)) < gtol:
            reason = "gtol"
            break
        p = -H @ g
        if float(g @ p) >= 0:  # not a descent direction: restart from steepest descent
            H = np.eye(n)
            p = -g
        alpha, f_new, g_new, nev = line_search(fg, x, f, g, p)
        nfev += nev
        if alpha is None:
            reason = "line_search"
            break
        s = alpha * p
        y = g_new - g
        x = x + s
        f, g = f_new, g_new
        sy = float(s @ y)
        if sy > 0:
            rho = 1.0 / sy
            I = np.eye(n)
            H = (I - rho * np.outer(s, y)) @ H @ (I - rho * np.outer(y, s)) + rho * np.outer(s, s)
    else:
        it = max_iter
    if np.max(np.abs(g)) < gtol:
        reason = "gtol"
    return dict(x=x, f=f, g=g, nit=it, nfev=nfev, H=H, reason=reason)
