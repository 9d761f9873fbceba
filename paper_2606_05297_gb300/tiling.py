"""Operator tiling (App. B): learn which generators ADAPT needs on a small,
classically cheap lattice and keep only their translates on the large one.

1. Run ADAPT on the small lattice with the full pool.
2. At every iteration collect the generator it selects and every generator
   whose |gradient| is degenerate with the selected one (within a relative
   `rel`), which stands for repeating the small runs until the degenerate
   choices have all been seen.
3. A generator's pattern is (type, phase, j - i) for a two-mode generator and
   (type, phase, None) for a single-mode one; the tiled pool of the large
   lattice is the large full pool restricted to the collected patterns, in
   the full pool's order (so ties resolve as they would in the full pool).

On a translationally invariant chain the tiled pool grows linearly with the
lattice like the full one, with a smaller constant (fewer gradients to
screen per iteration).
"""
from __future__ import annotations

import time
from typing import Iterable, List, Optional, Sequence, Set, Tuple

import numpy as np

from .adapt import Adapt, select
from .workloads import Model, Op

Pattern = Tuple[str, int, Optional[int]]


def pattern_of(op: Op) -> Pattern:
    return (op.type, int(op.phase), (op.j - op.i) if op.j is not None and op.j >= 0 else None)


def degenerate_patterns(pool: Sequence[Op], g, rel: float = 1e-6) -> Set[Pattern]:
    """Patterns of every pool element whose |g| lies within `rel` of max |g|."""
    a = np.abs(np.asarray(g))
    m = float(a.max(initial=0.0))
    if m <= 0.0:
        return set()
    return {pattern_of(pool[k]) for k in np.nonzero(a >= m * (1.0 - rel))[0]}


def tiled_pool(full_pool: Sequence[Op], patterns: Iterable[Pattern]) -> List[Op]:
    pats = set(patterns)
    return [op for op in full_pool if pattern_of(op) in pats]


def learn_patterns(model: Model, pool: Sequence[Op], init_occ: Sequence[int], warm_ops: Sequence[Op] = (),
                   warm_theta: Sequence[float] = (), max_ops: int = 20, grad_tol: float = 1e-6,
                   rel: float = 1e-6) -> Set[Pattern]:
    """Steps 1-2 on the GPU driver: the patterns of the selected and degenerate generators."""
    A = Adapt(model, pool, init_occ, warm_ops, warm_theta, n_max=max_ops + len(warm_ops) + 1)
    A.optimise_warm_start()
    pats: Set[Pattern] = set()
    for _ in range(max_ops):
        g = A.screen()
        k, gmax = select(g)
        if gmax < grad_tol:
            break
        pats |= degenerate_patterns(pool, g, rel)
        A._grow(k, gmax, 1000, time.perf_counter())
    return pats
