"""State features of the learned proposal, by their plain definitions (test
infrastructure, oracle): <n_r> and <n_r^2> as sums of |psi_x|^2 n_r(x)^k over
the sector basis, <a_i^dag a_j> as <psi|(a_i^dag a_j) psi> with the ladder
string applied by the oracle (truncated ladder rules of Sec. II.A)."""
from __future__ import annotations

import numpy as np

from .core import Operator


def features(sector, psi, pairs=()):
    occ = sector.tuples().astype(np.float64)
    p2 = np.abs(psi) ** 2
    out = [p2 @ occ[:, r] for r in range(sector.L)]
    out += [p2 @ occ[:, r] ** 2 for r in range(sector.L)]
    for (i, j) in pairs:
        op = Operator([(1.0, [(i, 1), (j, 0)])])  # a_i^dag a_j
        z = np.vdot(psi, sector.apply(op, psi))
        out += [z.real, z.imag]
    return np.array(out)
