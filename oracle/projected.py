"""Gates as projections of the untruncated gate, with the state renormalised
after every gate (test infrastructure, oracle).

Sec. V.A builds each gate's matrix elements for the infinite Fock space (by
recurrences) and keeps those between states inside the cutoff; since such a
truncated gate is not unitary, the state is normalised after each gate.  Here
the infinite-space elements are obtained as the matrix exponential of the
generator on the gate modes' local Fock space at a larger inner cutoff dc,
restricted to occupations below the sector's cutoff d:

    U_k = P exp(theta_k A_k^(dc)) P,   psi_k = U_k psi_{k-1} / ||U_k psi_{k-1}||.

For number-conserving two-mode generators every block is finite, and dc >=
2d - 1 gives the exact elements; for squeezers the elements converge as dc
grows.  The energy is E = <psi_n|H|psi_n>; its gradient follows the chain
rule through the normalisations, with every intermediate state stored:

    lambda_n = H psi_n;  for k = n..1:
      mu_k = (lambda_k - Re<psi_k|lambda_k> psi_k) / N_k,
      g_k = 2 Re <mu_k| D_k psi_{k-1}>,  D_k = P A_k exp(theta_k A_k) P,
      lambda_{k-1} = U_k^dag mu_k.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np
from scipy.linalg import expm

from .operators import generator_strings


def _ladder(dc: int) -> np.ndarray:
    a = np.zeros((dc, dc))
    for n in range(1, dc):
        a[n - 1, n] = np.sqrt(n)  # a|n> = sqrt(n)|n-1>
    return a


def gate_modes(op) -> Tuple[int, ...]:
    return (op.i,) if (op.j is None or op.j < 0 or op.type in ("kerr", "nn1", "rot", "sq1")) else (op.i, op.j)


def local_generator(op, dc: int) -> np.ndarray:
    """Generator A of pool element op on the Fock space of its modes cut at dc
    (dc or dc^2 square; mode order as in gate_modes, first mode most significant)."""
    modes = gate_modes(op)
    a = _ladder(dc)
    ops = {0: a, 1: a.T}
    eye = np.eye(dc)
    out = np.zeros((dc ** len(modes),) * 2, dtype=complex)
    for c, factors in generator_strings(op):
        term = np.eye(dc ** len(modes), dtype=complex)
        for mode, dag in factors:  # the product c o_0 o_1 ...; o_k on its mode
            f = ops[dag]
            full = f if len(modes) == 1 else (np.kron(f, eye) if mode == modes[0] else np.kron(eye, f))
            term = term @ full
        out += c * term
    return out


class Projected:
    """Projected gates of one pool on one sector (dense local matrices per gate)."""

    def __init__(self, sector, dc: int):
        self.s = sector
        self.dc = dc
        self.tup = sector.tuples()
        self._groups: Dict[Tuple[int, ...], List[Tuple[np.ndarray, np.ndarray]]] = {}

    def _groups_of(self, modes):
        """Sector indices grouped by the occupations of every other mode, with
        each member's local index (base dc) on the gate modes."""
        if modes not in self._groups:
            others = [r for r in range(self.s.L) if r not in modes]
            g: Dict[tuple, list] = {}
            for x, t in enumerate(self.tup):
                loc = 0
                for r in modes:
                    loc = loc * self.dc + int(t[r])
                g.setdefault(tuple(int(t[r]) for r in others), []).append((x, loc))
            self._groups[modes] = [(np.array([p[0] for p in v]), np.array([p[1] for p in v])) for v in g.values()]
        return self._groups[modes]

    def apply_local(self, op, M: np.ndarray, v: np.ndarray) -> np.ndarray:
        out = np.zeros_like(v)
        for xs, loc in self._groups_of(gate_modes(op)):
            out[xs] = M[np.ix_(loc, loc)] @ v[xs]
        return out

    def matrices(self, op, theta: float):
        A = local_generator(op, self.dc)
        U = expm(theta * A)
        return U, A @ U

    def forward(self, ops: Sequence, theta: Sequence[float], psi0: np.ndarray):
        states, norms = [np.asarray(psi0, dtype=complex)], []
        for op, th in zip(ops, theta):
            U, _ = self.matrices(op, th)
            phi = self.apply_local(op, U, states[-1])
            N = float(np.linalg.norm(phi))
            norms.append(N)
            states.append(phi / N)
        return states, norms

    def apply_ansatz(self, ops, theta, psi0):
        return self.forward(ops, theta, psi0)[0][-1]

    def energy_and_grad(self, ops: Sequence, theta: Sequence[float], psi0: np.ndarray):
        states, norms = self.forward(ops, theta, psi0)
        psi = states[-1]
        lam = self.s.apply_H(psi)
        E = float(np.vdot(psi, lam).real)
        g = np.zeros(len(ops))
        for k in range(len(ops) - 1, -1, -1):
            U, D = self.matrices(ops[k], theta[k])
            pk = states[k + 1]
            mu = (lam - np.vdot(pk, lam).real * pk) / norms[k]
            g[k] = 2.0 * np.vdot(mu, self.apply_local(ops[k], D, states[k])).real
            lam = self.apply_local(ops[k], U.conj().T, mu)
        return E, g
