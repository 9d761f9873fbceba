"""Dense full-Fock-space reference (test infrastructure, oracle).

Builds operators as Kronecker products of truncated D x D ladder matrices in
the full space of dimension D^L (mode 0 is the leftmost, most significant
factor), written out again from the paper's equations without the ladder
strings of operators.py, then restricts them to the symmetry sector by
brute-force filtering of the full basis.  Also exact diagonalisation and
dense matrix exponentials (scipy.linalg.expm).  Tiny systems only.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.linalg


def ladder(D: int) -> np.ndarray:
    """Truncated annihilation operator: a|n> = sqrt(n)|n-1> on span{|0>..|D-1>} (Sec. II.A)."""
    a = np.zeros((D, D))
    for n in range(1, D):
        a[n - 1, n] = np.sqrt(n)
    return a


def embed(m: np.ndarray, r: int, L: int) -> np.ndarray:
    D = m.shape[0]
    out = np.array([[1.0]])
    for q in range(L):
        out = np.kron(out, m if q == r else np.eye(D))
    return out


class FullSpace:
    def __init__(self, model):
        self.model = model
        self.L = model.L
        self.D = model.N + 1 if model.kind == "bh" else model.d
        a = ladder(self.D)
        self.a = [embed(a, r, self.L).astype(np.complex128) for r in range(self.L)]
        self.ad = [m.conj().T for m in self.a]
        self.n = [self.ad[r] @ self.a[r] for r in range(self.L)]
        occ = np.array(list(itertools.product(range(self.D), repeat=self.L)), dtype=np.int64)
        tot = occ.sum(axis=1)
        if model.kind == "bh":
            keep = tot == model.N
        else:
            keep = (tot % 2) == model.parity
        # full-space index of tuple n is sum_r n_r D^(L-1-r): itertools.product order
        self.sector_idx = np.nonzero(keep)[0]
        self.sector_occ = occ[keep]

    def hamiltonian(self) -> np.ndarray:
        m = self.model
        L = self.L
        H = np.zeros_like(self.a[0])
        bonds = [(r, (r + 1) % L) for r in range(L if m.periodic else L - 1)]
        for b, (r, s) in enumerate(bonds):
            hop = self.ad[r] @ self.a[s]
            H = H + m.hop[b] * (hop + hop.conj().T)
            if m.pair:
                pr = self.a[r] @ self.a[s]
                H = H + m.pair[b] * (pr + pr.conj().T)
        I = np.eye(H.shape[0])
        for r in range(L):
            nr = self.n[r]
            if m.nn1:
                H = H + m.nn1[r] * (nr @ (nr - I))
            if m.n2:
                H = H + m.n2[r] * (nr @ nr)
            if m.n1:
                H = H + m.n1[r] * nr
        return H

    def generator(self, op) -> np.ndarray:
        """Anti-Hermitian generator, written from Sec. II.B: BS, S2, S with
        e^{i phi} = i^phase; pair hopping; K, N(N-1), R, CK times i."""
        e = (1, 1j, -1, -1j)[op.phase % 4]
        i, j = op.i, op.j
        if op.type == "hop":
            X = self.a[i] @ self.ad[j]
            return e * X - (e * X).conj().T
        if op.type == "sq2":
            X = self.a[i] @ self.a[j]
            return e * X - (e * X).conj().T
        if op.type == "sq1":
            X = self.a[i] @ self.a[i]
            return 0.5 * (np.conj(e) * X - (np.conj(e) * X).conj().T)
        if op.type == "pairhop":
            X = self.a[i] @ self.a[i] @ self.ad[j] @ self.ad[j]
            return e * X - (e * X).conj().T
        I = np.eye(self.a[0].shape[0])
        if op.type == "kerr":
            return 1j * self.n[i] @ self.n[i]
        if op.type == "nn1":
            return 1j * self.n[i] @ (self.n[i] - I)
        if op.type == "rot":
            return 1j * self.n[i]
        if op.type == "xkerr":
            return 1j * self.n[i] @ self.n[j]
        raise ValueError(op.type)

    def restrict(self, M: np.ndarray) -> np.ndarray:
        ix = self.sector_idx
        return M[np.ix_(ix, ix)]

    def embed_state(self, v_sector: np.ndarray) -> np.ndarray:
        v = np.zeros(self.a[0].shape[0], dtype=np.complex128)
        v[self.sector_idx] = v_sector
        return v


def ground_energy(H: np.ndarray) -> float:
    return float(np.linalg.eigvalsh(H)[0])


def expm_apply(A: np.ndarray, theta: float, v: np.ndarray) -> np.ndarray:
    return scipy.linalg.expm(theta * A) @ v
