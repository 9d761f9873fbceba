"""Hamiltonians and pool generators as sums of ladder-operator strings.

Test infrastructure (oracle).  A string is (c, [(mode, dag), ...]) meaning
c * o_0 o_1 ... (rightmost factor acts first), dag = 1 for a^dag.  The C oracle
applies strings with the ladder rules of Sec. II.A.

Sources (arXiv 2606.05297):
  Eq. (BoseHubbard)             -J sum(a_r^dag a_{r+1} + h.c.) - U/2 sum N_r(N_r - 1) - mu sum N_r
  Eq. (BosonicKitaevChain)      -J sum(a_r^dag a_{r+1} + h.c.) - Delta sum(a_r a_{r+1} + h.c.) - mu sum N_r
  Eq. (BosonicKitaevChain_Kerr) H_BKC - U/2 sum N_r(N_r - 1)
  Sec. II.B gate generators: R = exp(i theta N), S(theta, phi) = exp[theta/2 (e^{-i phi} a^2 - e^{i phi} a^dag^2)],
  BS(theta, phi) = exp[theta (e^{i phi} a_1 a_2^dag - e^{-i phi} a_1^dag a_2)],
  S2(theta, phi) = exp[theta (e^{i phi} a_1 a_2 - e^{-i phi} a_1^dag a_2^dag)],
  K = exp(i theta N^2), CK = exp(i theta N_1 N_2); Sec. IV.B: O_r = exp(theta_r A_r).
The model coefficient vectors (hop, pair, nn1, n2, n1) are the inputs defined in
paper_2606_05297_gb300.workloads; the operator forms they multiply are written
out here.
"""
from __future__ import annotations

MAXF = 4
A, AD = 0, 1  # annihilation, creation


def _n(r):
    return [(r, AD), (r, A)]


def hamiltonian_strings(model):
    """H = sum_b hop_b (a_r^dag a_s + a_s^dag a_r) + pair_b (a_r a_s + a_r^dag a_s^dag)
           + sum_r nn1_r a_r^dag a_r^dag a_r a_r + n2_r (a_r^dag a_r)^2 + n1_r a_r^dag a_r."""
    out = []
    L = model.L
    nb = L if model.periodic else L - 1
    for b in range(nb):
        r, s = b, (b + 1) % L
        t = model.hop[b]
        if t != 0.0:
            out.append((t, [(r, AD), (s, A)]))
            out.append((t, [(s, AD), (r, A)]))
        p = model.pair[b] if model.pair else 0.0
        if p != 0.0:
            out.append((p, [(r, A), (s, A)]))
            out.append((p, [(r, AD), (s, AD)]))
    for r in range(L):
        if model.nn1 and model.nn1[r] != 0.0:
            out.append((model.nn1[r], [(r, AD), (r, AD), (r, A), (r, A)]))
        if model.n2 and model.n2[r] != 0.0:
            out.append((model.n2[r], _n(r) + _n(r)))
        if model.n1 and model.n1[r] != 0.0:
            out.append((model.n1[r], _n(r)))
    return out


def phase(p: int) -> complex:
    """e^{i phi} for phi = p * pi / 2, exact."""
    return (1, 1j, -1, -1j)[p % 4]


def generator_strings(op):
    """Anti-Hermitian generator A of the single-parameter gate exp(theta A)."""
    typ, i, j, p = op.type, op.i, op.j, op.phase
    e = phase(p)
    ec = e.conjugate()
    if typ == "hop":      # BS: e^{i phi} a_i a_j^dag - e^{-i phi} a_i^dag a_j
        return [(e, [(i, A), (j, AD)]), (-ec, [(i, AD), (j, A)])]
    if typ == "sq2":      # S2: e^{i phi} a_i a_j - e^{-i phi} a_i^dag a_j^dag
        return [(e, [(i, A), (j, A)]), (-ec, [(i, AD), (j, AD)])]
    if typ == "sq1":      # S: (e^{-i phi} a^2 - e^{i phi} a^dag^2) / 2
        return [(0.5 * ec, [(i, A), (i, A)]), (-0.5 * e, [(i, AD), (i, AD)])]
    if typ == "pairhop":  # e^{i phi} a_i^2 a_j^dag^2 - e^{-i phi} a_i^dag^2 a_j^2
        return [(e, [(i, A), (i, A), (j, AD), (j, AD)]), (-ec, [(i, AD), (i, AD), (j, A), (j, A)])]
    if typ == "kerr":     # K: i N^2
        return [(1j, _n(i) + _n(i))]
    if typ == "nn1":      # i N (N - 1)
        return [(1j, [(i, AD), (i, AD), (i, A), (i, A)])]
    if typ == "rot":      # R: i N
        return [(1j, _n(i))]
    if typ == "xkerr":    # CK: i N_i N_j
        return [(1j, _n(i) + _n(j))]
    raise ValueError(f"unknown op type {typ}")
