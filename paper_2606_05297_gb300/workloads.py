"""Seeded synthetic inputs shared by the CUDA path, the tests and the oracle.

This module describes *inputs* only: lattice models as coefficient vectors,
operator pools as (type, i, j, phase) tuples, initial occupation tuples and
seeded random states / angles.  It performs none of the method's arithmetic
(no operator is applied, no energy or gradient is formed), so that the oracle
and the CUDA path can both read it without sharing any of the method.

Conventions (arXiv 2606.05297):
  * Model coefficients multiply fixed operator forms.  For the bond b = (r, s)
    with s = (r + 1) mod L:
        hop[b]  * (a_r^dag a_s + a_s^dag a_r)
        pair[b] * (a_r a_s + a_r^dag a_s^dag)
    and on site r:
        nn1[r] * n_r (n_r - 1) + n2[r] * n_r^2 + n1[r] * n_r.
    Eq. (BoseHubbard) gives hop = -J, nn1 = -U/2, n1 = -mu (mu = 0 in the fixed
    N sector, Sec. III.A).  Eq. (BosonicKitaevChain) gives hop = -J,
    pair = -Delta, n1 = -mu; Eq. (BosonicKitaevChain_Kerr) adds nn1 = -U/2.
    The Kitaev-chain-with-Kerr workloads use H = sum_j[-t a_j^dag a_{j+1}
    + Delta a_j a_{j+1} + h.c.] + K sum_j n_j^2, i.e. hop = -t, pair = +Delta,
    n2 = K.
  * Pool elements are single-parameter gates exp(theta A) (Sec. IV.B) with
    anti-Hermitian generators A selected by a type name and a phase index p,
    e^{i phi} = i^p:
        hop     BS   : e^{i phi} a_i a_j^dag - e^{-i phi} a_i^dag a_j
        sq2     S2   : e^{i phi} a_i a_j     - e^{-i phi} a_i^dag a_j^dag
        sq1     S    : (e^{-i phi} a_i^2 - e^{i phi} a_i^dag^2) / 2
        pairhop      : e^{i phi} a_i^2 a_j^dag^2 - e^{-i phi} a_i^dag^2 a_j^2
        kerr    K    : i n_i^2          rot R : i n_i
        nn1          : i n_i (n_i - 1)  xkerr CK : i n_i n_j
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, NamedTuple, Sequence

import numpy as np

OP_TYPES = ("hop", "sq2", "sq1", "pairhop", "kerr", "nn1", "rot", "xkerr")


class Op(NamedTuple):
    type: str
    i: int
    j: int = -1
    phase: int = 0


@dataclasses.dataclass
class Model:
    kind: str            # "bh" (fixed N) or "bkc" (fixed parity)
    L: int
    N: int = 0           # BH total boson number (cutoff D = N + 1)
    d: int = 0           # BKC per-mode cutoff
    parity: int = 0      # BKC sector parity (0 = even)
    periodic: bool = False
    hop: List[float] = dataclasses.field(default_factory=list)
    pair: List[float] = dataclasses.field(default_factory=list)
    nn1: List[float] = dataclasses.field(default_factory=list)
    n2: List[float] = dataclasses.field(default_factory=list)
    n1: List[float] = dataclasses.field(default_factory=list)
    name: str = ""

    @property
    def nbonds(self) -> int:
        return self.L if self.periodic else self.L - 1

    def bonds(self):
        return [(r, (r + 1) % self.L) for r in range(self.nbonds)]


def _full(vals, n):
    return [float(v) for v in vals] if isinstance(vals, (list, tuple, np.ndarray)) else [float(vals)] * n


def bose_hubbard(L: int, N: int, J: float = 1.0, U: float = 0.0, periodic: bool = True,
                 mu: float = 0.0, name: str = "") -> Model:
    """Eq. (BoseHubbard) in its literal sign convention (U > 0 attractive)."""
    nb = L if periodic else L - 1
    return Model("bh", L, N=N, periodic=periodic, hop=[-float(J)] * nb, pair=[0.0] * nb,
                 nn1=[-0.5 * float(U)] * L, n2=[0.0] * L, n1=[-float(mu)] * L, name=name)


def bose_hubbard_coeffs(L: int, N: int, hop: float, onsite_nn1: float, periodic: bool, name: str = "") -> Model:
    """Bose-Hubbard chain given the raw coefficients of the hop and n(n-1) terms."""
    nb = L if periodic else L - 1
    return Model("bh", L, N=N, periodic=periodic, hop=[float(hop)] * nb, pair=[0.0] * nb,
                 nn1=[float(onsite_nn1)] * L, n2=[0.0] * L, n1=[0.0] * L, name=name)


def kitaev_paper(L: int, d: int, J: float = 1.0, Delta: float = 0.5, mu: float = -3.1, U: float = 0.0,
                 periodic: bool = True, parity: int = 0, name: str = "") -> Model:
    """Eqs. (BosonicKitaevChain) and (BosonicKitaevChain_Kerr), literal signs."""
    nb = L if periodic else L - 1
    return Model("bkc", L, d=d, parity=parity, periodic=periodic, hop=[-float(J)] * nb,
                 pair=[-float(Delta)] * nb, nn1=[-0.5 * float(U)] * L, n2=[0.0] * L,
                 n1=[-float(mu)] * L, name=name)


def kitaev_kerr(L: int, d: int, t: float = 1.0, Delta=0.5, K: float = 0.1, periodic: bool = False,
                parity: int = 0, name: str = "") -> Model:
    """H = sum_j[-t a_j^dag a_{j+1} + Delta a_j a_{j+1} + h.c.] + K sum_j n_j^2."""
    nb = L if periodic else L - 1
    return Model("bkc", L, d=d, parity=parity, periodic=periodic, hop=[-float(t)] * nb,
                 pair=_full(Delta, nb), nn1=[0.0] * L, n2=[float(K)] * L, n1=[0.0] * L, name=name)


# ------------------------------------------------------------------ pools

def bh_nn_pool(model: Model) -> List[Op]:
    """Nearest-neighbour number-conserving pool: real and imaginary hopping on
    every bond, then n_i(n_i - 1) on every site."""
    ops = []
    for (r, s) in model.bonds():
        ops.append(Op("hop", r, s, 0))
        ops.append(Op("hop", r, s, 1))
    for r in range(model.L):
        ops.append(Op("nn1", r))
    return ops


def bh_allpairs_pool(L: int) -> List[Op]:
    """All-pairs number-conserving pool: for every pair i < j real hopping,
    imaginary hopping and pair hopping (a_i^dag)^2 a_j^2 + h.c. (phase index 1
    makes A = i G with G that Hermitian form), then on-site Kerr per site."""
    ops = []
    for i in range(L):
        for j in range(i + 1, L):
            ops.append(Op("hop", i, j, 0))
            ops.append(Op("hop", i, j, 1))
            ops.append(Op("pairhop", i, j, 1))
    for r in range(L):
        ops.append(Op("kerr", r))
    return ops


def bkc_kerr_pool(L: int) -> List[Op]:
    """Parity-preserving pool: beam splitter and two-mode squeezing on all
    pairs with phi in {0, pi/2}, single-mode squeezing per site with both
    phases, Kerr per site."""
    ops = []
    for i in range(L):
        for j in range(i + 1, L):
            for p in (0, 1):
                ops.append(Op("hop", i, j, p))
            for p in (0, 1):
                ops.append(Op("sq2", i, j, p))
    for r in range(L):
        for p in (0, 1):
            ops.append(Op("sq1", r, -1, p))
    for r in range(L):
        ops.append(Op("kerr", r))
    return ops


def bkc_table_pool(L: int, kerr: bool = False) -> List[Op]:
    """Table I pool of the Kitaev chain as single-parameter generators: beam
    splitter and two-mode squeezer on all pairs (phi in {0, pi/2}),
    single-mode squeezer per site (both phases) and rotation per site, plus
    Kerr per site and cross-Kerr per pair with a Kerr term."""
    ops = []
    for i in range(L):
        for j in range(i + 1, L):
            ops += [Op("hop", i, j, p) for p in (0, 1)] + [Op("sq2", i, j, p) for p in (0, 1)]
            if kerr:
                ops.append(Op("xkerr", i, j))
    for r in range(L):
        ops += [Op("sq1", r, -1, p) for p in (0, 1)] + [Op("rot", r)]
        if kerr:
            ops.append(Op("kerr", r))
    return ops


def paper_bkc_pool_two_param(L: int, kerr: bool = False) -> List[tuple]:
    """Table I pools with two-parameter gates counted once: BS and S2 on all
    pairs, S and R per site; BKC+K adds K per site and CK per pair."""
    gates = []
    for i in range(L):
        for j in range(i + 1, L):
            gates += [("BS", i, j), ("S2", i, j)]
            if kerr:
                gates.append(("CK", i, j))
    for r in range(L):
        gates += [("S", r), ("R", r)]
        if kerr:
            gates.append(("K", r))
    return gates


def hva_layer(model: Model) -> List[Op]:
    """One layer of the Hamiltonian variational ansatz used as the warm start
    (Eq. HVA_ansatz, Fig. 3, Sec. IV.A): one single-parameter gate per
    Hamiltonian term.  Bose-Hubbard: beam splitter generated by the hopping
    term on every bond, then Kerr and rotation per site.  Kitaev chain: two-mode
    squeezing and beam splitter generated by the pair and hopping terms on
    every bond, Kerr per site when the model has one, rotation per site."""
    ops: List[Op] = []
    if model.kind == "bh":
        ops += [Op("hop", r, s, 1) for (r, s) in model.bonds()]
        ops += [Op("kerr", r) for r in range(model.L)]
        ops += [Op("rot", r) for r in range(model.L)]
    else:
        ops += [Op("sq2", r, s, 1) for (r, s) in model.bonds()]
        ops += [Op("hop", r, s, 1) for (r, s) in model.bonds()]
        if any(v != 0.0 for v in model.n2) or any(v != 0.0 for v in model.nn1):
            ops += [Op("kerr", r) for r in range(model.L)]
        ops += [Op("rot", r) for r in range(model.L)]
    return ops


# ------------------------------------------------------------ random inputs

def random_state(dim: int, seed: int) -> np.ndarray:
    """Complex Gaussian vector, normalised, complex128."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(dim) + 1j * rng.standard_normal(dim)
    v /= np.linalg.norm(v)
    return v.astype(np.complex128)


def random_real_state(dim: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(dim).astype(np.complex128)
    v /= np.linalg.norm(v)
    return v


def random_thetas(n: int, seed: int, scale: float = 0.2) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, n)


def random_ansatz(pool_size: int, depth: int, seed: int, scale: float = 0.2):
    """Ops drawn uniformly from the pool and theta ~ U[-scale, scale]."""
    rng = np.random.default_rng(seed)
    ids = rng.integers(0, pool_size, depth)
    th = rng.uniform(-scale, scale, depth)
    return [int(i) for i in ids], th


def warm_start_thetas(n: int, seed: int) -> np.ndarray:
    """Warm-start angles uniform in [-0.05, 0.05] (Sec. IV.A, App. C)."""
    return np.random.default_rng(seed).uniform(-0.05, 0.05, n)


def mott_occupation(L: int, N: int) -> List[int]:
    """Bosons spread over all sites (Sec. IV.A initial state for Lambda < 0);
    any remainder goes to the first sites."""
    base, rem = divmod(N, L)
    return [base + (1 if r < rem else 0) for r in range(L)]


def vacuum_occupation(L: int) -> List[int]:
    return [0] * L


# ------------------------------------------------------------- workloads

def c1_model() -> Model:
    """Bose-Hubbard open chain L=4, N=4, J=1, U=2, mu=0."""
    return bose_hubbard(4, 4, J=1.0, U=2.0, periodic=False, name="bh_open_L4_N4_U2")


def c2_model(U_over_J: float = 3.4, convention: str = "paper") -> Model:
    """Bose-Hubbard periodic chain L=12, N=12, J=1.  convention 'paper' uses the
    literal -U/2 n(n-1) of Eq. (BoseHubbard); 'repulsive' uses +U/2."""
    U = U_over_J if convention == "paper" else -U_over_J
    return bose_hubbard(12, 12, J=1.0, U=U, periodic=True, name=f"bh_pbc_L12_N12_U{U_over_J}_{convention}")


def c3_model(seed: int = 0, K: float = 0.1, L: int = 8, d: int = 8) -> Model:
    """Kitaev chain + Kerr, open, t=1, Delta ~ U[0,1] drawn once from the seed."""
    delta = float(np.random.default_rng(seed).uniform(0.0, 1.0))
    return kitaev_kerr(L, d, t=1.0, Delta=delta, K=K, periodic=False, name=f"bkck_open_L{L}_d{d}_K{K}_s{seed}")


def c4_instances(seed: int = 0, count: int = 64):
    """Batched Bose-Hubbard sweep: L ~ U{8..12}, N = L, U/J log-uniform in
    [0.5, 20], periodic, J = 1 (literal Eq. (BoseHubbard) sign)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        L = int(rng.integers(8, 13))
        u = float(math.exp(rng.uniform(math.log(0.5), math.log(20.0))))
        out.append(bose_hubbard(L, L, J=1.0, U=u, periodic=True, name=f"bh_pbc_L{L}_U{u:.3f}_i{k}"))
    return out


def c5_model(L: int = 10, d: int = 6) -> Model:
    """Kitaev chain + Kerr, open, L=10, d=6, t=1, Delta=0.6, K=0.3."""
    return kitaev_kerr(L, d, t=1.0, Delta=0.6, K=0.3, periodic=False, name=f"bkck_open_L{L}_d{d}")


def pool_for(model: Model) -> List[Op]:
    if model.kind == "bh":
        return bh_nn_pool(model) if not model.periodic and model.L <= 4 else bh_allpairs_pool(model.L)
    return bkc_kerr_pool(model.L)


def initial_occupation(model: Model) -> List[int]:
    return mott_occupation(model.L, model.N) if model.kind == "bh" else vacuum_occupation(model.L)


# ---------------------------------------------------------------- scorer inputs

SCORER_SHAPES = [(256, 32), (256,), (256, 256), (256,), (256,), ()]


def scorer_params(seed: int) -> np.ndarray:
    """A float32 parameter vector of the proposal scorer (He-scaled normal
    weights, small normal biases), in the order W1, b1, W2, b2, w3, b3."""
    rng = np.random.default_rng(seed)
    fan = [32, 1, 256, 1, 256, 1]
    parts = []
    for shape, f in zip(SCORER_SHAPES, fan):
        n = int(np.prod(shape))
        scale = math.sqrt(2.0 / f) if f > 1 else 0.1
        parts.append(rng.standard_normal(n) * scale)
    return np.concatenate(parts).astype(np.float32)


def scorer_inputs(rows: int, seed: int) -> np.ndarray:
    """Feature rows shaped like the proposal's inputs: a one-hot block, values
    in [0, 1] and signed log-magnitudes."""
    rng = np.random.default_rng(seed)
    X = np.zeros((rows, 32), dtype=np.float32)
    X[np.arange(rows), rng.integers(0, 8, rows)] = 1.0
    X[:, 8:20] = rng.random((rows, 12))
    X[:, 20:32] = rng.standard_normal((rows, 12)) * 3.0
    return X
