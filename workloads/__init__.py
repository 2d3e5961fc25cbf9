"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module only *describes* inputs: circuits as lists of gate records
(kind, targets, controls, parameter index or fixed angle), parameter vectors,
basis indices, random states and Pauli sums written as letters per qubit.
It holds none of the simulation arithmetic: no gate matrix is built from an
angle here and no gate is applied.  Each side (the CPU oracle and the GPU
library) turns these records into matrices and masks with its own code.

Conventions (the paper fixes none of them; Sec. 2, Eq. 1 only splits the
amplitude index into target bits tau and the rest q):

* qubit q is amplitude-index bit n-1-q (qubit 0 is the most significant bit);
* for targets (t_0 .. t_{k-1}) the row/column index of G is
  tau = sum_j b(t_j) 2^(k-1-j), so t_0 is the most significant bit of tau;
* a gate with controls acts only where every control qubit is 1;
* random numbers come from SplitMix64 (Steele, Lea, Flood, OOPSLA 2014):
  state += 0x9E3779B97F4A7C15, output = mix(state); a uniform draw is
  (next >> 11) * 2^-53 in [0, 1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MASK64 = (1 << 64) - 1

# Gate kinds.  Controlled forms are the same kinds with controls:
# CZ = Z + 1 control, CNOT = X + 1 control, CU1(l) = U1(l) + 1 control.
# PAULI(a) = exp(-i a P / 2) for the Pauli string P whose letters (one per
# target, in `paulis`) act on the targets; no controls.
BASE_KINDS = ("H", "X", "Y", "Z", "RX", "RY", "RZ", "U1", "SWAP", "MATRIX")
KINDS = BASE_KINDS + ("PAULI",)
PARAM_KINDS = ("RX", "RY", "RZ", "PAULI")
MAX_TARGETS = 5
MAX_CONTROLS = 8


# --------------------------------------------------------------------------
# SplitMix64
# --------------------------------------------------------------------------
def _mix64(z: int) -> int:
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


class SplitMix64:
    """Sequential SplitMix64 stream (scalar draws)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next(self) -> int:
        self.state = (self.state + GAMMA) & MASK64
        return _mix64(self.state)

    def uniform(self) -> float:
        return (self.next() >> 11) * (1.0 / 9007199254740992.0)

    def angle(self) -> float:
        return 2.0 * math.pi * self.uniform()


def splitmix64_block(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of the SplitMix64 stream with `seed`.

    Output k is mix(seed + (k+1) * GAMMA), so a block is computed without
    walking the stream.
    """
    k = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + k * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform_block(seed: int, start: int, count: int) -> np.ndarray:
    z = splitmix64_block(seed, start, count)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


# --------------------------------------------------------------------------
# Records
# --------------------------------------------------------------------------
@dataclass(frozen=True)
class Gate:
    kind: str
    targets: Tuple[int, ...]
    controls: Tuple[int, ...] = ()
    param: int = -1          # index into theta, -1 for a fixed angle
    angle: float = 0.0       # used when param == -1 (U1, or fixed rotations)
    matrix: Optional[np.ndarray] = field(default=None, compare=False)  # MATRIX only
    paulis: str = ""         # PAULI only: one letter X, Y or Z per target

    def __post_init__(self):
        assert self.kind in KINDS, self.kind
        if self.kind == "PAULI":
            assert len(self.paulis) == len(self.targets) and set(self.paulis) <= set("XYZ")
            assert not self.controls


@dataclass
class Circuit:
    n_qubits: int
    gates: List[Gate]
    n_params: int = 0
    name: str = ""

    def inverse_with(self, theta: np.ndarray) -> Tuple["Circuit", np.ndarray]:
        """Gates of U^dagger as records: reversed order, rotation angles and
        U1 angles negated, H/X/Y/Z/SWAP unchanged, MATRIX conjugate-transposed.
        Returns the inverse circuit with fixed angles (no parameters)."""
        inv = []
        for g in reversed(self.gates):
            if g.kind in PARAM_KINDS or g.kind == "U1":
                a = theta[g.param] if g.param >= 0 else g.angle
                inv.append(Gate(g.kind, g.targets, g.controls, -1, -float(a),
                                paulis=g.paulis))
            elif g.kind == "MATRIX":
                inv.append(Gate("MATRIX", g.targets, g.controls,
                                matrix=np.conj(g.matrix.T).copy()))
            else:
                inv.append(g)
        return Circuit(self.n_qubits, inv, 0, self.name + "^-1"), np.zeros(0)


# A Pauli sum: list of (coefficient, ((qubit, letter), ...)), letters in XYZ.
PauliTerm = Tuple[float, Tuple[Tuple[int, str], ...]]


# --------------------------------------------------------------------------
# Circuits shaped like the paper's workloads (Sec. 3: QFT, variational
# layers, VQE; Sec. 1: Schroedinger simulation cost linear in the gates)
# --------------------------------------------------------------------------
def random_layered(n: int, depth: int, seed: int) -> Tuple[Circuit, np.ndarray]:
    """Random layered circuit: each layer applies RX, RY, RZ on every qubit
    (angles uniform in [0, 2pi), drawn layer-major, then qubit, then
    RX, RY, RZ) followed by CZ(i, i+1) for i = l mod 2, l mod 2 + 2, ...
    (open chain, no wrap)."""
    rng = SplitMix64(seed)
    gates: List[Gate] = []
    theta: List[float] = []
    for layer in range(depth):
        for q in range(n):
            for kind in ("RX", "RY", "RZ"):
                theta.append(rng.angle())
                gates.append(Gate(kind, (q,), (), len(theta) - 1))
        for i in range(layer % 2, n - 1, 2):
            gates.append(Gate("Z", (i + 1,), (i,)))
    return Circuit(n, gates, len(theta), f"layered_n{n}_d{depth}"), np.array(theta)


def qft(n: int) -> Circuit:
    """Quantum Fourier transform: for each qubit i, H(i) then the controlled
    phase U1(pi / 2^(j-i)) with control j on target i for j > i; then
    SWAP(i, n-1-i) for i < n/2.  n + n(n-1)/2 + floor(n/2) gates."""
    gates: List[Gate] = []
    for i in range(n):
        gates.append(Gate("H", (i,)))
        for j in range(i + 1, n):
            gates.append(Gate("U1", (i,), (j,), -1, math.pi / (1 << (j - i))))
    for i in range(n // 2):
        gates.append(Gate("SWAP", (i, n - 1 - i)))
    return Circuit(n, gates, 0, f"qft_n{n}")


def hea(n: int, layers: int, seed: int) -> Tuple[Circuit, np.ndarray]:
    """Hardware-efficient ansatz: layer l is RY(theta[l*n + q]) on every
    qubit q, then CZ(0,1), CZ(1,2), ..., CZ(n-2, n-1) in that order."""
    rng = SplitMix64(seed)
    gates: List[Gate] = []
    theta = np.array([rng.angle() for _ in range(n * layers)])
    for layer in range(layers):
        for q in range(n):
            gates.append(Gate("RY", (q,), (), layer * n + q))
        for i in range(n - 1):
            gates.append(Gate("Z", (i + 1,), (i,)))
    return Circuit(n, gates, n * layers, f"hea_n{n}_L{layers}"), theta


def hea_theta(n: int, layers: int, seed: int) -> np.ndarray:
    """The parameter vector hea(n, layers, seed) draws, without the circuit."""
    rng = SplitMix64(seed)
    return np.array([rng.angle() for _ in range(n * layers)])


def grover(n: int, marked: int, iterations: int) -> Circuit:
    """Grover search for the basis state `marked` (Sec. 3: Grover's
    algorithm): H on every qubit, then per iteration the oracle (X on the
    qubits where `marked` has a 0, Z on qubit n-1 controlled by all others,
    the same X again) and the diffusion (H, X on every qubit, the same
    multi-controlled Z, X, H)."""
    hs = [Gate("H", (q,)) for q in range(n)]
    xs = [Gate("X", (q,)) for q in range(n)]
    flips = [Gate("X", (q,)) for q in range(n) if not (marked >> (n - 1 - q)) & 1]
    mcz = Gate("Z", (n - 1,), tuple(range(n - 1)))
    gates = list(hs)
    for _ in range(iterations):
        gates += flips + [mcz] + flips
        gates += hs + xs + [mcz] + xs + hs
    return Circuit(n, gates, 0, f"grover_n{n}_k{iterations}")


def ghz(n: int) -> Circuit:
    gates = [Gate("H", (0,))] + [Gate("X", (k + 1,), (k,)) for k in range(n - 1)]
    return Circuit(n, gates, 0, f"ghz_n{n}")


def tfim(n: int, h: float = 0.7) -> List[PauliTerm]:
    """Transverse-field Ising chain, open boundaries:
    H = sum_{i<n-1} Z_i Z_{i+1} + h sum_i X_i."""
    terms: List[PauliTerm] = [(1.0, ((i, "Z"), (i + 1, "Z"))) for i in range(n - 1)]
    terms += [(h, ((i, "X"),)) for i in range(n)]
    return terms


def sum_z(n: int) -> List[PauliTerm]:
    return [(1.0, ((i, "Z"),)) for i in range(n)]


def random_pauli_sum(n: int, n_terms: int, seed: int) -> List[PauliTerm]:
    """Random Pauli strings with random letters on a random subset of qubits
    and coefficients uniform in [-1, 1)."""
    rng = SplitMix64(seed)
    terms: List[PauliTerm] = []
    for _ in range(n_terms):
        ops = []
        for q in range(n):
            r = rng.next() % 4
            if r:
                ops.append((q, "XYZ"[r - 1]))
        terms.append((2.0 * rng.uniform() - 1.0, tuple(ops)))
    return terms


def random_basis_index(n: int, seed: int) -> int:
    return SplitMix64(seed).next() & ((1 << n) - 1)


def random_state(n: int, seed: int) -> np.ndarray:
    """Seeded complex Gaussian vector (Box-Muller on SplitMix64 uniforms),
    scaled to unit norm.  complex128, length 2^n."""
    dim = 1 << n
    u = uniform_block(seed, 0, 2 * dim)
    u1, u2 = 1.0 - u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    v = r * np.cos(2 * np.pi * u2) + 1j * r * np.sin(2 * np.pi * u2)
    return v / np.linalg.norm(v)


def random_unitary(k: int, rng: SplitMix64) -> np.ndarray:
    """2^k x 2^k unitary: QR of a seeded complex Gaussian, with the phases of
    R's diagonal divided out."""
    d = 1 << k
    u = np.array([rng.uniform() for _ in range(2 * d * d)])
    u1, u2 = 1.0 - u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = (r * np.cos(2 * np.pi * u2) + 1j * r * np.sin(2 * np.pi * u2)).reshape(d, d)
    q, rr = np.linalg.qr(z)
    ph = np.diag(rr) / np.abs(np.diag(rr))
    return q * ph[None, :]


def random_gates(n: int, n_gates: int, seed: int, max_tar: int = 5,
                 max_ctrl: int = 3, kinds: Sequence[str] = BASE_KINDS) -> Tuple[Circuit, np.ndarray]:
    """Random gate list over every kind: random distinct targets and
    controls, rotation angles as parameters, MATRIX gates with seeded
    unitaries on 1..max_tar targets."""
    rng = SplitMix64(seed)
    gates: List[Gate] = []
    theta: List[float] = []
    for _ in range(n_gates):
        kind = kinds[rng.next() % len(kinds)]
        if kind == "SWAP":
            k = 2
        elif kind in ("MATRIX", "PAULI"):
            k = 1 + rng.next() % min(max_tar, n)
        else:
            k = 1
        if kind == "SWAP" and n < 2:
            kind, k = "H", 1
        nc = rng.next() % (min(max_ctrl, n - k) + 1) if kind != "PAULI" else 0
        perm = list(range(n))
        for i in range(n - 1, 0, -1):          # Fisher-Yates
            j = rng.next() % (i + 1)
            perm[i], perm[j] = perm[j], perm[i]
        tg, ct = tuple(perm[:k]), tuple(perm[k:k + nc])
        if kind == "PAULI":
            letters = "".join("XYZ"[rng.next() % 3] for _ in range(k))
            theta.append(rng.angle())
            gates.append(Gate(kind, tg, (), len(theta) - 1, paulis=letters))
        elif kind in PARAM_KINDS:
            theta.append(rng.angle())
            gates.append(Gate(kind, tg, ct, len(theta) - 1))
        elif kind == "U1":
            gates.append(Gate(kind, tg, ct, -1, rng.angle()))
        elif kind == "MATRIX":
            gates.append(Gate(kind, tg, ct, matrix=random_unitary(k, rng)))
        else:
            gates.append(Gate(kind, tg, ct))
    return Circuit(n, gates, len(theta), f"random_n{n}_g{n_gates}"), np.array(theta)


def mixed_batch(count: int, seed: int, n_lo: int = 8, n_hi: int = 16,
                l_lo: int = 5, l_hi: int = 15):
    """`count` hardware-efficient ansatz items with qubit counts uniform in
    [n_lo, n_hi] and depths uniform in [l_lo, l_hi]; item i takes its
    angles from seed + 1 + i.  Returns a list of (circuit, theta, H)."""
    rng = SplitMix64(seed)
    items = []
    for i in range(count):
        n = n_lo + rng.next() % (n_hi - n_lo + 1)
        L = l_lo + rng.next() % (l_hi - l_lo + 1)
        c, th = hea(n, L, seed + 1 + i)
        items.append((c, th, tfim(n)))
    return items


# --------------------------------------------------------------------------
# QAOA for MaxCut (Sec. 3: pre-coded MaxCut Hamiltonian and QAOA models;
# QAOA as defined by Farhi, Goldstone, Gutmann, arXiv:1411.4028)
# --------------------------------------------------------------------------
def ring_graph(n: int) -> List[Tuple[int, int]]:
    """Edges (i, i+1 mod n) of the n-cycle."""
    return [(i, (i + 1) % n) for i in range(n)]


def random_regular_graph(n: int, d: int, seed: int) -> List[Tuple[int, int]]:
    """A seeded simple d-regular graph on n vertices (n d even): pair the
    n d half-edges by a Fisher-Yates shuffle and retry until no loop or
    repeated edge remains.  Edges as (i, j) with i < j, sorted."""
    assert (n * d) % 2 == 0 and d < n
    rng = SplitMix64(seed)
    while True:
        stubs = [v for v in range(n) for _ in range(d)]
        for i in range(len(stubs) - 1, 0, -1):
            j = rng.next() % (i + 1)
            stubs[i], stubs[j] = stubs[j], stubs[i]
        edges = set()
        ok = True
        for a, b in zip(stubs[0::2], stubs[1::2]):
            e = (min(a, b), max(a, b))
            if a == b or e in edges:
                ok = False
                break
            edges.add(e)
        if ok:
            return sorted(edges)


def maxcut(edges: Sequence[Tuple[int, int]]) -> List[PauliTerm]:
    """The MaxCut cost C = sum over edges (i, j) of (1 - Z_i Z_j) / 2 as a
    Pauli sum: the identity with coefficient |E| / 2 (empty string) and
    -1/2 Z_i Z_j per edge."""
    terms: List[PauliTerm] = [(0.5 * len(edges), ())]
    terms += [(-0.5, ((i, "Z"), (j, "Z"))) for i, j in edges]
    return terms


def qaoa(n: int, edges: Sequence[Tuple[int, int]], p: int, seed: int) -> Tuple[Circuit, np.ndarray]:
    """QAOA circuit with p layers on the MaxCut graph `edges`: H on every
    qubit (|+>^n), then per layer l the cost rotations PAULI "ZZ" on every
    edge with parameter 2l and the mixer rotations PAULI "X" on every qubit
    with parameter 2l + 1.  A gate PAULI(a) is exp(-i a P / 2), so Farhi et
    al.'s U(C, gamma) = exp(-i gamma C) is (up to a global phase) the cost
    rotations at a = -gamma and U(B, beta) = exp(-i beta sum_j X_j) the
    mixer at a = 2 beta.  Angles uniform in [0, 2pi) from the seed."""
    rng = SplitMix64(seed)
    gates: List[Gate] = [Gate("H", (q,)) for q in range(n)]
    for layer in range(p):
        for i, j in edges:
            gates.append(Gate("PAULI", (i, j), (), 2 * layer, paulis="ZZ"))
        for q in range(n):
            gates.append(Gate("PAULI", (q,), (), 2 * layer + 1, paulis="X"))
    theta = np.array([rng.angle() for _ in range(2 * p)])
    return Circuit(n, gates, 2 * p, f"qaoa_n{n}_p{p}"), theta
