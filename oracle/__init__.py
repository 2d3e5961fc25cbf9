"""CPU oracle for the state-vector gate-application path (complex128).

TEST INFRASTRUCTURE ONLY.  Imported by the tests, by the smoke check and by
the benchmark's CPU-baseline leg; never by the library.  The arithmetic lives
in sv_oracle.c (plain C, fp64, Eq. 1 of Sec. 2 written out as an index loop);
this module compiles it with gcc and marshals the seeded records from
`workloads` into the oracle's own flat arrays.

Gradients: `grad_param_shift` is the parameter-shift rule
dE/dtheta = (E(theta + pi/2) - E(theta - pi/2)) / 2 per gate occurrence,
which is exact for gates exp(-i theta P / 2) with P a Pauli matrix (RX, RY,
RZ); the paper's automatic gradients (Sec. 2, the tensorflow backend) give
the same derivative.  `grad_fd` is a plain central difference.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from typing import List, Optional, Sequence

import numpy as np

from workloads import KINDS, Circuit, Gate, PauliTerm

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sv_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

_KIND_CODE = {k: i for i, k in enumerate(KINDS)}   # same order as the C enum


def build(force: bool = False) -> str:
    """Compile sv_oracle.c to liboracle.so (gcc, -O2, OpenMP if available)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", _SRC, "-o", _LIB_PATH + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.orc_apply.argtypes = [I, P, I, P, I, P, P]
        L.orc_run.argtypes = [I, P, I, P, P, P, P, P, P, P, P, P, P, P, I, D]
        L.orc_expval.argtypes = [I, P, I, P, P, P, P, P, P, P]
        L.orc_probabilities.argtypes = [I, P, I, P, P]
        L.orc_sample.argtypes = [I, P, I, P, I, P, P]
        L.orc_sample_exact.argtypes = [I, P, I, P, I, P, P]
        L.orc_exact_total.argtypes = [I, P, P, P]
        L.orc_pauli_rotation.argtypes = [I, P, I, P, P, D]
        L.orc_norm2.argtypes = [I, P]
        L.orc_norm2.restype = D
        L.orc_dot.argtypes = [I, P, P, P, P]
        L.orc_init_basis.argtypes = [I, P, ctypes.c_uint64]
        L.orc_set_threads.argtypes = [I]
        L.orc_set_mutant.argtypes = [I]
        L.orc_get_threads.restype = I
        L.orc_have_openmp.restype = I
        _lib = L
    return _lib


def set_threads(t: int) -> None:
    lib().orc_set_threads(int(t))


def get_threads() -> int:
    return lib().orc_get_threads()


def have_openmp() -> bool:
    return bool(lib().orc_have_openmp())


def set_mutant(m: int) -> None:
    """Plant mistake m in the oracle (0 = none).  Pin-sensitivity tests only."""
    lib().orc_set_mutant(int(m))


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


class _Packed:
    def __init__(self, c: Circuit):
        ng = len(c.gates)
        self.ng = ng
        self.kind = np.zeros(ng, np.int32)
        self.ntar = np.zeros(ng, np.int32)
        self.tar = np.zeros(5 * max(ng, 1), np.int32)
        self.nctl = np.zeros(ng, np.int32)
        self.ctl = np.zeros(40 * max(ng, 1), np.int32)
        self.param = np.full(ng, -1, np.int32)
        self.angle = np.zeros(ng, np.float64)
        self.mat_off = np.zeros(ng, np.int64)
        self.letters = np.zeros(5 * max(ng, 1), np.uint8)
        pool: List[np.ndarray] = []
        off = 0
        for g, gate in enumerate(c.gates):
            self.kind[g] = _KIND_CODE[gate.kind]
            self.ntar[g] = len(gate.targets)
            self.tar[5 * g:5 * g + len(gate.targets)] = gate.targets
            self.nctl[g] = len(gate.controls)
            self.ctl[40 * g:40 * g + len(gate.controls)] = gate.controls
            self.param[g] = gate.param
            self.angle[g] = gate.angle
            for j, L in enumerate(gate.paulis):
                self.letters[5 * g + j] = ord(L)
            if gate.kind == "MATRIX":
                m = np.ascontiguousarray(gate.matrix, dtype=np.complex128).ravel()
                self.mat_off[g] = off
                pool.append(m)
                off += m.size
        self.pool = np.concatenate(pool) if pool else np.zeros(1, np.complex128)


def basis_state(n: int, x: int = 0) -> np.ndarray:
    psi = np.zeros(1 << n, np.complex128)
    lib().orc_init_basis(n, _ptr(psi), ctypes.c_uint64(x))
    return psi


def run(c: Circuit, theta: Optional[Sequence[float]] = None,
        psi0: Optional[np.ndarray] = None, basis: int = 0,
        shift_gate: int = -1, shift: float = 0.0) -> np.ndarray:
    """psi = U_N ... U_1 psi0 (psi0 = |basis> if not given)."""
    n = c.n_qubits
    psi = (np.array(psi0, dtype=np.complex128, copy=True) if psi0 is not None
           else basis_state(n, basis))
    th = np.ascontiguousarray(theta if theta is not None and len(theta) else [0.0],
                              dtype=np.float64)
    p = _Packed(c)
    rc = lib().orc_run(n, _ptr(psi), p.ng, _ptr(p.kind), _ptr(p.ntar), _ptr(p.tar),
                       _ptr(p.nctl), _ptr(p.ctl), _ptr(p.param), _ptr(p.angle),
                       _ptr(p.mat_off), _ptr(p.pool), _ptr(p.letters), _ptr(th), int(shift_gate),
                       float(shift))
    if rc:
        raise ValueError(f"oracle rejected the circuit (code {rc})")
    return psi


def apply_gate(psi: np.ndarray, n: int, targets: Sequence[int],
               controls: Sequence[int], G: np.ndarray) -> np.ndarray:
    """One Eq. (1) application of a dense matrix G (in place on a copy)."""
    out = np.array(psi, dtype=np.complex128, copy=True)
    t = np.ascontiguousarray(targets, np.int32)
    cc = np.ascontiguousarray(controls if len(controls) else [0], np.int32)
    g = np.ascontiguousarray(G, np.complex128)
    rc = lib().orc_apply(n, _ptr(out), len(targets), _ptr(t), len(controls),
                         _ptr(cc), _ptr(g))
    if rc:
        raise ValueError("oracle rejected the gate")
    return out


def probabilities(psi: np.ndarray, qubits: Sequence[int]) -> np.ndarray:
    """P(outcome) of measuring `qubits` (qubits[0] = most significant bit)."""
    n = int(psi.size).bit_length() - 1
    a = np.ascontiguousarray(psi, np.complex128)
    q = np.ascontiguousarray(qubits, np.int32)
    out = np.zeros(1 << len(q))
    if lib().orc_probabilities(n, _ptr(a), len(q), _ptr(q), _ptr(out)):
        raise ValueError("oracle rejected the measurement")
    return out


def sample(psi: np.ndarray, qubits: Sequence[int], uniforms: Sequence[float]) -> np.ndarray:
    """Inverse-CDF samples of `qubits` for the given uniforms in [0, 1)."""
    n = int(psi.size).bit_length() - 1
    a = np.ascontiguousarray(psi, np.complex128)
    q = np.ascontiguousarray(qubits, np.int32)
    u = np.ascontiguousarray(uniforms, np.float64)
    out = np.zeros(len(u), np.uint64)
    if lib().orc_sample(n, _ptr(a), len(q), _ptr(q), len(u), _ptr(u), _ptr(out)):
        raise ValueError("oracle rejected the sampling request")
    return out


def sample_exact(psi: np.ndarray, qubits: Sequence[int], uniforms: Sequence[float]) -> np.ndarray:
    """Inverse-CDF samples with the exact fixed-point CDF: q(v) = floor(v^2 2^120)
    per real component, 128-bit integer sums, T = floor(u * total)."""
    n = int(psi.size).bit_length() - 1
    a = np.ascontiguousarray(psi, np.complex128)
    q = np.ascontiguousarray(qubits, np.int32)
    u = np.ascontiguousarray(uniforms, np.float64)
    out = np.zeros(len(u), np.uint64)
    if lib().orc_sample_exact(n, _ptr(a), len(q), _ptr(q), len(u), _ptr(u), _ptr(out)):
        raise ValueError("oracle rejected the sampling request")
    return out


def exact_total(psi: np.ndarray) -> int:
    """sum over amplitudes of floor(re^2 2^120) + floor(im^2 2^120)."""
    n = int(psi.size).bit_length() - 1
    a = np.ascontiguousarray(psi, np.complex128)
    hi, lo = ctypes.c_uint64(), ctypes.c_uint64()
    lib().orc_exact_total(n, _ptr(a), ctypes.byref(hi), ctypes.byref(lo))
    return (hi.value << 64) | lo.value


def pauli_rotation(psi: np.ndarray, term_ops, a: float) -> np.ndarray:
    """exp(-i a P) psi for the Pauli string P = ((qubit, letter), ...)."""
    n = int(psi.size).bit_length() - 1
    out = np.array(psi, dtype=np.complex128, copy=True)
    q = np.ascontiguousarray([t[0] for t in term_ops] or [0], np.int32)
    L = np.ascontiguousarray([ord(t[1]) for t in term_ops] or [0], np.uint8)
    if lib().orc_pauli_rotation(n, _ptr(out), len(term_ops), _ptr(q), _ptr(L), float(a)):
        raise ValueError("oracle rejected the Pauli rotation")
    return out


def trotter(psi: np.ndarray, terms, t: float, steps: int, order: int = 1) -> np.ndarray:
    """Trotter product for exp(-i t H), H = sum_k c_k P_k: per step of
    dt = t / steps, first order applies exp(-i c_k dt P_k) for k = 1..K;
    second order applies exp(-i c_k dt/2 P_k) for k = 1..K, then k = K..1."""
    dt = t / steps
    out = np.array(psi, dtype=np.complex128, copy=True)
    for _ in range(steps):
        if order == 1:
            for c, ops in terms:
                out = pauli_rotation(out, ops, c * dt)
        else:
            for c, ops in terms:
                out = pauli_rotation(out, ops, 0.5 * c * dt)
            for c, ops in reversed(terms):
                out = pauli_rotation(out, ops, 0.5 * c * dt)
    return out


def norm2(psi: np.ndarray) -> float:
    n = int(psi.size).bit_length() - 1
    a = np.ascontiguousarray(psi, np.complex128)
    return lib().orc_norm2(n, _ptr(a))


def dot(a: np.ndarray, b: np.ndarray) -> complex:
    n = int(a.size).bit_length() - 1
    a = np.ascontiguousarray(a, np.complex128)
    b = np.ascontiguousarray(b, np.complex128)
    re, im = ctypes.c_double(), ctypes.c_double()
    lib().orc_dot(n, _ptr(a), _ptr(b), ctypes.byref(re), ctypes.byref(im))
    return complex(re.value, im.value)


def expval(psi: np.ndarray, terms: Sequence[PauliTerm], n: Optional[int] = None,
           per_term: bool = False):
    """<psi|H|psi> for H = sum_k c_k P_k (P_k a Pauli string)."""
    if n is None:
        n = int(psi.size).bit_length() - 1
    a = np.ascontiguousarray(psi, np.complex128)
    nt = len(terms)
    coeff = np.array([t[0] for t in terms] or [0.0], np.float64)
    nops = np.array([len(t[1]) for t in terms] or [0], np.int32)
    qubits = np.zeros(max(nt, 1) * n, np.int32)
    letters = np.zeros(max(nt, 1) * n, np.uint8)
    for k, (_, ops) in enumerate(terms):
        for j, (q, L) in enumerate(ops):
            qubits[k * n + j] = q
            letters[k * n + j] = ord(L)
    e = ctypes.c_double()
    tre = np.zeros(max(nt, 1))
    tim = np.zeros(max(nt, 1))
    rc = lib().orc_expval(n, _ptr(a), nt, _ptr(coeff), _ptr(nops), _ptr(qubits),
                          _ptr(letters), ctypes.byref(e), _ptr(tre), _ptr(tim))
    if rc:
        raise ValueError(f"oracle expval failed (code {rc})")
    if per_term:
        return e.value, tre[:nt] + 1j * tim[:nt]
    return e.value


def energy(c: Circuit, theta, terms, psi0=None, shift_gate=-1, shift=0.0) -> float:
    return expval(run(c, theta, psi0, shift_gate=shift_gate, shift=shift), terms, c.n_qubits)


def grad_param_shift(c: Circuit, theta, terms, params: Optional[Sequence[int]] = None,
                     psi0=None) -> np.ndarray:
    """Exact gradient by shift rules, summed over every gate that uses a
    parameter.  If `params` is given, only those entries are filled.

    Uncontrolled RX/RY/RZ and PAULI strings = exp(-i a P / 2) with P^2 = I:
    E(a) = A + B cos a + C sin a, so dE/da = (E(a + pi/2) - E(a - pi/2)) / 2.
    Controlled rotations = exp(-i a (Pc x P) / 2), Pc the all-ones projector
    of the controls: the generator's eigenvalues are 0 and +-1/2, so E(a)
    has frequencies 1/2 and 1.  For a component of frequency w,
    f(a + s) - f(a - s) = (2 sin(w s) / w) f'(a); requiring
    d+ (2 sin(w pi/2)/w) - d- (2 sin(w 3pi/2)/w) = 1 for w = 1 and w = 1/2
    gives d+ + d- = 1/2 and d+ - d- = 1/(2 sqrt 2), i.e. the exact rule
    dE/da = d+ [E(a+pi/2) - E(a-pi/2)] - d- [E(a+3pi/2) - E(a-3pi/2)],
    d+- = (sqrt2 +- 1) / (4 sqrt2)."""
    want = set(range(c.n_params)) if params is None else set(int(p) for p in params)
    g = np.zeros(c.n_params)
    dp = (math.sqrt(2) + 1) / (4 * math.sqrt(2))
    dm = (math.sqrt(2) - 1) / (4 * math.sqrt(2))
    for idx, gate in enumerate(c.gates):
        if gate.param >= 0 and gate.param in want:
            if gate.kind not in ("RX", "RY", "RZ", "PAULI"):
                raise ValueError("shift rules need RX, RY, RZ or PAULI gates")

            def E(s):
                return energy(c, theta, terms, psi0, idx, s)

            if not gate.controls:
                g[gate.param] += 0.5 * (E(math.pi / 2) - E(-math.pi / 2))
            else:
                g[gate.param] += (dp * (E(math.pi / 2) - E(-math.pi / 2))
                                  - dm * (E(1.5 * math.pi) - E(-1.5 * math.pi)))
    return g


def grad_fd(c: Circuit, theta, terms, h: float = 1e-3,
            params: Optional[Sequence[int]] = None, psi0=None) -> np.ndarray:
    """Central finite differences (E(theta + h e_j) - E(theta - h e_j)) / 2h."""
    theta = np.asarray(theta, np.float64)
    idx = range(c.n_params) if params is None else params
    g = np.zeros(c.n_params)
    for j in idx:
        tp = theta.copy(); tp[j] += h
        tm = theta.copy(); tm[j] -= h
        g[j] = (energy(c, tp, terms, psi0) - energy(c, tm, terms, psi0)) / (2 * h)
    return g
