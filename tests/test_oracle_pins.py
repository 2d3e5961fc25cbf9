"""Pins of the CPU oracle against facts that do not come from the oracle.

Each check below fixes one part of the oracle by something independent:
brute-force 2^n x 2^n operators built with numpy Kronecker products and
scipy's matrix exponential (Eq. 1 of Sec. 2 as a dense matrix product),
closed forms (the QFT of a basis state, GHZ, rotations of |0>, product-state
energies), hand-derived worked examples in tests/golden, and invariants
(unitarity, U followed by U^dagger, parameter shift against finite
differences).  A separate test plants known mistakes in the oracle and
checks that these pins catch each one.
"""
import math

import numpy as np
import pytest
import scipy.linalg

import oracle
import workloads as W
from golden_io import load as load_golden

PAULI = {
    "X": np.array([[0, 1], [1, 0]], np.complex128),
    "Y": np.array([[0, -1j], [1j, 0]], np.complex128),
    "Z": np.array([[1, 0], [0, -1]], np.complex128),
}


def textbook_matrix(g: W.Gate, theta) -> np.ndarray:
    """Gate matrices from their textbook definitions (scipy expm for the
    rotations exp(-i a P / 2)), independent of the oracle's gate table."""
    a = theta[g.param] if g.param >= 0 else g.angle
    if g.kind == "H":
        return scipy.linalg.hadamard(2).astype(np.complex128) / math.sqrt(2)
    if g.kind in PAULI:
        return PAULI[g.kind]
    if g.kind in ("RX", "RY", "RZ"):
        return scipy.linalg.expm(-0.5j * a * PAULI[g.kind[1]])
    if g.kind == "U1":
        return np.diag([1.0, np.exp(1j * a)])
    if g.kind == "SWAP":
        m = np.zeros((4, 4), np.complex128)
        for b0 in range(2):
            for b1 in range(2):
                m[2 * b1 + b0, 2 * b0 + b1] = 1
        return m
    return np.asarray(g.matrix, np.complex128)


def full_operator(n, targets, controls, G) -> np.ndarray:
    """The 2^n x 2^n operator of G on `targets` with `controls`: built in the
    qubit order (targets, controls, rest) as kron(G, P1) + kron(I, I - P1)
    (P1 the projector on controls = 1...1), extended by kron with the
    identity, then its tensor axes permuted to qubit order 0..n-1 (qubit 0 =
    most significant index bit)."""
    k, nc = len(targets), len(controls)
    rest = [q for q in range(n) if q not in targets and q not in controls]
    order = list(targets) + list(controls) + rest
    P1 = np.zeros((1 << nc, 1 << nc))
    P1[-1, -1] = 1.0
    core = np.kron(G, P1) + np.kron(np.eye(1 << k), np.eye(1 << nc) - P1)
    U = np.kron(core, np.eye(1 << len(rest)))
    T = U.reshape([2] * (2 * n))
    inv = [order.index(q) for q in range(n)]
    T = T.transpose(inv + [n + i for i in inv])
    return T.reshape(1 << n, 1 << n)


def pauli_operator(n, terms) -> np.ndarray:
    H = np.zeros((1 << n, 1 << n), np.complex128)
    for c, ops in terms:
        f = [np.eye(2, dtype=np.complex128)] * n
        for q, L in ops:
            f[q] = PAULI[L]
        P = f[0]
        for m in f[1:]:
            P = np.kron(P, m)
        H += c * P
    return H


def _single(c: W.Circuit, g: W.Gate) -> W.Circuit:
    return W.Circuit(c.n_qubits, [g], c.n_params)


# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,seed", [(1, 1), (2, 2), (3, 3), (4, 4), (5, 5),
                                    (6, 6), (7, 7), (8, 8)])
def test_eq1_against_bruteforce_kronecker(n, seed):
    circ, theta = W.random_gates(n, 40, seed, max_tar=min(5, n), max_ctrl=3)
    psi = W.random_state(n, 100 + seed)
    for g in circ.gates:
        ref = full_operator(n, g.targets, g.controls, textbook_matrix(g, theta)) @ psi
        got = oracle.run(_single(circ, g), theta, psi)
        assert np.max(np.abs(got - ref)) < 1e-13, g
        psi = got


def test_every_target_order_and_width():
    n = 7
    rng = W.SplitMix64(77)
    psi = W.random_state(n, 7)
    for k in range(1, 6):
        for _ in range(6):
            perm = list(range(n))
            for i in range(n - 1, 0, -1):
                j = rng.next() % (i + 1)
                perm[i], perm[j] = perm[j], perm[i]
            t, c = perm[:k], perm[k:k + rng.next() % (n - k + 1)][:3]
            G = W.random_unitary(k, rng)
            ref = full_operator(n, t, c, G) @ psi
            got = oracle.apply_gate(psi, n, t, c, G)
            assert np.max(np.abs(got - ref)) < 1e-13


def test_random_circuit_n10_bruteforce():
    n = 10
    circ, theta = W.random_gates(n, 25, 11, max_tar=4, max_ctrl=2)
    psi = W.random_state(n, 3)
    ref = psi.copy()
    for g in circ.gates:
        ref = full_operator(n, g.targets, g.controls, textbook_matrix(g, theta)) @ ref
    got = oracle.run(circ, theta, psi)
    assert np.max(np.abs(got - ref)) < 1e-12


def test_layered_n12_bruteforce_prefix():
    """Random layered circuit at n = 12 (4096 amplitudes): the first two
    layers as dense 4096 x 4096 operator products."""
    n = 12
    circ, theta = W.random_layered(n, 20, 1000)
    assert len(circ.gates) == 830 and circ.n_params == 720
    prefix = W.Circuit(n, circ.gates[:2 * 36 + 11], circ.n_params)
    ref = np.zeros(1 << n, np.complex128)
    ref[0] = 1
    for g in prefix.gates:
        ref = full_operator(n, g.targets, g.controls, textbook_matrix(g, theta)) @ ref
    got = oracle.run(prefix, theta)
    assert np.max(np.abs(got - ref)) < 1e-12


# --------------------------------------------------------------------------
@pytest.mark.parametrize("n", list(range(1, 11)) + [14])
def test_qft_closed_form(n):
    c = W.qft(n)
    assert len(c.gates) == n + n * (n - 1) // 2 + n // 2
    N = 1 << n
    rng = W.SplitMix64(500 + n)
    xs = {0, N - 1, rng.next() % N, rng.next() % N}
    y = np.arange(N, dtype=np.uint64)
    for x in xs:
        phase = ((np.uint64(x) * y) % np.uint64(N)).astype(np.float64) / N
        ref = np.exp(2j * np.pi * phase) / math.sqrt(N)
        got = oracle.run(c, None, basis=x)
        assert np.max(np.abs(got - ref)) < 1e-12


@pytest.mark.parametrize("n", [2, 3, 5, 9])
def test_ghz_and_bell(n):
    psi = oracle.run(W.ghz(n))
    ref = np.zeros(1 << n, np.complex128)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    assert np.max(np.abs(psi - ref)) < 1e-15


@pytest.mark.parametrize("block", load_golden(), ids=lambda b: b["name"])
def test_golden_worked_examples(block):
    psi = oracle.run(block["circuit"], None, basis=block["input"])
    if "amps" in block:
        assert np.max(np.abs(psi - block["amps"])) < 1e-15
    if "energy" in block:
        assert abs(oracle.expval(psi, W.tfim(block["n"])) - block["energy"]) < 1e-14


def test_rotation_closed_forms():
    for a in np.linspace(-7, 7, 23):
        c, s = math.cos(a / 2), math.sin(a / 2)
        for kind, ref0, ref1 in (("RX", c, -1j * s), ("RY", c, s)):
            psi = oracle.run(W.Circuit(1, [W.Gate(kind, (0,), (), -1, a)], 0))
            assert abs(psi[0] - ref0) < 1e-15 and abs(psi[1] - ref1) < 1e-15
        psi = oracle.run(W.Circuit(1, [W.Gate("RZ", (0,), (), -1, a)], 0), basis=1)
        assert abs(psi[1] - np.exp(0.5j * a)) < 1e-15


def test_involutions():
    n = 4
    psi = W.random_state(n, 9)
    for kind, t in (("H", (1,)), ("X", (2,)), ("Y", (0,)), ("Z", (3,)), ("SWAP", (0, 3))):
        c = W.Circuit(n, [W.Gate(kind, t), W.Gate(kind, t)], 0)
        assert np.max(np.abs(oracle.run(c, None, psi) - psi)) < 1e-15


# --------------------------------------------------------------------------
def test_norm_preserved_and_inverse_returns_zero_state():
    n = 10
    circ, theta = W.random_layered(n, 6, 42)
    psi = oracle.run(circ, theta)
    assert abs(oracle.norm2(psi) - 1.0) < 1e-13
    inv, _ = circ.inverse_with(theta)
    back = oracle.run(inv, None, psi)
    ref = np.zeros(1 << n, np.complex128)
    ref[0] = 1
    assert np.max(np.abs(back - ref)) < 1e-13
    rc, rth = W.random_gates(8, 60, 5)
    psi = oracle.run(rc, rth, W.random_state(8, 6))
    assert abs(oracle.norm2(psi) - 1.0) < 1e-13
    inv, _ = rc.inverse_with(rth)
    assert np.max(np.abs(oracle.run(inv, None, psi) - W.random_state(8, 6))) < 1e-13


def test_norm_and_dot_pairwise_exact_cases():
    n = 16
    psi = np.full(1 << n, 1 / 256.0, np.complex128)
    assert oracle.norm2(psi) == 1.0
    a = W.random_state(6, 1)
    b = W.random_state(6, 2)
    assert abs(oracle.dot(a, b) - np.vdot(a, b)) < 1e-15


# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,seed", [(2, 1), (4, 2), (6, 3), (7, 4)])
def test_expval_against_dense_pauli_operator(n, seed):
    terms = W.random_pauli_sum(n, 12, seed) + W.tfim(n)
    psi = W.random_state(n, seed + 10)
    H = pauli_operator(n, terms)
    ref = np.vdot(psi, H @ psi)
    e, per = oracle.expval(psi, terms, per_term=True)
    assert abs(e - ref.real) < 1e-13
    assert np.max(np.abs(per.imag)) < 1e-13


def test_energy_special_cases():
    n, L = 8, 3
    circ, theta = W.hea(n, L, 7)
    assert abs(oracle.energy(circ, np.zeros_like(theta), W.tfim(n)) - (n - 1)) < 1e-13
    th = theta[:n]
    ry = W.Circuit(n, [W.Gate("RY", (q,), (), q) for q in range(n)], n)
    e = oracle.energy(ry, th, W.tfim(n))
    ref = sum(math.cos(th[i]) * math.cos(th[i + 1]) for i in range(n - 1)) \
        + 0.7 * sum(math.sin(t) for t in th)
    assert abs(e - ref) < 1e-13
    # dE/dtheta_i of the product state, differentiated by hand
    g = oracle.grad_param_shift(ry, th, W.tfim(n))
    cs = [math.cos(t) for t in th]
    ref_g = [-math.sin(th[i]) * ((cs[i - 1] if i > 0 else 0) + (cs[i + 1] if i < n - 1 else 0))
             + 0.7 * math.cos(th[i]) for i in range(n)]
    assert np.max(np.abs(g - np.array(ref_g))) < 1e-13
    assert abs(oracle.energy(W.Circuit(3, [], 0), None, W.sum_z(3)) - 3.0) < 1e-15


def test_param_shift_matches_central_difference():
    n, L = 5, 3
    circ, theta = W.hea(n, L, 3)
    H = W.tfim(n)
    gs = oracle.grad_param_shift(circ, theta, H)
    gf = oracle.grad_fd(circ, theta, H, h=1e-4)
    assert np.max(np.abs(gs - gf)) / np.max(np.abs(gs)) < 1e-7
    lc, lth = W.random_layered(4, 2, 9)
    gs = oracle.grad_param_shift(lc, lth, W.random_pauli_sum(4, 5, 1))
    gf = oracle.grad_fd(lc, lth, W.random_pauli_sum(4, 5, 1), h=1e-4)
    assert np.max(np.abs(gs - gf)) < 1e-7


def test_controlled_rotation_shift_rule_matches_central_difference():
    n = 4
    gates = [W.Gate("H", (0,)), W.Gate("H", (1,)), W.Gate("RX", (2,), (0,), 0),
             W.Gate("RY", (3,), (1, 0), 1), W.Gate("RZ", (1,), (3,), 2),
             W.Gate("RY", (0,), (), 3), W.Gate("X", (2,), (3,))]
    c = W.Circuit(n, gates, 4)
    theta = np.array([0.4, -1.3, 2.2, 0.9])
    H = W.random_pauli_sum(n, 6, 3)
    gs = oracle.grad_param_shift(c, theta, H)
    gf = oracle.grad_fd(c, theta, H, h=1e-4)
    assert np.max(np.abs(gs - gf)) < 1e-7
    # the two-term rule alone is not exact for a controlled rotation
    two = 0.5 * (oracle.energy(c, theta, H, None, 2, math.pi / 2)
                 - oracle.energy(c, theta, H, None, 2, -math.pi / 2))
    assert abs(two - gs[0]) > 1e-4


def test_threads_do_not_change_results():
    if not oracle.have_openmp():
        pytest.skip("oracle built without OpenMP")
    circ, theta = W.random_layered(15, 2, 3)
    oracle.set_threads(1)
    a = oracle.run(circ, theta)
    oracle.set_threads(4)
    try:
        b = oracle.run(circ, theta)
    finally:
        oracle.set_threads(1)
    assert np.array_equal(a, b)


# --------------------------------------------------------------------------
def _pin_battery() -> bool:
    """True if every pin in a quick battery passes."""
    try:
        test_eq1_against_bruteforce_kronecker(4, 4)
        test_every_target_order_and_width()
        test_rotation_closed_forms()
        test_expval_against_dense_pauli_operator(4, 2)
        test_norm_and_dot_pairwise_exact_cases()
        for b in load_golden():
            test_golden_worked_examples(b)
    except AssertionError:
        return False
    return True


@pytest.mark.parametrize("mutant", [1, 2, 3, 4, 5, 6])
def test_pins_catch_planted_mistakes(mutant):
    """1: G transposed; 2: controls act on the wrong subspace; 3: tau bit
    order reversed; 4: RX sign flipped; 5: a term dropped from the sum;
    6: Y sign flipped."""
    assert _pin_battery()
    oracle.set_mutant(mutant)
    try:
        assert not _pin_battery()
    finally:
        oracle.set_mutant(0)
    assert _pin_battery()


# --------------------------------------------------------------------------
# measurement (Sec. 3: sampling of measurements)
def test_probabilities_against_numpy_marginals():
    n = 7
    psi = W.random_state(n, 31)
    p = np.abs(psi.reshape([2] * n)) ** 2          # axis q <-> qubit q (qubit 0 = MSB)
    for qubits in ([0], [6], [2, 5], [5, 2], [0, 3, 6], list(range(n)), [4, 1, 6, 0]):
        rest = tuple(q for q in range(n) if q not in qubits)
        marg = p.sum(axis=rest) if rest else p
        order = sorted(qubits)
        ref = np.transpose(marg, [order.index(q) for q in qubits]).reshape(-1)
        got = oracle.probabilities(psi, qubits)
        assert np.max(np.abs(got - ref)) < 1e-15
    assert abs(oracle.probabilities(psi, [3]).sum() - 1) < 1e-14


def test_probabilities_closed_forms():
    bell = oracle.run(W.Circuit(2, [W.Gate("H", (0,)), W.Gate("X", (1,), (0,))], 0))
    assert np.allclose(oracle.probabilities(bell, [0, 1]), [0.5, 0, 0, 0.5], atol=1e-15)
    # RY(a)|0>: P(1) = sin^2(a/2)
    a = 1.234
    psi = oracle.run(W.Circuit(1, [W.Gate("RY", (0,), (), -1, a)], 0))
    assert abs(oracle.probabilities(psi, [0])[1] - np.sin(a / 2) ** 2) < 1e-15


def test_sampling_against_numpy_searchsorted():
    n = 9
    psi = W.random_state(n, 32)
    u = W.uniform_block(77, 0, 5000)
    cdf = np.cumsum(np.abs(psi) ** 2)
    full = np.searchsorted(cdf, u * cdf[-1], side="right")
    got = oracle.sample(psi, list(range(n)), u)
    assert np.array_equal(got.astype(np.int64), full)
    # a subset is the projection of the full outcome: qubits (5, 0) -> 2 bits
    sub = oracle.sample(psi, [5, 0], u)
    ref = ((full >> (n - 1 - 5)) & 1) * 2 + ((full >> (n - 1 - 0)) & 1)
    assert np.array_equal(sub.astype(np.int64), ref)


def test_sampling_frequencies_follow_probabilities():
    n = 5
    psi = W.random_state(n, 33)
    u = W.uniform_block(78, 0, 200000)
    s = oracle.sample(psi, [1, 3], u).astype(np.int64)
    freq = np.bincount(s, minlength=4) / len(u)
    p = oracle.probabilities(psi, [1, 3])
    assert np.max(np.abs(freq - p)) < 5 * np.sqrt(0.25 / len(u))


def _q120_exact(v: float) -> int:
    """floor(v^2 * 2^120) with Python's exact rationals."""
    from fractions import Fraction
    f = Fraction(v)
    return (f * f * (1 << 120)).__floor__()


def test_exact_sampling_against_python_integers():
    n = 8
    for psi in (W.random_state(n, 34), W.random_state(n, 35).astype(np.complex64).astype(np.complex128)):
        q = [_q120_exact(float(a.real)) + _q120_exact(float(a.imag)) for a in psi]
        cdf = np.cumsum(np.array(q, dtype=object))
        total = int(cdf[-1])
        assert oracle.exact_total(psi) == total
        from fractions import Fraction
        u = list(W.uniform_block(79, 0, 3000)) + [0.0, 0.999999999999, 5e-324, 0.5]
        ref = []
        for uu in u:
            T = (Fraction(float(uu)) * total).__floor__()
            ref.append(next(i for i, c in enumerate(cdf) if c > T))
        got = oracle.sample_exact(psi, list(range(n)), u)
        assert got.astype(np.int64).tolist() == ref
    # small and large magnitudes: exact squares across the exponent range
    for v in (1.0, 0.5, 2.0 ** -60, 3.0e-20, 0.7071067811865476, 1.9999999999999998):
        psi = np.zeros(2, np.complex128)
        psi[0] = v
        assert oracle.exact_total(psi) == _q120_exact(v)


# --------------------------------------------------------------------------
# Pauli rotations and Trotter evolution (Sec. 3: time evolution, Trotter)
def test_pauli_rotation_against_expm():
    n = 5
    rng = W.SplitMix64(5)
    psi = W.random_state(n, 40)
    for c, ops in W.random_pauli_sum(n, 12, 41):
        if not ops:
            continue
        a = 2 * np.pi * rng.uniform() - np.pi
        P = pauli_operator(n, [(1.0, ops)])
        ref = scipy.linalg.expm(-1j * a * P) @ psi
        assert np.max(np.abs(oracle.pauli_rotation(psi, ops, a) - ref)) < 1e-13
    # single-qubit cases are the rotation gates: exp(-i a X) = RX(2a)
    ref = oracle.run(W.Circuit(n, [W.Gate("RX", (2,), (), -1, 1.1)], 0), None, psi)
    assert np.max(np.abs(oracle.pauli_rotation(psi, ((2, "X"),), 0.55) - ref)) < 1e-14


def test_trotter_exact_for_commuting_terms_and_converges_otherwise():
    n = 4
    psi = W.random_state(n, 42)
    zz = [(0.8, ((i, "Z"), (i + 1, "Z"))) for i in range(n - 1)] + [(0.3, ((1, "Z"),))]
    ref = scipy.linalg.expm(-1j * 0.9 * pauli_operator(n, zz)) @ psi
    assert np.max(np.abs(oracle.trotter(psi, zz, 0.9, 3) - ref)) < 1e-13
    H = W.tfim(n)
    ref = scipy.linalg.expm(-1j * 0.7 * pauli_operator(n, H)) @ psi
    e1 = [np.linalg.norm(oracle.trotter(psi, H, 0.7, s, 1) - ref) for s in (8, 16)]
    e2 = [np.linalg.norm(oracle.trotter(psi, H, 0.7, s, 2) - ref) for s in (8, 16)]
    assert 1.8 < e1[0] / e1[1] < 2.2      # first order: error ~ dt
    assert 3.6 < e2[0] / e2[1] < 4.4      # second order: error ~ dt^2


# --------------------------------------------------------------------------
# Grover search (Sec. 3: Grover's algorithm) and many-control gates
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_grover_success_probability_closed_form(n):
    N = 1 << n
    th = math.asin(1 / math.sqrt(N))
    marked = (0x5A5A5A >> (24 - n)) & (N - 1)
    for k in range(0, 4):
        psi = oracle.run(W.grover(n, marked, k))
        p = np.abs(psi) ** 2
        assert abs(p[marked] - math.sin((2 * k + 1) * th) ** 2) < 1e-12
        if N > 1:
            others = np.delete(p, marked)
            assert np.max(np.abs(others - math.cos((2 * k + 1) * th) ** 2 / (N - 1))) < 1e-12


def test_many_controls_against_bruteforce():
    n = 7
    psi = W.random_state(n, 44)
    g = W.Gate("Z", (6,), tuple(range(6)))
    ref = full_operator(n, g.targets, g.controls, PAULI["Z"]) @ psi
    assert np.max(np.abs(oracle.run(W.Circuit(n, [g], 0), None, psi) - ref)) < 1e-15


# ---- PAULI gates and QAOA (Sec. 3: QAOA, MaxCut) -----------------------------
def _pauli_string_matrix(letters) -> np.ndarray:
    P = np.ones((1, 1), np.complex128)
    for L in letters:
        P = np.kron(P, PAULI[L])
    return P


@pytest.mark.parametrize("n,seed", [(2, 21), (4, 22), (6, 23), (8, 24)])
def test_pauli_gate_against_expm_of_the_string(n, seed):
    """PAULI(a) on targets t_0.. with letters L_0..: expm(-i a/2 P) of the
    Kronecker product of the letters (t_0 most significant), placed by the
    brute-force operator builder."""
    circ, theta = W.random_gates(n, 30, seed, max_tar=min(5, n), kinds=("PAULI", "H", "RY"))
    assert any(g.kind == "PAULI" and len(g.targets) > 1 for g in circ.gates)
    psi = W.random_state(n, 200 + seed)
    for g in circ.gates:
        if g.kind == "PAULI":
            a = theta[g.param]
            G = scipy.linalg.expm(-0.5j * a * _pauli_string_matrix(g.paulis))
        else:
            G = textbook_matrix(g, theta)
        ref = full_operator(n, g.targets, g.controls, G) @ psi
        got = oracle.run(_single(circ, g), theta, psi)
        assert np.max(np.abs(got - ref)) < 1e-13, g
        psi = got


def test_pauli_gate_shift_rule_matches_central_difference():
    n = 6
    circ, theta = W.random_gates(n, 24, 31, max_tar=4, kinds=("PAULI", "RX", "H"))
    terms = W.random_pauli_sum(n, 6, 32)
    ps = [i for i, g in enumerate(circ.gates) if g.kind == "PAULI"]
    params = sorted({circ.gates[i].param for i in ps})[:5]
    g_ps = oracle.grad_param_shift(circ, theta, terms, params=params)
    g_fd = oracle.grad_fd(circ, theta, terms, h=1e-4, params=params)
    assert np.max(np.abs(g_ps[params] - g_fd[params])) < 1e-7


def _qaoa_p1_edge(gamma, beta, du, dv, lam):
    """<C_uv> after one QAOA layer, C_uv = (1 - Z_u Z_v) / 2, for vertices of
    degrees du, dv with lam common neighbours (Wang, Hadfield, Jiang, Rieffel,
    Phys. Rev. A 97, 022304 (2018), Theorem 1)."""
    s4b, s2b = math.sin(4 * beta), math.sin(2 * beta)
    cg = math.cos(gamma)
    return (0.5 + 0.25 * s4b * math.sin(gamma) * (cg ** (du - 1) + cg ** (dv - 1))
            - 0.25 * s2b ** 2 * cg ** (du + dv - 2 - 2 * lam) * (1 - math.cos(2 * gamma) ** lam))


@pytest.mark.parametrize("graph", ["ring7", "reg3_n8", "reg3_n10", "reg4_n9"])
def test_qaoa_p1_energy_closed_form(graph):
    """One QAOA layer on MaxCut: the oracle's <C> equals the published closed
    form, summed over edges (degrees and common neighbours per edge), for
    graphs with and without triangles.  The circuit's angles are
    (-gamma, 2 beta) for Farhi et al.'s exp(-i gamma C), exp(-i beta B)."""
    if graph == "ring7":
        n, edges = 7, W.ring_graph(7)
    else:
        d, n = (int(graph[3]), int(graph.split("_n")[1]))
        edges = W.random_regular_graph(n, d, 40 + n)
    adj = {v: set() for v in range(n)}
    for i, j in edges:
        adj[i].add(j)
        adj[j].add(i)
    c, _ = W.qaoa(n, edges, 1, 1)
    for gamma, beta in ((0.37, 0.91), (1.3, -0.25), (2.9, 2.2)):
        psi = oracle.run(c, np.array([-gamma, 2 * beta]))
        F = oracle.expval(psi, W.maxcut(edges))
        ref = sum(_qaoa_p1_edge(gamma, beta, len(adj[i]), len(adj[j]), len(adj[i] & adj[j]))
                  for i, j in edges)
        assert abs(F - ref) < 1e-12, (graph, gamma, beta, F, ref)
