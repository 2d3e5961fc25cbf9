"""Complex64 coefficient rounding does not bias the norm (the complex64 bar
|1 - ||psi||^2| <= 1e-5 for complex64, reached with no renormalisation).

fp32 rounds 1/sqrt2 to h with 2h^2 = 1 - 3.4e-8, so a rounded Hadamard
scales ||psi||^2 by exactly that factor on every state; an off-diagonal
Pauli rotation c I - i s P rounded scales it by c'^2 + s'^2 on every state.  Without
correction, N such gates move the norm by N times the factor's error.  The
library rounds every inexact matrix that acts on the whole state with error
feedback (the accumulated factor, kept per state, scales the next matrix
before it is rounded), so these long circuits keep |1 - ||psi||^2| within the
complex64 bar of 1e-5 - what remains is the rounding of the arithmetic
itself - while each amplitude still matches the oracle."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import TOL, max_err, oracle_threads, rounded

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle_threads()


def _hadamard_bricks(n, reps):
    """reps x (H on every qubit, then CZ(i, i+1) for every i)."""
    gates = []
    for _ in range(reps):
        gates += [W.Gate("H", (q,)) for q in range(n)]
        gates += [W.Gate("Z", (i + 1,), (i,)) for i in range(n - 1)]
    return W.Circuit(n, gates, 0)


@pytest.mark.parametrize("fuse_k", [0, 4])
def test_many_hadamards_keep_the_norm(fuse_k):
    """24 000 Hadamards on 12 qubits: a plain fp32 rounding would lose
    24 000 * 3.4e-8 = 8.2e-4 of the norm, 82 times the bar.  The circuit is
    periodic (a Clifford brick), so the arithmetic's own round-to-nearest
    errors also repeat from one period to the next; the fused passes take
    the dithered rounding for it, as long periodic circuits need (unfused
    1-qubit kernels dither by default)."""
    from paper_2202_07017_gb300 import State
    n, reps = 12, 2000
    c = _hadamard_bricks(n, reps)
    psi0 = rounded(W.random_state(n, 61), "c64")
    st = State(n, "c64").load(psi0)
    if fuse_k:
        st.set_rounding("dithered")
    try:
        st.apply_circuit(c, None, fuse_k)
        nrm = st.norm()
        got = st.numpy()
    finally:
        st.close()
    assert abs(1 - nrm) <= TOL["c64"]
    assert max_err(got, oracle.run(c, None, psi0)) <= TOL["c64"]


def _xy_chain(n):
    """0.7 sum X_i + 0.4 sum Y_i Y_(i+1): every term off-diagonal, so every
    exponential is one rounded pair of coefficients (c, s)."""
    return ([(0.7, ((i, "X"),)) for i in range(n)]
            + [(0.4, ((i, "Y"), (i + 1, "Y"))) for i in range(n - 1)])


def test_many_pauli_rotations_keep_the_norm():
    """A Trotter product of 3000 first-order steps on 10 qubits: 57 000
    rotations, each of the same 19 rounded coefficient pairs 3000 times."""
    from paper_2202_07017_gb300 import State
    n = 10
    psi0 = rounded(W.random_state(n, 62), "c64")
    H = _xy_chain(n)
    st = State(n, "c64").load(psi0)
    try:
        st.trotter(H, 1.5, 3000, 1)
        nrm = st.norm()
    finally:
        st.close()
    assert abs(1 - nrm) <= TOL["c64"]


def test_pauli_rotation_sequence_against_oracle():
    """300 second-order steps of the same chain: amplitudes against the
    oracle's product."""
    from paper_2202_07017_gb300 import State
    n = 10
    psi0 = rounded(W.random_state(n, 63), "c64")
    H = _xy_chain(n)
    st = State(n, "c64").load(psi0)
    try:
        st.trotter(H, 0.9, 300, 2)
        got = st.numpy()
        nrm = st.norm()
    finally:
        st.close()
    ref = oracle.trotter(psi0, H, 0.9, 300, 2)
    assert max_err(got, ref) <= TOL["c64"]
    assert abs(1 - nrm) <= TOL["c64"]


def test_feedback_restarts_with_a_new_state():
    """The factor is tracked per state and reset by init and load: the same
    circuit on a fresh state gives bit-identical amplitudes."""
    from paper_2202_07017_gb300 import State
    n = 9
    c = _hadamard_bricks(n, 7)
    st = State(n, "c64")
    try:
        a = st.init(5).apply_circuit(c).numpy()
        st.apply_circuit(c)  # moves the state's factor
        b = st.init(5).apply_circuit(c).numpy()
    finally:
        st.close()
    assert np.array_equal(a, b)
    assert abs(float(np.vdot(a, a).real) - 1) <= TOL["c64"]
