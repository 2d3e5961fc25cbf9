"""Pauli-sum energies of states of 16 qubits and more: the diagonal terms in
one streaming read (per register tile a Walsh-Hadamard transform of |psi|^2,
signs split over tile, thread and iteration bits), the other terms in
staged passes (the state read in shared-memory slices, terms with x bits
inside one tile pairing registers); terms that fit no pass fall back to the
per-amplitude kernel.  Against the oracle's <psi|H|psi> on random
states and Pauli sums of every shape, and against the closed form of a
product state at n = 30 and n = 33 (transverse-field Ising chain: three and
four passes)."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import TOL, oracle_threads, rounded

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle_threads()


def _terms_of_every_shape(n, seed):
    rng = W.SplitMix64(seed)
    terms = list(W.tfim(n))                                  # ZZ + X on every bit
    terms += [(0.3, ((i, "Y"), (i + 1, "Y"))) for i in range(0, n - 1, 3)]   # YY neighbours
    terms += [(0.2, ((i, "X"), ((i + 7) % n, "Z"))) for i in range(0, n, 5)]  # X with a far Z
    terms += [(-0.4, ((0, "X"), (n - 1, "X")))]             # x bits far apart
    terms += [(0.25, tuple((q, "X") for q in range(5)))]    # five x bits: per-amplitude kernel
    terms += [(0.5, ())]                                    # identity
    terms += W.random_pauli_sum(n, 12, seed)                 # dense random strings
    for _ in range(10):                                      # 1..3 factors anywhere
        k = 1 + rng.next() % 3
        qs = sorted({int(rng.next() % n) for _ in range(k)})
        terms.append((2 * rng.uniform() - 1, tuple((q, "XYZ"[rng.next() % 3]) for q in qs)))
    return terms


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n", [16, 19, 22])
def test_staged_energy_against_oracle(dtype, n):
    from paper_2202_07017_gb300 import State, sv_profile_start, sv_profile_stop
    psi = rounded(W.random_state(n, 300 + n), dtype)
    terms = _terms_of_every_shape(n, n)
    st = State(n, dtype).load(psi)
    try:
        sv_profile_start()
        e = st.expval(terms)
        prof = sv_profile_stop()
        e2 = st.expval(terms)
    finally:
        st.close()
    assert any(k.startswith("kpauli_energy") for k in prof), prof
    assert e == e2  # fixed reduction order
    scale = sum(abs(c) for c, _ in terms)
    assert abs(e - oracle.expval(psi, terms, n)) <= TOL[dtype] * scale


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_staged_energy_of_many_diagonal_terms(dtype):
    """200 diagonal strings (more than one pass holds) on n = 18."""
    from paper_2202_07017_gb300 import State
    n = 18
    rng = W.SplitMix64(5)
    terms = []
    for _ in range(200):
        qs = sorted({int(rng.next() % n) for _ in range(1 + rng.next() % 4)})
        terms.append((2 * rng.uniform() - 1, tuple((q, "Z") for q in qs)))
    psi = rounded(W.random_state(n, 6), dtype)
    st = State(n, dtype).load(psi)
    try:
        e = st.expval(terms)
    finally:
        st.close()
    assert abs(e - oracle.expval(psi, terms, n)) <= TOL[dtype] * sum(abs(c) for c, _ in terms)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_single_x_terms_take_the_lean_pass(dtype):
    """Only single-X terms (a field on every qubit, some qubits twice with
    other coefficients): every pass is the single-X kernel, and the energy
    matches the oracle's."""
    from paper_2202_07017_gb300 import State, sv_profile_start, sv_profile_stop
    n = 21
    rng = W.SplitMix64(17)
    terms = [(2 * rng.uniform() - 1, ((q, "X"),)) for q in range(n)]
    terms += [(2 * rng.uniform() - 1, ((q, "X"),)) for q in range(0, n, 4)]
    psi = rounded(W.random_state(n, 18), dtype)
    st = State(n, dtype).load(psi)
    try:
        sv_profile_start()
        e = st.expval(terms)
        prof = sv_profile_stop()
    finally:
        st.close()
    assert set(prof) == {f"kpauli_xbits_{dtype}", "kfinish"}, prof
    assert abs(e - oracle.expval(psi, terms, n)) <= TOL[dtype] * sum(abs(c) for c, _ in terms)


@pytest.mark.parametrize("n,x_passes", [(30, 3), (33, 4)])
def test_tfim_and_sum_z_on_a_product_state(n, x_passes):
    """RY(a_q) on every qubit of |0..0> (complex64, n = 30, and n = 33 with
    64-bit amplitude indices): <Z_q> = cos a_q and <X_q> = sin a_q exactly, so
    <sum Z> and the transverse-field Ising energy have closed forms; the
    chain's X terms need three passes at n = 30 and four at n = 33."""
    from paper_2202_07017_gb300 import State, sv_profile_start, sv_profile_stop
    a = np.array([0.1 + 0.9 * q / n for q in range(n)])
    c = W.Circuit(n, [W.Gate("RY", (q,), (), q) for q in range(n)], n)
    st = State(n, "c64").init(0)
    try:
        st.apply_circuit(c, a)
        sv_profile_start()
        ez = st.expval(W.sum_z(n))
        et = st.expval(W.tfim(n))
        prof = sv_profile_stop()
    finally:
        st.close()
    cz, sx = np.cos(a), np.sin(a)
    assert abs(ez - cz.sum()) <= TOL["c64"] * n
    ref = float(np.sum(cz[:-1] * cz[1:]) + 0.7 * sx.sum())
    assert abs(et - ref) <= TOL["c64"] * (n - 1 + 0.7 * n)
    # diagonal terms: one streaming read per call; the chain's X terms:
    # passes of the single-X kernel
    assert prof["kdiag_energy_c64"][0] == 2 and prof["kpauli_xbits_c64"][0] == x_passes, prof
    assert "kexpval" not in prof, prof
