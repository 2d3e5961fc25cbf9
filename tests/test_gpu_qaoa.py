"""QAOA on the gradient path (Sec. 3: pre-coded MaxCut Hamiltonian and QAOA
models): PAULI gates exp(-i a P / 2) on Pauli strings against the oracle,
MaxCut energies against the oracle and the published p = 1 closed form, and
adjoint gradients (unfused, fused, checkpointed, through torch.autograd)
against the oracle's exact two-term shift rule (P^2 = I)."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import TOL, gpu_run, max_err, oracle_threads, rounded

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DTYPES = ["c64", "c128"]
GRAD_TOL = {"c64": 1e-5, "c128": 1e-10}


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle_threads()


def _rel(g, ref):
    return float(np.max(np.abs(g - ref)) / max(np.max(np.abs(ref)), 1e-300))


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [2, 5, 11, 14])
@pytest.mark.parametrize("fuse_k", [0, 4])
def test_pauli_gates_against_oracle(dtype, n, fuse_k):
    c, theta = W.random_gates(n, 60, 500 + n, max_tar=min(5, n), max_ctrl=2,
                              kinds=("PAULI", "PAULI", "H", "RX", "U1", "Z"))
    assert any(g.kind == "PAULI" and len(g.targets) > 1 for g in c.gates) or n < 3
    psi = rounded(W.random_state(n, 510 + n), dtype)
    got = gpu_run(c, theta, psi, dtype, fuse_k=fuse_k)
    assert max_err(got, oracle.run(c, theta, psi)) <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
def test_qaoa_ring_energy_closed_form(dtype):
    """p = 1 on the 16-cycle: <C> = n (1/2 + sin(4 beta) sin(2 gamma) / 4)."""
    from paper_2202_07017_gb300 import State
    n = 16
    edges = W.ring_graph(n)
    c, _ = W.qaoa(n, edges, 1, 1)
    for gamma, beta in ((0.4, 0.3), (1.7, -0.9)):
        st = State(n, dtype).init(0)
        try:
            st.apply_circuit(c, np.array([-gamma, 2 * beta]))
            F = st.expval(W.maxcut(edges))
        finally:
            st.close()
        ref = n * (0.5 + 0.25 * math.sin(4 * beta) * math.sin(2 * gamma))
        assert abs(F - ref) <= TOL[dtype] * (len(edges) + 1)


def _qaoa_case(n, p, seed):
    edges = W.random_regular_graph(n, 3, seed)
    c, theta = W.qaoa(n, edges, p, seed)
    return c, theta, W.maxcut(edges)


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("fuse_k", [0, 4])
def test_qaoa_gradient_against_shift_rule(dtype, fuse_k):
    from paper_2202_07017_gb300 import State
    n = 12
    c, theta, H = _qaoa_case(n, 3, 71)
    st = State(n, dtype, guarded=True).init(0)
    try:
        e, g = st.grad(c, theta, H, [], fuse_k=fuse_k)
        st.check_guards()
        final = st.numpy()
    finally:
        st.close()
    scale = sum(abs(t[0]) for t in H)
    assert max_err(final, oracle.run(c, theta)) <= TOL[dtype]
    assert abs(e - oracle.energy(c, theta, H)) <= TOL[dtype] * scale
    assert _rel(g, oracle.grad_param_shift(c, theta, H)) <= GRAD_TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
def test_random_pauli_circuit_gradients(dtype):
    """Random strings on 1..5 targets (X, Y, Z letters), mixed with
    controlled rotations: every parameter against the shift rules."""
    from paper_2202_07017_gb300 import State
    n = 11
    c, theta = W.random_gates(n, 50, 77, max_tar=5, max_ctrl=2,
                              kinds=("PAULI", "RY", "RZ", "H", "Z"))
    terms = W.random_pauli_sum(n, 10, 78)
    psi0 = rounded(W.random_state(n, 79), dtype)
    for fuse_k in (0, 4):
        st = State(n, dtype).load(psi0)
        try:
            e, g = st.grad(c, theta, terms, [], fuse_k=fuse_k)
        finally:
            st.close()
        assert abs(e - oracle.energy(c, theta, terms, psi0)) <= TOL[dtype] * sum(
            abs(t[0]) for t in terms)
        assert _rel(g, oracle.grad_param_shift(c, theta, terms, psi0=psi0)) <= GRAD_TOL[dtype]


def test_qaoa_n16_checkpointed_gradient():
    """n = 16, p = 4 on a 3-regular graph (complex64), checkpoints before
    layers 2 and 3: energy and all 8 gradients against the oracle."""
    from paper_2202_07017_gb300 import State
    n = 16
    c, theta, H = _qaoa_case(n, 4, 73)
    per_layer = (len(c.gates) - n) // 4
    ck = [n + per_layer, n + 2 * per_layer]
    ref_e = oracle.energy(c, theta, H)
    ref_g = oracle.grad_param_shift(c, theta, H)
    for fuse_k in (0, 4):
        st = State(n, "c64").init(0)
        try:
            e, g = st.grad(c, theta, H, ck, fuse_k=fuse_k)
        finally:
            st.close()
        assert abs(e - ref_e) <= 1e-5 * (len(H))
        assert _rel(g, ref_g) <= GRAD_TOL["c64"]


def test_qaoa_through_torch_autograd():
    """The energy as a torch function of (gamma, beta): the circuit angles
    are (-gamma_l, 2 beta_l), the adjoint gradient flows back through that
    map, and the result matches the oracle's shift rule under the same
    chain rule."""
    from paper_2202_07017_gb300 import State, energy
    n = 14
    c, theta0, H = _qaoa_case(n, 2, 75)
    gb = torch.tensor(theta0, dtype=torch.float64, requires_grad=True)  # (gamma, beta) pairs
    scale = torch.tensor([-1.0, 2.0] * 2, dtype=torch.float64)
    st = State(n, "c64")
    try:
        E = energy(gb * scale, st, c, H)
        E.backward()
    finally:
        st.close()
    th = (theta0 * np.array([-1.0, 2.0] * 2))
    assert abs(E.item() - oracle.energy(c, th, H)) <= 1e-5 * len(H)
    ref = oracle.grad_param_shift(c, th, H) * np.array([-1.0, 2.0] * 2)
    assert _rel(gb.grad.numpy(), ref) <= GRAD_TOL["c64"]


def test_pauli_gate_rejects_bad_records():
    from paper_2202_07017_gb300 import State, SvError
    st = State(4, "c64").init(0)
    try:
        bad = W.Circuit(4, [W.Gate("PAULI", (0, 1), (), -1, 0.3, paulis="ZX")], 0)
        object.__setattr__(bad.gates[0], "controls", (2,))  # controls are not allowed
        with pytest.raises(SvError):
            st.apply_circuit(bad)
    finally:
        st.close()
