"""GPU parity of the fused adjoint gradient (sv_grad_fused: forward circuit
and reverse sweep as qubit-block passes over psi and lambda, each
parameterised gate's Im<lambda|P|psi> accumulated in its pass before the gate
is un-applied) against the oracle's exact parameter-shift gradient and
against the unfused sweep, with and without forward checkpoints."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import TOL, max_err, oracle_threads, rounded

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DTYPES = ["c64", "c128"]
GRAD_TOL = {"c64": 1e-5, "c128": 1e-10}


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle_threads()


def _rel(g, ref):
    return float(np.max(np.abs(g - ref)) / max(np.max(np.abs(ref)), 1e-300))


def _grad(c, theta, terms, dtype, psi0=None, checkpoints=(), fuse_k=4, profile=False):
    from paper_2202_07017_gb300 import State, sv_profile_start, sv_profile_stop
    st = State(c.n_qubits, dtype, guarded=True)
    try:
        if psi0 is None:
            st.init(0)
        else:
            st.load(np.asarray(psi0))
        if profile:
            sv_profile_start()
        e, g = st.grad(c, theta, terms, list(checkpoints), fuse_k=fuse_k)
        prof = sv_profile_stop() if profile else {}
        st.check_guards()  # state and both work states
        return e, g, st.numpy(), prof
    finally:
        st.close()


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("fuse_k", [3, 4])
@pytest.mark.parametrize("n,seed", [(11, 1), (13, 2)])
def test_fused_grad_random_circuits_vs_parameter_shift(dtype, fuse_k, n, seed):
    kinds = ("H", "X", "Y", "Z", "RX", "RY", "RZ", "U1", "SWAP", "MATRIX")
    c, theta = W.random_gates(n, 60, 900 + seed, max_tar=3, max_ctrl=2, kinds=kinds)
    terms = W.random_pauli_sum(n, 8, seed)
    psi0 = rounded(W.random_state(n, seed), dtype)
    e, g, final, prof = _grad(c, theta, terms, dtype, psi0, fuse_k=fuse_k, profile=True)
    assert f"kfused_adj_{dtype}" in prof, prof
    assert max_err(final, oracle.run(c, theta, psi0)) <= TOL[dtype]
    assert abs(e - oracle.energy(c, theta, terms, psi0)) <= TOL[dtype] * sum(abs(t[0]) for t in terms)
    assert c.n_params > 0
    assert _rel(g, oracle.grad_param_shift(c, theta, terms, psi0=psi0)) <= GRAD_TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("fuse_k", [3, 4])
def test_fused_grad_rotation_runs(dtype, fuse_k):
    """Runs of six rotations per qubit (two shared evaluations of up to four
    gradients each), a controlled rotation and a phase on some qubits between
    runs (no sharing across them), CZ bricks between layers."""
    n = 11
    gates, p = [], 0
    for layer in range(3):
        for q in range(n):
            for kind in ("RX", "RY", "RZ", "RX", "RY", "RZ"):
                gates.append(W.Gate(kind, (q,), (), p))
                p += 1
            if q % 4 == 1:
                gates.append(W.Gate("RY", (q,), ((q + 3) % n,), p))
                p += 1
                gates.append(W.Gate("RZ", (q,), (), p))
                p += 1
            if q % 4 == 2:
                gates.append(W.Gate("U1", (q,), (), -1, 0.3))
                gates.append(W.Gate("RX", (q,), (), p))
                p += 1
        for q in range(layer % 2, n - 1, 2):
            gates.append(W.Gate("Z", (q + 1,), (q,)))
    c = W.Circuit(n, gates, p)
    theta = np.array([W.SplitMix64(77 + i).angle() for i in range(p)])
    terms = W.tfim(n)
    psi0 = rounded(W.random_state(n, 5), dtype)
    e, g, _, prof = _grad(c, theta, terms, dtype, psi0, fuse_k=fuse_k, profile=True)
    assert f"kfused_adj_{dtype}" in prof, prof
    assert abs(e - oracle.energy(c, theta, terms, psi0)) <= TOL[dtype] * sum(abs(t[0]) for t in terms)
    assert _rel(g, oracle.grad_param_shift(c, theta, terms, psi0=psi0)) <= GRAD_TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
def test_fused_grad_shared_parameters_and_controls(dtype):
    """Parameters shared by several gates (gradients summed) and rotations
    with controls (the generator acts on the control subspace only)."""
    n = 12
    gates = []
    for layer in range(3):
        for q in range(n):
            gates.append(W.Gate("RY", (q,), (), q % 5))
        for q in range(0, n - 1, 2):
            gates.append(W.Gate("RX", (q + 1,), (q,), 5 + layer))
        gates.append(W.Gate("RZ", (0,), (3, 7), 8))
        gates.append(W.Gate("U1", (2,), (9,), -1, 0.4))
    c = W.Circuit(n, gates, 9)
    theta = np.array([W.SplitMix64(55 + i).angle() for i in range(9)])
    terms = W.tfim(n)
    e, g, _, prof = _grad(c, theta, terms, dtype, profile=True)
    assert f"kfused_adj_{dtype}" in prof, prof
    assert abs(e - oracle.energy(c, theta, terms)) <= TOL[dtype] * sum(abs(t[0]) for t in terms)
    assert _rel(g, oracle.grad_param_shift(c, theta, terms)) <= GRAD_TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
def test_fused_grad_checkpoints_match_unfused(dtype):
    """Random layered circuit n = 14, depth 12, checkpoints every 3 layers:
    fused and unfused sweeps give the same energy, gradient and final state."""
    n, depth = 14, 12
    c, theta = W.random_layered(n, depth, 77)
    starts = [i for i, gt in enumerate(c.gates) if gt.kind == "RX" and gt.targets == (0,)]
    ck = [starts[3], starts[6], starts[9]]
    terms = W.sum_z(n)
    e1, g1, s1, _ = _grad(c, theta, terms, dtype, checkpoints=ck, fuse_k=4)
    e0, g0, s0, _ = _grad(c, theta, terms, dtype, checkpoints=ck, fuse_k=0)
    ref_state = oracle.run(c, theta)
    assert max_err(s1, ref_state) <= TOL[dtype]
    assert max_err(s0, ref_state) <= TOL[dtype]
    assert abs(e1 - e0) <= TOL[dtype] * n
    assert _rel(g1, g0) <= 2 * GRAD_TOL[dtype]
    ps = [0, c.n_params // 3, c.n_params - 1]
    ref = oracle.grad_param_shift(c, theta, terms, params=ps)
    assert np.max(np.abs(g1[ps] - ref[ps])) <= GRAD_TOL[dtype] * max(1.0, np.max(np.abs(ref[ps])))


def test_fused_grad_hea20_against_unfused_and_shift_rule():
    """Hardware-efficient ansatz n = 20, L = 10 (200 parameters), TFIM,
    complex64: fused against the unfused sweep and sampled shift-rule
    gradients."""
    n = 20
    c, theta = W.hea(n, 10, 1002)
    terms = W.tfim(n)
    e1, g1, _, prof = _grad(c, theta, terms, "c64", profile=True)
    e0, g0, _, _ = _grad(c, theta, terms, "c64", fuse_k=0)
    assert "kfused_adj_c64" in prof
    assert abs(e1 - e0) <= 1e-5 * sum(abs(t[0]) for t in terms)
    assert _rel(g1, g0) <= 2e-5
    sample = [0, 57, 133, 199]
    ref = oracle.grad_param_shift(c, theta, terms, params=sample)
    assert np.max(np.abs(g1[sample] - ref[sample])) <= 1e-5 * max(1.0, np.max(np.abs(ref[sample])))


def test_fused_grad_layered_n28_checkpointed():
    """Random layered circuit n = 28, depth 40 (3900 gates, 3360 parameters),
    <sum Z_i>, checkpoints every 10 layers: fused and unfused checkpointed
    sweeps agree (complex64)."""
    n = 28
    c, theta = W.random_layered(n, 40, 1004)
    starts = [i for i, gt in enumerate(c.gates) if gt.kind == "RX" and gt.targets == (0,)]
    ck = [starts[10], starts[20], starts[30]]
    terms = W.sum_z(n)
    e1, g1, _, prof = _grad(c, theta, terms, "c64", checkpoints=ck, profile=True)
    e0, g0, _, _ = _grad(c, theta, terms, "c64", checkpoints=ck, fuse_k=0)
    assert "kfused_adj_c64" in prof
    assert abs(e1 - e0) <= 1e-5 * n
    assert np.max(np.abs(g1 - g0)) <= 1e-4 * max(1e-3, np.max(np.abs(g0)))


@pytest.mark.parametrize("dtype", DTYPES)
def test_fused_grad_small_states_use_unfused_sweep(dtype):
    """Below 10 qubits sv_grad_fused takes the unfused reverse sweep: no
    reverse-pass kernel runs and the result equals sv_grad's."""
    n = 7
    c, theta = W.random_layered(n, 6, 31)
    terms = W.tfim(n)
    e1, g1, s1, prof = _grad(c, theta, terms, dtype, profile=True)
    e0, g0, s0, _ = _grad(c, theta, terms, dtype, fuse_k=0)
    assert not any(k.startswith("kfused_adj") for k in prof), prof
    assert abs(e1 - e0) <= TOL[dtype] * n
    assert _rel(g1, g0) <= GRAD_TOL[dtype]
    ref_state = oracle.run(c, theta)  # the forward itself is fused
    assert max_err(s1, ref_state) <= TOL[dtype] and max_err(s0, ref_state) <= TOL[dtype]


def test_fused_grad_rejects_bad_group_width():
    from paper_2202_07017_gb300 import State, SvError
    c, theta = W.hea(4, 1, 3)
    st = State(4, "c64").init(0)
    try:
        with pytest.raises(SvError):
            st.grad(c, theta, W.tfim(4), [], fuse_k=1)
        with pytest.raises(SvError):
            st.grad(c, theta, W.tfim(4), [], fuse_k=6)
    finally:
        st.close()


@pytest.mark.parametrize("dtype", DTYPES)
def test_fused_grad_more_gradients_than_one_pass_holds(dtype):
    """400 rotations on 12 qubits with nothing else between them: the reverse
    sweep needs several passes of at most 200 gradient slots; sampled
    entries against the oracle's shift rule."""
    n = 12
    gates, p = [], 0
    for rep in range(400 // n + 1):
        for q in range(n):
            if p == 400:
                break
            gates.append(W.Gate(("RX", "RY", "RZ")[rep % 3], (q,), (), p))
            p += 1
        if rep % 7 == 6:
            for q in range(0, n - 1, 2):
                gates.append(W.Gate("Z", (q + 1,), (q,)))
    c = W.Circuit(n, gates, p)
    theta = np.array([W.SplitMix64(313 + i).angle() for i in range(p)])
    terms = W.tfim(n)
    psi0 = rounded(W.random_state(n, 11), dtype)
    e, g, _, prof = _grad(c, theta, terms, dtype, psi0, profile=True)
    assert f"kfused_adj_{dtype}" in prof, prof
    sample = list(range(0, p, 10)) + [p - 1]
    ref = oracle.grad_param_shift(c, theta, terms, params=sample, psi0=psi0)
    assert abs(e - oracle.energy(c, theta, terms, psi0)) <= TOL[dtype] * sum(abs(t[0]) for t in terms)
    assert _rel(g[sample], ref[sample]) <= GRAD_TOL[dtype]
