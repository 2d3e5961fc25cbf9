"""GPU parity of gate application (Sec. 2, Eq. 1) against the CPU oracle:
every gate kind on every target bit position, control placements including
bit 0 and neighbours, SWAP on every pair, dense 1..5-qubit matrices,
random circuits, the random layered circuit at n = 12 (complex128, full
4096-amplitude output) and the QFT on n = 30 against its closed form."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import TOL, gpu_run, max_err, oracle_threads, rounded

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DTYPES = ["c64", "c128"]


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle_threads()


def _one(n, gate, theta, dtype, seed):
    psi = rounded(W.random_state(n, seed), dtype)
    c = W.Circuit(n, [gate], len(theta))
    got = gpu_run(c, theta, psi, dtype)
    ref = oracle.run(c, theta, psi)
    return max_err(got, ref)


@pytest.mark.parametrize("dtype", DTYPES)
def test_one_qubit_kinds_every_position_and_control(dtype):
    n = 9
    theta = np.array([0.7313, -2.1, 5.9])
    kinds = [("H", -1, 0.0), ("X", -1, 0.0), ("Y", -1, 0.0), ("Z", -1, 0.0),
             ("RX", 0, 0.0), ("RY", 1, 0.0), ("RZ", 2, 0.0), ("U1", -1, 1.234),
             ("U1", -1, math.pi / 2), ("U1", -1, -math.pi / 2), ("U1", -1, math.pi)]
    worst = 0.0
    for q in range(n):
        ctrl_sets = [(), ((q + 1) % n,), ((q + n - 1) % n,), (n - 1,) if q != n - 1 else (0,),
                     tuple(c for c in (n - 1, (q + 3) % n) if c != q)]
        for kind, p, a in kinds:
            for cs in ctrl_sets:
                g = W.Gate(kind, (q,), tuple(sorted(set(cs))), p, a)
                worst = max(worst, _one(n, g, theta, dtype, 31 * q + len(cs)))
    assert worst <= TOL[dtype], worst


@pytest.mark.parametrize("dtype", DTYPES)
def test_swap_every_pair(dtype):
    n = 7
    worst = 0.0
    for a in range(n):
        for b in range(n):
            if a == b:
                continue
            for cs in ((), tuple(c for c in (n - 1,) if c not in (a, b)),
                       tuple(c for c in (0, 3) if c not in (a, b))):
                worst = max(worst, _one(n, W.Gate("SWAP", (a, b), cs), [], dtype, a * 7 + b))
    assert worst <= TOL[dtype], worst


@pytest.mark.parametrize("dtype", DTYPES)
def test_dense_matrices_one_to_five_targets(dtype):
    n = 10
    rng = W.SplitMix64(4242)
    worst = 0.0
    for k in range(1, 6):
        for trial in range(12):
            perm = list(range(n))
            for i in range(n - 1, 0, -1):
                j = rng.next() % (i + 1)
                perm[i], perm[j] = perm[j], perm[i]
            nc = trial % 4
            g = W.Gate("MATRIX", tuple(perm[:k]), tuple(perm[k:k + nc]),
                       matrix=W.random_unitary(k, rng))
            worst = max(worst, _one(n, g, [], dtype, 100 * k + trial))
    # diagonal matrices with a single phase and general diagonals
    g = W.Gate("MATRIX", (3, 6), (), matrix=np.diag([1, 1, 1, np.exp(0.3j)]))
    worst = max(worst, _one(n, g, [], dtype, 7))
    g = W.Gate("MATRIX", (0, 9, 4), (2,), matrix=np.diag(np.exp(1j * np.arange(8))))
    worst = max(worst, _one(n, g, [], dtype, 8))
    assert worst <= TOL[dtype], worst


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 13])
def test_random_circuits(dtype, n):
    c, theta = W.random_gates(n, 60, 900 + n, max_tar=min(5, n), max_ctrl=3)
    psi = rounded(W.random_state(n, n), dtype)
    got = gpu_run(c, theta, psi, dtype)
    ref = oracle.run(c, theta, psi)
    assert max_err(got, ref) <= TOL[dtype]


def test_random_layered_n12_complex128_full_state():
    """Plain random layered circuit, n = 12, depth 20, complex128, from
    |0...0>: all 4096 amplitudes against the oracle."""
    c, theta = W.random_layered(12, 20, 1000)
    got = gpu_run(c, theta, None, "c128")
    ref = oracle.run(c, theta)
    assert max_err(got, ref) <= 1e-12
    assert abs(1 - np.vdot(got, got).real) <= 1e-12


@pytest.mark.parametrize("dtype", DTYPES)
def test_layered_inverse_returns_zero_state(dtype):
    c, theta = W.random_layered(14, 6, 77)
    inv, _ = c.inverse_with(theta)
    full = W.Circuit(14, c.gates + inv.gates, c.n_params)
    got = gpu_run(full, theta, None, dtype)
    ref = np.zeros(1 << 14)
    ref[0] = 1
    assert max_err(got, ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
def test_qft_small_against_oracle(dtype):
    n = 14
    x = W.random_basis_index(n, 1001)
    got = gpu_run(W.qft(n), None, None, dtype, basis=x)
    ref = oracle.run(W.qft(n), None, basis=x)
    assert max_err(got, ref) <= TOL[dtype]


def _qft_closed_form(n, x, idx):
    N = np.uint64(1 << n)
    ph = ((np.uint64(x) * idx.astype(np.uint64)) % N).astype(np.float64) / float(1 << n)
    return np.exp(2j * np.pi * ph) / math.sqrt(1 << n)


@pytest.mark.parametrize("dtype", DTYPES)
def test_qft_n30_closed_form(dtype):
    """QFT on n = 30 qubits (8 GiB complex64 / 16 GiB complex128), one
    kernel per gate, from a seeded basis state: sampled amplitudes against
    exp(2 pi i x y / 2^n) / 2^(n/2), plus the norm."""
    from paper_2202_07017_gb300 import State
    n = 30
    x = W.random_basis_index(n, 1001)
    st = State(n, dtype)
    try:
        st.init(x)
        st.apply_circuit(W.qft(n), None)
        nrm = st.norm()
        N = 1 << n
        rs = np.random.default_rng(5)
        idx = np.unique(np.concatenate([np.arange(4096), np.arange(N - 4096, N),
                                        rs.integers(0, N, 1 << 20)]))
        assert idx.min() >= 0 and idx.max() < N  # checked on the host before indexing
        got =st.tensor[torch.from_numpy(idx.astype(np.int64)).to(st.tensor.device)].cpu().numpy()
    finally:
        st.close()
    ref = _qft_closed_form(n, x, idx)
    assert max_err(got, ref) <= TOL[dtype]
    # relative to the amplitude size 2^-15 the error stays at rounding level
    assert max_err(got, ref) * math.sqrt(N) <= (1e-3 if dtype == "c64" else 1e-10)
    assert abs(1 - nrm) <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
def test_basis_init_and_ghz(dtype):
    from paper_2202_07017_gb300 import State
    for n in (1, 2, 5, 11):
        st = State(n, dtype)
        for x in {0, 1 % (1 << n), (1 << n) - 1, (5 * n) % (1 << n)}:
            st.init(x)
            v = st.numpy()
            ref = np.zeros(1 << n)
            ref[x] = 1
            assert max_err(v, ref) == 0.0
        st.close()
    got = gpu_run(W.ghz(12), None, None, dtype)
    ref = np.zeros(1 << 12)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    assert max_err(got, ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
def test_many_controls_and_empty_circuit(dtype):
    n = 11
    psi = rounded(W.random_state(n, 3), dtype)
    gates = [W.Gate("X", (0,), tuple(range(1, n))), W.Gate("Z", (n - 1,), tuple(range(n - 1))),
             W.Gate("RY", (5,), tuple(q for q in range(n) if q != 5), -1, 0.9),
             W.Gate("SWAP", (0, n - 1), tuple(range(1, n - 1)))]
    c = W.Circuit(n, gates, 0)
    assert max_err(gpu_run(c, None, psi, dtype), oracle.run(c, None, psi)) <= TOL[dtype]
    empty = W.Circuit(n, [], 0)
    assert max_err(gpu_run(empty, None, psi, dtype), psi) == 0.0


def test_invalid_arguments_leave_state_untouched():
    from paper_2202_07017_gb300 import SvError, State
    n = 6
    st = State(n, "c64")
    psi = rounded(W.random_state(n, 1), "c64")
    st.load(psi)
    bad = [((0, 0), (), np.eye(4)), ((6,), (), np.eye(2)), ((1,), (1,), np.eye(2)),
           ((-1,), (), np.eye(2)), (tuple(range(6)), (), np.eye(64))]
    for t, c, m in bad:
        with pytest.raises(SvError) as e:
            st.apply_gate(t, c, m)
        assert e.value.status == 1
    c = W.Circuit(n, [W.Gate("H", (0,)), W.Gate("RX", (9,), (), 0)], 1)
    with pytest.raises(SvError):
        st.apply_circuit(c, [0.1])
    with pytest.raises(SvError):
        st.apply_circuit(W.Circuit(n, [W.Gate("RX", (1,), (), 3)], 1), [0.1])
    with pytest.raises(SvError):
        st.apply_circuit(W.Circuit(n + 1, [], 0), None)
    with pytest.raises(SvError):
        st.expval([(1.0, ((7, "Z"),))])
    assert max_err(st.numpy(), psi) == 0.0
    st.close()
