"""GPU parity of the fused qubit-block passes (sv_apply_circuit with fuse_k
>= 2) against the oracle and against the unfused path; the random layered
circuit at n = 33 (64 GiB complex64) checked by running it and its inverse
fused and comparing fused with unfused on its first layers."""
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


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("n", [1, 3, 8, 11, 14, 17])
@pytest.mark.parametrize("k", [2, 4, 5])
def test_fused_random_circuits(dtype, n, k):
    c, theta = W.random_gates(n, 120, 700 + n, max_tar=min(4, n), max_ctrl=min(3, n - 1) if n > 1 else 0)
    psi = rounded(W.random_state(n, n + 1), dtype)
    got = gpu_run(c, theta, psi, dtype, fuse_k=k)
    assert max_err(got, oracle.run(c, theta, psi)) <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("make", [lambda: W.random_layered(20, 12, 5), lambda: W.hea(20, 10, 1002),
                                  lambda: (W.qft(20), np.zeros(0))], ids=["layered", "hea", "qft"])
def test_fused_structured_n20(dtype, make):
    c, theta = make()
    psi = rounded(W.random_state(20, 4), dtype)
    got = gpu_run(c, theta, psi, dtype, fuse_k=4)
    assert max_err(got, oracle.run(c, theta, psi)) <= TOL[dtype]
    unfused = gpu_run(c, theta, psi, dtype, fuse_k=0)
    assert max_err(got, unfused) <= TOL[dtype]


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("max_ctrl", [0, 1])
def test_fused_layer_programs_n22(dtype, max_ctrl):
    """At n = 22 the passes stage 2^13 (complex64) amplitudes: 1-qubit gates of
    every kind (dense unitaries, rotations, H, X, Y with zero diagonals, phases)
    run as layer programs in rotation form - both rotation shapes, register
    relabelling, two sub-blocks per thread - and, with controls, beside gate
    lists in the same pass; against the oracle."""
    n = 22
    c, theta = W.random_gates(n, 160, 2200 + max_ctrl, max_tar=1, max_ctrl=max_ctrl,
                              kinds=("H", "X", "Y", "Z", "RX", "RY", "RZ", "U1", "MATRIX"))
    psi = rounded(W.random_state(n, 23), dtype)
    got = gpu_run(c, theta, psi, dtype, fuse_k=4)
    assert max_err(got, oracle.run(c, theta, psi)) <= TOL[dtype]


def test_fused_layered_n33_inverse_and_unfused_prefix():
    """Random layered circuit, n = 33 (64 GiB complex64), depth 40, fused
    k <= 4: U then U^dagger returns |0...0> (sampled amplitudes and norm);
    the first two layers fused agree with the unfused kernels."""
    from paper_2202_07017_gb300 import State
    n = 33
    c, theta = W.random_layered(n, 40, 1004)
    inv, _ = c.inverse_with(theta)
    st = State(n, "c64")
    try:
        st.init(0)
        st.apply_circuit(c, theta, 4)
        nrm = st.norm()
        st.apply_circuit(inv, None, 4)
        picks = [0, 1, 2, 3, 1 << 20, (1 << n) - 1, 1234567890]
        assert all(0 <= i < (1 << n) for i in picks)  # checked on the host before indexing
        idx = torch.tensor(picks, dtype=torch.int64, device=st.tensor.device)
        amps = st.tensor[idx].cpu().numpy()
        nrm2 = st.norm()
        # first two layers, fused vs unfused, on a random-looking start
        prefix = W.Circuit(n, c.gates[:230], c.n_params)
        st.init(0)
        st.apply_circuit(prefix, theta, 4)
        sample = torch.randint(0, 1 << n, (1 << 20,), generator=torch.Generator().manual_seed(3))
        sample = sample.to(st.tensor.device)
        fused = st.tensor[sample].cpu().numpy()
        st.init(0)
        st.apply_circuit(prefix, theta, 0)
        unfused = st.tensor[sample].cpu().numpy()
    finally:
        st.close()
    ref = np.zeros(len(amps), np.complex128)
    ref[0] = 1.0
    assert abs(1 - nrm) <= 1e-5 and abs(1 - nrm2) <= 1e-5
    assert max_err(amps, ref) <= 1e-5
    assert max_err(fused, unfused) <= 1e-5


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("make", [lambda: W.random_layered(20, 6, 9), lambda: (W.qft(20), np.zeros(0)),
                                  lambda: W.random_gates(16, 150, 77, max_tar=3, max_ctrl=2)],
                         ids=["layered", "qft", "random"])
def test_fused_passes_use_bulk_tensor_staging(dtype, make):
    """At n >= 10 every fused pass is staged by bulk tensor copies (the
    kfused_tma kernels): layer programs for the layered circuit, mixed
    groups for the QFT (its final SWAPs), gate lists for controlled gates;
    results equal the unfused path."""
    from paper_2202_07017_gb300 import State, sv_profile_start, sv_profile_stop
    c, theta = make()
    psi = rounded(W.random_state(c.n_qubits, 31), dtype)
    unfused = gpu_run(c, theta, psi, dtype, fuse_k=0)
    st = State(c.n_qubits, dtype).load(psi)
    try:
        sv_profile_start()
        st.apply_circuit(c, theta, 4)
        prof = sv_profile_stop()
        got = st.numpy()
    finally:
        st.close()
    fused = {k: v for k, v in prof.items() if k.startswith("kfused")}
    assert set(fused) == {f"kfused_tma_{dtype}"}, prof
    assert max_err(got, unfused) <= TOL[dtype]
