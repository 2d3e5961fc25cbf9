"""GPU parity of Pauli-string rotations exp(-i a P) and Trotter products
(Sec. 3: time evolution with the Trotter decomposition) against the oracle;
for commuting ZZ terms at n = 28 the product is exact and every sampled
amplitude has a closed form."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import TOL, max_err, rounded

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _state(n, dtype, psi):
    from paper_2202_07017_gb300 import State
    return State(n, dtype).load(np.asarray(psi))


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n", [1, 3, 9, 14])
def test_pauli_rotations(dtype, n):
    psi = rounded(W.random_state(n, 80 + n), dtype)
    rng = W.SplitMix64(n)
    terms = [t for t in W.random_pauli_sum(n, 20, 90 + n) if t[1]]
    terms += [(1.0, ((0, "Z"),)), (1.0, ((n - 1, "X"),)), (1.0, ((n // 2, "Y"),))]
    st = _state(n, dtype, psi)
    ref = psi.copy()
    try:
        for _, ops in terms:
            a = 4 * rng.uniform() - 2
            st.pauli_rotation(ops, a)
            ref = oracle.pauli_rotation(ref, ops, a)
        got = st.numpy()
    finally:
        st.close()
    assert max_err(got, ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("order", [1, 2])
def test_trotter_tfim_and_random(dtype, order):
    n = 10
    psi = rounded(W.random_state(n, 85), dtype)
    for H in (W.tfim(n), W.random_pauli_sum(n, 15, 86) + [(0.4, ((2, "Z"), (5, "Z")))]):
        st = _state(n, dtype, psi)
        try:
            st.trotter(H, 0.8, 6, order)
            got = st.numpy()
        finally:
            st.close()
        ref = oracle.trotter(psi, H, 0.8, 6, order)
        assert max_err(got, ref) <= TOL[dtype]


def test_trotter_commuting_zz_n28_closed_form():
    """H = sum_i J_i Z_i Z_{i+1} + h_i Z_i on n = 28 (complex64): diagonal,
    so exp(-i t H)|+...+> has amplitudes 2^-14 exp(-i t E(x)) exactly;
    sampled amplitudes against E(x) computed in fp64 on the host."""
    from paper_2202_07017_gb300 import State
    n, t = 28, 0.37
    J = np.linspace(0.3, 1.1, n - 1)
    hz = np.linspace(-0.5, 0.5, n)
    H = [(float(J[i]), ((i, "Z"), (i + 1, "Z"))) for i in range(n - 1)]
    H += [(float(hz[i]), ((i, "Z"),)) for i in range(n)]
    st = State(n, "c64")
    try:
        st.init(0)
        st.apply_circuit(W.Circuit(n, [W.Gate("H", (q,)) for q in range(n)], 0), None)
        st.trotter(H, t, 3, 2)
        nrm = st.norm()
        rs = np.random.default_rng(2)
        idx = np.unique(np.concatenate([[0, (1 << n) - 1], rs.integers(0, 1 << n, 4096)]))
        assert idx.max() < (1 << n)
        got = st.tensor[torch.from_numpy(idx.astype(np.int64)).to(st.tensor.device)].cpu().numpy()
    finally:
        st.close()
    bits = ((idx[:, None] >> (n - 1 - np.arange(n))[None, :]) & 1).astype(np.float64)
    z = 1 - 2 * bits                                   # Z eigenvalue per qubit
    E = (z[:, :-1] * z[:, 1:]) @ J + z @ hz
    ref = np.exp(-1j * t * E) / 2 ** (n / 2)
    assert max_err(got, ref) <= 1e-5
    assert abs(1 - nrm) <= 1e-5


def test_rotation_rejects_bad_arguments():
    from paper_2202_07017_gb300 import State, SvError
    st = State(3, "c64").init(0)
    try:
        with pytest.raises(SvError):
            st.pauli_rotation(((3, "X"),), 0.1)
        with pytest.raises(SvError):
            st.pauli_rotation(((0, "X"),), float("nan"))
        with pytest.raises(SvError):
            st.trotter(W.tfim(3), 1.0, 0)
    finally:
        st.close()
