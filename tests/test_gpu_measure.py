"""GPU parity of measurement (Sec. 3: sampling of measurements): outcome
probabilities of qubit subsets against the oracle, and inverse-CDF samples
for the same uniforms.  Both sides decide outcomes with the exact
fixed-point CDF (q(v) = floor(v^2 2^120), 128-bit integer sums), so the GPU
samples must equal the oracle's exactly; they must also lie on the step of
the oracle's fp64 CDF containing u * total (relative slack 1e-12).  At
n = 30 the QFT's uniform distribution gives a closed form."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import rounded

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _state(n, dtype, psi):
    from paper_2202_07017_gb300 import State
    return State(n, dtype).load(np.asarray(psi))


SUBSETS = [[0], "last", [1, 0], "all", "perm"]


def _subset(spec, n, rng):
    if spec == "last":
        return [n - 1]
    if spec == "all":
        return list(range(n))
    if spec == "perm":
        q = list(range(n))
        rng.shuffle(q)
        return q[:max(1, min(n, 6))]
    return [q for q in spec if q < n] or [0]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n", [1, 5, 12, 20])
def test_probabilities(dtype, n):
    psi = rounded(W.random_state(n, 60 + n), dtype)
    st = _state(n, dtype, psi)
    rng = np.random.default_rng(n)
    try:
        for spec in SUBSETS:
            q = _subset(spec, n, rng)
            if len(q) > 12:
                q = q[:12]
            got = st.probabilities(q)
            ref = oracle.probabilities(psi, q)
            assert np.max(np.abs(got - ref)) <= 1e-12, (spec, q)
            assert np.array_equal(got, st.probabilities(q))   # fixed order
    finally:
        st.close()


def _valid(psi, u, xs):
    """Every sample x lies on the oracle CDF step containing u * total."""
    cdf = np.cumsum(np.abs(psi) ** 2)
    t = u * cdf[-1]
    lo = np.concatenate([[0.0], cdf])[xs]
    hi = cdf[xs]
    slack = 1e-12 * cdf[-1]
    return np.all(lo <= t + slack) and np.all(hi >= t - slack)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n", [1, 4, 11, 16])
def test_sampling_against_oracle_cdf(dtype, n):
    psi = rounded(W.random_state(n, 70 + n), dtype)
    u = W.uniform_block(900 + n, 0, 20000)
    st = _state(n, dtype, psi)
    try:
        full = st.sample(list(range(n)), u).astype(np.int64)
        sub_q = [n - 1, 0] if n > 1 else [0]
        sub = st.sample(sub_q, u).astype(np.int64)
    finally:
        st.close()
    assert _valid(psi, u, full)
    # both sides decide with the exact fixed-point CDF: identical outcomes
    exact = oracle.sample_exact(psi, list(range(n)), u).astype(np.int64)
    assert np.array_equal(full, exact)
    ref = oracle.sample(psi, list(range(n)), u).astype(np.int64)
    assert np.mean(full != ref) <= 1e-3          # the fp64 CDF differs only at rounding ties
    proj = np.zeros_like(full)
    for q in sub_q:
        proj = (proj << 1) | ((full >> (n - 1 - q)) & 1)
    assert np.array_equal(sub, proj)


def test_sampling_qft_n30_uniform_closed_form():
    """QFT of a basis state on n = 30 (complex64): every outcome has
    probability 2^-30, so the inverse CDF of u is floor(u * 2^30) away from
    rounding ties; first-three-qubit probabilities are 1/8 each."""
    from paper_2202_07017_gb300 import State
    n = 30
    st = State(n, "c64")
    try:
        st.init(W.random_basis_index(n, 1001))
        st.apply_circuit(W.qft(n), None)
        u = W.uniform_block(31, 0, 100000)
        xs = st.sample(list(range(n)), u).astype(np.int64)
        p3 = st.probabilities([0, 1, 2])
    finally:
        st.close()
    # The complex64 amplitudes carry relative errors up to ~1e-3 after 480
    # gates (the parity bound max|dpsi| 2^15 <= 1e-3), so |psi_y|^2 = 2^-30
    # (1 + O(1e-3)) and the CDF wanders by a random walk of about
    # 2^-30 * 2e-3 * sqrt(2^29) ~ 50 outcomes: samples stay within that of
    # u * 2^30, far inside 2^12.
    d = np.abs(xs - u * (1 << n))
    assert np.max(d) < 2 ** 12 and np.median(d) < 256
    assert np.max(np.abs(p3 - 0.125)) < 1e-5


def test_measurement_rejects_bad_arguments():
    from paper_2202_07017_gb300 import State, SvError
    st = State(4, "c64").init(0)
    try:
        for q in ([4], [1, 1], [-1], []):
            with pytest.raises(SvError):
                st.probabilities(q)
        with pytest.raises(SvError):
            st.sample([0], [1.0])
        with pytest.raises(SvError):
            st.sample([0], [-0.1])
        assert st.sample([0, 1], [0.0, 0.5]).tolist() == [0, 0]
    finally:
        st.close()
