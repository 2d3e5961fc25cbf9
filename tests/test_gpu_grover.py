"""Multi-controlled gates at scale (Sec. 3: Grover's algorithm): gates with
up to n - 1 controls against the oracle, and Grover search on n = 20
(complex64, ~80k gates, unfused and fused) against the closed form
P(marked) = sin^2((2k + 1) asin(2^(-n/2))) with ||psi||^2 within 1e-5 of 1."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import TOL, gpu_run, max_err, oracle_threads, rounded

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle_threads()


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_many_control_gates(dtype):
    n = 14
    psi = rounded(W.random_state(n, 45), dtype)
    gates = [W.Gate("Z", (n - 1,), tuple(range(n - 1))),
             W.Gate("X", (0,), tuple(range(1, n))),
             W.Gate("U1", (5,), tuple(q for q in range(n) if q != 5), -1, 0.77),
             W.Gate("RY", (3,), tuple(q for q in range(n) if q not in (3, 9)), -1, 1.3),
             W.Gate("SWAP", (2, 11), tuple(q for q in range(n) if q not in (2, 11)))]
    for g in gates:
        c = W.Circuit(n, [g], 0)
        assert max_err(gpu_run(c, None, psi, dtype), oracle.run(c, None, psi)) <= TOL[dtype]


@pytest.mark.parametrize("fuse_k", [0, 4])
def test_grover_n20_closed_form(fuse_k):
    from paper_2202_07017_gb300 import State
    n = 20
    N = 1 << n
    th = math.asin(1 / math.sqrt(N))
    k = int(math.floor(math.pi / (4 * th)))
    marked = 0xB3C5A % N
    c = W.grover(n, marked, k)
    st = State(n, "c64").init(0)
    if fuse_k:
        st.set_rounding("dithered")
    try:
        st.apply_circuit(c, None, fuse_k)
        p = st.probabilities(list(range(n)))
    finally:
        st.close()
    # 32 180 Hadamards in complex64 on states with 2^20 - 1 equal
    # amplitudes: error-feedback coefficients (a plain rounding of 1/sqrt2
    # would lose 1.1e-3) and dithered roundings (round-to-nearest repeats one
    # error on all equal amplitudes: 2.5e-5 unfused, 1.4e-5 fused) keep
    # ||psi||^2 at 1 within the complex64 bar
    total = p.sum()
    assert abs(1 - total) <= 1e-5
    assert abs(p[marked] - math.sin((2 * k + 1) * th) ** 2) < 1e-4


def test_grover_small_against_oracle():
    n, marked = 10, 333
    c = W.grover(n, marked, 7)
    for dtype in ("c64", "c128"):
        got = gpu_run(c, None, None, dtype)
        assert max_err(got, oracle.run(c)) <= TOL[dtype]
