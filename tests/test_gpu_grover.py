"""Multi-controlled gates at scale (Sec. 3: Grover's algorithm): gates with
up to n - 1 controls against the oracle, and Grover search on n = 20
(complex64, ~80k gates, unfused and fused) against the closed form
P(marked) = sin^2((2k + 1) asin(2^(-n/2)))."""
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
    try:
        st.apply_circuit(c, None, fuse_k)
        p = st.probabilities(list(range(n)))
    finally:
        st.close()
    # complex64 rounds 1/sqrt2 to h with 2h^2 = 1 - 3.4e-8, so every
    # Hadamard scales ||psi||^2 by 2h^2; unfused Grover at n = 20 applies
    # 40 per iteration (804 iterations): ||psi||^2 ~ 0.9989.  The
    # distribution itself is checked normalised.
    h = float(np.float32(1 / math.sqrt(2)))
    n_h = sum(1 for g in c.gates if g.kind == "H")
    norm_model = (2 * h * h) ** n_h
    total = p.sum()
    assert abs(p[marked] / total - math.sin((2 * k + 1) * th) ** 2) < 1e-4
    assert norm_model - 1e-4 <= total <= 1 + 1e-5


def test_grover_small_against_oracle():
    n, marked = 10, 333
    c = W.grover(n, marked, 7)
    for dtype in ("c64", "c128"):
        got = gpu_run(c, None, None, dtype)
        assert max_err(got, oracle.run(c)) <= TOL[dtype]
