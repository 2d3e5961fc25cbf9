"""The fusion planner (host-only, runs without a GPU): every gate planned once,
the circuit order kept for every qubit, every fused gate inside its pass's
staged bits, and the reordered circuit equal to the original on the CPU
oracle (gates on disjoint qubits commute, Eq. 1 applied in plan order)."""
import numpy as np
import pytest

import oracle
import workloads as W
from paper_2202_07017_gb300 import C64, C128, sv_fusion_plan


def check_plan(c, theta, dtype, k):
    order, pass_of, npass, masks = sv_fusion_plan(c, theta, dtype, k)
    n = c.n_qubits
    assert sorted(order.tolist()) == list(range(len(c.gates)))
    # pass ids non-decreasing among fused gates
    seq = [p for p in pass_of.tolist() if p >= 0]
    assert seq == sorted(seq)
    assert len(set(seq)) == npass
    # per-qubit order preserved
    for q in range(n):
        orig = [i for i, g in enumerate(c.gates) if q in g.targets or q in g.controls]
        planned = [i for i in order.tolist()
                   if q in c.gates[i].targets or q in c.gates[i].controls]
        assert orig == planned, (q, orig[:8], planned[:8])
    # fused gates lie inside the staged bits
    for i, p in zip(order.tolist(), pass_of.tolist()):
        if p < 0:
            continue
        g = c.gates[i]
        for q in tuple(g.targets) + tuple(g.controls):
            assert (masks[p] >> (n - 1 - q)) & 1
    return order, pass_of, npass


CASES = [
    ("layered", lambda: W.random_layered(12, 10, 5)),
    ("layered33", lambda: W.random_layered(33, 40, 1004)),
    ("qft", lambda: (W.qft(16), np.zeros(0))),
    ("hea", lambda: W.hea(20, 10, 1002)),
    ("random", lambda: W.random_gates(11, 200, 3, max_tar=4, max_ctrl=3)),
    ("random_small", lambda: W.random_gates(3, 50, 4, max_tar=3, max_ctrl=1)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_plan_is_a_valid_reordering(name, make, k):
    c, theta = make()
    for dt in (C64, C128):
        check_plan(c, theta, dt, k)


@pytest.mark.parametrize("name,make", [CASES[0], CASES[4], CASES[5]], ids=["layered", "random", "small"])
def test_plan_order_gives_the_same_state_on_the_oracle(name, make):
    c, theta = make()
    order, _, _ = check_plan(c, theta, C64, 4)
    psi0 = W.random_state(c.n_qubits, 8)
    ref = oracle.run(c, theta, psi0)
    re = W.Circuit(c.n_qubits, [c.gates[i] for i in order], c.n_params)
    assert np.max(np.abs(oracle.run(re, theta, psi0) - ref)) < 1e-12


def test_layered_n33_pass_count():
    """Random layered circuit n = 33, depth 40 (4600 gates): passes are far
    fewer than gates (one HBM round trip each)."""
    c, theta = W.random_layered(33, 40, 1004)
    assert len(c.gates) == 4600
    _, pass_of, npass = check_plan(c, theta, C64, 4)
    assert (pass_of >= 0).all()
    assert npass < 200


def test_plan_rejects_bad_arguments():
    c, theta = W.random_layered(5, 2, 1)
    from paper_2202_07017_gb300 import SvError
    with pytest.raises(SvError):
        sv_fusion_plan(c, theta, C64, 1)
    with pytest.raises(SvError):
        sv_fusion_plan(c, None, C64, 4)   # parameters missing


@pytest.mark.parametrize("n", [10, 12, 16, 20, 30])
def test_staged_bits_per_pass(n):
    """Every pass stages m bits: 13 (complex64) or 12 (complex128) slices,
    fewer for mid-size states so that at least 2^8 slices remain, and at
    least min(n, 10); the lowest L bits (5 for complex64, 4 for complex128,
    fewer when the slice is small) are always staged."""
    c, theta = W.random_layered(n, 3, 17)
    for dt, mmax, lmax in ((C64, 13, 5), (C128, 12, 4)):
        m = min(n, mmax)
        if n > 10:
            m = max(min(m, n - 8), min(n, 10))
        _, _, npass, masks = sv_fusion_plan(c, theta, dt, 4)
        assert npass == len(masks) > 0
        low = (1 << min(lmax, m - 4)) - 1 if m - lmax < 4 else (1 << lmax) - 1
        for mk in masks:
            assert bin(mk).count("1") == m, (n, dt, bin(mk))
            assert mk & low == low
