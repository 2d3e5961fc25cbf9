"""The reverse-sweep planner of the fused adjoint gradient (host-only, no
GPU): every gate of the segment un-applied once and in reverse circuit order
on each qubit; every parameterised gate's gradient taken once, before its
un-apply; gradients that share one evaluation sit on one qubit with only
uncontrolled 1-qubit gates on that qubit between them (they then see the same
inner product: the other gates act on other qubits and commute with the
generator)."""
import numpy as np
import pytest

import workloads as W
from paper_2202_07017_gb300 import C64, C128, SvError, sv_fusion_plan_reverse


def _touches(g, q):
    return q in g.targets or q in g.controls


def check_reverse_plan(c, theta, dtype, k, lo=0, hi=None):
    hi = len(c.gates) if hi is None else hi
    ev, npass = sv_fusion_plan_reverse(c, theta, dtype, k, lo, hi)
    seg = range(lo, hi)
    unapply = [int(e[1]) for e in ev if e[0] == 0]
    grads = [int(e[1]) for e in ev if e[0] == 1]
    # every gate un-applied once, every parameterised gate differentiated once
    assert sorted(unapply) == list(seg)
    assert sorted(grads) == [i for i in seg if c.gates[i].param >= 0]
    pos_un = {int(e[1]): t for t, e in enumerate(ev) if e[0] == 0}
    pos_gr = {int(e[1]): t for t, e in enumerate(ev) if e[0] == 1}
    for i in grads:
        assert pos_gr[i] < pos_un[i], i
    # reverse circuit order kept on every qubit (the un-applies that touch it)
    for q in range(c.n_qubits):
        want = [i for i in reversed(seg) if _touches(c.gates[i], q)]
        got = [i for i in unapply if _touches(c.gates[i], q)]
        assert got == want, (q, want[:6], got[:6])
    # passes are contiguous in the event list
    passes = [int(e[2]) for e in ev if e[2] >= 0]
    assert passes == sorted(passes) and (not passes or passes[-1] + 1 == npass)
    # shared evaluations
    evals = {}
    for e in ev:
        if e[0] == 1:
            evals.setdefault(int(e[3]), []).append(int(e[1]))
    for members in evals.values():
        assert len(members) <= 4
        if len(members) == 1:
            continue
        qs = {c.gates[i].targets[0] for i in members}
        assert len(qs) == 1 and all(not c.gates[i].controls for i in members), members
        q = qs.pop()
        for j in range(min(members) + 1, max(members)):
            g = c.gates[j]
            if _touches(g, q):
                assert len(g.targets) == 1 and not g.controls, (members, j, g)
    return ev, npass, evals


CASES = [
    ("layered", lambda: W.random_layered(12, 10, 5)),
    ("layered28", lambda: W.random_layered(28, 10, 1004)),
    ("hea", lambda: W.hea(20, 10, 1002)),
    ("random", lambda: W.random_gates(11, 200, 3, max_tar=4, max_ctrl=3)),
    ("random_small", lambda: W.random_gates(4, 60, 4, max_tar=3, max_ctrl=1)),
    ("random_phases", lambda: W.random_gates(8, 160, 7, max_tar=2, max_ctrl=2,
                                             kinds=("H", "X", "Y", "Z", "RX", "RY", "RZ", "U1",
                                                    "SWAP", "MATRIX"))),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("k", [2, 3, 4])
@pytest.mark.parametrize("dtype", [C64, C128])
def test_reverse_plan_is_valid(name, make, k, dtype):
    c, theta = make()
    check_reverse_plan(c, theta, dtype, k)


def expected_evaluations(c):
    """Gradients of uncontrolled rotations on one qubit with only uncontrolled
    1-qubit gates on it in between, in chunks of at most 4 (reverse order);
    every other parameterised gate alone."""
    out = []
    run = {}
    for i in reversed(range(len(c.gates))):
        g = c.gates[i]
        if len(g.targets) == 1 and not g.controls:
            q = g.targets[0]
            if g.param >= 0:
                cur = run.setdefault(q, [])
                if len(cur) == 4:
                    out.append(cur)
                    cur = run[q] = []
                cur.append(i)
            continue
        for q in tuple(g.targets) + tuple(g.controls):
            if run.get(q):
                out.append(run.pop(q))
        if g.param >= 0:
            out.append([i])
    out.extend(v for v in run.values() if v)
    return sorted(sorted(m) for m in out)


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_shared_evaluations_match_the_rotation_runs(name, make):
    """On the layered circuit RX, RY, RZ of a layer share one evaluation; a
    qubit without a CZ in a layer joins two layers' rotations (6 = 4 + 2)."""
    c, theta = make()
    _, _, evals = check_reverse_plan(c, theta, C64, 4)
    assert sorted(sorted(m) for m in evals.values()) == expected_evaluations(c)


def test_run_longer_than_four_splits():
    n = 6
    gates, p = [], 0
    for kind in ("RX", "RY", "RZ", "RX", "RY", "RZ", "RX"):
        gates.append(W.Gate(kind, (2,), (), p))
        p += 1
    gates.append(W.Gate("Z", (3,), (2,)))
    for kind in ("RY", "RZ"):
        gates.append(W.Gate(kind, (2,), (), p))
        p += 1
    c = W.Circuit(n, gates, p)
    theta = np.linspace(0.1, 1.0, p)
    _, _, evals = check_reverse_plan(c, theta, C64, 4)
    groups = sorted(sorted(m) for m in evals.values())
    # the CZ on qubit 2 separates the last two rotations from the first seven
    assert [7, 8] not in [[g for g in m if g < 7] for m in groups]
    assert sorted(len(m) for m in groups) == [2, 3, 4]


def test_segments_and_bad_arguments():
    c, theta = W.random_layered(10, 4, 2)
    n = len(c.gates)
    for lo, hi in ((0, n // 2), (n // 2, n), (n // 3, 2 * n // 3), (5, 5)):
        check_reverse_plan(c, theta, C64, 4, lo, hi)
    for lo, hi in ((-1, 3), (4, 3), (0, n + 1)):
        with pytest.raises(SvError):
            sv_fusion_plan_reverse(c, theta, C64, 4, lo, hi)
    with pytest.raises(SvError):
        sv_fusion_plan_reverse(c, theta, C64, 6)


def test_gradient_capacity_per_pass():
    """A pass holds at most 200 gradients (its accumulator slots): 400 rotations
    on 12 qubits with nothing else between them need at least two passes, and
    the plan stays valid."""
    n = 12
    gates, p = [], 0
    for rep in range(400 // n + 1):
        for q in range(n):
            if p == 400:
                break
            gates.append(W.Gate(("RX", "RY", "RZ")[rep % 3], (q,), (), p))
            p += 1
    c = W.Circuit(n, gates, p)
    theta = np.linspace(0.0, 3.0, p)
    ev, npass, evals = check_reverse_plan(c, theta, C64, 4)
    per_pass = {}
    for e in ev:
        if e[0] == 1:
            per_pass[int(e[2])] = per_pass.get(int(e[2]), 0) + 1
    assert npass >= 2 and max(per_pass.values()) <= 200
