"""The batch planner on the host (no GPU): validation of the batch kernel's
limits and the register-group schedule for every group width, including
gates as wide as the group (the case that must not stall the schedule)."""
import numpy as np
import pytest

import workloads as W
from paper_2202_07017_gb300 import SvError, sv_batch_plan

ONEQ = ("H", "X", "Y", "Z", "RX", "RY", "RZ", "U1")


def test_groups_for_each_width():
    hea, _ = W.hea(14, 10, 1)
    g = {k: int(sv_batch_plan([hea], [W.tfim(14)], k)[0]) for k in (2, 3, 4, 5)}
    assert g[2] >= g[3] >= g[4] >= g[5] >= 1
    assert g[4] < len(hea.gates)
    with pytest.raises(SvError):  # 5 qubits is the widest register group
        sv_batch_plan([hea], [W.tfim(14)], 6)


def test_wide_gates_need_wide_groups():
    c, _ = W.random_gates(9, 80, 2, max_tar=1, max_ctrl=2, kinds=ONEQ)
    widest = max(1 + len(g.controls) for g in c.gates)
    assert widest == 3
    with pytest.raises(SvError):
        sv_batch_plan([c], [W.tfim(9)], 2)
    assert sv_batch_plan([c], [W.tfim(9)], 3)[0] > 0
    assert sv_batch_plan([c], [W.tfim(9)], 4)[0] > 0


def test_batch_limits_rejected_on_host():
    with pytest.raises(SvError):
        sv_batch_plan([W.Circuit(3, [W.Gate("SWAP", (0, 1))], 0)], [W.tfim(3)], 4)
    with pytest.raises(SvError):
        sv_batch_plan([W.hea(19, 1, 1)[0]], [W.tfim(19)], 4)
    with pytest.raises(SvError):
        sv_batch_plan([W.hea(4, 1, 1)[0]], [W.random_pauli_sum(4, 65, 1)], 4)
    mixed = W.mixed_batch(64, 5)
    out = sv_batch_plan([m[0] for m in mixed], [m[2] for m in mixed], 4)
    assert (out > 0).all()


def test_mixed_batch_recipe():
    """The C3 mixed batch: 1024 HEA circuits with n uniform in 8..16 and L in
    5..15 (every value drawn), each with its own open-chain TFIM and n*L
    parameters."""
    items = W.mixed_batch(1024, 1003)
    ns = [c.n_qubits for c, _, _ in items]
    Ls = [len(th) // c.n_qubits for c, th, _ in items]
    assert len(items) == 1024
    assert set(ns) == set(range(8, 17)) and set(Ls) == set(range(5, 16))
    for (c, th, H), L in zip(items, Ls):
        assert c.n_params == len(th) == c.n_qubits * L
        assert len(H) == 2 * c.n_qubits - 1
    # roughly uniform: every qubit count within 40 % of 1024 / 9
    counts = np.bincount(ns, minlength=17)[8:]
    assert counts.min() > 0.6 * 1024 / 9 and counts.max() < 1.4 * 1024 / 9


def test_real_amplitude_kernel_needs_real_gates_and_terms():
    """tune = 4 (the real-amplitude batch kernel) is refused on the host, before
    any device work, for a Y term (an odd number of Y factors is an imaginary
    matrix) or a complex gate (RX)."""
    from paper_2202_07017_gb300 import sv_batch_create
    hea, _ = W.hea(5, 2, 1)
    with pytest.raises(SvError, match="real amplitudes"):
        sv_batch_create([hea], [[(1.0, ((0, "Y"),))]], [0], 4)
    c, _ = W.random_gates(5, 20, 3, max_tar=1, max_ctrl=1, kinds=("RX", "RY"))
    with pytest.raises(SvError, match="real amplitudes"):
        sv_batch_create([c], [W.tfim(5)], [0], 4)
