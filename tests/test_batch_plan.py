"""The batch planner on the host (no GPU): validation of the batch kernel's
limits and the register-group schedule for every group width, including
gates as wide as the group (the case that must not stall the schedule)."""
import pytest

import workloads as W
from paper_2202_07017_gb300 import SvError, sv_batch_plan

ONEQ = ("H", "X", "Y", "Z", "RX", "RY", "RZ", "U1")


def test_groups_for_each_width():
    hea, _ = W.hea(14, 10, 1)
    g = {k: int(sv_batch_plan([hea], [W.tfim(14)], k)[0]) for k in (2, 3, 4)}
    assert g[2] >= g[3] >= g[4] >= 1
    assert g[4] < len(hea.gates)


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
