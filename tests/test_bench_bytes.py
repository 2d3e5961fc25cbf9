"""The bench's algorithmic bytes (host logic, CPU): B_alg = 2 * s * |A| per gate,
A the amplitudes the gate changes on a generic input (H: 2^n, controlled-U1:
2^(n-2), SWAP: 2^(n-1)), and one write of the state for the basis-state
initialisation.  Pinned by counting, for every gate of the n = 30 QFT, the
amplitudes its matrix changes on small n by brute force, and by the step total."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import workloads as W  # noqa: E402

KERNEL_OF = {"H": "k1q_c64_pair", "U1": "kphase_c64", "SWAP": "kswap_c64_vv"}


def changed_amplitudes(n, g):
    """Amplitudes that the gate's full 2^n operator moves on a generic state,
    by brute force: rows of (U - I) with a nonzero entry."""
    import oracle
    dim = 1 << n
    cols = []
    c = W.Circuit(n, [g], 0)
    for x in range(dim):
        e = np.zeros(dim, np.complex128)
        e[x] = 1.0
        cols.append(oracle.run(c, np.zeros(0), e))
    U = np.array(cols).T
    return int(np.count_nonzero(np.any(np.abs(U - np.eye(dim)) > 1e-12, axis=1)))


def test_bytes_per_gate_match_the_changed_amplitudes():
    n = 6
    for g in W.qft(n).gates:
        kind = "U1" if g.kind == "U1" else g.kind
        want = 2 * 8 * changed_amplitudes(n, g)
        assert bench.algorithmic_bytes(KERNEL_OF[kind], n, 8) == want, g


def test_qft_step_bytes_at_n30():
    n = 30
    c = W.qft(n)
    per_gate = sum(bench.algorithmic_bytes(KERNEL_OF[g.kind], n, 8) for g in c.gates)
    # 30 H x 17.18 GB + 435 CU1 x 4.295 GB + 15 SWAP x 8.59 GB
    assert per_gate == 30 * 2 * 8 * 2 ** 30 + 435 * 2 * 8 * 2 ** 28 + 15 * 2 * 8 * 2 ** 29
    assert abs(per_gate / 1e9 - 2512.6) < 0.1
    assert bench.algorithmic_bytes("kinit_c64", n, 8) == 8 * 2 ** n
