"""Writes tests/golden/layered_n28_d40.npz: the oracle's complex128 forward
state of the random layered circuit at n = 28, depth 40 (seed 1004: RX, RY,
RZ on every qubit, then the CZ brick of the layer's parity), sampled at
65536 seeded amplitude indices plus the first and last index, with
<sum_i Z_i> and ||psi||^2 of the full state.

The values come from the oracle alone (one run of its Eq. (1) index loop
over the 3900 gates; about an hour on 8 host threads, 4 GiB of state), so
the GPU parity test at this size does not have to repeat that run.

    python tests/golden/make_layered_n28.py [threads]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads as W  # noqa: E402

N, DEPTH, SEED = 28, 40, 1004
SAMPLE_SEED, N_SAMPLES = 2804, 1 << 16
OUT = os.path.join(HERE, "layered_n28_d40.npz")


def sample_indices():
    """Seeded amplitude indices: SplitMix64 outputs masked to 28 bits,
    with 0 and 2^28 - 1 added; unique and sorted."""
    raw = W.splitmix64_block(SAMPLE_SEED, 0, N_SAMPLES) & np.uint64((1 << N) - 1)
    idx = np.concatenate([raw, np.array([0, (1 << N) - 1], np.uint64)])
    return np.unique(idx)


def main():
    threads = int(sys.argv[1]) if len(sys.argv) > 1 else (os.cpu_count() or 1)
    oracle.set_threads(threads)
    c, theta = W.random_layered(N, DEPTH, SEED)
    t0 = time.time()
    psi = oracle.run(c, theta)
    t1 = time.time()
    energy = oracle.expval(psi, W.sum_z(N), N)
    norm = oracle.norm2(psi)
    idx = sample_indices()
    np.savez(OUT, idx=idx, amp=psi[idx.astype(np.int64)], energy=np.float64(energy),
             norm=np.float64(norm), gates=np.int64(len(c.gates)))
    print(f"wrote {OUT}: {idx.size} amplitudes, energy {energy!r}, norm {norm!r}, "
          f"{len(c.gates)} gates in {t1 - t0:.0f} s on {threads} threads")


if __name__ == "__main__":
    main()
