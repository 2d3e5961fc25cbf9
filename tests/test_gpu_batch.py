"""GPU parity of the batched persistent kernel (energies and adjoint
gradients of many circuits in one launch) against the oracle's energies and
exact shift-rule gradients; graph
replay and the autotuner; the batch shaped like 4096 parameter sets of the
n = 14 hardware-efficient ansatz plus 1024 mixed circuits (n 8..16, depth
5..15)."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import oracle_threads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ONEQ = ("H", "X", "Y", "Z", "RX", "RY", "RZ", "U1")


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle_threads()


def _rel(g, ref):
    return float(np.max(np.abs(g - ref)) / max(np.max(np.abs(ref)), 1e-300))


def _small_batch():
    circuits, hams = [], []
    for n in (1, 2, 3, 5, 8):
        c, _ = W.hea(n, 3, 10 + n)
        circuits.append(c)
        hams.append(W.tfim(n) if n > 1 else [(1.0, ((0, "X"),)), (0.5, ((0, "Z"),))])
    for n, seed in ((4, 1), (7, 2), (9, 3)):
        c, _ = W.random_gates(n, 50, seed, max_tar=1, max_ctrl=2, kinds=ONEQ)
        circuits.append(c)
        hams.append(W.random_pauli_sum(n, 12, seed))
    items = [i % len(circuits) for i in range(2 * len(circuits))]
    rng = W.SplitMix64(77)
    thetas = [np.array([rng.angle() for _ in range(circuits[ci].n_params)]) for ci in items]
    return circuits, hams, items, thetas


@pytest.mark.parametrize("tune", [0, 1, 2, 3], ids=["default", "tuned", "cluster", "smem-states"])
def test_batch_against_oracle(tune):
    from paper_2202_07017_gb300 import Batch
    circuits, hams, items, thetas = _small_batch()
    b = Batch(circuits, hams, items, tune=tune)
    theta = torch.tensor(np.concatenate(thetas), dtype=torch.float64, device="cuda")
    e, g = b.run(theta)
    e2, g2 = b.run(theta, graph=True)
    e3, g3 = b.run(theta, graph=True)
    torch.cuda.synchronize()
    e, g, e2, g2, e3, g3 = (t.cpu().numpy() for t in (e, g, e2, g2, e3, g3))
    b.close()
    assert np.array_equal(e, e2) and np.array_equal(g, g2)   # same kernel, fixed order
    assert np.array_equal(e2, e3) and np.array_equal(g2, g3)
    off = 0
    for i, ci in enumerate(items):
        c, H, th = circuits[ci], hams[ci], thetas[i]
        scale = sum(abs(t[0]) for t in H)
        assert abs(e[i] - oracle.energy(c, th, H)) <= 1e-5 * scale
        if c.n_params:
            gi = g[off:off + c.n_params]
            ref = oracle.grad_param_shift(c, th, H)
            assert _rel(gi, ref) <= 1e-5, (i, _rel(gi, ref))
        off += c.n_params


def test_batch_one_shot_matches_persistent_run():
    from paper_2202_07017_gb300 import Batch, sv_batch_grad
    circuits, hams, items, thetas = _small_batch()
    theta = np.concatenate(thetas)
    e1, g1 = sv_batch_grad(circuits, hams, items, theta)
    b = Batch(circuits, hams, items, tune=False)
    e2, g2 = b.run(torch.tensor(theta, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    assert np.array_equal(e1, e2.cpu().numpy()) and np.array_equal(g1, g2.cpu().numpy())
    b.close()


def test_batch_rejects_unsupported_gates():
    from paper_2202_07017_gb300 import Batch, SvError
    c = W.Circuit(3, [W.Gate("SWAP", (0, 1))], 0)
    with pytest.raises(SvError):
        Batch([c], [W.tfim(3)], [0], tune=False)
    c, th = W.hea(19, 1, 1)
    with pytest.raises(SvError):
        Batch([c], [W.tfim(19)], [0], tune=False)


def test_batch_hea14_and_mixed_shapes():
    """4096 parameter sets of the n = 14, L = 10 ansatz (TFIM) plus 1024
    mixed circuits (n uniform in 8..16, depth 5..15), one persistent launch,
    autotuned; sampled items' energies and gradient entries against the
    oracle (every energy and 20 full gradients: test_gpu_fullsize.py)."""
    from paper_2202_07017_gb300 import Batch
    hea14, _ = W.hea(14, 10, 1003)
    mixed = W.mixed_batch(1024, 1003)
    circuits = [hea14] + [m[0] for m in mixed]
    hams = [W.tfim(14)] + [m[2] for m in mixed]
    items = [0] * 4096 + list(range(1, 1025))
    thetas = [W.hea_theta(14, 10, 1003 + i) for i in range(4096)] + [m[1] for m in mixed]
    theta = np.concatenate(thetas)
    b = Batch(circuits, hams, items, tune=True)
    e, g = b.run(torch.tensor(theta, dtype=torch.float64, device="cuda"), graph=True)
    torch.cuda.synchronize()
    e, g = e.cpu().numpy(), g.cpu().numpy()
    b.close()
    offs = np.concatenate([[0], np.cumsum([circuits[ci].n_params for ci in items])])
    rs = np.random.default_rng(1)
    sample = [0, 4095, 4096, 4100, 5119] + list(rs.integers(0, 5120, 8))
    for i in sample:
        c, H, th = circuits[items[i]], hams[items[i]], thetas[i]
        assert abs(e[i] - oracle.energy(c, th, H)) <= 1e-5 * sum(abs(t[0]) for t in H)
        ps = [0, c.n_params // 2, c.n_params - 1]
        ref = oracle.grad_param_shift(c, th, H, params=ps)
        gi = g[offs[i]:offs[i + 1]]
        assert np.max(np.abs(gi[ps] - ref[ps])) <= 1e-5 * max(1.0, np.max(np.abs(ref[ps])))


@pytest.mark.parametrize("mode,cl,sm", [(0, 1, False), (2, 2, True), (3, 1, True)],
                         ids=["single-block", "cluster", "smem-states"])
def test_batch_kernel_choice_and_both_state_homes(mode, cl, sm):
    """tune = 0 runs single blocks on global workspace; tune = 2 runs
    two-block clusters (items up to 14 qubits keep psi and lambda split over
    the pair's shared memory, larger ones in the cluster's global slot), a
    gate with 3 controls falling back to the single-block kernel; tune = 3
    runs single blocks with psi (and lambda up to 13 qubits) in shared
    memory.  Energies and sampled gradient entries against the oracle."""
    from paper_2202_07017_gb300 import Batch
    mixed = W.mixed_batch(40, 2024)
    big = [m for m in mixed if m[0].n_qubits >= 15][:3] + [m for m in mixed if m[0].n_qubits <= 10][:3]
    c3, th3 = W.random_gates(9, 60, 5, max_tar=1, max_ctrl=3, kinds=ONEQ)
    cases = [([m[0] for m in big], [m[2] for m in big], [m[1] for m in big], (cl, sm)),
             ([c3], [W.random_pauli_sum(9, 10, 5)], [th3], (1, mode == 3))]
    for circuits, hams, thetas, want in cases:
        items = list(range(len(circuits)))
        b = Batch(circuits, hams, items, tune=mode)
        assert (b.cluster, b.smem_states) == want
        e, g = b.run(torch.tensor(np.concatenate(thetas), dtype=torch.float64, device="cuda"))
        torch.cuda.synchronize()
        e, g = e.cpu().numpy(), g.cpu().numpy()
        b.close()
        off = 0
        for i, (c, H, th) in enumerate(zip(circuits, hams, thetas)):
            scale = sum(abs(t[0]) for t in H)
            assert abs(e[i] - oracle.energy(c, th, H)) <= 1e-5 * scale
            if c.n_params:
                ps = sorted({0, c.n_params // 3, c.n_params // 2, c.n_params - 1})
                g_ref = oracle.grad_param_shift(c, th, H, params=ps)
                # normwise over the sample, with a floor for circuits whose
                # gradient vanishes (rotations whose controls are rarely set)
                err = np.max(np.abs(g[off:off + c.n_params][ps] - g_ref[ps]))
                assert err <= 1e-5 * max(np.max(np.abs(g_ref[ps])), 0.05 * scale), (i, err)
            off += c.n_params


REAL = ("H", "X", "Z", "RY")


def _real_terms(n, count, seed):
    """Random Pauli strings with an even number of Y factors (real matrices)."""
    terms = [t for t in W.random_pauli_sum(n, 4 * count, seed)
             if sum(1 for _, p in t[1] if p == "Y") % 2 == 0]
    return terms[:count]


def test_real_batch_against_oracle():
    """The real-amplitude kernel (tune = 4): HEA items and random circuits of
    real gates with up to 3 controls (H, X, Z, RY: CNOT, CZ, controlled RY
    ...), Hamiltonians of real terms (XX, YY, ZZ, X, Z strings); items of
    8..16 qubits put psi and lambda in shared memory (n <= 14), psi alone
    (n = 15) or neither (n = 16).  Energies and gradients against the oracle;
    graph replay repeats the launch bit for bit."""
    from paper_2202_07017_gb300 import Batch
    circuits, hams = [], []
    for n in (1, 2, 5, 9, 14, 15, 16):
        c, _ = W.hea(n, 3 if n < 15 else 2, 40 + n)
        circuits.append(c)
        hams.append(W.tfim(n) if n > 1 else [(1.0, ((0, "X"),)), (0.5, ((0, "Z"),))])
    for n, seed in ((4, 1), (8, 2), (11, 3)):
        c, _ = W.random_gates(n, 60, 300 + seed, max_tar=1, max_ctrl=3, kinds=REAL)
        circuits.append(c)
        hams.append(_real_terms(n, 10, seed))
    items = list(range(len(circuits))) + [1, 3, 7]
    rng = W.SplitMix64(78)
    thetas = [np.array([rng.angle() for _ in range(circuits[ci].n_params)]) for ci in items]
    b = Batch(circuits, hams, items, tune=4)
    assert b.real and b.smem_states and b.cluster == 1
    theta = torch.tensor(np.concatenate(thetas), dtype=torch.float64, device="cuda")
    e, g = b.run(theta)
    e2, g2 = b.run(theta, graph=True)
    torch.cuda.synchronize()
    e, g, e2, g2 = (t.cpu().numpy() for t in (e, g, e2, g2))
    b.close()
    assert np.array_equal(e, e2) and np.array_equal(g, g2)
    off = 0
    for i, ci in enumerate(items):
        c, H, th = circuits[ci], hams[ci], thetas[i]
        scale = sum(abs(t[0]) for t in H)
        assert abs(e[i] - oracle.energy(c, th, H)) <= 1e-5 * scale, i
        if c.n_params:
            ps = (list(range(c.n_params)) if c.n_qubits <= 11
                  else sorted({0, c.n_params // 3, c.n_params // 2, c.n_params - 1}))
            ref = oracle.grad_param_shift(c, th, H, params=ps)
            err = np.max(np.abs(g[off:off + c.n_params][ps] - ref[ps]))
            assert err <= 1e-5 * max(np.max(np.abs(ref[ps])), 0.05 * scale), (i, err)
        off += c.n_params


def test_real_batch_matches_complex_kernel():
    """The same real batch through the real-amplitude kernel and the complex
    shared-memory kernel: energies and gradients agree to fp32 rounding."""
    from paper_2202_07017_gb300 import Batch
    mixed = W.mixed_batch(24, 99)
    circuits = [m[0] for m in mixed]
    hams = [m[2] for m in mixed]
    theta = np.concatenate([m[1] for m in mixed])
    items = list(range(len(circuits)))
    out = {}
    for tune in (3, 4):
        b = Batch(circuits, hams, items, tune=tune)
        assert b.real == (tune == 4)
        e, g = b.run(torch.tensor(theta, dtype=torch.float64, device="cuda"))
        torch.cuda.synchronize()
        out[tune] = (e.cpu().numpy(), g.cpu().numpy())
        b.close()
    scale = max(sum(abs(t[0]) for t in H) for H in hams)
    assert np.max(np.abs(out[3][0] - out[4][0])) <= 2e-6 * scale
    assert np.max(np.abs(out[3][1] - out[4][1])) <= 2e-6 * scale


def test_real_kernel_refuses_complex_batches():
    from paper_2202_07017_gb300 import Batch, SvError
    c, _ = W.hea(5, 2, 1)
    with pytest.raises(SvError):  # a Y term is imaginary
        Batch([c], [[(1.0, ((0, "Y"),))]], [0], tune=4)
    c2, _ = W.random_gates(5, 20, 3, max_tar=1, max_ctrl=1, kinds=("RX", "RY"))
    with pytest.raises(SvError):  # RX is complex
        Batch([c2], [W.tfim(5)], [0], tune=4)
