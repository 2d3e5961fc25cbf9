"""Parity of the benchmark configurations at their stated sizes against the
complex128 oracle (not against another path of the library):

* hardware-efficient ansatz n = 20, L = 10, TFIM (complex64, fp64
  reductions): the final state, the energy and all 200 adjoint gradients
  against the oracle's exact parameter shift, unfused, fused and through
  torch.autograd;
* the batch of 4096 ansatz parameter sets at n = 14 plus 1024 mixed
  circuits (n 8..16, depth 5..15): every one of the 5120 energies against
  the oracle, and the full gradients of 20 items that cover every qubit
  count 8..16;
* the random layered circuit at n = 28, depth 40 (complex64): sampled
  amplitudes of the forward state (fused, unfused, and the one left by the
  checkpointed fused gradient), its norm and <sum Z_i> against one oracle
  run stored in tests/golden/layered_n28_d40.npz (written by
  tests/golden/make_layered_n28.py from the oracle alone); the same
  generator's checkpointed gradient at n = 18 against the shift rule.
"""
import os

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import TOL, max_err, oracle_threads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "layered_n28_d40.npz")


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle_threads()


def _rel(g, ref):
    return float(np.max(np.abs(np.asarray(g) - ref)) / max(np.max(np.abs(ref)), 1e-300))


# ---- hardware-efficient ansatz n = 20, L = 10 ----------------------------------------
@pytest.fixture(scope="module")
def hea20():
    c, theta = W.hea(20, 10, 1002)
    H = W.tfim(20)
    psi = oracle.run(c, theta)
    return {"c": c, "theta": theta, "H": H, "psi": psi, "e": oracle.expval(psi, H, 20),
            "g": oracle.grad_param_shift(c, theta, H)}


@pytest.mark.parametrize("fuse_k", [0, 4])
def test_hea20_state_energy_and_every_gradient(hea20, fuse_k):
    from paper_2202_07017_gb300 import State
    d = hea20
    st = State(20, "c64").init(0)
    try:
        e, g = st.grad(d["c"], d["theta"], d["H"], [], fuse_k=fuse_k)
        psi = st.numpy()
    finally:
        st.close()
    assert d["c"].n_params == 200
    assert max_err(psi, d["psi"]) <= TOL["c64"]
    assert abs(1 - float(np.vdot(psi, psi).real)) <= TOL["c64"]
    assert abs(e - d["e"]) <= TOL["c64"] * sum(abs(t[0]) for t in d["H"])
    assert _rel(g, d["g"]) <= 1e-5


@pytest.mark.parametrize("fuse_k", [0, 4])
def test_hea20_through_torch_autograd(hea20, fuse_k):
    from paper_2202_07017_gb300 import State, energy
    d = hea20
    st = State(20, "c64")
    try:
        th = torch.tensor(d["theta"], dtype=torch.float64, requires_grad=True)
        E = energy(th, st, d["c"], d["H"], fuse_k=fuse_k)
        E.backward()
    finally:
        st.close()
    assert abs(E.item() - d["e"]) <= TOL["c64"] * sum(abs(t[0]) for t in d["H"])
    assert _rel(th.grad.numpy(), d["g"]) <= 1e-5


# ---- the 5120-item batch ---------------------------------------------------------------
@pytest.fixture(scope="module")
def batch5120():
    hea14, _ = W.hea(14, 10, 1003)
    mixed = W.mixed_batch(1024, 1003)
    circuits = [hea14] + [m[0] for m in mixed]
    hams = [W.tfim(14)] + [m[2] for m in mixed]
    items = [0] * 4096 + list(range(1, 1025))
    thetas = [W.hea_theta(14, 10, 1003 + i) for i in range(4096)] + [m[1] for m in mixed]
    e_ref = np.array([oracle.energy(circuits[ci], thetas[i], hams[ci])
                      for i, ci in enumerate(items)])
    scale = np.array([sum(abs(t[0]) for t in hams[ci]) for ci in items])
    return {"circuits": circuits, "hams": hams, "items": items, "thetas": thetas,
            "e_ref": e_ref, "scale": scale}


def _run_batch(b5, tune):
    from paper_2202_07017_gb300 import Batch
    b = Batch(b5["circuits"], b5["hams"], b5["items"], tune=tune)
    try:
        th = torch.tensor(np.concatenate(b5["thetas"]), dtype=torch.float64, device="cuda")
        e, g = b.run(th, graph=True)
        torch.cuda.synchronize()
        return e.cpu().numpy(), g.cpu().numpy()
    finally:
        b.close()


@pytest.mark.parametrize("tune", [0, 1, 3, 4], ids=["default", "tuned", "smem-states", "real"])
def test_batch_every_energy(batch5120, tune):
    e, _ = _run_batch(batch5120, tune)
    err = np.abs(e - batch5120["e_ref"]) / batch5120["scale"]
    assert err.size == 5120
    assert float(err.max()) <= TOL["c64"], int(np.argmax(err))


_GRAD_REFS = {}


@pytest.mark.parametrize("tune", [1, 3], ids=["tuned", "smem-states"])
def test_batch_full_gradients_for_every_qubit_count(batch5120, tune):
    """Full gradients of 20 items (2 per qubit count) against the oracle: with
    the autotuner's kernel (the batch is real: the real-amplitude kernel) and
    with the complex shared-memory kernel."""
    b5 = batch5120
    e, g = _run_batch(b5, tune)
    items, circuits = b5["items"], b5["circuits"]
    offs = np.concatenate([[0], np.cumsum([circuits[ci].n_params for ci in items])])
    pick = [0, 4095]
    for nq in range(8, 17):
        pick += [i for i in range(4096, 5120) if circuits[items[i]].n_qubits == nq][:2]
    assert len(pick) == 20
    for i in pick:
        c, H, th = circuits[items[i]], b5["hams"][items[i]], b5["thetas"][i]
        if i not in _GRAD_REFS:
            _GRAD_REFS[i] = oracle.grad_param_shift(c, th, H)
        ref = _GRAD_REFS[i]
        assert _rel(g[offs[i]:offs[i + 1]], ref) <= 1e-5, (i, c.n_qubits)


# ---- random layered circuit, n = 28 ----------------------------------------------------
@pytest.fixture(scope="module")
def golden28():
    if not os.path.exists(GOLDEN):
        pytest.fail("tests/golden/layered_n28_d40.npz is missing "
                    "(python tests/golden/make_layered_n28.py writes it from the oracle)")
    z = np.load(GOLDEN)
    return {k: z[k] for k in z.files}


def _check28(st, z):
    idx = torch.from_numpy(z["idx"].astype(np.int64)).to(st.tensor.device)
    got = st.tensor[idx].cpu().numpy()
    e = st.expval(W.sum_z(28))
    nrm = st.norm()
    assert max_err(got, z["amp"]) <= TOL["c64"]
    # the amplitudes are ~2^-14: also bound the error relative to their size
    d = np.abs(got.astype(np.complex128) - z["amp"])
    assert float(np.sqrt(np.mean(d * d) / np.mean(np.abs(z["amp"]) ** 2))) <= 1e-4
    assert abs(1 - nrm) <= TOL["c64"]
    assert abs(e - float(z["energy"])) <= TOL["c64"] * 28


@pytest.mark.parametrize("fuse_k", [4, 0])
def test_layered_n28_forward_against_oracle_run(golden28, fuse_k):
    from paper_2202_07017_gb300 import State
    c, theta = W.random_layered(28, 40, 1004)
    assert int(golden28["gates"]) == len(c.gates) == 3900
    assert abs(float(golden28["norm"]) - 1) <= 1e-12   # the oracle's own unitarity
    st = State(28, "c64").init(0)
    try:
        st.apply_circuit(c, theta, fuse_k)
        _check28(st, golden28)
    finally:
        st.close()


def test_layered_n28_checkpointed_fused_gradient_state_and_energy(golden28):
    """sv_grad_fused with checkpoints every 10 layers: the forward state it
    leaves and the energy it returns against the oracle run."""
    from paper_2202_07017_gb300 import State
    c, theta = W.random_layered(28, 40, 1004)
    starts = [i for i, g in enumerate(c.gates) if g.kind == "RX" and g.targets == (0,)]
    st = State(28, "c64").init(0)
    try:
        e, g = st.grad(c, theta, W.sum_z(28), [starts[10], starts[20], starts[30]], fuse_k=4)
        _check28(st, golden28)
    finally:
        st.close()
    assert abs(e - float(golden28["energy"])) <= TOL["c64"] * 28
    assert g.shape == (3360,) and np.all(np.isfinite(g))


@pytest.mark.parametrize("fuse_k", [0, 4])
def test_layered_generator_n18_checkpointed_gradient(fuse_k):
    """The n = 28 gradient configuration's generator at n = 18: depth 40,
    <sum Z_i>, checkpoints every 10 layers; sampled gradients against the
    exact shift rule."""
    from paper_2202_07017_gb300 import State
    n = 18
    c, theta = W.random_layered(n, 40, 1004)
    starts = [i for i, g in enumerate(c.gates) if g.kind == "RX" and g.targets == (0,)]
    H = W.sum_z(n)
    st = State(n, "c64").init(0)
    try:
        e, g = st.grad(c, theta, H, [starts[10], starts[20], starts[30]], fuse_k=fuse_k)
    finally:
        st.close()
    ps = [0, 1, 2, 53, 700, 1079, 1080, 1500, 2000, 2157, 2158, 2159]
    ref = oracle.grad_param_shift(c, theta, H, params=ps)
    assert abs(e - oracle.energy(c, theta, H)) <= TOL["c64"] * n
    assert np.max(np.abs(g[ps] - ref[ps])) <= 1e-5 * max(1.0, np.max(np.abs(ref[ps])))
