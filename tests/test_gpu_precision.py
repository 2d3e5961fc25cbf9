"""The precision reading of the reductions over complex64 states: products of
fp32 amplitudes (relative rounding u = 2^-24 each), added per thread in a
compensated fp32 sum, the per-thread sums meeting in fp64 (blocks, then a
fixed-order finish).  Bound of that reading: |error| <= 3 u sum_x |term_x|
(one rounding of the product, 2 u for the compensated sum, independent of the
count); sum_x |term_x| <= sum_k |c_k| for a unit state.

Checked at n = 30 on a random layered state (2^30 terms per reduction)
against the oracle's fp64 pairwise sums over the same complex64 amplitudes,
beside the error that fp64 accumulation of the same fp32 products would
leave (the products formed in fp32 on the host and summed in fp64), which
is the floor any accumulation of fp32 products reaches.  The errors are
printed (pytest -s) for the record."""
import numpy as np
import pytest

import oracle
import workloads as W
from gpu_helpers import oracle_threads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

U = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def _threads():
    oracle_threads()


@pytest.fixture(scope="module")
def layered30():
    from paper_2202_07017_gb300 import State
    n = 30
    c, theta = W.random_layered(n, 2, 1030)
    st = State(n, "c64").init(0)
    try:
        st.apply_circuit(c, theta, 4)
        norm = st.norm()
        H = [(1.0, ((0, "Z"),)), (1.0, ((15, "Z"),)), (1.0, ((29, "Z"),)),
             (1.0, ((0, "Z"), (1, "Z"))), (1.0, ((14, "Z"), (15, "Z"))),
             (0.7, ((0, "X"),)), (0.7, ((15, "X"),)), (0.7, ((29, "X"),))]
        e = st.expval(H)
        e_terms = [st.expval([t]) for t in H]
        psi = st.numpy()  # complex64
    finally:
        st.close()
    return {"n": n, "psi": psi, "norm": norm, "H": H, "e": e, "e_terms": e_terms}


def test_norm_n30_within_the_bound_and_near_the_fp64_floor(layered30):
    d = layered30
    psi32 = d["psi"]
    psi = psi32.astype(np.complex128)
    ref = oracle.norm2(psi)
    re, im = psi32.real, psi32.imag
    floor = float(np.sum((re * re + im * im).astype(np.float64))) - ref  # fp32 products, fp64 sum
    err = d["norm"] - ref
    print(f"\nnorm n=30: gpu {d['norm']!r} oracle {ref!r} error {err:.3e} "
          f"(fp64 accumulation of fp32 products {floor:.3e}, bound {3 * U * ref:.3e})")
    assert abs(err) <= 3 * U * ref


def test_energy_terms_n30_within_the_bound(layered30):
    d = layered30
    psi = d["psi"].astype(np.complex128)
    ref, per_term = oracle.expval(psi, d["H"], d["n"], per_term=True)
    scale = sum(abs(c) for c, _ in d["H"])
    err = d["e"] - ref
    print(f"\nenergy n=30: gpu {d['e']!r} oracle {ref!r} error {err:.3e} (bound {3 * U * scale:.3e})")
    assert abs(err) <= 3 * U * scale
    for (c, ops), g, t in zip(d["H"], d["e_terms"], per_term):
        te = g - c * t.real
        print(f"  {c} {ops}: error {te:.3e}")
        assert abs(te) <= 3 * U * abs(c)
