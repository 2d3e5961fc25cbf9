"""sv_expval_noalloc: the energy entry point for callers that cannot allocate
device memory when they need it (code being captured into a CUDA graph,
where cudaMalloc is not allowed; processes whose device memory belongs to a
caching allocator or a fixed arena).  Its reduction scratch is a fixed
array inside the library, so the call itself allocates nothing.

Checked through the C ABI against sv_expval_async on the same state, for two
calls in a row (the second reuses the scratch the first left behind).  This
file is named to be collected last, and it passes both alone in a fresh
process and after the other tests."""
import ctypes

import numpy as np
import pytest

import workloads as W
from gpu_helpers import TOL, rounded

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_noalloc_energy_matches_sv_expval_on_two_calls(dtype):
    from paper_2202_07017_gb300 import State, sv
    lib = sv.load()
    n = 14
    psi = rounded(W.random_state(n, 21), dtype)
    first = W.tfim(n) + W.random_pauli_sum(n, 90, 3)      # two chunks of terms
    second = W.random_pauli_sum(n, 20, 4)                  # fewer terms next
    st = State(n, dtype).load(psi)
    stream = st.stream.cuda_stream
    ref = torch.zeros(2, dtype=torch.float64, device=st.tensor.device)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=st.tensor.device)
    try:
        for i, terms in enumerate((first, second)):
            pp = sv.pack_pauli(terms, n)
            sv.sv_expval_async(st.h, pp, ref[i:].data_ptr())
            rc = lib.sv_expval_noalloc(ctypes.c_void_p(st.tensor.data_ptr()), n, st.code,
                                       ctypes.byref(pp.s), ctypes.c_void_p(out[i:].data_ptr()),
                                       ctypes.c_void_p(stream))
            assert rc == 0, sv.sv_last_error()
        torch.cuda.synchronize()
        got, want = out.cpu().numpy(), ref.cpu().numpy()
    finally:
        st.close()
    for i, terms in enumerate((first, second)):
        scale = sum(abs(c) for c, _ in terms)
        assert abs(got[i] - want[i]) <= TOL[dtype] * scale, (i, got[i], want[i])


def test_noalloc_rejects_too_many_terms():
    from paper_2202_07017_gb300 import C64, State, sv
    lib = sv.load()
    n = 6
    st = State(n, "c64").init(0)
    out = torch.zeros(1, dtype=torch.float64, device=st.tensor.device)
    too_many = [(1.0, ((0, "Z"),))] * 1025
    pp = sv.pack_pauli(too_many, n)
    try:
        rc = lib.sv_expval_noalloc(ctypes.c_void_p(st.tensor.data_ptr()), n, C64,
                                   ctypes.byref(pp.s), ctypes.c_void_p(out.data_ptr()), None)
    finally:
        st.close()
    assert rc == 1
    assert "1024" in sv.sv_last_error()
