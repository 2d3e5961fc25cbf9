"""Failure paths on the GPU without a GPU fault: an allocation the device
cannot hold returns SV_ERR_OOM and leaves the library usable; a bulk-copy
pass whose barrier can never complete gives up after its bounded wait, the
host reads SV_ERR_TIMEOUT from sv_sync, the state is unchanged and the
context keeps working; the guard regions around a state report a write
outside it."""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import TOL, max_err

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SV_ERR_OOM, SV_ERR_TIMEOUT = 2, 4


def test_allocation_beyond_the_device_returns_oom():
    from paper_2202_07017_gb300 import C128, SvError, State, sv_alloc, sv_free
    held = []
    try:
        with pytest.raises(SvError) as err:
            for _ in range(3):  # 256 GiB each: at most one fits on a 288 GB part
                held.append(sv_alloc(34, C128))
        assert err.value.status == SV_ERR_OOM
    finally:
        for h in held:
            sv_free(h)
    st = State(12, "c64").init(5)  # the library still works
    try:
        v = st.numpy()
        assert v[5] == 1 and np.count_nonzero(v) == 1
    finally:
        st.close()


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_bounded_wait_gives_up_and_the_context_survives(dtype):
    from paper_2202_07017_gb300 import SvError, State, sv_selftest_wait
    n = 14
    psi = W.random_state(n, 8)
    c, theta = W.random_layered(n, 2, 4)
    st = State(n, dtype).load(psi)
    try:
        before = st.numpy()
        sv_selftest_wait(st.h)
        with pytest.raises(SvError) as err:
            st.sync()
        assert err.value.status == SV_ERR_TIMEOUT
        assert np.array_equal(st.numpy(), before)    # nothing was stored
        st.sync()                                     # the status was cleared
        st.apply_circuit(c, theta, 4)                 # fused passes work again
        ref = State(n, dtype).load(psi)
        try:
            ref.apply_circuit(c, theta, 0)
            assert max_err(st.numpy(), ref.numpy()) <= TOL[dtype]
        finally:
            ref.close()
    finally:
        st.close()


def test_bounded_wait_selftest_rejects_small_states():
    from paper_2202_07017_gb300 import SvError, State, sv_selftest_wait
    st = State(6, "c64").init(0)
    try:
        with pytest.raises(SvError):
            sv_selftest_wait(st.h)
    finally:
        st.close()


def test_guard_regions_report_a_write_outside_the_state():
    """The 4 KiB guards around an sv_alloc state: clean after a circuit, and a
    host-issued write of 16 bytes just below the state (inside the guard,
    within the allocation) is reported by sv_check_guards."""
    import ctypes
    from paper_2202_07017_gb300 import SvError, State, sv_info
    n = 12
    c, theta = W.random_layered(n, 4, 3)
    st = State(n, "c64", guarded=True).init(0)
    try:
        st.apply_circuit(c, theta, 4)
        st.check_guards()
        ptr = sv_info(st.h)[0]
        rt = ctypes.CDLL("libcudart.so.13")
        torch.cuda.synchronize()
        assert rt.cudaMemset(ctypes.c_void_p(ptr - 16), 0, ctypes.c_size_t(16)) == 0
        torch.cuda.synchronize()
        with pytest.raises(SvError):
            st.check_guards()
    finally:
        st.close()
