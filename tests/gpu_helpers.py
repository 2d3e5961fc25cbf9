"""Shared helpers of the GPU parity tests (imported only by tests marked gpu)."""
import os

import numpy as np

import oracle

# max |delta psi| and |1 - ||psi||^2| bars per state precision
TOL = {"c64": 1e-5, "c128": 1e-12}
NP_DTYPE = {"c64": np.complex64, "c128": np.complex128}


def oracle_threads():
    oracle.set_threads(os.cpu_count() or 1)


def gpu_run(circuit, theta, psi0, dtype, fuse_k=0, basis=None):
    """Run `circuit` on the GPU from psi0 (or |basis>) and return the state."""
    from paper_2202_07017_gb300 import State
    st = State(circuit.n_qubits, dtype, guarded=True)
    try:
        if psi0 is None:
            st.init(basis or 0)
        else:
            st.load(np.asarray(psi0, NP_DTYPE[dtype]))
        st.apply_circuit(circuit, theta, fuse_k)
        st.check_guards()  # nothing written outside the state
        return st.numpy()
    finally:
        st.close()


def rounded(psi, dtype):
    """psi rounded to the GPU state's precision and back to complex128, so
    both sides start from identical amplitudes."""
    return np.asarray(psi, NP_DTYPE[dtype]).astype(np.complex128)


def max_err(a, b):
    return float(np.max(np.abs(np.asarray(a, np.complex128) - np.asarray(b, np.complex128))))
