"""GB300 state-vector simulation of circuits (Sec. 2, Eq. 1 of the Qibo 0.1.7
paper): hand-written CUDA kernels for sm_103a behind the C ABI of
include/sv.h, with PyTorch providing device memory, streams and autograd.

    from paper_2202_07017_gb300 import State, Energy
    st = State(20, "c64")                 # torch-owned device buffer
    st.init(0)
    st.apply_circuit(circuit, theta)      # one kernel per gate (fuse_k = 0)
    e = st.expval(hamiltonian)            # fp64-accumulated <psi|H|psi>
"""
from __future__ import annotations

import numpy as np

from .sv import (C64, C128, EXPORTS, PackedBatch, sv_batch_create, sv_batch_free, sv_batch_grad,
                 sv_batch_plan,
                 sv_batch_info, sv_batch_kernel, sv_batch_run, sv_batch_run_graph, PackedCircuit, PackedPauli, SvError, load, pack_circuit,
                 pack_pauli, sv_adjoint, sv_alloc, sv_apply_circuit, sv_apply_gate,
                 sv_apply_pauli_sum, sv_copy, sv_download, sv_expval, sv_expval_async, sv_free,
                 sv_fusion_plan, sv_fusion_plan_reverse, sv_pauli_rotation, sv_probabilities, sv_sample, sv_trotter,
                 sv_grad, sv_grad_fused, sv_info, sv_init, sv_last_error, sv_launch_count, sv_norm, sv_profile_start,
                 sv_profile_stop, sv_set_stream, sv_set_rounding,
                 sv_sync, sv_upload, sv_version, sv_wrap, sv_host_alloc, sv_host_free,
                 sv_selftest_wait, sv_check_guards)

__all__ = ["State", "Batch", "Energy", "energy", "C64", "C128", "SvError", "pack_circuit", "pack_pauli",
           "load"] + list(EXPORTS)


def _dtype_code(dtype) -> int:
    if dtype in ("c64", "complex64", C64):
        return C64
    if dtype in ("c128", "complex128", C128):
        return C128
    raise ValueError(f"dtype {dtype!r}: expected c64 or c128")


class State:
    """A 2^n-amplitude state in a torch CUDA tensor, wrapped by an sv handle
    bound to a torch stream (the current stream by default).  guarded=True
    lets the library allocate the state instead (no torch tensor), between
    guard regions that check_guards() verifies."""

    def __init__(self, n_qubits: int, dtype="c64", device="cuda", stream=None, guarded=False):
        import torch
        self.n = int(n_qubits)
        self.code = _dtype_code(dtype)
        if guarded:
            self.tensor = None
            self.stream = stream if stream is not None else torch.cuda.current_stream()
            self.h = sv_alloc(self.n, self.code, self.stream.cuda_stream)
            return
        tdt = torch.complex64 if self.code == C64 else torch.complex128
        self.tensor = torch.empty(1 << self.n, dtype=tdt, device=device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.tensor.device)
        self.h = sv_wrap(self.tensor.data_ptr(), self.n, self.code, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "h", None):
            sv_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self.stream = stream
        sv_set_stream(self.h, stream.cuda_stream)

    def set_rounding(self, mode):
        """Complex64 rounding: "default" or "dithered" (see sv_set_rounding)."""
        sv_set_rounding(self.h, mode)
        return self

    def init(self, basis_index: int = 0):
        sv_init(self.h, basis_index)
        return self

    def load(self, amplitudes: np.ndarray):
        a = np.ascontiguousarray(amplitudes,
                                 dtype=np.complex64 if self.code == C64 else np.complex128)
        sv_upload(self.h, a)
        sv_sync(self.h)
        return self

    def numpy(self) -> np.ndarray:
        out = np.empty(1 << self.n, np.complex64 if self.code == C64 else np.complex128)
        sv_download(self.h, out)
        return out

    def apply_gate(self, targets, controls, matrix):
        sv_apply_gate(self.h, targets, controls, matrix)
        return self

    def apply_circuit(self, circuit, theta=None, fuse_k: int = 0):
        sv_apply_circuit(self.h, circuit, theta, fuse_k)
        return self

    def norm(self) -> float:
        return sv_norm(self.h)

    def pauli_rotation(self, term_ops, theta):
        sv_pauli_rotation(self.h, term_ops, theta)
        return self

    def trotter(self, terms, t, steps, order=1):
        sv_trotter(self.h, terms, t, steps, order)
        return self

    def probabilities(self, qubits):
        return sv_probabilities(self.h, qubits)

    def sample(self, qubits, uniforms):
        return sv_sample(self.h, qubits, uniforms)

    def expval(self, terms) -> float:
        return sv_expval(self.h, pack_pauli(terms, self.n))

    def adjoint(self, circuit, theta, terms):
        return sv_adjoint(self.h, circuit, theta, pack_pauli(terms, self.n))

    def grad(self, circuit, theta, terms, checkpoint_gates=(), fuse_k=0):
        """Forward pass from the current state plus adjoint gradient; fuse_k >= 2
        runs both as fused qubit-block passes."""
        if fuse_k:
            return sv_grad_fused(self.h, circuit, theta, pack_pauli(terms, self.n),
                                 checkpoint_gates, fuse_k)
        return sv_grad(self.h, circuit, theta, pack_pauli(terms, self.n), checkpoint_gates)

    def sync(self):
        sv_sync(self.h)

    def check_guards(self):
        """Raise SvError if a kernel wrote outside the state or its work states."""
        sv_check_guards(self.h)


class Batch:
    """Energies and adjoint gradients of many small circuits in one persistent
    launch (complex64 - or real fp32 states for a batch of real gates and
    terms - with fp64 accumulation).  theta / energy / grad are torch
    CUDA float64 tensors; parameters are packed per item in item order."""

    def __init__(self, circuits, hamiltonians, item_circuit, tune=True):
        self.h, self.packed = sv_batch_create(circuits, hamiltonians, item_circuit, tune)
        self.k, self.threads, self.blocks, self.total_params = sv_batch_info(self.h)
        self.cluster, self.smem_states, self.real = sv_batch_kernel(self.h)
        self.n_items = len(self.packed.items)

    def run(self, theta, energy=None, grad=None, graph: bool = False, stream=None):
        import torch
        dev = theta.device
        if energy is None:
            energy = torch.empty(self.n_items, dtype=torch.float64, device=dev)
        if grad is None:
            grad = torch.empty(max(1, self.total_params), dtype=torch.float64, device=dev)
        st = (stream or torch.cuda.current_stream(dev)).cuda_stream
        fn = sv_batch_run_graph if graph else sv_batch_run
        fn(self.h, theta.data_ptr(), energy.data_ptr(), grad.data_ptr(), st)
        return energy, grad

    def close(self):
        if getattr(self, "h", None):
            sv_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _energy_fn():
    import torch

    class Energy(torch.autograd.Function):
        """E(theta) = <psi(theta)|H|psi(theta)>, psi(theta) = U(theta)|basis>.

        forward: when theta requires a gradient, sv_grad (fuse_k = 0) or
        sv_grad_fused runs the circuit from |basis> and the adjoint sweep at
        once (checkpoints: gate indices whose forward states the sweep
        restores) and keeps dE/dtheta for backward; otherwise sv_init +
        sv_apply_circuit + sv_expval.  backward: the kept gradient times the
        incoming one.  The gate matrices are built on the host from theta in
        fp64, so theta is copied to the host once per forward."""

        @staticmethod
        def forward(ctx, theta, state, circuit, terms, basis=0, fuse_k=0, checkpoints=()):
            th = theta.detach().to("cpu", torch.float64).numpy().copy()
            pc = pack_circuit(circuit)
            pp = pack_pauli(terms, state.n)
            state.init(basis)
            if ctx.needs_input_grad[0]:
                if fuse_k:
                    e, g = sv_grad_fused(state.h, pc, th, pp, list(checkpoints), fuse_k)
                else:
                    e, g = sv_grad(state.h, pc, th, pp, list(checkpoints))
                ctx.grad = torch.from_numpy(np.asarray(g, np.float64)).to(theta.device)
            else:
                sv_apply_circuit(state.h, pc, th, fuse_k)
                e = sv_expval(state.h, pp)
                ctx.grad = None
            return torch.tensor(e, dtype=torch.float64, device=theta.device)

        @staticmethod
        def backward(ctx, grad_out):
            gt = None if ctx.grad is None else ctx.grad * grad_out
            return gt, None, None, None, None, None, None

    return Energy


class _Lazy:
    _cls = None

    def __getattr__(self, name):
        if _Lazy._cls is None:
            _Lazy._cls = _energy_fn()
        return getattr(_Lazy._cls, name)


Energy = _Lazy()


def energy(theta, state: State, circuit, terms, basis: int = 0, fuse_k: int = 0,
           checkpoints=()):
    """Differentiable energy (torch scalar) via the adjoint kernels; fuse_k >= 2
    runs the circuit and the reverse sweep as fused qubit-block passes."""
    return Energy.apply(theta, state, circuit, terms, basis, fuse_k, tuple(checkpoints))
