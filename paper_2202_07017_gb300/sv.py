"""Thin Python binding of libsv (include/sv.h): same names, argument
marshalling only.  Every step of the computation runs in the library's CUDA
kernels; if libsv.so cannot be built or loaded this module raises.

Records accepted by `pack_circuit` are any objects with the attributes
kind (str: H X Y Z RX RY RZ U1 SWAP MATRIX), targets, controls, param, angle
and matrix, e.g. the seeded records of the `workloads` module.  Pauli sums
are lists of (coeff, ((qubit, 'X'|'Y'|'Z'), ...)).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple

import numpy as np

from . import _build

C64, C128 = 0, 1
KIND_CODE = {"H": 0, "X": 1, "Y": 2, "Z": 3, "RX": 4, "RY": 5, "RZ": 6, "U1": 7,
             "SWAP": 8, "MATRIX": 9, "PAULI": 10}
LETTER_CODE = {"X": 1, "Y": 2, "Z": 3}
STATUS = {0: "SV_OK", 1: "SV_ERR_INVALID", 2: "SV_ERR_OOM", 3: "SV_ERR_CUDA",
          4: "SV_ERR_TIMEOUT", 5: "SV_ERR_UNSUPPORTED"}

c_i32, c_i64, c_u64, c_dbl, c_vp = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                    ctypes.c_double, ctypes.c_void_p)


class SvGate(ctypes.Structure):
    _fields_ = [("kind", c_i32), ("n_tar", c_i32), ("n_ctrl", c_i32), ("param", c_i32),
                ("targets", c_i32 * 5), ("controls", c_i32 * 33), ("angle", c_dbl),
                ("mat_off", c_i64), ("paulis", c_i32), ("reserved", c_i32)]


class SvCircuit(ctypes.Structure):
    _fields_ = [("n_qubits", c_i32), ("n_gates", c_i32), ("n_params", c_i32),
                ("gates", ctypes.POINTER(SvGate)), ("mat_pool", ctypes.POINTER(c_dbl))]


class SvPauliSum(ctypes.Structure):
    _fields_ = [("n_terms", c_i32), ("xmask", ctypes.POINTER(c_u64)),
                ("zmask", ctypes.POINTER(c_u64)), ("coeff", ctypes.POINTER(c_dbl))]


class SvError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


EXPORTS = ("sv_alloc", "sv_wrap", "sv_free", "sv_set_stream", "sv_set_rounding", "sv_info", "sv_init",
           "sv_upload", "sv_download", "sv_host_alloc", "sv_host_free", "sv_copy", "sv_apply_gate", "sv_apply_circuit",
           "sv_norm", "sv_expval", "sv_expval_async", "sv_apply_pauli_sum", "sv_adjoint",
           "sv_grad", "sv_grad_fused", "sv_sync", "sv_selftest_wait", "sv_check_guards", "sv_last_error", "sv_launch_count", "sv_version",
           "sv_profile_start", "sv_profile_stop", "sv_fusion_plan", "sv_fusion_plan_reverse",
           "sv_expval_noalloc",
           "sv_probabilities", "sv_sample", "sv_pauli_rotation", "sv_trotter",
           "sv_batch_create", "sv_batch_plan", "sv_batch_info", "sv_batch_kernel", "sv_batch_run", "sv_batch_run_graph", "sv_batch_grad",
           "sv_batch_free")

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build: bool = True):
    """Load libsv.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libsv.so is not built; run __graft_entry__.build()")
    L = ctypes.CDLL(_build.LIB)
    P = ctypes.POINTER
    sig = {
        "sv_alloc": [ctypes.c_int, ctypes.c_int, c_vp, P(c_vp)],
        "sv_wrap": [c_vp, ctypes.c_int, ctypes.c_int, c_vp, P(c_vp)],
        "sv_free": [c_vp],
        "sv_set_stream": [c_vp, c_vp],
        "sv_set_rounding": [c_vp, ctypes.c_int],
        "sv_info": [c_vp, P(c_vp), P(ctypes.c_int), P(ctypes.c_int)],
        "sv_init": [c_vp, c_u64],
        "sv_upload": [c_vp, c_vp],
        "sv_host_alloc": [ctypes.c_size_t, P(c_vp)],
        "sv_host_free": [c_vp],
        "sv_download": [c_vp, c_vp],
        "sv_copy": [c_vp, c_vp],
        "sv_apply_gate": [c_vp, P(ctypes.c_int), ctypes.c_int, P(ctypes.c_int), ctypes.c_int,
                          P(c_dbl)],
        "sv_apply_circuit": [c_vp, P(SvCircuit), P(c_dbl), ctypes.c_int],
        "sv_norm": [c_vp, P(c_dbl)],
        "sv_expval": [c_vp, P(SvPauliSum), P(c_dbl)],
        "sv_expval_async": [c_vp, P(SvPauliSum), c_vp],
        "sv_apply_pauli_sum": [c_vp, c_vp, P(SvPauliSum)],
        "sv_adjoint": [c_vp, P(SvCircuit), P(c_dbl), P(SvPauliSum), P(c_dbl), P(c_dbl)],
        "sv_grad": [c_vp, P(SvCircuit), P(c_dbl), P(SvPauliSum), P(c_i32), ctypes.c_int,
                    P(c_dbl), P(c_dbl)],
        "sv_grad_fused": [c_vp, P(SvCircuit), P(c_dbl), P(SvPauliSum), P(c_i32), ctypes.c_int,
                          ctypes.c_int, P(c_dbl), P(c_dbl)],
        "sv_sync": [c_vp],
        "sv_selftest_wait": [c_vp],
        "sv_check_guards": [c_vp],
        "sv_profile_start": [],
        "sv_pauli_rotation": [c_vp, c_u64, c_u64, c_dbl],
        "sv_trotter": [c_vp, P(SvPauliSum), c_dbl, ctypes.c_int, ctypes.c_int],
        "sv_probabilities": [c_vp, P(ctypes.c_int), ctypes.c_int, P(c_dbl)],
        "sv_sample": [c_vp, P(ctypes.c_int), ctypes.c_int, c_i64, P(c_dbl), P(c_u64)],
        "sv_batch_create": [P(SvCircuit), P(SvPauliSum), ctypes.c_int, P(c_i32), ctypes.c_int,
                            ctypes.c_int, P(c_vp)],
        "sv_batch_plan": [P(SvCircuit), P(SvPauliSum), ctypes.c_int, ctypes.c_int, P(c_i32)],
        "sv_batch_info": [c_vp, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int)],
        "sv_batch_kernel": [c_vp, P(ctypes.c_int), P(ctypes.c_int), P(ctypes.c_int)],
        "sv_batch_run": [c_vp, c_vp, c_vp, c_vp, c_vp],
        "sv_batch_run_graph": [c_vp, c_vp, c_vp, c_vp, c_vp],
        "sv_batch_grad": [P(SvCircuit), P(SvPauliSum), ctypes.c_int, P(c_i32), ctypes.c_int,
                          P(c_dbl), c_vp, P(c_dbl), P(c_dbl)],
        "sv_batch_free": [c_vp],
        "sv_expval_noalloc": [c_vp, ctypes.c_int, ctypes.c_int, P(SvPauliSum), c_vp, c_vp],
        "sv_fusion_plan": [P(SvCircuit), P(c_dbl), ctypes.c_int, ctypes.c_int, P(c_i32), P(c_i32),
                           P(c_i32), P(c_i32)],
        "sv_fusion_plan_reverse": [P(SvCircuit), P(c_dbl), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, P(c_i32), P(c_i32), P(c_i32)],
        "sv_profile_stop": [ctypes.c_char_p, ctypes.c_size_t],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.sv_last_error.restype = ctypes.c_char_p
    L.sv_last_error.argtypes = []
    L.sv_launch_count.restype = c_u64
    L.sv_launch_count.argtypes = []
    L.sv_version.restype = ctypes.c_int
    L.sv_version.argtypes = []
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        raise SvError(status, load().sv_last_error().decode())


# ---- marshalling ----------------------------------------------------------------------
class PackedCircuit:
    """An sv_circuit plus the numpy buffers it points into."""

    def __init__(self, circuit):
        gates = list(circuit.gates)
        n = circuit.n_qubits
        self.n_qubits = n
        self.n_params = int(getattr(circuit, "n_params", 0))
        self.n_gates = len(gates)
        self._arr = (SvGate * max(1, len(gates)))()
        pool = []
        off = 0
        for i, g in enumerate(gates):
            r = self._arr[i]
            r.kind = KIND_CODE[g.kind]
            r.n_tar = len(g.targets)
            r.n_ctrl = len(g.controls)
            if r.n_tar > 5 or r.n_ctrl > 33:
                raise SvError(1, f"gate {i}: too many targets or controls")
            for j, t in enumerate(g.targets):
                r.targets[j] = int(t)
            for j, c in enumerate(g.controls):
                r.controls[j] = int(c)
            r.param = int(g.param)
            r.angle = float(g.angle)
            letters = getattr(g, "paulis", "")
            if len(letters) > 5:
                raise SvError(1, f"gate {i}: too many Pauli letters")
            r.paulis = sum(LETTER_CODE[L] << (2 * j) for j, L in enumerate(letters))
            if g.kind == "MATRIX":
                m = np.ascontiguousarray(g.matrix, dtype=np.complex128).ravel()
                r.mat_off = off
                pool.append(m)
                off += m.size
        self._pool = (np.concatenate(pool) if pool else np.zeros(1, np.complex128)).view(np.float64)
        self.c = SvCircuit(n, len(gates), self.n_params,
                           ctypes.cast(self._arr, ctypes.POINTER(SvGate)),
                           self._pool.ctypes.data_as(ctypes.POINTER(c_dbl)))


def pack_circuit(circuit) -> PackedCircuit:
    return circuit if isinstance(circuit, PackedCircuit) else PackedCircuit(circuit)


class PackedPauli:
    """An sv_pauli_sum (masks in amplitude-index bits: qubit q -> bit n-1-q)."""

    def __init__(self, terms, n: int):
        self.n = n
        self.x = np.zeros(max(1, len(terms)), np.uint64)
        self.z = np.zeros(max(1, len(terms)), np.uint64)
        self.c = np.zeros(max(1, len(terms)), np.float64)
        for k, (coeff, ops) in enumerate(terms):
            x = z = 0
            for q, L in ops:
                if not 0 <= int(q) < n or L not in ("X", "Y", "Z"):
                    raise SvError(1, f"Pauli term {k}: bad factor {L}{q} for {n} qubits")
                b = 1 << (n - 1 - int(q))
                if L in "XY":
                    x |= b
                if L in "ZY":
                    z |= b
            self.x[k], self.z[k], self.c[k] = x, z, coeff
        P = ctypes.POINTER
        self.s = SvPauliSum(len(terms), self.x.ctypes.data_as(P(c_u64)),
                            self.z.ctypes.data_as(P(c_u64)), self.c.ctypes.data_as(P(c_dbl)))


def pack_pauli(terms, n: int) -> PackedPauli:
    return terms if isinstance(terms, PackedPauli) else PackedPauli(terms, n)


def _theta_ptr(theta):
    if theta is None or len(theta) == 0:
        return None, None
    a = np.ascontiguousarray(theta, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(c_dbl))


# ---- the C-ABI, name for name ------------------------------------------------------------
def sv_alloc(n_qubits: int, dtype: int = C64, stream: int = 0) -> int:
    h = c_vp()
    _check(load().sv_alloc(n_qubits, dtype, c_vp(stream), ctypes.byref(h)))
    return h.value


def sv_wrap(dev_ptr: int, n_qubits: int, dtype: int = C64, stream: int = 0) -> int:
    h = c_vp()
    _check(load().sv_wrap(c_vp(dev_ptr), n_qubits, dtype, c_vp(stream), ctypes.byref(h)))
    return h.value


def sv_free(h: int) -> None:
    _check(load().sv_free(c_vp(h)))


def sv_set_stream(h: int, stream: int) -> None:
    _check(load().sv_set_stream(c_vp(h), c_vp(stream)))


ROUNDING = {"default": 0, "dithered": 1}


def sv_set_rounding(h: int, mode) -> None:
    """Complex64 rounding mode: "default" (0) or "dithered" (1)."""
    _check(load().sv_set_rounding(c_vp(h), int(ROUNDING.get(mode, mode))))


def sv_info(h: int) -> Tuple[int, int, int]:
    p, n, d = c_vp(), ctypes.c_int(), ctypes.c_int()
    _check(load().sv_info(c_vp(h), ctypes.byref(p), ctypes.byref(n), ctypes.byref(d)))
    return p.value, n.value, d.value


def sv_init(h: int, basis_index: int = 0) -> None:
    _check(load().sv_init(c_vp(h), c_u64(basis_index)))


def sv_host_alloc(n_elems: int, dtype=np.complex64) -> np.ndarray:
    """A numpy array over a page-locked buffer from the library's CUDA runtime
    (free it with sv_host_free(array))."""
    nbytes = int(n_elems) * np.dtype(dtype).itemsize
    p = c_vp()
    _check(load().sv_host_alloc(ctypes.c_size_t(nbytes), ctypes.byref(p)))
    buf = (ctypes.c_char * nbytes).from_address(p.value)
    return np.frombuffer(buf, dtype=dtype, count=int(n_elems))


def sv_host_free(arr: np.ndarray) -> None:
    _check(load().sv_host_free(c_vp(arr.ctypes.data)))


def sv_upload(h: int, host: np.ndarray) -> None:
    _check(load().sv_upload(c_vp(h), c_vp(host.ctypes.data)))


def sv_download(h: int, host: np.ndarray) -> None:
    _check(load().sv_download(c_vp(h), c_vp(host.ctypes.data)))


def sv_copy(dst: int, src: int) -> None:
    _check(load().sv_copy(c_vp(dst), c_vp(src)))


def sv_apply_gate(h: int, targets: Sequence[int], controls: Sequence[int],
                  matrix: np.ndarray) -> None:
    t = (ctypes.c_int * max(1, len(targets)))(*targets)
    c = (ctypes.c_int * max(1, len(controls)))(*controls)
    m = np.ascontiguousarray(matrix, dtype=np.complex128).view(np.float64)
    _check(load().sv_apply_gate(c_vp(h), t, len(targets), c, len(controls),
                                m.ctypes.data_as(ctypes.POINTER(c_dbl))))


def sv_apply_circuit(h: int, circuit, theta=None, fuse_k: int = 0) -> None:
    pc = pack_circuit(circuit)
    keep, tp = _theta_ptr(theta)
    _check(load().sv_apply_circuit(c_vp(h), ctypes.byref(pc.c), tp, int(fuse_k)))


def sv_fusion_plan(circuit, theta=None, dtype: int = C64, fuse_k: int = 4):
    """Dry run of the fusion planner: (order, pass_of, n_passes, staged masks)."""
    pc = pack_circuit(circuit)
    keep, tp = _theta_ptr(theta)
    ng = max(1, pc.n_gates)
    order = np.zeros(ng, np.int32)
    pass_of = np.zeros(ng, np.int32)
    staged = np.zeros(2 * ng, np.int32)
    npass = c_i32()
    P = ctypes.POINTER
    _check(load().sv_fusion_plan(ctypes.byref(pc.c), tp, dtype, fuse_k,
                                 order.ctypes.data_as(P(c_i32)), pass_of.ctypes.data_as(P(c_i32)),
                                 ctypes.byref(npass), staged.ctypes.data_as(P(c_i32))))
    p = npass.value
    masks = [(int(staged[2 * i]) & 0xffffffff) | ((int(staged[2 * i + 1]) & 0xffffffff) << 32)
             for i in range(p)]
    return order[:pc.n_gates], pass_of[:pc.n_gates], p, masks


def sv_fusion_plan_reverse(circuit, theta=None, dtype: int = C64, fuse_k: int = 4, lo: int = 0,
                           hi=None):
    """Dry run of the reverse-sweep planner over gates [lo, hi): (events, n_passes),
    events an (n, 4) array of (kind 0 un-apply / 1 gradient, gate, pass, evaluation)."""
    pc = pack_circuit(circuit)
    keep, tp = _theta_ptr(theta)
    hi = pc.n_gates if hi is None else int(hi)
    ev = np.zeros(max(1, 8 * (hi - lo)), np.int32)
    nev, npass = c_i32(), c_i32()
    P = ctypes.POINTER
    _check(load().sv_fusion_plan_reverse(ctypes.byref(pc.c), tp, dtype, fuse_k, int(lo), hi,
                                         ev.ctypes.data_as(P(c_i32)), ctypes.byref(nev),
                                         ctypes.byref(npass)))
    return ev[:4 * nev.value].reshape(-1, 4), npass.value


def sv_pauli_rotation(h: int, term_ops, theta: float) -> None:
    """psi <- exp(-i theta P), P = ((qubit, letter), ...)."""
    pp = pack_pauli([(1.0, tuple(term_ops))], _n_of(h))
    _check(load().sv_pauli_rotation(c_vp(h), c_u64(int(pp.x[0])), c_u64(int(pp.z[0])),
                                    float(theta)))


def sv_trotter(h: int, terms, t: float, steps: int, order: int = 1) -> None:
    pp = pack_pauli(terms, _n_of(h))
    _check(load().sv_trotter(c_vp(h), ctypes.byref(pp.s), float(t), int(steps), int(order)))


def sv_probabilities(h: int, qubits: Sequence[int]) -> np.ndarray:
    q = (ctypes.c_int * max(1, len(qubits)))(*qubits)
    out = np.zeros(1 << len(qubits), np.float64)
    _check(load().sv_probabilities(c_vp(h), q, len(qubits),
                                   out.ctypes.data_as(ctypes.POINTER(c_dbl))))
    return out


def sv_sample(h: int, qubits: Sequence[int], uniforms) -> np.ndarray:
    q = (ctypes.c_int * max(1, len(qubits)))(*qubits)
    u = np.ascontiguousarray(uniforms, dtype=np.float64)
    out = np.zeros(max(1, len(u)), np.uint64)
    _check(load().sv_sample(c_vp(h), q, len(qubits), len(u),
                            u.ctypes.data_as(ctypes.POINTER(c_dbl)),
                            out.ctypes.data_as(ctypes.POINTER(c_u64))))
    return out[:len(u)]


def sv_norm(h: int) -> float:
    out = c_dbl()
    _check(load().sv_norm(c_vp(h), ctypes.byref(out)))
    return out.value


def _n_of(h: int) -> int:
    return sv_info(h)[1]


def sv_expval(h: int, terms) -> float:
    pp = pack_pauli(terms, _n_of(h))
    out = c_dbl()
    _check(load().sv_expval(c_vp(h), ctypes.byref(pp.s), ctypes.byref(out)))
    return out.value


def sv_expval_async(h: int, terms, dev_out_ptr: int) -> None:
    pp = pack_pauli(terms, _n_of(h))
    _check(load().sv_expval_async(c_vp(h), ctypes.byref(pp.s), c_vp(dev_out_ptr)))


def sv_expval_noalloc(dev_state: int, n_qubits: int, dtype: int, terms, dev_out: int,
                      stream: int = 0) -> None:
    """Allocation-free <psi|H|psi> into the device double at dev_out (no sync)."""
    pp = pack_pauli(terms, n_qubits)
    _check(load().sv_expval_noalloc(c_vp(dev_state), n_qubits, dtype, ctypes.byref(pp.s),
                                    c_vp(dev_out), c_vp(stream)))


def sv_apply_pauli_sum(out: int, inp: int, terms) -> None:
    pp = pack_pauli(terms, _n_of(inp))
    _check(load().sv_apply_pauli_sum(c_vp(out), c_vp(inp), ctypes.byref(pp.s)))


def sv_adjoint(h: int, circuit, theta, terms) -> Tuple[float, np.ndarray]:
    pc = pack_circuit(circuit)
    pp = pack_pauli(terms, pc.n_qubits)
    keep, tp = _theta_ptr(theta)
    e = c_dbl()
    g = np.zeros(max(1, pc.n_params), np.float64)
    _check(load().sv_adjoint(c_vp(h), ctypes.byref(pc.c), tp, ctypes.byref(pp.s),
                             ctypes.byref(e), g.ctypes.data_as(ctypes.POINTER(c_dbl))))
    return e.value, g[:pc.n_params]


def sv_grad(h: int, circuit, theta, terms, checkpoint_gates: Sequence[int] = ()) -> Tuple[float, np.ndarray]:
    pc = pack_circuit(circuit)
    pp = pack_pauli(terms, pc.n_qubits)
    keep, tp = _theta_ptr(theta)
    ck = np.ascontiguousarray(list(checkpoint_gates) or [0], dtype=np.int32)
    e = c_dbl()
    g = np.zeros(max(1, pc.n_params), np.float64)
    _check(load().sv_grad(c_vp(h), ctypes.byref(pc.c), tp, ctypes.byref(pp.s),
                          ck.ctypes.data_as(ctypes.POINTER(c_i32)), len(checkpoint_gates),
                          ctypes.byref(e), g.ctypes.data_as(ctypes.POINTER(c_dbl))))
    return e.value, g[:pc.n_params]


def sv_grad_fused(h: int, circuit, theta, terms, checkpoint_gates: Sequence[int] = (),
                  fuse_k: int = 4) -> Tuple[float, np.ndarray]:
    """sv_grad with the forward circuit and the reverse sweep in fused passes."""
    pc = pack_circuit(circuit)
    pp = pack_pauli(terms, pc.n_qubits)
    keep, tp = _theta_ptr(theta)
    ck = np.ascontiguousarray(list(checkpoint_gates) or [0], dtype=np.int32)
    e = c_dbl()
    g = np.zeros(max(1, pc.n_params), np.float64)
    _check(load().sv_grad_fused(c_vp(h), ctypes.byref(pc.c), tp, ctypes.byref(pp.s),
                                ck.ctypes.data_as(ctypes.POINTER(c_i32)), len(checkpoint_gates),
                                int(fuse_k), ctypes.byref(e),
                                g.ctypes.data_as(ctypes.POINTER(c_dbl))))
    return e.value, g[:pc.n_params]


def sv_sync(h: int) -> None:
    _check(load().sv_sync(c_vp(h)))


def sv_selftest_wait(h: int) -> None:
    _check(load().sv_selftest_wait(c_vp(h)))


def sv_check_guards(h: int) -> None:
    """Raise SvError if a kernel wrote into a guard region around the state."""
    _check(load().sv_check_guards(c_vp(h)))


def sv_last_error() -> str:
    return load().sv_last_error().decode()


def sv_launch_count() -> int:
    return int(load().sv_launch_count())


def sv_version() -> int:
    return int(load().sv_version())


def sv_profile_start() -> None:
    _check(load().sv_profile_start())


def sv_profile_stop() -> dict:
    """{kernel name: (launches, total ms)} since sv_profile_start()."""
    buf = ctypes.create_string_buffer(1 << 16)
    _check(load().sv_profile_stop(buf, len(buf)))
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt, ms = line.split()
        out[name] = (int(cnt), float(ms))
    return out


# ---- batched energies and gradients ----------------------------------------------------
class PackedBatch:
    """Arrays of sv_circuit / sv_pauli_sum for a batch, plus the item map."""

    def __init__(self, circuits, hamiltonians, item_circuit):
        self.pcs = [pack_circuit(c) for c in circuits]
        self.pps = [pack_pauli(h, pc.n_qubits) for h, pc in zip(hamiltonians, self.pcs)]
        if len(self.pcs) != len(self.pps):
            raise SvError(1, "one Hamiltonian per circuit")
        self.carr = (SvCircuit * len(self.pcs))(*[pc.c for pc in self.pcs])
        self.harr = (SvPauliSum * len(self.pps))(*[pp.s for pp in self.pps])
        self.items = np.ascontiguousarray(item_circuit, dtype=np.int32)
        self.n_params = [pc.n_params for pc in self.pcs]
        self.total_params = int(sum(self.n_params[i] for i in self.items))


def sv_batch_create(circuits, hamiltonians, item_circuit, tune=False):
    """tune: False/0 default tile, True/1 autotune, 2 the two-block cluster kernel,
    3 single blocks with states in shared memory, 4 the real-amplitude kernel
    (every gate H, X, Z or RY, every term with an even number of Y factors)."""
    pb = PackedBatch(circuits, hamiltonians, item_circuit)
    h = c_vp()
    _check(load().sv_batch_create(pb.carr, pb.harr, len(pb.pcs),
                                  pb.items.ctypes.data_as(ctypes.POINTER(c_i32)), len(pb.items),
                                  int(tune), ctypes.byref(h)))
    return h.value, pb


def sv_batch_plan(circuits, hamiltonians, k: int):
    """Host-only: register groups per circuit for group width k."""
    pb = PackedBatch(circuits, hamiltonians, [0])
    out = np.zeros(len(pb.pcs), np.int32)
    _check(load().sv_batch_plan(pb.carr, pb.harr, len(pb.pcs), int(k),
                                out.ctypes.data_as(ctypes.POINTER(c_i32))))
    return out


def sv_batch_info(h: int):
    k, t, b, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().sv_batch_info(c_vp(h), ctypes.byref(k), ctypes.byref(t), ctypes.byref(b),
                                ctypes.byref(p)))
    return k.value, t.value, b.value, p.value


def sv_batch_kernel(h: int):
    """(blocks per cluster, states in shared memory, real states) of the chosen
    batch kernel."""
    c, m, r = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().sv_batch_kernel(c_vp(h), ctypes.byref(c), ctypes.byref(m), ctypes.byref(r)))
    return c.value, bool(m.value), bool(r.value)


def sv_batch_run(h: int, dev_theta: int, dev_energy: int, dev_grad: int, stream: int = 0) -> None:
    _check(load().sv_batch_run(c_vp(h), c_vp(dev_theta), c_vp(dev_energy), c_vp(dev_grad),
                               c_vp(stream)))


def sv_batch_run_graph(h: int, dev_theta: int, dev_energy: int, dev_grad: int,
                       stream: int = 0) -> None:
    _check(load().sv_batch_run_graph(c_vp(h), c_vp(dev_theta), c_vp(dev_energy),
                                     c_vp(dev_grad), c_vp(stream)))


def sv_batch_grad(circuits, hamiltonians, item_circuit, theta, stream: int = 0):
    pb = PackedBatch(circuits, hamiltonians, item_circuit)
    th = np.ascontiguousarray(theta if len(theta) else [0.0], dtype=np.float64)
    if len(theta) != pb.total_params:
        raise SvError(1, f"theta has {len(theta)} entries, the batch needs {pb.total_params}")
    e = np.zeros(len(pb.items))
    g = np.zeros(max(1, pb.total_params))
    P = ctypes.POINTER
    _check(load().sv_batch_grad(pb.carr, pb.harr, len(pb.pcs),
                                pb.items.ctypes.data_as(P(c_i32)), len(pb.items),
                                th.ctypes.data_as(P(c_dbl)), c_vp(stream),
                                e.ctypes.data_as(P(c_dbl)), g.ctypes.data_as(P(c_dbl))))
    return e, g[:pb.total_params]


def sv_batch_free(h: int) -> None:
    _check(load().sv_batch_free(c_vp(h)))
