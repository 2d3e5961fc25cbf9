"""The C ABI: libsv.so builds, loads and exports every function include/sv.h
declares; host-side validation rejects bad arguments before touching the
GPU (these calls make no CUDA call, so they run without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2202_07017_gb300 import sv

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                      "include", "sv.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sv_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_documented_calls():
    names = declared_functions()
    for must in ("sv_alloc", "sv_init", "sv_apply_gate", "sv_apply_circuit", "sv_expval",
                 "sv_grad", "sv_norm", "sv_adjoint", "sv_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = sv.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) <= set(sv.EXPORTS) | {"sv_info"}
    assert lib.sv_version() >= 100


def test_host_validation_without_gpu():
    lib = sv.load()
    h = ctypes.c_void_p()
    assert lib.sv_alloc(0, 0, None, ctypes.byref(h)) == 1
    assert "n_qubits" in sv.sv_last_error()
    assert lib.sv_alloc(35, 0, None, ctypes.byref(h)) == 1
    assert lib.sv_alloc(10, 7, None, ctypes.byref(h)) == 1
    assert lib.sv_wrap(None, 10, 0, None, ctypes.byref(h)) == 1
    assert lib.sv_wrap(ctypes.c_void_p(8), 10, 0, None, ctypes.byref(h)) == 1  # misaligned
    assert lib.sv_init(None, 0) == 1
    assert lib.sv_apply_gate(None, None, 1, None, 0, None) == 1
    assert lib.sv_norm(None, None) == 1
    assert lib.sv_set_rounding(None, 0) == 1
    assert lib.sv_free(None) == 0
    with pytest.raises(sv.SvError) as e:
        sv.sv_alloc(40)
    assert e.value.status == 1


def test_struct_layout_matches_header(tmp_path):
    """The binding's ctypes records have the sizes and field offsets that a C
    compiler gives the header's structs."""
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "sv.h"\n'
        "int main(void) {\n"
        '  printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(sv_gate), offsetof(sv_gate, angle),\n'
        "         offsetof(sv_gate, mat_off), offsetof(sv_gate, paulis), sizeof(sv_circuit),\n"
        "         sizeof(sv_pauli_sum));\n"
        "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    c_sizes = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                              text=True).stdout.split()]
    py_sizes = [ctypes.sizeof(sv.SvGate), sv.SvGate.angle.offset, sv.SvGate.mat_off.offset,
                sv.SvGate.paulis.offset, ctypes.sizeof(sv.SvCircuit),
                ctypes.sizeof(sv.SvPauliSum)]
    assert c_sizes == py_sizes


def test_pauli_masks_follow_bit_convention():
    p = sv.PackedPauli([(0.5, ((0, "X"), (2, "Y"), (3, "Z")))], 4)
    assert int(p.x[0]) == 0b1010 and int(p.z[0]) == 0b0011 and p.c[0] == 0.5
