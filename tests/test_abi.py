"""Host-side checks of the C ABI (no GPU needed): the library builds and loads,
exports every entry point include/*.h declares, the record layouts agree, and
argument validation rejects bad input before any device work."""
import ctypes
import glob
import os
import subprocess
import re

import numpy as np
import pytest

import workloads as w

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_2212_14201_gb300 import build
    return build()


def declared_symbols():
    syms = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        syms += re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(qs_\w+)\s*\(", text, flags=re.M)
    return sorted(set(syms))


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    syms = declared_symbols()
    assert len(syms) >= 20
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing


def test_gate_codes_and_layouts_agree_with_header():
    text = open(os.path.join(ROOT, "include", "qsim.h")).read()
    for name, code in w.GATE_CODES.items():
        m = re.search(rf"QS_{name}\s*=\s*(\d+)", text)
        assert m and int(m.group(1)) == code, name
    from paper_2212_14201_gb300 import GATE_DTYPE, PAULI_DTYPE
    assert GATE_DTYPE == w.GATE_DTYPE and GATE_DTYPE.itemsize == 56
    assert PAULI_DTYPE == w.PAULI_DTYPE and PAULI_DTYPE.itemsize == 24


def test_program_codes_and_layout_agree_with_header(tmp_path):
    text = open(os.path.join(ROOT, "include", "qsim.h")).read()
    for name, code in w.PROGRAM_OPS.items():
        m = re.search(rf"QS_PI_{name}\s*=\s*(\d+)", text)
        assert m and int(m.group(1)) == code, name
    for name, code in w.CLASSICAL_OPS.items():
        m = re.search(rf"QS_CA_{name}\s*=\s*(\d+)", text)
        assert m and int(m.group(1)) == code, name
    from paper_2212_14201_gb300 import PINSTR_DTYPE
    assert PINSTR_DTYPE == w.PINSTR_DTYPE
    # the C compiler's layout of qs_pinstr against the numpy record
    src = tmp_path / "lay.c"
    fields = ["op", "qubit", "dst", "alu", "lhs", "rhs", "imm", "n_then", "n_else", "gate_begin", "gate_end"]
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "qsim.h"\nint main(void){printf("%zu'
                   + "".join(" %zu" for _ in fields) + '\\n", sizeof(qs_pinstr)'
                   + "".join(f", offsetof(qs_pinstr, {f})" for f in fields) + ");return 0;}\n")
    exe = tmp_path / "lay"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got == [w.PINSTR_DTYPE.itemsize] + [w.PINSTR_DTYPE.fields[f][1] for f in fields]


def test_noise_codes_and_layout_agree_with_header(tmp_path):
    text = open(os.path.join(ROOT, "include", "qsim.h")).read()
    for name, code in w.NOISE_MODELS.items():
        m = re.search(rf"QS_NOISE_{name}\s*=\s*(\d+)", text)
        assert m and int(m.group(1)) == code, name
    from paper_2212_14201_gb300 import NOISE_DTYPE
    assert NOISE_DTYPE == w.NOISE_DTYPE
    src = tmp_path / "lay.c"
    fields = ["model", "gate_type", "q0", "q1", "p", "t1", "t2", "tgate"]
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "qsim.h"\nint main(void){printf("%zu'
                   + "".join(" %zu" for _ in fields) + '\\n", sizeof(qs_noise_rule)'
                   + "".join(f", offsetof(qs_noise_rule, {f})" for f in fields) + ");return 0;}\n")
    exe = tmp_path / "lay"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got == [w.NOISE_DTYPE.itemsize] + [w.NOISE_DTYPE.fields[f][1] for f in fields]


def test_host_validation_without_gpu(built):
    import paper_2212_14201_gb300 as q
    with pytest.raises(q.QsimError) as e:
        q.qs_alloc(0)
    assert e.value.code == -1
    with pytest.raises(q.QsimError):
        q.qs_alloc(q.qs_max_qubits() + 1)
    with pytest.raises(q.QsimError) as e:
        q.qs_plan_create(4, w.pack([w.gate("H", 4)]), q.PLAN_PLAIN, 5)
    assert "out of range" in str(e.value)
    with pytest.raises(q.QsimError):
        q.qs_plan_create(4, w.pack([w.gate("CNOT", 2, 2)]), q.PLAN_PLAIN, 5)
    with pytest.raises(q.QsimError):
        q.qs_plan_create(4, w.pack([w.gate("X", 1, ctrl_mask=0b10)]), q.PLAN_PLAIN, 5)


def test_gate_list_dagger_reverses_and_flips(built):
    import paper_2212_14201_gb300 as q
    g = w.random_circuit(5, 30, 1)
    d = q.qs_gate_list_dagger(g)
    assert np.array_equal(d["type"], g["type"][::-1])
    assert np.array_equal(d["dagger"], 1 - g["dagger"][::-1])
    assert np.array_equal(d["p"], g["p"][::-1])
