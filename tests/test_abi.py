"""The C-ABI library builds for sm_103a, loads, and exports every entry
point declared in include/sv.h (no compute call: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(sv_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2309_16979_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert {"sv_create", "sv_apply_circuit", "sv_expect", "sv_amplitudes", "sv_destroy", "sv_grad",
            "sv_stats", "sv_last_error", "sv_codec_encode", "sv_codec_decode"} <= names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_lists_every_declared_symbol():
    from paper_2309_16979_gb300 import _abi
    assert set(_abi.EXPORTS) == _declared()


def test_struct_sizes_match_header_layout():
    from paper_2309_16979_gb300 import _abi
    assert ctypes.sizeof(_abi.SvGate) == 4 * 4 + 8 + 8 + 8 + 32 * 8
    assert ctypes.sizeof(_abi.SvPauliTerm) == 24
    assert ctypes.sizeof(_abi.SvConfig) == 4 + 4 + 8 + 4 * 12 + 4 * 8 + 8 + 8


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """Every ctypes struct of the binding has the size and field offsets that
    the C compiler gives the header's struct."""
    import shutil
    import subprocess
    from paper_2309_16979_gb300 import _abi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"sv_gate": _abi.SvGate, "sv_pauli_term": _abi.SvPauliTerm, "sv_config": _abi.SvConfig,
               "sv_stats_t": _abi.SvStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sv.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            cname, f, v = line.split()
            got[(cname, f)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_codec_max_bytes_without_gpu(lib):
    lib.sv_codec_max_bytes.restype = ctypes.c_size_t
    import oracle
    for c in (8, 10, 22):
        assert lib.sv_codec_max_bytes(c) == oracle.codec_max_bytes(c)
    assert lib.sv_codec_max_bytes(7) == 0


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    from paper_2309_16979_gb300 import StateVector, SvError
    with pytest.raises(SvError):
        StateVector(10, 8, 1e-6)


@pytest.mark.parametrize("kw,word", [
    (dict(lambda_cache=3), "lambda_cache"),
    (dict(lambda_cache=-1), "lambda_cache"),
    (dict(checkpoint_passes=-1), "checkpoint_passes"),
    (dict(max_group_qubits=9), "max_group_qubits"),
    (dict(max_group_qubits=1), "max_group_qubits"),
    (dict(pipeline_slots=1), "pipeline_slots"),
    (dict(pipeline_slots=5), "pipeline_slots"),
    (dict(tile_qubits=14), "tile_qubits"),
    (dict(init_index=1 << 10), "init_index"),
])
def test_create_rejects_bad_config_before_any_gpu_call(kw, word):
    """sv_create checks its arguments before it touches a device: each bad
    field gives SV_ERR_ARG (-1) and a message naming it, with or without a
    GPU."""
    from paper_2309_16979_gb300 import StateVector, SvError
    with pytest.raises(SvError) as ei:
        StateVector(10, 8, 1e-6, memory="cuda", **kw)
    assert ei.value.code == -1
    assert word in str(ei.value)
