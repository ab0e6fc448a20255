"""The sub-pass kernels generated at run time, checked on the host: the
generator's sources compile with NVRTC for sm_103a, depend on the circuit's
structure and not on its rotation angles, and fold thread-conditional
exchanges into the phase's store addresses. No GPU is used."""
import ctypes
import dataclasses
import os

import pytest

import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2309_16979_gb300", "csrc")
HEADERS = ["sv_dev_types.h", "codec_dev.cuh", "tile_dev.cuh"]


def _nvrtc():
    for name in ("libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("NVRTC is not available")


def _compile(lib, src):
    prog = ctypes.c_void_p()
    hdr = (ctypes.c_char_p * len(HEADERS))(*[open(os.path.join(CSRC, h), "rb").read() for h in HEADERS])
    names = (ctypes.c_char_p * len(HEADERS))(*[h.encode() for h in HEADERS])
    assert lib.nvrtcCreateProgram(ctypes.byref(prog), src.encode(), b"sv_subpass.cu", len(HEADERS), hdr, names) == 0
    opts = (ctypes.c_char_p * 2)(b"--gpu-architecture=sm_103a", b"--std=c++17")
    rc = lib.nvrtcCompileProgram(prog, 2, opts)
    n = ctypes.c_size_t()
    lib.nvrtcGetProgramLogSize(prog, ctypes.byref(n))
    log = ctypes.create_string_buffer(max(1, n.value))
    lib.nvrtcGetProgramLog(prog, log)
    lib.nvrtcDestroyProgram(ctypes.byref(prog))
    return rc, log.value.decode(errors="replace")


@pytest.fixture(scope="module")
def jit_sources():
    from paper_2309_16979_gb300 import jit_sources
    return jit_sources


@pytest.mark.parametrize("case", ["layers_c64_fused", "mixed_c128", "mixed_c64_uncompressed"])
def test_generated_kernels_compile(jit_sources, case):
    lib = _nvrtc()
    if case == "layers_c64_fused":
        srcs = jit_sources(16, 10, W.random_layers(16, 4, seed=3), max_group_qubits=3)
    elif case == "mixed_c128":
        srcs = jit_sources(14, 9, W.random_mixed(14, 120, seed=8), dtype="c128", max_group_qubits=3)
    else:
        srcs = jit_sources(13, 13, W.random_mixed(13, 120, seed=9), mode="uncompressed")
    srcs = [s for s in srcs if s]
    assert srcs
    # the first and the last sub-pass carry the fused decode / encode
    for src in (srcs[0], srcs[-1]):
        rc, log = _compile(lib, src)
        assert rc == 0, log


def test_sources_depend_on_structure_not_angles(jit_sources):
    # kernels are shared while each rotation keeps which entry is factored
    # out of it (the first one, unless the rotation is near pi)
    a = jit_sources(16, 10, W.random_layers(16, 4, seed=3), max_group_qubits=3)
    g = W.random_layers(16, 4, seed=3)
    for x in g:
        if x.kind in ("RX", "RY", "RZ"):
            x.theta = x.theta + 0.01
    b = jit_sources(16, 10, g, max_group_qubits=3)
    assert a == b
    # an angle that makes a rotation the identity changes the code (the gate is dropped)
    for x in g:
        if x.kind == "RX":
            x.theta = 0.0
            break
    c = jit_sources(16, 10, g, max_group_qubits=3)
    assert c != b


def test_conditional_exchange_folds_into_store_addresses(jit_sources):
    # CNOTs whose control is a thread bit and target a register bit, with no
    # later gate on the target in the phase: the exchange becomes an XOR of the
    # store base instead of register moves (the controls carry no mixing gate,
    # so no phase takes them as register bits)
    gates = [W.Gate("H", (q,)) for q in range(12) if q not in (7, 9)]
    gates += [W.Gate("CNOT", (1,), (7,)), W.Gate("CNOT", (2,), (9,))]
    srcs = [s for s in jit_sources(12, 12, gates, mode="uncompressed") if s]
    assert any("const uint32_t sb0 = sb" in s for s in srcs)


def test_x_gates_cost_no_arithmetic(jit_sources):
    gates = [W.Gate("X", (q,)) for q in range(12)]
    srcs = [s for s in jit_sources(12, 12, gates, mode="uncompressed") if s]
    assert srcs and all("p.m[" not in s for s in srcs)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_generated_adjoint_kernels_compile(jit_sources, dtype):
    """Reverse-sweep kernels of sv_grad: psi and lambda together, one
    gradient accumulation per parameterised gate."""
    lib = _nvrtc()
    gates, nparams = W.hea(14, 2)
    theta = W.normal_params(nparams)
    gates = [dataclasses.replace(g, theta=theta[g.param]) if g.param >= 0 else g for g in gates]
    srcs = [s for s in jit_sources(14, 9, gates, dtype=dtype, max_group_qubits=3, adjoint=True) if s]
    assert srcs
    assert sum(s.count("gw[") for s in srcs) - 3 * len(srcs) == nparams
    # complex64: psi's and lambda's updates share coefficients and run as
    # packed FP32x2 instructions; complex128 has no packed form
    packed = sum(s.count("__ffma2_rn(") + s.count("__fadd2_rn(") for s in srcs)
    assert (packed > 0) == (dtype == "c64")
    for s in srcs:
        rc, log = _compile(lib, s)
        assert rc == 0, log


def test_exchange_circuits_reach_every_store_form(jit_sources):
    """The circuits of the GPU parity tests for exchanges reach each way a
    phase stores: shared memory with pending exchanges folded into its bases,
    HBM directly (with and without pending exchanges), and real and
    imaginary parts packed into FP32x2 pairs."""
    from test_gpu_jit import _exchange_circuit
    srcs = [s for s in jit_sources(14, 14, _exchange_circuit(14, 41), mode="uncompressed") if s]
    assert any("const uint32_t sb0 = " in s for s in srcs)
    assert any("T* const gq = " in s for s in srcs)
    assert any("T* const gq0 = " in s for s in srcs)
    assert any("{ const float2 " in s for s in srcs)


def test_remapped_circuit_kernels_compile(jit_sources):
    """With qubit remapping the passes also run physical SWAPs (4x4
    permutation matrices: moves only); every kernel of such a plan compiles."""
    import paper_2309_16979_gb300 as P
    lib = _nvrtc()
    n, c, g = 16, 10, 2
    gates = W.random_layers(n, 6, seed=5)
    assert P.plan(n, c, gates, max_group_qubits=g, remap=True)["swaps"]
    plain = [s for s in jit_sources(n, c, gates, max_group_qubits=g) if s]
    srcs = [s for s in jit_sources(n, c, gates, max_group_qubits=g, remap=True) if s]
    assert srcs and srcs != plain
    for src in srcs:
        if src in plain:
            continue
        rc, log = _compile(lib, src)
        assert rc == 0, log
