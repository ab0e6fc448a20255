"""ctypes mirror of include/sv.h (argument marshalling only).

Loading fails loudly when libsvgb300.so is missing: there is no CPU or
Python fallback for any call.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsvgb300.so")

SV_OK = 0
ERRORS = {
    -1: "SV_ERR_ARG", -2: "SV_ERR_HOST_OOM", -3: "SV_ERR_DEVICE_OOM", -4: "SV_ERR_CORRUPT",
    -5: "SV_ERR_TIMEOUT", -6: "SV_ERR_NORM_COLLAPSE", -7: "SV_ERR_RANGE", -8: "SV_ERR_CUDA",
}
SV_C64, SV_C128 = 1, 2
SV_COMPRESSED, SV_UNCOMPRESSED = 0, 1

GATE_KIND = {"H": 0, "X": 1, "Y": 2, "Z": 3, "S": 4, "SDG": 5, "T": 6, "TDG": 7, "RX": 8,
             "RY": 9, "RZ": 10, "P": 11, "CNOT": 12, "CZ": 13, "CP": 14, "SWAP": 15, "CUSTOM": 16}


class SvGate(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("ntargets", C.c_uint32), ("ncontrols", C.c_uint32),
                ("param_index", C.c_int32), ("targets", C.c_uint32 * 2), ("controls", C.c_uint32 * 2),
                ("theta", C.c_double), ("mat", C.c_double * 32)]


class SvPauliTerm(C.Structure):
    _fields_ = [("coeff", C.c_double), ("xmask", C.c_uint64), ("zmask", C.c_uint64)]


DEVICE_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_int, C.c_void_p)
DEVICE_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_int, C.c_void_p)


class SvConfig(C.Structure):
    _fields_ = [("dtype", C.c_int32), ("mode", C.c_int32), ("init_index", C.c_uint64),
                ("max_group_qubits", C.c_int32), ("tile_qubits", C.c_int32),
                ("pipeline_slots", C.c_int32), ("renormalize", C.c_int32), ("device", C.c_int32),
                ("profile", C.c_int32), ("fuse_codec", C.c_int32), ("jit", C.c_int32),
                ("relative_bound", C.c_int32), ("remap_qubits", C.c_int32),
                ("checkpoint_passes", C.c_int32), ("lambda_cache", C.c_int32), ("device_alloc", DEVICE_ALLOC_FN), ("device_free", DEVICE_FREE_FN), ("alloc_ctx", C.c_void_p),
                ("stream", C.c_void_p), ("host_budget_bytes", C.c_uint64), ("timeout_s", C.c_double)]


class SvStats(C.Structure):
    _fields_ = [("passes", C.c_uint64), ("subpasses", C.c_uint64), ("groups", C.c_uint64),
                ("kernel_launches", C.c_uint64), ("bytes_h2d", C.c_uint64), ("bytes_d2h", C.c_uint64),
                ("compressed_bytes", C.c_uint64), ("raw_bytes", C.c_uint64),
                ("amp_gate_updates", C.c_uint64), ("gates_applied", C.c_uint64), ("norm2", C.c_double),
                ("last_call_seconds", C.c_double), ("quant_step", C.c_double),
                ("chunk_qubits", C.c_int32), ("group_qubits", C.c_int32),
                ("t_decode_s", C.c_double), ("t_apply_s", C.c_double), ("t_encode_s", C.c_double),
                ("n_decode", C.c_uint64), ("n_apply", C.c_uint64), ("n_encode", C.c_uint64),
                ("alg_bytes_decode", C.c_uint64), ("alg_bytes_apply", C.c_uint64),
                ("alg_bytes_encode", C.c_uint64),
                ("jit_kernels_compiled", C.c_uint64), ("jit_launches", C.c_uint64),
                ("t_jit_compile_s", C.c_double),
                ("t_h2d_s", C.c_double), ("t_d2h_s", C.c_double), ("t_encode_finish_s", C.c_double),
                ("t_host_prepare_s", C.c_double), ("t_host_wait_s", C.c_double),
                ("remap_swaps", C.c_uint64), ("jit_adjoint_launches", C.c_uint64),
                ("host_pinned_bytes", C.c_uint64), ("checkpoint_bytes", C.c_uint64),
                ("checkpoints", C.c_uint64), ("t_grad_forward_s", C.c_double), ("t_grad_lambda_s", C.c_double),
                ("t_grad_reverse_s", C.c_double)]


# every entry point declared in include/sv.h
EXPORTS = ("sv_config_default", "sv_create", "sv_apply_circuit", "sv_expect", "sv_amplitudes",
           "sv_amplitudes_range", "sv_grad", "sv_stats", "sv_last_error", "sv_destroy",
           "sv_codec_max_bytes", "sv_codec_encode", "sv_codec_decode", "sv_plan",
           "sv_codec_encode_noalloc", "sv_chunk_stream", "sv_jit_sources", "sv_set_profile",
           "sv_codec_encode_relative", "sv_copy_probe", "sv_plan_remap", "sv_inner",
           "sv_device_state")

_lib = None


class SvError(RuntimeError):
    def __init__(self, code: int, what: str, detail: str = ""):
        self.code = code
        super().__init__(f"{what}: {ERRORS.get(code, code)} {detail}".strip())


def load() -> C.CDLL:
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            f"{LIB_PATH} is missing: build it with `python -m paper_2309_16979_gb300.build` "
            "(nvcc, sm_103a). There is no fallback implementation.")
    L = C.CDLL(LIB_PATH)
    P, SZ = C.c_void_p, C.c_size_t
    L.sv_config_default.argtypes = [C.POINTER(SvConfig)]
    L.sv_config_default.restype = None
    L.sv_create.argtypes = [C.c_int, C.c_int, C.c_double, C.POINTER(SvConfig), C.POINTER(P)]
    L.sv_create.restype = C.c_int
    L.sv_apply_circuit.argtypes = [P, P, SZ]
    L.sv_apply_circuit.restype = C.c_int
    L.sv_expect.argtypes = [P, P, SZ, C.POINTER(C.c_double)]
    L.sv_expect.restype = C.c_int
    L.sv_amplitudes.argtypes = [P, P, SZ, P]
    L.sv_amplitudes.restype = C.c_int
    L.sv_amplitudes_range.argtypes = [P, C.c_uint64, SZ, P]
    L.sv_amplitudes_range.restype = C.c_int
    L.sv_inner.argtypes = [P, P, C.POINTER(C.c_double), C.POINTER(C.c_double)]
    L.sv_inner.restype = C.c_int
    L.sv_device_state.argtypes = [P, C.POINTER(C.c_void_p), P]
    L.sv_device_state.restype = C.c_int
    L.sv_grad.argtypes = [P, P, SZ, P, SZ, P, SZ, C.POINTER(C.c_double), P]
    L.sv_grad.restype = C.c_int
    L.sv_stats.argtypes = [P, C.POINTER(SvStats)]
    L.sv_stats.restype = C.c_int
    L.sv_last_error.argtypes = [P]
    L.sv_last_error.restype = C.c_char_p
    L.sv_destroy.argtypes = [P]
    L.sv_destroy.restype = None
    L.sv_codec_max_bytes.argtypes = [C.c_int]
    L.sv_codec_max_bytes.restype = SZ
    L.sv_codec_encode.argtypes = [C.c_int, C.c_int, C.c_double, P, P, SZ, C.POINTER(SZ)]
    L.sv_codec_encode.restype = C.c_int
    L.sv_codec_decode.argtypes = [C.c_int, C.c_int, P, SZ, P]
    L.sv_codec_decode.restype = C.c_int
    L.sv_plan.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, P, SZ, P, P, P, C.POINTER(SZ), C.POINTER(SZ),
                          C.POINTER(SZ)]
    L.sv_plan.restype = C.c_int
    L.sv_plan_remap.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, P, SZ, P, P, P, C.POINTER(SZ),
                                C.POINTER(SZ), C.POINTER(SZ), C.POINTER(SZ), P, P, P]
    L.sv_plan_remap.restype = C.c_int
    L.sv_codec_encode_noalloc.argtypes = [C.c_int, C.c_int, C.c_double, P, P, SZ, C.POINTER(SZ)]
    L.sv_codec_encode_noalloc.restype = C.c_int
    L.sv_codec_encode_relative.argtypes = [C.c_int, C.c_int, C.c_double, P, P, SZ, C.POINTER(SZ)]
    L.sv_codec_encode_relative.restype = C.c_int
    L.sv_copy_probe.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_uint64, C.POINTER(C.c_double),
                                C.POINTER(C.c_int)]
    L.sv_copy_probe.restype = C.c_int
    L.sv_chunk_stream.argtypes = [P, C.c_uint64, P, SZ, C.POINTER(SZ)]
    L.sv_chunk_stream.restype = C.c_int
    L.sv_jit_sources.argtypes = [C.c_int, C.c_int, C.POINTER(SvConfig), P, SZ, C.c_int, C.c_char_p, SZ,
                                 C.POINTER(SZ), C.POINTER(SZ)]
    L.sv_jit_sources.restype = C.c_int
    L.sv_set_profile.argtypes = [P, C.c_int]
    L.sv_set_profile.restype = C.c_int
    _lib = L
    return L


def gates_to_c(gates) -> C.Array:
    """Marshal gate descriptions (objects with kind/targets/controls/theta/param/mat)."""
    arr = (SvGate * max(1, len(gates)))()
    for i, g in enumerate(gates):
        s = arr[i]
        s.kind = GATE_KIND[g.kind]
        s.ntargets = len(g.targets)
        s.ncontrols = len(g.controls)
        s.param_index = getattr(g, "param", -1)
        for a, q in enumerate(g.targets):
            s.targets[a] = q
        for a, q in enumerate(g.controls):
            s.controls[a] = q
        s.theta = g.theta
        mat = getattr(g, "mat", None)
        if mat is not None:
            for a, z in enumerate(mat):
                s.mat[2 * a] = complex(z).real
                s.mat[2 * a + 1] = complex(z).imag
    return arr


def terms_to_c(terms) -> C.Array:
    arr = (SvPauliTerm * max(1, len(terms)))()
    for i, t in enumerate(terms):
        arr[i].coeff = t.coeff
        arr[i].xmask = t.xmask
        arr[i].zmask = t.zmask
    return arr
