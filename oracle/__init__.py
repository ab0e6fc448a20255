"""CPU FP64 oracle for compressed state-vector simulation (MEMQSim, arXiv 2309.16979).

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``. The product library never imports it.

The arithmetic lives in ``oracle.c`` (plain loops, FP64). This module only
compiles it with gcc, marshals gate lists / Pauli sums from ``workloads`` into
the oracle's own C structs, and wraps the calls. Every function names the part
of the method it follows in ``oracle.c``'s header.

Parity status per function:
  apply_gates / run      pinned (dense Kronecker-product unitaries, closed forms)
  expect / hamiltonian   pinned (closed forms on basis, |+>, GHZ states; dense matrix)
  adjoint                pinned (parameter shift, central finite differences)
  codec encode/decode    pinned (hand-worked streams in tests/golden, error bound,
                         bit-level invariants)
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess
import threading
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, f"liboracle.{platform.machine()}.so")
_lock = threading.Lock()
_lib = None

KIND = {"H": 0, "X": 1, "Y": 2, "Z": 3, "S": 4, "SDG": 5, "T": 6, "TDG": 7,
        "RX": 8, "RY": 9, "RZ": 10, "P": 11, "CNOT": 12, "CZ": 13, "CP": 14,
        "SWAP": 15, "CUSTOM": 16}

C64, C128 = 1, 2


class OrGate(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nt", C.c_int32), ("nc", C.c_int32),
                ("param", C.c_int32), ("t", C.c_int32 * 2), ("c", C.c_int32 * 2),
                ("theta", C.c_double), ("m", C.c_double * 32)]


class OrPauli(C.Structure):
    _fields_ = [("coeff", C.c_double), ("x", C.c_uint64), ("z", C.c_uint64)]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP, no FMA contraction)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.c_void_p
        L.or_apply_gates.argtypes = [C.c_int, P, P, C.c_int64, P]
        L.or_apply_gates.restype = C.c_int
        L.or_apply_gates_dagger_reversed.argtypes = [C.c_int, P, P, C.c_int64, P]
        L.or_apply_gates_dagger_reversed.restype = C.c_int
        L.or_expect.argtypes = [C.c_int, P, P, C.c_int64]
        L.or_expect.restype = C.c_double
        L.or_apply_hamiltonian.argtypes = [C.c_int, P, P, C.c_int64, P]
        L.or_apply_hamiltonian.restype = None
        L.or_adjoint.argtypes = [C.c_int, C.c_uint64, P, C.c_int64, P, C.c_int64, P,
                                 C.c_int64, P, P, P]
        L.or_adjoint.restype = C.c_int
        L.or_num_threads.restype = C.c_int
        L.or_set_num_threads.argtypes = [C.c_int]
        L.or_codec_step_exponent.argtypes = [C.c_double]
        L.or_codec_step_exponent.restype = C.c_int
        L.or_codec_meta_bytes.argtypes = [C.c_int]
        L.or_codec_meta_bytes.restype = C.c_size_t
        L.or_codec_max_bytes.argtypes = [C.c_int]
        L.or_codec_max_bytes.restype = C.c_size_t
        L.or_codec_encode.argtypes = [C.c_int, C.c_int, C.c_double, P, P, C.c_size_t,
                                      C.POINTER(C.c_size_t)]
        L.or_codec_encode.restype = C.c_int
        L.or_codec_decode.argtypes = [C.c_int, C.c_int, P, C.c_size_t, P]
        L.or_codec_decode.restype = C.c_int
        L.or_codec_relative_exponent.argtypes = [C.c_double, C.c_double]
        L.or_codec_relative_exponent.restype = C.c_int
        L.or_codec_chunk_max.argtypes = [C.c_int, C.c_int, P]
        L.or_codec_chunk_max.restype = C.c_double
        L.or_codec_encode_relative.argtypes = [C.c_int, C.c_int, C.c_double, P, P, C.c_size_t,
                                               C.POINTER(C.c_size_t)]
        L.or_codec_encode_relative.restype = C.c_int
        _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


def _check(status: int, what: str):
    if status != 0:
        raise OracleError(f"{what} failed with status {status}")


def gates_to_c(gates: Sequence) -> C.Array:
    arr = (OrGate * max(1, len(gates)))()
    for i, g in enumerate(gates):
        s = arr[i]
        s.kind = KIND[g.kind]
        s.nt = len(g.targets)
        s.nc = len(g.controls)
        s.param = g.param
        for a, q in enumerate(g.targets):
            s.t[a] = q
        for a, q in enumerate(g.controls):
            s.c[a] = q
        s.theta = g.theta
        if g.mat is not None:
            for a, z in enumerate(g.mat):
                s.m[2 * a] = z.real
                s.m[2 * a + 1] = z.imag
    return arr


def paulis_to_c(terms: Sequence) -> C.Array:
    arr = (OrPauli * max(1, len(terms)))()
    for i, t in enumerate(terms):
        arr[i].coeff = t.coeff
        arr[i].x = t.xmask
        arr[i].z = t.zmask
    return arr


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def basis_state(n: int, index: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[index] = 1.0
    return psi


def apply_gates(n: int, psi: np.ndarray, gates: Sequence,
                theta: Optional[Sequence[float]] = None, inplace: bool = False) -> np.ndarray:
    """psi <- U_L ... U_1 psi in FP64, on a complex128 copy (or, with inplace,
    on psi itself when it is already a contiguous complex128 array)."""
    out = np.ascontiguousarray(psi, dtype=np.complex128)
    if not (inplace and out is psi):
        out = out.copy()
    th = None if theta is None else np.ascontiguousarray(theta, dtype=np.float64)
    ga = gates_to_c(gates)
    _check(lib().or_apply_gates(n, _ptr(out), C.addressof(ga), len(gates),
                                None if th is None else _ptr(th)), "or_apply_gates")
    return out


def run(n: int, gates: Sequence, init: int = 0,
        theta: Optional[Sequence[float]] = None) -> np.ndarray:
    return apply_gates(n, basis_state(n, init), gates, theta)


def expect(n: int, psi: np.ndarray, terms: Sequence) -> float:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    ta = paulis_to_c(terms)
    return lib().or_expect(n, _ptr(psi), C.addressof(ta), len(terms))


def hamiltonian(n: int, psi: np.ndarray, terms: Sequence) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.empty_like(psi)
    ta = paulis_to_c(terms)
    lib().or_apply_hamiltonian(n, _ptr(psi), C.addressof(ta), len(terms), _ptr(out))
    return out


def energy(n: int, gates: Sequence, theta: Sequence[float], terms: Sequence,
           init: int = 0) -> float:
    return expect(n, run(n, gates, init, theta), terms)


def adjoint(n: int, gates: Sequence, theta: Sequence[float], terms: Sequence,
            init: int = 0) -> Tuple[float, np.ndarray]:
    th = np.ascontiguousarray(theta, dtype=np.float64)
    grad = np.zeros(len(th), dtype=np.float64)
    work = np.empty(4 << n, dtype=np.float64)
    e = C.c_double(0.0)
    ga = gates_to_c(gates)
    ta = paulis_to_c(terms)
    _check(lib().or_adjoint(n, init, C.addressof(ga), len(gates), _ptr(th), len(th),
                            C.addressof(ta), len(terms), C.byref(e), _ptr(grad), _ptr(work)),
           "or_adjoint")
    return e.value, grad


def param_shift(n: int, gates: Sequence, theta: Sequence[float], terms: Sequence,
                params: Optional[Sequence[int]] = None, init: int = 0) -> np.ndarray:
    """dE/dtheta_p = (E(theta_p + pi/2) - E(theta_p - pi/2)) / 2, exact for
    U = exp(-i theta G / 2) with G^2 = I when each parameter is used once."""
    th = np.array(theta, dtype=np.float64)
    idx = list(range(len(th))) if params is None else list(params)
    out = np.zeros(len(idx))
    for j, p in enumerate(idx):
        tp = th.copy(); tp[p] += np.pi / 2
        tm = th.copy(); tm[p] -= np.pi / 2
        out[j] = 0.5 * (energy(n, gates, tp, terms, init) - energy(n, gates, tm, terms, init))
    return out


def finite_diff(n: int, gates: Sequence, theta: Sequence[float], terms: Sequence,
                params: Sequence[int], h: float = 1e-5, init: int = 0) -> np.ndarray:
    th = np.array(theta, dtype=np.float64)
    out = np.zeros(len(params))
    for j, p in enumerate(params):
        tp = th.copy(); tp[p] += h
        tm = th.copy(); tm[p] -= h
        out[j] = (energy(n, gates, tp, terms, init) - energy(n, gates, tm, terms, init)) / (2 * h)
    return out


def num_threads() -> int:
    return lib().or_num_threads()


def set_num_threads(t: int) -> None:
    lib().or_set_num_threads(t)


# ------------------------------------------------------------------ codec

def step_exponent(eb: float) -> int:
    return lib().or_codec_step_exponent(eb)


def codec_meta_bytes(c: int) -> int:
    return lib().or_codec_meta_bytes(c)


def codec_max_bytes(c: int) -> int:
    return lib().or_codec_max_bytes(c)


def codec_relative_exponent(eb: float, m: float) -> int:
    """Step exponent of the relative bound for a chunk whose largest component
    magnitude is m."""
    return lib().or_codec_relative_exponent(eb, m)


def codec_encode(amps: np.ndarray, eb: float, relative: bool = False) -> bytes:
    """Encode one chunk of 2^c amplitudes (complex64 or complex128); with
    relative, the step follows the chunk's largest component (relative bound)."""
    amps = np.ascontiguousarray(amps)
    dtype = C64 if amps.dtype == np.complex64 else C128
    if amps.dtype not in (np.complex64, np.complex128):
        raise TypeError("complex64 or complex128 amplitudes expected")
    c = int(amps.size).bit_length() - 1
    if amps.size != (1 << c):
        raise ValueError("chunk size must be a power of two")
    cap = codec_max_bytes(c)
    out = np.zeros(cap, dtype=np.uint8)
    nb = C.c_size_t(0)
    fn = lib().or_codec_encode_relative if relative else lib().or_codec_encode
    _check(fn(dtype, c, eb, _ptr(amps), _ptr(out), cap, C.byref(nb)), "or_codec_encode")
    return out[: nb.value].tobytes()


def codec_decode(stream: bytes, c: int, dtype=np.complex64) -> np.ndarray:
    dt = C64 if dtype == np.complex64 else C128
    buf = np.frombuffer(stream, dtype=np.uint8).copy()
    out = np.zeros(1 << c, dtype=dtype)
    _check(lib().or_codec_decode(dt, c, _ptr(buf), buf.size, _ptr(out)), "or_codec_decode")
    return out


def codec_status_encode(amps: np.ndarray, eb: float) -> int:
    """Status code of an encode (for range / argument error tests)."""
    amps = np.ascontiguousarray(amps)
    dtype = C64 if amps.dtype == np.complex64 else C128
    c = int(amps.size).bit_length() - 1
    cap = codec_max_bytes(max(c, 8))
    out = np.zeros(cap, dtype=np.uint8)
    nb = C.c_size_t(0)
    return lib().or_codec_encode(dtype, c, eb, _ptr(amps), _ptr(out), cap, C.byref(nb))


def codec_status_decode(stream: bytes, c: int, dtype=np.complex64) -> int:
    dt = C64 if dtype == np.complex64 else C128
    buf = np.frombuffer(stream, dtype=np.uint8).copy()
    out = np.zeros(1 << c, dtype=dtype)
    return lib().or_codec_decode(dt, c, _ptr(buf), buf.size, _ptr(out))


def compress_roundtrip(psi: np.ndarray, c: int, eb: float, relative: bool = False) -> np.ndarray:
    """Quantise a whole state chunk by chunk through the reference codec."""
    out = np.empty_like(psi)
    for k in range(psi.size >> c):
        seg = psi[k << c:(k + 1) << c]
        out[k << c:(k + 1) << c] = codec_decode(codec_encode(seg, eb, relative), c, psi.dtype)
    return out
