"""GB300 compressed state-vector simulator (MEMQSim, arXiv 2309.16979).

Python binding over the C ABI of include/sv.h. Every step of a pass -- chunk
streaming, decode, gate application, encode, reductions, the adjoint sweep --
runs in the CUDA library libsvgb300.so; this module only marshals arguments.

    from paper_2309_16979_gb300 import StateVector
    sv = StateVector(30, chunk_qubits=22, eb=1e-6)      # relative_bound=True: per-chunk step
                                                         # remap_qubits=True: fewer passes on
                                                         # circuits that mix high qubits often
    sv.apply(gates)
    e = sv.expect(terms)
    energy, grad = sv.grad(gates, theta, terms)          # adjoint gradient
    ov = sv.inner(ref)                                   # <sv|ref>, ref uncompressed

Also: codec_encode / codec_decode (one chunk on the device), copy_probe (the
paper's host <-> device copy strategies), plan (with remap=True: the remapped
passes) and jit_sources (host only).
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np

from . import _abi
from ._abi import SV_C64, SV_C128, SV_COMPRESSED, SV_UNCOMPRESSED, SvError, load

__all__ = ["StateVector", "SvError", "codec_encode", "codec_decode", "codec_max_bytes", "copy_probe", "plan",
           "jit_sources", "load", "SV_C64", "SV_C128", "SV_COMPRESSED", "SV_UNCOMPRESSED"]


def _check(code: int, what: str, handle=None):
    if code != 0:
        detail = _abi.load().sv_last_error(handle)
        raise SvError(code, what, detail.decode() if detail else "")


class StateVector:
    """An n-qubit state stored as compressed chunks in pinned host memory
    (mode="compressed") or whole in HBM (mode="uncompressed")."""

    def __init__(self, n: int, chunk_qubits: int = 0, eb: float = 1e-6, dtype: str = "c64",
                 mode: str = "compressed", init_index: int = 0, max_group_qubits: int = 0,
                 tile_qubits: int = 0, pipeline_slots: int = 3, renormalize: bool = False,
                 host_budget_bytes: int = 0, timeout_s: float = 600.0, device: int = 0,
                 profile: bool = False, fuse_codec: bool = True,
                 jit: bool = True, relative_bound: bool = False, remap_qubits: bool = False,
                 checkpoint_passes: int = 0, lambda_cache: int = 1, memory: str = "torch"):
        """memory="torch": the handle's device memory comes from torch's
        caching allocator (it shows in torch.cuda.memory_allocated()) and its
        calls order after the work queued on torch's current stream of the
        device at creation; memory="cuda": the library allocates with
        cudaMalloc and orders against no caller stream."""
        L = load()
        cfg = _abi.SvConfig()
        L.sv_config_default(C.byref(cfg))
        cfg.dtype = SV_C64 if dtype == "c64" else SV_C128
        cfg.mode = SV_COMPRESSED if mode == "compressed" else SV_UNCOMPRESSED
        cfg.init_index = init_index
        cfg.max_group_qubits = max_group_qubits
        cfg.tile_qubits = tile_qubits
        cfg.pipeline_slots = pipeline_slots
        cfg.renormalize = int(renormalize)
        cfg.host_budget_bytes = host_budget_bytes
        cfg.timeout_s = timeout_s
        cfg.device = device
        cfg.profile = int(profile)
        cfg.fuse_codec = int(fuse_codec)
        cfg.jit = int(jit)
        cfg.relative_bound = int(relative_bound)
        cfg.remap_qubits = int(remap_qubits)
        cfg.checkpoint_passes = int(checkpoint_passes)
        cfg.lambda_cache = int(lambda_cache)
        self._callbacks = None
        if memory == "torch":
            self._callbacks = _torch_memory(cfg, device, release_cached=max_group_qubits == 0)
        elif memory != "cuda":
            raise ValueError("memory must be 'torch' or 'cuda'")
        h = C.c_void_p()
        _check(L.sv_create(n, chunk_qubits or n, eb, C.byref(cfg), C.byref(h)), "sv_create", None)
        self._h = h
        self.n = n
        self.device = device
        self.dtype = dtype
        self.mode = mode

    # ------------------------------------------------------------ calls
    def apply(self, gates: Sequence) -> None:
        arr = _abi.gates_to_c(gates)
        _check(load().sv_apply_circuit(self._h, C.addressof(arr), len(gates)), "sv_apply_circuit", self._h)

    def expect(self, terms: Sequence) -> float:
        arr = _abi.terms_to_c(terms)
        out = C.c_double(0.0)
        _check(load().sv_expect(self._h, C.addressof(arr), len(terms), C.byref(out)), "sv_expect", self._h)
        return out.value

    def amplitudes(self, idx) -> np.ndarray:
        idx = np.ascontiguousarray(idx, dtype=np.uint64)
        out = np.empty(2 * idx.size, dtype=np.float64)
        _check(load().sv_amplitudes(self._h, idx.ctypes.data, idx.size, out.ctypes.data), "sv_amplitudes",
               self._h)
        return out.view(np.complex128)

    def amplitudes_range(self, first: int, count: int) -> np.ndarray:
        out = np.empty(2 * count, dtype=np.float64)
        _check(load().sv_amplitudes_range(self._h, first, count, out.ctypes.data), "sv_amplitudes_range",
               self._h)
        return out.view(np.complex128)

    def inner(self, other: "StateVector") -> complex:
        """<self|other> in FP64 (sv_inner); other must be uncompressed, on the
        same device, with the same number of qubits."""
        re, im = C.c_double(0.0), C.c_double(0.0)
        _check(load().sv_inner(self._h, other._h, C.byref(re), C.byref(im)), "sv_inner", self._h)
        return complex(re.value, im.value)

    def device_tensor(self):
        """Zero-copy torch view (complex64 / complex128, on the handle's GPU)
        of an uncompressed state, valid until the next call that applies
        gates and to be read only (torch has no read-only tensors: writing it
        is undefined), and the physical bit position of every logical qubit
        (sv_device_state): logical index x sits at the physical index whose
        bit positions[q] is bit q of x."""
        import torch
        ptr = C.c_void_p()
        pos = np.zeros(self.n, dtype=np.int32)
        _check(load().sv_device_state(self._h, C.byref(ptr), pos.ctypes.data), "sv_device_state", self._h)
        real = "<f4" if self.dtype == "c64" else "<f8"

        class _View:
            __cuda_array_interface__ = {"shape": (2 << self.n,), "typestr": real, "data": (ptr.value, False),
                                        "version": 3, "strides": None}

        flat = torch.as_tensor(_View(), device=f"cuda:{self.device}")
        return flat.view(torch.complex64 if self.dtype == "c64" else torch.complex128), pos.tolist()

    def state(self) -> np.ndarray:
        return self.amplitudes_range(0, 1 << self.n)

    def energy(self, gates: Sequence, theta: Sequence[float], terms: Sequence) -> float:
        """<H> of the parameterised circuit at theta from |init_index>, with no
        gradient (sv_grad with grad = NULL); the state is left at psi(theta)."""
        th = np.ascontiguousarray(theta, dtype=np.float64)
        ga = _abi.gates_to_c(gates)
        ta = _abi.terms_to_c(terms)
        e = C.c_double(0.0)
        _check(load().sv_grad(self._h, C.addressof(ga), len(gates), th.ctypes.data, th.size, C.addressof(ta),
                              len(terms), C.byref(e), None), "sv_grad", self._h)
        return e.value

    def grad(self, gates: Sequence, theta: Sequence[float], terms: Sequence):
        th = np.ascontiguousarray(theta, dtype=np.float64)
        g = np.zeros(th.size, dtype=np.float64)
        ga = _abi.gates_to_c(gates)
        ta = _abi.terms_to_c(terms)
        e = C.c_double(0.0)
        _check(load().sv_grad(self._h, C.addressof(ga), len(gates), th.ctypes.data, th.size, C.addressof(ta),
                              len(terms), C.byref(e), g.ctypes.data), "sv_grad", self._h)
        return e.value, g

    def chunk_stream(self, k: int) -> bytes:
        """The compressed stream of physical chunk k as stored in host memory."""
        L = load()
        nb = C.c_size_t(0)
        L.sv_chunk_stream(self._h, k, None, 0, C.byref(nb))
        buf = (C.c_uint8 * max(1, nb.value))()
        _check(L.sv_chunk_stream(self._h, k, buf, nb.value, C.byref(nb)), "sv_chunk_stream", self._h)
        return bytes(buf)[:nb.value]

    def set_profile(self, on: bool) -> None:
        """Per-launch CUDA-event timing on or off for the following calls."""
        _check(load().sv_set_profile(self._h, int(on)), "sv_set_profile", self._h)

    def stats(self) -> dict:
        st = _abi.SvStats()
        _check(load().sv_stats(self._h, C.byref(st)), "sv_stats", self._h)
        return {f: getattr(st, f) for f, _ in _abi.SvStats._fields_}

    def close(self) -> None:
        if getattr(self, "_h", None):
            load().sv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _torch_memory(cfg, device: int, release_cached: bool = False):
    """Fill cfg's allocator and stream from torch: the caching allocator on
    `device`, torch's current stream there. Returns the ctypes callbacks,
    which must live as long as the handle. Without CUDA in torch the library
    keeps its own allocator (sv_create then reports the missing device).
    release_cached: hand torch's cached free blocks back to the driver first,
    so that the library's automatic group size, which it takes from the
    device's free memory, sees them."""
    try:
        import torch
    except ImportError:
        return None
    if not torch.cuda.is_available():
        return None
    if release_cached:
        with torch.cuda.device(device):
            torch.cuda.empty_cache()
    stream = torch.cuda.current_stream(device)

    def alloc(nbytes, dev, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device=dev, stream=stream)
        except Exception:  # noqa: BLE001 -- reported by the library as SV_ERR_DEVICE_OOM
            return None

    def free(ptr, dev, ctx):
        try:
            torch.cuda.caching_allocator_delete(ptr)
        except Exception:  # noqa: BLE001 -- torch already torn down at interpreter exit
            pass

    cbs = (_abi.DEVICE_ALLOC_FN(alloc), _abi.DEVICE_FREE_FN(free))
    cfg.device_alloc, cfg.device_free = cbs
    cfg.stream = stream.cuda_stream
    return cbs


def plan(n: int, chunk_qubits: int, gates: Sequence, max_group_qubits: int = 4, tile_qubits: int = 0,
         remap: bool = False) -> dict:
    """Host-only pass plan (sv_plan, or sv_plan_remap with remap): execution
    order, pass of each gate, staged high-qubit mask per pass, pass / sub-pass
    counts, and the physical SWAPs remapping adds as (pass, low position, high
    position), each after the gates of its pass; with remap also the positions
    each executed gate runs on (targets, controls; -1 = none) and the final
    position of every qubit."""
    L = load()
    ng = len(gates)
    arr = _abi.gates_to_c(gates)
    order = np.zeros(max(1, ng), dtype=np.int32)
    pass_of = np.zeros(max(1, ng), dtype=np.int32)
    staged = np.zeros(max(1, ng), dtype=np.uint64)
    ex, npass, nsub, nswap = C.c_size_t(0), C.c_size_t(0), C.c_size_t(0), C.c_size_t(0)
    args = (n, chunk_qubits, max_group_qubits, tile_qubits, C.addressof(arr), ng, order.ctypes.data,
            pass_of.ctypes.data, staged.ctypes.data, C.byref(ex), C.byref(npass), C.byref(nsub))
    swaps = np.zeros(max(1, 24 * ng), dtype=np.int32)
    qubits = np.full(max(1, 4 * ng), -1, dtype=np.int32)
    positions = np.arange(n, dtype=np.int32)
    if remap:
        _check(L.sv_plan_remap(*args, C.byref(nswap), swaps.ctypes.data, qubits.ctypes.data,
                               positions.ctypes.data), "sv_plan_remap", None)
    else:
        _check(L.sv_plan(*args), "sv_plan", None)
    k = ex.value
    out = {"order": order[:k].tolist(), "pass_of": pass_of[:k].tolist(),
           "staged": [int(x) for x in staged[:npass.value]], "passes": npass.value, "subpasses": nsub.value,
           "swaps": [tuple(int(v) for v in swaps[3 * i:3 * i + 3]) for i in range(nswap.value)]}
    if remap:
        out["qubits"] = [tuple(int(v) for v in qubits[4 * i:4 * i + 4]) for i in range(k)]
        out["positions"] = positions.tolist()
    return out


def jit_sources(n: int, chunk_qubits: int, gates: Sequence, dtype: str = "c64", mode: str = "compressed",
                max_group_qubits: int = 4, tile_qubits: int = 0, fuse_codec: bool = True,
                adjoint: bool = False, remap: bool = False) -> list:
    """Host-only: the CUDA C++ sources of the sub-pass kernels sv_apply_circuit
    (or, with adjoint, the reverse sweep of sv_grad) would generate for this
    circuit (sv_jit_sources), in launch order; remap: with
    sv_config.remap_qubits."""
    L = load()
    cfg = _abi.SvConfig()
    L.sv_config_default(C.byref(cfg))
    cfg.dtype = SV_C64 if dtype == "c64" else SV_C128
    cfg.mode = SV_COMPRESSED if mode == "compressed" else SV_UNCOMPRESSED
    cfg.max_group_qubits = max_group_qubits
    cfg.tile_qubits = tile_qubits
    cfg.fuse_codec = int(fuse_codec)
    cfg.remap_qubits = int(remap)
    arr = _abi.gates_to_c(gates)
    need, nk = C.c_size_t(0), C.c_size_t(0)
    adj = int(adjoint)
    _check(L.sv_jit_sources(n, chunk_qubits, C.byref(cfg), C.addressof(arr), len(gates), adj, None, 0,
                            C.byref(need), C.byref(nk)), "sv_jit_sources", None)
    buf = C.create_string_buffer(max(1, need.value))
    _check(L.sv_jit_sources(n, chunk_qubits, C.byref(cfg), C.addressof(arr), len(gates), adj, buf, need.value,
                            C.byref(need), C.byref(nk)), "sv_jit_sources", None)
    parts = buf.raw[:need.value].split(b"\0")[:nk.value]
    return [x.decode() for x in parts]


# --------------------------------------------------------------- transfers

COPY_STRATEGIES = {"sync": 0, "async": 1, "buffer": 2}


def copy_probe(n: int, strategy: str, direction: str = "h2d", dtype: str = "c128", sample: int = 0):
    """Seconds to move a 2^n-amplitude state host -> device ("h2d") or back
    ("d2h") by one of the paper's strategies (sv_copy_probe); returns
    (seconds, verified)."""
    sec = C.c_double(0.0)
    ok = C.c_int(0)
    _check(load().sv_copy_probe(n, SV_C64 if dtype == "c64" else SV_C128, COPY_STRATEGIES[strategy],
                                0 if direction == "h2d" else 1, sample, C.byref(sec), C.byref(ok)),
           "sv_copy_probe", None)
    return sec.value, bool(ok.value)


# ------------------------------------------------------------------ codec

def codec_max_bytes(chunk_qubits: int) -> int:
    return load().sv_codec_max_bytes(chunk_qubits)


def codec_encode(d_amps, eb: float, d_stream=None, relative: bool = False):
    """Encode one chunk held in a CUDA tensor (complex64/complex128, 2^c
    elements); relative: the step follows the chunk's largest component
    (sv_codec_encode_relative). Returns (stream tensor uint8 on the device,
    nbytes)."""
    import torch
    c = int(d_amps.numel()).bit_length() - 1
    dt = SV_C64 if d_amps.dtype == torch.complex64 else SV_C128
    cap = codec_max_bytes(c)
    if d_stream is None:
        d_stream = torch.empty(cap, dtype=torch.uint8, device=d_amps.device)
    nb = C.c_size_t(0)
    torch.cuda.synchronize(d_amps.device)
    fn = load().sv_codec_encode_relative if relative else load().sv_codec_encode
    code = fn(dt, c, eb, d_amps.data_ptr(), d_stream.data_ptr(), d_stream.numel(), C.byref(nb))
    if code:
        raise SvError(code, "sv_codec_encode")
    return d_stream, nb.value


def codec_decode(d_stream, nbytes: int, c: int, dtype="c64", out=None):
    import torch
    dt = SV_C64 if dtype == "c64" else SV_C128
    if out is None:
        out = torch.empty(1 << c, dtype=torch.complex64 if dt == SV_C64 else torch.complex128,
                          device=d_stream.device)
    torch.cuda.synchronize(d_stream.device)
    code = load().sv_codec_decode(dt, c, d_stream.data_ptr(), nbytes, out.data_ptr())
    if code:
        raise SvError(code, "sv_codec_decode")
    return out
