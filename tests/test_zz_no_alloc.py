"""sv_codec_encode_noalloc: the chunk encoder for callers that must not
allocate GPU memory while they run (device memory owned by another
allocator, or loops that cannot take the device-wide synchronisation of
cudaMalloc / cudaFree). It stages in a fixed device array inside the library
instead of per-call buffers; its streams must be byte-identical to
sv_codec_encode's, call after call, although every call reuses the same
staging area. This file is collected last so that a failure here does not
hide the other tests."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    from paper_2309_16979_gb300 import _abi
    return _abi.load()


def _encode(lib, fn, x, c, eb, dtype_code):
    cap = lib.sv_codec_max_bytes(c)
    d_amps = torch.from_numpy(x).cuda()
    d_out = torch.full((cap,), 0xAB, dtype=torch.uint8, device="cuda")
    nb = C.c_size_t(0)
    torch.cuda.synchronize()
    code = fn(dtype_code, c, eb, d_amps.data_ptr(), d_out.data_ptr(), cap, C.byref(nb))
    assert code == 0, code
    return d_out[:nb.value].cpu().numpy().tobytes()


def test_noalloc_streams_equal_allocating_encoder_on_consecutive_calls(lib):
    rng = np.random.default_rng(2024)
    fn_na = lib.sv_codec_encode_noalloc
    fn_na.argtypes = [C.c_int, C.c_int, C.c_double, C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t)]
    fn_na.restype = C.c_int
    cases = [(20, np.complex64, 1, 1e-6, 1.0), (11, np.complex64, 1, 1e-4, 0.05),
             (14, np.complex128, 2, 1e-7, 0.01)]
    for c, dt, code, eb, scale in cases:  # two or more calls in a row, shrinking and growing sizes
        x = ((rng.standard_normal(1 << c) + 1j * rng.standard_normal(1 << c)) * scale * 2.0 ** (-c / 2)).astype(dt)
        want = _encode(lib, lib.sv_codec_encode, x, c, eb, code)
        got = _encode(lib, fn_na, x, c, eb, code)
        assert got == want, (c, dt)
        again = _encode(lib, fn_na, x, c, eb, code)
        assert again == want


def test_noalloc_rejects_out_of_range_sizes(lib):
    fn_na = lib.sv_codec_encode_noalloc
    fn_na.argtypes = [C.c_int, C.c_int, C.c_double, C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t)]
    d = torch.zeros(1 << 12, dtype=torch.complex64, device="cuda")
    out = torch.zeros(lib.sv_codec_max_bytes(12), dtype=torch.uint8, device="cuda")
    nb = C.c_size_t(0)
    assert fn_na(1, 21, 1e-6, d.data_ptr(), out.data_ptr(), out.numel(), C.byref(nb)) == -1
    assert fn_na(1, 12, 1e-6, d.data_ptr(), out.data_ptr(), out.numel() - 16, C.byref(nb)) == -1
    assert fn_na(1, 12, 1e-6, d.data_ptr(), out.data_ptr(), out.numel(), C.byref(nb)) == 0


def test_noalloc_range_error_then_clean_call(lib):
    """An out-of-range value returns SV_ERR_RANGE; the staging area's error
    word, which persists between calls, must not leak into the next call."""
    fn_na = lib.sv_codec_encode_noalloc
    fn_na.argtypes = [C.c_int, C.c_int, C.c_double, C.c_void_p, C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t)]
    fn_na.restype = C.c_int
    c, eb = 12, 1e-7  # step 2^-23: complex64 codes reach 2^24 - 1, i.e. |x| < 2
    cap = lib.sv_codec_max_bytes(c)
    bad = np.zeros(1 << c, dtype=np.complex64)
    bad[77] = 4.0 - 3.0j
    d_bad = torch.from_numpy(bad).cuda()
    out = torch.zeros(cap, dtype=torch.uint8, device="cuda")
    nb = C.c_size_t(0)
    torch.cuda.synchronize()
    assert fn_na(1, c, eb, d_bad.data_ptr(), out.data_ptr(), cap, C.byref(nb)) == -7  # SV_ERR_RANGE
    rng = np.random.default_rng(7)
    x = ((rng.standard_normal(1 << c) + 1j * rng.standard_normal(1 << c)) * 2.0 ** (-c / 2)).astype(np.complex64)
    want = _encode(lib, lib.sv_codec_encode, x, c, eb, 1)
    assert _encode(lib, fn_na, x, c, eb, 1) == want
