"""GPU chunk codec vs the oracle's reference codec: byte-exact streams on
identical inputs, bit-exact decodes, the error bound, and corrupt-stream
rejection. Calls go through the C ABI (sv_codec_encode / sv_codec_decode)."""
import json
import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
GOLD = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def sv():
    import paper_2309_16979_gb300 as sv
    return sv


def _planes(kind, c, dtype, seed=0):
    rng = np.random.default_rng(seed)
    n = 1 << c
    if kind == "random":
        x = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * 2.0 ** (-c / 2)
    elif kind == "smooth":
        k = np.arange(n)
        x = np.exp(2j * np.pi * 37 * k / n) / np.sqrt(n)
    elif kind == "zero":
        x = np.zeros(n)
    elif kind == "constant":
        x = np.full(n, 0.3 - 0.2j)
    elif kind == "alternating":
        x = np.where(np.arange(n) % 2 == 0, 0.7, -0.7) + 0.1j
    elif kind == "unit":
        x = np.zeros(n, dtype=complex)
        x[rng.integers(n)] = 1.0
        x[rng.integers(n)] = -1j
    elif kind == "wide":
        x = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * 0.3
    else:
        raise ValueError(kind)
    return x.astype(dtype)


def _gpu_encode(sv, x, eb):
    d = torch.from_numpy(x).cuda()
    stream, nb = sv.codec_encode(d, eb)
    return stream[:nb].cpu().numpy().tobytes()


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
@pytest.mark.parametrize("kind", ["random", "smooth", "zero", "constant", "alternating", "unit", "wide"])
@pytest.mark.parametrize("c", [8, 11, 14])
def test_stream_bytes_match_oracle(sv, dtype, kind, c):
    for eb in (1e-4, 1e-6):
        x = _planes(kind, c, dtype, seed=c)
        assert _gpu_encode(sv, x, eb) == oracle.codec_encode(x, eb), (kind, c, eb)


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
def test_decode_bit_exact_and_bounded(sv, dtype):
    c = 13
    for seed, eb in [(1, 1e-5), (2, 3.3e-6), (3, 1e-3)]:
        x = _planes("random", c, dtype, seed)
        ref = oracle.codec_encode(x, eb)
        d_stream = torch.from_numpy(np.frombuffer(ref, dtype=np.uint8).copy()).cuda()
        got = sv.codec_decode(d_stream, len(ref), c, "c64" if dtype == np.complex64 else "c128").cpu().numpy()
        want = oracle.codec_decode(ref, c, dtype)
        assert np.array_equal(got.view(np.uint8), want.view(np.uint8))
        err = np.maximum(np.abs(got.real.astype(float) - x.real), np.abs(got.imag.astype(float) - x.imag))
        assert err.max() <= eb


def test_golden_streams_on_gpu(sv):
    for name in ("codec_ramp_c64.json", "codec_ties_c64.json"):
        g = json.load(open(os.path.join(GOLD, name)))
        if "re_head" in g:
            x = np.full(256, g["re_fill"] + 1j * g["im_fill"], dtype=np.complex64)
            x.real[:4] = g["re_head"]
        else:
            x = np.zeros(256, dtype=np.complex64)
            x.real = np.arange(256) * 2.0 ** -10
        assert _gpu_encode(sv, x, g["eb"]).hex() == "".join(g["stream_hex"])


def test_range_error_on_gpu(sv):
    x = np.zeros(256, dtype=np.complex64)
    x[5] = 2.0
    with pytest.raises(sv.SvError) as ei:
        _gpu_encode(sv, x, 1e-8)
    assert ei.value.code == -7
    x[5] = np.inf
    with pytest.raises(sv.SvError):
        _gpu_encode(sv, x, 1e-3)


def test_corrupt_streams_rejected_on_gpu(sv):
    c = 10
    x = _planes("random", c, np.complex64, 5)
    ref = bytearray(oracle.codec_encode(x, 1e-4))
    cases = []
    bad = bytearray(ref); bad[0] ^= 1; cases.append((bad, len(bad)))
    bad = bytearray(ref); bad[32] = 40; cases.append((bad, len(bad)))
    bad = bytearray(ref); bad[33] = (bad[33] + 3) % 32; cases.append((bad, len(bad)))
    cases.append((bytearray(ref), len(ref) - 64))
    for buf, nb in cases:
        d = torch.from_numpy(np.frombuffer(bytes(buf), dtype=np.uint8).copy()).cuda()
        with pytest.raises(sv.SvError) as ei:
            sv.codec_decode(d, nb, c)
        assert ei.value.code == -4


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
@pytest.mark.parametrize("kind", ["random", "smooth", "zero", "constant", "alternating", "unit", "wide", "tiny"])
@pytest.mark.parametrize("c", [8, 14])
def test_relative_stream_bytes_match_oracle(sv, dtype, kind, c):
    """Relative bound: the per-chunk step from the chunk maximum, GPU against
    the oracle byte for byte, and the bound max(eb m, 2^-61) on the decode."""
    for eb in (1e-2, 1e-5):
        x = _planes("random" if kind == "tiny" else kind, c, dtype, seed=c + 1)
        if kind == "tiny":
            x = (x * 1e-15).astype(dtype)
        d = torch.from_numpy(x).cuda()
        stream, nb = sv.codec_encode(d, eb, relative=True)
        got = stream[:nb].cpu().numpy().tobytes()
        assert got == oracle.codec_encode(x, eb, relative=True)
        back = sv.codec_decode(stream, nb, c, "c64" if dtype == np.complex64 else "c128").cpu().numpy()
        m = max(np.abs(x.real).max(), np.abs(x.imag).max())
        bound = max(eb * float(m), 2.0 ** -61)
        assert np.abs(back.real.astype(np.float64) - x.real.astype(np.float64)).max() <= bound
        assert np.abs(back.imag.astype(np.float64) - x.imag.astype(np.float64)).max() <= bound
