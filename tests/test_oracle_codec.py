"""Pins for the oracle's reference codec: hand-worked byte streams, the
pointwise error bound, exactness properties of a power-of-two step, and
rejection of out-of-range inputs and corrupt streams."""
import json
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def test_step_exponent_is_largest_power_of_two_below_2eb():
    for eb, k in [(1e-6, -19), (1e-5, -16), (1e-4, -13), (0.5, 0), (2.0 ** -11, -10),
                  (1e-3, -9), (0.3, -1)]:
        assert oracle.step_exponent(eb) == k
        assert 2.0 ** k <= 2 * eb < 2.0 ** (k + 1)


def test_golden_ramp_stream():
    g = _load("codec_ramp_c64.json")
    amps = np.zeros(256, dtype=np.complex64)
    amps.real = np.arange(256) * 2.0 ** -10
    s = oracle.codec_encode(amps, g["eb"])
    assert s.hex() == "".join(g["stream_hex"])
    assert len(s) == g["nbytes"]
    assert np.array_equal(oracle.codec_decode(s, 8), amps)


def test_golden_ties_stream():
    g = _load("codec_ties_c64.json")
    amps = np.full(256, g["re_fill"] + 1j * g["im_fill"], dtype=np.complex64)
    amps.real[:4] = g["re_head"]
    s = oracle.codec_encode(amps, g["eb"])
    assert s.hex() == "".join(g["stream_hex"])
    d = oracle.codec_decode(s, 8)
    assert list(d.real[:4]) == g["decoded_re_head"]
    assert np.all(d.imag == g["im_fill"])


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
@pytest.mark.parametrize("eb", [1e-3, 1e-5, 1e-6, 3.7e-7])
def test_error_bound_holds_pointwise(dtype, eb):
    rng = np.random.default_rng(7)
    c = 10
    x = (rng.standard_normal(1 << c) + 1j * rng.standard_normal(1 << c)) * 0.03
    x = x.astype(dtype)
    d = oracle.codec_decode(oracle.codec_encode(x, eb), c, dtype)
    assert np.abs(d.real.astype(np.float64) - x.real.astype(np.float64)).max() <= eb
    assert np.abs(d.imag.astype(np.float64) - x.imag.astype(np.float64)).max() <= eb
    # the reconstruction is an exact multiple of the step
    k = oracle.step_exponent(eb)
    q = d.real.astype(np.float64) * 2.0 ** -k
    assert np.array_equal(q, np.rint(q))


def test_reencode_of_decoded_is_identical():
    rng = np.random.default_rng(1)
    x = ((rng.standard_normal(2048) + 1j * rng.standard_normal(2048)) * 0.1).astype(np.complex64)
    s = oracle.codec_encode(x, 1e-5)
    d = oracle.codec_decode(s, 11)
    assert oracle.codec_encode(d, 1e-5) == s


def test_zero_and_constant_chunks_have_width_zero():
    c = 9
    for val in (0.0, 0.25 + 0.5j, -1.0):
        x = np.full(1 << c, val, dtype=np.complex64)
        s = oracle.codec_encode(x, 1e-6)
        nb = 2 * (1 << c) // 256
        assert s[32:32 + nb] == bytes(nb)
        assert len(s) == oracle.codec_meta_bytes(c)
        assert np.array_equal(oracle.codec_decode(s, c), x)


def test_alternating_sign_and_unit_magnitude():
    c = 8
    x = np.zeros(256, dtype=np.complex64)
    x.real = np.where(np.arange(256) % 2 == 0, 1.0, -1.0)
    x.imag[7] = 1.0
    s = oracle.codec_encode(x, 1e-6)
    d = oracle.codec_decode(s, c)
    assert np.abs(d - x).max() <= 1e-6
    # residuals alternate between -2q and +2q with q = 2^19: width = bitlen(2*2^20) = 22
    assert s[32] == 22


def test_basis_state_chunk_roundtrip_exact():
    x = np.zeros(1 << 12, dtype=np.complex64)
    x[1234] = 1.0
    d = oracle.codec_decode(oracle.codec_encode(x, 1e-5), 12)
    assert np.array_equal(d, x)


def test_range_errors():
    x = np.zeros(256, dtype=np.complex64)
    x[3] = 2.0
    assert oracle.codec_status_encode(x, 1e-8) == -7          # |q| = 2^25 > 2^24 - 1
    x[3] = np.nan
    assert oracle.codec_status_encode(x, 1e-3) == -7
    y = np.zeros(256, dtype=np.complex128)
    y[0] = 1.0
    assert oracle.codec_status_encode(y, 1e-9) == 0           # q = 2^29 fits complex128
    assert oracle.codec_status_encode(y, 1e-10) == -7


def test_corrupt_streams_rejected():
    rng = np.random.default_rng(3)
    x = ((rng.standard_normal(512) + 1j * rng.standard_normal(512)) * 0.1).astype(np.complex64)
    s = bytearray(oracle.codec_encode(x, 1e-4))
    assert oracle.codec_status_decode(bytes(s), 9) == 0
    bad = bytearray(s); bad[0] ^= 1
    assert oracle.codec_status_decode(bytes(bad), 9) == -4      # magic
    bad = bytearray(s); bad[32] = 33
    assert oracle.codec_status_decode(bytes(bad), 9) == -4      # width > 32
    bad = bytearray(s); bad[32] = (bad[32] + 1) % 32
    assert oracle.codec_status_decode(bytes(bad), 9) == -4      # offsets inconsistent
    assert oracle.codec_status_decode(bytes(s[:-4]), 9) == -4   # truncated payload
    assert oracle.codec_status_decode(bytes(s), 10) == -4       # wrong chunk size


# ------------------------------------------------------- relative bound
def test_relative_exponent_brackets_2_eb_m():
    """k = floor(log2(2 eb m)), checked against the power of two it must sit
    under, clamped to [-60, 0]; k = 0 for an all-zero chunk."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        eb = 10.0 ** rng.uniform(-7, -1)
        m = 10.0 ** rng.uniform(-12, 0.5)
        k = oracle.codec_relative_exponent(eb, m)
        v = 2 * eb * m
        if v >= 1.0:
            assert k == 0
        elif v < 2.0 ** -59:
            assert k == -60
        else:
            assert 2.0 ** k <= v < 2.0 ** (k + 1)
    assert oracle.codec_relative_exponent(1e-5, 0.0) == 0
    assert oracle.codec_relative_exponent(1e-5, 2.0 ** -18) == -34  # 2e-5 * 2^-18 = 7.6e-11 -> 2^-34


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
@pytest.mark.parametrize("scale", [1.0, 2.0 ** -9, 2.0 ** -18, 1e-12])
def test_relative_bound_holds_pointwise(dtype, scale):
    """|x - xhat| <= max(eb * m, 2^-61), m the chunk's largest component."""
    rng = np.random.default_rng(11)
    c, eb = 10, 1e-4
    x = ((rng.standard_normal(1 << c) + 1j * rng.standard_normal(1 << c)) * scale).astype(dtype)
    m = max(np.abs(x.real).max(), np.abs(x.imag).max())
    d = oracle.codec_decode(oracle.codec_encode(x, eb, relative=True), c, dtype)
    bound = max(eb * float(m), 2.0 ** -61)
    assert np.abs(d.real.astype(np.float64) - x.real.astype(np.float64)).max() <= bound
    assert np.abs(d.imag.astype(np.float64) - x.imag.astype(np.float64)).max() <= bound


def test_relative_equals_absolute_when_the_chunk_peaks_at_one():
    """A chunk whose largest component is exactly 1 gets the absolute step:
    the two encodings are the same bytes."""
    rng = np.random.default_rng(5)
    x = ((rng.standard_normal(1024) + 1j * rng.standard_normal(1024)) * 0.2).astype(np.complex64)
    x.real[17] = 1.0
    x.real = np.clip(x.real, -1, 1)
    x.imag = np.clip(x.imag, -1, 1)
    for eb in (1e-3, 1e-5, 1e-6):
        assert oracle.codec_encode(x, eb, relative=True) == oracle.codec_encode(x, eb)


def test_relative_bound_keeps_a_spread_state():
    """Amplitudes of 2^-8 under eb = 1e-2: the absolute step (2^-6) rounds
    every component to zero, the relative one keeps them to 1 %."""
    n = 16
    x = np.full(1 << 10, 2.0 ** -(n / 2) * np.exp(0.3j), dtype=np.complex64)
    da = oracle.codec_decode(oracle.codec_encode(x, 1e-2), 10)
    dr = oracle.codec_decode(oracle.codec_encode(x, 1e-2, relative=True), 10)
    assert not np.any(da)
    assert np.abs(dr - x).max() <= 1e-2 * 2.0 ** -(n / 2) * 2 ** 0.5
