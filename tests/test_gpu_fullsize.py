"""Parity at the full benchmark sizes, in the launch configuration bench.py
times (n = 30, complex64, chunks of 2^22, groups of 2^4 chunks), and beyond
HBM (n = 36): on outputs the oracle can produce one by one (its codec on
stored chunk streams, closed-form amplitudes) and on properties that hold at
any size."""
import math

import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

N, C, G = 30, 22, 4


@pytest.fixture(scope="module")
def SV():
    from paper_2309_16979_gb300 import StateVector
    return StateVector


def test_bench_workload_chunks_decode_bit_exact_with_oracle_codec(SV):
    """After the 1800-gate bench circuit, the oracle decodes stored chunk
    streams to exactly the amplitudes the GPU reads back."""
    gates = W.random_layers(N, 40, seed=1)
    with SV(N, C, 1e-6, init_index=W.basis_index(N), max_group_qubits=G) as s:
        s.apply(gates)
        st = s.stats()
        for k in (0, 77, 255):
            ref = oracle.codec_decode(s.chunk_stream(k), C, np.complex64)
            got = s.amplitudes_range(k << C, 1 << C)
            assert np.array_equal(got.real, ref.real.astype(np.float64))
            assert np.array_equal(got.imag, ref.imag.astype(np.float64))
    assert st["passes"] >= 10 and st["compressed_bytes"] < st["raw_bytes"]


def test_bench_workload_circuit_then_inverse(SV):
    """U then U^dagger returns the basis state up to the quantisation noise:
    each pass adds independent rounding of variance Delta^2/12 per stored real
    number, so the expected infidelity is about P * 2^(n+1) * Delta^2 / 12."""
    gates = W.random_layers(N, 40, seed=1)
    x = W.basis_index(N)
    with SV(N, C, 1e-6, init_index=x, max_group_qubits=G) as s:
        s.apply(gates)
        s.apply(W.inverse(gates))
        st = s.stats()
        a = s.amplitudes([x])[0]
    delta = 2.0 ** -19
    expected_loss = st["passes"] * (2 << N) * delta ** 2 / 12
    fid = abs(a) ** 2 / st["norm2"]
    assert fid >= 1 - 4 * expected_loss - 1e-3, (fid, expected_loss)


def test_ghz30_closed_form(SV):
    with SV(N, C, 1e-6, max_group_qubits=G) as s:
        s.apply(W.ghz(N))
        st = s.stats()
        rng = np.random.default_rng(0)
        idx = np.concatenate([[0, (1 << N) - 1], rng.integers(1, (1 << N) - 1, 2000)])
        a = s.amplitudes(idx)
    tol = st["passes"] * math.sqrt(2) * 1e-6
    assert abs(a[0] - 2 ** -0.5) <= tol and abs(a[1] - 2 ** -0.5) <= tol
    assert np.all(a[2:] == 0)


def test_qft30_sampled_against_closed_form(SV):
    """The error vector has ||e||^2 <= (P sqrt(2^(n+1)) eb)^2, so the mean
    squared error per amplitude is <= 2 P^2 eb^2; a 4096-point sample mean is
    checked against that with 50 % sampling slack."""
    eb = 1e-7
    x = W.basis_index(N)
    with SV(N, C, eb, init_index=x, max_group_qubits=G) as s:
        s.apply(W.qft(N))
        st = s.stats()
        k = np.random.default_rng(1).integers(0, 1 << N, 4096).astype(np.uint64)
        got = s.amplitudes(k)
    kk = k.astype(np.float64)
    phase = 2 * np.pi * ((x * k.astype(object)) % (1 << N)).astype(np.float64) / (1 << N)
    want = np.exp(1j * phase) / math.sqrt(1 << N)
    mse = np.mean(np.abs(got - want) ** 2)
    assert mse <= 1.5 * 2 * st["passes"] ** 2 * eb ** 2
    assert abs(st["norm2"] - 1) < 0.05
    del kk


@pytest.mark.slow
def test_ghz36_beyond_hbm(SV):
    """n = 36 complex64 is 512 GiB raw (more than HBM); the compressed store
    holds GHZ-36 in pinned host memory and streams it in 2^26-amplitude chunks."""
    n, c = 36, 26
    with SV(n, c, 1e-5, max_group_qubits=4) as s:
        s.apply(W.ghz(n))
        st = s.stats()
        a = s.amplitudes([0, (1 << n) - 1, 12345, (1 << n) - 2])
    assert st["raw_bytes"] == 8 << n
    assert st["compressed_bytes"] < st["raw_bytes"] // 50
    tol = st["passes"] * math.sqrt(2) * 1e-5
    assert abs(a[0] - 2 ** -0.5) <= tol and abs(a[1] - 2 ** -0.5) <= tol
    assert a[2] == 0 and a[3] == 0
