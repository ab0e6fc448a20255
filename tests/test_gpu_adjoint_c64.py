"""The complex64 generated adjoint kernels (psi and lambda updated together in
packed FP32x2 instructions, FP32 warp partials summed per CTA in FP64)
against the FP64 oracle's adjoint recursion and parameter shift.

These kernels run only when a tile sub-pass holds 2^12 amplitudes, i.e. when
the state (uncompressed) or a staged chunk group (compressed) has at least
12 + 2 local qubits of which 12 form the tile; every case asserts that the
reverse sweep launched them, so a fallback to the table-driven kernel cannot
pass silently.

Tolerance: 1e-5 * sum|c| for energy and every gradient entry (complex64
arithmetic: each gate rounds every output at 2^-24 relative and a unitary
carries earlier errors unchanged in norm; a few hundred gates on psi and
lambda stay well inside it); compressed cases add the quantisation bound of
both stores."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def SV():
    from paper_2309_16979_gb300 import StateVector
    return StateVector


def _scale(terms):
    return sum(abs(t.coeff) for t in terms)


@pytest.mark.parametrize("n,layers,seed", [(14, 2, 11), (14, 3, 12), (16, 3, 13)])
def test_c64_generated_adjoint_uncompressed(SV, n, layers, seed):
    gates, npar = W.hea(n, layers)
    theta = W.normal_params(npar, seed=seed)
    terms = W.ising(n, seed=seed)
    e_o, g_o = oracle.adjoint(n, gates, theta, terms)
    with SV(n, mode="uncompressed", dtype="c64") as s:
        e, g = s.grad(gates, theta, terms)
        st = s.stats()
    assert st["jit_adjoint_launches"] > 0
    tol = 1e-5 * _scale(terms)
    assert abs(e - e_o) <= tol
    assert np.abs(g - g_o).max() <= tol
    sub = list(range(0, npar, 9))
    ps = oracle.param_shift(n, gates, theta, terms, params=sub)
    assert np.abs(g[sub] - ps).max() <= tol


def test_c64_generated_adjoint_mixed_generators(SV):
    """RX, RY and RZ parameters, a parameter shared by two gates, fixed gates
    between them, and a Pauli sum with X, Y and Z factors on every qubit."""
    n = 14
    rng = np.random.default_rng(5)
    gates = []
    p = 0
    for layer in range(3):
        for q in range(n):
            kind = ("RX", "RY", "RZ")[(q + layer) % 3]
            gates.append(W.Gate(kind, (q,), param=p))
            p += 1
        for q in range(0, n - 1, 2):
            gates.append(W.Gate("CNOT", ((q + 1 + layer) % n,), (q,)))
        gates.append(W.Gate("H", (layer,)))
        gates.append(W.Gate("CP", (n - 1,), (layer + 2,), theta=0.37))
    gates.append(W.Gate("RY", (5,), param=3))  # parameter 3 used twice
    theta = rng.normal(0.0, 0.4, p)
    terms = W.random_pauli_sum(n, 24, seed=21)
    e_o, g_o = oracle.adjoint(n, gates, theta, terms, init=77)
    with SV(n, mode="uncompressed", dtype="c64", init_index=77) as s:
        e, g = s.grad(gates, theta, terms)
        assert s.stats()["jit_adjoint_launches"] > 0
    tol = 1e-5 * _scale(terms)
    assert abs(e - e_o) <= tol and np.abs(g - g_o).max() <= tol


@pytest.mark.parametrize("relative", [False, True])
def test_c64_generated_adjoint_compressed(SV, relative):
    """n = 16, chunks of 2^10, 3 staged high qubits: groups of 2^13
    amplitudes, so the reverse sweep's sub-passes run on 2^12 tiles. Bound:
    each re-encoding of psi moves every stored real number by at most eb
    (absolute) or eb * (largest component of the chunk) <= eb (relative), so
    by at most q = sqrt(2 * 2^n) eb in L2; lambda's step carries the next
    power of two of sum|c|. A gradient term moves by at most
    sum|c| (P + 2 (P + 1)) q over P passes."""
    n, c, gq, eb = 16, 10, 3, 1e-6
    gates, npar = W.hea(n, 2)
    theta = W.normal_params(npar, seed=17)
    terms = W.ising(n, seed=4)
    e_o, g_o = oracle.adjoint(n, gates, theta, terms, init=5)
    with SV(n, c, eb, dtype="c64", init_index=5, max_group_qubits=gq, relative_bound=relative) as s:
        e, g = s.grad(gates, theta, terms)
        st = s.stats()
    assert st["jit_adjoint_launches"] > 0
    P = st["passes"]
    scale = _scale(terms)
    q = np.sqrt(2.0 * (1 << n)) * eb
    arith = 1e-5 * scale
    assert abs(e - e_o) <= scale * P * q + arith
    assert np.abs(g - g_o).max() <= scale * (P + 2 * (P + 1)) * q + arith


@pytest.mark.slow
def test_c64_generated_adjoint_hea24_full_size(SV):
    """The adjoint gradient workload at full size: n = 24, 10 HEA layers (480
    parameters, 710 gates), open-chain Ising with J, h ~ U[-1, 1] (seed 4),
    complex64 uncompressed in HBM, in the launch configuration the benchmark
    times; every energy and gradient entry against the FP64 oracle."""
    n, layers = 24, 10
    gates, npar = W.hea(n, layers)
    assert npar == 480
    theta = W.normal_params(npar, seed=3)
    terms = W.ising(n)
    with SV(n, mode="uncompressed", dtype="c64") as s:
        e, g = s.grad(gates, theta, terms)
        st = s.stats()
    assert st["jit_adjoint_launches"] > 0
    e_o, g_o = oracle.adjoint(n, gates, theta, terms)
    tol = 1e-5 * _scale(terms)
    assert abs(e - e_o) <= tol
    assert np.abs(g - g_o).max() <= tol
