"""Pins for the oracle's state-vector update (plain FP64 loop), against
mathematics that does not depend on it: dense Kronecker-product unitaries,
closed forms (GHZ, QFT of a basis state), unitarity and inverses."""
import numpy as np
import pytest

import oracle
import workloads as W
from dense_ref import circuit_unitary, gate_unitary


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_every_gate_kind_matches_dense_unitary(n):
    gates = W.random_mixed(n, 60, seed=100 + n)
    rng = np.random.default_rng(n)
    psi0 = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi0 /= np.linalg.norm(psi0)
    got = oracle.apply_gates(n, psi0, gates)
    want = circuit_unitary(n, gates) @ psi0
    assert np.abs(got - want).max() < 1e-12


@pytest.mark.parametrize("kind", W.KINDS)
def test_single_gate_each_kind_each_position(kind):
    n = 4
    rng = W.SplitMix64(11)
    for q in range(n):
        for other in range(n):
            if other == q:
                continue
            if kind in ("CNOT", "CZ", "CP"):
                g = W.Gate(kind, (q,), (other,), theta=0.7 if kind == "CP" else 0.0)
            elif kind == "SWAP":
                g = W.Gate(kind, (q, other))
            elif kind == "CUSTOM":
                g = W.Gate(kind, (q, other), mat=W.random_unitary_4x4(rng))
            else:
                g = W.Gate(kind, (q,), theta=1.3 if kind in W.ANGLE_KINDS else 0.0)
            for idx in (0, 5, 15):
                got = oracle.run(n, [g], init=idx)
                want = gate_unitary(n, g)[:, idx]
                assert np.abs(got - want).max() < 1e-13, (kind, q, other, idx)


def test_two_controls_match_dense():
    n = 5
    g = W.Gate("RX", (2,), (0, 4), theta=0.9)
    rng = np.random.default_rng(1)
    psi0 = rng.standard_normal(32) + 1j * rng.standard_normal(32)
    assert np.abs(oracle.apply_gates(n, psi0, [g]) - gate_unitary(n, g) @ psi0).max() < 1e-13


@pytest.mark.parametrize("n", [2, 3, 7, 12])
def test_ghz_closed_form(n):
    psi = oracle.run(n, W.ghz(n))
    want = np.zeros(1 << n, dtype=complex)
    want[0] = want[-1] = 2 ** -0.5
    assert np.abs(psi - want).max() < 1e-14


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 11])
def test_qft_basis_state_closed_form(n):
    for x in {0, 1, (1 << n) - 1, W.basis_index(n)}:
        psi = oracle.run(n, W.qft(n), init=x)
        k = np.arange(1 << n)
        want = np.exp(2j * np.pi * x * k / (1 << n)) / np.sqrt(1 << n)
        assert np.abs(psi - want).max() < 1e-13, (n, x)


def test_qft_matches_dft_matrix():
    n = 6
    U = circuit_unitary(n, W.qft(n))
    N = 1 << n
    k = np.arange(N)
    F = np.exp(2j * np.pi * np.outer(k, k) / N) / np.sqrt(N)
    assert np.abs(U - F).max() < 1e-12
    # and the oracle reproduces each column
    for x in (0, 3, 17, 63):
        assert np.abs(oracle.run(n, W.qft(n), init=x) - F[:, x]).max() < 1e-13


@pytest.mark.parametrize("family", ["layers", "clifford", "mixed"])
def test_circuit_then_inverse_is_identity(family):
    n = 9
    if family == "layers":
        gates = W.random_layers(n, 8, seed=3)
    elif family == "clifford":
        gates = W.random_clifford_rz(n, 8, 3, seed=3)
    else:
        gates = W.random_mixed(n, 200, seed=3)
    rng = np.random.default_rng(2)
    psi0 = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    psi0 /= np.linalg.norm(psi0)
    mid = oracle.apply_gates(n, psi0, gates)
    assert abs(np.linalg.norm(mid) - 1) < 1e-13
    back = oracle.apply_gates(n, mid, W.inverse(gates))
    assert np.abs(back - psi0).max() < 1e-13


def test_dagger_reversed_undoes_circuit():
    n = 6
    gates = W.random_mixed(n, 80, seed=9)
    rng = np.random.default_rng(3)
    psi0 = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    mid = oracle.apply_gates(n, psi0, gates)
    back = mid.copy()
    ga = oracle.gates_to_c(gates)
    st = oracle.lib().or_apply_gates_dagger_reversed(n, back.ctypes.data, oracle.C.addressof(ga),
                                                     len(gates), None)
    assert st == 0
    assert np.abs(back - psi0).max() < 1e-12


def test_invalid_gates_are_rejected():
    with pytest.raises(oracle.OracleError):
        oracle.run(3, [W.Gate("H", (3,))])
    with pytest.raises(oracle.OracleError):
        oracle.run(3, [W.Gate("CNOT", (1,), (1,))])
    with pytest.raises(oracle.OracleError):
        oracle.run(3, [W.Gate("CNOT", (1,))])


def test_planted_mistake_is_caught():
    """A wrong RX sign (theta -> -theta) must fail the dense comparison."""
    n = 3
    g = W.Gate("RX", (1,), theta=0.8)
    wrong = W.Gate("RX", (1,), theta=-0.8)
    good = np.abs(oracle.run(n, [g]) - gate_unitary(n, g)[:, 0]).max()
    bad = np.abs(oracle.run(n, [wrong]) - gate_unitary(n, g)[:, 0]).max()
    assert good < 1e-14 and bad > 1e-2
