"""Pins for the oracle's Pauli-sum expectation, H|psi> and adjoint gradient:
closed forms, dense Pauli matrices (Kronecker products), parameter shift and
central finite differences."""
import numpy as np
import pytest

import oracle
import workloads as W
from dense_ref import hamiltonian_matrix, pauli_matrix


def test_z_on_basis_states():
    n = 6
    for x in (0, 1, 37, 63):
        psi = oracle.basis_state(n, x)
        for q in range(n):
            e = oracle.expect(n, psi, [W.PauliTerm(1.0, 0, 1 << q)])
            assert e == (-1.0) ** ((x >> q) & 1)


def test_x_on_plus_and_y_on_plus_i():
    n = 3
    plus = oracle.run(n, [W.Gate("H", (q,)) for q in range(n)])
    assert abs(oracle.expect(n, plus, [W.PauliTerm(1.0, 0b111, 0)]) - 1) < 1e-14
    plus_i = oracle.run(n, [W.Gate("H", (1,)), W.Gate("S", (1,))])
    assert abs(oracle.expect(n, plus_i, [W.PauliTerm(1.0, 0b010, 0b010)]) - 1) < 1e-14
    assert abs(oracle.expect(n, plus_i, [W.PauliTerm(1.0, 0b010, 0)])) < 1e-14


def test_ghz_correlators():
    n = 8
    psi = oracle.run(n, W.ghz(n))
    for i in range(n):
        for j in range(i + 1, n):
            assert abs(oracle.expect(n, psi, [W.PauliTerm(1.0, 0, (1 << i) | (1 << j))]) - 1) < 1e-14
    full = (1 << n) - 1
    assert abs(oracle.expect(n, psi, [W.PauliTerm(1.0, full, 0)]) - 1) < 1e-14
    assert abs(oracle.expect(n, psi, [W.PauliTerm(1.0, 0, 1)])) < 1e-14


def test_expect_matches_dense_pauli_matrices():
    n = 5
    rng = np.random.default_rng(5)
    psi = rng.standard_normal(32) + 1j * rng.standard_normal(32)
    psi /= np.linalg.norm(psi)
    terms = W.random_pauli_sum(n, 25, seed=8)
    for t in terms:
        want = np.vdot(psi, pauli_matrix(n, t) @ psi)
        assert abs(want.imag) < 1e-13
        assert abs(oracle.expect(n, psi, [t]) - want.real) < 1e-13
    Hm = hamiltonian_matrix(n, terms)
    assert np.abs(oracle.hamiltonian(n, psi, terms) - Hm @ psi).max() < 1e-13


def test_ising_terms_shape():
    terms = W.ising(24)
    assert len(terms) == 2 * 24 - 1
    assert all(-1 <= t.coeff <= 1 for t in terms)


@pytest.mark.parametrize("n,layers", [(3, 2), (5, 3)])
def test_adjoint_matches_parameter_shift_and_fd(n, layers):
    gates, npar = W.hea(n, layers)
    theta = W.normal_params(npar, seed=3)
    terms = W.ising(n)
    e, g = oracle.adjoint(n, gates, theta, terms)
    assert abs(e - oracle.energy(n, gates, theta, terms)) < 1e-13
    ps = oracle.param_shift(n, gates, theta, terms)
    assert np.abs(g - ps).max() < 1e-12
    fd = oracle.finite_diff(n, gates, theta, terms, range(npar), h=1e-5)
    assert np.abs(g - fd).max() < 1e-8


def test_adjoint_rx_and_nonzero_init_and_dense_energy():
    n = 4
    gates = [W.Gate("RX", (0,), param=0), W.Gate("CNOT", (1,), (0,)), W.Gate("RY", (2,), param=1),
             W.Gate("H", (3,)), W.Gate("RZ", (3,), param=2), W.Gate("CZ", (2,), (3,)),
             W.Gate("RX", (1,), param=3)]
    theta = [0.3, -1.2, 2.0, 0.7]
    terms = W.random_pauli_sum(n, 10, seed=2)
    e, g = oracle.adjoint(n, gates, theta, terms, init=5)
    psi = oracle.run(n, gates, init=5, theta=theta)
    assert abs(e - np.vdot(psi, hamiltonian_matrix(n, terms) @ psi).real) < 1e-13
    ps = oracle.param_shift(n, gates, theta, terms, init=5)
    assert np.abs(g - ps).max() < 1e-12


def test_adjoint_rejects_controlled_parameter():
    n = 2
    gates = [W.Gate("RX", (0,), (1,), param=0)]
    with pytest.raises(oracle.OracleError):
        oracle.adjoint(n, gates, [0.1], [W.PauliTerm(1.0, 0, 1)])
