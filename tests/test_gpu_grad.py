"""Adjoint gradients on the GPU vs the oracle's adjoint recursion, parameter
shift and central finite differences; the autograd wrapper."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def SV():
    from paper_2309_16979_gb300 import StateVector
    return StateVector


@pytest.mark.parametrize("n,layers", [(4, 2), (9, 3), (14, 2)])
def test_adjoint_c128_matches_oracle(SV, n, layers):
    gates, npar = W.hea(n, layers)
    theta = W.normal_params(npar, seed=3)
    terms = W.ising(n)
    e_o, g_o = oracle.adjoint(n, gates, theta, terms)
    with SV(n, mode="uncompressed", dtype="c128") as s:
        e, g = s.grad(gates, theta, terms)
    assert abs(e - e_o) <= 1e-11
    assert np.abs(g - g_o).max() <= 1e-10


def test_adjoint_c64_matches_oracle_and_param_shift(SV):
    n, layers = 10, 3
    gates, npar = W.hea(n, layers)
    theta = W.normal_params(npar, seed=5)
    terms = W.ising(n)
    e_o, g_o = oracle.adjoint(n, gates, theta, terms)
    with SV(n, mode="uncompressed", dtype="c64") as s:
        e, g = s.grad(gates, theta, terms)
    scale = sum(abs(t.coeff) for t in terms)
    assert abs(e - e_o) <= 1e-5 * scale
    assert np.abs(g - g_o).max() <= 1e-5 * scale
    ps = oracle.param_shift(n, gates, theta, terms, params=range(0, npar, 7))
    assert np.abs(g[::7] - ps).max() <= 1e-5 * scale


def test_adjoint_mixed_gates_and_rx(SV):
    n = 6
    gates = [W.Gate("H", (0,)), W.Gate("RX", (0,), param=0), W.Gate("CNOT", (3,), (0,)),
             W.Gate("RY", (5,), param=1), W.Gate("SWAP", (1, 5)), W.Gate("RZ", (1,), param=2),
             W.Gate("CP", (2,), (1,), theta=0.3), W.Gate("RX", (2,), param=0), W.Gate("T", (4,))]
    theta = [0.4, -0.9, 1.7]
    terms = W.random_pauli_sum(n, 12, seed=3)
    e_o, g_o = oracle.adjoint(n, gates, theta, terms, init=9)
    with SV(n, mode="uncompressed", dtype="c128", init_index=9) as s:
        e, g = s.grad(gates, theta, terms)
    assert abs(e - e_o) <= 1e-12 and np.abs(g - g_o).max() <= 1e-11


def test_autograd_function(SV):
    torch = pytest.importorskip("torch")
    from paper_2309_16979_gb300.autograd import expectation
    n, layers = 6, 2
    gates, npar = W.hea(n, layers)
    terms = W.ising(n)
    theta = torch.tensor(W.normal_params(npar, seed=8), dtype=torch.float64, requires_grad=True)
    with SV(n, mode="uncompressed", dtype="c128") as s:
        e = expectation(theta, s, gates, terms)
        (2.0 * e).backward()
    e_o, g_o = oracle.adjoint(n, gates, theta.detach().numpy(), terms)
    assert abs(e.item() - e_o) < 1e-12
    assert np.abs(theta.grad.numpy() - 2 * g_o).max() < 1e-11
