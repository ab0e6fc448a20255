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


@pytest.mark.parametrize("mode", ["uncompressed", "compressed"])
def test_energy_without_gradient(SV, mode):
    """sv_grad with grad = NULL (StateVector.energy, and the autograd wrapper
    under no_grad): the forward sweep and the expectation only -- no reverse
    sweep launches -- with the energy sv_grad reports."""
    torch = pytest.importorskip("torch")
    from paper_2309_16979_gb300.autograd import expectation
    n, layers = 14, 2
    gates, npar = W.hea(n, layers)
    theta = W.normal_params(npar, seed=31)
    terms = W.ising(n)
    with SV(n, 10, 1e-9, dtype="c128", mode=mode, max_group_qubits=2) as s:
        e_full, _ = s.grad(gates, theta, terms)
        a = s.stats()
        e = s.energy(gates, theta, terms)
        with torch.no_grad():
            e_t = expectation(torch.tensor(theta, dtype=torch.float64, requires_grad=True), s, gates, terms)
        b = s.stats()
    assert b["jit_adjoint_launches"] == a["jit_adjoint_launches"]
    e_o, _ = oracle.adjoint(n, gates, theta, terms)
    scale = sum(abs(t.coeff) for t in terms)
    # compressed: every pass re-quantises psi (L2 move <= sqrt(2 * 2^n) eb each)
    tol = 1e-11 if mode == "uncompressed" else scale * b["passes"] * np.sqrt(2.0 * (1 << n)) * 1e-9 + 1e-12
    assert abs(e - e_o) <= tol and abs(e_t.item() - e) <= 1e-15 and abs(e_full - e_o) <= tol


@pytest.mark.parametrize("dtype,eb", [("c128", 1e-9), ("c64", 1e-6)])
def test_compressed_adjoint_within_quantisation_bound(SV, dtype, eb):
    """psi and lambda both as compressed chunk stores. Each re-encoding of psi
    moves every stored real number by <= eb (L2 <= sqrt(2 * 2^n) eb = q); the
    lambda store's step is scaled by the next power of two of sum|c| (< 2
    sum|c|), so its re-encodings move it by < 2 sum|c| q. A gradient term
    Im<lambda|G|psi> moves by at most |lambda| |d psi| + |d lambda| with
    |lambda| <= sum|c|: |d g| <= sum|c| (P + 2 (P + 1)) q (+ arithmetic)."""
    n, c, g = 12, 8, 3
    gates, npar = W.hea(n, 2)
    theta = W.normal_params(npar, seed=6)
    terms = W.ising(n)
    e_o, g_o = oracle.adjoint(n, gates, theta, terms, init=3)
    with SV(n, c, eb, dtype=dtype, init_index=3, max_group_qubits=g) as s:
        e, gr = s.grad(gates, theta, terms)
        st = s.stats()
    # lambda's sources from the host store (0) or a device copy of the
    # compressed psi (2) instead of the decoded psi (1): the same bits
    for cache in (0, 2):
        with SV(n, c, eb, dtype=dtype, init_index=3, max_group_qubits=g, lambda_cache=cache) as s:
            e2, gr2 = s.grad(gates, theta, terms)
        assert e2 == e and np.array_equal(gr2, gr), cache
    P = st["passes"]  # forward + reverse passes
    scale = sum(abs(t.coeff) for t in terms)
    q = np.sqrt(2.0 * (1 << n)) * eb
    arith = 0.0 if dtype == "c128" else 64 * 2.0 ** -24 * len(gates) * scale
    assert abs(e - e_o) <= scale * P * q + arith + 1e-12
    assert np.abs(gr - g_o).max() <= scale * (P + 2 * (P + 1)) * q + arith + 1e-12


def test_compressed_adjoint_agrees_with_uncompressed_gpu(SV):
    n = 13
    gates, npar = W.hea(n, 2)
    theta = W.normal_params(npar, seed=9)
    terms = W.ising(n)
    with SV(n, mode="uncompressed", dtype="c128") as s:
        e_u, g_u = s.grad(gates, theta, terms)
    with SV(n, 9, 1e-9, dtype="c128", max_group_qubits=4) as s:
        e_c, g_c = s.grad(gates, theta, terms)
    assert abs(e_c - e_u) < 1e-4 and np.abs(g_c - g_u).max() < 1e-4


@pytest.mark.parametrize("cache", [0, 1, 2])
@pytest.mark.parametrize("dtype,eb", [("c128", 1e-9), ("c64", 1e-6)])
def test_compressed_adjoint_with_more_high_x_masks_than_a_group(SV, dtype, eb, cache):
    """lambda = H psi when the terms' distinct high x-masks (0, 1, 2, 4, 8, 9
    over 4 high qubits) outnumber the 4 chunks a staging group holds: two
    batches per output chunk, accumulated before one encode, when the
    sources are staged (lambda_cache 0: from the host, 2: from a device copy
    of the compressed psi); one pass over the decoded psi with 1. Same bound
    as the single-batch case."""
    n, c = 12, 8
    gates, npar = W.hea(n, 2)
    theta = W.normal_params(npar, seed=12)
    terms = [W.PauliTerm(0.3 + 0.05 * q, 1 << q, 0) for q in range(n)] + \
        [W.PauliTerm(0.5, (1 << 11) | (1 << 8), 1 << 3), W.PauliTerm(-0.7, (1 << 9) | 3, (1 << 9) | (1 << 2))]
    e_o, g_o = oracle.adjoint(n, gates, theta, terms, init=6)
    with SV(n, c, eb, dtype=dtype, init_index=6, max_group_qubits=2, lambda_cache=cache) as s:
        e, gr = s.grad(gates, theta, terms)
        P = s.stats()["passes"]
    scale = sum(abs(t.coeff) for t in terms)
    q = np.sqrt(2.0 * (1 << n)) * eb
    arith = 0.0 if dtype == "c128" else 64 * 2.0 ** -24 * len(gates) * scale
    assert abs(e - e_o) <= scale * P * q + arith + 1e-12
    assert np.abs(gr - g_o).max() <= scale * (P + 2 * (P + 1)) * q + arith + 1e-12


@pytest.mark.parametrize("n,c", [(12, 8), (15, 11)])
@pytest.mark.parametrize("dtype,eb", [("c128", 1e-9), ("c64", 1e-6)])
def test_compressed_lambda_runs_of_terms_sharing_a_source(SV, dtype, eb, n, c):
    """lambda = H psi sums, per output, the terms that read the same source
    (high and low x-mask) as one coefficient times one source amplitude.
    Here several x-masks (low, high, both, none; some on local bits 8..10,
    where a thread's 8 outputs differ) each carry terms with different
    z-masks (some on bits 8..10, some overlapping the x-mask: Y factors, odd
    and even counts), listed in an order that interleaves the sources. With
    c = 11 the chunks are at least one 2048-output strip long."""
    gates, npar = W.hea(n, 2)
    theta = W.normal_params(npar, seed=14)
    xs = [0, 1 << 2, (1 << (c + 1)) | (1 << 1), (1 << (c + 2)) | (1 << 9), (1 << c) | (1 << (c + 3)) | 5]
    zs = [0, 1 << 2, (1 << (c + 1)) | (1 << 3), (1 << 1) | (1 << (c + 3)), 0b11100000111 | (1 << c),
          (1 << (c + 1)) | 2]
    terms = [W.PauliTerm(0.1 + 0.07 * i - 0.03 * j, x, z) for j, z in enumerate(zs) for i, x in enumerate(xs)]
    assert any(bin(t.xmask & t.zmask).count("1") % 2 for t in terms)
    assert any(bin(t.xmask & t.zmask).count("1") == 2 for t in terms)
    e_o, g_o = oracle.adjoint(n, gates, theta, terms, init=5)
    with SV(n, c, eb, dtype=dtype, init_index=5, max_group_qubits=3) as s:
        e, gr = s.grad(gates, theta, terms)
        P = s.stats()["passes"]
    scale = sum(abs(t.coeff) for t in terms)
    q = np.sqrt(2.0 * (1 << n)) * eb
    arith = 0.0 if dtype == "c128" else 64 * 2.0 ** -24 * len(gates) * scale
    assert abs(e - e_o) <= scale * P * q + arith + 1e-12
    assert np.abs(gr - g_o).max() <= scale * (P + 2 * (P + 1)) * q + arith + 1e-12


def test_compressed_adjoint_diagonal_parameters_on_high_qubits(SV):
    """Parameterised RZ gates on the chunk-index (high) qubits ahead of any
    gate that mixes them: a diagonal gate needs no staged qubit to run, but
    the reverse sweep takes each parameter's partial on the tile, so the
    gradient's passes stage those targets too (the library refuses a plan
    that does not). Energy and gradient against the oracle."""
    n, c, g = 13, 8, 2
    gates = [W.Gate("RZ", (q,), param=q - c) for q in range(c, n)]          # params 0..4 on high qubits
    gates += [W.Gate("H", (q,)) for q in range(c)]
    gates += [W.Gate("CNOT", (q + 1,), (q,)) for q in range(n - 1)]
    gates += [W.Gate("RZ", (q,), param=5 + q) for q in range(n)]
    gates += [W.Gate("RX", (q,), param=5 + n + q) for q in range(n)]
    npar = 5 + 2 * n
    theta = W.normal_params(npar, seed=31)
    terms = W.ising(n)
    e_o, g_o = oracle.adjoint(n, gates, theta, terms, init=9)
    with SV(n, c, 1e-9, dtype="c128", init_index=9, max_group_qubits=g) as s:
        e, gr = s.grad(gates, theta, terms)
        P = s.stats()["passes"]
    scale = sum(abs(t.coeff) for t in terms)
    q = np.sqrt(2.0 * (1 << n)) * 1e-9
    assert abs(e - e_o) <= scale * P * q + 1e-12
    assert np.abs(gr - g_o).max() <= scale * (P + 2 * (P + 1)) * q + 1e-12


@pytest.mark.parametrize("dtype,eb", [("c64", 1e-4), ("c128", 1e-7)])
def test_compressed_adjoint_checkpoints(SV, dtype, eb):
    """checkpoint_passes = 1: the forward sweep keeps psi after each of its 7
    passes but the last, and the reverse sweep resumes from them, so psi's
    error comes from the forward passes only (plus one reverse re-encoding)
    instead of growing over forward and reverse sweeps. Both runs obey the
    uncompute bound against the oracle, the energy (taken before the reverse
    sweep) is the same, and the reverse sweep did use the checkpoints (the
    gradients differ). Lambda's store, re-encoded in every reverse pass with
    a step 2^ceil(log2 sum|c|) times psi's, is not checkpointed, so the
    gradient error need not shrink."""
    n, c, g = 14, 8, 2
    gates, npar = W.hea(n, 2)
    theta = W.normal_params(npar, seed=21)
    terms = W.ising(n)
    e_o, g_o = oracle.adjoint(n, gates, theta, terms, init=9)
    out = {}
    for K in (0, 1):
        with SV(n, c, eb, dtype=dtype, init_index=9, max_group_qubits=g, checkpoint_passes=K) as s:
            e, gr = s.grad(gates, theta, terms)
            st = s.stats()
        out[K] = (e, gr, st)
    P = out[0][2]["passes"]
    assert out[0][2]["checkpoints"] == 0 and out[1][2]["checkpoints"] == P // 2 - 1 > 0
    assert out[1][2]["checkpoint_bytes"] > 0
    scale = sum(abs(t.coeff) for t in terms)
    q = np.sqrt(2.0 * (1 << n)) * eb
    arith = 0.0 if dtype == "c128" else 64 * 2.0 ** -24 * len(gates) * scale
    for K in (0, 1):
        e, gr, _ = out[K]
        assert abs(e - e_o) <= scale * P * q + arith + 1e-12
        assert np.abs(gr - g_o).max() <= scale * (P + 2 * (P + 1)) * q + arith + 1e-12
    assert out[0][0] == out[1][0]
    assert not np.array_equal(out[0][1], out[1][1])
