"""GPU state-vector path vs the FP64 oracle, through the C ABI.

Uncompressed complex128: relative L2 <= 1e-12. Uncompressed complex64:
within the FP32 arithmetic bound of gpu_util.fp32_tol. Compressed: within the
quantisation bound of gpu_util.compressed_l2_bound (one re-quantisation per
pass, unitaries preserve error norms), plus the closed forms."""
import math

import numpy as np
import pytest

import oracle
import workloads as W
from gpu_util import compressed_l2_bound, fp32_tol, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def SV():
    from paper_2309_16979_gb300 import StateVector
    return StateVector


def _circuits(n):
    return {
        "ghz": W.ghz(n),
        "qft": W.qft(n),
        "layers": W.random_layers(n, 6, seed=4),
        "clifford": W.random_clifford_rz(n, 6, max(1, n // 3), seed=5),
        "mixed": W.random_mixed(n, 150, seed=6),
    }


@pytest.mark.parametrize("name", ["ghz", "qft", "layers", "clifford", "mixed"])
@pytest.mark.parametrize("n", [3, 9, 14])
def test_uncompressed_c128_matches_oracle(SV, name, n):
    gates = _circuits(n)[name]
    init = W.basis_index(n)
    want = oracle.run(n, gates, init=init)
    with SV(n, mode="uncompressed", dtype="c128", init_index=init) as s:
        s.apply(gates)
        got = s.state()
    assert rel_l2(got, want) <= 1e-12


@pytest.mark.parametrize("name", ["ghz", "qft", "layers", "clifford", "mixed"])
@pytest.mark.parametrize("n", [5, 13, 16])
def test_uncompressed_c64_matches_oracle(SV, name, n):
    gates = _circuits(n)[name]
    want = oracle.run(n, gates, init=3)
    with SV(n, mode="uncompressed", dtype="c64", init_index=3) as s:
        s.apply(gates)
        got = s.state()
    assert rel_l2(got, want) <= fp32_tol(len(gates))


@pytest.mark.parametrize("tile", [2, 5, 8, 13])
def test_tile_sizes_agree(SV, tile):
    n = 14
    gates = W.random_mixed(n, 120, seed=9)
    want = oracle.run(n, gates)
    with SV(n, mode="uncompressed", dtype="c128", tile_qubits=tile) as s:
        s.apply(gates)
        assert rel_l2(s.state(), want) <= 1e-12


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("name", ["ghz", "qft", "layers", "clifford", "mixed"])
@pytest.mark.parametrize("n,c,g", [(12, 8, 2), (14, 9, 3), (16, 10, 4), (10, 10, 2)])
def test_compressed_within_quantisation_bound(SV, dtype, name, n, c, g):
    gates = _circuits(n)[name]
    init = W.basis_index(n, seed=7)
    want = oracle.run(n, gates, init=init)
    eb = 1e-6
    with SV(n, c, eb, dtype=dtype, init_index=init, max_group_qubits=g) as s:
        s.apply(gates)
        got = s.state()
        st = s.stats()
    bound = compressed_l2_bound(n, eb, st["passes"], len(gates), dtype)
    assert np.linalg.norm(got - want) <= bound, (st["passes"], np.linalg.norm(got - want), bound)
    assert abs(st["norm2"] - np.vdot(got, got).real) <= 1e-9


def test_compressed_config0_workloads(SV):
    """n=16 complex128, chunk 2^10, eb 1e-6: QFT of a seeded basis state and 20
    random layers, checked against the oracle."""
    n = 16
    x = W.basis_index(n)
    for gates in (W.qft(n), W.random_layers(n, 20, seed=1)):
        want = oracle.run(n, gates, init=x)
        with SV(n, 10, 1e-6, dtype="c128", init_index=x) as s:
            s.apply(gates)
            got = s.state()
            st = s.stats()
        assert np.linalg.norm(got - want) <= compressed_l2_bound(n, 1e-6, st["passes"], len(gates), "c128")
        fid = abs(np.vdot(want, got)) ** 2 / np.vdot(got, got).real
        assert fid > 1 - 1e-3


def test_ghz_and_qft_closed_forms_compressed(SV):
    n, c = 18, 10
    with SV(n, c, 1e-6, max_group_qubits=3) as s:
        s.apply(W.ghz(n))
        a = s.amplitudes([0, (1 << n) - 1, 1, 12345])
    assert abs(a[0] - 2 ** -0.5) <= 1e-5 and abs(a[1] - 2 ** -0.5) <= 1e-5
    assert abs(a[2]) == 0 and abs(a[3]) == 0
    x = W.basis_index(n)
    with SV(n, c, 1e-7, init_index=x) as s:
        s.apply(W.qft(n))
        k = np.array([0, 1, 777, 4095, (1 << n) - 1], dtype=np.uint64)
        got = s.amplitudes(k)
        st = s.stats()
    want = np.exp(2j * np.pi * x * k.astype(float) / (1 << n)) / np.sqrt(1 << n)
    assert np.abs(got - want).max() <= compressed_l2_bound(n, 1e-7, st["passes"], len(W.qft(n)))


def test_swap_relabels_logical_order(SV):
    n = 10
    gates = [W.Gate("X", (0,)), W.Gate("H", (3,)), W.Gate("SWAP", (0, 9)), W.Gate("RY", (9,), theta=0.4),
             W.Gate("SWAP", (3, 5)), W.Gate("CNOT", (2,), (5,))]
    want = oracle.run(n, gates)
    for mode in ("uncompressed", "compressed"):
        with SV(n, 8, 1e-7, mode=mode, dtype="c128") as s:
            s.apply(gates)
            assert np.abs(s.state() - want).max() < 1e-6


def test_sequential_calls_accumulate(SV):
    n = 12
    g1, g2 = W.random_layers(n, 3, seed=1), W.random_layers(n, 3, seed=2)
    want = oracle.run(n, g1 + g2)
    with SV(n, 8, 1e-7, dtype="c128", max_group_qubits=2) as s:
        s.apply(g1)
        s.apply(g2)
        st = s.stats()
        assert np.linalg.norm(s.state() - want) <= compressed_l2_bound(n, 1e-7, st["passes"], 0, "c128")
        assert st["gates_applied"] == len(g1) + len(g2)


@pytest.mark.parametrize("mode", ["uncompressed", "compressed"])
def test_expectation_values(SV, mode):
    n = 12
    gates = W.random_layers(n, 5, seed=3)
    terms = W.ising(n) + W.random_pauli_sum(n, 20, seed=4)
    psi = oracle.run(n, gates)
    with SV(n, 8, 1e-8, mode=mode, dtype="c128", max_group_qubits=2) as s:
        s.apply(gates)
        got = s.expect(terms)
        st = s.stats()
        # against the oracle on the state the GPU holds (pure reduction check)
        held = s.state()
    assert abs(got - oracle.expect(n, held, terms)) <= 1e-12 * sum(abs(t.coeff) for t in terms) + 1e-12
    # and against the exact state, within what the stored-state error allows
    err = np.linalg.norm(held - psi)
    assert abs(got - oracle.expect(n, psi, terms)) <= 2 * err * sum(abs(t.coeff) for t in terms) + 1e-12


@pytest.mark.parametrize("mode", ["uncompressed", "compressed"])
def test_expectation_every_lowest_x_bit(SV, mode):
    """The all-terms energy kernel evaluates X-type terms whose lowest x bit
    is 8 or above on one amplitude of each pair: terms with every lowest x
    bit, with Y factors and z masks, over several strips and CTAs (n = 15),
    against the oracle on the state the GPU holds."""
    n = 15
    gates = W.random_layers(n, 4, seed=8)
    rng = np.random.default_rng(9)
    terms = []
    for b in range(n):
        z = int(rng.integers(0, 1 << n))
        terms += [W.PauliTerm(0.7, 1 << b, 0), W.PauliTerm(-0.4, 1 << b, z | (1 << b)),
                  W.PauliTerm(0.3, (1 << b) | (1 << (n - 1)), z)]
    terms += W.ising(n, seed=5)
    with SV(n, 9, 1e-9, mode=mode, dtype="c128", max_group_qubits=3) as s:
        s.apply(gates)
        got = s.expect(terms)
        held = s.state()
    assert abs(got - oracle.expect(n, held, terms)) <= 1e-12 * sum(abs(t.coeff) for t in terms)


def test_expectation_closed_forms(SV):
    n = 14
    with SV(n, 8, 1e-6, max_group_qubits=2) as s:
        s.apply(W.ghz(n))
        assert abs(s.expect([W.PauliTerm(1.0, 0, (1 << 2) | (1 << 13))]) - 1) < 1e-5
        assert abs(s.expect([W.PauliTerm(1.0, (1 << n) - 1, 0)]) - 1) < 1e-5
        assert abs(s.expect([W.PauliTerm(1.0, 0, 1 << 11)])) < 1e-5


def test_amplitude_indices_and_errors(SV):
    from paper_2309_16979_gb300 import SvError
    n = 11
    gates = W.random_mixed(n, 60, seed=2)
    want = oracle.run(n, gates)
    idx = np.random.default_rng(0).integers(0, 1 << n, 500)
    with SV(n, 8, 1e-7, dtype="c128") as s:
        s.apply(gates)
        got = s.amplitudes(idx)
        assert np.abs(got - want[idx]).max() < 1e-5
        with pytest.raises(SvError):
            s.amplitudes([1 << n])
        with pytest.raises(SvError):
            s.apply([W.Gate("H", (n,))])
        # a rejected circuit leaves the state unchanged
        assert np.abs(s.amplitudes(idx) - got).max() == 0


def test_create_argument_errors(SV):
    from paper_2309_16979_gb300 import SvError
    with pytest.raises(SvError):
        SV(12, 7, 1e-6)
    with pytest.raises(SvError):
        SV(12, 8, 1e-9)  # complex64 quantiser range
    with pytest.raises(SvError):
        SV(12, 8, 1e-6, max_group_qubits=1)


def test_pipeline_slots_agree(SV):
    n = 14
    gates = W.random_layers(n, 4, seed=8)
    outs = []
    for slots in (2, 3, 4):
        with SV(n, 8, 1e-6, pipeline_slots=slots, max_group_qubits=2) as s:
            s.apply(gates)
            outs.append(s.state())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])


def test_compressed_store_is_byte_exact_with_oracle_codec(SV):
    """After a circuit, re-encoding the stored (decoded) state chunk by chunk
    with the oracle codec gives amplitudes equal to what the GPU decodes."""
    n, c = 13, 9
    gates = W.random_layers(n, 3, seed=11)
    with SV(n, c, 1e-5) as s:
        s.apply(gates)
        held = s.state().astype(np.complex64)
    again = oracle.compress_roundtrip(held, c, 1e-5)
    assert np.array_equal(again, held)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_fused_codec_agrees_with_separate_kernels(SV, dtype):
    """Decode inside the first tile sub-pass / encode inside the last gives the
    same stored state, within the quantisation bound, as separate kernels."""
    n, c = 16, 9
    gates = W.random_layers(n, 6, seed=12)
    want = oracle.run(n, gates, init=5)
    outs = []
    for fuse in (True, False):
        with SV(n, c, 1e-6, dtype=dtype, init_index=5, max_group_qubits=3, fuse_codec=fuse) as s:
            s.apply(gates)
            outs.append((s.state(), s.stats()))
    for got, st in outs:
        assert np.linalg.norm(got - want) <= compressed_l2_bound(n, 1e-6, st["passes"], len(gates), dtype)
    assert outs[0][1]["kernel_launches"] < outs[1][1]["kernel_launches"]


def test_phase_kernel_every_gate_kind_and_control(SV):
    """Register-phase tiles (2^12 amplitudes) on every gate kind with controls
    inside, outside and across tiles, complex128 at 1e-12."""
    n = 15
    gates = W.random_mixed(n, 400, seed=21)
    want = oracle.run(n, gates, init=77)
    with SV(n, mode="uncompressed", dtype="c128", init_index=77) as s:
        s.apply(gates)
        assert rel_l2(s.state(), want) <= 1e-12


def test_relative_bound_keeps_a_spread_state(SV):
    """QFT-16 of a basis state at eb = 1e-2: every amplitude (2^-8) sits under
    half the absolute step (2^-7), so the absolute bound collapses the state;
    the relative bound (step from each chunk's largest component) keeps it."""
    import paper_2309_16979_gb300 as P
    n, c, eb = 16, 10, 1e-2
    x = W.basis_index(n)
    gates = W.qft(n)
    want = oracle.run(n, gates, init=x)
    with pytest.raises(P.SvError):
        with SV(n, c, eb, init_index=x) as s:
            s.apply(gates)
    with SV(n, c, eb, init_index=x, relative_bound=True) as s:
        s.apply(gates)
        got = s.state()
        st = s.stats()
    # each pass moves a stored component by at most eb times its chunk's
    # largest component (<= 1)
    assert np.linalg.norm(got - want) <= compressed_l2_bound(n, eb, st["passes"], len(gates))
    fid = abs(np.vdot(want, got)) ** 2 / np.vdot(got, got).real
    assert fid > 1 - 1e-3
    assert abs(st["norm2"] - np.vdot(got, got).real) <= 1e-6


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_relative_store_is_byte_exact_with_oracle_codec(SV, dtype):
    """Relative bound: re-encoding the stored state chunk by chunk with the
    oracle's relative codec reproduces it exactly (each chunk's step is the
    one its own maximum gives), and the circuit stays within the bound."""
    n, c, eb = 14, 9, 1e-4
    gates = W.random_layers(n, 4, seed=13)
    want = oracle.run(n, gates, init=3)
    with SV(n, c, eb, dtype=dtype, init_index=3, max_group_qubits=3, relative_bound=True) as s:
        s.apply(gates)
        held = s.state().astype(np.complex64 if dtype == "c64" else np.complex128)
        st = s.stats()
    assert np.array_equal(oracle.compress_roundtrip(held, c, eb, relative=True), held)
    assert np.linalg.norm(held - want) <= compressed_l2_bound(n, eb, st["passes"], len(gates), dtype)


def test_relative_bound_adjoint_gradient(SV):
    """Compressed adjoint gradient with the relative bound: both stores keep
    their spread amplitudes; the gradient matches the oracle's adjoint to the
    quantisation level."""
    n, c = 12, 8
    gates, npar = W.hea(n, 2)
    theta = np.array(W.normal_params(npar, seed=3))
    terms = W.ising(n, seed=4)
    e_ref, g_ref = oracle.adjoint(n, gates, theta, terms)
    with SV(n, c, 1e-5, max_group_qubits=3, relative_bound=True) as s:
        e, g = s.grad(gates, theta, terms)
    csum = sum(abs(t.coeff) for t in terms)
    assert abs(e - e_ref) <= 1e-3 * csum
    assert np.abs(g - g_ref).max() <= 1e-3 * csum


@pytest.mark.parametrize("n", [1, 2, 3, 5, 11, 12, 13])
def test_small_states_uncompressed(SV, n):
    """States smaller than, equal to and just above one 2^12 tile (the
    generated kernels need L >= 12; below it the table-driven kernels run)."""
    gates = W.random_mixed(n, 60, seed=40 + n)
    want = oracle.run(n, gates, init=1 % (1 << n))
    with SV(n, mode="uncompressed", dtype="c128", init_index=1 % (1 << n)) as s:
        s.apply(gates)
        assert rel_l2(s.state(), want) <= 1e-12


@pytest.mark.parametrize("n,c", [(8, 8), (9, 8), (13, 8), (12, 12)])
def test_degenerate_chunkings(SV, n, c):
    """One chunk (n = c), one or few high qubits, the smallest chunk (2^8):
    within the quantisation bound; an empty gate list changes nothing."""
    gates = W.random_layers(n, 4, seed=50 + n)
    want = oracle.run(n, gates, init=3)
    with SV(n, c, 1e-6, init_index=3, max_group_qubits=2 if n - c >= 2 else 0) as s:
        s.apply(gates)
        got = s.state()
        st = s.stats()
        s.apply([])
        assert np.array_equal(s.state(), got)
        assert s.stats()["passes"] == st["passes"]
    assert np.linalg.norm(got - want) <= compressed_l2_bound(n, 1e-6, st["passes"], len(gates))


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("name", ["layers", "clifford", "mixed"])
@pytest.mark.parametrize("n,c,g", [(16, 10, 2), (14, 8, 3)])
def test_remapped_passes_match_oracle(SV, dtype, name, n, c, g):
    """remap_qubits: physical SWAPs move qubits between chunk-index and
    in-chunk positions; the state, sampled amplitudes and an expectation read
    back in logical order match the oracle, with the pass count sv_plan_remap
    gives."""
    import paper_2309_16979_gb300 as P
    gates = _circuits(n)[name]
    init = W.basis_index(n, seed=7)
    want = oracle.run(n, gates, init=init)
    plan = P.plan(n, c, gates, max_group_qubits=g, remap=True)
    eb = 1e-6
    with SV(n, c, eb, dtype=dtype, init_index=init, max_group_qubits=g, remap_qubits=True) as s:
        s.apply(gates)
        got = s.state()
        st = s.stats()
        idx = np.array([0, 1, 5, (1 << n) - 1, 12345 % (1 << n)], dtype=np.uint64)
        amps = s.amplitudes(idx)
        terms = W.random_pauli_sum(n, 6, seed=11)
        e = s.expect(terms)
    assert st["passes"] == plan["passes"] and st["remap_swaps"] == len(plan["swaps"])
    bound = compressed_l2_bound(n, eb, st["passes"], len(gates) + st["remap_swaps"], dtype)
    assert np.linalg.norm(got - want) <= bound, (st["passes"], np.linalg.norm(got - want), bound)
    assert np.abs(amps - want[idx.astype(np.int64)]).max() <= bound
    assert abs(e - oracle.expect(n, want, terms)) <= 4 * bound * sum(abs(t.coeff) for t in terms)


def test_remapped_calls_accumulate_and_grad_resets(SV):
    """Two remapped calls in a row compose their moves; sv_grad afterwards
    starts again from the initial state on the original positions (g = 3:
    the Ising terms' 6 high x-masks and the identity fit a group of 8
    chunks)."""
    n, c, g = 16, 10, 3
    a, b = W.random_layers(n, 6, seed=4), W.random_mixed(n, 150, seed=6)
    want = oracle.run(n, a + b, init=3)
    gates, nparams = W.hea(n, 2)
    theta = np.array(W.normal_params(nparams, seed=3))
    H = W.ising(n, seed=4)
    e_want, g_want = oracle.adjoint(n, gates, theta, H, init=3)
    with SV(n, c, 1e-7, dtype="c128", init_index=3, max_group_qubits=g, remap_qubits=True) as s:
        s.apply(a)
        s.apply(b)
        got = s.state()
        st = s.stats()
        assert st["remap_swaps"] > 0
        bound = compressed_l2_bound(n, 1e-7, st["passes"], len(a) + len(b) + st["remap_swaps"], "c128")
        assert np.linalg.norm(got - want) <= bound
        e, gr = s.grad(gates, theta, H)
    csum = sum(abs(t.coeff) for t in H)
    assert abs(e - e_want) <= 1e-4 * csum
    assert np.abs(gr - g_want).max() <= 1e-4 * csum


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_expectation_tile_sets_and_remainder(SV, dtype):
    """Terms whose x bits above local bit 7 fit four tile positions are
    evaluated from shared-memory tiles, several tile sets per sweep; terms
    with five or more such bits by the strip kernel; one sum. n = 18, in HBM
    and as compressed groups of 2^15 amplitudes, against the oracle on the
    state the GPU holds."""
    n = 18
    gates = W.random_layers(n, 4, seed=12)
    rng = np.random.default_rng(13)
    terms = [W.PauliTerm(0.5 - 0.03 * q, 1 << q, int(rng.integers(0, 1 << n))) for q in range(n)]
    terms += [W.PauliTerm(0.2, (1 << 9) | (1 << 12) | (1 << 15) | 5, 1 << 16)]       # 3 high bits + low
    wide = 0
    for q in (8, 10, 11, 13, 14, 17):
        wide |= 1 << q
    terms += [W.PauliTerm(-0.35, wide, 3), W.PauliTerm(0.15, wide | 1, wide)]       # 6 high bits: remainder
    terms += W.ising(n, seed=6) + W.random_pauli_sum(n, 12, seed=14)
    tol = 1e-12 if dtype == "c128" else 2e-6
    for mode in ("uncompressed", "compressed"):
        with SV(n, 12, 1e-9 if dtype == "c128" else 1e-6, mode=mode, dtype=dtype, max_group_qubits=3) as s:
            s.apply(gates)
            got = s.expect(terms)
            held = s.state()
        assert abs(got - oracle.expect(n, held, terms)) <= tol * sum(abs(t.coeff) for t in terms), mode
