"""Host-side pass planning (sv_plan, no GPU): the execution order is a valid
reordering of the circuit (checked by running both orders through the FP64
oracle), every pass's mixing high qubits are staged, and pass counts of
circuits with a known structure."""
import numpy as np
import pytest

import oracle
import workloads as W


@pytest.fixture(scope="module")
def sv():
    from paper_2309_16979_gb300 import build
    build.build()
    import paper_2309_16979_gb300 as sv
    return sv


DIAG = {"Z", "S", "SDG", "T", "TDG", "RZ", "P", "CZ", "CP"}


def _mixing(g):
    if g.kind in DIAG:
        return set()
    return set(g.targets)


@pytest.mark.parametrize("family", ["layers", "clifford", "mixed", "qft_noswap", "ghz"])
@pytest.mark.parametrize("n,c,gmax", [(10, 6, 2), (12, 8, 3), (11, 9, 2)])
def test_plan_is_valid_reordering(sv, family, n, c, gmax):
    gates = {
        "layers": W.random_layers(n, 6, seed=2),
        "clifford": W.random_clifford_rz(n, 6, 3, seed=2),
        "mixed": [g for g in W.random_mixed(n, 150, seed=2) if g.kind != "SWAP"],
        "qft_noswap": W.qft(n, swaps=False),
        "ghz": W.ghz(n),
    }[family]
    p = sv.plan(n, c, gates, max_group_qubits=gmax)
    assert sorted(p["order"]) == list(range(len(gates)))
    assert p["pass_of"] == sorted(p["pass_of"])
    nh = n - c
    for k, gi in enumerate(p["order"]):
        high_mix = {q for q in _mixing(gates[gi]) if q >= c}
        staged = p["staged"][p["pass_of"][k]]
        assert all((staged >> q) & 1 for q in high_mix)
    for m in p["staged"]:
        assert bin(m).count("1") == min(gmax, nh)
        assert m & ((1 << c) - 1) == 0
    rng = np.random.default_rng(1)
    psi0 = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    a = oracle.apply_gates(n, psi0, gates)
    b = oracle.apply_gates(n, psi0, [gates[i] for i in p["order"]])
    assert np.abs(a - b).max() < 1e-12


@pytest.mark.parametrize("n,c,gmax", [(30, 22, 4), (36, 26, 4), (36, 26, 5), (16, 10, 2), (12, 12, 4)])
def test_ghz_pass_count(sv, n, c, gmax):
    p = sv.plan(n, c, W.ghz(n), max_group_qubits=gmax)
    want = max(1, -(-(n - c) // gmax))
    assert p["passes"] == want


def test_diagonal_gates_never_force_a_pass(sv):
    n, c = 20, 10
    gates = [W.Gate("H", (q,)) for q in range(c)]
    gates += [W.Gate("RZ", (q,), theta=0.1 * q) for q in range(n)]
    gates += [W.Gate("CZ", (q,), (q + 1,)) for q in range(n - 1)]
    gates += [W.Gate("CNOT", (q - 10,), (q,)) for q in range(c, n)]  # high controls, low targets
    p = sv.plan(n, c, gates, max_group_qubits=2)
    assert p["passes"] == 1


def test_swaps_relabel_without_passes(sv):
    n, c = 14, 8
    gates = [W.Gate("SWAP", (0, 13)), W.Gate("H", (0,))]   # logical 0 now lives on physical 13
    p = sv.plan(n, c, gates, max_group_qubits=2)
    assert p["order"] == [1] and p["passes"] == 1
    assert (p["staged"][0] >> 13) & 1


def test_invalid_gates_rejected(sv):
    with pytest.raises(sv.SvError):
        sv.plan(8, 8, [W.Gate("H", (8,))])
    with pytest.raises(sv.SvError):
        sv.plan(8, 8, [W.Gate("CNOT", (1,), (1,))])
    with pytest.raises(sv.SvError):
        sv.plan(8, 8, [W.Gate("H", (1,))], max_group_qubits=1)


def test_subpass_counts_small_tiles_terminate(sv):
    n = 16
    gates = W.random_mixed(n, 200, seed=4)
    gates = [g for g in gates if g.kind != "SWAP"]
    for tile in (2, 3, 5, 8, 13):
        p = sv.plan(n, 10, gates, max_group_qubits=3, tile_qubits=tile)
        assert p["subpasses"] >= p["passes"] >= 1


def test_plan_cache_replays_the_fresh_plan():
    """Sub-pass plans are cached by the ops' structure and replayed with the
    current matrices: the kernels generated for a circuit seen before (and
    for the same circuit with new angles) equal those of a fresh process."""
    import os
    import subprocess
    import sys
    from paper_2309_16979_gb300 import jit_sources
    ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    n, c = 20, 14
    g1 = W.random_layers(n, 12, seed=5)
    g2 = [W.Gate(x.kind, x.targets, x.controls, theta=x.theta * 0.731 + 0.2) if x.kind in W.ANGLE_KINDS else x
          for x in g1]
    code = ("import sys, json; sys.path.insert(0, %r); import workloads as W; "
            "from paper_2309_16979_gb300 import jit_sources; "
            "g = W.random_layers(%d, 12, seed=5); "
            "g = [W.Gate(x.kind, x.targets, x.controls, theta=x.theta * 0.731 + 0.2) if x.kind in W.ANGLE_KINDS else x "
            "for x in g]; print(json.dumps(jit_sources(%d, %d, g, max_group_qubits=3)))") % (ROOT, n, n, c)
    fresh = subprocess.run([sys.executable, "-c", code], check=True, capture_output=True, text=True).stdout
    import json
    jit_sources(n, c, g1, max_group_qubits=3)  # fills the cache with g1's structure
    cached = jit_sources(n, c, g2, max_group_qubits=3)
    assert cached == json.loads(fresh)
    for adjoint in (False, True):
        a = jit_sources(n, c, g1, max_group_qubits=3, adjoint=adjoint)
        b = jit_sources(n, c, g1, max_group_qubits=3, adjoint=adjoint)
        assert a == b


def test_commuting_gates_run_ahead_of_deferred_ones(sv):
    """A gate may run in an earlier pass than a deferred gate it shares
    qubits with when, on every shared qubit, both commute with Z (controls,
    diagonal gates) or both with X (CNOT's target, RX); a gate that breaks
    both families waits. Here g = 2 stages qubits 10 and 13 first (the
    gates on them outnumber the rest), so H(11), the CNOT it blocks and the
    CNOT onto 12 wait for a later pass."""
    n, c = 16, 10
    gates = [W.Gate("H", (q,)) for q in (10, 13, 10, 13, 10, 13, 10, 13)]
    gates += [W.Gate("H", (11,)), W.Gate("CNOT", (5,), (11,)),
              W.Gate("RX", (5,), theta=0.3),   # 10: X family on 5, like the CNOT's target: runs ahead
              W.Gate("RZ", (5,), theta=0.7),   # 11: Z family against the target's X: waits
              W.Gate("CNOT", (12,), (4,)),     # 12: mixes 12, deferred in pass 0
              W.Gate("RZ", (4,), theta=0.2),   # 13: Z family, like the CNOT's control: runs ahead
              W.Gate("H", (4,))]               # 14: neither: waits
    p = sv.plan(n, c, gates, max_group_qubits=2)
    assert p["staged"][0] == (1 << 10) | (1 << 13)
    pass_of = dict(zip(p["order"], p["pass_of"]))
    assert {k for k, v in pass_of.items() if v == 0} == set(range(8)) | {10, 13}
    assert pass_of[11] >= pass_of[9] >= pass_of[8] > 0 and pass_of[14] >= pass_of[12] > 0
    rng = np.random.default_rng(3)
    psi0 = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    a = oracle.apply_gates(n, psi0, gates)
    b = oracle.apply_gates(n, psi0, [gates[i] for i in p["order"]])
    assert np.abs(a - b).max() < 1e-12
