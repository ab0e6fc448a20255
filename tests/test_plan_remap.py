"""Host-side qubit remapping (sv_plan_remap, no GPU). The library reports
the physical circuit its remapped passes run: for every caller gate, in
execution order, the positions it runs on, the SWAPs it adds, and the final
position of every qubit. The tests rebuild that circuit and run it through the
FP64 oracle against the logical circuit, the result read back through the
reported final positions; they also replay the positions from the SWAPs
alone, check that every pass's mixing high positions (the SWAPs' included)
are staged, that the remapped plan never has more passes than the plain one,
and that circuits whose high qubits are mixed often need fewer passes."""
import numpy as np
import pytest

import oracle
import workloads as W

DIAG = {"Z", "S", "SDG", "T", "TDG", "RZ", "P", "CZ", "CP"}


@pytest.fixture(scope="module")
def sv():
    from paper_2309_16979_gb300 import build
    build.build()
    import paper_2309_16979_gb300 as sv
    return sv


def physical_circuit(gates, plan):
    """The gate list the remapped passes run, on the library's positions,
    each with its pass."""
    out = []
    swaps = list(plan["swaps"])
    si = 0
    for k, (gi, p) in enumerate(zip(plan["order"], plan["pass_of"])):
        while si < len(swaps) and swaps[si][0] < p:
            out.append((W.Gate("SWAP", swaps[si][1:]), swaps[si][0]))
            si += 1
        g = gates[gi]
        q = plan["qubits"][k]
        out.append((W.Gate(g.kind, tuple(q[:len(g.targets)]), tuple(q[2:2 + len(g.controls)]), theta=g.theta,
                           param=g.param, mat=g.mat), p))
    out += [(W.Gate("SWAP", s[1:]), s[0]) for s in swaps[si:]]
    return out


def replay_positions(gates, plan, n):
    """Positions of every gate and the final map, recomputed from the SWAPs."""
    pos = list(range(n))
    swaps = list(plan["swaps"])
    si = 0
    qubits = []
    for gi, p in zip(plan["order"], plan["pass_of"]):
        while si < len(swaps) and swaps[si][0] < p:
            _, lo, hi = swaps[si]
            a, b = pos.index(lo), pos.index(hi)
            pos[a], pos[b] = hi, lo
            si += 1
        g = gates[gi]
        t = [pos[q] for q in g.targets] + [-1] * (2 - len(g.targets))
        c = [pos[q] for q in g.controls] + [-1] * (2 - len(g.controls))
        qubits.append(tuple(t + c))
    for _, lo, hi in swaps[si:]:
        a, b = pos.index(lo), pos.index(hi)
        pos[a], pos[b] = hi, lo
    return qubits, pos


def to_physical(psi, pos, n):
    idx = np.arange(1 << n, dtype=np.int64)
    phys = np.zeros_like(idx)
    for q in range(n):
        phys |= ((idx >> q) & 1) << pos[q]
    out = np.empty_like(psi)
    out[phys] = psi
    return out


@pytest.mark.parametrize("family", ["layers", "clifford", "mixed", "hea"])
@pytest.mark.parametrize("n,c,gmax", [(10, 6, 2), (12, 7, 3), (11, 5, 2), (12, 8, 4)])
def test_remapped_plan_runs_the_circuit(sv, family, n, c, gmax):
    gates = {
        "layers": W.random_layers(n, 8, seed=3),
        "clifford": W.random_clifford_rz(n, 10, n - c, seed=3),
        "mixed": [g for g in W.random_mixed(n, 200, seed=3) if g.kind != "SWAP"],
        "hea": W.hea(n, 4)[0],
    }[family]
    plain = sv.plan(n, c, gates, max_group_qubits=gmax)
    p = sv.plan(n, c, gates, max_group_qubits=gmax, remap=True)
    assert sorted(p["order"]) == list(range(len(gates)))
    assert p["pass_of"] == sorted(p["pass_of"])
    assert p["passes"] <= plain["passes"]
    if not p["swaps"]:
        assert p["order"] == plain["order"] and p["staged"] == plain["staged"]
    qubits, pos = replay_positions(gates, p, n)
    assert qubits == p["qubits"] and pos == p["positions"]
    assert sorted(pos) == list(range(n))
    phys = physical_circuit(gates, p)
    for g, pi in phys:
        high_mix = {q for q in g.targets if q >= c} if g.kind not in DIAG else set()
        assert all((p["staged"][pi] >> q) & 1 for q in high_mix), (g, pi)
    for _, lo, hi in p["swaps"]:
        assert lo < c <= hi
    rng = np.random.default_rng(5)
    psi0 = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    want = to_physical(oracle.apply_gates(n, psi0, gates), p["positions"], n)
    got = oracle.apply_gates(n, psi0, [g for g, _ in phys])
    assert np.abs(got - want).max() < 1e-11


def test_remap_keeps_plans_that_do_not_gain(sv):
    """GHZ and QFT stage each high qubit about once: nothing to gain, and the
    plain plan is kept."""
    for n, c, gates in ((30, 22, W.ghz(30)), (36, 26, W.qft(36, swaps=False))):
        a = sv.plan(n, c, gates, max_group_qubits=6)
        b = sv.plan(n, c, gates, max_group_qubits=6, remap=True)
        assert b["swaps"] == [] and b["passes"] == a["passes"] and b["order"] == a["order"]


@pytest.mark.parametrize("name,n,c,gmax,most", [
    ("clifford", 36, 26, 6, 4),   # plain: 8 passes
    ("clifford", 30, 22, 4, 5),   # plain: 11
    ("hea", 32, 24, 6, 2),        # plain: 4
    ("layers", 30, 22, 6, 7),     # plain: 10
])
def test_remap_cuts_passes_of_high_heavy_circuits(sv, name, n, c, gmax, most):
    gates = {"clifford": lambda: W.random_clifford_rz(n, 30, n - c, seed=1),
             "hea": lambda: W.hea(n, 8)[0],
             "layers": lambda: W.random_layers(n, 40, seed=1)}[name]()
    a = sv.plan(n, c, gates, max_group_qubits=gmax)
    b = sv.plan(n, c, gates, max_group_qubits=gmax, remap=True)
    assert b["passes"] <= most < a["passes"], (a["passes"], b["passes"])


@pytest.mark.parametrize("n,c,gmax", [(11, 5, 2), (12, 7, 3)])
def test_remapped_plan_with_caller_swaps(sv, n, c, gmax):
    """Caller SWAPs relabel qubits before the remapping moves them: the
    physical circuit the library reports (its own positions for every gate)
    still equals the logical circuit read back through the final map."""
    gates = W.random_mixed(n, 200, seed=13)
    assert any(g.kind == "SWAP" for g in gates)
    p = sv.plan(n, c, gates, max_group_qubits=gmax, remap=True)
    assert p["swaps"]
    assert sorted(p["order"]) == [i for i, g in enumerate(gates) if g.kind != "SWAP"]
    assert sorted(p["positions"]) == list(range(n))
    phys = physical_circuit(gates, p)
    rng = np.random.default_rng(6)
    psi0 = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    want = to_physical(oracle.apply_gates(n, psi0, gates), p["positions"], n)
    got = oracle.apply_gates(n, psi0, [g for g, _ in phys])
    assert np.abs(got - want).max() < 1e-11


def test_remap_plan_degenerate_inputs(sv):
    """No gates, SWAPs only, all high qubits stageable at once (one pass:
    nothing to remap), and invalid sizes."""
    from paper_2309_16979_gb300 import SvError
    for gates in ([], [W.Gate("SWAP", (0, 9)), W.Gate("SWAP", (3, 11))]):
        p = sv.plan(12, 8, gates, max_group_qubits=2, remap=True)
        assert p["passes"] == 0 and p["order"] == [] and p["swaps"] == []
    swapped = sv.plan(12, 8, [W.Gate("SWAP", (0, 9)), W.Gate("SWAP", (3, 11))], max_group_qubits=2, remap=True)
    pos = list(range(12))
    pos[0], pos[9] = 9, 0
    pos[3], pos[11] = 11, 3
    assert swapped["positions"] == pos
    gates = W.random_layers(12, 6, seed=7)
    p = sv.plan(12, 8, gates, max_group_qubits=4, remap=True)
    assert p["passes"] == 1 and p["swaps"] == []
    with pytest.raises(SvError):
        sv.plan(12, 8, gates, max_group_qubits=1, remap=True)
    with pytest.raises(SvError):
        sv.plan(12, 13, gates, max_group_qubits=2, remap=True)
