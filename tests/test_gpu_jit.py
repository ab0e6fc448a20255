"""Sub-pass kernels generated at run time (sv_config.jit) against the FP64
oracle and against the table-driven kernel, through the C ABI."""
import copy

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


@pytest.mark.parametrize("jit", [False, True])
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_generated_and_table_kernels_match_oracle(SV, jit, dtype):
    n = 15
    gates = W.random_mixed(n, 400, seed=21)
    want = oracle.run(n, gates, init=77)
    with SV(n, mode="uncompressed", dtype=dtype, init_index=77, jit=jit) as s:
        s.apply(gates)
        st = s.stats()
        got = s.state()
    assert rel_l2(got, want) <= (1e-12 if dtype == "c128" else fp32_tol(len(gates)))
    assert (st["jit_launches"] > 0) == jit


def _exchange_circuit(n, seed):
    """CNOTs between random qubits (controls often thread bits of a phase,
    targets register bits), each followed or not by gates on the target or
    the control, so that exchanges are both deferred to the stores and
    applied to the registers."""
    rng = W.SplitMix64(seed)
    g = [W.Gate("H", (q,)) for q in range(n)]
    for _ in range(120):
        c, t = rng.below(n), rng.below(n)
        if c == t:
            continue
        g.append(W.Gate("CNOT", (t,), (c,)))
        r = rng.below(4)
        if r == 0:
            g.append(W.Gate("RX", (t,), theta=0.1 + 0.01 * rng.below(50)))
        elif r == 1:
            g.append(W.Gate("RZ", (c,), theta=0.2 + 0.01 * rng.below(50)))
        elif r == 2:
            g.append(W.Gate("CZ", (t,), (rng.below(n) if rng.below(2) else c,)) if c != t else W.Gate("Z", (t,)))
    return [x for x in g if not (x.kind == "CZ" and x.targets[0] in x.controls)]


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_deferred_exchanges(SV, dtype):
    n = 14
    gates = _exchange_circuit(n, 41)
    want = oracle.run(n, gates, init=5)
    with SV(n, mode="uncompressed", dtype=dtype, init_index=5) as s:
        s.apply(gates)
        got = s.state()
    assert rel_l2(got, want) <= (1e-12 if dtype == "c128" else fp32_tol(len(gates)))


def test_compressed_generated_kernels_with_fused_codec(SV):
    n, c = 17, 10
    gates = _exchange_circuit(n, 43) + W.random_layers(n, 4, seed=44)
    want = oracle.run(n, gates, init=11)
    outs = []
    for jit in (True, False):
        with SV(n, c, 1e-6, init_index=11, max_group_qubits=3, jit=jit) as s:
            s.apply(gates)
            outs.append((s.state(), s.stats()))
    for got, st in outs:
        assert np.linalg.norm(got - want) <= compressed_l2_bound(n, 1e-6, st["passes"], len(gates), "c64")
    assert outs[0][1]["jit_launches"] > 0 and outs[1][1]["jit_launches"] == 0


def test_kernels_reused_when_only_angles_change(SV):
    """Kernels are keyed by structure: new angles that keep every rotation on
    the same side of the factoring threshold (away from pi) compile nothing."""
    n, c = 16, 10
    g1 = W.random_layers(n, 5, seed=31)
    rng = W.SplitMix64(77)
    for x in g1:
        if x.kind in ("RX", "RY", "RZ"):
            x.theta = 2.0 * rng.uniform() - 1.0
    g2 = copy.deepcopy(g1)
    for x in g2:
        if x.kind in ("RX", "RY", "RZ"):
            x.theta = 0.9 * x.theta + 0.05
    with SV(n, c, 1e-6, max_group_qubits=3, init_index=9) as s:
        s.apply(g1)
        k1 = s.stats()["jit_kernels_compiled"]
        s.apply(g2)
        st = s.stats()
        got = s.state()
    assert st["jit_kernels_compiled"] == k1
    want = oracle.run(n, g1 + g2, init=9)
    assert np.linalg.norm(got - want) <= compressed_l2_bound(n, 1e-6, st["passes"], len(g1) + len(g2), "c64")
