"""Failure paths made on the host, with no GPU fault: a pinned-memory budget
too small for the compressed store (SV_ERR_HOST_OOM), and a host wait
deadline shorter than the GPU work (SV_ERR_TIMEOUT: the host gives up while
the kernels finish on their own). After either, the handle can still be
destroyed and a fresh handle runs a circuit correctly."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

SV_ERR_HOST_OOM = -2
SV_ERR_TIMEOUT = -5


@pytest.fixture(scope="module")
def mod():
    import paper_2309_16979_gb300 as m
    return m


def _fresh_handle_works(mod):
    n, c = 12, 8
    gates = W.qft(n)
    x = W.basis_index(n)
    with mod.StateVector(n, c, 1e-7, dtype="c128", init_index=x, max_group_qubits=2) as s:
        s.apply(gates)
        got = s.state()
        P = s.stats()["passes"]
    want = oracle.run(n, gates, init=x)
    assert np.linalg.norm(got - want) <= P * np.sqrt(2.0 * (1 << n)) * 1e-7 + 1e-12


def test_host_budget_too_small_for_the_store(mod):
    # a basis state needs two slots (the shared all-zero chunk stream and the
    # basis amplitude's chunk), a few hundred bytes: 64 bytes cannot hold it
    with pytest.raises(mod.SvError) as ei:
        mod.StateVector(16, 10, 1e-6, host_budget_bytes=64)
    assert ei.value.code == SV_ERR_HOST_OOM
    _fresh_handle_works(mod)


def test_host_wait_deadline_then_destroy_and_recover(mod):
    """A deadline of one microsecond on a circuit that keeps the GPU busy for
    tens of milliseconds: some host wait (at creation or during the passes)
    gives up with SV_ERR_TIMEOUT; destroying the handle waits for the GPU
    work it issued, and a new handle computes correctly."""
    n, c = 24, 18
    gates = W.random_layers(n, 12)
    code = None
    try:
        s = mod.StateVector(n, c, 1e-6, max_group_qubits=3, timeout_s=1e-6)
    except mod.SvError as e:
        code = e.code
    else:
        try:
            s.apply(gates)
        except mod.SvError as e:
            code = e.code
        s.close()
    assert code == SV_ERR_TIMEOUT
    _fresh_handle_works(mod)


def test_store_holds_one_copy_of_the_state(mod):
    """The pinned store keeps one slot per chunk, rewritten in place: after a
    circuit that spreads the state, pinned memory is about the compressed
    size (1/32 headroom per slot, released slots, segment granularity), and a
    budget of 1.3x that runs the same circuit to the same state. A budget
    below the compressed size fails in the pass that outgrows it, with
    SV_ERR_HOST_OOM."""
    n, c, eb = 20, 12, 1e-6
    gates = W.random_layers(n, 6)
    kw = dict(max_group_qubits=3, init_index=5)
    with mod.StateVector(n, c, eb, **kw) as s:
        s.apply(gates)
        st = s.stats()
        ref = s.state()
    comp, pinned = st["compressed_bytes"], st["host_pinned_bytes"]
    seg = max(4 * mod.codec_max_bytes(c), (8 << n) // 8)
    assert comp > 4096 * (1 << (n - c))  # the state has spread (a basis state: ~340 bytes per chunk)
    assert pinned <= 1.3 * comp + 2 * seg
    budget = int(1.3 * comp) + 2 * seg
    with mod.StateVector(n, c, eb, host_budget_bytes=budget, **kw) as s:
        s.apply(gates)
        assert s.stats()["host_pinned_bytes"] <= budget
        assert np.array_equal(s.state(), ref)
    with mod.StateVector(n, c, eb, host_budget_bytes=comp // 3, **kw) as s:
        with pytest.raises(mod.SvError) as ei:
            s.apply(gates)
        assert ei.value.code == SV_ERR_HOST_OOM
    _fresh_handle_works(mod)
