"""Device memory and streams from torch: a handle created with torch's
caching allocator shows its device footprint in torch.cuda.memory_allocated()
and gives it back on destroy; calls order after the work queued on torch's
current stream; an uncompressed state is read by torch kernels in place
(sv_device_state) without an explicit synchronise."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mod():
    import paper_2309_16979_gb300 as m
    return m


def test_torch_allocator_holds_the_handle_memory(mod):
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    n = 24
    s = mod.StateVector(n, mode="uncompressed", dtype="c64", memory="torch")
    grown = torch.cuda.memory_allocated() - base
    assert grown >= 8 << n  # the whole state (complex64) comes from torch
    s.apply(W.random_layers(n, 2))
    s.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == base
    c = mod.StateVector(n, 18, 1e-6, max_group_qubits=3, memory="torch")
    assert torch.cuda.memory_allocated() - base >= (8 << 18) << 3  # a staged group of decoded chunks
    c.close()
    assert torch.cuda.memory_allocated() == base


def test_cuda_allocator_is_invisible_to_torch(mod):
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    with mod.StateVector(20, mode="uncompressed", memory="cuda"):
        assert torch.cuda.memory_allocated() == base


@pytest.mark.parametrize("mode", ["uncompressed", "compressed"])
def test_torch_memory_results_match_oracle(mod, mode):
    n = 13
    gates = W.qft(n)
    x = W.basis_index(n)
    with mod.StateVector(n, 8, 1e-9, dtype="c128", mode=mode, init_index=x, max_group_qubits=2,
                         memory="torch") as s:
        s.apply(gates)
        got = s.state()
        P = s.stats()["passes"]
    want = oracle.run(n, gates, init=x)
    bound = 1e-12 if mode == "uncompressed" else P * np.sqrt(2.0 * (1 << n)) * 1e-9 + 1e-12
    assert np.linalg.norm(got - want) <= bound


def test_device_state_consumed_by_torch_on_the_current_stream(mod):
    """The state a call leaves in HBM, read by torch kernels on the current
    stream right after the call; QFT's SWAPs leave a non-trivial qubit map."""
    n = 14
    gates = W.qft(n)
    x = W.basis_index(n)
    want = oracle.run(n, gates, init=x)
    with mod.StateVector(n, mode="uncompressed", dtype="c128", init_index=x, memory="torch") as s:
        # queue work on torch's stream before the call: the call must order after it
        junk = torch.randn(4096, 4096, device="cuda")
        for _ in range(8):
            junk = junk @ junk
            junk = junk / junk.norm()
        s.apply(gates)
        t, pos = s.device_tensor()
        assert sorted(pos) == list(range(n)) and pos != list(range(n))
        # logical index x -> physical index: a gather on the GPU
        idx = torch.arange(1 << n, device="cuda", dtype=torch.int64)
        phys = torch.zeros_like(idx)
        for q, p in enumerate(pos):
            phys |= ((idx >> q) & 1) << p
        logical = t[phys]
        ref = torch.from_numpy(want).to("cuda")
        err = torch.linalg.vector_norm(logical - ref).item()
    assert err <= 1e-12
