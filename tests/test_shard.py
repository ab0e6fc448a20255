"""Sharding the compressed store over ranks, on the CPU: the relabel plan
keeps owner qubits out of every pass's staged set, its chunk moves form a
permutation, and two gloo ranks exchange compressed chunk streams so that
each ends up holding exactly the streams of the relabelled state (checked
against the oracle codec) and the FP64 all-reduce of their norms equals the
whole state's."""
import os
import socket

import numpy as np
import pytest

import oracle
import workloads as W
from paper_2309_16979_gb300 import shard


def _staged_lists(n, c, g, gates):
    from paper_2309_16979_gb300 import plan
    p = plan(n, c, gates, max_group_qubits=g)
    return [[q for q in range(c, n) if (m >> q) & 1] for m in p["staged"]]


@pytest.mark.parametrize("r", [1, 2])
def test_plan_keeps_owner_qubits_unstaged(r):
    n, c, g = 20, 12, 3
    staged = _staged_lists(n, c, g, W.random_layers(n, 12))
    assert any(set(S) & set(shard.owner_qubits(n, r)) for S in staged)  # the device plan does stage them
    sp = shard.plan_shards(n, c, r, staged)
    owners = set(shard.owner_qubits(n, r))
    assert len(sp.staged) == len(staged) and sp.relabels
    for S in sp.staged:
        assert not owners & set(S)
    for rl in sp.relabels:
        assert rl.a in owners and rl.b not in owners and c <= rl.b < n
    # every relabel moves chunks as a permutation of the whole store, half of each rank's
    for rl in sp.relabels:
        dest = []
        for rank in range(1 << r):
            partner, moves = shard.relabel_moves(rank, n, c, r, rl.a, rl.b)
            assert len(moves) == len(shard.local_chunks(rank, n, c, r)) // 2
            for src, dst in moves:
                assert shard.owner_of(src, n, c, r) == rank and shard.owner_of(dst, n, c, r) == partner
                dest.append(dst)
        stay = [k for k in range(1 << (n - c)) if ((k >> (rl.a - c)) & 1) == ((k >> (rl.b - c)) & 1)]
        assert sorted(dest + stay) == list(range(1 << (n - c)))


def _swap_qubits(psi, n, a, b):
    idx = np.arange(1 << n)
    ba, bb = (idx >> a) & 1, (idx >> b) & 1
    j = idx ^ ((ba ^ bb) << a) ^ ((ba ^ bb) << b)
    return psi[j]


def _rank_main(rank, world, port, n, c, eb, a, b, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r = world.bit_length() - 1
        rng = np.random.default_rng(11)
        psi = (rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)).astype(np.complex64)
        psi /= np.linalg.norm(psi)
        cs = 1 << c
        store = {k: oracle.codec_encode(psi[k * cs:(k + 1) * cs], eb) for k in shard.local_chunks(rank, n, c, r)}
        new = shard.exchange(store, rank, n, c, r, a, b, dist)
        want = _swap_qubits(psi, n, a, b)
        ok = sorted(new) == shard.local_chunks(rank, n, c, r)
        part = 0.0
        for k, st in new.items():
            # a stream moves whole: the relabelled state's chunk k encodes to the same bytes
            ok = ok and st == oracle.codec_encode(want[k * cs:(k + 1) * cs], eb)
            x = oracle.codec_decode(st, c, np.complex64).astype(np.complex128)
            part += float(np.vdot(x, x).real)
        total = shard.allreduce_fp64([part], dist)[0]
        q.put((rank, ok, total))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_exchange_compressed_chunks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    n, c, eb = 12, 8, 1e-5
    a, b = n - 1, c + 1  # the owner qubit trades places with chunk qubit 1
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(rank, 2, port, n, c, eb, a, b, q)) for rank in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    rng = np.random.default_rng(11)
    psi = (rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)).astype(np.complex64)
    psi /= np.linalg.norm(psi)
    whole = 0.0
    for k in range(1 << (n - c)):
        x = oracle.codec_decode(oracle.codec_encode(psi[k << c:(k + 1) << c], eb), c, np.complex64)
        whole += float(np.vdot(x.astype(np.complex128), x.astype(np.complex128)).real)
    for rank, ok, total in res:
        assert ok, rank
        assert abs(total - whole) <= 1e-12 * whole
