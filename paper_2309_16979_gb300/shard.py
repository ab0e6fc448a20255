"""Sharding the compressed chunk store over 2^r ranks (host side).

The chunk groups of a pass are independent (Sec. 2, "Online stage": each
stage streams every chunk once), so the store splits over ranks by the top
r high qubits: rank rho owns the chunks whose physical qubits n-r .. n-1
(the owner qubits) spell rho. A pass whose staged set holds no owner qubit
runs on every rank over its own chunks with no exchange. Before a pass
that stages an owner qubit, that qubit trades places with a high qubit the
pass neither stages nor owns (a relabel, as the library's SWAP absorption
and qubit remapping do): chunks whose two bits differ move to the partner
rank that differs in the owner bit, as compressed streams, half of every
rank's chunks per relabelled qubit. Norms, expectation values and gradient
sums are per-rank partial sums reduced in FP64.

This module holds the plan and the host exchange (torch.distributed with
any backend: gloo on CPU, NCCL between GPUs); it moves bytes only and
computes nothing of the method.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Sequence, Tuple


def owner_qubits(n: int, r: int) -> List[int]:
    """Physical qubits whose bits name the owning rank (rank bit i = qubit n - r + i)."""
    return list(range(n - r, n))


def owner_of(k: int, n: int, c: int, r: int) -> int:
    """Rank owning physical chunk k (chunk bit j = physical qubit c + j)."""
    return k >> (n - c - r)


def local_chunks(rank: int, n: int, c: int, r: int) -> List[int]:
    """Physical chunk indices rank owns, ascending."""
    per = 1 << (n - c - r)
    return list(range(rank * per, (rank + 1) * per))


@dataclass
class Relabel:
    """Exchange physical qubits a (an owner qubit) and b (a high qubit that
    is neither staged nor an owner qubit) before pass `before_pass`."""
    before_pass: int
    a: int
    b: int


@dataclass
class ShardPlan:
    n: int
    c: int
    r: int
    relabels: List[Relabel] = field(default_factory=list)
    # staged physical qubits of every pass after the relabels before it
    staged: List[List[int]] = field(default_factory=list)


def plan_shards(n: int, c: int, r: int, staged_per_pass: Sequence[Sequence[int]]) -> ShardPlan:
    """Relabels that keep every pass's staged set off the owner qubits.

    staged_per_pass: the staged physical high qubits of each pass as planned
    for one device (e.g. from sv_plan's staged masks). Qubits are tracked
    through the relabels: a logical position that a relabel moved onto a
    low-owner slot is staged at its new place. The free qubit for a relabel
    is the high, non-owner qubit staged furthest in the future (or never)."""
    if r < 0 or n - c < r:
        raise ValueError("need 0 <= r <= n - c")
    owners = set(owner_qubits(n, r))
    where = list(range(n))  # where[q] = current physical position of planned qubit q
    plan = ShardPlan(n, c, r)
    for p, S in enumerate(staged_per_pass):
        phys = [where[q] for q in S]
        for q in S:
            if where[q] not in owners:
                continue
            staged_now = {where[x] for x in S}

            def next_use(pos):
                for pp in range(p + 1, len(staged_per_pass)):
                    if pos in {where[x] for x in staged_per_pass[pp]}:
                        return pp
                return len(staged_per_pass) + 1

            free = [b for b in range(c, n) if b not in owners and b not in staged_now]
            if not free:
                raise ValueError(f"pass {p}: no free high qubit to relabel an owner qubit with")
            b = max(free, key=next_use)
            a = where[q]
            plan.relabels.append(Relabel(p, a, b))
            qb = where.index(b)
            where[q], where[qb] = b, a
        phys = [where[q] for q in S]
        assert not owners & set(phys)
        plan.staged.append(sorted(phys))
    return plan


def relabel_moves(rank: int, n: int, c: int, r: int, a: int, b: int) -> Tuple[int, List[Tuple[int, int]]]:
    """The chunks rank sends for the relabel of owner qubit a with high qubit
    b: (partner rank, [(chunk index before, chunk index after)]). A chunk
    whose bits a and b differ takes the other value of both (the qubits
    trade places), which flips its owner bit, so it goes to the partner;
    the partner's chunks of the opposite pattern come back in its place."""
    ja, jb = a - c, b - c
    partner = rank ^ (1 << (a - (n - r)))
    out = []
    for k in local_chunks(rank, n, c, r):
        if ((k >> ja) & 1) != ((k >> jb) & 1):
            out.append((k, k ^ (1 << ja) ^ (1 << jb)))
    return partner, out


def exchange(store: Dict[int, bytes], rank: int, n: int, c: int, r: int, a: int, b: int, dist) -> Dict[int, bytes]:
    """Apply one relabel to this rank's share of the store: send the moving
    chunk streams to the partner and receive its moving ones (lengths
    first, then the bytes), with torch.distributed point-to-point calls.
    Returns the rank's new store (chunk index -> compressed stream)."""
    import torch
    partner, moves = relabel_moves(rank, n, c, r, a, b)
    _, back = relabel_moves(partner, n, c, r, a, b)
    send_lens = torch.tensor([len(store[k]) for k, _ in moves], dtype=torch.int64)
    recv_lens = torch.empty(len(back), dtype=torch.int64)
    payload = torch.frombuffer(bytearray(b"".join(store[k] for k, _ in moves)) or bytearray(1), dtype=torch.uint8)
    # lower rank sends first: no deadlock with blocking calls
    if rank < partner:
        dist.send(send_lens, partner)
        dist.recv(recv_lens, partner)
    else:
        dist.recv(recv_lens, partner)
        dist.send(send_lens, partner)
    total = int(recv_lens.sum().item())
    incoming = torch.empty(max(1, total), dtype=torch.uint8)
    if rank < partner:
        dist.send(payload, partner)
        dist.recv(incoming, partner)
    else:
        dist.recv(incoming, partner)
        dist.send(payload, partner)
    out = dict(store)
    for k, _ in moves:
        del out[k]
    raw = incoming.numpy().tobytes()
    off = 0
    for (k_src, k_dst), ln in zip(back, recv_lens.tolist()):
        out[k_dst] = raw[off:off + ln]
        off += ln
    return out


def allreduce_fp64(values: Sequence[float], dist) -> List[float]:
    """Sum per-rank FP64 partial sums (norm^2, <H>, gradient entries) over ranks."""
    import torch
    t = torch.tensor(list(values), dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.tolist()
