"""Seeded synthetic inputs shared by the oracle and the GPU path.

This module only *describes* inputs: gate lists (kind, qubits, angle,
parameter index), Pauli sums (coefficient, x-mask, z-mask) and basis-state
indices. It holds none of the simulation arithmetic: no gate matrix, no state
update, no codec. Each side (``oracle/`` and the CUDA library) turns these
descriptions into its own data structures and matrices.

Circuit families follow the workloads of the compressed state-vector method
(MEMQSim, Sec. 2 "Offline stage": a circuit partitioned into stages over a
chunked state): GHZ, QFT on a basis state, random layered circuits,
random Clifford+RZ circuits with a chosen share of gates on high qubits, and a
hardware-efficient ansatz with a 1-D Ising observable for gradients.

Random numbers come from splitmix64 (Steele, Lea & Flood, OOPSLA 2014),
implemented here from its published definition.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

MASK64 = (1 << 64) - 1

# Gate kinds understood by both sides. Matrices are defined separately by each.
KINDS = ("H", "X", "Y", "Z", "S", "SDG", "T", "TDG", "RX", "RY", "RZ", "P",
         "CNOT", "CZ", "CP", "SWAP", "CUSTOM")
# kinds that carry an angle
ANGLE_KINDS = ("RX", "RY", "RZ", "P", "CP")
# kinds whose angle may be a trainable parameter (U = exp(-i theta G / 2))
PARAM_KINDS = ("RX", "RY", "RZ")


class SplitMix64:
    """splitmix64: state += golden gamma; output = mix(state)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """U[0,1) with 53 random bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def below(self, m: int) -> int:
        """Integer in [0, m) (multiply-shift; bias < 2^-40 for m < 2^24)."""
        return int(self.uniform() * m)

    def normal(self) -> float:
        """Standard normal by Box-Muller (one of the pair)."""
        u1 = self.uniform()
        u2 = self.uniform()
        u1 = max(u1, 1e-300)
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


@dataclass
class Gate:
    """One gate. ``targets``/``controls`` are qubit numbers (qubit 0 = LSB of
    the amplitude index). For 2-target gates the matrix row/column index has
    bit b <-> targets[b]. ``mat`` (CUSTOM only) is the row-major 2^k x 2^k
    complex matrix as a flat list of complex numbers. ``param`` >= 0 marks a
    trainable angle (index into the parameter vector)."""
    kind: str
    targets: Tuple[int, ...]
    controls: Tuple[int, ...] = ()
    theta: float = 0.0
    param: int = -1
    mat: Optional[Tuple[complex, ...]] = None

    def qubits(self) -> Tuple[int, ...]:
        return tuple(self.targets) + tuple(self.controls)


@dataclass
class PauliTerm:
    """coeff * prod_q sigma(x_q, z_q); sigma(1,0)=X, (0,1)=Z, (1,1)=Y."""
    coeff: float
    xmask: int
    zmask: int


# --------------------------------------------------------------------------
# circuit families
# --------------------------------------------------------------------------

def basis_index(n: int, seed: int = 2) -> int:
    """Seeded basis-state index in [0, 2^n)."""
    return SplitMix64(seed).next_u64() % (1 << n)


def ghz(n: int) -> List[Gate]:
    """H on qubit 0, then a CNOT chain 0->1->...->n-1."""
    gates = [Gate("H", (0,))]
    for i in range(n - 1):
        gates.append(Gate("CNOT", (i + 1,), (i,)))
    return gates


def qft(n: int, swaps: bool = True) -> List[Gate]:
    """QFT|x> = 2^{-n/2} sum_k exp(2 pi i x k / 2^n) |k> with qubit 0 = LSB.

    Textbook circuit: for j from n-1 down to 0, H(j) then controlled phases
    CP(pi / 2^(j-m)) from every lower qubit m (control m, target j); the final
    SWAPs reverse the qubit order."""
    gates: List[Gate] = []
    for j in range(n - 1, -1, -1):
        gates.append(Gate("H", (j,)))
        for m in range(j - 1, -1, -1):
            gates.append(Gate("CP", (j,), (m,), theta=math.pi / (1 << (j - m))))
    if swaps:
        for i in range(n // 2):
            gates.append(Gate("SWAP", (i, n - 1 - i)))
    return gates


def random_layers(n: int, depth: int, seed: int = 1) -> List[Gate]:
    """Each layer: every qubit gets one gate drawn uniformly from
    {H, RX(theta), RZ(theta)} with theta ~ U[0, 2 pi); then a seeded random
    perfect matching of the qubits (Fisher-Yates shuffle, consecutive pairs,
    first of a pair = control) gets one CNOT per pair."""
    rng = SplitMix64(seed)
    gates: List[Gate] = []
    for _ in range(depth):
        for q in range(n):
            pick = rng.below(3)
            if pick == 0:
                gates.append(Gate("H", (q,)))
            else:
                th = 2.0 * math.pi * rng.uniform()
                gates.append(Gate("RX" if pick == 1 else "RZ", (q,), theta=th))
        perm = list(range(n))
        for i in range(n - 1, 0, -1):
            j = rng.below(i + 1)
            perm[i], perm[j] = perm[j], perm[i]
        for i in range(0, n - 1, 2):
            gates.append(Gate("CNOT", (perm[i + 1],), (perm[i],)))
    return gates


def random_clifford_rz(n: int, depth: int, n_high: int, p_high: float = 0.4,
                       seed: int = 1) -> List[Gate]:
    """Each layer has n gate slots. A slot's first qubit comes from the
    n_high top qubits with probability p_high, else from the others; its gate
    is H / S / RZ(theta) / CNOT with weights 0.3 / 0.2 / 0.2 / 0.3. A CNOT's
    second qubit (the target) is any other qubit."""
    rng = SplitMix64(seed)
    lo = n - n_high
    gates: List[Gate] = []
    for _ in range(depth):
        for _slot in range(n):
            if rng.uniform() < p_high:
                q = lo + rng.below(n_high)
            else:
                q = rng.below(lo)
            u = rng.uniform()
            if u < 0.3:
                gates.append(Gate("H", (q,)))
            elif u < 0.5:
                gates.append(Gate("S", (q,)))
            elif u < 0.7:
                gates.append(Gate("RZ", (q,), theta=2.0 * math.pi * rng.uniform()))
            else:
                t = rng.below(n - 1)
                if t >= q:
                    t += 1
                gates.append(Gate("CNOT", (t,), (q,)))
    return gates


def hea(n: int, layers: int) -> Tuple[List[Gate], int]:
    """Hardware-efficient ansatz: per layer RY(theta) then RZ(theta) on every
    qubit, then a CNOT ladder i -> i+1 (open). Parameters are numbered in gate
    order; returns (gates, n_params)."""
    gates: List[Gate] = []
    p = 0
    for _ in range(layers):
        for q in range(n):
            gates.append(Gate("RY", (q,), param=p)); p += 1
            gates.append(Gate("RZ", (q,), param=p)); p += 1
        for i in range(n - 1):
            gates.append(Gate("CNOT", (i + 1,), (i,)))
    return gates, p


def normal_params(count: int, sigma: float = 0.1, seed: int = 3) -> List[float]:
    """theta ~ N(0, sigma^2) (sigma = 0.1 reading of 'N(0, 0.1)')."""
    rng = SplitMix64(seed)
    return [sigma * rng.normal() for _ in range(count)]


def ising(n: int, seed: int = 4) -> List[PauliTerm]:
    """Open-chain 1-D Ising H = sum_i J_i Z_i Z_{i+1} + sum_i h_i X_i,
    J, h ~ U[-1, 1]."""
    rng = SplitMix64(seed)
    J = [2.0 * rng.uniform() - 1.0 for _ in range(n - 1)]
    h = [2.0 * rng.uniform() - 1.0 for _ in range(n)]
    terms = [PauliTerm(J[i], 0, (1 << i) | (1 << (i + 1))) for i in range(n - 1)]
    terms += [PauliTerm(h[i], 1 << i, 0) for i in range(n)]
    return terms


def random_pauli_sum(n: int, count: int, seed: int = 5) -> List[PauliTerm]:
    """Random Pauli strings with U[-1,1] coefficients (test input)."""
    rng = SplitMix64(seed)
    out = []
    for _ in range(count):
        x = rng.next_u64() & ((1 << n) - 1)
        z = rng.next_u64() & ((1 << n) - 1)
        out.append(PauliTerm(2.0 * rng.uniform() - 1.0, x, z))
    return out


def random_unitary_2x2(rng: SplitMix64) -> Tuple[complex, ...]:
    """A seeded unitary built from three angles: the matrix is written out
    here only as test input data for CUSTOM gates."""
    a = 2 * math.pi * rng.uniform(); b = 2 * math.pi * rng.uniform()
    c = 2 * math.pi * rng.uniform(); t = math.pi * rng.uniform()
    ct, st = math.cos(t / 2), math.sin(t / 2)
    e = lambda ang: complex(math.cos(ang), math.sin(ang))
    return (e(a) * ct, -e(a + c) * st, e(a + b) * st, e(a + b + c) * ct)


def random_unitary_4x4(rng: SplitMix64) -> Tuple[complex, ...]:
    """Seeded 4x4 unitary as test input: Gram-Schmidt on a random complex
    matrix (plain Python, no numpy)."""
    cols = []
    for _ in range(4):
        v = [complex(rng.normal(), rng.normal()) for _ in range(4)]
        for u in cols:
            d = sum(u[i].conjugate() * v[i] for i in range(4))
            v = [v[i] - d * u[i] for i in range(4)]
        nv = math.sqrt(sum(abs(x) ** 2 for x in v))
        cols.append([x / nv for x in v])
    # row-major: M[r][c] = cols[c][r]
    return tuple(cols[c][r] for r in range(4) for c in range(4))


def random_mixed(n: int, count: int, seed: int = 7, custom: bool = True) -> List[Gate]:
    """Every gate kind on seeded random qubits (test input for brute-force
    comparison)."""
    rng = SplitMix64(seed)
    one = ["H", "X", "Y", "Z", "S", "SDG", "T", "TDG", "RX", "RY", "RZ", "P"]
    two = ["CNOT", "CZ", "CP", "SWAP"]
    kinds = one + (two if n >= 2 else []) + (["CUSTOM"] if custom else [])
    gates: List[Gate] = []
    for _ in range(count):
        k = kinds[rng.below(len(kinds))]
        th = 2 * math.pi * rng.uniform() - math.pi
        q = rng.below(n)
        if k in one:
            ctrls: Tuple[int, ...] = ()
            if n >= 2 and rng.uniform() < 0.2:
                c = rng.below(n - 1)
                ctrls = (c + 1 if c >= q else c,)
            gates.append(Gate(k, (q,), ctrls, theta=th if k in ANGLE_KINDS else 0.0))
        elif k in ("CNOT", "CZ", "CP"):
            c = rng.below(n - 1)
            c = c + 1 if c >= q else c
            gates.append(Gate(k, (q,), (c,), theta=th if k == "CP" else 0.0))
        elif k == "SWAP":
            r = rng.below(n - 1)
            r = r + 1 if r >= q else r
            gates.append(Gate("SWAP", (q, r)))
        else:
            if n >= 2 and rng.uniform() < 0.5:
                r = rng.below(n - 1)
                r = r + 1 if r >= q else r
                gates.append(Gate("CUSTOM", (q, r), mat=random_unitary_4x4(rng)))
            else:
                gates.append(Gate("CUSTOM", (q,), mat=random_unitary_2x2(rng)))
    return gates


def inverse(gates: Sequence[Gate]) -> List[Gate]:
    """The inverse circuit: gates in reverse order, each replaced by its
    inverse (self-inverse kinds unchanged, S<->SDG, T<->TDG, angles negated,
    CUSTOM conjugate-transposed)."""
    swap = {"S": "SDG", "SDG": "S", "T": "TDG", "TDG": "T"}
    out: List[Gate] = []
    for g in reversed(gates):
        if g.kind in swap:
            out.append(Gate(swap[g.kind], g.targets, g.controls))
        elif g.kind in ANGLE_KINDS:
            out.append(Gate(g.kind, g.targets, g.controls, theta=-g.theta, param=-1))
        elif g.kind == "CUSTOM":
            k = 1 << len(g.targets)
            m = g.mat
            mt = tuple(m[c * k + r].conjugate() for r in range(k) for c in range(k))
            out.append(Gate("CUSTOM", g.targets, g.controls, mat=mt))
        else:
            out.append(Gate(g.kind, g.targets, g.controls))
    return out


def amp_gate_updates(n: int, gates: Sequence[Gate]) -> int:
    """Work unit of the throughput metric: every gate touches all 2^n
    amplitudes (SWAPs included)."""
    return len(gates) * (1 << n)
