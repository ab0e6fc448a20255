"""Independent dense-matrix construction of gates and Pauli strings for
pinning the oracle (test helper; numpy/scipy only).

Gate matrices come from their generators via the matrix exponential and
full operators from Kronecker products of 2x2 factors, so none of this
shares the oracle's index loops or closed-form matrix entries."""
import numpy as np
from scipy.linalg import expm

I2 = np.eye(2, dtype=complex)
X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
Z = np.array([[1, 0], [0, -1]], dtype=complex)
P0 = np.array([[1, 0], [0, 0]], dtype=complex)
P1 = np.array([[0, 0], [0, 1]], dtype=complex)


def E(r, c):
    m = np.zeros((2, 2), dtype=complex)
    m[r, c] = 1
    return m


def op_on(n, ops):
    """Kronecker product with ops[q] on qubit q (qubit 0 = rightmost factor)."""
    m = np.array([[1.0 + 0j]])
    for q in range(n - 1, -1, -1):
        m = np.kron(m, ops.get(q, I2))
    return m


def single_matrix(kind, theta):
    if kind == "H":
        return (X + Z) / np.sqrt(2)
    if kind in ("X", "CNOT"):
        return X
    if kind == "Y":
        return Y
    if kind in ("Z", "CZ"):
        return Z
    proj1 = (I2 - Z) / 2
    if kind == "S":
        return expm(1j * (np.pi / 2) * proj1)
    if kind == "SDG":
        return expm(-1j * (np.pi / 2) * proj1)
    if kind == "T":
        return expm(1j * (np.pi / 4) * proj1)
    if kind == "TDG":
        return expm(-1j * (np.pi / 4) * proj1)
    if kind == "RX":
        return expm(-0.5j * theta * X)
    if kind == "RY":
        return expm(-0.5j * theta * Y)
    if kind == "RZ":
        return expm(-0.5j * theta * Z)
    if kind in ("P", "CP"):
        return expm(1j * theta * proj1)
    raise ValueError(kind)


def gate_unitary(n, g, theta=None):
    th = g.theta if (theta is None or g.param < 0) else theta[g.param]
    dim = 1 << n
    if g.kind == "SWAP":
        a, b = g.targets
        full = 0.5 * (op_on(n, {}) + op_on(n, {a: X, b: X}) + op_on(n, {a: Y, b: Y})
                      + op_on(n, {a: Z, b: Z}))
    elif g.kind == "CUSTOM" and len(g.targets) == 2:
        M = np.array(g.mat, dtype=complex).reshape(4, 4)
        t0, t1 = g.targets
        full = np.zeros((dim, dim), dtype=complex)
        for r in range(4):
            for c in range(4):
                if M[r, c] != 0:
                    full += M[r, c] * op_on(n, {t0: E(r & 1, c & 1), t1: E(r >> 1, c >> 1)})
    elif g.kind == "CUSTOM":
        full = op_on(n, {g.targets[0]: np.array(g.mat, dtype=complex).reshape(2, 2)})
    else:
        full = op_on(n, {g.targets[0]: single_matrix(g.kind, th)})
    if g.controls:
        proj = op_on(n, {c: P1 for c in g.controls})
        full = np.eye(dim) - proj + proj @ full
    return full


def circuit_unitary(n, gates, theta=None):
    U = np.eye(1 << n, dtype=complex)
    for g in gates:
        U = gate_unitary(n, g, theta) @ U
    return U


def pauli_matrix(n, t):
    ops = {}
    for q in range(n):
        x, z = (t.xmask >> q) & 1, (t.zmask >> q) & 1
        if x and z:
            ops[q] = Y
        elif x:
            ops[q] = X
        elif z:
            ops[q] = Z
    return t.coeff * op_on(n, ops)


def hamiltonian_matrix(n, terms):
    return sum(pauli_matrix(n, t) for t in terms)
