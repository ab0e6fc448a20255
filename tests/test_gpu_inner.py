"""sv_inner: <a|b> in FP64 on the GPU against the same sum taken in NumPy
over the two states as read back (sv_amplitudes_range), for compressed and
uncompressed first states, both amplitude types, and qubit maps that differ
between the states (caller SWAPs, remapping passes)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mod():
    import paper_2309_16979_gb300 as m
    return m


def _check(a, b):
    want = np.vdot(a.state(), b.state())
    got = a.inner(b)
    scale = np.linalg.norm(a.state()) * np.linalg.norm(b.state())
    assert abs(got - want) <= 1e-12 * scale, (got, want)
    return got


@pytest.mark.parametrize("dtype_a", ["c64", "c128"])
@pytest.mark.parametrize("dtype_b", ["c64", "c128"])
def test_inner_compressed_vs_uncompressed(mod, dtype_a, dtype_b):
    n = 13
    x = W.basis_index(n)
    qft = W.qft(n)  # its SWAPs leave the qubit map permuted
    with mod.StateVector(n, 8, 1e-6 if dtype_a == "c64" else 1e-9, dtype=dtype_a, init_index=x,
                         max_group_qubits=3) as a, \
            mod.StateVector(n, mode="uncompressed", dtype=dtype_b, init_index=x) as b:
        a.apply(qft)
        b.apply(qft[: len(qft) // 2])
        b.apply(W.random_layers(n, 2, seed=9))
        _check(a, b)
        b2 = mod.StateVector(n, mode="uncompressed", dtype=dtype_b, init_index=x)
        b2.apply(qft)
        ov = _check(a, b2)
        assert abs(abs(ov) - 1.0) < 1e-3  # the same state up to quantisation
        b2.close()


def test_inner_remapped_and_self(mod):
    n = 14
    gates = W.random_clifford_rz(n, 12, 4, seed=3)
    with mod.StateVector(n, 8, 1e-7, dtype="c128", max_group_qubits=2, remap_qubits=True) as a, \
            mod.StateVector(n, mode="uncompressed", dtype="c128") as b, \
            mod.StateVector(n, mode="uncompressed", dtype="c64") as p:
        a.apply(gates)
        assert a.stats()["remap_swaps"] > 0
        b.apply(gates)
        p.apply(gates)
        _check(a, b)
        _check(p, b)
        nb = b.inner(b)
        assert abs(nb - 1.0) < 1e-12 and abs(nb.imag) < 1e-15
        assert abs(a.inner(b)) ** 2 / (a.stats()["norm2"] * nb.real) > 1 - 1e-6


def test_inner_rejects(mod):
    with mod.StateVector(10, 8, 1e-6) as a, mod.StateVector(10, 8, 1e-6) as c, \
            mod.StateVector(11, mode="uncompressed") as d:
        with pytest.raises(mod.SvError) as ei:
            a.inner(c)  # second state compressed
        assert ei.value.code == -1
        with pytest.raises(mod.SvError):
            a.inner(d)  # qubit counts differ
