"""Helpers shared by the GPU parity tests."""
import numpy as np

U32 = 2.0 ** -24


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def fp32_tol(ngates):
    """Bound on the relative L2 error of complex64 gate arithmetic: each gate
    rounds every output (a 2x2 complex product, a few roundings of 2^-24) and a
    unitary carries earlier errors unchanged in norm, so errors add at most
    linearly in the number of gates; the gate matrices themselves are rounded
    to FP32 once."""
    return 16 * U32 * max(1, ngates) + 1e-6


def compressed_l2_bound(n, eb, passes, ngates, dtype="c64"):
    """||psi_gpu - psi_exact||_2 bound for the compressed path: every pass
    ends with a re-quantisation that moves each stored real number by at most
    eb (L2 at most sqrt(2 * 2^n) * eb); unitaries keep earlier errors' norm."""
    arith = fp32_tol(ngates) if dtype == "c64" else 1e-12
    return passes * np.sqrt(2.0 * (1 << n)) * eb + arith
