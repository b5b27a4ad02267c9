"""The FP32 energy tolerance shared by the GPU parity tests.

FP32 statevector results must agree with the complex128 oracle within 1e-6
relative energy error.  The energy of a random-like n-qubit state is a
near-cancellation: sum_k c_k <P_k> has typical size
E_typ = ||c||_2 2^(-n/2), far below sum_k |c_k|, and for the few tasks whose
energy lands near zero any relative error diverges whatever the precision.
The error is therefore taken relative to max(|E_ref|, E_typ): plain relative
error for every task whose energy is at least typical, the same 1e-6 of
E_typ for the near-zero ones.
"""
import numpy as np

FP32_ENERGY_TOL = 1e-6


def energy_scale(terms, n: int) -> float:
    """E_typ = ||c||_2 2^(-n/2), the typical |E| of a random-like state."""
    c = np.asarray(terms["coef"], dtype=np.float64)
    return float(np.sqrt(np.sum(c * c))) * 2.0 ** (-n / 2)


def energy_error(e: float, e_ref: float, terms, n: int) -> float:
    """|E - E_ref| / max(|E_ref|, E_typ)."""
    return abs(e - e_ref) / max(abs(e_ref), energy_scale(terms, n))


def energy_ok(e: float, e_ref: float, terms, n: int, fp64: bool) -> bool:
    """FP64: 1e-12 relative (at least 1e-12 absolute); FP32: FP32_ENERGY_TOL
    on the error above."""
    if fp64:
        return abs(e - e_ref) <= 1e-12 * max(1.0, abs(e_ref))
    return energy_error(e, e_ref, terms, n) <= FP32_ENERGY_TOL
