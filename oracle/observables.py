"""Pauli-sum expectation values on the FP64 state (test infrastructure only).

An expectation <psi|H|psi> with H = sum_t c_t P_t is evaluated by applying each
Pauli string P_t to psi qubit by qubit (the Sec. 2.1 rule psi' = U psi with the
Pauli matrices) and taking the inner product with psi.
"""
from __future__ import annotations

from typing import Optional

import numpy as np

from paper_2108_06831_gb300.circuits import Circuit, PauliSum
from . import gates as G
from .statevector import apply_matrix, simulate_state


def apply_pauli_string(psi: np.ndarray, n: int, s: str) -> np.ndarray:
    out = psi
    for q, p in enumerate(s):
        if p != "I":
            out = apply_matrix(out, n, G.PAULI[p], (q,))
    return out


def expectation_of_state(psi: np.ndarray, H: PauliSum) -> float:
    total = 0.0 + 0.0j
    for c, s in zip(H.coef, H.strings):
        total += c * np.vdot(psi, apply_pauli_string(psi, H.n_qubits, s))
    return float(total.real)


def apply_hamiltonian(psi: np.ndarray, H: PauliSum) -> np.ndarray:
    out = np.zeros_like(psi)
    for c, s in zip(H.coef, H.strings):
        out += c * apply_pauli_string(psi, H.n_qubits, s)
    return out


def expectation(c: Circuit, H: PauliSum, params: Optional[np.ndarray] = None, angle_overrides=None) -> float:
    return expectation_of_state(simulate_state(c, params, angle_overrides), H)


def hamiltonian_matrix(H: PauliSum) -> np.ndarray:
    """Dense 2^N x 2^N matrix of H from Kronecker products (qubit 0 leftmost), small N."""
    dim = 1 << H.n_qubits
    M = np.zeros((dim, dim), dtype=np.complex128)
    for c, s in zip(H.coef, H.strings):
        K = np.array([[1.0 + 0j]])
        for p in s:
            K = np.kron(K, G.PAULI[p])
        M += c * K
    return M
