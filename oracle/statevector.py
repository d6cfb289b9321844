"""Plain FP64 state-vector simulation (test infrastructure only).

Sec. 2.1: an N-qubit state is a vector in C^(2^N) whose basis index spells the
qubits most-significant-first (|00>,|01>,|10>,|11> = |0>..|3>), a gate acts as
psi' = U psi, and an operator on several qubits is a Kronecker product.  This
module applies each gate to the state viewed as an order-N tensor with one
axis of size 2 per qubit (axis q = qubit q), which is exactly that ordering.
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np

from paper_2108_06831_gb300.circuits import Circuit, Gate
from . import gates as G


def basis_state(n: int, x: int) -> np.ndarray:
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[x] = 1.0
    return psi


def gate_matrix(c: Circuit, g: Gate, params: Optional[np.ndarray], angles_override=None) -> np.ndarray:
    ang = angles_override if angles_override is not None else c.angles_for(g, params)
    return G.matrix(g.kind, ang, g.mat)


def apply_matrix(psi: np.ndarray, n: int, U: np.ndarray, qubits: Sequence[int]) -> np.ndarray:
    """psi' = (U on ``qubits``, identity elsewhere) psi.

    The k-qubit matrix U is reshaped to an order-2k tensor U[out..., in...];
    its input axes are summed against the state's axes ``qubits`` and its
    output axes put back in their place.
    """
    k = len(qubits)
    t = psi.reshape((2,) * n)
    Ut = U.reshape((2,) * (2 * k))
    out = np.tensordot(Ut, t, axes=(list(range(k, 2 * k)), list(qubits)))
    out = np.moveaxis(out, list(range(k)), list(qubits))
    return np.ascontiguousarray(out).reshape(-1)


def simulate_state(c: Circuit, params: Optional[np.ndarray] = None, angle_overrides=None) -> np.ndarray:
    """U_G ... U_1 |x0> for the circuit's gates in time order (complex128).

    ``angle_overrides`` maps a gate position to replacement angles (used by the
    parameter-shift rule to shift one occurrence of a parameter).
    """
    psi = basis_state(c.n_qubits, c.init_basis)
    for i, g in enumerate(c.gates):
        ov = None if angle_overrides is None else angle_overrides.get(i)
        psi = apply_matrix(psi, c.n_qubits, gate_matrix(c, g, params, ov), g.qubits)
    return psi


def full_operator(n: int, U: np.ndarray, qubits: Sequence[int]) -> np.ndarray:
    """The 2^N x 2^N matrix of U acting on ``qubits`` (brute force, small N).

    Built entry by entry from the definition: <y| U_full |x> equals
    U[out bits of y on qubits, in bits of x on qubits] when x and y agree on
    every other qubit, and 0 otherwise.
    """
    dim = 1 << n
    k = len(qubits)
    M = np.zeros((dim, dim), dtype=np.complex128)
    bitpos = [n - 1 - q for q in qubits]
    others = ~sum(1 << b for b in bitpos) & (dim - 1)
    for x in range(dim):
        col_in = 0
        for b in bitpos:
            col_in = (col_in << 1) | ((x >> b) & 1)
        for row_out in range(1 << k):
            y = x & others
            for j, b in enumerate(bitpos):
                if (row_out >> (k - 1 - j)) & 1:
                    y |= 1 << b
            M[y, x] = U[row_out, col_in]
    return M


def circuit_unitary(c: Circuit, params: Optional[np.ndarray] = None) -> np.ndarray:
    """Product of full 2^N x 2^N gate matrices, last gate leftmost (small N only)."""
    dim = 1 << c.n_qubits
    Ufull = np.eye(dim, dtype=np.complex128)
    for g in c.gates:
        Ufull = full_operator(c.n_qubits, gate_matrix(c, g, params), g.qubits) @ Ufull
    return Ufull
