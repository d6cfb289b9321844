"""Gate matrices in complex128 (test infrastructure only; see ``oracle/__init__``).

Sec. 2.1 states that a gate is a unitary U acting as psi' = U psi and that
multi-qubit operators are Kronecker products, with ``U (x) V`` laid out in
blocks ``U_ij V``.  The paper names but does not define H, CNOT, Rz, Rx and CZ
(Fig. 2.1, Fig. 3.1); the textbook definitions used here are:

* H = [[1, 1], [1, -1]] / sqrt 2;  X, Y, Z the Pauli matrices;
* RX/RY/RZ(t) = exp(-i t P / 2) for P = X/Y/Z;
* U3(t, p, l) = [[cos t/2, -e^{il} sin t/2], [e^{ip} sin t/2, e^{i(p+l)} cos t/2]];
* SX = RX(pi/2), SY = RY(pi/2), SW = exp(-i pi/4 W) with W = (X + Y)/sqrt 2;
* CZ = diag(1, 1, 1, -1), CP(p) = diag(1, 1, 1, e^{ip}), CNOT with the control
  listed first, SWAP; two-qubit matrices are indexed 2*bit(first) + bit(second).
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np

I2 = np.eye(2, dtype=np.complex128)
X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
Z = np.array([[1, 0], [0, -1]], dtype=np.complex128)
PAULI = {"I": I2, "X": X, "Y": Y, "Z": Z}


def _expm_pauli(theta: float, P: np.ndarray) -> np.ndarray:
    """exp(-i theta P / 2) for an involutory P (P^2 = I): cos(t/2) I - i sin(t/2) P."""
    return math.cos(theta / 2) * I2 - 1j * math.sin(theta / 2) * P


def rx(t: float) -> np.ndarray:
    return _expm_pauli(t, X)


def ry(t: float) -> np.ndarray:
    return _expm_pauli(t, Y)


def rz(t: float) -> np.ndarray:
    return _expm_pauli(t, Z)


def u3(t: float, p: float, l: float) -> np.ndarray:
    c, s = math.cos(t / 2), math.sin(t / 2)
    return np.array([[c, -np.exp(1j * l) * s],
                     [np.exp(1j * p) * s, np.exp(1j * (p + l)) * c]], dtype=np.complex128)


def matrix(kind: str, angles: Sequence[float] = (), mat=None) -> np.ndarray:
    """The unitary of a named gate (2x2 or 4x4, complex128)."""
    if kind == "H":
        return np.array([[1, 1], [1, -1]], dtype=np.complex128) / math.sqrt(2.0)
    if kind == "X":
        return X.copy()
    if kind == "Y":
        return Y.copy()
    if kind == "Z":
        return Z.copy()
    if kind == "S":
        return np.diag([1, 1j]).astype(np.complex128)
    if kind == "SDG":
        return np.diag([1, -1j]).astype(np.complex128)
    if kind == "T":
        return np.diag([1, np.exp(1j * math.pi / 4)]).astype(np.complex128)
    if kind == "TDG":
        return np.diag([1, np.exp(-1j * math.pi / 4)]).astype(np.complex128)
    if kind == "SX":
        return rx(math.pi / 2)
    if kind == "SY":
        return ry(math.pi / 2)
    if kind == "SW":
        W = (X + Y) / math.sqrt(2.0)
        return _expm_pauli(math.pi / 2, W)
    if kind == "RX":
        return rx(angles[0])
    if kind == "RY":
        return ry(angles[0])
    if kind == "RZ":
        return rz(angles[0])
    if kind == "U3":
        return u3(angles[0], angles[1], angles[2])
    if kind == "CZ":
        return np.diag([1, 1, 1, -1]).astype(np.complex128)
    if kind == "CP":
        return np.diag([1, 1, 1, np.exp(1j * angles[0])]).astype(np.complex128)
    if kind == "CNOT":
        m = np.zeros((4, 4), dtype=np.complex128)
        m[0, 0] = m[1, 1] = m[2, 3] = m[3, 2] = 1
        return m
    if kind == "SWAP":
        m = np.zeros((4, 4), dtype=np.complex128)
        m[0, 0] = m[1, 2] = m[2, 1] = m[3, 3] = 1
        return m
    if kind in ("MAT1", "MAT2"):
        d = 2 if kind == "MAT1" else 4
        return np.asarray(mat, dtype=np.complex128).reshape(d, d)
    raise ValueError(f"unknown gate kind {kind!r}")
