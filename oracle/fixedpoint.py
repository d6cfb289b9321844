"""Complex Q4.28 fixed-point state-vector simulation (test infrastructure only; see ``oracle/__init__``).

Sec. 3 reports that the FPGA implementations did their complex arithmetic in 32-bit fixed point
with 28 bits behind the binary point.  The paper fixes no rounding, accumulator width or overflow
rule; the reading restated here (the same one the library's ABI documents):

* an int32 value q stands for q / 2^28;
* a gate matrix is quantised once: q = floor(x 2^28 + 1/2) for the real and the imaginary part of
  every entry (FP64 arithmetic), saturated to the int32 range;
* applying a gate to the state, every output component is the exact integer sum of the complex
  products Uq[i][k] psi[k] (re: ur pr - ui pi, im: ur pi + ui pr), rounded half up to Q4.28,
  floor((acc + 2^27) / 2^28), and saturated to the int32 range.

Gates act one after another in circuit order, each on the state as a tensor with one binary leg
per qubit (Sec. 2.1; qubit q is the most significant leg first, as in ``oracle.statevector``).
Integer sums are exact, so the result does not depend on the order of summation.
"""
from __future__ import annotations

import math
from typing import Sequence, Tuple

import numpy as np

from paper_2108_06831_gb300.circuits import Circuit
from .statevector import gate_matrix

FRAC = 28
ONE = 1 << FRAC
INT32_MIN, INT32_MAX = -(1 << 31), (1 << 31) - 1


def quantize(x: float) -> int:
    """Nearest Q4.28 value of x, halves rounded up, saturated to int32."""
    return int(min(max(math.floor(x * ONE + 0.5), INT32_MIN), INT32_MAX))


def quantize_matrix(U: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """(re, im) of the quantised matrix, int64."""
    re = np.array([[quantize(float(v.real)) for v in row] for row in U], dtype=np.int64)
    im = np.array([[quantize(float(v.imag)) for v in row] for row in U], dtype=np.int64)
    return re, im


def round_q(acc: np.ndarray) -> np.ndarray:
    """floor((acc + 2^27) / 2^28) saturated to int32 (acc: exact int64 sums)."""
    return np.clip((acc + (1 << (FRAC - 1))) >> FRAC, INT32_MIN, INT32_MAX)


def apply_gate_q(re: np.ndarray, im: np.ndarray, n: int, Ur: np.ndarray, Ui: np.ndarray,
                 qubits: Sequence[int]) -> Tuple[np.ndarray, np.ndarray]:
    """psi' = Uq psi on the given qubits, every output component rounded once."""
    k = len(qubits)
    d = 1 << k
    # int64 sums stay exact while every |value| <= 2^29 (products <= 2^58, at most 8 terms)
    assert max(int(np.abs(Ur).max()), int(np.abs(Ui).max())) <= 1 << 29
    assert int(np.abs(re).max(initial=0)) <= 1 << 29 and int(np.abs(im).max(initial=0)) <= 1 << 29
    axes = list(qubits)
    tr = np.moveaxis(re.reshape((2,) * n), axes, list(range(k))).reshape(d, -1)
    ti = np.moveaxis(im.reshape((2,) * n), axes, list(range(k))).reshape(d, -1)
    out_r = np.empty_like(tr)
    out_i = np.empty_like(ti)
    for l in range(d):
        acc_r = np.zeros(tr.shape[1], dtype=np.int64)
        acc_i = np.zeros(tr.shape[1], dtype=np.int64)
        for m in range(d):
            acc_r += Ur[l, m] * tr[m] - Ui[l, m] * ti[m]
            acc_i += Ur[l, m] * ti[m] + Ui[l, m] * tr[m]
        out_r[l] = round_q(acc_r)
        out_i[l] = round_q(acc_i)
    back = lambda t: np.moveaxis(t.reshape((2,) * n), list(range(k)), axes).reshape(-1)
    return back(out_r), back(out_i)


def simulate_state_q428(c: Circuit) -> Tuple[np.ndarray, np.ndarray]:
    """The circuit applied to |init_basis> in Q4.28: (re, im) int64 arrays of the int32 values."""
    n = c.n_qubits
    re = np.zeros(1 << n, dtype=np.int64)
    im = np.zeros(1 << n, dtype=np.int64)
    re[c.init_basis] = ONE
    for g in c.gates:
        Ur, Ui = quantize_matrix(gate_matrix(c, g, None))
        re, im = apply_gate_q(re, im, n, Ur, Ui, g.qubits)
    return re, im


def to_complex(re: np.ndarray, im: np.ndarray) -> np.ndarray:
    """The represented values, complex128 (exact: |q| < 2^31 < 2^53)."""
    return (re.astype(np.float64) + 1j * im.astype(np.float64)) / ONE
