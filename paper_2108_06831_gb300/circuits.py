"""Seeded synthetic workload generators (gate lists, parameters, bitstrings, Hamiltonians).

This module only *describes* inputs: gate names, the qubits they act on, and the
random angles a workload draws.  It builds no gate matrix and applies nothing, so
that the FP64 oracle and the CUDA library each turn these descriptions into
arithmetic with their own code.

Conventions shared by every consumer:

* qubit ``q`` of an ``n``-qubit register is bit ``n-1-q`` of a basis index
  (most-significant-bit first, the ordering of the paper's Sec. 2.1 where
  ``|00>,|01>,|10>,|11>`` are labelled ``|0>..|3>``);
* a two-qubit gate lists its qubits as ``(a, b)``; its 4x4 matrix is indexed by
  ``2*bit(a) + bit(b)`` (the Kronecker order ``U (x) V`` of Sec. 2.1);
* parameterised gates read their angles from a per-batch parameter vector at
  ``params[param_idx : param_idx + arity]`` (arity 3 for ``U3``, 1 for
  ``RX/RY/RZ/CP``); ``param_idx = -1`` means the angles are stored in the gate.

Workload recipes (seeded PCG64 streams; seed = 1000 * workload_index + item_index
unless a caller passes its own):

* brickwork: layer l applies U3(theta, phi, lambda) with all three angles
  uniform in [0, 2 pi) on every qubit, then CZ(2i, 2i+1) for even l and
  CZ(2i+1, 2i+2) for odd l;
* grid: qubit = cols*r + c; each layer draws an i.i.d. uniform gate from
  {sqrt X, sqrt Y, sqrt W} per qubit, then CZ on edge pattern l mod 4
  (A: horizontal, even left column; B: horizontal, odd; C: vertical, even top
  row; D: vertical, odd);
* hardware-efficient ansatz: per layer RY(theta) on all, RZ(theta) on all, then
  CNOT(i, i+1) for i = 0..n-2; parameter index = 2n*layer + {0..n-1 RY, n..2n-1 RZ};
* QFT on a basis state: H / controlled-phase ladder followed by the
  qubit-reversal SWAPs, applied to a seeded random basis state;
* the paper's test circuit (Fig. 3.1): H on every qubit, then k rounds of
  CNOT(2i -> 2i+1), Rz on every qubit, CZ(2i+1, 2i+2), Rx on every qubit, then H
  on every qubit; rotation angles uniform in [0, 2 pi).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

# Gate names understood by both the oracle and the library, with their qubit
# count and the number of angles they take.
GATE_ARITY = {
    "H": (1, 0), "X": (1, 0), "Y": (1, 0), "Z": (1, 0),
    "S": (1, 0), "SDG": (1, 0), "T": (1, 0), "TDG": (1, 0),
    "SX": (1, 0), "SY": (1, 0), "SW": (1, 0),
    "RX": (1, 1), "RY": (1, 1), "RZ": (1, 1), "U3": (1, 3),
    "CZ": (2, 0), "CNOT": (2, 0), "CP": (2, 1), "SWAP": (2, 0),
    "MAT1": (1, 0), "MAT2": (2, 0),
}


@dataclass(frozen=True)
class Gate:
    kind: str
    qubits: Tuple[int, ...]
    angles: Tuple[float, ...] = ()
    param_idx: int = -1
    # row-major complex matrix for MAT1 (2x2) / MAT2 (4x4); None otherwise
    mat: Optional[Tuple[complex, ...]] = None

    @property
    def n_angles(self) -> int:
        return GATE_ARITY[self.kind][1]


@dataclass
class Circuit:
    n_qubits: int
    gates: List[Gate]
    init_basis: int = 0
    name: str = ""
    n_params: int = 0

    def angles_for(self, gate: Gate, params: Optional[np.ndarray]) -> Tuple[float, ...]:
        """Angles of ``gate`` for one parameter vector (no arithmetic beyond lookup)."""
        if gate.param_idx < 0:
            return tuple(gate.angles)
        assert params is not None, "parameterised circuit needs params"
        return tuple(float(params[gate.param_idx + i]) for i in range(gate.n_angles))


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ----------------------------------------------------------------------------
# textbook circuits (pins)
# ----------------------------------------------------------------------------

def bell() -> Circuit:
    return Circuit(2, [Gate("H", (0,)), Gate("CNOT", (0, 1))], name="bell")


def ghz(n: int) -> Circuit:
    gates = [Gate("H", (0,))] + [Gate("CNOT", (0, q)) for q in range(1, n)]
    return Circuit(n, gates, name=f"ghz{n}")


def fig21_as_drawn() -> Circuit:
    """The 3-qubit circuit of the paper's Fig. 2.1 exactly as drawn."""
    g = [Gate("H", (0,)), Gate("H", (1,)), Gate("H", (2,)),
         Gate("CNOT", (0, 1)), Gate("CNOT", (0, 2)),
         Gate("H", (1,)), Gate("H", (2,))]
    return Circuit(3, g, name="fig21")


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def brickwork(n: int, depth: int, seed: int, parameterized: bool = False) -> Tuple[Circuit, Optional[np.ndarray]]:
    """1D brickwork of U3 layers and alternating nearest-neighbour CZ.

    Returns (circuit, params).  With ``parameterized`` the U3 angles live in the
    returned parameter vector (param_idx set), otherwise in the gates and
    params is None.
    """
    rng = _rng(seed)
    gates: List[Gate] = []
    params: List[float] = []
    for layer in range(depth):
        ang = rng.uniform(0.0, 2.0 * math.pi, size=(n, 3))
        for q in range(n):
            a = tuple(float(x) for x in ang[q])
            if parameterized:
                gates.append(Gate("U3", (q,), (), len(params)))
                params.extend(a)
            else:
                gates.append(Gate("U3", (q,), a))
        start = 0 if layer % 2 == 0 else 1
        for a in range(start, n - 1, 2):
            gates.append(Gate("CZ", (a, a + 1)))
    c = Circuit(n, gates, name=f"brickwork_n{n}_d{depth}", n_params=len(params))
    return c, (np.asarray(params, dtype=np.float64) if parameterized else None)


def grid_edges(rows: int, cols: int, pattern: int) -> List[Tuple[int, int]]:
    """CZ pairs of edge pattern A/B/C/D (0..3) on a rows x cols grid."""
    e = []
    if pattern in (0, 1):
        for r in range(rows):
            for c in range(pattern, cols - 1, 2):
                e.append((cols * r + c, cols * r + c + 1))
    else:
        start = pattern - 2
        for r in range(start, rows - 1, 2):
            for c in range(cols):
                e.append((cols * r + c, cols * (r + 1) + c))
    return e


def grid(rows: int, cols: int, depth: int, seed: int) -> Circuit:
    rng = _rng(seed)
    n = rows * cols
    names = ("SX", "SY", "SW")
    gates: List[Gate] = []
    for layer in range(depth):
        pick = rng.integers(0, 3, size=n)
        for q in range(n):
            gates.append(Gate(names[int(pick[q])], (q,)))
        for a, b in grid_edges(rows, cols, layer % 4):
            gates.append(Gate("CZ", (a, b)))
    return Circuit(n, gates, name=f"grid{rows}x{cols}_d{depth}")


def hea(n: int, layers: int) -> Circuit:
    """Hardware-efficient ansatz: RY, RZ on every qubit, then a CNOT ladder."""
    gates: List[Gate] = []
    for layer in range(layers):
        base = 2 * n * layer
        for q in range(n):
            gates.append(Gate("RY", (q,), (), base + q))
        for q in range(n):
            gates.append(Gate("RZ", (q,), (), base + n + q))
        for q in range(n - 1):
            gates.append(Gate("CNOT", (q, q + 1)))
    return Circuit(n, gates, name=f"hea_n{n}_l{layers}", n_params=2 * n * layers)


def hea_params(n_params: int, batch: int, seed: int) -> np.ndarray:
    """theta ~ U[-pi, pi], shape (batch, n_params)."""
    return _rng(seed).uniform(-math.pi, math.pi, size=(batch, n_params))


def qft(n: int, init_basis: int = 0) -> Circuit:
    gates: List[Gate] = []
    for j in range(n):
        gates.append(Gate("H", (j,)))
        for k in range(j + 1, n):
            gates.append(Gate("CP", (k, j), (2.0 * math.pi / float(1 << (k - j + 1)),)))
    for j in range(n // 2):
        gates.append(Gate("SWAP", (j, n - 1 - j)))
    return Circuit(n, gates, init_basis=init_basis, name=f"qft{n}")


def paper_fig31(n: int, k: int, seed: int) -> Circuit:
    """The paper's Fig. 3.1 test circuit with n qubits and k rounds."""
    rng = _rng(seed)
    gates: List[Gate] = [Gate("H", (q,)) for q in range(n)]
    for _ in range(k):
        for i in range(0, n - 1, 2):
            gates.append(Gate("CNOT", (i, i + 1)))
        for q, a in enumerate(rng.uniform(0.0, 2.0 * math.pi, size=n)):
            gates.append(Gate("RZ", (q,), (float(a),)))
        for i in range(1, n - 1, 2):
            gates.append(Gate("CZ", (i, i + 1)))
        for q, a in enumerate(rng.uniform(0.0, 2.0 * math.pi, size=n)):
            gates.append(Gate("RX", (q,), (float(a),)))
    gates += [Gate("H", (q,)) for q in range(n)]
    return Circuit(n, gates, name=f"fig31_n{n}_k{k}")


def random_circuit(n: int, n_gates: int, seed: int) -> Circuit:
    """Mixed random circuit over every gate kind (for brute-force pins)."""
    rng = _rng(seed)
    one = ["H", "X", "Y", "Z", "S", "SDG", "T", "TDG", "SX", "SY", "SW", "RX", "RY", "RZ", "U3", "MAT1"]
    two = ["CZ", "CNOT", "CP", "SWAP", "MAT2"]
    gates: List[Gate] = []
    for _ in range(n_gates):
        if n >= 2 and rng.uniform() < 0.4:
            kind = two[int(rng.integers(0, len(two)))]
            a, b = (int(x) for x in rng.choice(n, size=2, replace=False))
            qs: Tuple[int, ...] = (a, b)
        else:
            kind = one[int(rng.integers(0, len(one)))]
            qs = (int(rng.integers(0, n)),)
        mat = None
        if kind in ("MAT1", "MAT2"):
            d = 2 if kind == "MAT1" else 4
            z = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
            # a Haar-like unitary from the QR factorisation of a Gaussian matrix
            qm, rm = np.linalg.qr(z)
            qm = qm * (np.diag(rm) / np.abs(np.diag(rm)))
            mat = tuple(complex(x) for x in qm.reshape(-1))
        ang = tuple(float(x) for x in rng.uniform(0, 2 * math.pi, size=GATE_ARITY[kind][1]))
        gates.append(Gate(kind, qs, ang, -1, mat))
    return Circuit(n, gates, name=f"random_n{n}_g{n_gates}")


def random_basis(n: int, seed: int) -> int:
    return int(_rng(seed).integers(0, 1 << n)) if n < 63 else int(_rng(seed).integers(0, 1 << 62))


def random_bitstrings(n: int, count: int, seed: int) -> np.ndarray:
    """``count`` uniform n-bit basis indices as uint64 (MSB-first qubit order)."""
    rng = _rng(seed)
    out = np.zeros(count, dtype=np.uint64)
    for lo in range(0, n, 32):
        w = min(32, n - lo)
        out |= rng.integers(0, 1 << w, size=count, dtype=np.uint64) << np.uint64(lo)
    return out


def serving_mix(n_circuits: int, seed: int, n_min: int = 8, n_max: int = 22,
                d_min: int = 4, d_max: int = 30) -> List[Circuit]:
    """Half brickwork (n ~ U[n_min, n_max], depth ~ U[d_min, d_max]), half QFT on a random basis state."""
    rng = _rng(seed)
    out: List[Circuit] = []
    for i in range(n_circuits):
        n = int(rng.integers(n_min, n_max + 1))
        if i % 2 == 0:
            d = int(rng.integers(d_min, d_max + 1))
            c, _ = brickwork(n, d, seed * 100003 + i)
        else:
            c = qft(n, random_basis(n, seed * 100003 + i))
        out.append(c)
    return out


def serving_mix_params(n_circuits: int, seed: int, n_min: int = 8, n_max: int = 22,
                       d_min: int = 4, d_max: int = 30) -> Tuple[List[Circuit], List[np.ndarray]]:
    """serving_mix with the brickwork halves' U3 angles as parameters: (circuits, per-circuit
    parameter vectors; empty for the QFT halves).  The parameter values equal the angles
    serving_mix(n_circuits, seed) draws, so the states are the same."""
    rng = _rng(seed)
    circs: List[Circuit] = []
    params: List[np.ndarray] = []
    for i in range(n_circuits):
        n = int(rng.integers(n_min, n_max + 1))
        if i % 2 == 0:
            d = int(rng.integers(d_min, d_max + 1))
            c, p = brickwork(n, d, seed * 100003 + i, parameterized=True)
        else:
            c, p = qft(n, random_basis(n, seed * 100003 + i)), np.zeros(0)
        circs.append(c)
        params.append(p)
    return circs, params


# ----------------------------------------------------------------------------
# observables
# ----------------------------------------------------------------------------

@dataclass
class PauliSum:
    """H = sum_t coef[t] * P_t with P_t a string over {I, X, Y, Z} (index q = qubit q)."""
    n_qubits: int
    coef: List[float] = field(default_factory=list)
    strings: List[str] = field(default_factory=list)

    def add(self, c: float, ops: Sequence[Tuple[int, str]]) -> "PauliSum":
        s = ["I"] * self.n_qubits
        for q, p in ops:
            s[q] = p
        self.coef.append(float(c))
        self.strings.append("".join(s))
        return self


def tfim(n: int, j: float = 1.0, h: float = 1.0) -> PauliSum:
    """Open-chain transverse-field Ising model H = -J sum Z_i Z_{i+1} - h sum X_i."""
    H = PauliSum(n)
    for i in range(n - 1):
        H.add(-j, [(i, "Z"), (i + 1, "Z")])
    for i in range(n):
        H.add(-h, [(i, "X")])
    return H


def random_pauli_sum(n: int, n_terms: int, seed: int) -> PauliSum:
    rng = _rng(seed)
    H = PauliSum(n)
    for _ in range(n_terms):
        s = "".join("IXYZ"[int(x)] for x in rng.integers(0, 4, size=n))
        H.coef.append(float(rng.normal()))
        H.strings.append(s)
    return H
