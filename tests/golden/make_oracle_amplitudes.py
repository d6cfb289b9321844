"""Writes the stored oracle amplitudes of the two circuits too large for the oracle at test time.

Every value comes from the FP64 oracle (``oracle/tn.py``) and nothing else; the GPU tests
read the files this script writes.  Run from the repository root:

    python tests/golden/make_oracle_amplitudes.py [grid36|fig31_28_14|all]

grid36       6x6 grid of 36 qubits, depth 12, seed 3003 (the 36-qubit amplitude workload);
             the 64 bitstrings random_bitstrings(36, 64, 3004) of its first call, by the
             oracle's qubit-sweep contraction (about 10 s each on 8 host cores).
fig31_28_14  the Fig. 3.1 test circuit with n = 28, k = 14, seed 6042 (the largest point of
             the paper's grid); 8 bitstrings random_bitstrings(28, 8, 6242), by the oracle's
             greedy pairwise contraction (about 1 min and 9 GB of host memory each).
"""
from __future__ import annotations

import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle.tn import contract_amplitude, contract_amplitude_sweep  # noqa: E402
from paper_2108_06831_gb300 import circuits as C  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def _write(name: str, header: list, xs, amps) -> None:
    path = os.path.join(HERE, name)
    with open(path, "w") as f:
        for h in header:
            f.write("# " + h + "\n")
        f.write("# bitstring(decimal)  real  imag   (qubit q is bit n-1-q)\n")
        for x, a in zip(xs, amps):
            f.write(f"{int(x)} {a.real!r} {a.imag!r}\n")
    print("wrote", path, file=sys.stderr)


def grid36() -> None:
    c = C.grid(6, 6, 12, 3003)
    xs = C.random_bitstrings(36, 64, 3004)
    amps = []
    t0 = time.time()
    for i, x in enumerate(xs):
        amps.append(contract_amplitude_sweep(c, int(x)))
        print(f"grid36 {i + 1}/64 {time.time() - t0:.0f}s", file=sys.stderr)
    _write("oracle_grid6x6_d12_s3003.txt",
           ["<x|C|0> of C = grid(6, 6, 12, seed 3003): 36 qubits, depth 12, {sqrtX, sqrtY, sqrtW} + CZ",
            "in four alternating edge patterns; x = random_bitstrings(36, 64, seed 3004).",
            "FP64 oracle, oracle.tn.contract_amplitude_sweep (written by tests/golden/make_oracle_amplitudes.py)."],
           xs, amps)


def fig31_28_14() -> None:
    c = C.paper_fig31(28, 14, 6042)
    xs = C.random_bitstrings(28, 8, 6242)
    amps = []
    t0 = time.time()
    for i, x in enumerate(xs):
        amps.append(contract_amplitude(c, int(x)))
        print(f"fig31 {i + 1}/8 {time.time() - t0:.0f}s", file=sys.stderr)
    _write("oracle_fig31_n28_k14_s6042.txt",
           ["<x|C|0> of C = paper_fig31(28, 14, seed 6042): the Fig. 3.1 test circuit, n = 28 qubits,",
            "k = 14 rounds, angles U[0, 2pi); x = random_bitstrings(28, 8, seed 6242).",
            "FP64 oracle, oracle.tn.contract_amplitude (written by tests/golden/make_oracle_amplitudes.py)."],
           xs, amps)


if __name__ == "__main__":
    which = sys.argv[1] if len(sys.argv) > 1 else "all"
    if which in ("grid36", "all"):
        grid36()
    if which in ("fig31_28_14", "all"):
        fig31_28_14()
