"""Stored oracle amplitudes (tests/golden/oracle_*.txt) against the oracle run here (CPU).

The GPU parity tests of the 36-qubit grid read amplitudes that the oracle needs ~10 s each
to compute; they are written by tests/golden/make_oracle_amplitudes.py, which calls only
the oracle.  This recomputes one of them, so a stored file that no longer matches the
circuit generator or the oracle fails here.
"""
import os

import numpy as np

from paper_2108_06831_gb300 import circuits as C

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _read(name):
    rows = [l.split() for l in open(os.path.join(HERE, name)) if l.strip() and not l.startswith("#")]
    return (np.array([int(r[0]) for r in rows], dtype=np.uint64),
            np.array([complex(float(r[1]), float(r[2])) for r in rows]))


def test_grid36_fixture_matches_generator_and_oracle():
    from oracle.tn import contract_amplitude_sweep
    xs, ref = _read("oracle_grid6x6_d12_s3003.txt")
    assert len(xs) == 64 and np.array_equal(xs, C.random_bitstrings(36, 64, 3004))
    c = C.grid(6, 6, 12, 3003)
    a = contract_amplitude_sweep(c, int(xs[5]))
    assert abs(a - ref[5]) <= 1e-12 * np.abs(ref).max()
    # Porter-Thomas: the mean of |a|^2 2^36 over 64 amplitudes is near 1 (weak sanity check)
    assert 0.5 < float(np.mean(np.abs(ref) ** 2) * 2.0 ** 36) < 1.6


def test_fig31_fixture_matches_generator():
    xs, ref = _read("oracle_fig31_n28_k14_s6042.txt")
    assert len(xs) == 8 and np.array_equal(xs, C.random_bitstrings(28, 8, 6242))
    assert np.all(np.isfinite(ref)) and np.all(np.abs(ref) < 1.0)
