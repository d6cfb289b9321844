"""GB300-native tensor-network contraction of quantum circuits.

The compute path lives in the CUDA library ``libtnq.so`` (sources in ``csrc/``,
C ABI in ``include/tn.h``); :mod:`paper_2108_06831_gb300.tn` is its thin ctypes
binding and :mod:`paper_2108_06831_gb300.circuits` describes seeded workloads.
Importing this package loads nothing; the binding loads the library on first use
and raises if it has not been built.
"""
