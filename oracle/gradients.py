"""Gradients of an expectation value w.r.t. circuit parameters (test infrastructure only).

Two independent FP64 methods:

* parameter shift: in each of its angles a, every parameterised gate of this
  library has the form exp(-i a G / 2) times a constant, with G having exactly
  two eigenvalues that differ by 2 (RX/RY/RZ: G = X/Y/Z; U3 = e^{i(p+l)/2}
  RZ(p) RY(t) RZ(l); CP(a) = exp(-i a G/2) with G = -2|11><11|, eigenvalues 0
  and -2).  For such gates the expectation is a + b cos a + c sin a, so
  d<H>/da = (<H>(a + pi/2) - <H>(a - pi/2)) / 2 exactly, summed over every
  occurrence of a parameter;
* central finite differences with step h on the parameter vector.
"""
from __future__ import annotations

import math
from typing import Optional

import numpy as np

from paper_2108_06831_gb300.circuits import Circuit, PauliSum
from .observables import expectation


def param_shift_grad(c: Circuit, H: PauliSum, params: np.ndarray) -> np.ndarray:
    grad = np.zeros(len(params), dtype=np.float64)
    for gi, g in enumerate(c.gates):
        if g.param_idx < 0:
            continue
        base = list(c.angles_for(g, params))
        for a in range(g.n_angles):
            vals = []
            for sgn in (+1.0, -1.0):
                ang = list(base)
                ang[a] += sgn * math.pi / 2
                vals.append(expectation(c, H, params, {gi: tuple(ang)}))
            grad[g.param_idx + a] += 0.5 * (vals[0] - vals[1])
    return grad


def finite_diff_grad(c: Circuit, H: PauliSum, params: np.ndarray, h: float = 1e-4) -> np.ndarray:
    grad = np.zeros(len(params), dtype=np.float64)
    for p in range(len(params)):
        up = params.copy()
        dn = params.copy()
        up[p] += h
        dn[p] -= h
        grad[p] = (expectation(c, H, up) - expectation(c, H, dn)) / (2 * h)
    return grad
