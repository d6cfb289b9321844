"""FP64 CPU oracle for tensor-network quantum-circuit contraction.

TEST INFRASTRUCTURE ONLY.  Nothing on the library's product path may import,
call or link this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` use it.  It shares no code with the
CUDA library (no gate tables, no planners, no helpers); the only thing both
sides read is the seeded workload description in
``paper_2108_06831_gb300/circuits.py``, which holds names and random angles but
no arithmetic of the method.

Contents (each function cites the part of the paper it restates):

* :mod:`oracle.gates`        - gate matrices in complex128 (Sec. 2.1 unitaries,
  Kronecker convention), plus the conventions the paper leaves open;
* :mod:`oracle.statevector`  - plain state-vector simulation psi' = U psi,
  gate by gate (Sec. 2.1), and a brute-force full-matrix builder for small N;
* :mod:`oracle.tn`           - the circuit as a tensor network (Sec. 2.2.2,
  Eq. 2.3) contracted pairwise by explicit sums over shared indices
  (Sec. 2.2.1, Eq. 2.2), with output legs left open (state) or closed by a
  basis bra (amplitude, Sec. 2.2.3);
* :mod:`oracle.observables`  - Pauli-sum expectation values on the FP64 state;
* :mod:`oracle.gradients`    - parameter-shift and central finite-difference
  gradients of an expectation value.

Parity status: every function is pinned by tests in ``tests/test_oracle_*.py``
against closed forms, textbook identities or brute force (none is unpinned).
"""
