"""The circuit as a tensor network, contracted pairwise (test infrastructure only).

Sec. 2.2.2 (Eq. 2.3) writes the N-qubit state as the coefficient tensor
C^{i_1..i_N} whose legs are the qubits; Sec. 2.2.3 obtains one amplitude by
representing the final basis state as tensors too and contracting every index,
with the contraction order a free choice because contraction is associative.
Sec. 2.2.1 defines the two operations used: the tensor product (orders add)
and the contraction of a shared index (a sum over that index, Eq. 2.2).

The network built here has one node per input qubit (the vector |x0_q>), one
node per gate (a k-qubit gate is the order-2k tensor U[out_1..out_k, in_1..in_k]),
and optionally one node per output qubit (the covector <x_q|).  Every index
label joins exactly two nodes or is open.  Pairs of connected nodes are merged
by summing over all their shared labels (``numpy.tensordot``), choosing at each
step the pair whose merged tensor is smallest; this order is the oracle's own.
"""
from __future__ import annotations

from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from paper_2108_06831_gb300.circuits import Circuit
from .statevector import gate_matrix


class _Node:
    __slots__ = ("data", "labels")

    def __init__(self, data: np.ndarray, labels: List[int]):
        assert data.ndim == len(labels)
        self.data = data
        self.labels = labels


def build_network(c: Circuit, params: Optional[np.ndarray] = None,
                  close_with: Optional[int] = None) -> Tuple[List[_Node], List[int]]:
    """Nodes of the circuit's network and the open output labels (qubit order).

    ``close_with`` = a basis index x closes every output leg with <x_q| so the
    network evaluates the single amplitude <x|C|x0> (Sec. 2.2.3).
    """
    n = c.n_qubits
    nodes: List[_Node] = []
    next_label = 0
    wire = []
    for q in range(n):
        v = np.zeros(2, dtype=np.complex128)
        v[(c.init_basis >> (n - 1 - q)) & 1] = 1.0
        nodes.append(_Node(v, [next_label]))
        wire.append(next_label)
        next_label += 1
    for g in c.gates:
        U = gate_matrix(c, g, params)
        k = len(g.qubits)
        outs = list(range(next_label, next_label + k))
        next_label += k
        ins = [wire[q] for q in g.qubits]
        nodes.append(_Node(U.reshape((2,) * (2 * k)), outs + ins))
        for j, q in enumerate(g.qubits):
            wire[q] = outs[j]
    if close_with is None:
        return nodes, wire
    for q in range(n):
        v = np.zeros(2, dtype=np.complex128)
        v[(close_with >> (n - 1 - q)) & 1] = 1.0
        nodes.append(_Node(v, [wire[q]]))
    return nodes, []


def _merge(a: _Node, b: _Node) -> _Node:
    """Contract every label shared by a and b (sum over shared indices)."""
    shared = [l for l in a.labels if l in b.labels]
    ax_a = [a.labels.index(l) for l in shared]
    ax_b = [b.labels.index(l) for l in shared]
    data = np.tensordot(a.data, b.data, axes=(ax_a, ax_b))
    labels = [l for l in a.labels if l not in shared] + [l for l in b.labels if l not in shared]
    return _Node(data, labels)


def contract(nodes: List[_Node], open_labels: Sequence[int], max_log2: int = 34) -> np.ndarray:
    """Greedy pairwise contraction of the whole network.

    At every step the connected pair with the smallest merged tensor is merged
    (ties: lowest node positions).  Disconnected pieces are joined last by
    tensor products.  The result's axes follow ``open_labels``.
    """
    nodes = list(nodes)
    while len(nodes) > 1:
        best = None
        owner: Dict[int, List[int]] = {}
        for i, nd in enumerate(nodes):
            for l in nd.labels:
                owner.setdefault(l, []).append(i)
        pairs = set()
        for l, own in owner.items():
            if len(own) == 2:
                pairs.add((min(own), max(own)))
        for i, j in sorted(pairs):
            a, b = nodes[i], nodes[j]
            shared = set(a.labels) & set(b.labels)
            size = len(a.labels) + len(b.labels) - 2 * len(shared)
            if best is None or size < best[0]:
                best = (size, i, j)
        if best is None:  # no shared labels left: tensor product of two pieces
            best = (len(nodes[0].labels) + len(nodes[1].labels), 0, 1)
        size, i, j = best
        if size > max_log2:
            raise MemoryError(f"oracle contraction would create a 2^{size} tensor")
        merged = _merge(nodes[i], nodes[j])
        nodes = [nd for k, nd in enumerate(nodes) if k not in (i, j)] + [merged]
    last = nodes[0]
    if not open_labels:
        return np.asarray(last.data).reshape(())
    perm = [last.labels.index(l) for l in open_labels]
    return np.transpose(last.data, perm)


def contract_state(c: Circuit, params: Optional[np.ndarray] = None) -> np.ndarray:
    """The full state (open output legs), flattened MSB-first (small N only)."""
    nodes, wire = build_network(c, params)
    return contract(nodes, wire).reshape(-1)


def contract_amplitude(c: Circuit, x: int, params: Optional[np.ndarray] = None, max_log2: int = 34) -> complex:
    """<x| C |x0> by closing every output leg with a basis covector."""
    nodes, _ = build_network(c, params, close_with=int(x))
    return complex(contract(nodes, [], max_log2=max_log2))


def contract_amplitudes(c: Circuit, xs: Sequence[int], params: Optional[np.ndarray] = None,
                        max_log2: int = 34) -> np.ndarray:
    return np.array([contract_amplitude(c, int(x), params, max_log2) for x in xs], dtype=np.complex128)


# ----------------------------------------------------------------------------------------
# Amplitudes of larger circuits: diagonal two-qubit gates as shared indices, qubit sweep.
# ----------------------------------------------------------------------------------------

def _diag2(kind):
    return kind in ("CZ", "CP")


def build_network_shared(c: Circuit, x: int, params: Optional[np.ndarray] = None):
    """Nodes (data, labels, group) of <x|C|x0> with every diagonal two-qubit gate as a rank-2
    factor on the two qubits' current indices.

    A diagonal gate leaves both basis values unchanged (Sec. 2.1 action on basis states), so
    its tensor d[a,b] = U[ab,ab] joins the indices that carry those values before and after
    it; an index may then be shared by more than two nodes.  A node's group is the largest
    qubit it touches; the output leg of qubit q is closed by the covector <x_q| (Sec. 2.2.3).
    """
    n = c.n_qubits
    nodes = []
    nxt = [0]

    def new():
        nxt[0] += 1
        return nxt[0] - 1

    cur = []
    for q in range(n):
        lab = new()
        v = np.zeros(2, dtype=np.complex128)
        v[(c.init_basis >> (n - 1 - q)) & 1] = 1.0
        nodes.append((v, [lab], q))
        cur.append(lab)
    for g in c.gates:
        U = gate_matrix(c, g, params)
        if len(g.qubits) == 1:
            q = g.qubits[0]
            out = new()
            nodes.append((U, [out, cur[q]], q))
            cur[q] = out
        elif _diag2(g.kind):
            a, b = g.qubits
            nodes.append((np.diag(U).reshape(2, 2), [cur[a], cur[b]], max(a, b)))
        else:
            a, b = g.qubits
            oa, ob = new(), new()
            nodes.append((U.reshape(2, 2, 2, 2), [oa, ob, cur[a], cur[b]], max(a, b)))
            cur[a], cur[b] = oa, ob
    for q in range(n):
        v = np.zeros(2, dtype=np.complex128)
        v[(x >> (n - 1 - q)) & 1] = 1.0
        nodes.append((v, [cur[q]], q))
    return nodes


def _einsum_merge(a, la, b, lb, keep):
    """Sum over the labels of a and b that are not in `keep`; result labels in first-seen order."""
    labels = []
    for l in la + lb:
        if l not in labels:
            labels.append(l)
    out = [l for l in labels if l in keep]
    idx = {l: i for i, l in enumerate(labels)}
    data = np.einsum(a, [idx[l] for l in la], b, [idx[l] for l in lb], [idx[l] for l in out])
    return data, out


def contract_amplitude_sweep(c: Circuit, x: int, params: Optional[np.ndarray] = None) -> complex:
    """<x|C|x0>: the nodes of each qubit (by group) are multiplied into one block, and the
    blocks are absorbed into a running tensor in qubit order, summing every index as soon
    as no remaining node carries it."""
    nodes = build_network_shared(c, int(x), params)
    remaining = {}
    for _, labs, _ in nodes:
        for l in labs:
            remaining[l] = remaining.get(l, 0) + 1
    F, LF = np.ones(()), []
    for q in range(c.n_qubits):
        group = [(d, l) for d, l, g in nodes if g == q]
        if not group:
            continue
        blk, lb = group[0]
        for l in lb:
            remaining[l] -= 1
        for d, l in group[1:]:
            for ll in l:
                remaining[ll] -= 1
            keep = {ll for ll in set(lb) | set(l) if remaining[ll] > 0 or (ll in LF)}
            blk, lb = _einsum_merge(blk, lb, d, l, keep)
        keep = {ll for ll in set(LF) | set(lb) if remaining[ll] > 0}
        F, LF = _einsum_merge(F, LF, blk, lb, keep)
    assert LF == [], LF
    return complex(F)
