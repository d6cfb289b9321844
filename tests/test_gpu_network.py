"""Amplitudes by network contraction (permutations + batched complex GEMMs) vs the FP64 oracle."""
import numpy as np
import pytest

from paper_2108_06831_gb300 import circuits as C

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-5


def _amps(circ, xs, B, precision, max_log2=0, order_search=0):
    from paper_2108_06831_gb300 import tn
    ch = tn.CircuitHandle(circ)
    p = tn.Plan(ch, target=tn.TARGET_AMPLITUDES, network_bitstrings=B, precision=precision,
                max_intermediate_log2=max_log2, order_search=order_search)
    ws = torch.empty(max(p.workspace_bytes, 16), dtype=torch.uint8, device="cuda")
    x = torch.as_tensor(np.asarray(xs, dtype=np.uint64).astype(np.int64), device="cuda")
    out = torch.full((len(xs),), complex(float("nan"), 0), dtype=torch.complex64, device="cuda")
    tn.contract_amplitudes(p, None, x, out, ws)
    torch.cuda.synchronize()
    assert tn.sync_status() == tn.OK
    return out.cpu().numpy(), p.stats()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_grid_4x4_depth12(precision):
    from oracle.statevector import simulate_state
    c = C.grid(4, 4, 12, 21)
    psi = simulate_state(c)
    xs = C.random_bitstrings(16, 200, 5)
    got, st = _amps(c, xs, 256, precision)
    assert st["net_merges"] > 0
    assert _rel(got, psi[xs.astype(np.int64)]) <= TOL


@pytest.mark.parametrize("maker,B", [
    (lambda: C.random_circuit(10, 90, 41), 64),
    (lambda: C.brickwork(14, 8, 9)[0], 128),
    (lambda: C.qft(9, 300), 16),
    (lambda: C.paper_fig31(12, 4, 6), 32),
    (lambda: C.ghz(11), 8),
])
def test_circuit_families(maker, B):
    from oracle.statevector import simulate_state
    c = maker()
    psi = simulate_state(c)
    xs = C.random_bitstrings(c.n_qubits, B - 3, 77)  # fewer than the plan's batch: padded
    xs[0], xs[-1] = 0, (1 << c.n_qubits) - 1  # GHZ has weight only on these two
    got, _ = _amps(c, xs, B, 1)
    assert _rel(got, psi[xs.astype(np.int64)]) <= TOL


def test_grid_4x5_split_bf16_against_fp32():
    """Same bitstrings through the FP32 and the split-BF16 GEMMs: both within the bar of the oracle."""
    from oracle.statevector import simulate_state
    c = C.grid(4, 5, 12, 33)
    psi = simulate_state(c)
    xs = C.random_bitstrings(20, 256, 8)
    ref = psi[xs.astype(np.int64)]
    a32, _ = _amps(c, xs, 256, 0)
    abf, _ = _amps(c, xs, 256, 2)
    assert _rel(a32, ref) <= TOL and _rel(abf, ref) <= TOL


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_grid_5x5_depth12(precision):
    """25 qubits, the same generator as the 36-qubit configuration: sampled amplitudes against
    the oracle's FP64 sweep (itself pinned to state vectors on 4x4 and 4x5 grids)."""
    from oracle.tn import contract_amplitude_sweep
    c = C.grid(5, 5, 12, 55)
    xs = C.random_bitstrings(25, 64, 56)
    got, st = _amps(c, xs, 64, precision)
    ref = np.array([contract_amplitude_sweep(c, int(x)) for x in xs[:6]])
    assert _rel(got[:6], ref) <= TOL


def read_golden_amplitudes(name):
    """(bitstrings, amplitudes) stored by tests/golden/make_oracle_amplitudes.py (FP64 oracle)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    xs, amps = [], []
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            x, re, im = line.split()
            xs.append(int(x))
            amps.append(complex(float(re), float(im)))
    return np.array(xs, dtype=np.uint64), np.array(amps)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_cfg3_grid_6x6_depth12_against_stored_oracle(precision):
    """The 36-qubit configuration in the bench's launch configuration (64 bitstrings per call)
    in each merge precision (FP32, 3xTF32, split BF16): all 64 amplitudes of the call against
    the oracle's FP64 sweep contraction (stored; the oracle needs ~10 s per amplitude), element
    by element within the relative L2 bar, and the Porter-Thomas statistic (mean |a|^2 2^36
    near 1)."""
    c = C.grid(6, 6, 12, 3003)
    xs = C.random_bitstrings(36, 64, 3004)
    gx, ref = read_golden_amplitudes("oracle_grid6x6_d12_s3003.txt")
    assert np.array_equal(gx, xs)  # the generator still makes the stored bitstrings
    got, st = _amps(c, xs, 64, precision)
    assert st["net_max_log2"] <= 28
    err = _rel(got, ref)
    assert err <= TOL, err
    # element by element: no amplitude is off by more than the bar times the vector's RMS
    rms = np.linalg.norm(ref) / np.sqrt(len(ref))
    assert np.max(np.abs(got - ref)) <= TOL * rms * 4, np.max(np.abs(got - ref)) / rms
    print(f"cfg3 precision {precision}: rel L2 error vs FP64 {err:.2e}")
    pt = float(np.mean(np.abs(got.astype(np.complex128)) ** 2) * 2.0 ** 36)
    assert 0.5 < pt < 1.6


# (circuit, bitstrings per call, bitstrings passed, cap): the planner takes every route on
# these -- slicing only, smaller passes only, both (test_network_plan_routes_host_only checks
# that it still does); grid 3x4 at cap 2^4 slices legs of output closures
CAPPED_CASES = [
    (lambda: C.qft(8, 77), 4, 4, 5),
    (lambda: C.brickwork(12, 10, 3)[0], 16, 13, 8),
    (lambda: C.grid(3, 4, 8, 2), 4, 3, 5),
    (lambda: C.random_circuit(10, 120, 5), 4, 4, 7),
    (lambda: C.grid(3, 4, 8, 2), 4, 4, 4),
    (lambda: C.random_circuit(10, 120, 5), 1, 1, 6),
]


@pytest.mark.parametrize("maker,B,n,cap", CAPPED_CASES)
@pytest.mark.parametrize("precision", [0, 1])
def test_capped_contraction(maker, B, n, cap, precision):
    """A cap below every order's peak: the planner contracts the bitstrings in smaller passes
    and/or slices indices (each slice contracted, the slices' amplitudes summed in FP64).
    Both are exact, so the bar is the same as for an uncapped plan; the largest intermediate
    obeys the cap.  n < B leaves padded bitstrings in the last pass."""
    from oracle.statevector import simulate_state
    c = maker()
    psi = simulate_state(c)
    xs = C.random_bitstrings(c.n_qubits, n, 4000 + cap)
    got, st = _amps(c, xs, B, precision, max_log2=cap)
    assert st["net_max_log2"] <= cap
    assert st["net_sliced"] > 0 or (1 << st["net_batch_log2"]) < B
    assert _rel(got, psi[xs.astype(np.int64)]) <= TOL


@pytest.mark.parametrize("cap", [14, 10])
def test_capped_grid_5x5(cap):
    """25 qubits, 16 bitstrings per call with 13 passed: cap 2^14 takes passes of 2 bitstrings
    (the last one padded), cap 2^10 passes of one bitstring with 4 sliced indices; against the
    oracle's FP64 sweep, and the same amplitudes as the uncapped plan."""
    from oracle.tn import contract_amplitude_sweep
    c = C.grid(5, 5, 10, 7)
    xs = C.random_bitstrings(25, 13, 4100)
    got, st = _amps(c, xs, 16, 1, max_log2=cap)
    assert st["net_max_log2"] <= cap and st["net_batch_log2"] < 4
    assert (st["net_sliced"] > 0) == (cap == 10)
    ref = np.array([contract_amplitude_sweep(c, int(x)) for x in xs[:4]])
    assert _rel(got[:4], ref) <= TOL
    whole, st0 = _amps(c, xs, 16, 1)
    assert st0["net_sliced"] == 0 and st0["net_batch_log2"] == 4
    assert _rel(got, whole) <= TOL


@pytest.mark.parametrize("n,k", [(2, 2), (8, 14), (14, 8), (20, 14)])
def test_fig31_amplitude_mode(n, k):
    """Fig. 3.1 circuits in amplitude mode (network contraction, 64 bitstrings per call,
    3xTF32 merges) against the FP64 state vector."""
    from oracle.statevector import simulate_state
    c = C.paper_fig31(n, k, 6100 + n + k)
    psi = simulate_state(c)
    xs = C.random_bitstrings(n, 64, 6200 + n + k)
    got, _ = _amps(c, xs, 64, 1)
    assert _rel(got, psi[xs.astype(np.int64)]) <= TOL


def test_fig31_amplitude_mode_28_qubits():
    """n = 28, k = 8 in the bench's launch configuration (64 bitstrings per call, 3xTF32):
    sampled amplitudes against the oracle's FP64 greedy network contraction."""
    from oracle.tn import contract_amplitude
    c = C.paper_fig31(28, 8, 6136)
    xs = C.random_bitstrings(28, 64, 6236)
    got, st = _amps(c, xs, 64, 1)
    assert st["net_max_log2"] <= 28
    ref = np.array([contract_amplitude(c, int(x)) for x in xs[:4]])
    assert _rel(got[:4], ref) <= TOL


@pytest.mark.parametrize("maker,B", [(lambda: C.grid(4, 5, 10, 81), 64), (lambda: C.paper_fig31(20, 8, 82), 64),
                                     (lambda: C.random_circuit(16, 200, 83), 16)])
def test_adaptive_order_search_plans(maker, B):
    """Orders from the adaptive search (order_search = 1, the cross-entropy hyper-optimiser) run on
    the GPU and give the same amplitudes as the state vector."""
    from oracle.statevector import simulate_state
    c = maker()
    psi = simulate_state(c)
    xs = C.random_bitstrings(c.n_qubits, B, 84)
    got, st = _amps(c, xs, B, 1, order_search=1)
    assert st["net_merges"] > 0
    assert _rel(got, psi[xs.astype(np.int64)]) <= TOL
