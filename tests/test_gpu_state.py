"""Parity of the CUDA contraction path with the FP64 oracle (GPU).

Bar (complex64 states and amplitude vectors): relative L2 error <= 1e-5 against the
oracle's complex128 result; expectations |E - E_ref| <= 1e-4 max(1, |E_ref|).
"""
import numpy as np
import pytest

from paper_2108_06831_gb300 import circuits as C

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

STATE_TOL = 1e-5


def _tn():
    from paper_2108_06831_gb300 import tn
    return tn


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def gpu_state(circ, params=None, batch=1, tile=0, specialize=True):
    tn = _tn()
    ctr = tn.Contractor(circ, target=tn.TARGET_STATE, batch=batch, tile_qubits=tile, specialize=specialize)
    p = None if params is None else torch.as_tensor(np.asarray(params, dtype=np.float64).reshape(batch, -1),
                                                    device="cuda").contiguous()
    out = ctr.state(p)
    torch.cuda.synchronize()
    assert tn.sync_status() == tn.OK
    return out.cpu().numpy()


@pytest.mark.parametrize("specialize", [True, False])
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 8, 9, 11, 12])
def test_random_circuits_small(n, specialize):
    """Every gate kind, both the plan-specialised kernels and the interpreting kernel."""
    from oracle.statevector import simulate_state
    for seed in range(3):
        c = C.random_circuit(n, 12 * n + 5, 100 * n + seed)
        c.init_basis = (seed * 7919) % (1 << n)
        ref = simulate_state(c)
        got = gpu_state(c, specialize=specialize)[0]
        assert rel_l2(got, ref) <= STATE_TOL, (n, seed)


@pytest.mark.parametrize("specialize", [True, False])
@pytest.mark.parametrize("n,tile", [(13, 6), (14, 6), (15, 8), (16, 10), (17, 12), (18, 13), (16, 7)])
def test_random_circuits_multipass(n, tile, specialize):
    """Several tiles and passes; tile sizes from the smallest allowed upwards."""
    from oracle.statevector import simulate_state
    c = C.random_circuit(n, 10 * n, 7 * n + tile)
    c.init_basis = (n * 104729) % (1 << n)
    ref = simulate_state(c)
    got = gpu_state(c, tile=tile, specialize=specialize)[0]
    assert rel_l2(got, ref) <= STATE_TOL


def test_cfg1_brickwork_10q_depth8():
    from oracle.statevector import simulate_state
    c, _ = C.brickwork(10, 8, 1000)
    ref = simulate_state(c)
    got = gpu_state(c)[0]
    assert rel_l2(got, ref) <= STATE_TOL


@pytest.mark.parametrize("maker", [
    lambda: C.brickwork(16, 12, 5)[0],
    lambda: C.qft(16, 12345),
    lambda: C.paper_fig31(16, 6, 3),
    lambda: C.grid(4, 4, 10, 8),
    lambda: C.ghz(14),
])
def test_workload_families(maker):
    from oracle.statevector import simulate_state
    c = maker()
    ref = simulate_state(c)
    for tile in (0, 9):
        got = gpu_state(c, tile=tile)[0]
        assert rel_l2(got, ref) <= STATE_TOL


def test_parameterized_batch():
    """Per-batch parameters: every batch element matches the oracle with its own angles."""
    from oracle.statevector import simulate_state
    c, p0 = C.brickwork(12, 6, 77, parameterized=True)
    rng = np.random.default_rng(5)
    params = np.stack([p0] + [rng.uniform(0, 2 * np.pi, size=p0.shape) for _ in range(4)])
    got = gpu_state(c, params, batch=5)
    for b in range(5):
        assert rel_l2(got[b], simulate_state(c, params[b])) <= STATE_TOL


def test_cfg2_full_size_sampled():
    """24-qubit brickwork, depth 20, in the bench's launch configuration (parameterised
    U3 angles, plan-specialised kernels): sampled amplitudes against the oracle's network
    contraction, plus the norm."""
    from oracle.tn import contract_amplitude
    c, params = C.brickwork(24, 20, 1001, parameterized=True)
    got = gpu_state(c, params)[0]
    c, _ = C.brickwork(24, 20, 1001)
    assert abs(np.linalg.norm(got.astype(np.complex128)) - 1.0) < 1e-5
    xs = C.random_bitstrings(24, 10, 4242)
    ref = np.array([contract_amplitude(c, int(x)) for x in xs])
    assert rel_l2(got[xs.astype(np.int64)], ref) <= STATE_TOL


def test_amplitudes_gather():
    from oracle.statevector import simulate_state
    tn = _tn()
    c = C.grid(4, 4, 8, 11)
    ref = simulate_state(c)
    ctr = tn.Contractor(c, target=tn.TARGET_AMPLITUDES)
    xs = C.random_bitstrings(16, 300, 9)
    got = ctr.amplitudes(torch.as_tensor(xs.astype(np.int64), device="cuda")).cpu().numpy()[0]
    assert rel_l2(got, ref[xs.astype(np.int64)]) <= STATE_TOL
    # empty batch of bitstrings is a no-op
    ctr.amplitudes(torch.empty(0, dtype=torch.int64, device="cuda"))
    torch.cuda.synchronize()


def test_empty_circuit_and_basis():
    c = C.Circuit(7, [], init_basis=93)
    got = gpu_state(c)[0]
    ref = np.zeros(128, dtype=np.complex128)
    ref[93] = 1
    assert np.abs(got - ref).max() == 0


def test_invalid_arguments_rejected():
    tn = _tn()
    with pytest.raises(tn.TnError):
        tn.CircuitHandle(C.Circuit(3, [C.Gate("H", (3,))]))
    with pytest.raises(tn.TnError):
        tn.CircuitHandle(C.Circuit(3, [C.Gate("CZ", (1, 1))]))
    with pytest.raises(tn.TnError):
        tn.CircuitHandle(C.Circuit(3, [], init_basis=8))
    ctr = tn.Contractor(C.brickwork(6, 2, 1, parameterized=True)[0])
    with pytest.raises(tn.TnError):
        ctr.state(None)  # parameterised circuit without parameters


@pytest.mark.parametrize("n,k", [(2, 14), (6, 2), (14, 8), (20, 14)])
def test_fig31_sweep_points(n, k):
    """Points of the paper-shaped sweep (Fig. 3.1 circuits) against the FP64 oracle."""
    from oracle.statevector import simulate_state
    from paper_2108_06831_gb300 import tn
    c = C.paper_fig31(n, k, 6000 + n + k)
    ctr = tn.Contractor(c)
    out = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    tn.contract_state(ctr.plan, None, out, ctr.workspace)
    torch.cuda.synchronize()
    assert tn.sync_status() == tn.OK
    ref = simulate_state(c)
    got = out.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5


def test_fig31_largest_point_against_stored_oracle():
    """n = 28, k = 14 (2 GiB state), the largest point of the Fig. 3.1 grid, in the bench's
    launch configuration: 8 amplitudes against the oracle's FP64 greedy network contraction
    (stored: ~1 min and 9 GB of host memory per amplitude), plus the norm."""
    import os
    from paper_2108_06831_gb300 import tn
    c = C.paper_fig31(28, 14, 6042)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_fig31_n28_k14_s6042.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    xs = np.array([int(r[0]) for r in rows], dtype=np.int64)
    ref = np.array([complex(float(r[1]), float(r[2])) for r in rows])
    assert np.array_equal(xs.astype(np.uint64), C.random_bitstrings(28, 8, 6242))
    a = tn.Contractor(c)
    x = torch.empty(1 << 28, dtype=torch.complex64, device="cuda")
    tn.contract_state(a.plan, None, x, a.workspace)
    torch.cuda.synchronize()
    assert tn.sync_status() == tn.OK
    nx = torch.linalg.vector_norm(x.to(torch.complex128)).item()
    assert abs(nx - 1.0) <= 1e-5
    got = x[torch.as_tensor(xs, device="cuda")].cpu().numpy()
    # amplitudes of a 2^28-entry state are ~2^-14: compare them against the state's RMS scale
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= 1e-5, err


def test_max_size_32_qubits_closed_form():
    """32 qubits (a 32 GiB complex64 state): U3 on every qubit, then CZ on every neighbour pair.
    Every amplitude has a closed form, amp(x) = prod_q (U3_q|0>)[x_q] * (-1)^(sum_q x_q x_{q+1}),
    evaluated in FP64 on 4096 sampled indices."""
    from oracle.gates import matrix
    from paper_2108_06831_gb300 import tn
    n = 32
    rng = np.random.default_rng(3232)
    angles = rng.uniform(0.0, 2.0 * np.pi, size=(n, 3))
    gates = [C.Gate("U3", (q,), tuple(float(a) for a in angles[q])) for q in range(n)]
    gates += [C.Gate("CZ", (q, q + 1)) for q in range(n - 1)]
    c = C.Circuit(n, gates)
    ctr = tn.Contractor(c)
    out = torch.empty((1, 1 << n), dtype=torch.complex64, device="cuda")
    tn.contract_state(ctr.plan, None, out, ctr.workspace)
    torch.cuda.synchronize()
    assert tn.sync_status() == tn.OK
    xs = rng.integers(0, 1 << n, size=4096, dtype=np.int64)
    got = out[0, torch.as_tensor(xs, device="cuda")].cpu().numpy().astype(np.complex128)
    col = np.array([matrix("U3", tuple(angles[q]))[:, 0] for q in range(n)])  # U3_q |0>
    bits = (xs[:, None] >> (n - 1 - np.arange(n))[None, :]) & 1  # bit of qubit q (MSB first)
    ref = np.prod(col[np.arange(n)[None, :], bits], axis=1)
    ref = ref * (-1.0) ** np.sum(bits[:, :-1] * bits[:, 1:], axis=1)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= STATE_TOL


def test_tile_autotuner_single_plan():
    """tn_plan_contraction_tuned: the circuit planned at each candidate tile size, each plan's
    contraction timed, the fastest returned; its tile is a candidate and its state matches the
    oracle (parameterised circuit, batch of 2)."""
    from oracle.statevector import simulate_state
    tn = _tn()
    c, p0 = C.brickwork(16, 10, 91, parameterized=True)
    params = np.stack([p0, np.random.default_rng(92).uniform(0, 2 * np.pi, size=p0.shape)])
    ctr = tn.Contractor(c, batch=2, tune={"candidates": (8, 10, 12), "reps": 2})
    assert ctr.plan.tuned_tile in (8, 10, 12)
    assert ctr.plan.stats()["tile_qubits"] == ctr.plan.tuned_tile
    got = ctr.state(torch.as_tensor(params, device="cuda")).cpu().numpy()
    torch.cuda.synchronize()
    assert tn.sync_status() == tn.OK
    for b in range(2):
        assert rel_l2(got[b], simulate_state(c, params[b])) <= STATE_TOL
    with pytest.raises(tn.TnError):  # tile_qubits is the tuner's choice
        tn.Plan(tn.CircuitHandle(c), tile_qubits=10, tune={})
