"""Persistent batched executor (many circuits, one launch) against the FP64 oracle (GPU)."""
import numpy as np
import pytest

from paper_2108_06831_gb300 import circuits as C

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-5


def _mix():
    rng = np.random.default_rng(11)
    out = []
    for i in range(20):
        n = int(rng.integers(6, 17))
        if i % 3 == 0:
            out.append(C.qft(n, int(rng.integers(0, 1 << n))))
        elif i % 3 == 1:
            out.append(C.brickwork(n, int(rng.integers(2, 12)), 300 + i)[0])
        else:
            c = C.random_circuit(n, 6 * n, 500 + i)
            c.init_basis = int(rng.integers(0, 1 << n))
            out.append(c)
    return out


def _run_batch(circs, tile=0):
    from paper_2108_06831_gb300 import tn
    handles = [tn.CircuitHandle(c) for c in circs]
    plans = [tn.Plan(h, tile_qubits=min(tile, c.n_qubits) if tile else 0, specialize=False)
             for h, c in zip(handles, circs)]
    b = tn.Batch(plans)
    states = torch.full((b.state_elems,), complex(float("nan"), 0), dtype=torch.complex64, device="cuda")
    ws = torch.empty(b.workspace_bytes, dtype=torch.uint8, device="cuda")
    return tn, b, plans, handles, states, ws


def test_batch_matches_oracle():
    from oracle.statevector import simulate_state
    circs = _mix()
    tn, b, plans, handles, states, ws = _run_batch(circs)
    tn.batch_run(b, states, ws)
    torch.cuda.synchronize()
    assert tn.sync_status() == tn.OK
    got = states.cpu().numpy()
    for c, off in zip(circs, b.offsets):
        ref = simulate_state(c)
        s = got[off:off + (1 << c.n_qubits)]
        assert np.linalg.norm(s - ref) / np.linalg.norm(ref) <= TOL, c.name


def test_batch_small_tiles_many_passes_and_graph_replay():
    """8-qubit tiles force multi-pass circuits; the launch is captured in a CUDA graph and replayed."""
    from oracle.statevector import simulate_state
    circs = _mix()[:10]
    tn, b, plans, handles, states, ws = _run_batch(circs, tile=8)
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    tn.batch_run(b, states, ws)  # first call outside capture (sets kernel attributes)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            tn.batch_run(b, states, ws)
    for _ in range(2):
        states.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert tn.sync_status() == tn.OK
        got = states.cpu().numpy()
        for c, off in zip(circs, b.offsets):
            ref = simulate_state(c)
            s = got[off:off + (1 << c.n_qubits)]
            assert np.linalg.norm(s - ref) / np.linalg.norm(ref) <= TOL, c.name


def test_batch_with_parameterised_circuits():
    """Parameterised circuits in the persistent launch: every circuit's gate table is built in the
    run from its own parameters (one kernel for all), fixed-angle circuits beside them; the run is
    captured in a CUDA graph and replayed with new parameter values written into the same buffer."""
    from oracle.statevector import simulate_state
    from paper_2108_06831_gb300 import tn
    rng = np.random.default_rng(12)
    circs, params = [], []
    for i in range(12):
        n = int(rng.integers(6, 17))
        if i % 3 == 2:
            circs.append(C.qft(n, int(rng.integers(0, 1 << n))))
            params.append(np.zeros(0))
        elif i % 3 == 1:
            c = C.hea(n, 3)
            circs.append(c)
            params.append(C.hea_params(c.n_params, 1, 100 + i)[0])
        else:
            c, p = C.brickwork(n, int(rng.integers(2, 10)), 600 + i, parameterized=True)
            circs.append(c)
            params.append(p)
    plans = [tn.Plan(tn.CircuitHandle(c), tile_qubits=min(8 + (i % 4), c.n_qubits) if c.n_qubits >= 6 else 0,
                     specialize=False) for i, c in enumerate(circs)]
    b = tn.Batch(plans)
    assert b.n_params == sum(len(p) for p in params)
    flat = np.zeros(max(b.n_params, 1))
    for p, off in zip(params, b.param_offsets):
        flat[off:off + len(p)] = p
    d_params = torch.as_tensor(flat, device="cuda")
    states = torch.full((b.state_elems,), complex(float("nan"), 0), dtype=torch.complex64, device="cuda")
    ws = torch.empty(b.workspace_bytes, dtype=torch.uint8, device="cuda")
    with pytest.raises(tn.TnError):  # parameters are required
        tn.batch_run(b, states, ws)

    def check():
        got = states.cpu().numpy()
        for c, p, off in zip(circs, params, b.offsets):
            ref = simulate_state(c, p if len(p) else None)
            s_ = got[off:off + (1 << c.n_qubits)]
            assert np.linalg.norm(s_ - ref) / np.linalg.norm(ref) <= TOL, c.name
    tn.batch_run(b, states, ws, params=d_params)
    torch.cuda.synchronize()
    assert tn.sync_status() == tn.OK
    check()
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            tn.batch_run(b, states, ws, params=d_params)
    for rep in range(2):
        params = [rng.uniform(-np.pi, np.pi, size=len(p)) for p in params]
        for p, off in zip(params, b.param_offsets):
            flat[off:off + len(p)] = p
        d_params.copy_(torch.as_tensor(flat))
        states.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        assert tn.sync_status() == tn.OK
        check()


def test_batch_rejects_batched_plans():
    from paper_2108_06831_gb300 import tn
    c, _ = C.brickwork(8, 2, 1, parameterized=True)
    p = tn.Plan(tn.CircuitHandle(c), batch=2, specialize=False)
    with pytest.raises(tn.TnError) as e:
        tn.Batch([p])
    assert e.value.status == tn.ERR_UNSUPPORTED


def test_tuned_batch_matches_oracle():
    """The tile autotuner: every chosen tile is a candidate (or the circuit's own width), the
    batch it returns owns its plans, and its states match the oracle."""
    from oracle.statevector import simulate_state
    from paper_2108_06831_gb300 import tn
    circs = _mix()[:12]
    handles = [tn.CircuitHandle(c) for c in circs]
    b = tn.Batch.tuned(handles, candidates=(6, 8, 10, 12), reps=1)
    for c, t in zip(circs, b.tiles):
        assert t in (6, 8, 10, 12) or t == c.n_qubits
        assert t <= min(c.n_qubits, 12)
    del handles  # the batch must not depend on the circuit handles
    states = torch.full((b.state_elems,), complex(float("nan"), 0), dtype=torch.complex64, device="cuda")
    ws = torch.empty(b.workspace_bytes, dtype=torch.uint8, device="cuda")
    tn.batch_run(b, states, ws)
    torch.cuda.synchronize()
    assert tn.sync_status() == tn.OK
    got = states.cpu().numpy()
    for c, off in zip(circs, b.offsets):
        ref = simulate_state(c)
        s = got[off:off + (1 << c.n_qubits)]
        assert np.linalg.norm(s - ref) / np.linalg.norm(ref) <= TOL, c.name


def test_tuned_batch_rejects_bad_options():
    from paper_2108_06831_gb300 import tn
    h = [tn.CircuitHandle(C.brickwork(8, 3, 1)[0])]
    with pytest.raises(tn.TnError):
        tn.Batch.tuned(h, candidates=(5,))
    with pytest.raises(tn.TnError):
        tn.Batch.tuned(h, candidates=(13,))
    hp = [tn.CircuitHandle(C.brickwork(8, 3, 1, parameterized=True)[0])]
    with pytest.raises(tn.TnError):
        tn.Batch.tuned(hp)


# The 512-circuit serving mix at its own sizes: a subset of serving_mix(512, 5000) that reaches
# 22 qubits and depth 28-30 (both halves, brickwork and QFT, including the largest circuit of
# each), through the tile autotuner and one launch, every state against the oracle.
SERVING_SUBSET = [i * 31 for i in range(16)] + [494, 441]


def test_serving_mix_subset_tuned_matches_oracle():
    import multiprocessing as mp
    import os
    from oracle.statevector import simulate_state
    from paper_2108_06831_gb300 import tn
    mix = C.serving_mix(512, 5000)
    circs = [mix[i] for i in SERVING_SUBSET]
    assert max(c.n_qubits for c in circs) == 22
    # the oracle runs in spawned worker processes while the GPU works
    ctx = mp.get_context("spawn")
    with ctx.Pool(max(1, min(8, os.cpu_count() or 1))) as pool:
        pending = pool.map_async(simulate_state, circs, chunksize=1)
        handles = [tn.CircuitHandle(c) for c in circs]
        b = tn.Batch.tuned(handles, reps=1)
        states = torch.full((b.state_elems,), complex(float("nan"), 0), dtype=torch.complex64, device="cuda")
        ws = torch.empty(b.workspace_bytes, dtype=torch.uint8, device="cuda")
        tn.batch_run(b, states, ws)
        torch.cuda.synchronize()
        assert tn.sync_status() == tn.OK
        got = states.cpu().numpy()
        refs = pending.get(timeout=1800)
    for c, off, ref in zip(circs, b.offsets, refs):
        s = got[off:off + (1 << c.n_qubits)]
        assert np.linalg.norm(s - ref) / np.linalg.norm(ref) <= TOL, c.name


def test_batch_wide_circuits_on_side_streams():
    """Circuits of 19 qubits and more with plan-specialised kernels run those kernels on the batch's
    side streams, beside the persistent launch of the small ones: six wide circuits on four streams
    (fixed angles, a QFT, and one parameterised plan used twice with different parameters), every
    state against the oracle, directly and as a replayed CUDA graph with new parameter values."""
    from oracle.statevector import simulate_state
    from paper_2108_06831_gb300 import tn
    rng = np.random.default_rng(21)
    wide_fixed = [C.brickwork(19, 5, 700)[0], C.brickwork(20, 4, 701)[0], C.qft(19, int(rng.integers(0, 1 << 19))),
                  C.brickwork(21, 3, 702)[0]]
    cp, pp = C.brickwork(19, 4, 703, parameterized=True)
    small = [C.brickwork(10, 6, 704)[0], C.qft(14, 12345), C.brickwork(16, 5, 705)[0]]
    hp = tn.CircuitHandle(cp)
    p_wide = tn.Plan(hp)  # one parameterised plan, two entries of the batch
    plans = [tn.Plan(tn.CircuitHandle(c)) for c in wide_fixed] + [p_wide, p_wide] + \
            [tn.Plan(tn.CircuitHandle(c), specialize=False) for c in small]
    assert all(p.stats()["specialized"] for p in plans[:6])
    circs = wide_fixed + [cp, cp] + small
    b = tn.Batch(plans)
    params = [np.zeros(0)] * 4 + [pp, rng.uniform(-np.pi, np.pi, size=len(pp))] + [np.zeros(0)] * 3
    flat = np.zeros(max(b.n_params, 1))
    d_params = torch.empty(len(flat), dtype=torch.float64, device="cuda")

    def load(ps):
        for p, off in zip(ps, b.param_offsets):
            flat[off:off + len(p)] = p
        d_params.copy_(torch.as_tensor(flat))

    states = torch.full((b.state_elems,), complex(float("nan"), 0), dtype=torch.complex64, device="cuda")
    ws = torch.empty(b.workspace_bytes, dtype=torch.uint8, device="cuda")

    def check(ps):
        got = states.cpu().numpy()
        for c, p, off in zip(circs, ps, b.offsets):
            ref = simulate_state(c, p if len(p) else None)
            s_ = got[off:off + (1 << c.n_qubits)]
            assert np.linalg.norm(s_ - ref) / np.linalg.norm(ref) <= TOL, c.name
    load(params)
    tn.batch_run(b, states, ws, params=d_params)
    torch.cuda.synchronize()
    assert tn.sync_status() == tn.OK
    check(params)
    stream = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            tn.batch_run(b, states, ws, params=d_params)
    params = params[:4] + [rng.uniform(-np.pi, np.pi, size=len(pp)) for _ in range(2)] + params[6:]
    load(params)
    states.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    assert tn.sync_status() == tn.OK
    check(params)
