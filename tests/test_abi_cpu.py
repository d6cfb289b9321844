"""Host-side checks of the C ABI that need no GPU: the library loads, exports every symbol
include/tn.h declares, validates arguments and plans (host-only) without touching a device."""
import os
import re

import numpy as np
import pytest

from paper_2108_06831_gb300 import circuits as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _tn():
    from paper_2108_06831_gb300 import _build
    if not os.path.exists(os.path.join(ROOT, "paper_2108_06831_gb300", "libtnq.so")):
        _build.build()
    from paper_2108_06831_gb300 import tn
    return tn


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tn_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol():
    tn = _tn()
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(tn._lib, name), name
    assert set(names) <= set(tn.EXPORTED)


def test_version_and_errors():
    tn = _tn()
    assert "sm_103a" in tn.version()
    with pytest.raises(tn.TnError) as e:
        tn.CircuitHandle(C.Circuit(0, []))
    assert "n_qubits" in str(e.value)
    with pytest.raises(tn.TnError):
        tn.CircuitHandle(C.Circuit(4, [C.Gate("RX", (0,), (), -5)]))
    with pytest.raises(tn.TnError):
        tn.CircuitHandle(C.Circuit(4, [C.Gate("H", (0,), (), 0)]))


def test_host_only_plans():
    tn = _tn()
    c, _ = C.brickwork(24, 20, 1001)
    ch = tn.CircuitHandle(c)
    n_u3 = sum(1 for g in c.gates if g.kind == "U3")
    n_cz = sum(1 for g in c.gates if g.kind == "CZ")
    for T in (8, 10, 12, 13):
        s = tn.Plan(ch, tile_qubits=T, host_only=True, fuse=False).stats()
        # every U3 becomes V = RY P (the pushed phase P(phi) merges into the qubit's next V),
        # so the plan holds every gate once plus one final phase gate per qubit
        assert s["n_ops"] == len(c.gates) + 24 and s["n_fused"] == 0
        assert s["tile_qubits"] == T and s["reg_qubits"] == 4
        assert s["n_passes"] >= 2
        # flops as executed: V costs 10 real flops per amplitude, a final phase 3, CZ none; the
        # first pass computes only the tile holding |x0> (the rest of a basis state stays zero)
        full = (10.0 * n_u3 + 3.0 * 24) * (1 << 24)
        assert 0.8 * full < s["flops"] < full
        # precontracted: each even-layer CZ pair with the U3s of its two qubits in that layer and
        # the next becomes one dense 4x4 (12 per two layers); the odd-layer CZs stay
        f = tn.Plan(ch, tile_qubits=T, host_only=True).stats()
        assert f["n_fused"] == 12 * 10
        assert f["n_ops"] == 120 + (n_cz - 120)
        assert 0.8 * 30.0 * 120 * (1 << 24) < f["flops"] < 30.0 * 120 * (1 << 24)
        assert f["n_phases"] < s["n_phases"]
    small = tn.Plan(tn.CircuitHandle(C.brickwork(10, 8, 1000)[0]), host_only=True).stats()
    assert small["tile_qubits"] == 10 and small["n_passes"] <= 2  # one tile; code budget may split it


def test_plan_option_validation():
    tn = _tn()
    ch = tn.CircuitHandle(C.ghz(5))
    with pytest.raises(tn.TnError):
        tn.Plan(ch, tile_qubits=5, host_only=True)
    with pytest.raises(tn.TnError):
        tn.Plan(ch, tile_qubits=20, host_only=True)
    with pytest.raises(tn.TnError):
        tn.Plan(ch, batch=-1, host_only=True)
    p = tn.Plan(ch, target=tn.TARGET_EXPECTATION, batch=4, host_only=True)
    assert p.workspace_bytes >= 2 * 4 * 8 * 32


def test_block_plans_host_only():
    """Uniform square blocks (TN_PLAN_BLOCKS): the 24-qubit brickwork cut into blocks of 6 and 7
    qubits (windows at alternating offsets take their light cones), one GEMM launch per block
    after the first, and the options the mode rejects."""
    tn = _tn()
    ch = tn.CircuitHandle(C.brickwork(24, 20, 1001, parameterized=True)[0])
    for k, most in ((6, 30), (7, 26)):
        s = tn.Plan(ch, host_only=True, block_qubits=k, precision=tn.PREC_3XTF32).stats()
        assert s["tile_qubits"] == k and 2 <= s["n_fused"] <= most
        assert s["n_passes"] == s["n_fused"] - 1
        assert s["flops"] == pytest.approx(8.0 * (1 << (24 - k)) * (1 << k) ** 2 * s["n_passes"])
    small = tn.CircuitHandle(C.brickwork(12, 4, 1)[0])
    with pytest.raises(tn.TnError):  # fewer than k + 7 qubits
        tn.Plan(small, host_only=True, block_qubits=6)
    with pytest.raises(tn.TnError):
        tn.Plan(ch, host_only=True, block_qubits=5)
    with pytest.raises(tn.TnError):
        tn.Plan(ch, host_only=True, block_qubits=6, batch=3)
    with pytest.raises(tn.TnError):
        tn.Plan(ch, host_only=True, block_qubits=6, target=tn.TARGET_EXPECTATION)


def test_network_plan_6x6_grid_host_only():
    """Network lowering for the 6x6 depth-12 grid (64 bitstrings per call), without a device:
    every merge is either folded at plan time or launched, the largest intermediate stays within
    2^27 entries, and the dense merges (and only fitting shapes) go to the tensor cores."""
    from paper_2108_06831_gb300 import tn
    ch = tn.CircuitHandle(C.grid(6, 6, 12, 3003))
    stats = {}
    for prec in (tn.PREC_FP32, tn.PREC_3XTF32, tn.PREC_SPLIT_BF16):
        p = tn.Plan(ch, target=tn.TARGET_AMPLITUDES, host_only=True, network_bitstrings=64, precision=prec)
        stats[prec] = s = p.stats()
        assert s["net_max_log2"] <= 27
        assert s["net_merges"] + s["net_folded_merges"] == stats[tn.PREC_FP32]["net_merges"] + \
            stats[tn.PREC_FP32]["net_folded_merges"]
        assert 0 < s["net_merges"] < 200 and s["net_folded_merges"] > 300
        assert p.workspace_bytes < 4 << 30
    assert stats[tn.PREC_FP32]["net_tensor_merges"] == 0
    assert stats[tn.PREC_3XTF32]["net_tensor_merges"] >= 8
    assert stats[tn.PREC_SPLIT_BF16]["net_tensor_merges"] >= 8
    # the planner is deterministic: the same circuit gives the same plan
    again = tn.Plan(ch, target=tn.TARGET_AMPLITUDES, host_only=True, network_bitstrings=64,
                    precision=tn.PREC_3XTF32).stats()
    assert again == stats[tn.PREC_3XTF32]


def test_network_plan_rejects_bad_options():
    from paper_2108_06831_gb300 import tn
    ch = tn.CircuitHandle(C.grid(3, 3, 4, 1))
    with pytest.raises(tn.TnError):  # bitstring batch must be a power of two
        tn.Plan(ch, target=tn.TARGET_AMPLITUDES, host_only=True, network_bitstrings=48)
    chp = tn.CircuitHandle(C.brickwork(6, 2, 1, parameterized=True)[0])
    with pytest.raises(tn.TnError):  # network plans take fixed angles
        tn.Plan(chp, target=tn.TARGET_AMPLITUDES, host_only=True, network_bitstrings=16)


def test_network_plan_capped_host_only():
    """A cap below every contraction order's peak: bitstrings are contracted in smaller passes
    and/or indices sliced until the largest intermediate fits; a cap that no slicing within
    2^16 slices reaches is rejected; the default cap needs neither."""
    from paper_2108_06831_gb300 import tn
    ch = tn.CircuitHandle(C.grid(5, 5, 10, 7))
    kw = dict(target=tn.TARGET_AMPLITUDES, host_only=True, network_bitstrings=16, precision=tn.PREC_3XTF32)
    whole = tn.Plan(ch, **kw).stats()
    assert whole["net_sliced"] == 0 and whole["net_batch_log2"] == 4
    prev_batch, prev_sliced = 4, 0
    for cap in (16, 14, 12, 10, 8, 6):
        s = tn.Plan(ch, max_intermediate_log2=cap, **kw).stats()
        assert s["net_max_log2"] <= cap and s["net_sliced"] <= 16
        assert s["net_batch_log2"] < 4 or s["net_sliced"] > 0
        # tighter caps never take larger passes or fewer slices here
        assert s["net_batch_log2"] <= prev_batch and s["net_sliced"] >= prev_sliced
        prev_batch, prev_sliced = s["net_batch_log2"], s["net_sliced"]
    assert prev_sliced > 0 and prev_batch == 0
    with pytest.raises(tn.TnError) as e:
        tn.Plan(ch, max_intermediate_log2=4, **kw)
    assert e.value.status == tn.ERR_UNSUPPORTED


def test_network_plan_routes_host_only():
    """The capped plans the GPU parity tests run take every route of the planner: slicing only,
    smaller bitstring passes only, and both."""
    from paper_2108_06831_gb300 import tn
    cases = [(C.qft(8, 77), 4, 5), (C.brickwork(12, 10, 3)[0], 16, 8), (C.grid(3, 4, 8, 2), 4, 5),
             (C.random_circuit(10, 120, 5), 4, 7), (C.grid(3, 4, 8, 2), 4, 4), (C.random_circuit(10, 120, 5), 1, 6)]
    routes = set()
    for c, B, cap in cases:
        s = tn.Plan(tn.CircuitHandle(c), target=tn.TARGET_AMPLITUDES, host_only=True, network_bitstrings=B,
                    max_intermediate_log2=cap).stats()
        assert s["net_max_log2"] <= cap
        routes.add((s["net_sliced"] > 0, (1 << s["net_batch_log2"]) < B))
    assert {(True, False), (False, True), (True, True)} <= routes


def test_network_order_search_never_worse_than_greedy():
    """The randomised search includes the deterministic greedy at every bitstring pass size, so
    its planned cost is never above the greedy's alone (order_trials = 1); other trial counts
    outside 4..4096 are rejected."""
    from paper_2108_06831_gb300 import tn
    for c in (C.paper_fig31(12, 6, 1), C.grid(4, 4, 8, 2), C.qft(9, 5), C.random_circuit(10, 80, 3)):
        ch = tn.CircuitHandle(c)
        kw = dict(target=tn.TARGET_AMPLITUDES, host_only=True, network_bitstrings=16)
        greedy = tn.Plan(ch, order_trials=1, **kw).stats()["net_cost"]
        search = tn.Plan(ch, **kw).stats()["net_cost"]
        few = tn.Plan(ch, order_trials=8, **kw).stats()["net_cost"]
        assert search <= greedy and few <= greedy
    for bad in (2, 3, 5000, -1):
        with pytest.raises(tn.TnError):
            tn.Plan(tn.CircuitHandle(C.ghz(4)), order_trials=bad, **kw)


def test_q428_plan_host_only():
    """A fixed-point plan: one launch per gate, each reading and writing every amplitude (int32
    pairs) after the basis state is written; fixed-angle circuits with batch 1 only, and not
    together with network planning."""
    from paper_2108_06831_gb300 import tn
    c = C.brickwork(12, 6, 4)[0]
    s = tn.Plan(tn.CircuitHandle(c), q428=True, host_only=True).stats()
    assert s["n_passes"] == len(c.gates)
    assert s["hbm_bytes"] == 8.0 * (1 << 12) * (1 + 2 * len(c.gates))
    with pytest.raises(tn.TnError):
        tn.Plan(tn.CircuitHandle(C.brickwork(6, 2, 1, parameterized=True)[0]), q428=True, host_only=True)
    with pytest.raises(tn.TnError):
        tn.Plan(tn.CircuitHandle(c), q428=True, batch=2, host_only=True)
    with pytest.raises(tn.TnError):
        tn.Plan(tn.CircuitHandle(c), q428=True, network_bitstrings=4, target=tn.TARGET_AMPLITUDES, host_only=True)


def test_network_planner_invariants_random_circuits():
    """Over seeded random circuits, bitstring batches and caps: the largest intermediate obeys the
    cap; passes never hold more bitstrings than a call; at most 16 indices are sliced; the planned
    cost covers the algorithmic bytes (it adds launch costs to max(bytes, flops / 32)); the same
    inputs give the same plan; a larger search is never worse than the greedy alone."""
    from paper_2108_06831_gb300 import tn
    rng = np.random.default_rng(2024)
    for trial in range(12):
        n = int(rng.integers(4, 12))
        c = C.random_circuit(n, int(rng.integers(2 * n, 10 * n)), 5000 + trial)
        B = 1 << int(rng.integers(0, 5))
        cap = int(rng.choice([0, 6, 8, 10]))
        ch = tn.CircuitHandle(c)
        kw = dict(target=tn.TARGET_AMPLITUDES, host_only=True, network_bitstrings=B, max_intermediate_log2=cap)
        try:
            s = tn.Plan(ch, **kw).stats()
        except tn.TnError as e:  # a cap no slicing within 2^16 slices reaches
            assert e.status == tn.ERR_UNSUPPORTED and cap
            continue
        assert s["net_max_log2"] <= (cap or 28)
        assert (1 << s["net_batch_log2"]) <= B and 0 <= s["net_sliced"] <= 16
        assert s["net_cost"] >= s["net_bytes"] > 0
        assert tn.Plan(ch, **kw).stats() == s
        assert s["net_cost"] <= tn.Plan(ch, order_trials=1, **kw).stats()["net_cost"]


def test_network_adaptive_search():
    """order_search = 1 (the adaptive hyper-optimiser over the order generator): deterministic,
    never worse than the greedy alone, within the cap; other values are rejected."""
    from paper_2108_06831_gb300 import tn
    kw = dict(target=tn.TARGET_AMPLITUDES, host_only=True, network_bitstrings=16)
    for c, cap in ((C.paper_fig31(14, 8, 2), 0), (C.grid(4, 4, 8, 11), 9), (C.random_circuit(10, 90, 6), 0)):
        ch = tn.CircuitHandle(c)
        a = tn.Plan(ch, order_search=1, max_intermediate_log2=cap, **kw).stats()
        assert tn.Plan(ch, order_search=1, max_intermediate_log2=cap, **kw).stats() == a
        greedy = tn.Plan(ch, order_trials=1, max_intermediate_log2=cap, **kw).stats()
        assert a["net_cost"] <= greedy["net_cost"] and a["net_max_log2"] <= (cap or 28)
    with pytest.raises(tn.TnError):
        tn.Plan(tn.CircuitHandle(C.ghz(4)), order_search=2, **kw)


def test_sliced_network_plans_search_wider():
    """A network plan that had to slice is searched again with four times the orders and the cheaper
    plan by the order cost is kept: under a 2^20 cap the default plan costs no more than the plan of
    the 256-order search alone, and both fit the cap."""
    from paper_2108_06831_gb300 import tn
    ch = tn.CircuitHandle(C.grid(6, 6, 12, 3003))
    kw = dict(target=tn.TARGET_AMPLITUDES, host_only=True, network_bitstrings=64, precision=tn.PREC_3XTF32,
              max_intermediate_log2=20)
    narrow = tn.Plan(ch, order_trials=256, **kw).stats()
    default = tn.Plan(ch, **kw).stats()
    assert narrow["net_sliced"] > 0
    assert default["net_max_log2"] <= 20 and narrow["net_max_log2"] <= 20
    assert default["net_cost"] <= narrow["net_cost"]


def test_generated_kernels_compile_without_a_device(tmp_path, monkeypatch):
    """The plan-specialised kernels (forward passes with fused 4x4 blocks and constant tables, the
    adjoint passes with derivative dots) are generated and compiled by NVRTC for sm_103a on the host,
    without loading them: a code-generation error fails the plan here, before any GPU run."""
    from paper_2108_06831_gb300 import tn
    dump = tmp_path / "src"
    monkeypatch.setenv("TNQ_JIT_COMPILE_CHECK", "1")
    monkeypatch.setenv("TNQ_JIT_DUMP_DIR", str(dump))
    monkeypatch.setenv("TNQ_CACHE_DIR", str(tmp_path / "cache"))
    circ, _ = C.brickwork(16, 6, 5, parameterized=True)  # fused blocks (16 >= 14 qubits), first-pass skip
    tn.Plan(tn.CircuitHandle(circ), host_only=True)
    tn.Plan(tn.CircuitHandle(C.qft(15, 1234)), host_only=True)  # SWAPs as register exchanges
    tn.Plan(tn.CircuitHandle(C.hea(14, 2)), target=tn.TARGET_EXPECTATION, batch=4, host_only=True)
    srcs = [f.read_text() for f in dump.glob("*.cu")]
    assert any("tnq_p" in t for t in srcs) and any("tnq_b" in t for t in srcs)
    assert all("griddepcontrol.wait" in t for t in srcs)  # every pass waits for its predecessor
    assert any("fma.rn.f32x2" in t for t in srcs)
