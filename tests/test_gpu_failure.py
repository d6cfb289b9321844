"""Failure path of the persistent executor: a dependency wait that can never be met (GPU).

The executor's tiles wait, bounded, for the previous pass of their circuit (a spin on a
counter in global memory).  tn_batch_test_stall makes one pass wait for one more tile than
its predecessor has, with a short bound; the run must then end by itself, the device status
word must read TN_ERR_TIMEOUT, and the context must stay usable: a normal run right after
(the table restored) matches the oracle.  No kernel faults, traps or hangs here: the wait is
on a counter nothing will raise, and it gives up after a few milliseconds.
"""
import time

import numpy as np
import pytest

from paper_2108_06831_gb300 import circuits as C

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _batch(tn):
    circs = [C.brickwork(12, 6, 41)[0], C.qft(11, 5), C.brickwork(10, 4, 42)[0]]
    plans = [tn.Plan(tn.CircuitHandle(c), tile_qubits=8, specialize=False) for c in circs]
    assert plans[0].stats()["n_passes"] >= 2
    b = tn.Batch(plans)
    states = torch.full((b.state_elems,), complex(float("nan"), 0), dtype=torch.complex64, device="cuda")
    ws = torch.empty(b.workspace_bytes, dtype=torch.uint8, device="cuda")
    return circs, plans, b, states, ws


def test_unmet_dependency_times_out_and_context_stays_usable():
    from oracle.statevector import simulate_state
    from paper_2108_06831_gb300 import tn
    circs, plans, b, states, ws = _batch(tn)
    assert tn.sync_status() == tn.OK  # nothing pending from earlier tests
    tn.batch_test_stall(b, 0, 1, 5_000_000)  # 5 ms bound
    t0 = time.perf_counter()
    tn.batch_run(b, states, ws)
    torch.cuda.synchronize()  # the kernel returns by itself
    elapsed = time.perf_counter() - t0
    assert tn.sync_status() == tn.ERR_TIMEOUT
    assert tn.sync_status() == tn.OK  # reading the word cleared it
    assert elapsed < 1.5, elapsed  # the short bound, not the default 2 s
    # the same batch, restored: a normal run is correct
    tn.batch_test_stall(b, -1)
    states.fill_(float("nan"))
    tn.batch_run(b, states, ws)
    torch.cuda.synchronize()
    assert tn.sync_status() == tn.OK
    got = states.cpu().numpy()
    for c, off in zip(circs, b.offsets):
        ref = simulate_state(c)
        s = got[off:off + (1 << c.n_qubits)]
        assert np.linalg.norm(s - ref) / np.linalg.norm(ref) <= 1e-5, c.name


def test_stall_arguments_validated():
    from paper_2108_06831_gb300 import tn
    circs, plans, b, states, ws = _batch(tn)
    for args in [(5, 1, 5_000_000), (0, 0, 5_000_000), (0, 99, 5_000_000), (0, 1, 10), (0, 1, 10 ** 11)]:
        with pytest.raises(tn.TnError) as e:
            tn.batch_test_stall(b, *args)
        assert e.value.status == tn.ERR_INVALID_ARG
