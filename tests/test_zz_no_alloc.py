"""The workspace-free expectation entry point, checked against the workspace one (GPU).

tn_state_expectation_noalloc exists for callers that cannot hand the library device memory
(their memory is owned by another allocator, or an allocation would synchronise the
device).  Its partial sums live in an array compiled into the library and shared by every
call, so this test makes two calls in a row with different sizes and checks both against
tn_state_expectation with a caller workspace.  Kept in a file that is collected last.
"""
import numpy as np
import pytest

from paper_2108_06831_gb300 import circuits as C

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _expect_both(tn, obs, batch, states):
    ws_bytes = tn.state_expectation_workspace_bytes(obs, batch)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    ref = torch.empty(batch, dtype=torch.float64, device="cuda")
    tn.state_expectation(obs, batch, states, ref, ws, ws_bytes)
    got = torch.full((batch,), float("nan"), dtype=torch.float64, device="cuda")
    tn.state_expectation_noalloc(obs, batch, states, got)
    torch.cuda.synchronize()
    assert tn.sync_status() == tn.OK
    return got.cpu().numpy(), ref.cpu().numpy()


def test_noalloc_matches_workspace_entry_point_twice():
    from paper_2108_06831_gb300 import tn
    n = 14
    c, p0 = C.brickwork(n, 8, 31, parameterized=True)
    rng = np.random.default_rng(2)
    params = np.stack([p0] + [rng.uniform(0, 2 * np.pi, size=p0.shape) for _ in range(2)])
    ctr = tn.Contractor(c, batch=3)
    states = ctr.state(torch.as_tensor(params, device="cuda"))
    # first call: TFIM (two reduction passes), three states
    obs1 = tn.Observable(C.tfim(n))
    got, ref = _expect_both(tn, obs1, 3, states)
    assert np.all(np.abs(got - ref) <= 1e-4 * np.maximum(1.0, np.abs(ref)))
    # and against the FP64 oracle (state-vector simulation, explicit Pauli application)
    from oracle import observables as OB
    H1 = C.tfim(n)
    exact = np.array([OB.expectation(c, H1, params[b]) for b in range(3)])
    assert np.all(np.abs(got - exact) <= 1e-4 * np.maximum(1.0, np.abs(exact)))
    # second call right after: another observable and fewer states over the same scratch
    obs2 = tn.Observable(C.random_pauli_sum(n, 17, 5))
    got2, ref2 = _expect_both(tn, obs2, 2, states)
    assert np.all(np.abs(got2 - ref2) <= 1e-4 * np.maximum(1.0, np.abs(ref2)))
    H2 = C.random_pauli_sum(n, 17, 5)
    exact2 = np.array([OB.expectation(c, H2, params[b]) for b in range(2)])
    assert np.all(np.abs(got2 - exact2) <= 1e-4 * np.maximum(1.0, np.abs(exact2)))


def test_noalloc_rejects_requests_beyond_its_scratch():
    from paper_2108_06831_gb300 import tn
    n = 14
    obs = tn.Observable(C.tfim(n))
    big = 4096  # 4096 states x 2 passes x 512 partial sums > 131072
    states = torch.zeros((1, 1 << n), dtype=torch.complex64, device="cuda")
    out = torch.zeros(big, dtype=torch.float64, device="cuda")
    with pytest.raises(tn.TnError) as e:
        tn.state_expectation_noalloc(obs, big, states, out)
    assert "built-in scratch" in str(e.value)
