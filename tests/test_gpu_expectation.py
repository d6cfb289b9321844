"""Expectation values and adjoint gradients against the FP64 oracle (GPU).

Bars: |E - E_ref| <= 1e-4 max(1, |E_ref|); per parameter set
||g - g_ref|| / max(||g_ref||, 1e-3) <= 1e-4, with g_ref the oracle's parameter-shift
gradient (cross-checked there against finite differences).
"""
import numpy as np
import pytest

from paper_2108_06831_gb300 import circuits as C

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _tn():
    from paper_2108_06831_gb300 import tn
    return tn


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


@pytest.mark.parametrize("n,layers,tile", [(4, 2, 0), (8, 3, 0), (12, 2, 7), (14, 3, 9)])
def test_hea_tfim_expectation_and_gradient(n, layers, tile):
    from oracle import gradients as GR
    from oracle import observables as OB
    tn = _tn()
    c = C.hea(n, layers)
    H = C.tfim(n)
    batch = 3
    params = C.hea_params(c.n_params, batch, 40 + n)
    ctr = tn.Contractor(c, target=tn.TARGET_EXPECTATION, batch=batch, tile_qubits=tile)
    obs = tn.Observable(H)
    E = ctr.expectation(obs, _dev(params)).cpu().numpy()
    G = ctr.expectation_backward(obs, _dev(params)).cpu().numpy()
    for b in range(batch):
        Eref = OB.expectation(c, H, params[b])
        assert abs(E[b] - Eref) <= 1e-4 * max(1.0, abs(Eref))
        gref = GR.param_shift_grad(c, H, params[b])
        assert np.linalg.norm(G[b] - gref) / max(np.linalg.norm(gref), 1e-3) <= 1e-4


@pytest.mark.parametrize("n,layers,tile,ham", [(6, 3, 0, "tfim"), (13, 2, 8, "tfim"), (11, 2, 8, "pauli")])
def test_value_and_grad_matches_separate_calls_and_oracle(n, layers, tile, ham):
    """tn_expectation_value_and_grad contracts the forward state once; energies and gradients
    equal the two-call path and the oracle (parameter shift).  Its energy is Re <psi|H psi> summed
    from lambda = H psi, the two-call path's the direct term sum: both in FP32 per amplitude, so they
    agree to FP32 rounding of the state's norm-sized sums, not bit for bit."""
    from oracle import gradients as GR
    from oracle import observables as OB
    tn = _tn()
    c = C.hea(n, layers)
    H = C.tfim(n) if ham == "tfim" else C.random_pauli_sum(n, 30, 90 + n)  # X, Y and Z factors
    batch = 2
    params = C.hea_params(c.n_params, batch, 70 + n)
    ctr = tn.Contractor(c, target=tn.TARGET_EXPECTATION, batch=batch, tile_qubits=tile)
    obs = tn.Observable(H)
    e1, g1 = ctr.expectation_value_and_grad(obs, _dev(params))
    e0 = ctr.expectation(obs, _dev(params))
    g0 = ctr.expectation_backward(obs, _dev(params))
    torch.cuda.synchronize()
    assert tn.sync_status() == tn.OK
    E, G = e1.cpu().numpy(), g1.cpu().numpy()
    assert np.allclose(E, e0.cpu().numpy(), rtol=1e-5, atol=1e-5)
    assert np.allclose(G, g0.cpu().numpy(), rtol=1e-9, atol=1e-12)
    for b in range(batch):
        Eref = OB.expectation(c, H, params[b])
        assert abs(E[b] - Eref) <= 1e-4 * max(1.0, abs(Eref))
        gref = GR.param_shift_grad(c, H, params[b])
        assert np.linalg.norm(G[b] - gref) / max(np.linalg.norm(gref), 1e-3) <= 1e-4


def test_theta_zero_energy_20q():
    tn = _tn()
    n = 20
    c = C.hea(n, 10)
    ctr = tn.Contractor(c, target=tn.TARGET_EXPECTATION, batch=2)
    obs = tn.Observable(C.tfim(n))
    E = ctr.expectation(obs, _dev(np.zeros((2, c.n_params)))).cpu().numpy()
    assert np.abs(E + 19.0).max() <= 1e-4 * 19


def test_cfg4_full_size_sampled():
    """20-qubit HEA, 400 parameters, batch 64 (bench launch configuration); the oracle checks
    the energy of two batch elements and, by parameter shift, three sampled gradient entries
    (a full 400-parameter shift at 2^20 amplitudes would take the oracle minutes)."""
    from oracle import observables as OB
    from oracle.statevector import simulate_state
    tn = _tn()
    n, layers, batch = 20, 10, 64
    c = C.hea(n, layers)
    H = C.tfim(n)
    params = C.hea_params(c.n_params, batch, 4000)
    ctr = tn.Contractor(c, target=tn.TARGET_EXPECTATION, batch=batch)
    obs = tn.Observable(H)
    E = ctr.expectation(obs, _dev(params)).cpu().numpy()
    G = ctr.expectation_backward(obs, _dev(params)).cpu().numpy()
    e2, g2 = ctr.expectation_value_and_grad(obs, _dev(params))  # the call the benchmark times
    E2, G2 = e2.cpu().numpy(), g2.cpu().numpy()
    assert np.allclose(G2, G, rtol=1e-9, atol=1e-12)
    rng = np.random.default_rng(1)
    for b in (0, 37):
        Eref = OB.expectation(c, H, params[b])
        assert abs(E[b] - Eref) <= 1e-4 * max(1.0, abs(Eref))
        assert abs(E2[b] - Eref) <= 1e-4 * max(1.0, abs(Eref))
    for b in (37,):
        ks = rng.choice(c.n_params, size=3, replace=False)
        for k in ks:
            gate_idx = [i for i, g in enumerate(c.gates) if g.param_idx == k]
            vals = []
            for sgn in (1, -1):
                ov = {gi: (params[b][k] + sgn * np.pi / 2,) for gi in gate_idx}
                vals.append(OB.expectation_of_state(simulate_state(c, params[b], ov), H))
            gk = 0.5 * (vals[0] - vals[1])
            assert abs(G[b, k] - gk) <= 1e-4 * max(np.linalg.norm(G[b]), 1e-3)


def test_random_pauli_sum_state_expectation():
    from oracle import observables as OB
    from oracle.statevector import simulate_state
    tn = _tn()
    n = 11
    c = C.random_circuit(n, 120, 3)
    H = C.random_pauli_sum(n, 25, 8)
    psi = simulate_state(c)
    ctr = tn.Contractor(c)
    st = ctr.state()
    obs = tn.Observable(H)
    ws_bytes = tn.state_expectation_workspace_bytes(obs, 1)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    tn.state_expectation(obs, 1, st, out, ws, ws_bytes)
    Eref = OB.expectation_of_state(psi, H)
    assert abs(out.item() - Eref) <= 1e-4 * max(1.0, abs(Eref))


def test_autograd_function():
    tn = _tn()
    from oracle import gradients as GR
    n = 6
    c = C.hea(n, 2)
    H = C.tfim(n)
    params = C.hea_params(c.n_params, 2, 9)
    ctr = tn.Contractor(c, target=tn.TARGET_EXPECTATION, batch=2)
    obs = tn.Observable(H)
    th = torch.tensor(params, device="cuda", requires_grad=True)
    E = tn.expectation_autograd(th, ctr, obs)
    (E * torch.tensor([1.0, -2.0], device="cuda", dtype=torch.float64)).sum().backward()
    g = th.grad.cpu().numpy()
    for b, w in ((0, 1.0), (1, -2.0)):
        gref = w * GR.param_shift_grad(c, H, params[b])
        assert np.linalg.norm(g[b] - gref) / max(np.linalg.norm(gref), 1e-3) <= 1e-4
