"""State contraction by uniform square blocks (TN_PLAN_BLOCKS) against the FP64 oracle (GPU).

The circuit is cut into blocks of gates on k qubits, each precontracted per call into one
2^k x 2^k matrix and applied to the state by the batched complex GEMM in FP32 (CUDA cores),
3xTF32 or split BF16 (tensor cores).  Same bar as every state: relative L2 <= 1e-5.
"""
import numpy as np
import pytest

from paper_2108_06831_gb300 import circuits as C

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-5


def _state(circ, k, precision, params=None, batch=1):
    from paper_2108_06831_gb300 import tn
    ctr = tn.Contractor(circ, batch=batch, precision=precision, block_qubits=k)
    st = ctr.plan.stats()
    assert st["n_fused"] >= 1 and st["tile_qubits"] == k
    p = None if params is None else torch.as_tensor(np.asarray(params, dtype=np.float64).reshape(batch, -1),
                                                    device="cuda").contiguous()
    out = torch.full((batch, 1 << circ.n_qubits), complex(float("nan"), 0), dtype=torch.complex64, device="cuda")
    tn.contract_state(ctr.plan, p, out, ctr.workspace)
    torch.cuda.synchronize()
    assert tn.sync_status() == tn.OK
    return out.cpu().numpy(), st


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CIRCUITS = [
    lambda: C.brickwork(14, 10, 71)[0],
    lambda: C.grid(4, 4, 12, 72),
    lambda: C.paper_fig31(16, 6, 73),
    lambda: C.qft(14, 5000),                # long-range phases: blocks seeded by single gates
    lambda: C.random_circuit(15, 220, 74),  # every gate kind, arbitrary qubit pairs
]


@pytest.mark.parametrize("k", [6, 7])
@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("maker", CIRCUITS)
def test_blocks_match_oracle(maker, precision, k):
    from oracle.statevector import simulate_state
    c = maker()
    if c.n_qubits < k + 7:
        pytest.skip("needs k + 7 qubits")
    c.init_basis = (0x5A5A5 * (k + precision)) % (1 << c.n_qubits)
    got, st = _state(c, k, precision)
    ref = simulate_state(c)
    err = _rel(got[0], ref)
    assert err <= TOL, (err, st)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_blocks_parameterised_batch(precision):
    """Block matrices precontracted per call from each parameter set (batch of 2)."""
    from oracle.statevector import simulate_state
    c, p0 = C.brickwork(16, 8, 75, parameterized=True)
    rng = np.random.default_rng(76)
    params = np.stack([p0, rng.uniform(0, 2 * np.pi, size=p0.shape)])
    got, _ = _state(c, 6, precision, params, batch=2)
    for b in range(2):
        assert _rel(got[b], simulate_state(c, params[b])) <= TOL


@pytest.mark.parametrize("precision", [1, 2])
def test_blocks_cfg2_full_size_sampled(precision):
    """The 24-qubit brickwork of depth 20 with parameterised U3 angles, in the launch
    configuration the bench times for the tensor-core arm (k = 6): sampled amplitudes against
    the oracle's network contraction, and the norm."""
    from oracle.tn import contract_amplitude
    c, params = C.brickwork(24, 20, 1001, parameterized=True)
    got, st = _state(c, 6, precision, params)
    assert st["n_passes"] == st["n_fused"] - 1
    assert abs(np.linalg.norm(got[0].astype(np.complex128)) - 1.0) < 1e-5
    cf, _ = C.brickwork(24, 20, 1001)
    xs = C.random_bitstrings(24, 10, 4242)
    ref = np.array([contract_amplitude(cf, int(x)) for x in xs])
    assert _rel(got[0][xs.astype(np.int64)], ref) <= TOL
