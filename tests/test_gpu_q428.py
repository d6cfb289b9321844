"""Fixed-point (Q4.28) state contraction against the oracle's fixed-point simulation (GPU).

Integer work: the bar is bit-exact equality of every int32 component.  The error of the
fixed-point state against the FP64 oracle is measured next to that of the FP32 path.
"""
import numpy as np
import pytest

from paper_2108_06831_gb300 import circuits as C

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _q428(circ):
    from paper_2108_06831_gb300 import tn
    p = tn.Plan(tn.CircuitHandle(circ), q428=True)
    st = torch.full((1 << circ.n_qubits, 2), 12345, dtype=torch.int32, device="cuda")
    tn.contract_state_q428(p, st)
    torch.cuda.synchronize()
    assert tn.sync_status() == tn.OK
    a = st.cpu().numpy().astype(np.int64)
    return a[:, 0], a[:, 1]


def _assert_bit_exact(circ):
    from oracle import fixedpoint as F
    re, im = _q428(circ)
    rr, ri = F.simulate_state_q428(circ)
    bad = np.flatnonzero((re != rr) | (im != ri))
    assert bad.size == 0, (bad[:5], re[bad[:5]], rr[bad[:5]])


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 11, 14])
def test_random_circuits_bit_exact(n):
    """Every gate kind (one- and two-qubit, diagonal and dense, both qubit orders)."""
    for seed in range(2):
        c = C.random_circuit(n, 12 * n + 5, 7700 + 10 * n + seed)
        c.init_basis = (seed * 40503) % (1 << n)
        _assert_bit_exact(c)


@pytest.mark.parametrize("maker", [
    lambda: C.brickwork(16, 10, 17)[0],
    lambda: C.paper_fig31(12, 6, 18),
    lambda: C.qft(10, 321),
    lambda: C.ghz(13),
    lambda: C.Circuit(6, [], init_basis=37),
])
def test_workload_families_bit_exact(maker):
    _assert_bit_exact(maker())


def test_brickwork_20_depth_20_bit_exact():
    """20 qubits, depth 20 (the 24-qubit workload's generator at a size the oracle runs in seconds)."""
    _assert_bit_exact(C.brickwork(20, 20, 1002)[0])


@pytest.mark.parametrize("n", [12, 16, 20])
def test_error_against_fp64(n):
    """Relative 2-norm error of the Q4.28 state against FP64, within the rounding bound (every gate
    adds at most 2^(n/2) 2^-28.5 + 4 2^-28.5 in the 2-norm); the FP32 path's error alongside."""
    from oracle import fixedpoint as F
    from oracle.statevector import simulate_state
    from paper_2108_06831_gb300 import tn
    c, _ = C.brickwork(n, 20, 2000 + n)
    ref = simulate_state(c)
    re, im = _q428(c)
    err_q = np.linalg.norm(F.to_complex(re, im) - ref) / np.linalg.norm(ref)
    ctr = tn.Contractor(c)
    out = ctr.state(None)
    torch.cuda.synchronize()
    got32 = out.cpu().numpy()[0].astype(np.complex128)
    err_32 = np.linalg.norm(got32 - ref) / np.linalg.norm(ref)
    bound = len(c.gates) * (2.0 ** (n / 2) + 4.0) * 2.0 ** -28.5
    print(f"n={n}: Q4.28 relative error {err_q:.3e}, FP32 {err_32:.3e}")
    assert 0 < err_q <= bound
    assert err_32 <= 1e-5


def test_wrong_plan_kinds_rejected():
    from paper_2108_06831_gb300 import tn
    c = C.brickwork(6, 2, 1)[0]
    fixed = tn.Plan(tn.CircuitHandle(c), q428=True)
    plain = tn.Plan(tn.CircuitHandle(c))
    st = torch.zeros((64, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(tn.TnError):
        tn.contract_state_q428(plain, st)
    with pytest.raises(tn.TnError):
        tn.contract_state(fixed, None, torch.zeros(64, dtype=torch.complex64, device="cuda"),
                          torch.empty(16, dtype=torch.uint8, device="cuda"))
    with pytest.raises(tn.TnError):
        tn.Plan(tn.CircuitHandle(C.brickwork(6, 2, 1, parameterized=True)[0]), q428=True)


def test_30_qubits_closed_form():
    """30 qubits (an 8 GiB int32-pair state): H on every qubit, CZ on every neighbour pair, X on
    qubit 0.  Each H meets a qubit still in |0>, so it maps every amplitude a to
    round(quantize(1/sqrt 2) a / 2^28) on both branches; CZ (entries +-1) negates exactly and X
    permutes exactly.  Every entry is then +-a_30 (real), the sign (-1)^(sum_q x_q x_{q+1}) of the
    index before the X."""
    from paper_2108_06831_gb300 import tn
    n = 30
    gates = [C.Gate("H", (q,)) for q in range(n)] + [C.Gate("CZ", (q, q + 1)) for q in range(n - 1)]
    gates.append(C.Gate("X", (0,)))
    p = tn.Plan(tn.CircuitHandle(C.Circuit(n, gates)), q428=True)
    st = torch.empty((1 << n, 2), dtype=torch.int32, device="cuda")
    tn.contract_state_q428(p, st)
    torch.cuda.synchronize()
    assert tn.sync_status() == tn.OK
    # quantize(1/sqrt 2) = floor(2^28 / sqrt 2 + 1/2) = 189812531 (2^28 / sqrt 2 = 189812531.25)
    qh = 189812531
    assert abs(qh - (1 << 28) / np.sqrt(2.0)) < 0.5
    # each H: a <- floor((qh a + 2^27) / 2^28), the reading's round half up written out in
    # Python integers (exact); a stays positive, far from the int32 limits
    a = 1 << 28
    for _ in range(n):
        a = (qh * a + (1 << 27)) // (1 << 28)
    assert not bool((st[:, 1] != 0).any())
    assert bool((st[:, 0].abs() == a).all())
    rng = np.random.default_rng(30)
    xs = rng.integers(0, 1 << n, size=4096, dtype=np.int64)
    got = st[torch.as_tensor(xs, device="cuda"), 0].cpu().numpy().astype(np.int64)
    pre = xs ^ (1 << (n - 1))  # undo the X on qubit 0 (the most significant bit)
    bits = (pre[:, None] >> (n - 1 - np.arange(n))[None, :]) & 1
    sign = 1 - 2 * (np.sum(bits[:, :-1] * bits[:, 1:], axis=1) & 1)
    assert np.array_equal(got, sign * a)
