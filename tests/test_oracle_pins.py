"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Every check here compares the oracle with something other than itself: a value
printed in the paper (fixtures under tests/golden/, each citing its section),
a closed form, a textbook identity, or a brute-force construction.
"""
import cmath
import math
import os

import numpy as np
import pytest

from oracle import gates as G
from oracle import gradients as GR
from oracle import observables as OB
from oracle import statevector as SV
from oracle import tn as TN
from paper_2108_06831_gb300 import circuits as C

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


# ---------------------------------------------------------------- gates

ALL1 = ["H", "X", "Y", "Z", "S", "SDG", "T", "TDG", "SX", "SY", "SW", "RX", "RY", "RZ", "U3"]
ALL2 = ["CZ", "CNOT", "CP", "SWAP"]


@pytest.mark.parametrize("kind", ALL1 + ALL2)
def test_gate_unitary(kind):
    rng = np.random.default_rng(3)
    for _ in range(5):
        ang = rng.uniform(0, 2 * math.pi, size=3)
        U = G.matrix(kind, ang)
        d = U.shape[0]
        assert np.abs(U @ U.conj().T - np.eye(d)).max() < 1e-14


def test_textbook_identities():
    X, Y, Z = G.X, G.Y, G.Z
    H = G.matrix("H")
    assert np.allclose(H @ Z @ H, X, atol=1e-15)
    assert np.allclose(G.rx(math.pi), -1j * X, atol=1e-15)
    assert np.allclose(G.ry(math.pi), -1j * Y, atol=1e-15)
    assert np.allclose(G.rz(math.pi), -1j * Z, atol=1e-15)
    # U3(pi, 0, pi) = X and U3(pi/2, 0, pi) = H (standard special cases)
    assert np.allclose(G.u3(math.pi, 0, math.pi), X, atol=1e-15)
    assert np.allclose(G.u3(math.pi / 2, 0, math.pi), H, atol=1e-15)
    # U3(t, p, l) = e^{i(p+l)/2} RZ(p) RY(t) RZ(l)
    t, p, l = 0.3, 1.1, -2.0
    assert np.allclose(G.u3(t, p, l), cmath.exp(0.5j * (p + l)) * G.rz(p) @ G.ry(t) @ G.rz(l), atol=1e-15)
    # square roots: SX^2 = RX(pi) = -iX, SY^2 = -iY, SW^2 = -iW
    W = (X + Y) / math.sqrt(2)
    assert np.allclose(G.matrix("SX") @ G.matrix("SX"), -1j * X, atol=1e-15)
    assert np.allclose(G.matrix("SY") @ G.matrix("SY"), -1j * Y, atol=1e-15)
    assert np.allclose(G.matrix("SW") @ G.matrix("SW"), -1j * W, atol=1e-15)
    S, T = G.matrix("S"), G.matrix("T")
    assert np.allclose(T @ T, S, atol=1e-15) and np.allclose(S @ S, Z, atol=1e-15)
    # CZ = (I (x) H) CNOT (I (x) H); SWAP = three CNOTs
    IH = np.kron(np.eye(2), H)
    assert np.allclose(IH @ G.matrix("CNOT") @ IH, G.matrix("CZ"), atol=1e-15)
    CN = G.matrix("CNOT")
    P = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]])  # swaps the qubits
    CN_rev = P @ CN @ P
    assert np.allclose(CN @ CN_rev @ CN, G.matrix("SWAP"), atol=1e-15)
    assert np.allclose(G.matrix("CP", (math.pi,)), G.matrix("CZ"), atol=1e-15)


# ---------------------------------------------------------------- Sec. 2.1 fixtures

def _unitary_with_first_column(a, b):
    return np.array([[a, -np.conj(b)], [b, np.conj(a)]], dtype=np.complex128)


def test_product_state_order_sec21():
    rng = np.random.default_rng(0)
    v = rng.normal(size=4) + 1j * rng.normal(size=4)
    a, b = v[:2] / np.linalg.norm(v[:2])
    a2, b2 = v[2:] / np.linalg.norm(v[2:])
    circ = C.Circuit(2, [C.Gate("MAT1", (0,), mat=tuple(_unitary_with_first_column(a, b).reshape(-1))),
                         C.Gate("MAT1", (1,), mat=tuple(_unitary_with_first_column(a2, b2).reshape(-1)))])
    psi = SV.simulate_state(circ)
    val = {"alpha": a, "beta": b, "alpha'": a2, "beta'": b2}
    for idx, f0, f1 in _rows("sec21_product_order.txt"):
        assert abs(psi[int(idx)] - val[f0] * val[f1]) < 1e-15


def test_kron_layout_sec21():
    rng = np.random.default_rng(1)
    U = G.u3(*rng.uniform(0, 6, 3))
    V = G.u3(*rng.uniform(0, 6, 3))
    rows = _rows("sec21_kron_layout.txt")
    K = np.zeros((4, 4), dtype=np.complex128)
    for r, row in enumerate(rows):
        for c, tok in enumerate(row):
            K[r, c] = U[int(tok[1]), int(tok[2])] * V[int(tok[4]), int(tok[5])]
    # U on qubit 0, V on qubit 1 applied by the simulator must act as K
    for col in range(4):
        psi = SV.apply_matrix(SV.apply_matrix(SV.basis_state(2, col), 2, U, (0,)), 2, V, (1,))
        assert np.abs(psi - K[:, col]).max() < 1e-15
    # and as one two-qubit MAT2 gate with matrix K
    for col in range(4):
        psi = SV.apply_matrix(SV.basis_state(2, col), 2, K, (0, 1))
        assert np.abs(psi - K[:, col]).max() < 1e-15


def test_bell_sec21():
    psi = SV.simulate_state(C.bell())
    ref = np.zeros(4, dtype=np.complex128)
    for idx, re, im in _rows("sec21_bell.txt"):
        ref[int(idx)] = float(re) + 1j * float(im)
    assert np.abs(psi - ref).max() < 1e-15


def test_fig21_as_drawn_and_ghz():
    psi = SV.simulate_state(C.fig21_as_drawn())
    ref = np.zeros(8, dtype=np.complex128)
    for idx, re, im in _rows("fig21_as_drawn.txt"):
        ref[int(idx)] = float(re) + 1j * float(im)
    assert np.abs(psi - ref).max() < 1e-15
    for n in (2, 3, 5, 8):
        psi = SV.simulate_state(C.ghz(n))
        ref = np.zeros(1 << n, dtype=np.complex128)
        ref[0] = ref[-1] = 1 / math.sqrt(2)
        assert np.abs(psi - ref).max() < 1e-15


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 11])
def test_qft_closed_form(n):
    rng = np.random.default_rng(n)
    for x in {0, (1 << n) - 1, int(rng.integers(0, 1 << n))}:
        psi = SV.simulate_state(C.qft(n, x))
        y = np.arange(1 << n)
        ref = np.exp(2j * math.pi * x * y / (1 << n)) / math.sqrt(1 << n)
        assert np.abs(psi - ref).max() < 1e-12
        assert np.allclose(np.abs(psi), 2.0 ** (-n / 2), atol=1e-13)


def test_norm_preserved():
    for seed in range(3):
        c, _ = C.brickwork(12, 10, seed)
        psi = SV.simulate_state(c)
        assert abs(np.linalg.norm(psi) - 1) < 1e-12
    psi = SV.simulate_state(C.random_circuit(10, 200, 7))
    assert abs(np.linalg.norm(psi) - 1) < 1e-12


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (3, 2), (5, 3), (7, 4), (8, 5)])
def test_bruteforce_unitary_product(n, seed):
    """Simulator == product of full 2^N x 2^N gate matrices built entry by entry."""
    c = C.random_circuit(n, 6 * n + 4, seed)
    c.init_basis = (seed * 2654435761) % (1 << n)
    Ufull = SV.circuit_unitary(c)
    psi = SV.simulate_state(c)
    assert np.abs(psi - Ufull[:, c.init_basis]).max() < 1e-12
    assert np.abs(Ufull @ Ufull.conj().T - np.eye(1 << n)).max() < 1e-12


def test_bruteforce_kron_adjacent():
    """For adjacent qubits the full operator equals I (x) U (x) I (Sec. 2.1 Kronecker rule)."""
    rng = np.random.default_rng(9)
    n = 5
    for q in range(n):
        U = G.u3(*rng.uniform(0, 6, 3))
        K = np.kron(np.kron(np.eye(1 << q), U), np.eye(1 << (n - 1 - q)))
        assert np.abs(SV.full_operator(n, U, (q,)) - K).max() < 1e-15
    for q in range(n - 1):
        U4 = G.matrix("CNOT") @ np.kron(G.u3(1, 2, 3), G.u3(0.5, 0.1, 0.2))
        K = np.kron(np.kron(np.eye(1 << q), U4), np.eye(1 << (n - 2 - q)))
        assert np.abs(SV.full_operator(n, U4, (q, q + 1)) - K).max() < 1e-15


# ---------------------------------------------------------------- the network path

@pytest.mark.parametrize("maker", [
    lambda: C.brickwork(10, 8, 1)[0],
    lambda: C.random_circuit(9, 80, 11),
    lambda: C.qft(7, 45),
    lambda: C.paper_fig31(8, 4, 2),
    lambda: C.grid(3, 3, 8, 5),
])
def test_tn_equals_statevector(maker):
    c = maker()
    a = TN.contract_state(c)
    b = SV.simulate_state(c)
    assert np.abs(a - b).max() < 1e-12


def test_tn_amplitudes_equal_state_entries():
    c = C.grid(4, 4, 8, 3)
    psi = SV.simulate_state(c)
    xs = C.random_bitstrings(16, 12, 4)
    amps = TN.contract_amplitudes(c, xs)
    assert np.abs(amps - psi[xs.astype(np.int64)]).max() < 1e-12


# ---------------------------------------------------------------- expectation

def test_expectation_theta_zero_tfim():
    n = 20
    c = C.hea(n, 10)
    H = C.tfim(n)
    assert abs(OB.expectation(c, H, np.zeros(c.n_params)) - (-(n - 1))) < 1e-12


@pytest.mark.parametrize("n", [2, 4, 7])
def test_expectation_vs_dense_hamiltonian(n):
    c = C.hea(n, 3)
    p = C.hea_params(c.n_params, 1, 5)[0]
    psi = SV.simulate_state(c, p)
    for H in (C.tfim(n), C.random_pauli_sum(n, 9, n)):
        M = OB.hamiltonian_matrix(H)
        ref = float(np.real(np.vdot(psi, M @ psi)))
        assert abs(OB.expectation_of_state(psi, H) - ref) < 1e-12
        assert np.abs(OB.apply_hamiltonian(psi, H) - M @ psi).max() < 1e-12


# ---------------------------------------------------------------- gradients

def test_gradient_closed_form_single_qubit():
    # <Z> after RY(t)|0> is cos t, so the derivative is -sin t
    c = C.Circuit(1, [C.Gate("RY", (0,), (), 0)], n_params=1)
    H = C.PauliSum(1, [1.0], ["Z"])
    for t in (0.0, 0.4, 2.5, -1.3):
        p = np.array([t])
        assert abs(OB.expectation(c, H, p) - math.cos(t)) < 1e-14
        assert abs(GR.param_shift_grad(c, H, p)[0] + math.sin(t)) < 1e-14
    # <X> after RZ(p) RY(pi/2)|0> is cos p
    c = C.Circuit(1, [C.Gate("RY", (0,), (math.pi / 2,)), C.Gate("RZ", (0,), (), 0)], n_params=1)
    H = C.PauliSum(1, [1.0], ["X"])
    for t in (0.1, 1.7):
        assert abs(GR.param_shift_grad(c, H, np.array([t]))[0] + math.sin(t)) < 1e-14


def test_param_shift_equals_finite_difference():
    c = C.hea(4, 2)
    H = C.tfim(4)
    p = C.hea_params(c.n_params, 1, 2)[0]
    ps = GR.param_shift_grad(c, H, p)
    fd = GR.finite_diff_grad(c, H, p, h=1e-4)
    assert np.abs(ps - fd).max() < 1e-7


def test_param_shift_u3_and_cp():
    gates = [C.Gate("H", (0,)), C.Gate("H", (1,)), C.Gate("U3", (0,), (), 0),
             C.Gate("CP", (0, 1), (), 3), C.Gate("U3", (1,), (), 4), C.Gate("CNOT", (1, 0))]
    c = C.Circuit(2, gates, n_params=7)
    H = C.random_pauli_sum(2, 6, 1)
    p = np.random.default_rng(3).uniform(-3, 3, size=7)
    assert np.abs(GR.param_shift_grad(c, H, p) - GR.finite_diff_grad(c, H, p, h=1e-4)).max() < 1e-7


@pytest.mark.parametrize("maker", [
    lambda: C.grid(4, 4, 12, 21),
    lambda: C.grid(3, 5, 9, 2),
    lambda: C.grid(4, 5, 12, 33),
    lambda: C.random_circuit(9, 70, 13),
    lambda: C.qft(8, 77),
    lambda: C.hea(6, 2),
])
def test_sweep_amplitudes_equal_state_entries(maker):
    """The shared-index network (diagonal gates as couplings), swept qubit by qubit, gives the
    state-vector entries."""
    c = maker()
    p = C.hea_params(c.n_params, 1, 3)[0] if c.n_params else None
    psi = SV.simulate_state(c, p)
    xs = C.random_bitstrings(c.n_qubits, 6, 12)
    for x in xs:
        assert abs(TN.contract_amplitude_sweep(c, int(x), p) - psi[int(x)]) < 1e-12


# --- Q4.28 fixed-point oracle (Sec. 3: 32-bit fixed point, 28 fractional bits) -------------

def test_q428_quantize_rounding_and_saturation():
    """floor(x 2^28 + 1/2): halves round up, values beyond the int32 range saturate."""
    from oracle import fixedpoint as F
    assert F.quantize(1.0) == 1 << 28 and F.quantize(-1.0) == -(1 << 28)
    assert F.quantize(2.0 ** -29) == 1 and F.quantize(-(2.0 ** -29)) == 0  # ties toward +inf
    assert F.quantize(3 * 2.0 ** -30) == 1 and F.quantize(-3 * 2.0 ** -30) == -1
    assert F.quantize(2.0 ** -30) == 0
    assert F.quantize(8.0) == 2 ** 31 - 1 and F.quantize(-9.0) == -(2 ** 31)
    assert F.quantize(-8.0) == -(2 ** 31)  # -8 is representable


def test_q428_output_rounding_on_hand_computed_sums():
    """One gate on a hand-built Q4.28 state whose exact integer sums fall on the rounding
    boundaries.  With U = diag(u0, u1) (imaginary parts 0) the output components are
    round(u_l psi_l / 2^28); the reading fixes round half up, floor((acc + 2^27) / 2^28), and
    saturation to int32.  Expected values are literals worked out by hand:
      acc = +2^27        -> 1  (a tie rounds up)      acc = -2^27     -> 0  (toward +inf)
      acc = 2^27 - 1     -> 0                         acc = 3 2^27    -> 2
      acc = -3 2^27      -> -1                        acc = 2^27 + 1  -> 1
    and, on a two-qubit gate with rows (2^29, 2^29, 2^29, 2^29) and -(same) applied to the
    state (2^29, 2^29, 2^29, 2^29): acc = +-2^60, i.e. +-2^32 after the shift, saturated to
    2^31 - 1 and -2^31.
    A floor (no half added), a truncation toward zero or a missing clip fails at least one."""
    from oracle import fixedpoint as F
    z = np.zeros((2, 2), dtype=np.int64)
    cases = [  # (u0, psi0, u1, psi1, out0, out1)
        (1 << 13, 1 << 14, -(1 << 13), 1 << 14, 1, 0),
        ((1 << 27) - 1, 1, 3, 1 << 27, 0, 2),
        (-3, 1 << 27, (1 << 27) + 1, 1, -1, 1),
    ]
    for u0, p0, u1, p1, o0, o1 in cases:
        Ur = np.array([[u0, 0], [0, u1]], dtype=np.int64)
        re = np.array([p0, p1], dtype=np.int64)
        # the imaginary parts mirror the real ones: acc_im = u_l im_l, same boundaries
        out_r, out_i = F.apply_gate_q(re.copy(), re.copy(), 1, Ur, z, [0])
        assert out_r.tolist() == [o0, o1], (u0, p0, u1, p1, out_r)
        assert out_i.tolist() == [o0, o1]
    U4 = np.zeros((4, 4), dtype=np.int64)
    U4[0, :] = 1 << 29
    U4[1, :] = -(1 << 29)
    big = np.full(4, 1 << 29, dtype=np.int64)
    out_r, out_i = F.apply_gate_q(big.copy(), big.copy(), 2, U4, np.zeros((4, 4), dtype=np.int64), [0, 1])
    assert out_r.tolist() == [(1 << 31) - 1, -(1 << 31), 0, 0]
    assert out_i.tolist() == [(1 << 31) - 1, -(1 << 31), 0, 0]
    # a complex entry mixes the parts: (u_r + i u_i)(p_r + i p_i) with u = (2^13, 2^13),
    # psi = (2^14, -2^14 + 1): re acc = 2^27 + 2^27 - 2^13 = 2^28 - 2^13 -> 1 (rounded up from
    # 0.99997), im acc = 2^13 (-2^14 + 1) + 2^27 = 2^13 -> 0
    Ur = np.array([[1 << 13, 0], [0, 0]], dtype=np.int64)
    Ui = np.array([[1 << 13, 0], [0, 0]], dtype=np.int64)
    out_r, out_i = F.apply_gate_q(np.array([1 << 14, 0], dtype=np.int64),
                                  np.array([-(1 << 14) + 1, 0], dtype=np.int64), 1, Ur, Ui, [0])
    assert out_r.tolist() == [1, 0] and out_i.tolist() == [0, 0]


def test_q428_exact_permutations_and_signs():
    """X, CNOT, SWAP and CZ have entries 0 and +-1: in Q4.28 they permute and negate exactly."""
    from oracle import fixedpoint as F
    c = C.Circuit(3, [C.Gate("X", (0,)), C.Gate("CNOT", (0, 2)), C.Gate("SWAP", (1, 2)), C.Gate("CZ", (0, 1))],
                  init_basis=0)
    re, im = F.simulate_state_q428(c)
    # |000> -X0-> |100> -CNOT(0,2)-> |101> -SWAP(1,2)-> |110> -CZ(0,1)-> -|110>
    expect = np.zeros(8, dtype=np.int64)
    expect[0b110] = -(1 << 28)
    assert np.array_equal(re, expect) and not im.any()


def test_q428_hadamard_on_basis_is_the_quantised_entry():
    """H|0>: each output is Uq[i][0] * 2^28 rounded back, i.e. exactly quantize(1/sqrt 2)."""
    from oracle import fixedpoint as F
    re, im = F.simulate_state_q428(C.Circuit(1, [C.Gate("H", (0,))]))
    q = F.quantize(1.0 / np.sqrt(2.0))
    assert re.tolist() == [q, q] and not im.any()


@pytest.mark.parametrize("n,seed", [(1, 1), (3, 2), (6, 3), (9, 4)])
def test_q428_within_rounding_bound_of_fp64(n, seed):
    """Error bound: one gate adds at most 2^-29 per output component from rounding (2^-28.5 per
    complex amplitude) plus the matrix quantisation error (each entry within 2^-29 per part, so
    the operator error is at most d 2^-28.5 for a d x d gate, d <= 4); unitaries do not grow
    errors in the 2-norm.  So ||psi_q - psi|| <= G (2^(n/2) 2^-28.5 + 4 2^-28.5).  A dropped term,
    wrong sign or transposed operand gives an O(1) error."""
    from oracle import fixedpoint as F
    from oracle.statevector import simulate_state
    c = C.random_circuit(n, 15 * n + 5, 900 + seed)
    re, im = F.simulate_state_q428(c)
    err = np.linalg.norm(F.to_complex(re, im) - simulate_state(c))
    bound = len(c.gates) * (2.0 ** (n / 2) + 4.0) * 2.0 ** -28.5
    assert err <= bound, (err, bound)
    assert err > 0 or n == 1  # rounding does happen
