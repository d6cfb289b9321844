"""Guard words around every output buffer and workspace (GPU).

Each buffer a call may write sits inside a larger allocation whose bytes before and after it are
set to a sentinel pattern; after the call the guards must be unchanged (no write outside the
buffer's extent, and no workspace use beyond the size the library asks for).  The results
themselves are checked by the parity tests; here only the guards are.
"""
import numpy as np
import pytest

from paper_2108_06831_gb300 import circuits as C

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GUARD = 64 << 10  # bytes on each side (a multiple of 256, so the buffer keeps its alignment)
SENTINEL = 0xA5


class Guarded:
    """nbytes of device memory with sentinel guards on both sides."""

    def __init__(self, nbytes: int):
        self.nbytes = max(int(nbytes), 16)
        self.raw = torch.full((self.nbytes + 2 * GUARD,), SENTINEL, dtype=torch.uint8, device="cuda")
        self.buf = self.raw[GUARD:GUARD + self.nbytes]

    def view(self, dtype, shape):
        return self.buf.view(dtype).view(shape)

    def intact(self) -> bool:
        torch.cuda.synchronize()
        return bool((self.raw[:GUARD] == SENTINEL).all()) and bool((self.raw[GUARD + self.nbytes:] == SENTINEL).all())


def _ok():
    from paper_2108_06831_gb300 import tn
    torch.cuda.synchronize()
    assert tn.sync_status() == tn.OK


@pytest.mark.parametrize("n,tile", [(9, 0), (14, 7), (17, 0)])
def test_state_contraction(n, tile):
    from paper_2108_06831_gb300 import tn
    c, p = C.brickwork(n, 6, 40 + n, parameterized=True)
    plan = tn.Plan(tn.CircuitHandle(c), batch=2, tile_qubits=tile)
    st = Guarded(2 * 8 << n)
    ws = Guarded(plan.workspace_bytes)
    params = torch.as_tensor(np.stack([p, p[::-1].copy()]), device="cuda")
    tn.contract_state(plan, params, st.view(torch.complex64, (2, 1 << n)), ws.buf)
    _ok()
    assert st.intact() and ws.intact()


@pytest.mark.parametrize("cap", [0, 12])
def test_network_amplitudes(cap):
    """Network contraction, uncapped and under a cap (bitstring passes, slices, FP64 slice sum)."""
    from paper_2108_06831_gb300 import tn
    c = C.grid(4, 4, 8, 11)
    plan = tn.Plan(tn.CircuitHandle(c), target=tn.TARGET_AMPLITUDES, network_bitstrings=16,
                   precision=tn.PREC_3XTF32, max_intermediate_log2=cap)
    xs = torch.as_tensor(C.random_bitstrings(16, 13, 5).astype(np.int64), device="cuda")
    amps = Guarded(13 * 8)
    ws = Guarded(plan.workspace_bytes)
    tn.contract_amplitudes(plan, None, xs, amps.view(torch.complex64, (13,)), ws.buf)
    _ok()
    assert amps.intact() and ws.intact()


@pytest.mark.parametrize("prec,shape", [(0, (3, 130, 9, 17)), (0, (1, 3, 5, 3000)), (0, (1, 128, 64, 4096)),
                                        (1, (2, 256, 64, 64)), (1, (1, 384, 256, 256)), (2, (2, 128, 128, 64))])
def test_batched_gemm(prec, shape):
    """Every form of kernel (c): ragged FP32, split K (few and many outputs), 3xTF32 streaming and
    prep-split, split BF16."""
    from paper_2108_06831_gb300 import tn
    b, M, N, K = shape
    g = torch.Generator(device="cuda").manual_seed(sum(shape))
    A = torch.randn((b, M, K), dtype=torch.complex64, device="cuda", generator=g)
    B = torch.randn((b, N, K), dtype=torch.complex64, device="cuda", generator=g)
    out = Guarded(b * M * N * 8)
    wsb = tn.cgemm_workspace_bytes(prec, b, M, N, K)
    ws = Guarded(wsb)
    tn.cgemm_batched(prec, b, M, N, K, A, B, out.view(torch.complex64, (b, M, N)), ws.buf, wsb)
    _ok()
    assert out.intact() and ws.intact()


def test_permute():
    from paper_2108_06831_gb300 import tn
    n = 20
    x = torch.randn(2 << n, dtype=torch.complex64, device="cuda")
    out = Guarded(2 * 8 << n)
    perm = [int(v) for v in np.random.default_rng(3).permutation(n)]
    tn.permute(n, perm, 2, x, out.view(torch.complex64, (2 << n,)))
    _ok()
    assert out.intact()


def test_expectation_value_and_grad():
    from paper_2108_06831_gb300 import tn
    n = 10
    c = C.hea(n, 3)
    plan = tn.Plan(tn.CircuitHandle(c), target=tn.TARGET_EXPECTATION, batch=3)
    obs = tn.Observable(C.tfim(n))
    params = torch.as_tensor(C.hea_params(c.n_params, 3, 77), device="cuda")
    e = Guarded(3 * 8)
    gr = Guarded(3 * c.n_params * 8)
    ws = Guarded(plan.workspace_bytes)
    tn.expectation_value_and_grad(plan, obs, params, e.view(torch.float64, (3,)),
                                  gr.view(torch.float64, (3, c.n_params)), ws.buf)
    _ok()
    assert e.intact() and gr.intact() and ws.intact()


def test_batched_executor():
    from paper_2108_06831_gb300 import tn
    circs = [C.brickwork(n, 4, 90 + n)[0] for n in (6, 9, 13, 15)]
    bat = tn.Batch([tn.Plan(tn.CircuitHandle(c), specialize=False) for c in circs])
    st = Guarded(bat.state_elems * 8)
    ws = Guarded(bat.workspace_bytes)
    tn.batch_run(bat, st.view(torch.complex64, (bat.state_elems,)), ws.buf)
    _ok()
    assert st.intact() and ws.intact()


def test_q428_state():
    from paper_2108_06831_gb300 import tn
    n = 15
    plan = tn.Plan(tn.CircuitHandle(C.random_circuit(n, 60, 8)), q428=True)
    st = Guarded(8 << n)
    tn.contract_state_q428(plan, st.view(torch.int32, (1 << n, 2)))
    _ok()
    assert st.intact()
