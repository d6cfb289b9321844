"""Kernel (c): batched complex GEMM against an FP64 product (GPU).

C[b][m][n] = sum_k A[b][m][k] B[b][n][k].  Bar: relative Frobenius error <= 1e-5 for
every precision (plain FP32 on CUDA cores, 3xTF32 and 3-way split BF16 on tcgen05).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-5


def _tn():
    from paper_2108_06831_gb300 import tn
    return tn


def _run(prec, batch, M, N, K, seed=0, scale=1.0):
    tn = _tn()
    rng = np.random.default_rng(seed)
    A = (rng.normal(size=(batch, M, K)) + 1j * rng.normal(size=(batch, M, K))) * scale
    B = (rng.normal(size=(batch, N, K)) + 1j * rng.normal(size=(batch, N, K))) * scale
    a = torch.as_tensor(A.astype(np.complex64), device="cuda")
    b = torch.as_tensor(B.astype(np.complex64), device="cuda")
    c = torch.full((batch, M, N), complex(float("nan"), 0), dtype=torch.complex64, device="cuda")
    wsb = tn.cgemm_workspace_bytes(prec, batch, M, N, K)
    ws = torch.empty(max(wsb, 16), dtype=torch.uint8, device="cuda")
    tn.cgemm_batched(prec, batch, M, N, K, a, b, c, ws, wsb)
    torch.cuda.synchronize()
    assert tn.sync_status() == tn.OK
    # reference from the complex64 inputs the GPU saw, in complex128
    ref = np.einsum("bmk,bnk->bmn", A.astype(np.complex64).astype(np.complex128),
                    B.astype(np.complex64).astype(np.complex128))
    got = c.cpu().numpy().astype(np.complex128)
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


@pytest.mark.parametrize("shape", [(1, 128, 64, 16), (2, 256, 128, 64), (3, 128, 192, 32), (1, 384, 256, 256)])
@pytest.mark.parametrize("prec", [0, 1, 2])
def test_cgemm_precisions(prec, shape):
    batch, M, N, K = shape
    assert _run(prec, batch, M, N, K, seed=sum(shape) + prec) <= TOL


@pytest.mark.parametrize("shape", [(2, 256, 64, 8), (1, 128, 128, 4), (3, 128, 64, 24), (1, 256, 256, 40)])
@pytest.mark.parametrize("prec", [1, 2])
def test_cgemm_k_not_a_tile_multiple(prec, shape):
    # K tiles partly (or, for split BF16, wholly) beyond K are zero-filled by the TMA
    assert _run(prec, *shape, seed=sum(shape) + 5 * prec) <= TOL


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_cgemm_deep_contraction(prec):
    # K = 4096: a long sum, where tensor-core accumulation truncates addends against the
    # running total; the split accumulators keep the error within the FP32 bar
    assert _run(prec, 1, 256, 128, 4096, seed=11 + prec) <= TOL


def test_cgemm_fp32_ragged_shapes():
    # the first four take the one-thread-per-output kernel (at most 2^18 multiply-adds), the last
    # three the tiled kernel with ragged edges in M, N and K
    for shape in [(1, 5, 7, 3), (2, 65, 33, 17), (1, 1, 1, 1), (3, 130, 70, 9),
                  (2, 300, 70, 20), (1, 1000, 9, 40), (1, 77, 200, 100)]:
        assert _run(0, *shape, seed=7) <= TOL


def test_cgemm_large_dynamic_range():
    # entries spanning several orders of magnitude: the split keeps FP32-level relative error
    assert _run(1, 1, 256, 128, 128, seed=3, scale=1e-3) <= TOL
    assert _run(2, 1, 256, 128, 128, seed=4, scale=1e3) <= TOL


def test_cgemm_unsupported_tensor_shape():
    tn = _tn()
    a = torch.zeros((1, 100, 16), dtype=torch.complex64, device="cuda")
    b = torch.zeros((1, 64, 16), dtype=torch.complex64, device="cuda")
    c = torch.zeros((1, 100, 64), dtype=torch.complex64, device="cuda")
    with pytest.raises(tn.TnError) as e:
        tn.cgemm_batched(1, 1, 100, 64, 16, a, b, c)
    assert e.value.status == tn.ERR_UNSUPPORTED


def test_cgemm_fp32_more_than_65535_row_tiles():
    """A tall, narrow product (8.4M rows, 3 columns, K 5: more than 65535 row tiles of 128 rows,
    ragged in every dimension), as operand exchange in network merges produces."""
    assert _run(0, 1, (1 << 23) + 200, 3, 5, seed=11) <= TOL


@pytest.mark.parametrize("shape", [(1, 1, 1, 65536), (3, 5, 7, 3000), (2, 130, 9, 1024), (1, 64, 64, 8192),
                                   (1, 128, 64, 4096)])
def test_cgemm_fp32_split_k(shape):
    """Few output tiles and a long K (a merge contracting two large operands into a small
    result): K is split over CTAs and the partials summed in a second kernel."""
    tn = _tn()
    batch, M, N, K = shape
    assert tn.cgemm_workspace_bytes(0, batch, M, N, K) > 0  # the split path is taken
    assert _run(0, batch, M, N, K, seed=sum(shape)) <= TOL


def test_block_diagonal_matricisation_is_the_batched_gemm():
    """Sec. 3 lays an order-(p, q) tensor out as one matrix: block_diag of its trailing d x d slices
    t[idx] over the leading indices.  Multiplying that block-diagonal matrix by a stacked operand
    is the batched GEMM with the leading indices as the batch (the form every network merge
    takes), with no zero block stored or multiplied."""
    scipy_linalg = pytest.importorskip("scipy.linalg")
    tn = _tn()
    rng = np.random.default_rng(31)
    t = rng.normal(size=(2, 2, 2, 4, 4)) + 1j * rng.normal(size=(2, 2, 2, 4, 4))
    mats = [t[idx] for idx in np.ndindex(t.shape[:-2])]
    X = rng.normal(size=(8 * 4, 6)) + 1j * rng.normal(size=(8 * 4, 6))
    ref = (scipy_linalg.block_diag(*mats) @ X).reshape(8, 4, 6)  # [block][row][column]
    a = torch.as_tensor(np.stack(mats).astype(np.complex64), device="cuda")                    # [b][m][k]
    b = torch.as_tensor(X.reshape(8, 4, 6).transpose(0, 2, 1).copy().astype(np.complex64), device="cuda")  # [b][n][k]
    c = torch.empty((8, 4, 6), dtype=torch.complex64, device="cuda")
    ws = torch.empty(16, dtype=torch.uint8, device="cuda")
    tn.cgemm_batched(0, 8, 4, 6, 4, a, b, c, ws, tn.cgemm_workspace_bytes(0, 8, 4, 6, 4))
    torch.cuda.synchronize()
    got = c.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= TOL
