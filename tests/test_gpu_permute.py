"""Kernel (b) permutation against numpy transposes (bit-exact: it only moves data)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _ref(x, n, perm):
    t = x.reshape((-1,) + (2,) * n)
    return np.ascontiguousarray(np.transpose(t, [0] + [1 + p for p in perm])).reshape(x.shape)


@pytest.mark.parametrize("n,batch,seed", [(1, 3, 0), (3, 2, 1), (4, 1, 2), (5, 2, 3), (6, 1, 4), (9, 3, 5),
                                          (12, 2, 6), (16, 1, 7), (20, 1, 8), (22, 2, 9)])
def test_random_permutations(n, batch, seed):
    from paper_2108_06831_gb300 import tn
    rng = np.random.default_rng(seed)
    for _ in range(3):
        perm = [int(v) for v in rng.permutation(n)]
        x = (rng.normal(size=(batch, 1 << n)) + 1j * rng.normal(size=(batch, 1 << n))).astype(np.complex64)
        xin = torch.as_tensor(x, device="cuda")
        out = torch.empty_like(xin)
        tn.permute(n, perm, batch, xin, out)
        torch.cuda.synchronize()
        assert tn.sync_status() == tn.OK
        assert np.array_equal(out.cpu().numpy(), _ref(x, n, perm))


def test_identity_and_reversal_24():
    from paper_2108_06831_gb300 import tn
    n = 24
    x = torch.randn(1 << n, dtype=torch.complex64, device="cuda")
    for perm in (list(range(n)), list(range(n))[::-1]):
        out = torch.empty_like(x)
        tn.permute(n, perm, 1, x, out)
        torch.cuda.synchronize()
        ref = x.reshape((2,) * n).permute(*perm).contiguous().reshape(-1)
        assert torch.equal(out, ref)


def test_rejects_bad_perm():
    from paper_2108_06831_gb300 import tn
    x = torch.zeros(16, dtype=torch.complex64, device="cuda")
    y = torch.zeros(16, dtype=torch.complex64, device="cuda")
    with pytest.raises(tn.TnError):
        tn.permute(4, [0, 1, 1, 2], 1, x, y)
    with pytest.raises(tn.TnError):
        tn.permute(4, [0, 1, 2, 3], 1, x, x)
