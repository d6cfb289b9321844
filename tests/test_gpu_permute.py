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


@pytest.mark.parametrize("n", [5, 6, 7, 8, 11, 14, 20])
@pytest.mark.parametrize("n_low_moved", [0, 1, 2, 5])
def test_low_leg_classes(n, n_low_moved):
    """Permutations that move exactly `n_low_moved` of the five fastest legs (tiles whose rows
    mix transposed and passive legs), batch 2."""
    from paper_2108_06831_gb300 import tn
    if n_low_moved and n < 5 + n_low_moved:
        pytest.skip("not enough slow legs to swap with")
    rng = np.random.default_rng(100 * n + n_low_moved)
    perm = list(range(n))
    high = perm[: n - 5]
    rng.shuffle(high)
    perm[: n - 5] = high
    low_pos = list(rng.choice(np.arange(n - 5, n), size=n_low_moved, replace=False))
    high_pos = list(rng.choice(np.arange(0, n - 5), size=n_low_moved, replace=False))
    for a, b in zip(low_pos, high_pos):
        perm[a], perm[b] = perm[b], perm[a]
    perm = [int(v) for v in perm]
    x = (rng.normal(size=(2, 1 << n)) + 1j * rng.normal(size=(2, 1 << n))).astype(np.complex64)
    xin = torch.as_tensor(x, device="cuda")
    out = torch.empty_like(xin)
    tn.permute(n, perm, 2, xin, out)
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
