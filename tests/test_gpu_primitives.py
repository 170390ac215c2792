"""Device primitives through the C ABI against the oracle and Python's exact
arithmetic: Philox, the Feistel permutation, u256 -> double rounding and the
binomial tails of the Boruta test."""
import math
from fractions import Fraction

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import torch

    import __graft_entry__

    __graft_entry__.build()
    assert torch.cuda.is_available()
    return torch.device("cuda:0")


def test_philox_matches_oracle(dev):
    import torch

    import oracle
    from paper_2605_09950_gb300 import boruta

    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2**32, size=(5000, 4), dtype=np.uint64).astype(np.uint32)
    ctr[0] = 0
    ctr[1] = 0xFFFFFFFF
    for key in ([0, 0], [0xFFFFFFFF, 0xFFFFFFFF], [0xA4093822, 0x299F31D0], [123, 456]):
        k = np.array(key, np.uint32)
        got = boruta.boruta_philox(torch.from_numpy(ctr.view(np.int32)).to(dev).contiguous(),
                                   torch.from_numpy(k.view(np.int32)).to(dev)).cpu().numpy().view(np.uint32)
        want = np.stack([oracle.philox(c, k) for c in ctr[:300]])
        np.testing.assert_array_equal(got[:300], want)
    # the published known answer, through the GPU
    c = torch.zeros(4, dtype=torch.int32, device=dev)
    out = boruta.boruta_philox(c, torch.zeros(2, dtype=torch.int32, device=dev)).cpu().numpy().view(np.uint32)
    assert [hex(v) for v in out] == ["0x6627e8d5", "0xe169c58d", "0xbc57ac4c", "0x9b00dbd8"]


@pytest.mark.parametrize("n", [1, 2, 3, 5, 17, 64, 65, 1000, 100_003, 1 << 20])
def test_perm_matches_oracle(dev, n):
    import torch

    import oracle
    from paper_2605_09950_gb300 import boruta

    idx = np.arange(min(n, 200_000), dtype=np.uint64)
    got = boruta.boruta_perm(n, 77, 3, 1 << 24, 2 << 24,
                             torch.from_numpy(idx.view(np.int64)).to(dev)).cpu().numpy().view(np.uint64)
    np.testing.assert_array_equal(got, oracle.perm(n, 77, 3, 1 << 24, 2 << 24, idx))
    if n <= 200_000:
        assert np.array_equal(np.sort(got), idx)


def test_u256_to_double_rounding(dev):
    import torch

    from paper_2605_09950_gb300 import boruta

    vals = [0, 1, 2**53 - 1, 2**53, 2**53 + 1, 2**53 + 3, 2**54 + 2, 2**64 - 1, 2**127 + 2**74,
            2**127 + 2**74 + 1, 2**255 + 1, 2**256 - 1, ((2**53 - 1) << 100) + (1 << 99)]
    rng = np.random.default_rng(5)
    for _ in range(5000):
        vals.append((int(rng.integers(1, 2**63)) << int(rng.integers(0, 190))) + int(rng.integers(0, 2**63)))
    limbs = np.array([[(v >> (64 * i)) & (2**64 - 1) for i in range(4)] for v in vals], dtype=np.uint64)
    got = boruta.boruta_u256_to_double(torch.from_numpy(limbs.view(np.int64)).to(dev).reshape(-1)).cpu().numpy()
    for v, g in zip(vals, got):
        assert g == float(v), hex(v)


def test_binomial_tails(dev):
    import torch

    from paper_2605_09950_gb300 import boruta

    ts, hs = [], []
    for t in (1, 2, 13, 17, 64, 100, 126):
        for h in range(t + 1):
            ts.append(t)
            hs.append(h)
    t = torch.tensor(ts, dtype=torch.int32, device=dev)
    h = torch.tensor(hs, dtype=torch.int32, device=dev)
    pa, pr = boruta.boruta_binom_tails(t, h)
    for tt, hh, a, r in zip(ts, hs, pa.cpu().numpy(), pr.cpu().numpy()):
        up = sum(math.comb(tt, k) for k in range(hh, tt + 1))
        lo = sum(math.comb(tt, k) for k in range(0, hh + 1))
        assert a == float(Fraction(up, 2**tt)) and r == float(Fraction(lo, 2**tt))


def test_binomial_tails_rejects_bad_t(dev):
    import torch

    from paper_2605_09950_gb300 import boruta

    t = torch.tensor([127], dtype=torch.int32, device=dev)
    with pytest.raises(boruta.BorutaError):
        boruta.boruta_binom_tails(t, t)
