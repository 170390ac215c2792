"""boruta_quantise against its definition, bin = min(B-1, floor(B rank/N))
with rank = number of strictly smaller values (the numpy statement of it in
synth.quantise): ties, negative zero, ragged N, two and 256 bins."""
import numpy as np
import pytest

from paper_2605_09950_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,p,B", [(1, 3, 2), (17, 5, 2), (1000, 7, 64), (4099, 6, 256), (100_000, 3, 256)])
def test_quantise_matches_rank_definition(N, p, B):
    import torch

    from paper_2605_09950_gb300 import boruta

    rng = np.random.default_rng(N * 31 + B)
    F = rng.standard_normal((p, N)).astype(np.float32)
    F[0] = np.round(F[0] * 3) / 3  # heavy ties
    if p > 2:
        F[1] = rng.integers(0, 3, size=N).astype(np.float32)  # three values (genotype-like)
        F[2, : N // 2] = -0.0
        F[2, N // 2 :] = 0.0
    got = boruta.boruta_quantise(torch.from_numpy(F).cuda(), B).cpu().numpy()
    want = synth.quantise(F.astype(np.float64), B)
    np.testing.assert_array_equal(got, want)


def test_quantise_rejects_nan_and_bad_bins():
    import torch

    from paper_2605_09950_gb300 import boruta

    F = torch.zeros((2, 10), dtype=torch.float32, device="cuda")
    with pytest.raises(boruta.BorutaError, match="n_bins"):
        boruta.boruta_quantise(F, 1)
    F[1, 3] = float("nan")
    with pytest.raises(boruta.BorutaError, match="NaN"):
        boruta.boruta_quantise(F, 8)
