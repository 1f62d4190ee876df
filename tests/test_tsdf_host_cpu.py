"""Host-side sizing of the TSDF grid: the band sample count the table is
sized with agrees with the oracle's band, and the power-of-two rounding."""
import numpy as np

from oracle import tsdf as T
from paper_2408_12677_gb300 import tsdf as G


def test_band_samples_match_the_oracle():
    rng = np.random.default_rng(0)
    cases = [(0.08, 0.01), (0.05, 0.01), (0.02, 0.01), (0.3, 0.01), (0.011, 0.02)]
    cases += [(float(rng.uniform(0.005, 0.3)), float(rng.uniform(0.004, 0.05))) for _ in range(200)]
    for eps, s in cases:
        assert G.band_samples(eps, s) == T.n_band_steps(eps, s) + 1 == len(T.band_offsets(eps, s))


def test_pow2():
    assert [G._pow2(n) for n in (1, 2, 3, 4, 5, 1000, 1024, 1025)] == [2, 2, 4, 4, 8, 1024, 1024, 2048]
