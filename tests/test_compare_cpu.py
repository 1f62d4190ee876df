"""The parity comparison (tests/_util.compare) itself: the tolerance, the
flip audit (an element beyond the tolerance must sit within FLIP_EPS of a
decision threshold, else it fails) and the budget, counted per element or,
with groups, per flipped Gaussian."""
import numpy as np
import pytest

from tests._util import FLIP_EPS, compare


def _case():
    ref = np.linspace(1.0, 2.0, 96)
    got = ref * (1 + 1e-7)
    return ref, got


def test_within_tolerance_passes():
    ref, got = _case()
    info = compare("x", got, ref, 1e-5, 0.0, 1e-5)
    assert info["bad"] == 0


def test_excess_far_from_every_threshold_fails():
    ref, got = _case()
    got[10] *= 1.01
    margins = np.full(ref.size, 0.5)  # every decision far from its threshold
    with pytest.raises(AssertionError, match="away from every threshold"):
        compare("x", got, ref, 1e-5, 0.0, 1e-2, flip_budget=5, margins=margins, kinds=np.zeros(ref.size, int))


def test_explained_flips_count_against_the_budget():
    ref, got = _case()
    got[[3, 50]] *= 1.01
    margins = np.full(ref.size, 0.5)
    margins[[3, 50]] = 0.1 * FLIP_EPS
    kinds = np.zeros(ref.size, int)
    info = compare("x", got, ref, 1e-5, 0.0, 1e-2, flip_budget=2, margins=margins, kinds=kinds)
    assert info["bad"] == 2 and all(f["kind"] == "q = 9" for f in info["flips"])
    with pytest.raises(AssertionError, match="flips"):
        compare("x", got, ref, 1e-5, 0.0, 1e-2, flip_budget=1, margins=margins, kinds=kinds)


def test_grouped_budget_counts_gaussians():
    """48 SH elements per Gaussian: seven elements of one Gaussian beyond the
    tolerance are one flip; the same count spread over two Gaussians is two."""
    per, n_g = 48, 2
    ref = np.linspace(1.0, 2.0, per * n_g)
    got = ref.copy()
    margins = np.full(ref.size, 0.5)
    one = np.arange(10, 17)
    got[one] *= 1.01
    margins[:per] = 0.1 * FLIP_EPS
    groups = np.repeat(np.arange(n_g), per)
    info = compare("sh", got, ref, 1e-5, 0.0, 1e-2, flip_budget=1, margins=margins,
                   kinds=np.zeros(ref.size, int), groups=groups)
    assert info["bad"] == 7 and info["flipped_groups"] == 1
    got[per + 3] *= 1.01
    margins[per:] = 0.1 * FLIP_EPS
    with pytest.raises(AssertionError, match="flips"):
        compare("sh", got, ref, 1e-5, 0.0, 1e-2, flip_budget=1, margins=margins,
                kinds=np.zeros(ref.size, int), groups=groups)
