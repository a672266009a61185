"""Host-side statistics of Tables 2 and 3 (Sec. III) on constructed inputs
with hand-computed answers."""
import numpy as np
import pytest

from paper_0807_0264_gb300.analysis import transition_tables


def test_transition_tables_hand_computed():
    # 4 configurations, 3 levels
    V = [[0.80, 0.81, 0.82],
         [0.80, 0.79, 0.83],
         [0.80, 0.81, 0.81],
         [0.80, 0.82, 0.80]]
    n = [[100, 50, 40],
         [100, 120, 60],
         [100, 80, 80],
         [100, 100, 90]]
    t = transition_tables(V, n)
    f, r, h, g = t["fewer_vortices_pct"], t["vortex_reduction_pct"], t["higher_max_pct"], t["fewer_given_higher_pct"]
    # level 0 -> 1: fewer vortices in configs 0, 2 (50 %); reductions 50 %, 20 % -> mean 35
    assert f[0, 1] == 50.0 and r[1, 0] == pytest.approx(35.0) and t["vortex_reduction_std"][1, 0] == pytest.approx(15.0)
    # level 0 -> 2: all four fewer; reductions 60, 40, 20, 10 -> mean 32.5
    assert f[0, 2] == 100.0 and r[2, 0] == pytest.approx(32.5)
    # level 1 -> 2: configs 0 (50->40), 1 (120->60), 3 (100->90) fewer; 2 equal -> 75 %
    assert f[1, 2] == 75.0 and r[2, 1] == pytest.approx((20 + 50 + 10) / 3)
    # higher maxima 0 -> 1: configs 0, 2, 3 (75 %); of those fewer vortices: 0, 2 -> 66.67 %
    assert h[0, 1] == 75.0 and g[1, 0] == pytest.approx(200 / 3)
    # 1 -> 2: higher in configs 0 (0.82 > 0.81), 1 (0.83 > 0.79); both fewer -> 100 %
    assert h[1, 2] == 50.0 and g[2, 1] == 100.0
    # diagonal and the unused triangles stay NaN
    assert np.isnan(f[1, 0]) and np.isnan(h[2, 2]) and np.isnan(r[0, 1])


def test_transition_tables_no_reductions():
    t = transition_tables([[1, 1], [1, 1]], [[5, 5], [5, 6]])
    assert t["fewer_vortices_pct"][0, 1] == 0.0 and np.isnan(t["vortex_reduction_pct"][1, 0])
    assert t["higher_max_pct"][0, 1] == 0.0 and np.isnan(t["fewer_given_higher_pct"][1, 0])
    with pytest.raises(ValueError):
        transition_tables([[1, 2]], [[1, 2, 3]])
