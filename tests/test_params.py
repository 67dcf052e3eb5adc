"""The parameter chooser (rambo_suggest_params) against the paper's formulas.

Host-only: B from Lemma 4.4's optimum sqrt(K V / eta), R the smallest value
meeting Lemma 4.2's failure bound, m and eta from Bloom-filter sizing."""
import math

import pytest


def test_suggested_parameters_follow_lemmas_4_2_and_4_4():
    from paper_1910_02611_gb300 import suggest_params

    for K, n_mean, V, p, delta in [(2000, 1e6, 2.0, 0.01, 0.01), (100, 1e4, 1.0, 0.05, 0.1),
                                   (10**5, 500, 20.0, 0.01, 0.05)]:
        got = suggest_params(K, n_mean, V, p, delta)
        eta0 = min(max(math.log(1 / p) / math.log(2), 1), 4)
        assert got["B"] == min(max(round(math.sqrt(K * V / eta0)), 2), 4096)
        B = got["B"]
        f = 1 - (1 - p) * (1 - 1 / B) ** V
        R = got["R"]
        assert K * f ** R <= delta  # Lemma 4.2 bound met ...
        assert R == 1 or K * f ** (R - 1) > delta  # ... by the smallest R
        n = n_mean * K / B
        m = got["m"]
        assert m & (m - 1) == 0 and m >= n * math.log(1 / p) / math.log(2) ** 2 > m / 2
        assert got["eta"] == min(max(round(math.log(2) * m / n), 1), 4)


def test_unreachable_failure_rate_reports_erange():
    from paper_1910_02611_gb300 import ERANGE, RamboError, suggest_params

    with pytest.raises(RamboError) as e:
        suggest_params(10**6, 1000, V=500.0, p=0.2, delta=1e-9)
    assert e.value.code == ERANGE and e.value.params["R"] == 8
