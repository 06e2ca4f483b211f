"""The Wilson interval against scipy's binomial test (an independent library)."""
import pytest

from paper_2509_17837_gb300.stats import ler_record, wilson_interval


@pytest.mark.parametrize("k,n", [(0, 10), (3, 10), (50, 100), (999, 1000), (1000, 1000), (17, 100000)])
def test_wilson_matches_scipy(k, n):
    stats = pytest.importorskip("scipy.stats")
    ci = stats.binomtest(k, n).proportion_ci(confidence_level=0.95, method="wilson")
    lo, hi = wilson_interval(k, n)
    assert lo == pytest.approx(ci.low, abs=1e-12) and hi == pytest.approx(ci.high, abs=1e-12)


def test_record():
    r = ler_record(0.1, 5, 100)
    assert r["ler"] == 0.05 and r["ci95"][0] < 0.05 < r["ci95"][1]
