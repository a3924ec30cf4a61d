"""The paper's experiments as synthetic GPU runs (small sizes): E3's error
distributions fall with p and are smaller at theta 0.25 than at 0.5; E2's
runtime grows about linearly in N and the FMM beats the direct sum at large N."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("method", ["fmm", "bh"])
def test_e3_error_falls_with_order(method):
    from paper_2005_12351_gb300 import experiments
    res = list(experiments.e3(n=6_000, thetas=(0.25, 0.5), orders=(1, 3, 5, 7), methods=(method,)))
    assert all(r["method"] == method for r in res)
    med = {(r["theta"], r["p"]): r["potential_error"]["median"] for r in res}
    rms = {(r["theta"], r["p"]): r["field_error"]["rel_rms"] for r in res}
    for th in (0.25, 0.5):
        m = [med[(th, p)] for p in (1, 3, 5, 7)]
        assert all(a > b for a, b in zip(m, m[1:])), m
        f = [rms[(th, p)] for p in (1, 3, 5, 7)]
        assert all(a > b for a, b in zip(f, f[1:])), f
    for p in (1, 3, 5, 7):
        assert med[(0.25, p)] < med[(0.5, p)]
    r0 = res[0]["potential_error"]
    assert sum(r0["log10_hist"]["counts"]) == 6_000


def test_e2_scaling_bh():
    from paper_2005_12351_gb300 import experiments
    res = list(experiments.e2(nmin=20_000, nmax=320_000, points=3, thetas=(0.5,), orders=(4,),
                              direct_max=0, methods=("bh",)))
    t = [r["ms_evaluate"] for r in res]
    assert [r["method"] for r in res] == ["bh"] * 3
    assert t[0] < t[1] < t[2] and t[-1] / t[0] < 64


def test_e2_scaling():
    from paper_2005_12351_gb300 import experiments
    res = list(experiments.e2(nmin=20_000, nmax=320_000, points=3, thetas=(0.5,), orders=(4,),
                              direct_max=320_000, methods=("fmm",)))
    ns = [r["n"] for r in res]
    t = [r["ms_evaluate"] for r in res]
    assert ns == sorted(ns) and len(ns) == 3
    # 16x more particles: evaluate time grows sub-quadratically (O(N) up to tree-depth steps)
    assert t[-1] / t[0] < 64
    assert res[-1]["ms_direct"] > res[-1]["ms_whole"]
