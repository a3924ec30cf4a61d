"""Continuous-batching server: each result is the same alone and in a concurrent mix;
admission respects the device-memory budget."""
import numpy as np
import pytest
from gpu_util import close

from paper_2005_12351_gb300 import synth

pytestmark = pytest.mark.gpu


def request_mix(count, seed, nmax=60_000):
    """Mixed requests: N log-uniform, s in {0,1,2}, p in {4..10}, uniform/Plummer."""
    sizes = synth.log_uniform_int(count, 1000, nmax, seed)
    u = synth.uniform01(seed, 17, 3 * count).reshape(count, 3)
    out = []
    for k in range(count):
        s = int(u[k, 0] * 3)
        p = 4 + int(u[k, 1] * 7)
        dist = "plummer" if u[k, 2] < 0.5 else "uniform"
        pos, mom = synth.make_system(int(sizes[k]), s, dist, seed * 31 + k)
        out.append(dict(positions=pos, moments=mom, source_order=s, p=p, max_leaf=64))
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32", "3xtf32"])
def test_results_same_alone_and_in_mix(precision):
    from paper_2005_12351_gb300 import fmm
    reqs = request_mix(10, 5)
    alone = []
    with_one = fmm.Server(slots=1, precision=precision)
    for r in reqs:
        t = with_one.submit(**r)
        alone.append(with_one.wait(t)[:2])
    with_one.close()
    mix = fmm.Server(slots=4, precision=precision)
    tickets = [mix.submit(**r) for r in reqs]
    slots_used, overlap = set(), 0
    outs = []
    for t in tickets:
        phi, E, info = mix.wait(t)
        outs.append((phi, E, info))
        slots_used.add(info["slot"])
    spans = sorted((o[2]["start_s"], o[2]["end_s"]) for o in outs)
    overlap = sum(1 for a, b in zip(spans, spans[1:]) if b[0] < a[1])
    assert len(slots_used) > 1 and overlap > 0          # the mix did run concurrently
    for (phi_a, E_a), (phi_m, E_m, _) in zip(alone, outs):
        assert np.array_equal(phi_a, phi_m) and np.array_equal(E_a, E_m)
    mix.close()


def test_server_matches_handle_api(orc):
    from gpu_util import rel_rms
    from paper_2005_12351_gb300 import fmm
    r = request_mix(1, 9)[0]
    sv = fmm.Server(slots=2)
    phi, E, _ = sv.wait(sv.submit(**r))
    sv.close()
    t = orc.Tree(r["positions"], 64)
    t.lists(0.5)
    phi_o, E_o = t.fmm(r["moments"], r["source_order"], r["p"])
    assert close(phi, phi_o, 1e-12) and close(E, E_o, 1e-12)


def test_admission_respects_budget():
    from paper_2005_12351_gb300 import fmm
    reqs = request_mix(8, 13, nmax=200_000)
    budget = 700 << 20
    sv = fmm.Server(slots=4, mem_budget_bytes=budget)
    tickets = [sv.submit(**r) for r in reqs]
    for t in tickets:
        sv.wait(t)
    st = sv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert 0 < st["peak_device_bytes"] <= budget
    with pytest.raises(fmm.FMMError) as ei:           # could never fit
        big, mom = synth.make_system(3_000_000, 0, "uniform", 3)
        sv.submit(big, mom, 0, 10)
    assert ei.value.status == fmm.FMM_EBUDGET
    sv.close()
