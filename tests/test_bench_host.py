"""Host-side pieces of bench.py on the CPU: the algorithmic work counts that the
roofline numbers divide by, checked against independent enumerations, and the
parsing of the nvidia-smi clock samples that decides whether a run is kept."""
import itertools

import bench


def _multi_indices(k):
    return [(a, b, k - a - b) for a in range(k + 1) for b in range(k + 1 - a)]


def _m2l_terms_enumerated(s, p, want_phi):
    """Pairs (n, m) with |m| >= s, |n| >= (0 if the potential is wanted else 1)
    and |n| + |m| <= p + s, counted by listing the multi-indices."""
    lo = 0 if want_phi else 1
    count = 0
    for kn in range(lo, p + 1):
        for km in range(s, p + s - kn + 1):
            count += len(_multi_indices(kn)) * len(_multi_indices(km))
    return count


def test_m2l_term_counts_match_enumeration():
    for s, p, phi in itertools.product((0, 1, 2), (1, 4, 6, 9), (False, True)):
        assert bench.m2l_macs_per_pair(s, p, phi) == _m2l_terms_enumerated(s, p, phi), (s, p, phi)
    # the full Cartesian dipole field-only M2L at p = 6 quoted with the results
    assert bench.m2l_macs_per_pair(1, 6, False) == 1477


def test_pair_flop_counts_quoted_with_the_results():
    assert bench.flops_per_pair(1, False, True) == 31          # dipole field
    assert bench.flops_per_pair(0, False, True) + bench.flops_per_pair(1, False, True) == 49
    for s in (0, 1, 2):                                        # more outputs never cost less
        f = bench.flops_per_pair(s, False, True)
        assert bench.flops_per_pair(s, True, True) > f > 0
        assert bench.flops_per_pair(s, True, False) < bench.flops_per_pair(s, True, True)


def test_m2p_flops_grow_with_order_and_outputs():
    for s in (0, 1, 2):
        prev = 0
        for p in range(max(s, 1), 9):
            f = bench.m2p_flops(s, p, False, True)
            assert f > prev
            assert bench.m2p_flops(s, p, True, True) > f
            prev = f


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(lines):
    cs = bench.ClockSampler(0)
    cs.proc = _FakeProc()
    cs.lines = list(lines)
    return cs


def test_clock_sampler_median_and_reasons(monkeypatch):
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)
    idle = "Not Active"
    lines = ["0, 2070, 2070, 900.1, 0x0, %s, %s, %s, %s" % (idle, idle, idle, idle),
             "0, 2055, 2070, 1390.5, 0x4, %s, %s, %s, Active" % (idle, idle, idle),
             "0, 2070, 2070, 1201.0, 0x0, %s, %s, %s, %s" % (idle, idle, idle, idle),
             "garbage line"]
    out = _sampler(lines).stop()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3


def test_clock_sampler_reports_thermal_slowdown(monkeypatch):
    monkeypatch.setattr(bench.time, "sleep", lambda s: None)
    lines = ["0, 1500, 2070, 1000.0, 0x40, Not Active, Active, Not Active, Not Active"]
    out = _sampler(lines).stop()
    assert out["reasons"] == ["hw_thermal_slowdown"] and out["sm_mhz"] == 1500.0


def test_clock_sampler_without_nvidia_smi():
    out = bench.ClockSampler(0).stop()
    assert out["sm_mhz"] is None and out["reasons"] == ["nvidia-smi unavailable"]


def test_reference_arm_line_on_the_small_workload(orc, capsys):
    """bench.py --impl reference times the oracle and prints the contract's line;
    its value counts the particles one step evaluated (all 2,000 here)."""
    import json
    assert bench.main(["--impl", "reference", "--workload", "monopole_2k_p4", "--steps", "2",
                       "--warmup", "1"]) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 1
    assert line["unit"] == "particles/s" and line["higher_is_better"] is True
    assert abs(line["value"] - 2000 / (line["ms_per_step"] / 1e3)) < 1e-6 * line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    assert "all 2000 particles" in cb["sample"]


def test_full_rate_fit_recovers_fixed_and_per_particle_costs():
    """The reference arm's step times t(k) = fixed + per * k at two sample sizes
    give the oracle's rate on the whole workload, n / (fixed + per * n)."""
    fixed, per, n = 3.0, 1.25e-5, 1_000_000
    counts = [32768, 131072] * 3
    times = [fixed + per * k for k in counts]
    value, f, p = bench.fit_full_rate(counts, times, n)
    assert abs(f - fixed) < 1e-9 and abs(p - per) < 1e-15
    assert abs(value - n / (fixed + per * n)) < 1e-6 * value
    # one sample size: the plain sampled rate
    assert bench.fit_full_rate([5000, 5000], [1.0, 1.0], n)[0] == 5000.0
