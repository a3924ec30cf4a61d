"""GPU FP64 FMM parity against the oracle (same tree), plus edge cases."""
import numpy as np
import pytest
from gpu_util import close

from paper_2005_12351_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12        # relative RMS, GPU FP64 form vs CPU FP64 oracle on the same tree


@pytest.mark.parametrize("s", [0, 1, 2])
def test_direct_sum_matches_oracle(orc, s):
    from gpu_util import rel_rms, to_dev
    from paper_2005_12351_gb300 import fmm
    pos, S = synth.make_system(3001, s, "plummer", 300 + s)
    phi, E = fmm.direct_sum(to_dev(pos), to_dev(S), s)
    phi_o, E_o = orc.direct(pos, S, s)
    assert close(phi.cpu().numpy(), phi_o, 1e-13)
    assert close(E.cpu().numpy(), E_o, 1e-13)
    tg = synth.sample_indices(3001, 37, 5)
    import torch
    phi2, E2 = fmm.direct_sum(to_dev(pos), to_dev(S), s, targets=to_dev(tg.astype(np.int32)))
    assert np.array_equal(phi2.cpu().numpy(), phi.cpu().numpy()[tg])
    torch.cuda.synchronize()


@pytest.mark.parametrize("s,p,dist,n,ncrit", [
    (0, 4, "uniform", 2000, 64),        # the 2k monopole workload
    (0, 1, "uniform", 9000, 32),
    (0, 9, "plummer", 6000, 24),
    (1, 6, "uniform", 20_000, 128),
    (1, 3, "plummer", 15_000, 32),
    (1, 8, "plummer", 8000, 64),
    (2, 5, "uniform", 12_000, 128),
    (2, 2, "plummer", 9000, 16),
    (2, 10, "uniform", 4000, 64),       # largest total order p + s = 12
])
def test_fmm_matches_oracle(orc, s, p, dist, n, ncrit):
    from gpu_util import gpu_fmm, rel_rms
    pos, S = synth.make_system(n, s, dist, 400 + 10 * s + p)
    (phi, E), tree = gpu_fmm(pos, S, s, p, 0.5, ncrit)
    t = orc.Tree(pos, ncrit)
    t.lists(0.5)
    phi_o, E_o = t.fmm(S, s, p)
    assert close(phi, phi_o, TOL), rel_rms(phi, phi_o)
    assert close(E, E_o, TOL), rel_rms(E, E_o)
    tree.destroy()


def test_monopole_2k_against_direct(orc):
    """2,000 monopoles, p=4: the GPU error vs the FP64 direct sum is the oracle's truncation error."""
    from gpu_util import gpu_fmm, rel_rms
    w = synth.WORKLOADS["monopole_2k_p4"]
    pos, S = synth.make_system(w["n"], w["s"], w["dist"], w["seed"])
    (phi, E), _ = gpu_fmm(pos, S, 0, 4, 0.5, 64)
    phi_d, E_d = orc.direct(pos, S, 0)
    phi_o, E_o = orc.fmm(pos, S, 0, 4, 0.5, 64)
    assert abs(rel_rms(E, E_d) - rel_rms(E_o, E_d)) < 1e-10
    assert abs(rel_rms(phi, phi_d) - rel_rms(phi_o, phi_d)) < 1e-10
    assert rel_rms(E, E_d) < 5e-3


def test_dipole_1m_sampled(orc):
    """1M dipoles, p=6, theta 0.5, n_crit 128, field only (the benchmarked launch):
    4096 sampled particles against the oracle FMM on the same tree."""
    from gpu_util import gpu_fmm, rel_rms, to_dev
    from paper_2005_12351_gb300 import fmm
    w = synth.WORKLOADS["dipole_1m_p6"]
    pos, S = synth.make_system(w["n"], w["s"], w["dist"], w["seed"])
    (_, E), tree = gpu_fmm(pos, S, 1, 6, 0.5, 128, want_phi=False)
    tg = synth.sample_indices(len(pos), 4096, 7)
    t = orc.Tree(pos, 128)
    t.lists(0.5)
    _, E_o = t.fmm(S, 1, 6, targets=tg)
    assert close(E[tg], E_o, TOL)
    # and the truncation error against the GPU FP64 direct sum is small
    _, E_d = fmm.direct_sum(to_dev(pos), to_dev(S), 1, targets=to_dev(tg[:512].astype(np.int32)),
                            want_potential=False)
    assert rel_rms(E[tg[:512]], E_d.cpu().numpy()) < 1e-3


def test_single_leaf_is_direct(orc):
    from gpu_util import gpu_fmm, rel_rms
    pos, S = synth.make_system(700, 2, "uniform", 501)
    (phi, E), _ = gpu_fmm(pos, S, 2, 3, 0.5, 1000)
    phi_d, E_d = orc.direct(pos, S, 2)
    assert close(phi, phi_d, 1e-13) and close(E, E_d, 1e-13)


def test_field_only_and_potential_only_agree(orc):
    from gpu_util import gpu_fmm
    pos, S = synth.make_system(5000, 1, "plummer", 502)
    (phi, E), _ = gpu_fmm(pos, S, 1, 5, 0.5, 32)
    (phi2, _), _ = gpu_fmm(pos, S, 1, 5, 0.5, 32, want_field=False)
    (_, E2), _ = gpu_fmm(pos, S, 1, 5, 0.5, 32, want_phi=False)
    assert np.allclose(phi2, phi, rtol=1e-13, atol=1e-13 * np.abs(phi).max())
    assert np.allclose(E2, E, rtol=1e-13, atol=1e-13 * np.abs(E).max())


def test_repeat_is_deterministic_and_theta_change_rebuilds(orc):
    import torch
    from gpu_util import rel_rms, to_dev
    from paper_2005_12351_gb300 import fmm
    pos, S = synth.make_system(8000, 0, "uniform", 503)
    tree = fmm.create_tree(max_leaf=32)
    tree.set_sources(to_dev(pos), to_dev(S), 0)
    a = [x.clone() for x in tree.evaluate(4, 0.5)]
    b = [x.clone() for x in tree.evaluate(4, 0.5)]
    assert all(torch.equal(x, y) for x, y in zip(a, b))
    phi3, _ = tree.evaluate(4, 0.35)
    assert tree.info()["theta"] == 0.35
    phi_o, _ = orc.fmm(pos, S, 0, 4, 0.35, 32)
    assert close(phi3.cpu().numpy(), phi_o, TOL)
    phi4, _ = tree.evaluate(7, 0.35)     # p change: new derivative tables, same lists
    phi_o, _ = orc.fmm(pos, S, 0, 7, 0.35, 32)
    assert close(phi4.cpu().numpy(), phi_o, TOL)


def test_linear_in_sources():
    from gpu_util import gpu_fmm
    pos, S1 = synth.make_system(6000, 1, "uniform", 504)
    S2 = synth.unit_dipoles(6000, 505)
    (f1, e1), _ = gpu_fmm(pos, S1, 1, 4, 0.5, 64)
    (f2, e2), _ = gpu_fmm(pos, S2, 1, 4, 0.5, 64)
    (f3, e3), _ = gpu_fmm(pos, S1 - 3.0 * S2, 1, 4, 0.5, 64)
    assert np.allclose(f3, f1 - 3.0 * f2, rtol=0, atol=1e-12 * np.abs(f3).max())
    assert np.allclose(e3, e1 - 3.0 * e2, rtol=0, atol=1e-12 * np.abs(e3).max())


def test_edge_cases_and_errors():
    import torch
    from gpu_util import to_dev
    from paper_2005_12351_gb300 import fmm
    tree = fmm.create_tree(max_leaf=8)
    with pytest.raises(fmm.FMMError) as ei:
        tree.evaluate(4, 0.5)
    assert ei.value.status == fmm.FMM_ESTATE
    # N = 0
    tree.set_sources(torch.zeros((0, 3), dtype=torch.float64, device="cuda"),
                     torch.zeros((0, 1), dtype=torch.float64, device="cuda"), 0)
    phi, E = tree.evaluate(3, 0.5)
    assert phi.numel() == 0 and E.numel() == 0
    # N = 1: no other source, zero field
    tree.set_sources(to_dev(np.array([[0.3, 0.4, 0.5]])), to_dev(np.array([[2.0]])), 0)
    phi, E = tree.evaluate(3, 0.5)
    assert phi.item() == 0.0 and not E.any()
    # bad arguments
    pos = synth.uniform_cube(100, 1)
    bad = pos.copy()
    bad[17, 1] = np.nan
    with pytest.raises(fmm.FMMError) as ei:
        tree.set_sources(to_dev(bad), to_dev(np.ones((100, 1))), 0)
    assert ei.value.status == fmm.FMM_EINVAL
    tree.set_sources(to_dev(pos), to_dev(np.ones((100, 1))), 0)
    for p, th, st in [(0, 0.5, fmm.FMM_EORDER), (13, 0.5, fmm.FMM_EORDER), (4, 0.0, fmm.FMM_EINVAL),
                      (4, 1.0, fmm.FMM_EINVAL)]:
        with pytest.raises(fmm.FMMError) as ei:
            tree.evaluate(p, th, True, True)
        assert ei.value.status == st
    with pytest.raises(fmm.FMMError) as ei:
        tree.set_sources(to_dev(pos), to_dev(np.ones((100, 10))), 3)
    assert ei.value.status == fmm.FMM_EORDER
    # memory budget
    small = fmm.create_tree(max_leaf=8, mem_budget_bytes=64 * 1024)
    with pytest.raises(fmm.FMMError) as ei:
        small.set_sources(to_dev(synth.uniform_cube(20000, 3)), to_dev(np.ones((20000, 1))), 0)
    assert ei.value.status == fmm.FMM_EBUDGET
    assert small.info()["device_bytes"] <= 64 * 1024
