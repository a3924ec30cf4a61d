"""Mixed source orders on the GPU (every particle carries the orders s_lo..s_hi,
§2 "mixed systems"): FMM, direct sum and Barnes-Hut against the oracle's
mixed-order versions, the P2P kernel variants (the symmetric one against the
one-way one), moment updates and graph replay,
and the calls a mixed system is refused by."""
import numpy as np
import pytest
from gpu_util import close

from paper_2005_12351_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12


def gpu_mixed(pos, S, lo, hi, ncrit, variant=None):
    from gpu_util import to_dev
    from paper_2005_12351_gb300 import fmm
    t = fmm.create_tree(max_leaf=ncrit)
    if variant is not None:
        t.set_tuning(p2p_variant=variant)
    t.set_sources_mixed(to_dev(pos), to_dev(S), lo, hi)
    return t


@pytest.mark.parametrize("lo,hi,p,dist,n,ncrit,outs,variant", [
    (0, 1, 6, "uniform", 20_000, 64, "both", None),
    (0, 1, 3, "plummer", 8000, 16, "field", 0),
    (1, 2, 5, "plummer", 10_000, 32, "both", None),
    (1, 2, 2, "uniform", 6000, 300, "phi", 1),
    (0, 2, 4, "uniform", 8000, 64, "field", 1),
    (0, 2, 8, "plummer", 6000, 16, "both", 2),
])
def test_mixed_fmm_matches_oracle(orc, lo, hi, p, dist, n, ncrit, outs, variant):
    import torch
    from gpu_util import rel_rms
    pos, S = synth.make_system_mixed(n, lo, hi, dist, 1500 + 10 * lo + hi + p)
    wp, wf = outs in ("phi", "both"), outs in ("field", "both")
    t = gpu_mixed(pos, S, lo, hi, ncrit, variant)
    assert t.info()["source_order_hi"] == hi and t.info()["source_order"] == lo
    phi, E = t.evaluate(p, 0.5, wp, wf)
    torch.cuda.synchronize()
    ot = orc.Tree(pos, ncrit)
    ot.lists(0.5)
    phi_o, E_o = ot.fmm(S, lo, p, s_hi=hi)
    if wp:
        assert close(phi.cpu().numpy(), phi_o, TOL)
    if wf:
        assert close(E.cpu().numpy(), E_o, TOL)
    t.destroy()


@pytest.mark.parametrize("lo,hi", [(0, 1), (1, 2), (0, 2)])
@pytest.mark.parametrize("outs", ["phi", "field", "both"])
def test_mixed_symmetric_p2p_matches_one_way(lo, hi, outs):
    """The symmetric near field (each shell's reverse term with its own parity)
    against the one-way kernel on the same tree: the same sums in another order."""
    import torch
    from gpu_util import rel_rms
    pos, S = synth.make_system_mixed(30_000, lo, hi, "plummer", 1900 + 3 * lo + hi)
    wp, wf = outs in ("phi", "both"), outs in ("field", "both")
    res = {}
    for v in (1, 2):
        t = gpu_mixed(pos, S, lo, hi, 64, v)
        phi, E = t.evaluate(4, 0.5, wp, wf)
        torch.cuda.synchronize()
        res[v] = (phi.cpu().numpy() if wp else None, E.cpu().numpy() if wf else None)
        t.destroy()
    if wp:
        assert close(res[2][0], res[1][0], 1e-14)
    if wf:
        assert close(res[2][1], res[1][1], 1e-14)


@pytest.mark.parametrize("lo,hi", [(0, 1), (1, 2), (0, 2)])
def test_mixed_direct_and_bh_match_oracle(orc, lo, hi):
    import torch
    from gpu_util import rel_rms, to_dev
    from paper_2005_12351_gb300 import fmm
    pos, S = synth.make_system_mixed(4000, lo, hi, "plummer", 1600 + lo + hi)
    phi, E = fmm.direct_sum(to_dev(pos), to_dev(S), lo, source_order_hi=hi)
    phi_o, E_o = orc.direct(pos, S, lo, s_hi=hi)
    assert close(phi.cpu().numpy(), phi_o, 1e-13) and close(E.cpu().numpy(), E_o, 1e-13)
    t = gpu_mixed(pos, S, lo, hi, 32)
    phi_b, E_b = t.evaluate_bh(5, 0.4)
    torch.cuda.synchronize()
    phi_bo, E_bo = orc.Tree(pos, 32).bh(S, lo, 5, 0.4, s_hi=hi)
    assert close(phi_b.cpu().numpy(), phi_bo, TOL) and close(E_b.cpu().numpy(), E_bo, TOL)
    t.destroy()


def test_mixed_update_moments_and_graph():
    """New mixed moments on the same geometry, replayed as one graph launch,
    give the bits of a fresh handle."""
    import torch
    from gpu_util import to_dev
    from paper_2005_12351_gb300 import fmm
    pos, S = synth.make_system_mixed(20_000, 0, 2, "uniform", 1701)
    S2 = synth.sources_mixed(len(pos), 1702, 0, 2)
    t = gpu_mixed(pos, S, 0, 2, 64)
    t.evaluate_graph(5, 0.5)
    t.update_moments(to_dev(S2))
    phi, E = t.evaluate_graph(5, 0.5)
    torch.cuda.synchronize()
    u = gpu_mixed(pos, S2, 0, 2, 64)
    phi_u, E_u = u.evaluate(5, 0.5)
    torch.cuda.synchronize()
    assert np.array_equal(E.cpu().numpy(), E_u.cpu().numpy())
    assert np.array_equal(phi.cpu().numpy(), phi_u.cpu().numpy())
    t.destroy()
    u.destroy()


def test_mixed_refusals():
    from gpu_util import to_dev
    from paper_2005_12351_gb300 import fmm
    pos, S = synth.make_system_mixed(500, 0, 1, "uniform", 1801)
    for prec in ("fp32", "3xtf32"):
        t = fmm.create_tree(max_leaf=32, precision=prec)
        with pytest.raises(fmm.FMMError):
            t.set_sources_mixed(to_dev(pos), to_dev(S), 0, 1)
        t.destroy()
    t = fmm.create_tree(max_leaf=32)
    with pytest.raises(Exception):
        t.set_sources_mixed(to_dev(pos), to_dev(S), 1, 0)
    t.set_sources_mixed(to_dev(pos), to_dev(S), 0, 1)
    with pytest.raises(fmm.FMMError):
        t.evaluate(13, 0.5)                  # p + s_lo <= 12: the limit refers to the lowest order
    t.destroy()
