"""GPU multipolar Barnes-Hut (FP64) against the oracle's Barnes-Hut on the same
tree, the theta = 0 limit against the GPU direct sum, systems of a batch
against the same systems alone, and the handle's FMM after a Barnes-Hut call."""
import numpy as np
import pytest
from gpu_util import close

from paper_2005_12351_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12        # relative RMS, GPU FP64 vs CPU FP64 oracle, same tree and walk


def gpu_bh(pos, S, s, p, theta, ncrit, want_phi=True, want_field=True):
    import torch
    from gpu_util import to_dev
    from paper_2005_12351_gb300 import fmm
    t = fmm.create_tree(max_leaf=ncrit)
    t.set_sources(to_dev(pos), to_dev(S), s)
    phi, E = t.evaluate_bh(p, theta, want_phi, want_field)
    torch.cuda.synchronize()
    return (phi.cpu().numpy() if phi is not None else None,
            E.cpu().numpy() if E is not None else None), t


# theta 0.8 lets a cell that holds the target pass (r/|d| >= 1/sqrt(3) inside a cell);
# p = 12 takes D to order 13 (one warp per block)
@pytest.mark.parametrize("s,p,theta,dist,n,ncrit,outs", [
    (0, 0, 0.5, "uniform", 4000, 32, "both"),
    (0, 4, 0.5, "uniform", 8000, 64, "both"),
    (0, 8, 0.3, "plummer", 6000, 32, "phi"),
    (1, 6, 0.5, "uniform", 20_000, 128, "field"),
    (1, 3, 0.25, "plummer", 10_000, 32, "both"),
    (1, 12, 0.5, "uniform", 3000, 64, "both"),
    (1, 2, 0.8, "plummer", 5000, 16, "both"),
    (2, 5, 0.4, "uniform", 6000, 64, "both"),
    (2, 2, 0.6, "plummer", 5000, 16, "field"),
])
def test_bh_matches_oracle(orc, s, p, theta, dist, n, ncrit, outs):
    from gpu_util import rel_rms
    pos, S = synth.make_system(n, s, dist, 1300 + 10 * s + p)
    wp, wf = outs in ("phi", "both"), outs in ("field", "both")
    (phi, E), t = gpu_bh(pos, S, s, p, theta, ncrit, wp, wf)
    phi_o, E_o = orc.Tree(pos, ncrit).bh(S, s, p, theta)
    if wp:
        assert close(phi, phi_o, TOL), rel_rms(phi, phi_o)
    else:
        assert phi is None
    if wf:
        assert close(E, E_o, TOL), rel_rms(E, E_o)
    t.destroy()


@pytest.mark.parametrize("s", [0, 1, 2])
def test_bh_theta_zero_is_direct_sum(s):
    from gpu_util import rel_rms, to_dev
    from paper_2005_12351_gb300 import fmm
    pos, S = synth.make_system(5000, s, "plummer", 1400 + s)
    (phi, E), t = gpu_bh(pos, S, s, s + 1, 0.0, 32)
    phi_d, E_d = fmm.direct_sum(to_dev(pos), to_dev(S), s)
    assert close(phi, phi_d.cpu().numpy(), 1e-13)
    assert close(E, E_d.cpu().numpy(), 1e-13)
    t.destroy()


def test_bh_batch_matches_alone():
    """Warps that straddle systems walk several roots; every system gets the
    bits it gets alone."""
    import torch
    from gpu_util import to_dev
    from paper_2005_12351_gb300 import fmm
    pos, S, off = synth.make_batch(40, 3, 3000, 1, 1411, dist="plummer")
    tb = fmm.create_tree(max_leaf=32)
    tb.set_sources_batch(to_dev(pos), to_dev(S), off, 1)
    phi_b, E_b = tb.evaluate_bh(5, 0.5)
    torch.cuda.synchronize()
    phi_b, E_b = phi_b.cpu().numpy(), E_b.cpu().numpy()
    for k in range(0, 40, 7):
        a, b = int(off[k]), int(off[k + 1])
        (phi, E), t = gpu_bh(pos[a:b], S[a:b], 1, 5, 0.5, 32)
        assert np.array_equal(phi, phi_b[a:b]) and np.array_equal(E, E_b[a:b]), k
        t.destroy()
    tb.destroy()


def test_fmm_after_bh_unchanged():
    """Barnes-Hut rebuilds the handle's tables and multipoles; the next FMM
    evaluate (and a captured one) gives the same bits as before."""
    import torch
    from gpu_util import to_dev
    from paper_2005_12351_gb300 import fmm
    pos, S = synth.make_system(20_000, 1, "uniform", 1421)
    t = fmm.create_tree(max_leaf=64)
    t.set_sources(to_dev(pos), to_dev(S), 1)
    phi0, E0 = t.evaluate(5, 0.5)
    phi0, E0 = phi0.cpu().numpy(), E0.cpu().numpy()
    t.evaluate_graph(5, 0.5)
    t.evaluate_bh(4, 0.4)
    phi1, E1 = t.evaluate(5, 0.5)
    phi2, E2 = t.evaluate_graph(5, 0.5)
    torch.cuda.synchronize()
    assert np.array_equal(phi1.cpu().numpy(), phi0) and np.array_equal(E1.cpu().numpy(), E0)
    assert np.array_equal(E2.cpu().numpy(), E0)
    t.destroy()


def test_bh_edge_cases():
    import torch
    from gpu_util import to_dev
    from paper_2005_12351_gb300 import fmm
    t = fmm.create_tree(max_leaf=8)
    t.set_sources(to_dev(np.array([[0.3, 0.4, 0.5]])), to_dev(np.array([[1.0, 0.0, 0.0]])), 1)
    phi, E = t.evaluate_bh(3, 0.5)
    assert phi.item() == 0.0 and not E.any()
    for p, theta in ((0, 0.5), (13, 0.5), (3, -0.1), (3, float("inf"))):
        with pytest.raises(Exception):
            t.evaluate_bh(p, theta)
    t.set_sources(torch.zeros((0, 3), dtype=torch.float64, device="cuda"),
                  torch.zeros((0, 3), dtype=torch.float64, device="cuda"), 1)
    phi, E = t.evaluate_bh(3, 0.5)
    assert phi.numel() == 0
    t.destroy()
