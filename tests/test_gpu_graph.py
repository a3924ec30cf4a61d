"""Repeated evaluation of one geometry: moment updates, the evaluate replayed as a
CUDA graph, and the autotuner.  Same tree, same kernels, same order: a replay and a
moment update give bitwise the results of an ordinary evaluate."""
import numpy as np
import pytest

from paper_2005_12351_gb300 import synth

pytestmark = pytest.mark.gpu


def fresh(pos, S, s, p, prec, ncrit=64, want_phi=True):
    import torch
    from gpu_util import to_dev
    from paper_2005_12351_gb300 import fmm
    t = fmm.create_tree(max_leaf=ncrit, precision=prec)
    t.set_sources(to_dev(pos), to_dev(S), s)
    phi, E = t.evaluate(p, 0.5, want_phi, True)
    torch.cuda.synchronize()
    out = (phi.cpu().numpy() if phi is not None else None), E.cpu().numpy()
    t.destroy()
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32", "3xtf32"])
def test_update_moments_and_graph_replay(prec):
    import torch
    from gpu_util import to_dev
    from paper_2005_12351_gb300 import fmm
    s, p = 1, 5
    pos, S1 = synth.make_system(30_000, s, "plummer", 501)
    _, S2 = synth.make_system(30_000, s, "plummer", 502)
    t = fmm.create_tree(max_leaf=64, precision=prec)
    t.set_sources(to_dev(pos), to_dev(S1), s)
    phi, E = t.evaluate_graph(p, 0.5)          # evaluates, then captures
    ref1 = fresh(pos, S1, s, p, prec)
    assert np.array_equal(E.cpu().numpy(), ref1[1]) and np.array_equal(phi.cpu().numpy(), ref1[0])
    launches = t.launch_count()
    phi, E = t.evaluate_graph(p, 0.5)          # one graph launch
    torch.cuda.synchronize()
    assert t.launch_count() == launches + 1
    assert np.array_equal(E.cpu().numpy(), ref1[1])
    t.update_moments(to_dev(S2))
    phi, E = t.evaluate_graph(p, 0.5)          # same graph, new moments
    torch.cuda.synchronize()
    ref2 = fresh(pos, S2, s, p, prec)
    assert np.array_equal(E.cpu().numpy(), ref2[1]) and np.array_equal(phi.cpu().numpy(), ref2[0])
    # another parameter set recaptures
    phi, E = t.evaluate_graph(p + 1, 0.5, want_potential=False)
    torch.cuda.synchronize()
    assert phi is None
    ref3 = fresh(pos, S2, s, p + 1, prec, want_phi=False)
    assert np.array_equal(E.cpu().numpy(), ref3[1])
    # a new tree drops the graph
    pos4, S4 = synth.make_system(20_000, s, "uniform", 503)
    t.set_sources(to_dev(pos4), to_dev(S4), s)
    phi, E = t.evaluate_graph(p, 0.5)
    phi, E = t.evaluate_graph(p, 0.5)
    torch.cuda.synchronize()
    assert np.array_equal(E.cpu().numpy(), fresh(pos4, S4, s, p, prec)[1])
    t.destroy()


def test_batch_graph_replay():
    """A forest of uneven systems: every phase for all systems in one graph launch."""
    import torch
    from gpu_util import to_dev
    from paper_2005_12351_gb300 import fmm
    pos, S, off = synth.make_batch(64, 100, 4000, 2, 611)
    _, S2, _ = synth.make_batch(64, 100, 4000, 2, 611)
    S2 = S2[::-1].copy()
    t = fmm.create_tree(max_leaf=64, precision="3xtf32")
    t.set_sources_batch(to_dev(pos), to_dev(S), off, 2)
    t.evaluate_graph(4, 0.5, want_potential=False)
    t.update_moments(to_dev(S2))
    _, E = t.evaluate_graph(4, 0.5, want_potential=False)
    torch.cuda.synchronize()
    u = fmm.create_tree(max_leaf=64, precision="3xtf32")
    u.set_sources_batch(to_dev(pos), to_dev(S2), off, 2)
    _, Eu = u.evaluate(4, 0.5, False, True)
    torch.cuda.synchronize()
    assert np.array_equal(E.cpu().numpy(), Eu.cpu().numpy())


# candidates: the three FP64 P2P kernels; FP32: 8/16/32 rows per chunk of the
# tiled SIMT M2L or its per-cell kernel; 3xTF32: 8/16/32 rows per chunk on the
# tensor cores or the tiled SIMT M2L; each FP32 form then the winner with the
# other P2P tile
@pytest.mark.parametrize("prec,ncand", [("fp64", 3), ("fp32", 5), ("3xtf32", 5)])
def test_autotune(prec, ncand):
    import torch
    from gpu_util import rel_rms, to_dev
    from paper_2005_12351_gb300 import fmm
    s, p = 1, 5
    pos, S = synth.make_system(40_000, s, "uniform", 521)
    t = fmm.create_tree(max_leaf=64, precision=prec)
    t.set_sources(to_dev(pos), to_dev(S), s)
    phi0, E0 = t.evaluate(p, 0.5)
    E0 = E0.cpu().numpy()
    tune = t.autotune(p, 0.5, reps=2)
    assert tune["candidates"] == ncand and tune["ms_per_evaluate"] > 0
    assert tune["p2p_variant"] in ((0, 1, 2) if prec == "fp64" else (1,))
    assert tune["p2p_targets"] in (1, 2)
    if prec == "3xtf32":
        assert tune["tc_chunk_rows"] in (8, 16, 32) and tune["m2l_tensor"] in (0, 1)
    if prec == "fp32":
        assert tune["tc_chunk_rows"] in (8, 16, 32) and tune["m2l_tiled"] in (0, 1)
    phi1, E1 = t.evaluate_graph(p, 0.5)
    torch.cuda.synchronize()
    tol = 1e-13 if prec == "fp64" else 1e-6
    assert rel_rms(E1.cpu().numpy(), E0) < tol


@pytest.mark.parametrize("prec", ["fp64", "fp32", "3xtf32"])
def test_launches_per_evaluate_do_not_grow_with_depth(prec):
    """The upward pass (P2M + M2M) and the L2L shifts each run as one launch
    whatever the tree depth: a shallow uniform tree and a deep Plummer tree
    take the same number of kernel launches per evaluate (and a batch of
    systems as few)."""
    import torch
    from gpu_util import to_dev
    from paper_2005_12351_gb300 import fmm
    counts = []
    for dist, n, ncrit in (("uniform", 20_000, 64), ("plummer", 60_000, 16)):
        pos, S = synth.make_system(n, 1, dist, 777)
        t = fmm.create_tree(max_leaf=ncrit, precision=prec)
        t.set_sources(to_dev(pos), to_dev(S), 1)
        t.evaluate(4, 0.5)                        # lists, tables, plans
        torch.cuda.synchronize()
        c0 = t.launch_count()
        t.evaluate(4, 0.5)
        torch.cuda.synchronize()
        counts.append((t.info()["nlevels"], t.launch_count() - c0))
    (l0, a), (l1, b) = counts
    assert l1 >= l0 + 3, counts
    assert a == b and a <= 10, counts
