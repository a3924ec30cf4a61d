"""GPU octree and interaction lists are bit-exact against the oracle."""
import numpy as np
import pytest

from paper_2005_12351_gb300 import synth

pytestmark = pytest.mark.gpu


def _gpu_tree(pos, ncrit, theta):
    from gpu_util import to_dev
    from paper_2005_12351_gb300 import fmm
    tree = fmm.create_tree(max_leaf=ncrit)
    tree.set_sources(to_dev(pos), to_dev(np.ones((len(pos), 1))), 0)
    if theta is not None and len(pos):
        import torch
        tree.evaluate(1, theta, True, False)
        torch.cuda.synchronize()
    return tree


@pytest.mark.parametrize("n,dist", [(1, "uniform"), (7, "uniform"), (4097, "uniform"),
                                    (50_000, "plummer"), (1_000_000, "uniform")])
def test_morton_order_bit_exact(orc, n, dist):
    from gpu_util import to_dev
    from paper_2005_12351_gb300 import fmm
    pos = synth.make_system(n, 0, dist, 100 + n)[0]
    keys, perm = fmm.morton_order(to_dev(pos))
    t = orc.Tree(pos, 1 << 30)
    assert np.array_equal(keys.cpu().numpy().view(np.uint64), t.keys)
    assert np.array_equal(perm.cpu().numpy().astype(np.int64), t.perm)


def test_morton_order_stable_with_repeated_points(orc):
    """300,000 particles on 997 distinct points: runs of equal keys span many
    sort tiles, and the sort keeps them in original-index order."""
    from gpu_util import to_dev
    from paper_2005_12351_gb300 import fmm
    base = synth.make_system(997, 0, "uniform", 4242)[0]
    pick = np.minimum((synth.uniform01(4243, 1, 300_000) * 997).astype(np.int64), 996)
    pos = base[pick]
    keys, perm = fmm.morton_order(to_dev(pos))
    t = orc.Tree(pos, 1 << 30)
    assert np.array_equal(keys.cpu().numpy().view(np.uint64), t.keys)
    assert np.array_equal(perm.cpu().numpy().astype(np.int64), t.perm)


def _compare_trees(orc, pos, ncrit, theta):
    t = orc.Tree(pos, ncrit)
    t.lists(theta)
    g = _gpu_tree(pos, ncrit, theta)
    info = g.info()
    assert info["ncells"] == t.ncells and info["nlevels"] == t.nlevels
    assert np.array_equal(info["lo"], t.lo) and info["side"] == t.side
    assert np.array_equal(g.copy_array("keys").numpy().view(np.uint64), t.keys)
    assert np.array_equal(g.copy_array("perm").numpy(), t.perm)
    assert np.array_equal(g.copy_array("level").numpy(), t.level)
    assert np.array_equal(g.copy_array("coord").numpy(), t.ci)
    rng = g.copy_array("range").numpy()
    assert np.array_equal(rng[:, 0], t.begin) and np.array_equal(rng[:, 1], t.end)
    assert np.array_equal(g.copy_array("parent").numpy(), t.parent)
    ch = g.copy_array("child").numpy()
    assert np.array_equal(ch[:, 0], t.child_first) and np.array_equal(ch[:, 1], t.nchild)
    # geometry: bit-exact doubles
    assert np.array_equal(g.copy_array("centre").numpy().view(np.uint64), t.centre.view(np.uint64))
    assert np.array_equal(g.copy_array("half").numpy().view(np.uint64), t.halfw.view(np.uint64))
    # lists, sorted by (target, source)
    assert info["n_m2l"] == len(t.m2l) and info["n_p2p"] == len(t.p2p)
    assert np.array_equal(g.copy_array("m2l").numpy(), t.m2l)
    assert np.array_equal(g.copy_array("p2p").numpy(), t.p2p)
    cnt = t.end - t.begin
    assert info["n_p2p_interactions"] == int((cnt[t.p2p[:, 0]] * cnt[t.p2p[:, 1]]).sum())
    g.destroy()


@pytest.mark.parametrize("n,dist,ncrit,theta", [
    (2000, "uniform", 64, 0.5),          # the 2k monopole workload's tree
    (20_000, "uniform", 32, 0.5),
    (30_000, "plummer", 16, 0.5),        # adaptive: cross-level pairs, deep leaves
    (10_000, "plummer", 40, 0.3),
    (5000, "uniform", 8, 0.8),
])
def test_tree_and_lists_bit_exact(orc, n, dist, ncrit, theta):
    pos = synth.make_system(n, 0, dist, 200 + n)[0]
    _compare_trees(orc, pos, ncrit, theta)


def test_lists_with_rows_longer_than_a_warp_sort(orc):
    """theta 0.2 on 30,000 uniform points gives M2L rows of about 2,000
    sources: those rows are sorted by a whole block, and the lists stay
    bit-exact."""
    pos = synth.make_system(30_000, 0, "uniform", 230_000)[0]
    t = orc.Tree(pos, 8)
    t.lists(0.2)
    assert np.bincount(t.m2l[:, 0]).max() > 1024
    _compare_trees(orc, pos, 8, 0.2)


@pytest.mark.parametrize("limit", [2, 64])
def test_lists_when_rows_exceed_the_row_sort(orc, monkeypatch, limit):
    """Rows longer than the row sort takes send both lists through the radix
    sort of (target, source) keys; FMM_ROW_SORT_LIMIT lowers that length so
    that the path runs on ordinary trees.  Same lists either way."""
    monkeypatch.setenv("FMM_ROW_SORT_LIMIT", str(limit))
    _compare_trees(orc, synth.make_system(30_000, 0, "plummer", 230_030)[0], 16, 0.5)
    _compare_trees(orc, synth.make_system(20_000, 0, "uniform", 220_000)[0], 32, 0.5)


def test_tree_duplicates_and_tiny(orc):
    pos = np.concatenate([np.repeat([[0.1, 0.2, 0.3]], 300, axis=0), synth.uniform_cube(200, 9)])
    _compare_trees(orc, pos, 16, 0.5)
    _compare_trees(orc, synth.uniform_cube(3, 1), 1, 0.5)
    _compare_trees(orc, -5.0 + 1e-6 * synth.uniform_cube(1000, 2), 10, 0.5)


def test_tree_full_size_dipole_workload(orc):
    """1M uniform points, n_crit 128, theta 0.5: the benchmarked tree and lists."""
    pos = synth.make_system(1_000_000, 1, "uniform", 20260001)[0]
    _compare_trees(orc, pos, 128, 0.5)
