"""Batches of independent systems (a forest): per-system bit-exact trees and lists,
and per-system FMM parity with the oracle, in one set of launches."""
import numpy as np
import pytest
from gpu_util import close

from paper_2005_12351_gb300 import synth

pytestmark = pytest.mark.gpu


def uneven_batch(s):
    """Systems of uneven size, distribution, offset and scale (so root sides differ),
    including an empty system and a one-particle system."""
    parts = []
    specs = [(300, "uniform", 1.0, 0.0), (0, "uniform", 1.0, 0.0), (1, "uniform", 1.0, 0.0),
             (2000, "plummer", 1.0, 5.0), (57, "uniform", 1e-3, -2.0), (5000, "plummer", 40.0, 0.0),
             (129, "uniform", 1.0, 0.25), (3000, "uniform", 0.125, 100.0)]
    for k, (n, dist, scale, shift) in enumerate(specs):
        p, m = synth.make_system(n, s, dist, 1000 + k)
        parts.append((p * scale + shift, m))
    off = np.zeros(len(parts) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(p) for p, _ in parts])
    pos = np.concatenate([p for p, _ in parts]) if off[-1] else np.zeros((0, 3))
    mom = np.concatenate([m for _, m in parts])
    return pos, mom, off


def build(pos, mom, off, s, ncrit, precision="fp64"):
    from gpu_util import to_dev
    from paper_2005_12351_gb300 import fmm
    tree = fmm.create_tree(max_leaf=ncrit, precision=precision)
    tree.set_sources_batch(to_dev(pos), to_dev(mom), list(off), s)
    return tree


def test_forest_trees_and_lists_bit_exact(orc):
    import torch
    pos, mom, off = uneven_batch(0)
    ncrit, theta = 16, 0.5
    g = build(pos, mom, off, 0, ncrit)
    g.evaluate(2, theta)
    torch.cuda.synchronize()
    assert g.info()["nsystems"] == len(off) - 1
    sysid = g.copy_array("system").numpy()
    level = g.copy_array("level").numpy()
    coord = g.copy_array("coord").numpy()
    rng = g.copy_array("range").numpy()
    parent = g.copy_array("parent").numpy()
    child = g.copy_array("child").numpy()
    centre = g.copy_array("centre").numpy()
    half = g.copy_array("half").numpy()
    perm = g.copy_array("perm").numpy()
    keys = g.copy_array("keys").numpy().view(np.uint64)
    m2l = g.copy_array("m2l").numpy()
    p2p = g.copy_array("p2p").numpy()
    for s in range(len(off) - 1):
        a, b = off[s], off[s + 1]
        cells = np.nonzero(sysid == s)[0]
        loc = -np.ones(len(sysid), dtype=np.int64)
        loc[cells] = np.arange(len(cells))
        t = orc.Tree(pos[a:b], ncrit)
        t.lists(theta)
        assert len(cells) == max(t.ncells, 1)
        if b == a:
            continue
        assert np.array_equal(perm[a:b] - a, t.perm) and np.array_equal(keys[a:b], t.keys)
        assert np.array_equal(level[cells], t.level) and np.array_equal(coord[cells], t.ci)
        assert np.array_equal(rng[cells, 0] - a, t.begin) and np.array_equal(rng[cells, 1] - a, t.end)
        par = parent[cells]
        assert np.array_equal(np.where(par >= 0, loc[np.maximum(par, 0)], -1), t.parent)
        fc = child[cells, 0]
        assert np.array_equal(np.where(fc >= 0, loc[np.maximum(fc, 0)], -1), t.child_first)
        assert np.array_equal(child[cells, 1], t.nchild)
        assert np.array_equal(centre[cells].view(np.uint64), t.centre.view(np.uint64))
        assert np.array_equal(half[cells].view(np.uint64), t.halfw.view(np.uint64))
        for L_g, L_o in ((m2l, t.m2l), (p2p, t.p2p)):
            mine = L_g[sysid[L_g[:, 0]] == s]
            assert (sysid[mine[:, 1]] == s).all()            # never across systems
            assert np.array_equal(loc[mine], L_o)


@pytest.mark.parametrize("s,p", [(0, 4), (1, 6), (2, 5)])
def test_forest_fmm_matches_oracle_per_system(orc, s, p):
    import torch
    from gpu_util import rel_rms
    pos, mom, off = uneven_batch(s)
    g = build(pos, mom, off, s, 32)
    phi, E = g.evaluate(p, 0.5)
    torch.cuda.synchronize()
    phi, E = phi.cpu().numpy(), E.cpu().numpy()
    for k in range(len(off) - 1):
        a, b = off[k], off[k + 1]
        if b - a < 2:
            if b > a:
                assert phi[a] == 0.0 and not E[a].any()
            continue
        phi_o, E_o = orc.fmm(pos[a:b], mom[a:b], s, p, 0.5, 32)
        assert close(phi[a:b], phi_o, 1e-12) and close(E[a:b], E_o, 1e-12), k


def test_forest_fp32_matches_per_system(orc):
    import torch
    from gpu_util import rel_rms
    pos, mom, off = uneven_batch(2)
    g = build(pos, mom, off, 2, 32, precision="fp32")
    phi, E = g.evaluate(5, 0.5)
    torch.cuda.synchronize()
    phi, E = phi.cpu().numpy(), E.cpu().numpy()
    for k in range(len(off) - 1):
        a, b = off[k], off[k + 1]
        if b - a < 50:
            continue
        phi_o, E_o = orc.fmm(pos[a:b], mom[a:b], 2, 5, 0.5, 32)
        assert rel_rms(phi[a:b], phi_o) < 1e-6 and rel_rms(E[a:b], E_o) < 1e-6, k


def test_quadrupole_batch_4096_sampled(orc):
    """4,096 uniform systems, N log-uniform in [256, 65536], quadrupoles, p=5:
    the batched FP64 and FP32 results on sampled systems match the oracle."""
    import torch
    from gpu_util import rel_rms
    w = synth.WORKLOADS["quadrupole_batch_4096_p5"]
    pos, mom, off = synth.make_batch(w["batch"], w["nlo"], w["nhi"], w["s"], w["seed"])
    for prec, tol in (("fp64", 1e-12), ("fp32", 1e-6)):
        g = build(pos, mom, off, 2, w["ncrit"], precision=prec)
        phi, E = g.evaluate(5, 0.5)
        torch.cuda.synchronize()
        phi, E = phi.cpu().numpy(), E.cpu().numpy()
        for k in (0, 1, 777, 2048, 4095):
            a, b = off[k], off[k + 1]
            phi_o, E_o = orc.fmm(pos[a:b], mom[a:b], 2, 5, 0.5, w["ncrit"])
            assert rel_rms(E[a:b], E_o) < tol and rel_rms(phi[a:b], phi_o) < tol, (prec, k)
        g.destroy()
