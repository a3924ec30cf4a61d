"""Mixed-precision forms: FMM_FP32 (scaled FP32 expansions and pair terms, FP64 D
tables and outputs) and FMM_3XTF32 (the same with the M2L on the tcgen05 tensor
cores in 3xTF32: FP32 operands split into two TF32 halves, FP32 accumulation in
tensor memory over chunks of keys, double-float across chunks).

Tolerances: the FP32 form is compared with the FP64 oracle FMM on the same tree
(difference = FP32 rounding only: ~2e-7 measured, bounded here by 1e-6 relative
RMS = ~16 FP32 ulps), and -- the criterion that matters -- its error against the
FP64 direct sum must stay within 1.1x the FP64 FMM truncation error at the same
p, with no additive allowance.  That needs the near field's rounding well below
FP32's: the quadrupole field's FP64 truncation error at p = 5 is ~5e-8, under
one FP32 ulp, and all-FP32 pair terms leave ~3e-7 of noise, set by each
particle's nearest neighbours.  The one-way FP32 P2P therefore evaluates the
pairs closer than one mean spacing of the target leaf in double-float.
"""
import numpy as np
import pytest
from gpu_util import close

from paper_2005_12351_gb300 import synth

pytestmark = pytest.mark.gpu


def gpu_eval(pos, S, s, p, theta, ncrit, precision, want_phi=True, want_field=True, harmonic=1,
             p2p_variant=-1, m2l_tiled=-1):
    import torch
    from gpu_util import to_dev
    from paper_2005_12351_gb300 import fmm
    tree = fmm.create_tree(max_leaf=ncrit, precision=precision)
    tree.set_tuning(m2l_harmonic=harmonic, p2p_variant=p2p_variant, m2l_tiled=m2l_tiled)
    tree.set_sources(to_dev(pos), to_dev(S), s)
    phi, E = tree.evaluate(p, theta, want_phi, want_field)
    torch.cuda.synchronize()
    return (phi.cpu().numpy() if phi is not None else None,
            E.cpu().numpy() if E is not None else None), tree


FORMS = ["fp32", "3xtf32"]


def assert_tc_ran(tree, precision):
    """The 3xTF32 form must have taken the tensor-core M2L (no silent SIMT path)."""
    info = tree.info()
    if precision == "3xtf32" and info["n_m2l"] > 0:
        assert info["tc_rows"] > 0 and info["tc_chunks"] > 0, info
        assert info["tc_rows"] * 128 >= info["n_m2l"]


@pytest.mark.parametrize("variant", [-1, 2])        # the form's default P2P, and the symmetric one
@pytest.mark.parametrize("precision", FORMS)
@pytest.mark.parametrize("s,p,dist,n,ncrit", [
    (0, 4, "uniform", 2000, 64),
    (0, 6, "plummer", 20_000, 32),
    (1, 6, "uniform", 30_000, 128),
    (1, 5, "plummer", 20_000, 64),
    (2, 5, "uniform", 15_000, 128),
    (2, 3, "plummer", 10_000, 16),
])
def test_fp32_close_to_fp64_oracle(orc, precision, s, p, dist, n, ncrit, variant):
    from gpu_util import rel_rms
    pos, S = synth.make_system(n, s, dist, 700 + 10 * s + p)
    (phi, E), tree = gpu_eval(pos, S, s, p, 0.5, ncrit, precision, p2p_variant=variant)
    assert_tc_ran(tree, precision)
    t = orc.Tree(pos, ncrit)
    t.lists(0.5)
    phi_o, E_o = t.fmm(S, s, p)
    assert rel_rms(phi, phi_o) < 1e-6, rel_rms(phi, phi_o)
    assert rel_rms(E, E_o) < 1e-6, rel_rms(E, E_o)


@pytest.mark.parametrize("precision", FORMS)
@pytest.mark.parametrize("s,p,dist", [(0, 4, "plummer"), (0, 8, "plummer"), (1, 6, "plummer"),
                                       (1, 8, "plummer"), (2, 3, "plummer"), (2, 5, "plummer"),
                                       (2, 5, "uniform"), (2, 8, "uniform"), (1, 10, "uniform")])
def test_fp32_error_within_1p1_of_fp64_truncation(orc, precision, s, p, dist):
    """The precision criterion, with no additive term: the mixed form's error against the
    FP64 direct sum (oracle) is within 1.1x the FP64 FMM's, for the field and the
    potential.  Quadrupoles at p >= 5 and dipoles at p = 10 have field truncation
    errors of 1e-8..1e-7, at or below FP32 resolution."""
    from gpu_util import rel_rms
    pos, S = synth.make_system(12_000, s, dist, 800 + s)
    (phi32, E32), tree = gpu_eval(pos, S, s, p, 0.5, 64, precision)
    assert_tc_ran(tree, precision)
    (phi64, E64), _ = gpu_eval(pos, S, s, p, 0.5, 64, "fp64")
    phi_d, E_d = orc.direct(pos, S, s)
    e32, e64 = rel_rms(E32, E_d), rel_rms(E64, E_d)
    assert e32 <= 1.1 * e64, (e32, e64)
    f32, f64 = rel_rms(phi32, phi_d), rel_rms(phi64, phi_d)
    assert f32 <= 1.1 * f64, (f32, f64)


@pytest.mark.parametrize("precision", FORMS)
def test_quadrupole_batch_4096_p5_within_1p1(orc, precision):
    """The 4,096-system quadrupole batch (N log-uniform in [256, 65536], uniform
    cube, p = 5, theta 0.5, n_crit 128): on 32 sampled systems, each mixed form's
    field and potential error against the oracle's direct sum is within 1.1x the
    FP64 batch's, and the FP64 batch matches the oracle FMM system by system."""
    import torch
    from gpu_util import rel_rms, to_dev
    from paper_2005_12351_gb300 import fmm
    w = synth.WORKLOADS["quadrupole_batch_4096_p5"]
    pos, S, off = synth.make_batch(w["batch"], w["nlo"], w["nhi"], w["s"], w["seed"], w["dist"])
    P, Sd = to_dev(pos), to_dev(S)
    out = {}
    for prec in ("fp64", precision):
        t = fmm.create_tree(max_leaf=w["ncrit"], precision=prec)
        t.set_sources_batch(P, Sd, list(off), w["s"])
        phi, E = t.evaluate(w["p"], w["theta"], True, True)
        torch.cuda.synchronize()
        if prec != "fp64":
            assert_tc_ran(t, prec)
        out[prec] = (phi.cpu().numpy(), E.cpu().numpy())
        t.destroy()
    ks = synth.sample_indices(w["batch"], 32, 29)
    num = {k: np.zeros(2) for k in out}
    den = np.zeros(2)
    for i, k in enumerate(ks):
        a, b = int(off[k]), int(off[k + 1])
        # big systems: the direct sum at 1,024 sampled targets of the system
        tg = synth.sample_indices(b - a, min(b - a, 1024), 31 + int(k))
        phi_d, E_d = orc.direct(pos[a:b], S[a:b], w["s"], targets=tg)
        den += [(phi_d ** 2).sum(), (E_d ** 2).sum()]
        for prec, (phi, E) in out.items():
            num[prec] += [((phi[a:b][tg] - phi_d) ** 2).sum(), ((E[a:b][tg] - E_d) ** 2).sum()]
        if i < 4:
            ot = orc.Tree(pos[a:b], w["ncrit"])
            ot.lists(w["theta"])
            phi_o, E_o = ot.fmm(S[a:b], w["s"], w["p"], targets=tg[:256])
            assert close(out["fp64"][0][a:b][tg[:256]], phi_o, 1e-12)
            assert close(out["fp64"][1][a:b][tg[:256]], E_o, 1e-12)
    e64 = np.sqrt(num["fp64"] / den)
    e32 = np.sqrt(num[precision] / den)
    assert e32[0] <= 1.1 * e64[0], (e32, e64)
    assert e32[1] <= 1.1 * e64[1], (e32, e64)


def test_plummer_4m_p8_fp32_vs_fp64(orc):
    """4M Plummer dipoles, p=8, n_crit 128: the field error of each mixed form
    against the FP64 direct sum (4,096 sampled particles) is within 1.1x that of
    the FP64 GPU form, and the FP64 form matches the oracle FMM on the same tree."""
    import torch
    from gpu_util import rel_rms, to_dev
    from paper_2005_12351_gb300 import fmm
    w = synth.WORKLOADS["dipole_plummer_4m_p8"]
    pos, S = synth.make_system(w["n"], w["s"], w["dist"], w["seed"])
    E_mixed = {}
    for prec in FORMS:
        (_, E_mixed[prec]), tm = gpu_eval(pos, S, 1, 8, 0.5, 128, prec, want_phi=False)
        assert_tc_ran(tm, prec)
        tm.destroy()
    (_, E64), t64 = gpu_eval(pos, S, 1, 8, 0.5, 128, "fp64", want_phi=False)
    t64.destroy()
    tg = synth.sample_indices(len(pos), 4096, 11)
    _, E_d = fmm.direct_sum(to_dev(pos), to_dev(S), 1, targets=to_dev(tg.astype(np.int32)),
                            want_potential=False)
    E_d = E_d.cpu().numpy()
    e64 = rel_rms(E64[tg], E_d)
    for prec in FORMS:
        e = rel_rms(E_mixed[prec][tg], E_d)
        assert e <= 1.1 * e64, (prec, e, e64)
    ot = orc.Tree(pos, 128)
    ot.lists(0.5)
    _, E_o = ot.fmm(S, 1, 8, targets=tg[:1024])
    assert close(E64[tg[:1024]], E_o, 1e-12)
    torch.cuda.synchronize()


@pytest.mark.parametrize("precision", FORMS)
def test_fp32_edge_cases(precision):
    import torch
    from gpu_util import to_dev
    from paper_2005_12351_gb300 import fmm
    tree = fmm.create_tree(max_leaf=8, precision=precision)
    tree.set_sources(to_dev(np.array([[0.3, 0.4, 0.5]])), to_dev(np.array([[1.0, 0.0, 0.0]])), 1)
    phi, E = tree.evaluate(3, 0.5)
    assert phi.item() == 0.0 and not E.any()
    tree.set_sources(torch.zeros((0, 3), dtype=torch.float64, device="cuda"),
                     torch.zeros((0, 3), dtype=torch.float64, device="cuda"), 1)
    phi, E = tree.evaluate(3, 0.5)
    assert phi.numel() == 0


@pytest.mark.parametrize("s,p,dist,n,h", [(1, 6, "uniform", 60_000, 1), (2, 5, "plummer", 40_000, 1),
                                           (0, 9, "plummer", 30_000, 1), (1, 11, "uniform", 20_000, 1),
                                           (1, 6, "uniform", 60_000, 0), (1, 9, "uniform", 20_000, 0),
                                           (1, 10, "uniform", 20_000, 0)])
def test_3xtf32_matches_fp32_form(s, p, dist, n, h):
    """Both mixed forms round the same scaled FP32 expansions; their results agree
    to FP32 rounding: the field within 1e-6, the potential (whose local term sums
    ~10^2 contributions of mixed sign per key row in tensor-core FP32) within 2e-6.
    Harmonic M2L (h=1): the tensor-core columns are the (p+1)^2 locals with
    n_z <= 1, two column groups from p = 11.  Full M2L (h=0): two column groups
    at p = 9; p = 10 has n_L = 286 > 256 and takes the SIMT M2L."""
    from gpu_util import rel_rms
    pos, S = synth.make_system(n, s, dist, 900 + s + p)
    (phi_a, E_a), ta = gpu_eval(pos, S, s, p, 0.5, 64, "fp32", harmonic=h)
    (phi_b, E_b), tb = gpu_eval(pos, S, s, p, 0.5, 64, "3xtf32", harmonic=h)
    if h == 1 or p < 10:
        assert_tc_ran(tb, "3xtf32")
    else:
        assert tb.info()["tc_rows"] == 0
    # local expansions column by column: with n_L > 128 the columns from 128 on
    # come from the second column group of the tensor-core M2L.  A cell stores
    # the (p+1)^2 traceless components (n_z <= 1) with the harmonic M2L, all
    # n_L otherwise.
    nL = (p + 1) ** 2 if h else (p + 1) * (p + 2) * (p + 3) // 6
    La, Lb = ta.copy_array("local", nL).numpy(), tb.copy_array("local", nL).numpy()
    assert La.dtype == np.float32 and La.shape[1] == Lb.shape[1]
    for c0 in range(0, La.shape[1], 128):
        assert rel_rms(Lb[:, c0:c0 + 128], La[:, c0:c0 + 128]) < 1e-5, c0
    assert rel_rms(E_b, E_a) < 1e-6, rel_rms(E_b, E_a)
    assert rel_rms(phi_b, phi_a) < 2e-6, rel_rms(phi_b, phi_a)


@pytest.mark.parametrize("precision", FORMS)
def test_tile_chunk_boundaries(monkeypatch, precision):
    """Chunks of one key row each and chunks longer than any tile's rows give the
    same result within FP32 rounding (the chunk partials are summed in double-float), on
    the tensor cores (3xTF32) and in the tiled SIMT M2L (FP32).  The chunk length
    is read when a handle builds its first plan."""
    from gpu_util import rel_rms
    pos, S = synth.make_system(20_000, 1, "plummer", 77)
    out = {}
    for g in ("1", "100000"):
        monkeypatch.setenv("FMM_TC_CHUNK", g)
        (_, out[g]), tree = gpu_eval(pos, S, 1, 6, 0.5, 32, precision, want_phi=False)
        info = tree.info()
        assert info["tc_chunks"] == (info["tc_rows"] if g == "1" else info["tc_tiles"])
    assert rel_rms(out["1"], out["100000"]) < 1e-6


@pytest.mark.parametrize("precision", FORMS)
def test_mixed_falls_back_to_per_cell_m2l_within_budget(precision):
    """When the tile plan and operator images (of the tensor-core M2L, or of the
    tiled SIMT M2L it falls back to first) do not fit the handle's memory budget,
    a mixed form takes the SIMT FP32 M2L with one block per target cell: the
    evaluate succeeds and is bitwise the FP32 form's result on that kernel."""
    import torch
    from gpu_util import to_dev
    from paper_2005_12351_gb300 import fmm
    pos, S = synth.make_system(40_000, 2, "plummer", 931)
    P, Sd = to_dev(pos), to_dev(S)
    f32 = fmm.create_tree(max_leaf=64, precision="fp32")
    f32.set_tuning(m2l_tiled=0)
    f32.set_sources(P, Sd, 2)
    _, E32 = f32.evaluate(9, 0.5, False, True)
    torch.cuda.synchronize()
    assert f32.info()["tc_rows"] == 0
    need32 = f32.info()["device_bytes"]
    full = fmm.create_tree(max_leaf=64, precision=precision)
    full.set_sources(P, Sd, 2)
    full.evaluate(9, 0.5, False, True)
    torch.cuda.synchronize()
    assert full.info()["tc_rows"] > 0 and full.info()["device_bytes"] > need32 * 1.05
    t = fmm.create_tree(max_leaf=64, precision=precision, mem_budget_bytes=int(need32 * 1.02))
    t.set_sources(P, Sd, 2)
    _, E = t.evaluate(9, 0.5, False, True)
    torch.cuda.synchronize()
    assert t.info()["tc_rows"] == 0
    assert np.array_equal(E.cpu().numpy(), E32.cpu().numpy())


@pytest.mark.parametrize("s,p,dist,n,h", [(1, 6, "uniform", 60_000, 1), (2, 5, "plummer", 40_000, 1),
                                           (0, 10, "plummer", 30_000, 1), (1, 6, "uniform", 40_000, 0),
                                           (1, 3, "plummer", 20_000, 0), (0, 12, "uniform", 10_000, 1),
                                           (0, 1, "uniform", 8_000, 1), (2, 2, "plummer", 8_000, 1)])
@pytest.mark.parametrize("want_phi", [True, False])
def test_fp32_tiled_m2l_matches_per_cell(orc, s, p, dist, n, h, want_phi):
    """The FP32 form's two SIMT M2L kernels -- over the tile plan (a block per
    chunk of key rows, a thread per target, the operator broadcast) and one block
    per target cell -- sum the same FP32 products in another order: the stored
    locals agree within 1e-5 column block by column block, the outputs within
    FP32 rounding, and the tiled result is within 1e-6 of the FP64 oracle.
    Column counts: 1 to 16 blocks of 8 (two targets per thread, the blocks
    split between two warp pairs; from p = 10 one target per thread); the
    harmonic p = 12 has 169 columns, more than the tiled kernel holds, and
    takes the per-cell kernel (no plan).  p = 1 and 2: a single block whose
    multipole groups are mostly padding.  Field only: the columns start at
    order 1."""
    import torch
    from gpu_util import rel_rms, to_dev
    from paper_2005_12351_gb300 import fmm
    pos, S = synth.make_system(n, s, dist, 1200 + 10 * s + p)
    out, Ls = {}, {}
    nL = (p + 1) ** 2 if h else (p + 1) * (p + 2) * (p + 3) // 6
    for tiled in (1, 0):
        t = fmm.create_tree(max_leaf=64, precision="fp32")
        t.set_tuning(m2l_harmonic=h, m2l_tiled=tiled)
        t.set_sources(to_dev(pos), to_dev(S), s)
        phi, E = t.evaluate(p, 0.5, want_phi, True)
        torch.cuda.synchronize()
        rows = t.info()["tc_rows"]
        assert (rows > 0) == (tiled == 1 and nL - (0 if want_phi else 1) <= 128 and p < 12), rows
        out[tiled] = (phi.cpu().numpy() if want_phi else None, E.cpu().numpy())
        Ls[tiled] = t.copy_array("local", nL).numpy()
        t.destroy()
    c0 = 0 if want_phi else 1                   # the order-0 local is not formed for the field alone
    for a in range(c0, nL, 64):
        assert rel_rms(Ls[1][:, a:a + 64], Ls[0][:, a:a + 64]) < 1e-5, a
    assert rel_rms(out[1][1], out[0][1]) < 1e-6
    if want_phi:
        assert rel_rms(out[1][0], out[0][0]) < 2e-6
    if p <= 6:
        ot = orc.Tree(pos, 64)
        ot.lists(0.5)
        phi_o, E_o = ot.fmm(S, s, p)
        assert rel_rms(out[1][1], E_o) < 1e-6
        if want_phi:
            assert rel_rms(out[1][0], phi_o) < 1e-6


@pytest.mark.parametrize("s", [1, 2])
def test_fp32_symmetric_batch_matches_alone(s):
    """The FP32 symmetric P2P gives each system of a batch the bits it gets alone
    (with the FP32 form's per-cell M2L: the tiles of the tiled and tensor-core
    M2L mix systems, and their chunks of key rows depend on the tile's other
    targets)."""
    import torch
    from gpu_util import to_dev
    from paper_2005_12351_gb300 import fmm
    pos, S, off = synth.make_batch(24, 300, 5000, s, 1901 + s, dist="plummer")
    tb = fmm.create_tree(max_leaf=32, precision="fp32")
    tb.set_tuning(p2p_variant=2, m2l_tiled=0)
    tb.set_sources_batch(to_dev(pos), to_dev(S), off, s)
    phi_b, E_b = tb.evaluate(4, 0.5)
    torch.cuda.synchronize()
    phi_b, E_b = phi_b.cpu().numpy(), E_b.cpu().numpy()
    for k in (0, 11, 23):
        a, b = int(off[k]), int(off[k + 1])
        (phi, E), t = gpu_eval(pos[a:b], S[a:b], s, 4, 0.5, 32, "fp32", p2p_variant=2, m2l_tiled=0)
        assert np.array_equal(phi, phi_b[a:b]) and np.array_equal(E, E_b[a:b]), k
        t.destroy()
    tb.destroy()


@pytest.mark.parametrize("precision", FORMS)
@pytest.mark.parametrize("s,dist", [(1, "uniform"), (2, "plummer")])
def test_p2p_tile_shapes_agree(orc, precision, s, dist):
    """The autotuner's P2P tile shapes (one or two targets per thread) sum the
    same pairs in another order: within FP32 rounding of each other, and each
    within 1e-6 of the oracle."""
    from gpu_util import rel_rms
    pos, S = synth.make_system(15_000, s, dist, 990 + s)
    out = {}
    for tt in (1, 2):
        import torch
        from gpu_util import to_dev
        from paper_2005_12351_gb300 import fmm
        tree = fmm.create_tree(max_leaf=64, precision=precision)
        tree.set_tuning(p2p_targets=tt)
        tree.set_sources(to_dev(pos), to_dev(S), s)
        phi, E = tree.evaluate(5, 0.5)
        torch.cuda.synchronize()
        out[tt] = (phi.cpu().numpy(), E.cpu().numpy())
    t = orc.Tree(pos, 64)
    t.lists(0.5)
    phi_o, E_o = t.fmm(S, s, 5)
    for tt in (1, 2):
        assert rel_rms(out[tt][1], E_o) < 1e-6 and rel_rms(out[tt][0], phi_o) < 1e-6
    assert rel_rms(out[1][1], out[2][1]) < 1e-6
