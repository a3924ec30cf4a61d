"""Pins of the CPU oracle to things other than itself (CPU only).

Each test ties one oracle function to the paper's printed example, a closed
form, an identity of the mathematics, or brute force, so that a dropped
term, a wrong sign or index, or a transposed operand fails somewhere here.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2005_12351_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def shells(order):
    """Multi-indices |n| <= order in the order the tests expect (independent enumeration)."""
    out = []
    for k in range(order + 1):
        for nx in range(k, -1, -1):
            for ny in range(k - nx, -1, -1):
                out.append((nx, ny, k - nx - ny))
    return out


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


# ------------------------------------------------------------- index map
def test_index_order_matches_paper_prefix(orc):
    g = json.load(open(os.path.join(GOLD, "index_order.json")))
    for i, n in enumerate(g["prefix"]):
        assert orc.multi_index(i) == tuple(n)
        assert orc.index(*n) == i


def test_index_roundtrip_and_counts(orc):
    ns = shells(12)
    assert orc.ntot(12) == len(ns) == 455
    for i, n in enumerate(ns):
        assert orc.index(*n) == i and orc.multi_index(i) == n
    # storage sizes used by the scope table: s=1,p=6 -> 119 / 84; s=2,p=10 -> 451 / 286
    assert orc.n_multipole(1, 6) == 119 and orc.n_local(6) == 84
    assert orc.n_multipole(1, 8) == 219 and orc.n_local(8) == 165
    assert orc.n_multipole(2, 5) == 116 and orc.n_multipole(2, 10) == 451


# ------------------------------------------------------ derivative tensors
R0 = np.array([0.37, -0.52, 0.81])


def test_derivatives_closed_forms_orders_0_to_3(orc):
    x = R0
    r = np.linalg.norm(x)
    D = orc.derivatives(x, 3)
    d = np.eye(3)
    for n in shells(3):
        axes = [a for a in range(3) for _ in range(n[a])]
        k = len(axes)
        if k == 0:
            ref = 1 / r
        elif k == 1:
            i, = axes
            ref = -x[i] / r ** 3
        elif k == 2:
            i, j = axes
            ref = 3 * x[i] * x[j] / r ** 5 - d[i, j] / r ** 3
        else:
            i, j, l = axes
            ref = (-15 * x[i] * x[j] * x[l] / r ** 7
                   + 3 * (d[i, j] * x[l] + d[i, l] * x[j] + d[j, l] * x[i]) / r ** 5)
        assert abs(D[orc.index(*n)] - ref) <= 1e-14 * max(1.0, abs(ref)), n


@pytest.mark.parametrize("order", [4, 6, 9])
def test_derivatives_against_finite_differences(orc, order):
    """D_{n+e_k} from Richardson-extrapolated central differences of D_n."""
    D = orc.derivatives(R0, order)
    scale = np.abs(D).max()
    for n in shells(order - 1):
        for k in range(3):
            def f(h):
                e = np.zeros(3)
                e[k] = h
                return (orc.derivatives(R0 + e, order - 1)[orc.index(*n)]
                        - orc.derivatives(R0 - e, order - 1)[orc.index(*n)]) / (2 * h)
            h = 1e-3
            fd = (4 * f(h / 2) - f(h)) / 3
            m = list(n)
            m[k] += 1
            assert abs(fd - D[orc.index(*m)]) < 2e-6 * scale, (n, k)


def test_derivatives_traceless_euler_parity_homogeneity(orc):
    P = 12
    D = orc.derivatives(R0, P)
    Dm = orc.derivatives(-R0, P)
    D2 = orc.derivatives(2.0 * R0, P)
    r = np.linalg.norm(R0)
    for n in shells(P - 2):
        nx, ny, nz = n
        tr = (D[orc.index(nx + 2, ny, nz)] + D[orc.index(nx, ny + 2, nz)]
              + D[orc.index(nx, ny, nz + 2)])
        mag = max(abs(D[orc.index(nx + 2, ny, nz)]), abs(D[orc.index(nx, ny + 2, nz)]),
                  abs(D[orc.index(nx, ny, nz + 2)]), 1e-300)
        assert abs(tr) <= 1e-12 * mag, n            # Laplace (§3.1 harmonic relation)
    for n in shells(P - 1):
        nx, ny, nz = n
        k = nx + ny + nz
        euler = (R0[0] * D[orc.index(nx + 1, ny, nz)] + R0[1] * D[orc.index(nx, ny + 1, nz)]
                 + R0[2] * D[orc.index(nx, ny, nz + 1)])
        assert abs(euler + (k + 1) * D[orc.index(*n)]) <= 1e-12 * abs(D).max() * r
    for n in shells(P):
        i = orc.index(*n)
        k = sum(n)
        assert Dm[i] == pytest.approx((-1) ** k * D[i], rel=1e-13, abs=1e-13 * abs(D).max())
        # power-of-two scaling is exact in IEEE arithmetic
        assert D2[i] == math.ldexp(D[i], -(k + 1))


# ------------------------------------------------- the printed M2L example
def test_m2l_1_listing(orc):
    g = json.load(open(os.path.join(GOLD, "m2l_1_listing.json")))
    s, p = g["s"], g["p"]
    for i, n in enumerate(g["index_order"]):
        assert orc.multi_index(i) == tuple(n)
    rng = np.random.default_rng(3)
    for _ in range(5):
        zt, zs = rng.normal(size=3), rng.normal(size=3)
        M = rng.normal(size=4)
        x, y, z = zt - zs
        R = math.sqrt(x * x + y * y + z * z)
        Dl = [eval(e, {"__builtins__": {}}, dict(x=x, y=y, z=z, R=R)) for e in g["D"]]
        Lref = [sum(Dl[d] * M[m] for d, m in terms) for terms in g["L_terms"]]
        L = orc.m2l(s, p, zt, zs, M)
        assert np.allclose(L, Lref, rtol=1e-14, atol=0)


# --------------------------------------------------------------------- P2M
def test_p2m_charge_matches_eq3(orc):
    """Eq. (3): M_n(z) = (-1)^|n| q (x - z)^n / n!."""
    rng = np.random.default_rng(5)
    z = np.array([0.5, 0.5, 0.5])
    x = z + rng.uniform(-0.1, 0.1, size=3)
    q = 0.7
    p = 5
    M = orc.p2m(0, p, z, x[None], [q])
    for n in shells(p):
        ref = (-1) ** sum(n) * q * np.prod([(x[a] - z[a]) ** n[a] / math.factorial(n[a])
                                             for a in range(3)])
        assert abs(M[orc.index(*n)] - ref) <= 1e-15 * max(1, abs(ref))


@pytest.mark.parametrize("s", [1, 2])
def test_p2m_source_at_centre(orc, s):
    """A source sitting on the expansion centre is its own lowest shell."""
    z = np.array([0.1, 0.2, 0.3])
    S = np.arange(1, 4 if s == 1 else 7, dtype=float)
    M = orc.p2m(s, 4, z, z[None], S)
    nS = len(S)
    assert np.array_equal(M[:nS], S) and not M[nS:].any()


def test_multipole_reproduces_far_potential(orc):
    """sum_n M_n D_n(x - z) tends to the exact source potential (Eq. (6) as read)."""
    rng = np.random.default_rng(8)
    z = np.zeros(3)
    pos = rng.uniform(-0.1, 0.1, size=(20, 3))
    S = rng.normal(size=(20, 3))
    xt = np.array([0.9, -0.6, 0.7])
    exact = sum(orc.p2p_pair(1, xt, pos[j], S[j])[0] for j in range(20))
    errs = []
    for p in (1, 3, 5, 7):
        M = orc.p2m(1, p, z, pos, S)
        D = orc.derivatives(xt - z, p + 1)
        approx = sum(M[i] * D[i + 1] for i in range(len(M)))
        errs.append(abs(approx - exact) / abs(exact))
    assert errs == sorted(errs, reverse=True) and errs[-1] < 1e-6


# -------------------------------------------------------------- M2M / L2L
@pytest.mark.parametrize("s,p", [(0, 4), (1, 6), (2, 5)])
def test_m2m_exact_composition(orc, s, p):
    """P2M at the children then M2M to the parent equals P2M at the parent."""
    rng = np.random.default_rng(11)
    zp = np.array([0.5, 0.5, 0.5])
    nS = (s + 1) * (s + 2) // 2
    Mp = np.zeros(orc.n_multipole(s, p))
    allpos, allS = [], []
    for o in range(8):
        zc = zp + 0.25 * np.array([1 if o & 4 else -1, 1 if o & 2 else -1, 1 if o & 1 else -1])
        pos = zc + rng.uniform(-0.25, 0.25, size=(7, 3))
        S = rng.normal(size=(7, nS))
        Mc = orc.p2m(s, p, zc, pos, S)
        Mp = orc.m2m(s, p, zc, zp, Mc, Mp)
        allpos.append(pos)
        allS.append(S)
    Mref = orc.p2m(s, p, zp, np.concatenate(allpos), np.concatenate(allS))
    assert rel(Mp, Mref) < 1e-13


def test_l2l_exact_polynomial_shift(orc):
    """L2P(L2L(L)) equals L2P(L): re-centring a degree-p polynomial is exact."""
    rng = np.random.default_rng(12)
    p = 7
    zp, zc = np.array([0.5, 0.5, 0.5]), np.array([0.25, 0.75, 0.25])
    L = rng.normal(size=orc.n_local(p))
    Lc = orc.l2l(p, zp, zc, L)
    for _ in range(5):
        x = zc + rng.uniform(-0.25, 0.25, size=3)
        f0, g0 = orc.l2p(p, zp, L, x)
        f1, g1 = orc.l2p(p, zc, Lc, x)
        assert abs(f1 - f0) <= 1e-13 * np.abs(L).sum() and rel(g1, g0) < 1e-12


def test_l2p_derivative_matches_finite_difference(orc):
    rng = np.random.default_rng(13)
    p = 6
    z = np.zeros(3)
    L = rng.normal(size=orc.n_local(p))
    x = np.array([0.1, -0.2, 0.15])
    f, g = orc.l2p(p, z, L, x)
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1e-5
        fd = (orc.l2p(p, z, L, x + e)[0] - orc.l2p(p, z, L, x - e)[0]) / 2e-5
        assert abs(fd - g[k]) < 1e-7 * np.abs(L).sum()


@pytest.mark.parametrize("s", [0, 1, 2])
def test_m2l_l2p_converges_to_direct(orc, s):
    """Well separated clusters: P2M -> M2L -> L2P approaches the direct sum in p."""
    rng = np.random.default_rng(14 + s)
    zs, zt = np.zeros(3), np.array([2.0, 0.8, -0.6])
    nS = (s + 1) * (s + 2) // 2
    src = rng.uniform(-0.15, 0.15, size=(15, 3))
    S = rng.normal(size=(15, nS))
    x = zt + rng.uniform(-0.15, 0.15, size=3)
    ef, eg = 0.0, np.zeros(3)
    for j in range(15):
        f, g = orc.p2p_pair(s, x, src[j], S[j])
        ef += f
        eg += g
    prev = np.inf
    for p in (2, 4, 6, 8):
        M = orc.p2m(s, p, zs, src, S)
        L = orc.m2l(s, p, zt, zs, M)
        f, g = orc.l2p(p, zt, L, x)
        err = np.linalg.norm(g - eg) / np.linalg.norm(eg)
        assert err < prev
        prev = err
    assert prev < 1e-5


# --------------------------------------------------------------------- P2P
def test_p2p_closed_forms(orc):
    rng = np.random.default_rng(21)
    xs = rng.normal(size=3)
    xt = xs + np.array([0.3, -0.4, 0.5])
    R = xt - xs
    r = np.linalg.norm(R)
    # charge: phi = q/r, E = q R / r^3 (Eq. (1))
    f, g = orc.p2p_pair(0, xt, xs, [2.5])
    assert f == pytest.approx(2.5 / r, rel=1e-15)
    assert np.allclose(-g, 2.5 * R / r ** 3, rtol=1e-14)
    # dipole in the S convention: phi = -S.R/r^3, E = S/r^3 - 3 (S.R) R / r^5
    S = np.array([0.2, -0.7, 0.4])
    f, g = orc.p2p_pair(1, xt, xs, S)
    assert f == pytest.approx(-S @ R / r ** 3, rel=1e-14)
    assert np.allclose(-g, S / r ** 3 - 3 * (S @ R) * R / r ** 5, rtol=1e-13)
    # quadrupole tensor Q with S_n = Q_n / n!: phi = 3/2 R.Q.R / r^5
    Q = synth.quadrupole_tensors(1, 99)[0]
    Sq = synth.quadrupole_sources(Q[None])[0]
    f, g = orc.p2p_pair(2, xt, xs, Sq)
    assert f == pytest.approx(1.5 * R @ Q @ R / r ** 5, rel=1e-13)
    grad = 3 * (Q @ R) / r ** 5 - 7.5 * (R @ Q @ R) * R / r ** 7
    assert np.allclose(g, grad, rtol=1e-12)
    # coincident points contribute nothing
    f, g = orc.p2p_pair(1, xs, xs, S)
    assert f == 0.0 and not g.any()


def test_direct_sum_brute_force(orc):
    rng = np.random.default_rng(22)
    n = 40
    pos = rng.uniform(size=(n, 3))
    q = rng.uniform(-1, 1, size=n)
    phi, E = orc.direct(pos, q[:, None], 0)
    for i in range(n):
        R = pos[i] - np.delete(pos, i, axis=0)
        r = np.linalg.norm(R, axis=1)
        qq = np.delete(q, i)
        assert phi[i] == pytest.approx((qq / r).sum(), rel=1e-13)
        assert np.allclose(E[i], (qq[:, None] * R / r[:, None] ** 3).sum(0), rtol=1e-12)
    tg = np.array([3, 17, 0])
    phi2, E2 = orc.direct(pos, q[:, None], 0, targets=tg)
    assert np.array_equal(phi2, phi[tg]) and np.array_equal(E2, E[tg])


# ------------------------------------------------------------------- tree
def _coverage(t):
    cov = np.zeros((t.n, t.n), dtype=np.int32)
    for a, b in np.concatenate([t.m2l, t.p2p]):
        ia = t.perm[t.begin[a]:t.end[a]]
        ib = t.perm[t.begin[b]:t.end[b]]
        cov[np.ix_(ia, ib)] += 1
    return cov


@pytest.mark.parametrize("dist,theta,ncrit", [("uniform", 0.5, 8), ("plummer", 0.5, 6),
                                              ("uniform", 0.3, 4), ("plummer", 0.8, 10)])
def test_tree_lists_cover_every_pair_once(orc, dist, theta, ncrit):
    pos, _ = synth.make_system(700, 0, dist, 31)
    t = orc.Tree(pos, ncrit)
    t.lists(theta)
    assert (_coverage(t) == 1).all()
    # accepted pairs satisfy the MAC of Eq. (13) geometrically (r = half side)
    a, b = t.m2l[:, 0], t.m2l[:, 1]
    R = np.linalg.norm(t.centre[a] - t.centre[b], axis=1)
    assert ((t.halfw[a] + t.halfw[b]) / R < theta * (1 + 1e-12)).all()
    # P2P pairs are leaf pairs; lists are sorted by (target, source)
    assert (t.nchild[t.p2p].ravel() == 0).all()
    for L in (t.m2l, t.p2p):
        key = L[:, 0] * t.ncells + L[:, 1]
        assert (np.diff(key) > 0).all()


def test_tree_structure_invariants(orc):
    pos, _ = synth.make_system(5000, 0, "plummer", 32)
    t = orc.Tree(pos, 16)
    # keys sorted, perm a permutation, equal keys in original-index order
    assert (np.diff(t.keys.astype(object)) >= 0).all()
    assert np.array_equal(np.sort(t.perm), np.arange(t.n))
    eq = t.keys[1:] == t.keys[:-1]
    assert (t.perm[1:][eq] > t.perm[:-1][eq]).all()
    # cells in (level, prefix) order; children partition the parent's range
    assert (np.diff(t.level) >= 0).all()
    for c in range(t.ncells):
        if t.nchild[c]:
            ch = np.arange(t.child_first[c], t.child_first[c] + t.nchild[c])
            assert t.begin[ch[0]] == t.begin[c] and t.end[ch[-1]] == t.end[c]
            assert (t.begin[ch[1:]] == t.end[ch[:-1]]).all()
            assert (t.parent[ch] == c).all() and (t.level[ch] == t.level[c] + 1).all()
            assert t.end[c] - t.begin[c] > 16
        else:
            assert t.end[c] - t.begin[c] <= 16 or t.level[c] == 21
    # every particle lies in its leaf's box
    for c in np.nonzero(t.nchild == 0)[0]:
        x = pos[t.perm[t.begin[c]:t.end[c]]]
        assert (np.abs(x - t.centre[c]) <= t.halfw[c] * (1 + 1e-12)).all()


def test_tree_duplicates_and_degenerate_sizes(orc):
    # many coincident points: a leaf cannot split below level 21
    pos = np.repeat(np.array([[0.25, 0.5, 0.75]]), 50, axis=0)
    pos = np.concatenate([pos, synth.uniform_cube(30, 4)])
    t = orc.Tree(pos, 8)
    t.lists(0.5)
    assert (_coverage(t) == 1).all()
    assert t.level.max() == 21
    S = np.ones((len(pos), 1))
    phid, Ed = orc.direct(pos, S, 0)
    errs = []
    for p in (2, 5, 8):
        phi, E = t.fmm(S, 0, p)
        assert np.isfinite(phi).all() and np.isfinite(E).all()
        errs.append(rel(E, Ed))
    # r_cell is half the side, so a corner particle converges at sqrt(3) theta: slow but monotone
    assert errs == sorted(errs, reverse=True) and errs[-1] < 0.5 * errs[0]
    # N = 1 and N = 0
    t1 = orc.Tree(np.array([[0.3, 0.3, 0.3]]), 8)
    t1.lists(0.5)
    assert t1.ncells == 1 and len(t1.p2p) == 1
    phi, E = t1.fmm(np.ones((1, 1)), 0, 4)
    assert phi[0] == 0.0 and not E.any()
    t0 = orc.Tree(np.zeros((0, 3)), 8)
    t0.lists(0.5)
    assert t0.n == 0 and t0.ncells == 0


def test_tree_keys_match_independent_morton(orc):
    pos = synth.uniform_cube(300, 5) * 3.0 - 1.0
    t = orc.Tree(pos, 8)
    lo = pos.min(0)
    ext = (pos.max(0) - lo).max()
    side = 2.0 ** math.ceil(math.log2(ext))
    assert t.side == side and np.array_equal(t.lo, lo)
    q = np.minimum(np.floor((pos - lo) * (2 ** 21 / side)).astype(np.int64), 2 ** 21 - 1)
    keys = np.zeros(len(pos), dtype=np.uint64)
    for b in range(21):
        for a in range(3):
            keys |= (((q[:, a] >> b) & 1).astype(np.uint64) << np.uint64(3 * b + 2 - a))
    order = np.lexsort((np.arange(len(pos)), keys))
    assert np.array_equal(t.perm, order) and np.array_equal(t.keys, keys[order])


# -------------------------------------------------------------------- FMM
@pytest.mark.parametrize("s", [0, 1, 2])
def test_fmm_single_leaf_is_direct(orc, s):
    pos, S = synth.make_system(64, s, "uniform", 40 + s)
    phi, E = orc.fmm(pos, S, s, 4, 0.5, ncrit=64)
    phid, Ed = orc.direct(pos, S, s)
    assert rel(phi, phid) < 1e-13 and rel(E, Ed) < 1e-13


@pytest.mark.parametrize("s", [0, 1, 2])
def test_fmm_error_falls_with_order(orc, s):
    pos, S = synth.make_system(1500, s, "uniform", 50 + s)
    t = orc.Tree(pos, 32)
    t.lists(0.5)
    phid, Ed = orc.direct(pos, S, s)
    errs = []
    for p in (2, 4, 6, 8):
        _, E = t.fmm(S, s, p)
        errs.append(np.sqrt(((E - Ed) ** 2).sum() / (Ed ** 2).sum()))
    assert errs == sorted(errs, reverse=True)
    assert errs[-1] < 0.25 * errs[0]


def test_fmm_linear_in_sources(orc):
    pos, S1 = synth.make_system(800, 1, "plummer", 60)
    S2 = synth.unit_dipoles(800, 61)
    t = orc.Tree(pos, 16)
    t.lists(0.5)
    f1, e1 = t.fmm(S1, 1, 5)
    f2, e2 = t.fmm(S2, 1, 5)
    f3, e3 = t.fmm(S1 + 2.0 * S2, 1, 5)
    assert rel(f3, f1 + 2.0 * f2) < 1e-13 and rel(e3, e1 + 2.0 * e2) < 1e-13


def test_fmm_scale_invariance(orc):
    """Power-of-two scaling: same tree, phi scales by 2^-(k(s+1)), E by 2^-(k(s+2))."""
    pos, S = synth.make_system(600, 1, "uniform", 62)
    phi, E = orc.fmm(pos, S, 1, 5, 0.5, 16)
    phi2, E2 = orc.fmm(pos * 2.0 ** -30, S, 1, 5, 0.5, 16)
    assert rel(phi2 * 2.0 ** -60, phi) < 1e-12 and rel(E2 * 2.0 ** -90, E) < 1e-12


def test_fmm_sampled_targets_equal_full(orc):
    pos, S = synth.make_system(3000, 2, "uniform", 63)
    t = orc.Tree(pos, 40)
    t.lists(0.5)
    phi, E = t.fmm(S, 2, 4)
    tg = synth.sample_indices(3000, 50, 1)
    phis, Es = t.fmm(S, 2, 4, targets=tg)
    assert rel(phis, phi[tg]) < 1e-14 and rel(Es, E[tg]) < 1e-14


def test_fmm_small_theta_is_direct(orc):
    pos, S = synth.make_system(400, 0, "uniform", 64)
    phi, E = orc.fmm(pos, S, 0, 3, 1e-3, 8)
    phid, Ed = orc.direct(pos, S, 0)
    assert rel(phi, phid) < 1e-12 and rel(E, Ed) < 1e-12


# ----------------------------------------------------------------- inputs
def test_synth_inputs():
    a = synth.uniform_cube(1000, 1)
    assert np.array_equal(a, synth.uniform_cube(1000, 1)) and (a >= 0).all() and (a < 1).all()
    d = synth.unit_dipoles(1000, 2)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0)
    assert abs(d.mean(0)).max() < 0.1
    Q = synth.quadrupole_tensors(100, 3)
    assert np.allclose(np.trace(Q, axis1=1, axis2=2), 0) and np.allclose(Q, Q.transpose(0, 2, 1))
    pl = synth.plummer(20000, 4)
    r = np.linalg.norm(pl - 0.5, axis=1)
    assert r.max() <= 1.0 + 1e-12 and 0.05 < np.median(r) < 0.2
    n = synth.log_uniform_int(5000, 256, 65536, 5)
    assert n.min() >= 256 and n.max() <= 65536 and 9000 < n.mean() < 14000
