"""Pin of the harmonic M2L reading (§3.1 harmonic derivatives, Eq. (8)): the
GPU M2L folds each multipole onto the components with m_z <= 1, contracts
only the n with n_z <= 1 and derives the other L_n from the Laplace identity
D_{k+2x} + D_{k+2y} + D_{k+2z} = 0.  Restated here in numpy from the identity
and checked against the oracle's plain contraction (no GPU, no CUDA code)."""
import numpy as np
import pytest

import oracle as orc


def harmonic_m2l(s, p, zt, zs, Ms):
    m0 = orc.ntot(s - 1)
    nM, nL = orc.n_multipole(s, p), orc.n_local(p)
    mi = [orc.multi_index(i) for i in range(orc.ntot(p + s))]
    idx = {k: i for i, k in enumerate(mi)}
    v = np.array(Ms, dtype=float)
    # D_{n+m} M_m with m_z >= 2 is -(D_{n+m-2z+2x} + D_{n+m-2z+2y}) M_m
    for z in range(p + s - 2, -1, -1):
        for k in range(nM):
            x, y, zz = mi[k + m0]
            if zz != z:
                continue
            if x >= 2:
                v[k] -= v[idx[(x - 2, y, zz + 2)] - m0]
            if y >= 2:
                v[k] -= v[idx[(x, y - 2, zz + 2)] - m0]
    D = orc.derivatives(np.asarray(zt) - np.asarray(zs), p + s)
    L = np.zeros(nL)
    for n in range(nL):
        a = mi[n]
        if a[2] > 1:
            continue
        for k in range(nM):
            m = mi[k + m0]
            if m[2] <= 1 and sum(a) + sum(m) <= p + s:
                L[n] += D[idx[(a[0] + m[0], a[1] + m[1], a[2] + m[2])]] * v[k]
    for z in range(2, p + 1):
        for n in range(nL):
            a = mi[n]
            if a[2] == z:
                L[n] = -L[idx[(a[0] + 2, a[1], z - 2)]] - L[idx[(a[0], a[1] + 2, z - 2)]]
    return L


@pytest.mark.parametrize("s", [0, 1, 2])
@pytest.mark.parametrize("p", [1, 3, 6, 9])
def test_harmonic_m2l_equals_plain_contraction(s, p):
    rng = np.random.default_rng(100 * s + p)
    Ms = rng.standard_normal(orc.n_multipole(s, p))
    zt, zs = np.array([0.1, -0.2, 0.3]), np.array([2.1, 1.3, -1.7])
    Lf = orc.m2l(s, p, zt, zs, Ms)
    Lh = harmonic_m2l(s, p, zt, zs, Ms)
    assert np.abs(Lh - Lf).max() <= 1e-14 * np.abs(Lf).max()


def test_harmonic_count_at_p6():
    """Terms kept, s = 1, p = 6, field only (|n| >= 1): 749 of 1477."""
    s, p = 1, 6
    mi = [orc.multi_index(i) for i in range(orc.ntot(p + s))]
    full = sum(1 for n in mi[1:orc.ntot(p)] for m in mi[orc.ntot(s - 1):]
               if sum(n) + sum(m) <= p + s)
    harm = sum(1 for n in mi[1:orc.ntot(p)] for m in mi[orc.ntot(s - 1):]
               if sum(n) + sum(m) <= p + s and n[2] <= 1 and m[2] <= 1)
    assert (full, harm) == (1477, 749)


def unfold_locals(p, L):
    """The L_n with n_z >= 2 from the n_z <= 1 components, by the trace identity
    L_n = -L_{n+2x-2z} - L_{n+2y-2z} in increasing n_z (the stored form of the
    GPU's local expansions); the input's n_z >= 2 entries are ignored."""
    mi = [orc.multi_index(i) for i in range(orc.n_local(p))]
    idx = {k: i for i, k in enumerate(mi)}
    out = np.array(L, dtype=float)
    for n, a in enumerate(mi):
        if a[2] >= 2:
            out[n] = np.nan
    for z in range(2, p + 1):
        for n, a in enumerate(mi):
            if a[2] == z:
                out[n] = -out[idx[(a[0] + 2, a[1], z - 2)]] - out[idx[(a[0], a[1] + 2, z - 2)]]
    return out


@pytest.mark.parametrize("s", [0, 1, 2])
@pytest.mark.parametrize("p", [2, 5, 8])
def test_local_expansions_keep_only_the_traceless_components(s, p):
    """Storing only the (p+1)^2 locals with n_z <= 1 loses nothing: the oracle's
    M2L output (the plain Eq. (8) contraction, which knows nothing of the
    identity) satisfies L_n + ... = 0 for every n_z >= 2, an L2L shift of such
    an expansion (Eq. (9)-type Taylor shift) satisfies it again, and L2P at any
    point gives the same potential and field from the unfolded stored
    components as from the full row."""
    rng = np.random.default_rng(17 * s + p)
    zt, zs = np.array([0.1, -0.2, 0.3]), np.array([2.1, 1.3, -1.7])
    L = orc.m2l(s, p, zt, zs, rng.standard_normal(orc.n_multipole(s, p)))
    mi = [orc.multi_index(i) for i in range(orc.n_local(p))]
    assert sum(1 for a in mi if a[2] <= 1) == (p + 1) ** 2
    scale = np.abs(L).max()
    assert np.abs(unfold_locals(p, L) - L).max() <= 1e-13 * scale
    zc = zt + np.array([0.125, -0.0625, 0.25])
    Lc = orc.l2l(p, zt, zc, L)
    assert np.abs(unfold_locals(p, Lc) - Lc).max() <= 1e-13 * np.abs(Lc).max()
    for x in (zc + np.array([0.05, 0.1, -0.07]), zt - np.array([0.2, 0.01, 0.13])):
        phi_f, g_f = orc.l2p(p, zt, L, x)
        phi_s, g_s = orc.l2p(p, zt, unfold_locals(p, L), x)
        assert abs(phi_s - phi_f) <= 1e-13 * abs(phi_f) + 1e-300
        assert np.abs(g_s - g_f).max() <= 1e-13 * np.abs(g_f).max()


def test_a_dropped_trace_term_is_caught():
    """The unfold must use both partners of the identity: with one of them left
    out the stored form no longer reproduces the oracle's locals."""
    p = 5
    L = orc.m2l(1, p, np.zeros(3), np.array([1.7, -2.3, 1.1]),
                np.random.default_rng(3).standard_normal(orc.n_multipole(1, p)))
    mi = [orc.multi_index(i) for i in range(orc.n_local(p))]
    idx = {k: i for i, k in enumerate(mi)}
    bad = np.array(L)
    for z in range(2, p + 1):
        for n, a in enumerate(mi):
            if a[2] == z:
                bad[n] = -bad[idx[(a[0] + 2, a[1], z - 2)]]
    assert np.abs(bad - L).max() > 1e-3 * np.abs(L).max()
