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
