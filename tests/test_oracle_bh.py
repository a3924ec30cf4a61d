"""Pins of the oracle's multipolar Barnes-Hut (§2 multipole potential, §3.2
Methods): closed forms of M2P, its exact gradient, the theta -> 0 limit
(every cell opened: the direct sum), convergence with p, and the paper's
remark that p = 1 dipoles can miss the field by over 100 % on single
particles (§4)."""
import numpy as np
import pytest

import oracle as orc
from paper_2005_12351_gb300 import synth


def rel_rms(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def cluster(n, s, seed, radius=0.1):
    rng = np.random.default_rng(seed)
    x = rng.uniform(-radius, radius, (n, 3)) / np.sqrt(3)
    S = synth.sources(n, seed, s)
    return x, S


def test_m2p_charge_is_total_charge_over_r():
    x, q = cluster(40, 0, 1)
    z = np.zeros(3)
    M = orc.p2m(0, 0, z, x, q)                      # order 0: M_0 = sum q
    X = np.array([1.3, -0.7, 2.1])
    f, g = orc.m2p(0, 0, z, M, X)
    Q, r = q.sum(), np.linalg.norm(X)
    assert f == pytest.approx(Q / r, rel=1e-14)
    assert np.allclose(g, -Q * X / r ** 3, rtol=1e-13, atol=0)


def test_m2p_dipole_order_one_is_net_dipole():
    x, mu = cluster(40, 1, 2)
    z = np.zeros(3)
    M = orc.p2m(1, 0, z, x, mu)                     # s = 1, order p = 1: M_(e_k) = sum mu_k
    assert np.allclose(M, mu.sum(axis=0), rtol=1e-14)
    X = np.array([-1.1, 0.4, 1.9])
    f, g = orc.m2p(1, 1, z, M, X)
    m, r = mu.sum(axis=0), np.linalg.norm(X)
    assert f == pytest.approx(-m.dot(X) / r ** 3, rel=1e-13)
    assert np.allclose(g, -m / r ** 3 + 3 * m.dot(X) * X / r ** 5, rtol=1e-12, atol=0)


@pytest.mark.parametrize("s", [0, 1, 2])
def test_m2p_field_is_gradient_of_potential(s):
    x, S = cluster(30, s, 3 + s)
    z = np.array([0.01, -0.02, 0.03])
    p = 5
    M = orc.p2m(s, p - s, z, x, S)
    X = np.array([0.9, 1.2, -0.8])
    _, g = orc.m2p(s, p, z, M, X)
    h = 1e-5
    fd = np.array([(orc.m2p(s, p, z, M, X + h * e)[0] - orc.m2p(s, p, z, M, X - h * e)[0]) / (2 * h)
                   for e in np.eye(3)])
    assert np.allclose(g, fd, rtol=1e-7, atol=1e-9 * np.abs(g).max())


@pytest.mark.parametrize("s", [0, 1, 2])
def test_m2p_converges_to_direct_far_away(s):
    x, S = cluster(60, s, 5 + s, radius=0.1)
    z = np.zeros(3)
    X = np.array([0.35, 0.2, -0.25])          # |X| ~ 4.7 x the cluster radius
    f_d, E_d = orc.direct(np.vstack([X, x]), np.vstack([np.zeros_like(S[:1]), S]), s, targets=np.array([0]))
    errs = []
    for p in range(s, s + 9):
        M = orc.p2m(s, p - s, z, x, S)
        f, g = orc.m2p(s, p, z, M, X)
        errs.append(np.linalg.norm(-g - E_d[0]) / np.linalg.norm(E_d[0]))
    assert all(b < a for a, b in zip(errs[2:], errs[3:]))
    assert errs[-1] < 1e-4


@pytest.mark.parametrize("s", [0, 1, 2])
def test_bh_theta_zero_is_direct_sum(s):
    pos, S = synth.make_system(1500, s, "plummer", 21 + s)
    phi, E = orc.bh(pos, S, s, s + 2, 0.0, 32)
    phi_d, E_d = orc.direct(pos, S, s)
    assert rel_rms(phi, phi_d) < 1e-13 and rel_rms(E, E_d) < 1e-13


def test_bh_error_falls_with_order_and_p1_dipoles_can_exceed_100_percent():
    pos, S = synth.make_system(20_000, 1, "uniform", 11)
    t = orc.Tree(pos, 128)
    _, E_d = orc.direct(pos, S, 1)
    med, worst = [], []
    for p in (1, 2, 4):
        _, E = t.bh(S, 1, p, 0.5)
        err = np.linalg.norm(E - E_d, axis=1) / np.linalg.norm(E_d, axis=1)
        med.append(np.median(err))
        worst.append(err.max())
    assert med[0] > med[1] > med[2]
    assert worst[0] > 1.0                       # §4: over 100 % on individual particles
    _, E8 = t.bh(S, 1, 8, 0.25)
    assert rel_rms(E8, E_d) < 1e-5
