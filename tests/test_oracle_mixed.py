"""Pins of the oracle's mixed source orders (§2: "mixed systems"; the expansion
starts at the lowest order present, s_lo).  Every step is linear in the
moments, so a mixed system is the sum of its shells; with the truncation of
R1 the FMM of the mixed system at order p equals the sum over shells s of the
single-order FMM at order p - (s - s_lo) (same multipole range s_lo..p+s_lo,
same M2L cut |n| + |m| <= p + s_lo; the extra local terms carry zero), and the
Barnes-Hut sum at order p that of the single-order Barnes-Hut at the same p."""
import numpy as np
import pytest

import oracle as orc
from paper_2005_12351_gb300 import synth

RANGES = [(0, 1), (1, 2), (0, 2)]


def rel_rms(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def shells(S, lo, hi):
    offs = [orc.ntot(s - 1) - orc.ntot(lo - 1) for s in range(lo, hi + 2)]
    return {s: S[:, offs[s - lo]:offs[s - lo + 1]] for s in range(lo, hi + 1)}


@pytest.mark.parametrize("lo,hi", RANGES)
def test_mixed_pair_and_direct_are_sums_of_shells(lo, hi):
    pos, S = synth.make_system_mixed(1500, lo, hi, "plummer", 31 + lo + hi)
    assert S.shape[1] == orc.n_source(lo, hi)
    sh = shells(S, lo, hi)
    f, g = orc.p2p_pair(lo, pos[0], pos[1], S[1], s_hi=hi)
    f2 = sum(orc.p2p_pair(s, pos[0], pos[1], sh[s][1])[0] for s in sh)
    g2 = sum(orc.p2p_pair(s, pos[0], pos[1], sh[s][1])[1] for s in sh)
    assert f == pytest.approx(f2, rel=1e-14) and np.allclose(g, g2, rtol=1e-14, atol=0)
    phi, E = orc.direct(pos, S, lo, s_hi=hi)
    parts = [orc.direct(pos, sh[s], s) for s in sh]
    assert rel_rms(phi, sum(q[0] for q in parts)) < 1e-14
    assert rel_rms(E, sum(q[1] for q in parts)) < 1e-14


@pytest.mark.parametrize("lo,hi", RANGES)
def test_mixed_fmm_is_sum_of_single_orders_at_shifted_p(lo, hi):
    pos, S = synth.make_system_mixed(4000, lo, hi, "plummer", 41 + lo + hi)
    t = orc.Tree(pos, 32)
    t.lists(0.5)
    p = 6
    phi, E = t.fmm(S, lo, p, s_hi=hi)
    parts = [t.fmm(Ss, s, p - (s - lo)) for s, Ss in shells(S, lo, hi).items()]
    assert rel_rms(phi, sum(q[0] for q in parts)) < 1e-13
    assert rel_rms(E, sum(q[1] for q in parts)) < 1e-13
    phi_d, E_d = orc.direct(pos, S, lo, s_hi=hi)
    assert rel_rms(E, E_d) < 1e-3


@pytest.mark.parametrize("lo,hi", RANGES)
def test_mixed_bh_is_sum_of_single_orders(lo, hi):
    pos, S = synth.make_system_mixed(3000, lo, hi, "uniform", 51 + lo + hi)
    t = orc.Tree(pos, 32)
    phi, E = t.bh(S, lo, 5, 0.4, s_hi=hi)
    parts = [t.bh(Ss, s, 5, 0.4) for s, Ss in shells(S, lo, hi).items()]
    assert rel_rms(phi, sum(q[0] for q in parts)) < 1e-13
    assert rel_rms(E, sum(q[1] for q in parts)) < 1e-13
