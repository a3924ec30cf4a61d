"""Seeded synthetic inputs for the Cartesian FMM workloads.

This module holds no FMM arithmetic: it only draws positions and source
moments.  Both the GPU path (tests, bench) and the CPU oracle's tests take
their inputs from here, so the two sides see identical bytes.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used counter-style -- value i of stream t is
``mix(key(seed, t) + (i + 1) * GOLDEN)`` -- and converted to a double in
[0, 1) as ``(z >> 11) * 2**-53``.  Everything is vectorised numpy uint64
arithmetic (wrapping), so results are identical on x86-64 and aarch64.

Source moments follow the paper's source convention (S_n with |n| = s, §2,
Eq. (5) and the text around it): a charge is S_(000) = q, a dipole is
S_(100), S_(010), S_(001), a quadrupole is the six S_n with |n| = 2 stored in
graded-lexicographic order (200), (110), (101), (020), (011), (002).  A
physical quadrupole tensor Q enters as S_n = Q_n / n!, i.e.
(Qxx/2, Qxy, Qxz, Qyy/2, Qyz, Qzz/2).
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream tags: one independent counter stream per drawn quantity
_POS, _MOM, _AUX, _PLUMMER_R, _PLUMMER_DIR, _SAMPLE = 1, 2, 3, 4, 5, 6


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        a = _mix(np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF)], dtype=np.uint64))
        b = _mix(np.array([np.uint64((stream * 0x632BE59BD9B4E019) & 0xFFFFFFFFFFFFFFFF)],
                          dtype=np.uint64))
    return np.uint64(a[0] ^ b[0])


def uniform01(seed: int, stream: int, count: int) -> np.ndarray:
    """``count`` doubles in [0, 1) from stream ``stream`` of ``seed``."""
    i = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _mix(_key(seed, stream) + i * _GOLDEN)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def gaussian(seed: int, stream: int, count: int) -> np.ndarray:
    """Standard normal draws by Box-Muller from two uniform streams."""
    u = uniform01(seed, stream, 2 * count).reshape(count, 2)
    u1 = 1.0 - u[:, 0]            # (0, 1]
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u[:, 1])


# ---------------------------------------------------------------- positions
def uniform_cube(n: int, seed: int) -> np.ndarray:
    """Positions uniform in the unit cube [0, 1)^3, shape (n, 3)."""
    return uniform01(seed, _POS, 3 * n).reshape(n, 3)


def plummer(n: int, seed: int, a: float = 0.1, r_max_over_a: float = 10.0) -> np.ndarray:
    """Plummer-sphere positions centred on (0.5, 0.5, 0.5).

    Enclosed mass fraction of a Plummer sphere is m(r) = x^3 / (1 + x^2)^{3/2}
    with x = r / a; inverting, r = a / sqrt(m^{-2/3} - 1).  Drawing m uniform
    in (0, m(r_max)] truncates the sphere at r_max = r_max_over_a * a.
    """
    x = r_max_over_a
    m_max = x ** 3 / (1.0 + x * x) ** 1.5
    m = m_max * (1.0 - uniform01(seed, _PLUMMER_R, n))          # (0, m_max]
    r = a / np.sqrt(m ** (-2.0 / 3.0) - 1.0)
    u = uniform01(seed, _PLUMMER_DIR, 2 * n).reshape(n, 2)
    cos_t = 2.0 * u[:, 0] - 1.0
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    ph = 2.0 * math.pi * u[:, 1]
    out = np.empty((n, 3))
    out[:, 0] = 0.5 + r * sin_t * np.cos(ph)
    out[:, 1] = 0.5 + r * sin_t * np.sin(ph)
    out[:, 2] = 0.5 + r * cos_t
    return out


# ------------------------------------------------------------------ moments
def charges(n: int, seed: int) -> np.ndarray:
    """Monopole sources S_(000) = q with q uniform in [-1, 1), shape (n, 1)."""
    return (2.0 * uniform01(seed, _MOM, n) - 1.0).reshape(n, 1)


def unit_dipoles(n: int, seed: int) -> np.ndarray:
    """Dipole sources (S_(100), S_(010), S_(001)): isotropic unit vectors."""
    g = gaussian(seed, _MOM, 3 * n).reshape(n, 3)
    nrm = np.sqrt((g * g).sum(axis=1, keepdims=True))
    nrm[nrm == 0.0] = 1.0
    return g / nrm


def quadrupole_tensors(n: int, seed: int) -> np.ndarray:
    """Symmetric traceless 3x3 tensors Q = (G + G^T)/2 - tr(G)/3 I, G ~ N(0,1)."""
    g = gaussian(seed, _MOM, 9 * n).reshape(n, 3, 3)
    q = 0.5 * (g + np.transpose(g, (0, 2, 1)))
    tr = np.trace(q, axis1=1, axis2=2) / 3.0
    q[:, 0, 0] -= tr
    q[:, 1, 1] -= tr
    q[:, 2, 2] -= tr
    return q


def quadrupole_sources(q: np.ndarray) -> np.ndarray:
    """S_n = Q_n / n! in graded-lexicographic order, shape (n, 6)."""
    return np.stack([q[:, 0, 0] / 2.0, q[:, 0, 1], q[:, 0, 2],
                     q[:, 1, 1] / 2.0, q[:, 1, 2], q[:, 2, 2] / 2.0], axis=1)


def sources(n: int, seed: int, s: int) -> np.ndarray:
    """Moments for source order s (0 charge, 1 unit dipole, 2 quadrupole)."""
    if s == 0:
        return charges(n, seed)
    if s == 1:
        return unit_dipoles(n, seed)
    if s == 2:
        return quadrupole_sources(quadrupole_tensors(n, seed))
    raise ValueError("source order must be 0, 1 or 2")


def sources_mixed(n: int, seed: int, s_lo: int, s_hi: int) -> np.ndarray:
    """Moments of every order s_lo..s_hi per particle (charge, dipole, quadrupole
    shells side by side in graded order), each shell drawn as sources(., ., s)."""
    return np.hstack([sources(n, seed + 101 * s, s) for s in range(s_lo, s_hi + 1)])


def sample_indices(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct particle indices in [0, n), sorted (for sampled checks)."""
    k = min(k, n)
    if k == n:
        return np.arange(n, dtype=np.int64)
    u = uniform01(seed, _SAMPLE, n)
    return np.sort(np.argsort(u, kind="stable")[:k]).astype(np.int64)


def log_uniform_int(count: int, lo: int, hi: int, seed: int, stream: int = _AUX) -> np.ndarray:
    """round(exp(U(ln lo, ln hi))) -- system sizes for the batch and serving mixes."""
    u = uniform01(seed, stream, count)
    return np.rint(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)


# ------------------------------------------------------------ named workloads
WORKLOADS = {
    # name: (n, source order, p, theta, n_crit, distribution, seed)
    "monopole_2k_p4": dict(n=2000, s=0, p=4, theta=0.5, ncrit=64, dist="uniform", seed=20260000),
    "dipole_1m_p6": dict(n=1_000_000, s=1, p=6, theta=0.5, ncrit=128, dist="uniform", seed=20260001),
    # same leaf occupancy as the 1M workload (leaves one level higher): profiling-size case
    "dipole_125k_p6": dict(n=125_000, s=1, p=6, theta=0.5, ncrit=128, dist="uniform", seed=20260011),
    # inputs larger than L2 (4M x 48 B): the case for HBM counters of the per-particle kernels
    "dipole_4m_p6": dict(n=4_000_000, s=1, p=6, theta=0.5, ncrit=128, dist="uniform", seed=20260012),
    "dipole_plummer_4m_p8": dict(n=4_000_000, s=1, p=8, theta=0.5, ncrit=128, dist="plummer",
                                 seed=20260002),
    # 4,096 independent uniform-cube systems, N log-uniform in [256, 65536], quadrupoles
    "quadrupole_batch_4096_p5": dict(batch=4096, nlo=256, nhi=65536, s=2, p=5, theta=0.5,
                                     ncrit=128, dist="uniform", seed=20260003),
}


def make_batch(count: int, lo: int, hi: int, s: int, seed: int, dist: str = "uniform"):
    """A batch of independent systems with sizes round(exp(U(ln lo, ln hi))).

    Returns (positions (N,3), moments (N, T(s)), offsets (count+1,)), systems
    concatenated; system k is drawn from seed*7919 + k.
    """
    sizes = log_uniform_int(count, lo, hi, seed)
    off = np.zeros(count + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    pos = np.empty((int(off[-1]), 3))
    mom = np.empty((int(off[-1]), (s + 1) * (s + 2) // 2))
    for k in range(count):
        p_k, m_k = make_system(int(sizes[k]), s, dist, seed * 7919 + k)
        pos[off[k]:off[k + 1]] = p_k
        mom[off[k]:off[k + 1]] = m_k
    return pos, mom, off


def make_system(n: int, s: int, dist: str, seed: int):
    """(positions (n,3), moments (n, T(s))) for a named distribution."""
    if dist == "uniform":
        pos = uniform_cube(n, seed)
    elif dist == "plummer":
        pos = plummer(n, seed)
    else:
        raise ValueError(dist)
    return pos, sources(n, seed, s)


def make_system_mixed(n: int, s_lo: int, s_hi: int, dist: str, seed: int):
    """(positions, moments (n, T(s_lo..s_hi))) with every order s_lo..s_hi per particle."""
    pos, _ = make_system(n, s_lo, dist, seed)
    return pos, sources_mixed(n, seed, s_lo, s_hi)
