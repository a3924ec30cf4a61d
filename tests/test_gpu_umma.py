"""Tensor-core building blocks of the FMM_3XTF32 M2L (tcgen05.mma kind::tf32,
32-byte-swizzled K-major tiles, accumulator in tensor memory), checked against
an FP64 product on the host.

Bounds: one TF32 product keeps 11 significant bits per operand, so hi.hi
alone is within ~2^-10 of the exact product (relative to sum |a||b|); the
3xTF32 form (hi.hi + hi.lo + lo.hi) carries ~22 bits per operand and
accumulates in FP32: within 2^-19 relative to sum |a||b| over K <= 32.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def reference(A, B, kbn):
    D = np.zeros((A.shape[0], B.shape[0]))
    for kb, nb in enumerate(kbn):
        sl = slice(8 * kb, 8 * kb + 8)
        D[:, :nb] += A[:, sl] @ B[:nb, sl].T
    scale = np.zeros_like(D)
    for kb, nb in enumerate(kbn):
        sl = slice(8 * kb, 8 * kb + 8)
        scale[:, :nb] += np.abs(A[:, sl]) @ np.abs(B[:nb, sl]).T
    return D, scale


@pytest.mark.parametrize("a_tmem", [False, True])
@pytest.mark.parametrize("kbn", [[16], [96, 64, 48, 32], [256, 256], [48, 16, 16]])
def test_umma_3xtf32(a_tmem, kbn):
    import torch
    from paper_2005_12351_gb300 import fmm
    rng = np.random.default_rng(len(kbn) * 1000 + kbn[0] + a_tmem)
    K, N = 8 * len(kbn), kbn[0]
    A = rng.standard_normal((128, K)) * np.exp(rng.uniform(-3, 3, (128, 1)))
    B = rng.standard_normal((N, K)) * np.exp(rng.uniform(-3, 3, (1, K)))
    A32, B32 = A.astype(np.float32), B.astype(np.float32)
    D = fmm.check_umma(torch.from_numpy(A32).cuda(), torch.from_numpy(B32).cuda(), kbn,
                       a_tmem=a_tmem, passes=3).cpu().numpy().astype(np.float64)
    ref, scale = reference(A32.astype(np.float64), B32.astype(np.float64), kbn)
    err = np.abs(D - ref) / np.maximum(scale, 1e-300)
    assert err.max() < 2.0 ** -19, err.max()
    D1 = fmm.check_umma(torch.from_numpy(A32).cuda(), torch.from_numpy(B32).cuda(), kbn,
                        a_tmem=a_tmem, passes=1).cpu().numpy().astype(np.float64)
    err1 = np.abs(D1 - ref) / np.maximum(scale, 1e-300)
    assert err1.max() < 2.0 ** -9, err1.max()
    assert err1.max() > 4 * err.max()      # the lo terms matter


def test_umma_rejects_bad_shapes():
    import torch
    from paper_2005_12351_gb300 import fmm
    A = torch.zeros((128, 8), dtype=torch.float32, device="cuda")
    B = torch.zeros((24, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(fmm.FMMError):
        fmm.check_umma(A, B, [24])
