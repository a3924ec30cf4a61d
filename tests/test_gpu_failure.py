"""Failure paths that run without faulting the GPU.

* The radix sort's bounded look-back wait: with FMM_SORT_POLLS=0 every look-back
  of a sort tile gives up at once, so every tile after the first recounts the
  digits before it from the input.  The call must report FMM_ETIMEOUT and still
  return the exact Morton order.
* Device allocation failure: FMM_FAIL_ALLOC=k (read when a handle is created)
  makes that handle's k-th device allocation fail as cudaMalloc would.  Every
  allocation of create + set_sources + evaluate is failed once in turn; each
  failing call returns FMM_ENOMEM, the handle then refuses to evaluate until
  set_sources succeeds again, and from there on gives the same bits as a fresh
  handle.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2005_12351_gb300 import synth

pytestmark = pytest.mark.gpu

FMM_ENOMEM, FMM_ETIMEOUT, FMM_ESTATE = -2, -5, -7


def _morton_abi(P, n):
    """fmm_morton_order through the C ABI: (status, keys, perm)."""
    import torch
    from paper_2005_12351_gb300 import fmm
    keys = torch.empty(n, dtype=torch.int64, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    st = fmm.lib().fmm_morton_order(C.c_void_p(torch.cuda.current_stream().cuda_stream),
                                    C.c_void_p(P.data_ptr()), n, C.c_void_p(keys.data_ptr()),
                                    C.c_void_p(perm.data_ptr()))
    torch.cuda.synchronize()
    return st, keys.cpu().numpy().view(np.uint64), perm.cpu().numpy().astype(np.int64)


@pytest.mark.parametrize("n,dist", [(300_000, "plummer"), (1_000_000, "uniform")])
def test_sort_wait_gives_up_and_recounts_exactly(orc, monkeypatch, n, dist):
    from gpu_util import to_dev
    pos = synth.make_system(n, 0, dist, 611)[0]
    P = to_dev(pos)
    t = orc.Tree(pos, 1 << 30)
    monkeypatch.setenv("FMM_SORT_POLLS", "0")
    st, keys, perm = _morton_abi(P, n)
    assert st == FMM_ETIMEOUT
    assert np.array_equal(keys, t.keys) and np.array_equal(perm, t.perm)
    monkeypatch.delenv("FMM_SORT_POLLS")
    st, keys, perm = _morton_abi(P, n)
    assert st == 0
    assert np.array_equal(keys, t.keys) and np.array_equal(perm, t.perm)


def test_set_sources_reports_sort_wait_then_recovers(monkeypatch):
    from gpu_util import to_dev
    from paper_2005_12351_gb300 import fmm
    pos, S = synth.make_system(50_000, 1, "uniform", 612)
    P, Sd = to_dev(pos), to_dev(S)
    ref = fmm.create_tree(max_leaf=64)
    ref.set_sources(P, Sd, 1)
    _, E_ref = ref.evaluate(4, 0.5, False, True)
    tree = fmm.create_tree(max_leaf=64)
    monkeypatch.setenv("FMM_SORT_POLLS", "0")
    with pytest.raises(fmm.FMMError) as ei:
        tree.set_sources(P, Sd, 1)
    assert ei.value.status == FMM_ETIMEOUT
    monkeypatch.delenv("FMM_SORT_POLLS")
    tree.set_sources(P, Sd, 1)
    _, E = tree.evaluate(4, 0.5, False, True)
    assert np.array_equal(E.cpu().numpy(), E_ref.cpu().numpy())


@pytest.mark.parametrize("precision", ["fp64", "fp32", "3xtf32"])
def test_every_allocation_failure_leaves_a_usable_handle(monkeypatch, precision):
    import torch
    from gpu_util import to_dev
    from paper_2005_12351_gb300 import fmm
    pos, S = synth.make_system(6000, 2, "plummer", 613)
    P, Sd = to_dev(pos), to_dev(S)
    p, theta = 4, 0.5

    def run(tree):
        tree.set_sources(P, Sd, 2)
        phi, E = tree.evaluate(p, theta, True, True)
        torch.cuda.synchronize()
        return phi.cpu().numpy(), E.cpu().numpy()

    phi_ref, E_ref = run(fmm.create_tree(max_leaf=32, precision=precision))
    k, injected = 0, 0
    while True:
        k += 1
        assert k < 500, "allocation count did not end"
        monkeypatch.setenv("FMM_FAIL_ALLOC", str(k))
        try:
            tree = fmm.create_tree(max_leaf=32, precision=precision)
        except fmm.FMMError as e:         # the k-th allocation was one of create's own
            assert e.status == FMM_ENOMEM and k <= 2
            injected += 1
            continue
        finally:
            monkeypatch.delenv("FMM_FAIL_ALLOC")
        failed = False
        try:
            tree.set_sources(P, Sd, 2)
        except fmm.FMMError as e:
            assert e.status == FMM_ENOMEM, (k, e)
            failed = True
        if not failed:
            try:
                tree.evaluate(p, theta, True, True)
                torch.cuda.synchronize()
            except fmm.FMMError as e:
                assert e.status == FMM_ENOMEM, (k, e)
                failed = True
        if not failed:
            tree.destroy()
            break                              # k is past the last allocation
        injected += 1
        # the handle lost its tree: evaluate refuses until set_sources succeeds
        with pytest.raises(fmm.FMMError) as ei:
            tree.evaluate(p, theta, True, True)
        assert ei.value.status == FMM_ESTATE
        phi, E = run(tree)
        assert np.array_equal(phi, phi_ref) and np.array_equal(E, E_ref), k
        tree.destroy()
    assert injected == k - 1 and injected > 20, (k, injected)
