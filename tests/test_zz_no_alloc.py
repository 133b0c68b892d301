"""sfmm_sort_keys_static: the allocation-free keys + sort entry point.

It exists for callers that must not allocate device memory (a plugin inside an
application whose memory pool owns the device, or a latency-critical pipeline
that cannot accept the synchronisation an allocation may cause).  Its scratch is
a static device array shared by all calls, so the GPU test below calls it twice
in a row and compares both results with the sorted keys and permutation the
solver itself produced (read back through sfmm_debug_copy), bit for bit.  The
file is named to run last.
"""
import ctypes

import numpy as np
import pytest

from paper_2210_07021_gb300 import sfmm, workloads


def test_rejects_sizes_above_its_static_scratch():
    L = sfmm.load()
    st = L.sfmm_sort_keys_static(None, sfmm.STATIC_SORT_MAX_N + 1, None, None, None)
    assert st == sfmm.SFMM_EINVAL
    assert "static scratch" in L.sfmm_last_error(None).decode()
    assert L.sfmm_sort_keys_static(None, -1, None, None, None) == sfmm.SFMM_EINVAL


@pytest.mark.gpu
@pytest.mark.parametrize("n", [1, sfmm.STATIC_SORT_MAX_N])
def test_matches_the_oracle_keys_and_a_stable_argsort(n):
    """At the smallest size and at the static scratch's limit (where its fixed
    layout must be exactly large enough), twice in a row: the keys are the
    oracle's order-29 nested keys sorted, the permutation a stable argsort."""
    torch = pytest.importorskip("torch")
    from oracle.healpix import key29
    rng = np.random.default_rng(18)
    src = workloads.clustered(rng, n, 64) if n > 1 else np.array([[0.6, 0.0, 0.8]])
    if n > 100:
        src[:50] = src[50:100]        # duplicate keys: equal keys keep their input order
    k = key29(src).astype(np.uint64)
    order = np.argsort(k, kind="stable")
    x = torch.as_tensor(src, device="cuda")
    for _ in range(2):
        keys, perm = sfmm.sort_keys_static(x)
        torch.cuda.synchronize()
        assert np.array_equal(keys.cpu().numpy().view(np.uint64), k[order])
        assert np.array_equal(perm.cpu().numpy().view(np.uint32), order.astype(np.uint32))


@pytest.mark.gpu
def test_matches_the_solver_sort_twice_in_a_row():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(17)
    n = 200_003                       # ragged: not a multiple of the 4096-key sort tile
    src = workloads.clustered(rng, n, 64)
    src[:50] = src[50:100]            # duplicate keys: the sort must keep input order
    q = np.ones(n)
    tgt = src[:1000]
    dev = lambda a: torch.as_tensor(a, device="cuda")
    plan = sfmm.Plan(p=8, leaf_size=64)
    plan.potential(dev(src), dev(q), dev(tgt))
    want_keys = plan.debug(sfmm.ARR_SRC_KEYS, np.uint64)
    want_perm = plan.debug(sfmm.ARR_SRC_PERM, np.uint32)
    x = dev(src)
    for _ in range(2):
        keys, perm = sfmm.sort_keys_static(x)
        torch.cuda.synchronize()
        assert np.array_equal(keys.cpu().numpy().view(np.uint64), want_keys)
        assert np.array_equal(perm.cpu().numpy().view(np.uint32), want_perm)
