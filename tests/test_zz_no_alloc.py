"""The allocation-free neighbor-list build.

Callers that can hand the library only their own input and output buffers
(no workspace, no cudaMalloc) use md_neighbor_list_build_noalloc, which
takes its scratch from a fixed pool inside the library.  This checks,
through the C ABI, that two calls in a row (different systems, so the
second call starts from the first one's leftovers in the pool) give exactly
the rows and counts of the ordinary md_neighbor_list_build.

Kept in its own file, named to be collected last.
"""
import numpy as np
import pytest

import workloads as W
from gpu_helpers import dev, status_word, to_dev

pytestmark = pytest.mark.gpu


def _reference_rows(P, s, r, N, cap):
    import torch
    nl = P.NeighborList(s, N, 2.5, 0.3, cap)
    st = status_word()
    nl.build(r, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    return nl.cnt.cpu().numpy(), nl.nbr.cpu().numpy()


def test_noalloc_build_matches_workspace_build_twice():
    import torch
    import paper_1912_04232_b300 as P
    cases = [W.lj_small(seed=0), W.lj_fluid("sc", 12, seed=5)]   # N = 4096, then N = 1728
    cap = 128
    for c in cases:
        s = P.md_space_periodic(3, [c.L] * 3)
        r = to_dev(c.r, torch.float32)
        nbr = torch.full((c.N, cap), -7, dtype=torch.int32, device=dev())
        cnt = torch.full((c.N,), -7, dtype=torch.int32, device=dev())
        st = status_word()
        P.md_neighbor_list_build_noalloc(s, r, c.N, 2.5, 0.3, cap, nbr, cnt, st)
        torch.cuda.synchronize()
        assert P.md_status_poll(st) == 0
        cnt_ref, nbr_ref = _reference_rows(P, s, r, c.N, cap)
        np.testing.assert_array_equal(cnt.cpu().numpy(), cnt_ref)
        np.testing.assert_array_equal(nbr.cpu().numpy(), nbr_ref)


def test_noalloc_build_rejects_sizes_beyond_the_pool():
    import torch
    import paper_1912_04232_b300 as P
    N = P.md_noalloc_scratch_bytes() // 16          # positions alone would fill the pool
    s = P.md_space_periodic(3, [200.0] * 3)
    # full-size buffers, so nothing could be read out of bounds even if the
    # size check were missing
    r = torch.zeros((N, 4), dtype=torch.float32, device=dev())
    nbr = torch.zeros((N, 8), dtype=torch.int32, device=dev())
    cnt = torch.zeros(N, dtype=torch.int32, device=dev())
    with pytest.raises(P.MDError) as e:
        P.md_neighbor_list_build_noalloc(s, r, N, 2.5, 0.3, 8, nbr, cnt, None)
    assert e.value.code == P.MD_ERR_INVALID


def test_noalloc_build_at_the_pool_boundary():
    # LJ at density 0.84 in a fixed box: the largest N whose scratch fits the
    # pool gives the workspace build's rows bit for bit; one particle more is
    # refused before anything runs
    import torch
    import paper_1912_04232_b300 as P
    from test_host_noalloc import noalloc_limit
    c = W.lj_fluid("fcc", 25, seed=3)          # N = 62,500, L = 42.06
    s = P.md_space_periodic(3, [c.L] * 3)
    n = noalloc_limit(P, s, c.N)
    cap = 128
    for N, ok in ((n, True), (n + 1, False)):
        r = to_dev(c.r[:N], torch.float32)
        nbr = torch.full((N, cap), -7, dtype=torch.int32, device=dev())
        cnt = torch.full((N,), -7, dtype=torch.int32, device=dev())
        st = status_word()
        if not ok:
            with pytest.raises(P.MDError) as e:
                P.md_neighbor_list_build_noalloc(s, r, N, 2.5, 0.3, cap, nbr, cnt, st)
            assert e.value.code == P.MD_ERR_INVALID
            assert (cnt == -7).all().item()
            continue
        P.md_neighbor_list_build_noalloc(s, r, N, 2.5, 0.3, cap, nbr, cnt, st)
        torch.cuda.synchronize()
        assert P.md_status_poll(st) == 0
        cnt_ref, nbr_ref = _reference_rows(P, s, r, N, cap)
        np.testing.assert_array_equal(cnt.cpu().numpy(), cnt_ref)
        np.testing.assert_array_equal(nbr.cpu().numpy(), nbr_ref)
