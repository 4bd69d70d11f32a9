"""Host-side sizing of the allocation-free neighbor-list build: the pool's
capacity follows from md_nbr_plan's workspace plus 16 bytes per particle of
build positions, about 68 bytes per particle plus 8 per cell.  No GPU."""
import workloads as W


def noalloc_need(P, space, N, r_cut=2.5, skin=0.3, cap=128):
    nb = P.md_nbr_plan(space, N, r_cut, skin, cap)
    return ((int(nb.ws_bytes) + 255) // 256) * 256 + 16 * N, nb


def noalloc_limit(P, space, n_hi):
    """Largest N <= n_hi whose scratch fits the pool (binary search; the
    need grows with N at a fixed box)."""
    pool = P.md_noalloc_scratch_bytes()
    lo, hi = 1, n_hi
    assert noalloc_need(P, space, lo)[0] <= pool < noalloc_need(P, space, hi)[0]
    while hi - lo > 1:
        m = (lo + hi) // 2
        if noalloc_need(P, space, m)[0] <= pool:
            lo = m
        else:
            hi = m
    return lo


def test_noalloc_capacity_lj_density_084():
    import paper_1912_04232_b300 as P
    c = W.lj_fluid("fcc", 25, seed=3)          # N = 62,500, L = 42.06
    s = P.md_space_periodic(3, [c.L] * 3)
    n = noalloc_limit(P, s, c.N)
    assert n == 61248
    need, nb = noalloc_need(P, s, n)
    assert list(nb.ncell) == [15, 15, 15]
    per_particle = (need - 8 * nb.ncell_total) / n
    assert 67.0 < per_particle < 69.0
    assert noalloc_need(P, s, n + 1)[0] > P.md_noalloc_scratch_bytes()
