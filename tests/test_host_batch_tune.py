"""Host logic of the batched-replica autotuner: size classes, the replica
key, and the coordinate descent (with a synthetic cost whose optimum is
known).  No GPU."""
import paper_1912_04232_b300.batch_tune as T
import paper_1912_04232_b300 as P


def test_size_classes_and_key():
    assert [T.size_class(n) for n in (64, 511, 512, 2047, 2048, 8192)] == [0, 0, 1, 1, 2, 2]
    d = P.md_replica_desc()
    d.N, d.L, d.kind, d.r_cut, d.skin = 100, 6.0, P.MD_LJ, 2.5, 0.3
    e = P.md_replica_desc.from_buffer_copy(d)
    assert T.replica_key([d]) == T.replica_key([e])
    e.N = 101
    assert T.replica_key([d]) != T.replica_key([e])
    m = T.with_mults([d, e], [2.0, 1.5, 1.0])
    assert [x.cell_mult for x in m] == [2.0, 2.0] and d.cell_mult == 0.0
    assert T.tpp_per_replica([d], [16, 8, 4]) == [16]


def test_coordinate_descent_finds_separable_optimum():
    opt_m, opt_t = [2.0, 1.0, 1.5], [16, 4, 8]
    calls = []

    def cost(mult, tpp):
        calls.append((tuple(mult), tuple(tpp)))
        return sum((m - a) ** 2 for m, a in zip(mult, opt_m)) + sum(abs(t - b) / 100.0 for t, b in zip(tpp, opt_t)) + 1.0

    mult, tpp, t0, t = T.coordinate_descent(cost, [True, True, True])
    assert mult == opt_m and tpp == opt_t
    assert t == 1.0 and t0 > t
    # one start, two other multipliers and two other thread counts per class
    assert len(calls) == 1 + 3 * 2 + 3 * 2


def test_coordinate_descent_skips_empty_classes():
    mult, tpp, t0, t = T.coordinate_descent(lambda m, q: 1.0 + m[1] + q[1] / 100.0, [False, True, False])
    assert mult == [1.0, 1.0, 1.0] and tpp == [4, 4, 4] and t0 == t
