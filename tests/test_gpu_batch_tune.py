"""GPU: the batched engine's tuning knobs change nothing but the time --
per-class cell multipliers and threads per particle give the same rows (as
sets), forces and energies to rounding, and the same trajectories to
rounding; per-class launches with the default threads per particle give the
default's bits; a tuned configuration matches the FP64 oracle; the
autotuner returns a configuration no slower than the default and caches
it."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import dev, force_error, status_word, to_dev

pytestmark = pytest.mark.gpu

CAP = 128


@pytest.fixture(scope="module")
def P():
    import paper_1912_04232_b300 as P
    return P


def _desc(P, sp):
    d = P.md_replica_desc()
    d.N, d.L = sp.N, sp.L
    if sp.kind == "lj":
        pot = P.lj_pot()
        d.kind, d.eps, d.sigma, d.r_cut, d.e_shift = P.MD_LJ, pot.eps, pot.sigma, pot.r_cut, pot.e_shift
    else:
        d.kind, d.eps, d.alpha, d.r_cut = P.MD_SOFT_SPHERE, 1.0, 2.0, 1.4
    d.skin, d.dt, d.mass = 0.3, sp.dt, 1.0
    return d


def _state(specs):
    import torch
    st = [W.replica_initial(sp) for sp in specs]
    return (to_dev(np.concatenate([s[0] for s in st]), torch.float32),
            to_dev(np.concatenate([s[1] for s in st]), torch.float32))


def _rows(b):
    cnt = b.cnt.cpu().numpy()
    nbr = b.nbr.cpu().numpy()
    return cnt, [np.sort(nbr[i, :cnt[i]]) for i in range(len(cnt))]


def test_tuned_knobs_keep_rows_forces_and_trajectories(P):
    import torch
    import paper_1912_04232_b300.batch_tune as T
    specs = W.replica_plan(R=64, n_max=4096, seed=3)
    descs = [_desc(P, sp) for sp in specs]
    assert {T.size_class(d.N) for d in descs} == {0, 1, 2}
    r0, v0 = _state(specs)
    st = status_word()
    out = {}
    for name, mult, tpp in (("default", [1.0, 1.0, 1.0], None), ("tuned", [2.0, 1.5, 2.0], [16, 8, 4])):
        b = P.Batch(T.with_mults(descs, mult), cap=CAP)
        if tpp is not None:
            P.md_batch_set_class_tpp(b.plan, T.tpp_per_replica(descs, tpp))
        r, v = r0.clone(), v0.clone()
        f = torch.zeros_like(r)
        P.md_batch_build(b.plan, r, st)
        P.md_batch_forces(b.plan, r, f, st)
        torch.cuda.synchronize()
        out[name] = dict(b=b, ncell=int(b.plan.ncell_total), rows=_rows(b), f=f.cpu().numpy())
    assert P.md_status_poll(st) == 0
    assert out["tuned"]["ncell"] < out["default"]["ncell"]   # larger cells really used
    c0, rows0 = out["default"]["rows"]
    c1, rows1 = out["tuned"]["rows"]
    np.testing.assert_array_equal(c0, c1)
    for a, b in zip(rows0, rows1):
        np.testing.assert_array_equal(a, b)
    f0, f1 = out["default"]["f"], out["tuned"]["f"]
    scale = np.abs(f0[:, :3]).max()
    assert np.abs(f1[:, :3] - f0[:, :3]).max() <= 1e-5 * scale
    # 20 NVE steps of the LJ replicas (soft spheres start overlapping)
    lj = [sp for sp in specs if sp.kind == "lj"]
    dl = [_desc(P, sp) for sp in lj]
    r0, v0 = _state(lj)
    res = {}
    for name, mult, tpp in (("default", [1.0, 1.0, 1.0], None), ("tuned", [2.0, 1.5, 2.0], [16, 8, 4])):
        b = P.Batch(T.with_mults(dl, mult), cap=CAP)
        if tpp is not None:
            P.md_batch_set_class_tpp(b.plan, T.tpp_per_replica(dl, tpp))
        r, v = r0.clone(), v0.clone()
        f = torch.zeros_like(r)
        PE = torch.zeros((len(lj), 20), dtype=torch.float64, device=dev())
        KE = torch.zeros_like(PE)
        P.md_batch_build(b.plan, r, st)
        P.md_batch_forces(b.plan, r, f, st)
        P.md_batch_run_nve(b.plan, r, v, f, 20, PE, KE, True, st)
        torch.cuda.synchronize()
        res[name] = (r.cpu().numpy(), PE.cpu().numpy(), KE.cpu().numpy())
    assert P.md_status_poll(st) == 0
    (ra, pa, ka), (rb, pb, kb) = res["default"], res["tuned"]
    L = np.repeat([sp.L for sp in lj], [sp.N for sp in lj])[:, None]
    d = rb[:, :3] - ra[:, :3]
    d -= L * np.round(d / L)
    assert np.abs(d).max() < 1e-4
    np.testing.assert_allclose(pb, pa, rtol=1e-5, atol=1e-6 * np.abs(pa).max())
    np.testing.assert_allclose(kb, ka, rtol=1e-5)


def test_class_tpp_rejects_other_values(P):
    specs = W.replica_plan(R=8, n_max=1024, seed=4)
    b = P.Batch([_desc(P, sp) for sp in specs], cap=CAP)
    with pytest.raises(P.MDError) as e:
        P.md_batch_set_class_tpp(b.plan, [4, 8, 16, 32, 4, 4, 4, 4])
    assert e.value.code == P.MD_ERR_INVALID
    P.md_batch_set_class_tpp(b.plan, [4, 8, 16, 16, 4, 4, 8, 4])
    P.md_batch_set_class_tpp(b.plan, None)


def test_autotuner_picks_and_caches(P, tmp_path):
    import paper_1912_04232_b300.batch_tune as T
    specs = [sp for sp in W.replica_plan(R=96, n_max=8192, seed=5) if sp.kind == "lj"]
    descs = [_desc(P, sp) for sp in specs]
    r0, v0 = _state(specs)
    path = str(tmp_path / "tune.json")
    res = T.tune(descs, r0, v0, probe=10, cache_path=path)
    assert not res["cached"]
    assert res["ms_tuned"] <= res["ms_default"]
    assert all(m in T.MULTS for m in res["cell_mult"]) and all(t in T.TPPS for t in res["tpp"])
    again = T.tune(descs, r0, v0, probe=10, cache_path=path)
    assert again["cached"] and again["cell_mult"] == res["cell_mult"] and again["tpp"] == res["tpp"]


def _run(P, descs, r0, v0, mult, tpp, steps):
    import torch
    import paper_1912_04232_b300.batch_tune as T
    b = P.Batch(T.with_mults(descs, mult), cap=CAP)
    if tpp is not None:
        P.md_batch_set_class_tpp(b.plan, T.tpp_per_replica(descs, tpp))
    r, v = r0.clone(), v0.clone()
    f = torch.zeros_like(r)
    st = status_word()
    P.md_batch_build(b.plan, r, st)
    P.md_batch_forces(b.plan, r, f, st)
    f0 = f.cpu().numpy()
    if steps:
        P.md_batch_run_nve(b.plan, r, v, f, steps, None, None, True, st)
    torch.cuda.synchronize()
    assert P.md_status_poll(st) == 0
    return f0, r.cpu().numpy(), v.cpu().numpy()


def test_class_launches_with_default_threads_are_bitwise_default(P):
    # the per-class force launches (grouped particle list) with 4 threads
    # per particle everywhere: the same arithmetic per particle as the one
    # launch, so the same bits after 20 steps
    specs = [sp for sp in W.replica_plan(R=64, n_max=4096, seed=6) if sp.kind == "lj"]
    descs = [_desc(P, sp) for sp in specs]
    r0, v0 = _state(specs)
    a = _run(P, descs, r0, v0, [1.0, 1.0, 1.0], None, 20)
    b = _run(P, descs, r0, v0, [1.0, 1.0, 1.0], [4, 4, 4], 20)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_tuned_configuration_matches_oracle(P):
    # larger cells and other threads per particle on every class: forces of
    # sampled replicas after the build, and 20-step trajectories of two LJ
    # replicas, against the FP64 oracle
    import paper_1912_04232_b300.batch_tune as T
    specs = [sp for sp in W.replica_plan(R=64, n_max=4096, seed=7) if sp.kind == "lj"]
    descs = [_desc(P, sp) for sp in specs]
    states = [W.replica_initial(sp) for sp in specs]
    import torch
    r0 = to_dev(np.concatenate([s[0] for s in states]), torch.float32)
    v0 = to_dev(np.concatenate([s[1] for s in states]), torch.float32)
    f0, rg, vg = _run(P, descs, r0, v0, [2.0, 1.5, 2.0], [16, 8, 4], 20)
    offs = np.concatenate([[0], np.cumsum([sp.N for sp in specs])])
    order = sorted(range(len(specs)), key=lambda k: specs[k].N)
    for k in (order[0], order[len(order) // 2], order[-1]):
        sp, (r, v) = specs[k], states[k]
        a, z = offs[k], offs[k + 1]
        U, F, e = O.lj(r, sp.L)
        assert force_error(f0[a:z], F) <= 1e-4, (k, sp.N)
        ro, vo, _, _ = O.nve(r, v, sp.L, "lj", dt=sp.dt, nsteps=20)
        d = rg[a:z, :3] - ro
        d -= sp.L * np.round(d / sp.L)
        assert np.abs(d).max() < 2e-4, (k, sp.N)
        assert np.abs(vg[a:z, :3] - vo).max() < 2e-3, (k, sp.N)
