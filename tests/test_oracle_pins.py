"""Pins for the FP64 oracle: values fixed by the paper, closed forms,
invariants, brute force and finite differences -- never the oracle's own
formula retyped.  CPU only.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()[:2]
            vals[k] = float(v)
    return vals


def _rand_fluid(N, L, seed, dim=3, rmin=0.0):
    """Random positions with a minimum separation (rejection), float32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = []
    while len(pts) < N:
        p = rng.uniform(0, L, size=dim)
        ok = True
        for q in pts:
            d = p - q
            d -= L * np.round(d / L)
            if np.dot(d, d) < rmin * rmin:
                ok = False
                break
        if ok:
            pts.append(p)
    r = np.zeros((N, 4), np.float32)
    r[:, :dim] = np.array(pts, dtype=np.float32)
    return r


# ---------------------------------------------------------------------------
# Periodic space and neighbor sets (Sec. 3.2.1, 3.2.3)
# ---------------------------------------------------------------------------
def test_min_image_hand_case():
    # two particles 0.1 inside opposite faces of a box of edge 10: separation 0.2
    L = 10.0
    r = np.array([[0.1, 5.0, 5.0, 0], [9.9, 5.0, 5.0, 0]], np.float32)
    cnt, nb = O.neighbor_list(r, L, 0.25, fp32_decision=False, use_cells=False)
    assert list(cnt) == [1, 1]
    cnt, nb = O.neighbor_list(r, L, 0.19, fp32_decision=False, use_cells=False)
    assert list(cnt) == [0, 0]


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("ncell", [1, 2, 3, 4])
def test_cell_list_equals_brute_force_tiny_boxes(dim, ncell):
    r_list = 1.3
    L = ncell * r_list * 1.05 if ncell > 1 else 2.7  # 1 cell: box < 2 r_list
    N = 48 if dim == 3 else 24
    for seed in range(3):
        r = _rand_fluid(N, L, seed, dim=dim)
        for mode in (True, False):
            c1, n1 = O.neighbor_list(r, L, r_list, dim=dim, fp32_decision=mode, use_cells=True, cap=N)
            c0, n0 = O.neighbor_list(r, L, r_list, dim=dim, fp32_decision=mode, use_cells=False, cap=N)
            np.testing.assert_array_equal(c1, c0)
            np.testing.assert_array_equal(n1, n0)


def test_neighbor_set_is_symmetric_and_sorted():
    c = W.lj_small()
    cnt, nb = O.neighbor_list(c.r, c.L, 2.8)
    N = c.N
    pairs = set()
    for i in range(N):
        row = nb[i, : cnt[i]]
        assert np.all(np.diff(row) > 0)
        assert np.all(nb[i, cnt[i]:] == N)
        pairs.update((i, int(j)) for j in row)
    assert all((j, i) in pairs for (i, j) in pairs)
    # mean count close to rho * 4/3 pi r_list^3
    assert abs(cnt.mean() - 0.84 * 4 / 3 * math.pi * 2.8 ** 3) < 3.0


def test_fp32_and_fp64_sets_agree_away_from_cutoff():
    c = W.lj_small()
    r_list = 2.8
    c32, n32 = O.neighbor_list(c.r, c.L, r_list, fp32_decision=True)
    c64, n64 = O.neighbor_list(c.r, c.L, r_list, fp32_decision=False)
    x = c.r[:, :3].astype(np.float64)
    diff = 0
    for i in range(c.N):
        a = set(n32[i, : c32[i]].tolist())
        b = set(n64[i, : c64[i]].tolist())
        for j in a ^ b:
            d = x[i] - x[j]
            d -= c.L * np.round(d / c.L)
            assert abs(np.linalg.norm(d) - r_list) < 1e-5
            diff += 1
    assert diff < 10


# ---------------------------------------------------------------------------
# Lennard-Jones (Sec. 3.3.2, benchmark Sec. 3.1)
# ---------------------------------------------------------------------------
def test_lj_closed_forms():
    g = _golden("lj_reduced.txt")
    u, du = O.lj_pair(g["r_min"])
    assert abs(u - g["u_min"]) < 1e-14 and abs(du) < 1e-12
    u1, du1 = O.lj_pair(1.0)
    assert abs(u1) < 1e-15 and abs(-du1 - g["f_at_r1"]) < 1e-12
    uc, _ = O.lj_pair(2.5)
    assert abs(uc - g["u_shift_2p5"]) < 1e-13
    # curvature at the minimum by central differences of the derivative
    h = 1e-5
    k = (O.lj_pair(g["r_min"] + h)[1] - O.lj_pair(g["r_min"] - h)[1]) / (2 * h)
    assert abs(k - g["k_min"]) < 1e-5


def test_lj_two_and_three_particle_hand_cases():
    g = _golden("lj_reduced.txt")
    L = 20.0
    # dimer at the minimum: shifted energy, zero force
    r = np.array([[5, 5, 5, 0], [5 + g["r_min"], 5, 5, 0]], np.float32)
    U, F, e = O.lj(r, L, use_cells=False)
    rm = float(np.float32(5 + g["r_min"])) - 5.0
    u, du = O.lj_pair(rm)
    assert abs(U - (u - g["u_shift_2p5"])) < 1e-12
    # dimer at r = 1: |F| = 24 along the axis, repulsive
    r = np.array([[5, 5, 5, 0], [6, 5, 5, 0]], np.float32)
    U, F, e = O.lj(r, L, shifted=False, use_cells=False)
    assert abs(U) < 1e-14
    np.testing.assert_allclose(F[0], [-24, 0, 0], atol=1e-12)
    np.testing.assert_allclose(F[1], [24, 0, 0], atol=1e-12)
    np.testing.assert_allclose(e, [0, 0], atol=1e-14)
    # equilateral triangle of side 1: U = 0, each force has magnitude 24*sqrt(3)
    r = np.array([[5, 5, 5, 0], [6, 5, 5, 0], [5.5, 5 + math.sqrt(3) / 2, 5, 0]], np.float64)
    U, F, e = O.lj(r, L, shifted=False, use_cells=False)
    assert abs(U) < 1e-6
    np.testing.assert_allclose(np.linalg.norm(F, axis=1), 24 * math.sqrt(3), rtol=1e-6)
    # outside the cutoff nothing interacts
    r = np.array([[5, 5, 5, 0], [7.6, 5, 5, 0]], np.float32)
    U, F, e = O.lj(r, L, use_cells=False)
    assert U == 0.0 and np.all(F == 0)


def test_lj_perfect_fcc_has_zero_force():
    # box and sites exactly representable: 4 x 4 x 4 FCC cells of edge 1.75
    r = W.fcc_lattice(4, 7.0)
    U, F, e = O.lj(r, 7.0, r_cut=2.5)
    assert np.abs(F).max() < 1e-11
    assert np.ptp(e) < 1e-12


def _fd_check(energy, r, h=1e-6):
    U, F = energy(r)
    rng = np.random.Generator(np.random.PCG64(5))
    idx = rng.choice(r.shape[0], size=min(8, r.shape[0]), replace=False)
    for i in idx:
        for k in range(3):
            rp = r.copy(); rp[i, k] += h
            rm = r.copy(); rm[i, k] -= h
            fd = -(energy(rp)[0] - energy(rm)[0]) / (2 * h)
            assert abs(fd - F[i, k]) <= 1e-7 * max(1.0, abs(F[i, k])), (i, k, fd, F[i, k])


def test_lj_forces_are_minus_gradient():
    r = _rand_fluid(64, 5.0, 1, rmin=0.9).astype(np.float64)

    def en(x):
        U, F, e = O.lj(x, 5.0, r_cut=2.4, shifted=True, use_cells=False)
        return U, F
    # keep every pair away from the cutoff so a displacement of h cannot cross it
    x = r[:, :3]
    d = x[:, None, :] - x[None, :, :]
    d -= 5.0 * np.round(d / 5.0)
    dist = np.sqrt((d ** 2).sum(-1))
    assert np.abs(dist - 2.4).min() > 1e-4
    _fd_check(en, r)


def test_lj_net_force_zero_and_energy_sum():
    c = W.lj_small()
    U, F, e = O.lj(c.r, c.L)
    scale = np.abs(F).sum()
    assert np.abs(F.sum(0)).max() <= 1e-10 * scale
    assert abs(e.sum() - U) < 1e-9 * abs(U)


def test_lj_cells_equal_brute_force():
    c = W.lj_small()
    U1, F1, e1 = O.lj(c.r, c.L, use_cells=True)
    U0, F0, e0 = O.lj(c.r, c.L, use_cells=False)
    assert abs(U1 - U0) < 1e-9 * abs(U0)
    np.testing.assert_allclose(F1, F0, rtol=0, atol=1e-10)


# ---------------------------------------------------------------------------
# Soft spheres (Sec. 3.3.2, App. A)
# ---------------------------------------------------------------------------
def test_soft_sphere_two_disk_closed_form_and_no_overlap():
    L = 10.0
    for r12 in (0.3, 0.75, 0.999):
        r = np.array([[2, 2, 0, 0], [2 + r12, 2, 0, 0]], np.float64)
        U, F, e = O.soft(r, [1.0, 1.0], L, dim=2)
        assert abs(U - 0.5 * (1 - r12) ** 2) < 1e-14
        np.testing.assert_allclose(F[1, :2], [(1 - r12), 0.0], atol=1e-14)
    # mixed diameters: sigma = (1.4 + 1)/2 = 1.2
    r = np.array([[2, 2, 0, 0], [2, 3.0, 0, 0]], np.float64)
    U, F, e = O.soft(r, [1.4, 1.0], L, dim=2)
    assert abs(U - 0.5 * (1 - 1.0 / 1.2) ** 2) < 1e-14
    r = np.array([[2, 2, 0, 0], [2, 3.3, 0, 0]], np.float64)
    U, F, e = O.soft(r, [1.4, 1.0], L, dim=2)
    assert U == 0.0 and np.all(F == 0.0)


def test_soft_sphere_scale_invariance_and_fd():
    p = W.packing_2d(N=64, D=1.4, seed=3)
    L = W.packing_box(64, 1.4, 0.9)
    r = np.zeros((64, 3)); r[:, :2] = p.s0 * L
    U, F, e = O.soft(r, p.diam, L, dim=2)
    s = 1.7
    U2, F2, _ = O.soft(r * s, p.diam * s, L * s, dim=2)
    assert abs(U2 - U) < 1e-12 * abs(U)
    np.testing.assert_allclose(F2 * s, F, rtol=1e-10, atol=1e-12)

    def en(x):
        U, F, _ = O.soft(x, p.diam, L, dim=2)
        F[:, 2] = 0.0
        return U, F
    _fd_check(en, r)


# ---------------------------------------------------------------------------
# Stillinger-Weber (Sec. 3.3.2)
# ---------------------------------------------------------------------------
def test_sw_diamond_cohesive_energy_and_zero_force():
    g = _golden("sw_silicon.txt")
    v, d = O.sw_phi2(2 ** (1 / 6) * g["sigma_A"])
    assert abs(v + g["eps_eV"]) < 1e-6 and abs(d) < 1e-6
    s = W.sw_silicon(3, a=g["diamond_a_A"], T_K=0)
    U, F, e = O.sw(s.r, s.L)
    assert abs(U / s.N - g["cohesive_energy_eV_per_atom"]) < 1e-4
    assert np.abs(F).max() < 1e-3


def test_sw_three_body_vanishes_at_tetrahedral_angle():
    # centre atom with two legs at the tetrahedral angle, both inside the cutoff,
    # legs themselves beyond the cutoff (3.84 A > a sigma): only 2-body energy
    L = 40.0
    b = 2.35163
    u = np.array([1, 1, 1]) / math.sqrt(3) * b
    w = np.array([1, -1, -1]) / math.sqrt(3) * b
    c = np.array([20.0, 20.0, 20.0])
    r = np.stack([c, c + u, c + w]).astype(np.float64)
    U, F, e = O.sw(r, L)
    p2, _ = O.sw_phi2(b)
    assert abs(U - 2 * p2) < 1e-10
    # bend the angle: three-body energy appears and is positive
    w2 = np.array([1, -1, 0.2]) / np.linalg.norm([1, -1, 0.2]) * b
    r2 = np.stack([c, c + u, c + w2])
    U2, _, _ = O.sw(r2, L)
    assert U2 > 2 * p2 + 1e-3


def test_sw_forces_fd_net_force_and_rotation_invariance():
    s = W.sw_silicon(2, T_K=0, jitter=0.15, seed=2)
    r = s.r.astype(np.float64)

    def en(x):
        U, F, _ = O.sw(x, s.L)
        return U, F
    _fd_check(en, r, h=1e-6)
    U, F, e = O.sw(r, s.L)
    assert np.abs(F.sum(0)).max() < 1e-10 * np.abs(F).sum()
    # a free cluster in a large box: rotation leaves U invariant and rotates F
    cl = r[:, :3][:20] + 30.0
    rng = np.random.Generator(np.random.PCG64(0))
    A = np.linalg.qr(rng.normal(size=(3, 3)))[0]
    c0 = cl.mean(0)
    cl2 = (cl - c0) @ A.T + c0
    U1, F1, _ = O.sw(cl, 100.0)
    U2, F2, _ = O.sw(cl2, 100.0)
    assert abs(U1 - U2) < 1e-10 * abs(U1)
    np.testing.assert_allclose(F1 @ A.T, F2, atol=1e-9)


# ---------------------------------------------------------------------------
# Dynamics (Sec. 3.3.1)
# ---------------------------------------------------------------------------
def test_nve_time_reversibility():
    c = W.lj_fluid("sc", 6, seed=4)
    r1, v1, PE, KE = O.nve(c.r, c.v, c.L, "lj", dt=0.005, nsteps=100)
    r2, v2, _, _ = O.nve(r1, -v1, c.L, "lj", dt=0.005, nsteps=100)
    d = r2 - c.r[:, :3].astype(np.float64)
    d -= c.L * np.round(d / c.L)
    assert np.abs(d).max() < 1e-9
    np.testing.assert_allclose(-v2, c.v[:, :3], atol=1e-9)


def test_nve_energy_error_is_second_order_and_bounded():
    # velocity Verlet is second order: the energy fluctuation scales as dt^2.
    # On the N=4,096 LJ start (jittered simple-cubic lattice, far from
    # equilibrium) the largest excursion at dt = 0.005 stays below 1.5e-3 per
    # particle; halving dt divides it by four.
    c = W.lj_small()
    dev = []
    for dt, n in ((0.005, 100), (0.0025, 200)):
        _, _, PE, KE = O.nve(c.r, c.v, c.L, "lj", dt=dt, nsteps=n)
        E = PE + KE
        dev.append(np.abs(E - E[0]).max() / c.N)
    assert dev[0] <= 1.5e-3
    assert 3.5 <= dev[0] / dev[1] <= 4.5


def test_nve_lj_dimer_small_oscillation_period():
    g = _golden("lj_reduced.txt")
    amp = 1e-3
    L = 20.0
    r = np.array([[5, 5, 5, 0], [5 + g["r_min"] + amp, 5, 5, 0]], np.float64)
    v = np.zeros((2, 4))
    dt = 1e-4
    period = 2 * math.pi * math.sqrt(0.5 / g["k_min"])
    n = int(round(1.5 * period / dt))
    # record separation over time by stepping in chunks of 1
    x, vv = r.copy(), v.copy()
    seps = []
    for _ in range(n):
        x, vv, _, _ = O.nve(x, vv, L, "lj", dt=dt, nsteps=1, shifted=False, r_cut=5.0)
        seps.append(x[1, 0] - x[0, 0])
    seps = np.array(seps)
    # time of the first return to maximum separation = one period
    t = np.arange(1, n + 1) * dt
    k = np.argmax(seps[int(0.5 * period / dt):]) + int(0.5 * period / dt)
    assert abs(t[k] - period) < 3 * dt + 2e-3 * period


def test_gd_dimer_closed_form_and_monotone():
    # two overlapping unit disks: (sigma - r_{t+1}) = (1 - 2 eta k)(sigma - r_t), k = eps/sigma^2
    eta = 0.05
    r = np.array([[2, 2, 0, 0], [2.6, 2, 0, 0]], np.float64)
    x, E = O.gd(r, 10.0, "soft", eta=eta, nsteps=5, dim=2, diam=[1.0, 1.0])
    gap = 1.0 - 0.6
    for _ in range(5):
        gap *= (1 - 2 * eta)
    assert abs((x[1, 0] - x[0, 0]) - (1.0 - gap)) < 1e-14
    p = W.packing_2d(N=128, D=1.4, seed=0)
    L = W.packing_box(128, 1.4, 0.9)
    r = np.zeros((128, 3)); r[:, :2] = p.s0 * L
    _, E = O.gd(r, L, "soft", eta=eta, nsteps=200, dim=2, diam=p.diam)
    assert np.all(np.diff(E) <= 1e-12)


# ---------------------------------------------------------------------------
# Differentiation through minimisation (Sec. 4.2, App. A)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N,D,T,seed", [(32, 1.3, 20, 0), (64, 1.1, 60, 1), (64, 1.6, 40, 2)])
def test_adjoint_matches_finite_differences(N, D, T, seed):
    p = W.packing_2d(N=N, D=D, seed=seed)
    E, g, _ = O.gd_adjoint(p.s0, D, T=T)
    h = 1e-5 * D
    fd = (O.gd_final_energy(p.s0, D + h, T=T) - O.gd_final_energy(p.s0, D - h, T=T)) / (2 * h)
    assert abs(g - fd) <= 1e-6 * max(1.0, abs(fd)), (g, fd)


def test_adjoint_T1_dimer_forward_mode_closed_form():
    # N=2 (one disk of diameter D, one of diameter 1), low packing fraction so
    # the pair overlaps through one image only; one GD step; forward-mode by hand.
    phi, eps, eta, D, delta = 0.1, 1.0, 0.05, 1.3, 0.22
    s0 = np.array([[0.3, 0.5], [0.3 + delta, 0.5]])
    E, g, _ = O.gd_adjoint(s0, D, phi=phi, eta=eta, T=1)
    L = math.sqrt(math.pi * (1 + D * D) / 4 / phi)
    Lp = math.pi * D / (4 * phi * L)
    sg, sgp = (D + 1) / 2, 0.5
    r0, r0p = L * delta, Lp * delta
    x0 = 1 - r0 / sg
    x0p = -(r0p * sg - r0 * sgp) / sg ** 2
    r1 = r0 + 2 * eta * eps * x0 / sg
    r1p = r0p + 2 * eta * eps * (x0p * sg - x0 * sgp) / sg ** 2
    x1 = 1 - r1 / sg
    x1p = -(r1p * sg - r1 * sgp) / sg ** 2
    assert r1 < sg and r0 < L / 2
    assert abs(E - 0.5 * eps * x1 ** 2) < 1e-14
    assert abs(g - eps * x1 * x1p) < 1e-13


# ---------------------------------------------------------------------------
# Counter-based noise and Langevin (Sec. 3.3.1)
# ---------------------------------------------------------------------------
def test_philox_known_answers():
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_normals_moments():
    z = np.array([O.normal3(i, 7, 0, 12345) for i in range(20000)])
    assert abs(z.mean()) < 0.02
    assert abs(z.var() - 1.0) < 0.03
    assert abs((z ** 4).mean() - 3.0) < 0.15


def test_langevin_free_particles_equipartition():
    # non-interacting particles (LJ with eps = 0): the O-steps alone drive
    # the velocity distribution to kT/m per component
    N = 512
    L = 40.0
    r = W.uniform_box_positions(N, L, 3, np.random.Generator(np.random.PCG64(1)))
    r4 = np.zeros((N, 4), np.float32); r4[:, :3] = r
    v = np.zeros((N, 4))
    kT, m = 0.7, 2.0
    x, vv, PE, KE = O.langevin(r4, v, L, "lj", mass=m, dt=1.0, gamma=0.05, kT=kT, seed=9, nsteps=400,
                               eps=0.0)
    assert np.all(PE == 0.0)
    ke_tail = KE[200:].mean() / N
    assert abs(ke_tail - 1.5 * kT) < 0.04 * 1.5 * kT
