"""The training-data augmentation of the graph network (its periodic form
of the paper's random rotations and flips): every symmetry operation of the
cubic box keeps all minimum-image distances and the energy, maps forces as
it maps displacements, and keeps positions in [0, L)."""
import numpy as np
import torch

from paper_1912_04232_b300 import learned as LP


def _dists(r, L):
    d = r[:, None, :3] - r[None, :, :3]
    d -= L * np.round(d / L)
    return np.sort(np.sqrt((d ** 2).sum(-1)).ravel())


def test_cubic_symmetry_copies():
    rng = np.random.Generator(np.random.PCG64(0))
    S, n, L = 3, 20, 7.5
    r = np.zeros((S, n, 4), np.float32)
    r[:, :, :3] = rng.uniform(0, L, (S, n, 3))
    r[:, :, 3] = 1.0
    F = np.zeros((S, n, 4), np.float32)
    F[:, :, :3] = rng.normal(size=(S, n, 3))
    ds = LP.Dataset(r=torch.from_numpy(r), F=torch.from_numpy(F), E=torch.arange(S, dtype=torch.float64),
                    T=np.arange(S, dtype=float), L=L, n=n)
    da = LP.augment_cubic(ds, 0, 2, 5, seed=1, keep=(2, 3))
    assert da.r.shape == (2 * 5 + 1, n, 4)
    ra, Fa = da.r.numpy(), da.F.numpy()
    assert np.all(ra[:, :, :3] >= 0) and np.all(ra[:, :, :3] < L)
    for k in range(10):
        s = k // 5
        np.testing.assert_allclose(_dists(ra[k], L), _dists(r[s], L), atol=2e-5)
        assert da.E[k].item() == float(s)
        # the same orthogonal map takes displacements and forces: F.d is kept
        d0 = r[s, 1, :3] - r[s, 0, :3]
        d0 -= L * np.round(d0 / L)
        d1 = ra[k, 1, :3] - ra[k, 0, :3]
        d1 -= L * np.round(d1 / L)
        assert abs(float(F[s, 0, :3] @ d0) - float(Fa[k, 0, :3] @ d1)) < 1e-4
        np.testing.assert_allclose(np.linalg.norm(Fa[k, :, :3], axis=1), np.linalg.norm(F[s, :, :3], axis=1),
                                   rtol=1e-6)
    np.testing.assert_array_equal(ra[10], r[2])
