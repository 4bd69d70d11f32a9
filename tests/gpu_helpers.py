"""Helpers for the GPU parity tests (CUDA path through the C ABI vs oracle)."""
from __future__ import annotations

import numpy as np


def dev():
    import torch
    assert torch.cuda.is_available(), "GPU test run without a CUDA device"
    return torch.device("cuda:0")


def to_dev(a, dtype=None):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(dev()).contiguous()


def status_word():
    import torch
    return torch.zeros(1, dtype=torch.int32, device=dev())


def force_error(F_gpu, F_ref):
    """Max over particles of |dF_i| / max(|F_i|, F_rms) (the F_rms floor
    keeps near-zero net forces from dominating)."""
    F_gpu = np.asarray(F_gpu, np.float64)[:, :3]
    F_ref = np.asarray(F_ref, np.float64)[:, :3]
    d = np.linalg.norm(F_gpu - F_ref, axis=1)
    mag = np.linalg.norm(F_ref, axis=1)
    frms = np.sqrt((mag ** 2).mean())
    return float((d / np.maximum(mag, frms)).max())


def rows_equal(cnt_g, nbr_g, cnt_o, nbr_o):
    """Bit-exact comparison of neighbor rows as sets: counts equal, each
    GPU row's valid entries sorted equal the oracle's sorted row, entries
    unique, padding equal to N."""
    cnt_g = np.asarray(cnt_g)
    nbr_g = np.asarray(nbr_g)
    np.testing.assert_array_equal(cnt_g, cnt_o)
    N = nbr_g.shape[0]
    cap = min(nbr_g.shape[1], nbr_o.shape[1])
    n = np.minimum(cnt_g, cap)
    col = np.arange(nbr_g.shape[1])[None, :]
    valid = col < n[:, None]
    assert np.all(nbr_g[~valid] == N)
    big = np.where(valid, nbr_g, np.iinfo(np.int32).max)
    srt = np.sort(big, axis=1)[:, :cap]
    want = np.where(np.arange(cap)[None, :] < n[:, None], nbr_o[:, :cap], np.iinfo(np.int32).max)
    np.testing.assert_array_equal(srt, want)


def rows_equal_off_cutoff(cnt_g, nbr_g, cnt_o, nbr_o, r, L, r_list, tol=1e-6):
    """Neighbor rows as sets against the oracle's FP32-decision sets, with
    the pairs within tol (sigma) of r_list excluded (their membership may be
    decided by another FP32 rounding): every pair present on one side only
    lies within tol of r_list (FP64 nearest-image distance); rows hold no
    duplicates, padding equals N."""
    cnt_g = np.asarray(cnt_g)
    nbr_g = np.asarray(nbr_g)
    N = nbr_g.shape[0]
    x = np.asarray(r, np.float64)[:, :3]
    col = np.arange(nbr_g.shape[1])[None, :]
    n = np.minimum(cnt_g, nbr_g.shape[1])
    assert np.all(nbr_g[col >= n[:, None]] == N)
    bad = 0
    for i in range(N):
        g = nbr_g[i, : n[i]]
        assert len(np.unique(g)) == len(g), i
        o = nbr_o[i, : cnt_o[i]]
        diff = np.setxor1d(g, o)
        if diff.size:
            d = x[diff] - x[i]
            d -= L * np.round(d / L)
            dist = np.sqrt((d * d).sum(1))
            bad += int(np.sum(np.abs(dist - r_list) > tol))
    assert bad == 0, bad
