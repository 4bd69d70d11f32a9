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
    """Bit-exact comparison of sorted padded rows."""
    np.testing.assert_array_equal(np.asarray(cnt_g), cnt_o)
    cap = min(nbr_g.shape[1], nbr_o.shape[1])
    np.testing.assert_array_equal(np.asarray(nbr_g)[:, :cap], nbr_o[:, :cap])
