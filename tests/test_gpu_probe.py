"""The FP32 FMA probe behind the ALU-bound rooflines does the work it
claims: every thread's stored sum equals the closed form of its 8 affine
recurrences x <- a x + b (a = 0.999, b = 1e-3), and the reported FLOP count
is 2 x 8 x iters per thread."""
import numpy as np
import pytest

from gpu_helpers import dev

pytestmark = pytest.mark.gpu


def test_fma_probe_values_and_flop_count():
    import torch
    import paper_1912_04232_b300 as P
    blocks, threads, iters = 3, 96, 1000
    out = torch.full((blocks * threads,), float("nan"), dtype=torch.float32, device=dev())
    fl = P.md_fma_probe(out, blocks, threads, iters)
    torch.cuda.synchronize()
    assert fl == 2 * 8 * iters * threads * blocks
    a, b = np.float64(np.float32(0.999)), np.float64(np.float32(1e-3))
    t = np.arange(threads, dtype=np.float64)
    x0 = np.stack([np.float32(1e-3) * (t + k).astype(np.float32) for k in range(8)]).astype(np.float64)
    an = a ** iters
    xs = (an * x0 + b * (1.0 - an) / (1.0 - a)).sum(0)
    got = out.cpu().numpy().reshape(blocks, threads).astype(np.float64)
    assert np.allclose(got, xs[None, :], rtol=1e-4, atol=0)


def test_fma_probe_rejects_bad_shapes():
    import torch
    import paper_1912_04232_b300 as P
    out = torch.zeros(1024, dtype=torch.float32, device=dev())
    for blocks, threads, iters in ((0, 32, 1), (1, 48, 1), (1, 2048, 1), (1, 32, 0)):
        with pytest.raises(P.MDError):
            P.md_fma_probe(out, blocks, threads, iters)
