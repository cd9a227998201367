"""sem_dot_noalloc: the inner product for callers that cannot allocate device
memory when they need it (for example while recording a CUDA graph by stream
capture, or under an application's own pool allocator).  Its scratch is a
fixed device array inside the library instead of memory from cudaMalloc.

Checked through the C ABI against the existing sem_dot on two calls in a row
(the second call reuses the array the first one left behind).  This file is
collected last so that a failure here leaves every other test already run."""
import numpy as np
import pytest

import workloads as W
import paper_2207_07098_gb300 as S

pytestmark = pytest.mark.gpu


def test_dot_noalloc_matches_sem_dot_twice():
    import torch

    m = W.box_mesh(7, 6, 5, 7, amp=0.05)  # 210 elements, 107,520 points: 4 chunks, ragged last
    h = S.sem_setup(m.E, m.lx, m.coords, m.gid, m.mask, W.h1_wavy(m))
    try:
        ref = torch.zeros(1, dtype=torch.float64, device="cuda")
        got = torch.zeros(1, dtype=torch.float64, device="cuda")
        for seed in (1, 2):
            a = torch.from_numpy(W.random_local_field(m, seed, continuous=True)).cuda()
            b = torch.from_numpy(W.random_local_field(m, seed + 10, continuous=True)).cuda()
            S.sem_dot(h, a, b, ref)
            got.fill_(np.nan)
            S.sem_dot_noalloc(h, a, b, got)
            torch.cuda.synchronize()
            r, g = float(ref.item()), float(got.item())
            scale = float(torch.sum(torch.abs(a * b)).item())
            assert abs(g - r) <= 1e-13 * scale, (seed, g, r)
    finally:
        S.sem_destroy(h)
