"""sem_dot_noalloc: the inner product for callers that cannot allocate device
memory when they need it (for example while recording a CUDA graph by stream
capture, or under an application's own pool allocator).  Its scratch is a
fixed device array inside the library instead of memory from cudaMalloc.

Checked through the C ABI against the existing sem_dot on two calls in a row
(the second call reuses the array the first one left behind), and against the
oracle's inner product on a batch handle of uneven meshes, with calls issued
back to back on one stream before any host synchronisation.  This file is
collected last so that a failure here leaves every other test already run."""
import numpy as np
import pytest

import oracle
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


def test_dot_noalloc_batch_matches_oracle_back_to_back():
    """A batch handle of meshes of uneven sizes and orders (one result per
    mesh; the shared ticket counter is cleared before each mesh's launch):
    two products issued back to back on one stream, read only after both,
    each against the oracle's inner product of every member."""
    import torch

    meshes = [W.box_mesh(1, 1, 1, 2), W.box_mesh(9, 8, 7, 7, amp=0.05), W.box_mesh(2, 3, 1, 4, amp=0.03),
              W.box_mesh(5, 4, 4, 9, amp=0.06)]
    h = S.sem_setup_batch([(m.E, m.lx, m.coords, m.gid, m.mask, None) for m in meshes])
    try:
        fields = []
        for seed in (3, 4):
            a = np.concatenate([W.random_local_field(m, seed + 7 * q, continuous=True) for q, m in enumerate(meshes)])
            b = np.concatenate([W.random_local_field(m, seed + 50 + q, continuous=True) for q, m in enumerate(meshes)])
            fields.append((a, b))
        outs = [torch.full((len(meshes),), np.nan, dtype=torch.float64, device="cuda") for _ in fields]
        devs = [(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()) for a, b in fields]
        torch.cuda.synchronize()
        for (ad, bd), out in zip(devs, outs):  # no host synchronisation between the two calls
            S.sem_dot_noalloc(h, ad, bd, out)
        torch.cuda.synchronize()
        off = np.cumsum([0] + [m.n_local for m in meshes])
        for (a, b), out in zip(fields, outs):
            got = out.cpu().numpy()
            for q, m in enumerate(meshes):
                P = oracle.Problem(m)
                aq, bq = a[off[q]:off[q + 1]], b[off[q]:off[q + 1]]
                ref = P.dot(aq, bq)
                scale = float(np.sum(np.abs(aq * bq) / P.mult()))
                assert abs(got[q] - ref) <= 1e-13 * scale, (q, got[q], ref)
    finally:
        S.sem_destroy(h)
