"""Parity of the MSM forms that bench.py times, against the oracle.

* ecc_msm_ragged recorded once in a CUDA graph and replayed on two fresh scalar
  sets written into the same input buffer: every instance of each replay
  against its closed form (sum_i k_i a_i mod r) G, the bases being a_i G made by
  the oracle.  Instance sizes span several window widths and include an empty
  and a one-point instance.
* Resident bases with window multiples at the width the BLS12-381 line runs
  (c = 20, one shared set of 2^19 buckets): every vector against the closed
  form, and the same handle's ragged form.
"""
import numpy as np
import pytest

from oracle import curves, ec
from paper_2501_03245_gb300 import synth
from tests.helpers import from_cuda, limbs_to_points, points_to_limbs, random_points, to_cuda

pytestmark = pytest.mark.gpu


def _closed_form(C, a_ints, k_ints):
    acc = sum(x * y for x, y in zip(a_ints, k_ints))
    return ec.mul(C, acc % C.n, C.G)


def test_ragged_msm_graph_replay_fresh_scalars(gpu_lib):
    import torch

    cid, C = 2, curves.BN254
    widths = {10: 8, 12: 8, 14: 13, 17: 15}  # the tuned widths of the 256-MSM line's classes
    sizes = [0, 1, 1024, 5000, 16384, 150000, 5, 3000]
    total = sum(sizes)
    pts, a_ints = random_points(C, total, 0x6ECC2B00)
    pts_l = points_to_limbs(C, pts)
    _, ks = synth.msm_raw(0x6ECC2C00, total, C.n, 2)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    for k, c in widths.items():
        gpu_lib.ecc_msm_set_window(cid, k, c)
    try:
        d_pts = to_cuda(pts_l.view(np.int32))
        d_sc = to_cuda(ks[0].view(np.int32))
        out = torch.zeros((len(sizes), 16), dtype=torch.int32, device="cuda")
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            gpu_lib.ecc_msm_ragged(cid, len(sizes), offs, d_pts, d_sc, out, s)  # warm-up
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            gpu_lib.ecc_msm_ragged(cid, len(sizes), offs, d_pts, d_sc, out, s)
        for v in range(2):
            d_sc.copy_(to_cuda(ks[v].view(np.int32)))
            out.zero_()
            g.replay()
            torch.cuda.synchronize()
            got = limbs_to_points(C, from_cuda(out).view(np.uint32))
            k_ints = synth.limbs_to_ints(ks[v])
            for i in range(len(sizes)):
                lo, hi = int(offs[i]), int(offs[i + 1])
                assert got[i] == _closed_form(C, a_ints[lo:hi], k_ints[lo:hi]), (v, i)
    finally:
        for k in widths:
            gpu_lib.ecc_msm_set_window(cid, k, 0)


def test_window_multiples_at_benched_width(gpu_lib):
    import torch

    cid, C, c = 3, curves.BLS12_381, 20
    n, V = 3000, 2
    pts, a_ints = random_points(C, n, 0x6ECC2D00)
    _, ks = synth.msm_raw(0x6ECC2E00, n, C.n, V)
    ks[1][:100] = ks[1][100:200]  # repeated digits: buckets with many entries
    h = gpu_lib.ecc_bases_create(cid, n, to_cuda(points_to_limbs(C, pts).view(np.int32)))
    try:
        gpu_lib.ecc_bases_precompute(h, c)
        assert gpu_lib.ecc_bases_window(h) == c
        out = torch.zeros((V, 24), dtype=torch.int32, device="cuda")
        gpu_lib.ecc_msm_bases(h, V, to_cuda(np.concatenate(ks).view(np.int32)), out)
        sizes = np.array([n, 1, 1777], np.uint64)
        rk = np.concatenate([ks[0], ks[1][:1], ks[1][:1777]], axis=0)
        rout = torch.zeros((3, 24), dtype=torch.int32, device="cuda")
        gpu_lib.ecc_msm_bases_ragged(h, 3, sizes, to_cuda(rk.view(np.int32)), rout)
        torch.cuda.synchronize()
    finally:
        gpu_lib.ecc_bases_destroy(h)
    got = limbs_to_points(C, from_cuda(out).view(np.uint32))
    for v in range(V):
        assert got[v] == _closed_form(C, a_ints, synth.limbs_to_ints(ks[v])), v
    rgot = limbs_to_points(C, from_cuda(rout).view(np.uint32))
    k1 = synth.limbs_to_ints(ks[1])
    assert rgot[0] == got[0]
    assert rgot[1] == ec.mul(C, a_ints[0] * k1[0] % C.n, C.G)
    assert rgot[2] == _closed_form(C, a_ints[:1777], k1[:1777])
