"""Device-resident instance sizes, the device status word, point validation and
the caller's workspace allocator.

* ecc_msm_ragged_dev / ecc_msm_bases_ragged_dev read the instance boundaries
  from device memory: one CUDA graph, captured once with a capacity, is
  replayed on two different size mixes written into the same device buffer,
  and every instance of each replay must equal its closed form
  (sum_i k_i a_i mod r) G (bases a_i G made by the oracle).
* Sizes the device refuses (decreasing offsets) give O outputs and ECC_EINVAL
  from ecc_sync_status; the next valid call is unaffected.
* ecc_validate_points against the curve equation checked by the oracle.
* Every workspace taken from a caller allocator (torch's caching allocator)
  gives the same results as the default.
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


@pytest.mark.parametrize("cid", [2, 3])
def test_ragged_dev_one_graph_two_size_mixes(gpu_lib, cid):
    import torch

    C = curves.BY_ID[cid]
    L = 2 * C.limbs
    cap, num = 40000, 6
    pts, a_ints = random_points(C, cap, 0x6ECC3000 + cid)
    _, ks = synth.msm_raw(0x6ECC3100 + cid, cap, C.n, 2)
    mixes = [[0, 1, 7000, 300, 20000, 5000], [12000, 12000, 0, 2, 999, 14999]]  # the second fills cap
    d_pts = to_cuda(points_to_limbs(C, pts).view(np.int32))
    d_sc = to_cuda(ks[0].view(np.int32))
    d_off = torch.zeros(num + 1, dtype=torch.int64, device="cuda")
    out = torch.zeros((num, L), dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    d_off.copy_(torch.from_numpy(np.concatenate([[0], np.cumsum(mixes[0])]).astype(np.int64)))
    with torch.cuda.stream(s):
        gpu_lib.ecc_msm_ragged_dev(cid, num, cap, d_off, d_pts, d_sc, out, 0, s)  # warm-up
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        gpu_lib.ecc_msm_ragged_dev(cid, num, cap, d_off, d_pts, d_sc, out, 0, s)
    for v, sizes in enumerate(mixes):
        offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        d_off.copy_(torch.from_numpy(offs))
        d_sc.copy_(to_cuda(ks[v].view(np.int32)))
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        got = limbs_to_points(C, from_cuda(out).view(np.uint32))
        k_ints = synth.limbs_to_ints(ks[v])
        for i in range(num):
            lo, hi = int(offs[i]), int(offs[i + 1])
            assert got[i] == _closed_form(C, a_ints[lo:hi], k_ints[lo:hi]), (v, i)
    gpu_lib.ecc_sync_status(torch.cuda.current_stream())


@pytest.mark.parametrize("table_c", [0, 11])
def test_bases_ragged_dev_one_graph_two_size_mixes(gpu_lib, table_c):
    import torch

    cid, C = 2, curves.BN254
    n, num = 9000, 5
    pts, a_ints = random_points(C, n, 0x6ECC3200 + table_c)
    _, ks = synth.msm_raw(0x6ECC3300 + table_c, 3 * n, C.n, 1)
    mixes = [[n, 1, 0, 4000, 777], [3, 8999, 2500, 2500, 0]]
    cap = max(sum(m) for m in mixes)
    h = gpu_lib.ecc_bases_create(cid, n, to_cuda(points_to_limbs(C, pts).view(np.int32)))
    try:
        if table_c:
            gpu_lib.ecc_bases_precompute(h, table_c)
        d_sizes = torch.zeros(num, dtype=torch.int64, device="cuda")
        d_sc = to_cuda(ks[0].view(np.int32))
        out = torch.zeros((num, 16), dtype=torch.int32, device="cuda")
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        d_sizes.copy_(torch.tensor(mixes[0], dtype=torch.int64))
        with torch.cuda.stream(s):
            gpu_lib.ecc_msm_bases_ragged_dev(h, num, cap, d_sizes, d_sc, out, s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            gpu_lib.ecc_msm_bases_ragged_dev(h, num, cap, d_sizes, d_sc, out, s)
        k_all = synth.limbs_to_ints(ks[0])
        for v, sizes in enumerate(mixes):
            d_sizes.copy_(torch.tensor(sizes, dtype=torch.int64))
            out.zero_()
            g.replay()
            torch.cuda.synchronize()
            got = limbs_to_points(C, from_cuda(out).view(np.uint32))
            row = 0
            for i, m in enumerate(sizes):
                assert got[i] == _closed_form(C, a_ints[:m], k_all[row:row + m]), (v, i)
                row += m
    finally:
        gpu_lib.ecc_bases_destroy(h)


def test_refused_device_sizes_set_the_status_word(gpu_lib):
    import torch

    cid, C = 2, curves.BN254
    cap, num = 4000, 3
    pts, a_ints = random_points(C, cap, 0x6ECC3400)
    _, ks = synth.msm_raw(0x6ECC3500, cap, C.n, 1)
    d_pts = to_cuda(points_to_limbs(C, pts).view(np.int32))
    d_sc = to_cuda(ks[0].view(np.int32))
    out = torch.ones((num, 16), dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    gpu_lib.ecc_sync_status(stream)  # nothing pending
    for bad in ([0, 100, 50, 200], [5, 100, 200, 300], [0, 100, 200, cap + 1]):
        d_off = torch.tensor(bad, dtype=torch.int64, device="cuda")
        gpu_lib.ecc_msm_ragged_dev(cid, num, cap, d_off, d_pts, d_sc, out, 0)
        with pytest.raises(gpu_lib.EccError) as e:
            gpu_lib.ecc_sync_status(stream)
        assert e.value.code == gpu_lib.ECC_EINVAL
        assert not out.any()  # every output is O
    # the word is cleared, and a valid call that follows is unaffected
    offs = np.array([0, 100, 1000, cap], np.int64)
    gpu_lib.ecc_msm_ragged_dev(cid, num, cap, to_cuda(offs), d_pts, d_sc, out, 0)
    gpu_lib.ecc_sync_status(stream)
    got = limbs_to_points(C, from_cuda(out).view(np.uint32))
    k_ints = synth.limbs_to_ints(ks[0])
    for i in range(num):
        assert got[i] == _closed_form(C, a_ints[offs[i]:offs[i + 1]], k_ints[offs[i]:offs[i + 1]])


@pytest.mark.parametrize("cid", [0, 1, 2, 3, 4])
def test_validate_points(gpu_lib, cid):
    import torch

    C = curves.BY_ID[cid]
    pts, _ = random_points(C, 64, 0x6ECC3600 + cid)
    L = points_to_limbs(C, pts + [None]).astype(np.uint32)
    rows = [L]
    # off the curve: y + 1; x replaced by p (not canonical); y = p - y + p (not canonical)
    bad = L[:3].copy()
    bad[0] = points_to_limbs(C, [pts[0]])[0]
    bad[0][C.limbs:] = synth.ints_to_limbs([(pts[0][1] + 1) % C.p], C.limbs)[0]
    bad[1][:C.limbs] = synth.ints_to_limbs([C.p], C.limbs)[0]
    bad[2][C.limbs:] = synth.ints_to_limbs([C.p + pts[2][1] if C.p + pts[2][1] < (1 << (32 * C.limbs)) else C.p],
                                           C.limbs)[0]
    rows.append(bad)
    allp = np.concatenate(rows)
    want = [1] * 65 + [int(ec.on_curve(C, (pts[0][0], (pts[0][1] + 1) % C.p))), 0, 0]
    ok = torch.zeros(len(allp), dtype=torch.uint8, device="cuda")
    gpu_lib.ecc_validate_points(cid, len(allp), to_cuda(allp.view(np.int32)), ok)
    torch.cuda.synchronize()
    assert from_cuda(ok).tolist() == want


def test_caller_allocator_gives_the_same_results(gpu_lib):
    import torch

    calls = {"alloc": 0, "free": 0}

    def alloc(nbytes, stream):
        calls["alloc"] += 1
        return torch.cuda.caching_allocator_alloc(nbytes, torch.cuda.current_device(), stream)

    def release(ptr, stream):
        calls["free"] += 1
        torch.cuda.caching_allocator_delete(ptr)

    cid, C = 3, curves.BLS12_381
    pts, _ = random_points(C, 3000, 0x6ECC3700)
    _, ks = synth.msm_raw(0x6ECC3800, 3000, C.n, 1)
    d_pts = to_cuda(points_to_limbs(C, pts).view(np.int32))
    d_sc = to_cuda(ks[0].view(np.int32))
    want = torch.zeros((1, 24), dtype=torch.int32, device="cuda")
    gpu_lib.ecc_msm(cid, 3000, d_pts, d_sc, want)
    got = torch.zeros_like(want)
    gpu_lib.ecc_set_allocator(alloc, release)
    try:
        gpu_lib.ecc_msm(cid, 3000, d_pts, d_sc, got)
        torch.cuda.synchronize()
    finally:
        gpu_lib.ecc_set_allocator(None, None)
    assert torch.equal(got, want)
    assert calls["alloc"] > 0 and calls["alloc"] == calls["free"]
