"""GPU parity of the Pippenger MSM (digits, counting sort by bucket id, batched
affine bucket accumulation, bucket reduction, window combination) against the
oracle's definition sum_i k_i P_i, bit-exact, including ragged batches, resident
bases and degenerate inputs."""
import numpy as np
import pytest

from oracle import cpp_oracle, curves, ec
from paper_2501_03245_gb300 import synth
from tests.helpers import from_cuda, limbs_to_points, points_to_limbs, random_points, to_cuda

pytestmark = pytest.mark.gpu


def _pts_limbs(C, pts):
    return points_to_limbs(C, pts)


def _oracle_msm(cid, pts_l, k_l):
    C = curves.BY_ID[cid]
    return limbs_to_points(C, cpp_oracle.msm(cid, pts_l, k_l)[None, :])[0]


def _gpu_msm(gpu_lib, cid, pts_l, k_l):
    import torch

    C = curves.BY_ID[cid]
    out = torch.zeros((1, 2 * C.limbs), dtype=torch.int32, device="cuda")
    gpu_lib.ecc_msm(cid, pts_l.shape[0], to_cuda(pts_l), to_cuda(k_l), out)
    torch.cuda.synchronize()
    return limbs_to_points(C, from_cuda(out).view(np.uint32))[0]


@pytest.mark.parametrize("cid", [2, 3])
@pytest.mark.parametrize("n", [1, 37, 1000])
def test_msm_random(gpu_lib, cid, n):
    C = curves.BY_ID[cid]
    pts, _ = random_points(C, n, 0x6ECC0A00 + cid + n)
    _, ks = synth.msm_raw(0x6ECC0B00 + n, n, C.n, 1)
    K = synth.limbs_to_ints(ks[0])
    if n >= 37:
        K[0] = 0
        K[1] = C.n               # reduces to 0
        K[2] = (1 << 256) - 1    # reduced mod r on the device
        pts[3] = pts[4]          # the same base twice (bucket collisions)
        pts[5] = ec.neg(C, pts[6])
        K[5] = K[6]              # P and -P with equal digits cancel
    pts_l, k_l = _pts_limbs(C, pts), synth.ints_to_limbs(K, 8)
    assert _gpu_msm(gpu_lib, cid, pts_l, k_l) == _oracle_msm(cid, pts_l, k_l)


@pytest.mark.parametrize("cid", [2, 3])
def test_msm_degenerate(gpu_lib, cid):
    C = curves.BY_ID[cid]
    pts, _ = random_points(C, 64, 0x6ECC0C00 + cid)
    pts_l = _pts_limbs(C, pts)
    zero = np.zeros((64, 8), np.uint32)
    assert _gpu_msm(gpu_lib, cid, pts_l, zero) is None
    # k P + (r - k) P = O
    K = [5, C.n - 5] + [0] * 62
    same = _pts_limbs(C, [pts[0], pts[0]] + pts[2:])
    assert _gpu_msm(gpu_lib, cid, same, synth.ints_to_limbs(K, 8)) is None
    # all scalars equal -> one bucket per window holds every point
    K = [0x1234567] * 64
    pts_l2 = _pts_limbs(C, pts)
    assert _gpu_msm(gpu_lib, cid, pts_l2, synth.ints_to_limbs(K, 8)) == \
        _oracle_msm(cid, pts_l2, synth.ints_to_limbs(K, 8))


@pytest.mark.parametrize("cid", [2, 3])
def test_msm_ragged(gpu_lib, cid):
    import torch

    C = curves.BY_ID[cid]
    sizes = [0, 1, 5, 300, 33, 700, 2, 128]
    total = sum(sizes)
    pts, _ = random_points(C, total, 0x6ECC0D00 + cid)
    _, ks = synth.msm_raw(0x6ECC0E00 + cid, total, C.n, 1)
    pts_l, k_l = _pts_limbs(C, pts), ks[0]
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    out = torch.zeros((len(sizes), 2 * C.limbs), dtype=torch.int32, device="cuda")
    gpu_lib.ecc_msm_ragged(cid, len(sizes), offs, to_cuda(pts_l), to_cuda(k_l), out)
    torch.cuda.synchronize()
    got = limbs_to_points(C, from_cuda(out).view(np.uint32))
    for i in range(len(sizes)):
        lo, hi = int(offs[i]), int(offs[i + 1])
        want = _oracle_msm(cid, pts_l[lo:hi], k_l[lo:hi]) if hi > lo else None
        assert got[i] == want, i
    # each instance alone gives the same result as inside the mix
    for i in (3, 5):
        lo, hi = int(offs[i]), int(offs[i + 1])
        assert _gpu_msm(gpu_lib, cid, pts_l[lo:hi], k_l[lo:hi]) == got[i]


@pytest.mark.parametrize("cid", [2, 3])
def test_msm_resident_bases(gpu_lib, cid):
    import torch

    C = curves.BY_ID[cid]
    n, V = 500, 3
    pts, _ = random_points(C, n, 0x6ECC0F00 + cid)
    _, ks = synth.msm_raw(0x6ECC1000 + cid, n, C.n, V)
    pts_l = _pts_limbs(C, pts)
    h = gpu_lib.ecc_bases_create(cid, n, to_cuda(pts_l))
    try:
        k_all = np.concatenate(ks, axis=0)
        out = torch.zeros((V, 2 * C.limbs), dtype=torch.int32, device="cuda")
        gpu_lib.ecc_msm_bases(h, V, to_cuda(k_all), out)
        torch.cuda.synchronize()
        got = limbs_to_points(C, from_cuda(out).view(np.uint32))
        for v in range(V):
            assert got[v] == _oracle_msm(cid, pts_l, ks[v]), v
    finally:
        gpu_lib.ecc_bases_destroy(h)


def test_msm_window_override_same_result(gpu_lib):
    cid = 2
    C = curves.BY_ID[cid]
    pts, _ = random_points(C, 700, 0x6ECC1100)
    _, ks = synth.msm_raw(0x6ECC1200, 700, C.n, 1)
    pts_l = _pts_limbs(C, pts)
    want = _oracle_msm(cid, pts_l, ks[0])
    for c in (3, 7, 12, 16):
        gpu_lib.ecc_msm_set_window(cid, 9, c)  # size class 2^9 .. 2^10 - 1
        assert gpu_lib.ecc_msm_window(cid, 700) == c
        assert _gpu_msm(gpu_lib, cid, pts_l, ks[0]) == want, c
    gpu_lib.ecc_msm_set_window(cid, 9, 0)


@pytest.mark.parametrize("cid", [2, 3])
def test_msm_reduce_chunk_override_same_result(gpu_lib, cid):
    """The bucket layout of the reduction (first-level chunks of 2^k buckets)
    changes the rounds, never the sum: every k against the oracle, with
    several window widths so chunks straddle or exceed a bucket row."""
    C = curves.BY_ID[cid]
    pts, _ = random_points(C, 700, 0x6ECC1800 + cid)
    _, ks = synth.msm_raw(0x6ECC1900 + cid, 700, C.n, 1)
    pts_l = _pts_limbs(C, pts)
    want = _oracle_msm(cid, pts_l, ks[0])
    try:
        for c in (4, 9):
            gpu_lib.ecc_msm_set_window(cid, 9, c)
            for k in (1, 2, 3, 5, 7, 10):
                gpu_lib.ecc_msm_set_reduce_chunk(cid, 9, k)
                assert gpu_lib.ecc_msm_reduce_chunk(cid, 700) == k
                assert _gpu_msm(gpu_lib, cid, pts_l, ks[0]) == want, (c, k)
    finally:
        gpu_lib.ecc_msm_set_window(cid, 9, 0)
        gpu_lib.ecc_msm_set_reduce_chunk(cid, 9, 0)


def test_msm_unsupported_curve(gpu_lib):
    import torch

    a = torch.zeros((4, 16), dtype=torch.int32, device="cuda")
    with pytest.raises(gpu_lib.EccError) as e:
        gpu_lib.ecc_msm(0, 4, a, a, a)
    assert e.value.code == gpu_lib.ECC_EUNSUPPORTED


@pytest.mark.parametrize("cid,n,c,same", [(3, 4096, 15, False), (2, 8192, 0, True)])
def test_msm_heavy_buckets(gpu_lib, cid, n, c, same):
    """Buckets holding hundreds of partial sums: BLS12-381 at c = 15 (the top
    window holds only the carry, so about half the points share one bucket) and
    BN254 with every scalar equal (each window's only bucket holds all n)."""
    C = curves.BY_ID[cid]
    pts, _ = random_points(C, n, 0x6ECC1300 + cid)
    _, ks = synth.msm_raw(0x6ECC1400 + cid, n, C.n, 1)
    k_l = ks[0]
    if same:
        k_l = np.repeat(k_l[:1], n, axis=0)
    pts_l = _pts_limbs(C, pts)
    log2n = n.bit_length() - 1
    if c:
        gpu_lib.ecc_msm_set_window(cid, log2n, c)
    try:
        assert _gpu_msm(gpu_lib, cid, pts_l, k_l) == _oracle_msm(cid, pts_l, k_l)
    finally:
        if c:
            gpu_lib.ecc_msm_set_window(cid, log2n, 0)


@pytest.mark.parametrize("cid,c", [(2, 7), (2, 13), (3, 5), (3, 12)])
def test_msm_bases_precomputed_windows(gpu_lib, cid, c):
    """Resident bases with window multiples 2^(c w) P_i: every vector against the
    oracle and against the same handle without the table, the ragged form too."""
    import torch

    C = curves.BY_ID[cid]
    n, V = 700, 3
    pts, _ = random_points(C, n, 0x6ECC1500 + cid)
    _, ks = synth.msm_raw(0x6ECC1600 + cid + c, n, C.n, V)
    ks[1][:50] = ks[1][50:100]          # repeated digits: buckets with many entries
    ks[2][0] = synth.ints_to_limbs([C.n - 1], 8)[0]
    pts_l = _pts_limbs(C, pts)
    h = gpu_lib.ecc_bases_create(cid, n, to_cuda(pts_l))
    try:
        k_all = to_cuda(np.concatenate(ks, axis=0))
        plain = torch.zeros((V, 2 * C.limbs), dtype=torch.int32, device="cuda")
        gpu_lib.ecc_msm_bases(h, V, k_all, plain)
        assert gpu_lib.ecc_bases_window(h) == 0
        gpu_lib.ecc_bases_precompute(h, c)
        assert gpu_lib.ecc_bases_window(h) == c
        out = torch.zeros_like(plain)
        gpu_lib.ecc_msm_bases(h, V, k_all, out)
        sizes = np.array([n, 1, 333], np.uint64)
        rk = np.concatenate([ks[0], ks[1][:1], ks[2][:333]], axis=0)
        rout = torch.zeros((3, 2 * C.limbs), dtype=torch.int32, device="cuda")
        gpu_lib.ecc_msm_bases_ragged(h, 3, sizes, to_cuda(rk), rout)
        torch.cuda.synchronize()
        got = limbs_to_points(C, from_cuda(out).view(np.uint32))
        assert got == limbs_to_points(C, from_cuda(plain).view(np.uint32))
        for v in range(V):
            assert got[v] == _oracle_msm(cid, pts_l, ks[v]), v
        rgot = limbs_to_points(C, from_cuda(rout).view(np.uint32))
        assert rgot[0] == got[0]
        assert rgot[1] == _oracle_msm(cid, pts_l[:1], ks[1][:1])
        assert rgot[2] == _oracle_msm(cid, pts_l[:333], ks[2][:333])
    finally:
        gpu_lib.ecc_bases_destroy(h)


def test_msm_bases_precompute_rejects(gpu_lib):
    from paper_2501_03245_gb300 import ecc

    C = curves.BN254
    pts, _ = random_points(C, 8, 0x6ECC1700)
    h = gpu_lib.ecc_bases_create(2, 8, to_cuda(_pts_limbs(C, pts)))
    try:
        for c in (1, 25):
            with pytest.raises(ecc.EccError):
                gpu_lib.ecc_bases_precompute(h, c)
        assert gpu_lib.ecc_bases_window(h) == 0
    finally:
        gpu_lib.ecc_bases_destroy(h)


def test_msm_rejects_digit_overflow(gpu_lib):
    """A resident-bases call whose (point, window) digits would pass 2^31 is
    refused before any work (sizes are checked on the host)."""
    import torch

    from paper_2501_03245_gb300 import ecc

    C = curves.BN254
    n = 1 << 20
    pts = torch.zeros((n, 16), dtype=torch.int32, device="cuda")
    h = gpu_lib.ecc_bases_create(2, n, pts)
    try:
        sc = torch.zeros((8, 8), dtype=torch.int32, device="cuda")  # never read
        out = torch.zeros((4096, 16), dtype=torch.int32, device="cuda")
        with pytest.raises(ecc.EccError) as ex:
            gpu_lib.ecc_msm_bases(h, 4096, sc, out)  # 4096 x 2^20 x W digits
        assert ex.value.code == ecc.ECC_EINVAL
    finally:
        gpu_lib.ecc_bases_destroy(h)
