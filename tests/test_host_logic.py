"""Host-side logic that runs without a GPU: the MSM window-width table behind
ecc_msm_window / ecc_msm_set_window, argument checks that reject a call before
any device work, and the serving loop's request trace and latency summary."""
import math
import os
import shutil

import numpy as np
import pytest

from paper_2501_03245_gb300 import costmodel, serving, synth


@pytest.fixture(scope="module")
def ecc():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2501_03245_gb300 import build, ecc as binding

    build.build()
    binding.load()
    return binding


MSM_CURVES = [(2, 254), (3, 255)]  # (curve id, bits of the group order r)


@pytest.mark.parametrize("cid,bits", MSM_CURVES, ids=["BN254", "BLS12-381"])
def test_default_window_is_near_work_optimal(ecc, cid, bits):
    # The library's default width per size class, against the algorithmic count
    # of a Pippenger MSM (digits, bucket reduction, window combination)
    prev = 0
    for l in range(6, 27):
        n = 1 << l
        c = ecc.ecc_msm_window(cid, n)
        assert 2 <= c <= 20
        assert c >= prev  # wider windows as n grows
        prev = c
        cost = {k: costmodel.msm_modmul(n, costmodel.msm_windows(bits, k), k) for k in range(2, 21)}
        assert cost[c] <= 1.05 * min(cost.values()), (l, c)


def test_window_override_covers_its_size_class_and_resets(ecc):
    cid, l = 2, 14
    model = ecc.ecc_msm_window(cid, 1 << l)
    below, above = ecc.ecc_msm_window(cid, (1 << l) - 1), ecc.ecc_msm_window(cid, 1 << (l + 1))
    other = ecc.ecc_msm_window(3, 1 << l)
    pick = 9 if model != 9 else 10
    try:
        ecc.ecc_msm_set_window(cid, l, pick)
        assert ecc.ecc_msm_window(cid, 1 << l) == pick
        assert ecc.ecc_msm_window(cid, (1 << (l + 1)) - 1) == pick   # floor(log2 n) = l
        assert ecc.ecc_msm_window(cid, (1 << l) - 1) == below        # neighbouring classes keep theirs
        assert ecc.ecc_msm_window(cid, 1 << (l + 1)) == above
        assert ecc.ecc_msm_window(3, 1 << l) == other                # so does the other curve
    finally:
        ecc.ecc_msm_set_window(cid, l, 0)
    assert ecc.ecc_msm_window(cid, 1 << l) == model


@pytest.mark.parametrize("args", [(2, 14, 1), (2, 14, 21), (2, -1, 8), (2, 41, 8), (9, 3, 8)])
def test_window_override_rejects_bad_arguments(ecc, args):
    with pytest.raises(ecc.EccError) as e:
        ecc.ecc_msm_set_window(*args)
    assert e.value.code == ecc.ECC_EINVAL


def test_calls_rejected_before_device_work(ecc):
    z = np.zeros(64, np.uint8)
    w = z.view(np.uint32)
    cases = [
        (lambda: ecc.ecc_verify_batch(2, 4, z, z, z, z, z), ecc.ECC_EUNSUPPORTED, "ECDSA"),
        (lambda: ecc.ecc_verify_batch(1, 4, None, z, z, z, z), ecc.ECC_EINVAL, "NULL"),
        (lambda: ecc.ecc_verify_batch(1, (1 << 26) + 1, z, z, z, z, z), ecc.ECC_EINVAL, "2^26"),
        (lambda: ecc.ecc_sign_batch(2, 4, z, z, z, z, z, z), ecc.ECC_EUNSUPPORTED, "ECDSA"),
        (lambda: ecc.ecc_msm(0, 4, w, w, w), ecc.ECC_EUNSUPPORTED, "MSM"),
        (lambda: ecc.ecc_msm_ragged(1, 1, np.array([0, 4], np.uint64), w, w, w), ecc.ECC_EUNSUPPORTED, "MSM"),
        (lambda: ecc.ecc_fp_mul(1, 2, 4, z, z, z), ecc.ECC_EINVAL, "field"),
        (lambda: ecc.ecc_bases_create(3, 4, None), ecc.ECC_EINVAL, "NULL"),
        (lambda: ecc.ecc_fp_inv_batch_noalloc(1, 0, 65537, z, z), ecc.ECC_EINVAL, "capacity"),
    ]
    for call, code, text in cases:
        with pytest.raises(ecc.EccError) as e:
            call()
        assert e.value.code == code and text in str(e.value), str(e.value)
    assert ecc.ecc_verify_batch(1, 0, z, z, z, z, z) == ecc.ECC_OK  # n = 0: no work, no error


def test_trace_shape_and_determinism():
    count, rate = 20000, 500.0
    a = serving.make_trace(synth.SEED_BASE + 4, count, rate)
    b = serving.make_trace(synth.SEED_BASE + 4, count, rate)
    assert [(q.kind, q.size, q.arrival, q.offset) for q in a] == \
        [(q.kind, q.size, q.arrival, q.offset) for q in b]
    t = [q.arrival for q in a]
    assert all(x <= y for x, y in zip(t, t[1:]))
    gaps = np.diff([0.0] + t)
    # exponential inter-arrival times: mean 1/rate, coefficient of variation 1
    assert abs(gaps.mean() * rate - 1) < 0.05
    assert abs(gaps.std() / gaps.mean() - 1) < 0.05
    nv = sum(q.kind == "verify" for q in a)
    assert abs(nv / count - 0.5) < 0.02
    for q in a:
        if q.kind == "verify":
            assert 1 <= q.size <= 4096 and q.offset + q.size <= 1 << 16
        else:
            assert 1 << 12 <= q.size <= 1 << 20 and q.offset + q.size <= 1 << 22
    # log-uniform sizes: about half the MSM requests below 2^16
    msm = [q.size for q in a if q.kind == "msm"]
    assert abs(sum(s < 1 << 16 for s in msm) / len(msm) - 0.5) < 0.03
    burst = serving.make_trace(1, 50, math.inf)
    assert all(q.arrival == 0.0 for q in burst)


def test_summary_percentiles_are_nearest_rank():
    reqs = []
    for i in range(100):
        q = serving.Request(i, "verify" if i % 2 else "msm", 10, 0.0, 0)
        q.done = (i + 1) / 1000.0  # latencies 1 .. 100 ms
        reqs.append(q)
    s = serving.summarise(reqs, span=2.0)
    assert s["p50_ms"] == pytest.approx(50.0) and s["p99_ms"] == pytest.approx(99.0)
    assert s["mean_ms"] == pytest.approx(50.5)
    assert s["throughput_req_s"] == pytest.approx(50.0)
    assert s["verify_triples_s"] == pytest.approx(250.0) and s["msm_points_s"] == pytest.approx(250.0)


def test_round_admission_by_workspace_and_ring_contiguity():
    """A round takes waiting requests in arrival order while their payloads are
    contiguous in the ring, within the item limit and the workspace budget; a
    request whose workspace does not fit what is left waits."""
    R = serving.Request
    reqs = [R(0, "verify", 100, 0.0, 0), R(1, "verify", 50, 0.0, 100), R(2, "verify", 30, 0.0, 150),
            R(3, "verify", 40, 0.0, 0)]                       # the ring wrapped before request 3
    cost = lambda items: 1000 + 10 * items  # noqa: E731
    batch, items = serving.take_round(reqs, 1 << 20, 10 ** 9, cost)
    assert [q.rid for q in batch] == [0, 1, 2] and items == 180
    batch, _ = serving.take_round(reqs, 160, 10 ** 9, cost)    # item limit
    assert [q.rid for q in batch] == [0, 1]
    batch, _ = serving.take_round(reqs, 1 << 20, cost(150), cost)  # budget: the third does not fit
    assert [q.rid for q in batch] == [0, 1]
    batch, items = serving.take_round(reqs, 1 << 20, cost(99), cost)  # not even the first: wait
    assert batch == [] and items == 0


def test_request_work_follows_the_cost_model():
    v = serving.request_work("verify", 10, 16)
    assert v == 10 * costmodel.verify_imad()
    m = serving.request_work("msm", 1 << 12, 16)
    W = costmodel.msm_windows(254, 16)
    assert m == costmodel.msm_modmul_precomputed(1 << 12, W, 16) * 136
