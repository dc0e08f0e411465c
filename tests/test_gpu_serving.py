"""Serving loop: every result is bit-identical alone and in the continuous-batched
mix, and matches the oracle (ECDSA bits and MSM points)."""
import math

import numpy as np
import pytest

from oracle import cpp_oracle, curves
from paper_2501_03245_gb300 import serving
from tests.helpers import limbs_to_points

pytestmark = pytest.mark.gpu


def test_serving_mix_equals_alone_and_oracle(gpu_lib):
    import torch

    srv = serving.Server(torch, pool_triples=4096, n_bases=4096, pool_scalars=1 << 14,
                         hbm_budget=64 << 20, max_verify_round=3000, max_msm_round_points=6000)
    try:
        trace = serving.make_trace(0x6ECC5000, 24, rate=2000.0, verify_max_log2=9,
                                   msm_lo_log2=6, msm_hi_log2=11, pool_triples=4096,
                                   pool_scalars=1 << 14)
        srv.run(trace)
        assert all(q.done is not None and q.done >= q.arrival - 1e-3 for q in trace)
        kinds = {q.kind for q in trace}
        assert kinds == {"verify", "msm"}
        e, r, s, pub = (t.cpu().numpy() for t in (srv.e, srv.r, srv.s, srv.pub))
        pts = srv.bases_pts.cpu().numpy().view(np.uint32)
        sc = srv.scalars.cpu().numpy().view(np.uint32)
        C = curves.BN254
        for q in trace:
            alone = srv.run_alone(q)
            assert np.array_equal(alone, q.result), q.rid
            lo, hi = q.offset, q.offset + q.size
            if q.kind == "verify":
                want = cpp_oracle.verify(0, e[lo:hi], r[lo:hi], s[lo:hi], pub[lo:hi])
                assert np.array_equal(q.result, want), q.rid
            else:
                want = cpp_oracle.msm(2, pts[:q.size], sc[lo:hi])
                assert limbs_to_points(C, q.result[None, :]) == limbs_to_points(C, want[None, :])
        summary = serving.summarise(trace)
        assert summary["requests"] == 24 and summary["p99_ms"] >= summary["p50_ms"] > 0
        assert math.isfinite(summary["throughput_req_s"])
    finally:
        srv.close()
