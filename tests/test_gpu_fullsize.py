"""Parity at the workloads' full sizes, in the configuration bench.py times.

* P-256 verification of 2^20 triples with the 1/16 corruption recipe applied
  over the full 2^20 positions: a pool of 4096 oracle-signed triples is tiled,
  and the oracle verifies every distinct (triple, corruption) combination, so
  every one of the 2^20 output bits has an oracle value.
* BLS12-381 MSM, 2^20 resident bases a_i G, 16 scalar vectors: each result
  against the closed form (sum_i k_i a_i mod r) G (one oracle scalar
  multiplication); a sample of the bases against the oracle.
* BN254 ragged batch of 256 MSMs with log-uniform sizes 2^10..2^18: every
  instance against its closed form.
"""
import numpy as np
import pytest

from oracle import cpp_oracle, curves, ec
from paper_2501_03245_gb300 import synth
from tests.helpers import from_cuda, limbs_to_points, to_cuda

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_verify_p256_full_size(gpu_lib):
    import torch

    C = curves.P256
    n, pool = 1 << 20, 4096
    raw = synth.ecdsa_raw(synth.SEED_BASE + 1, pool, C.n, 0)
    r0, s0, pub0 = cpp_oracle.sign(1, raw["d"], raw["e"], raw["k"])
    reps = n // pool
    e, r, s, pub = (np.tile(a, (reps, 1)) for a in (raw["e"], r0, s0, pub0))
    cor = synth.ecdsa_raw(synth.SEED_BASE + 1, n, C.n, 16)  # corruption recipe over 2^20 positions
    r, s = synth.apply_corruption(r, s, cor["corrupt_idx"], cor["corrupt_kind"], cor["corrupt_bit"])
    want = np.tile(cpp_oracle.verify(1, raw["e"], r0, s0, pub0), reps)
    idx = cor["corrupt_idx"]
    want[idx] = cpp_oracle.verify(1, e[idx], r[idx], s[idx], pub[idx])
    ok = torch.zeros(n, dtype=torch.uint8, device="cuda")
    gpu_lib.ecc_verify_batch(1, n, to_cuda(e), to_cuda(r), to_cuda(s), to_cuda(pub), ok)
    torch.cuda.synchronize()
    assert np.array_equal(from_cuda(ok), want)
    assert want.sum() == n - len(idx)


def _bases(gpu_lib, cid, a_limbs):
    import torch

    C = curves.BY_ID[cid]
    n = a_limbs.shape[0]
    out = torch.empty((n, 2 * C.limbs), dtype=torch.int32, device="cuda")
    gpu_lib.ecc_fixed_base_mul(cid, n, to_cuda(a_limbs.view(np.int32)), out)
    torch.cuda.synchronize()
    return out


def _closed_form(C, a_ints, k_ints):
    acc = 0
    for x, y in zip(a_ints, k_ints):
        acc += x * y
    return ec.mul(C, acc % C.n, C.G)


def test_msm_bls12_381_full_size(gpu_lib):
    import torch

    cid, C = 3, curves.BLS12_381
    n, V = 1 << 20, 16
    a, ks = synth.msm_raw(synth.SEED_BASE + 2, n, C.n, V)
    bases = _bases(gpu_lib, cid, a)
    # the bases themselves, sampled, against the oracle
    a_ints = synth.limbs_to_ints(a)
    pts = from_cuda(bases).view(np.uint32)
    for i in np.linspace(0, n - 1, 24).astype(int):
        assert limbs_to_points(C, pts[i:i + 1])[0] == ec.mul(C, a_ints[i], C.G)
    h = gpu_lib.ecc_bases_create(cid, n, bases)
    try:
        out = torch.empty((V, 2 * C.limbs), dtype=torch.int32, device="cuda")
        gpu_lib.ecc_msm_bases(h, V, to_cuda(np.concatenate(ks).view(np.int32)), out)
        torch.cuda.synchronize()
        got = limbs_to_points(C, from_cuda(out).view(np.uint32))
    finally:
        gpu_lib.ecc_bases_destroy(h)
    for v in range(V):
        assert got[v] == _closed_form(C, a_ints, synth.limbs_to_ints(ks[v])), v


def test_msm_bn254_ragged_full_size(gpu_lib):
    import torch

    cid, C = 2, curves.BN254
    sizes = synth.ragged_sizes(synth.SEED_BASE + 3, 256)
    total = int(sizes.sum())
    a, ks = synth.msm_raw(synth.SEED_BASE + 3, total, C.n, 1)
    bases = _bases(gpu_lib, cid, a)
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    out = torch.empty((256, 2 * C.limbs), dtype=torch.int32, device="cuda")
    gpu_lib.ecc_msm_ragged(cid, 256, offs, bases, to_cuda(ks[0].view(np.int32)), out)
    torch.cuda.synchronize()
    got = limbs_to_points(C, from_cuda(out).view(np.uint32))
    a_ints, k_ints = synth.limbs_to_ints(a), synth.limbs_to_ints(ks[0])
    for i in range(256):
        lo, hi = int(offs[i]), int(offs[i + 1])
        assert got[i] == _closed_form(C, a_ints[lo:hi], k_ints[lo:hi]), i
