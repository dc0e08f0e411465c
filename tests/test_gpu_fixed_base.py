"""GPU parity of batched FPMUL (k G through the fixed-base table) and batched
ECDSA signing, against the oracle, bit-exact."""
import numpy as np
import pytest

from oracle import cpp_oracle, curves, ec
from paper_2501_03245_gb300 import synth
from tests.helpers import from_cuda, limbs_to_points, to_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cid", [0, 1, 2, 3, 4])
def test_fixed_base_mul(gpu_lib, cid):
    import torch

    C = curves.BY_ID[cid]
    n = 2 * 256 * 3 + 11
    a, ks = synth.msm_raw(0x6ECC0800 + cid, n, C.n, 1)
    K = synth.limbs_to_ints(ks[0])
    # edge scalars: 0, 1, n - 1, n (gives O), 2^256 - 1 (not reduced)
    K[:5] = [0, 1, C.n - 1, C.n, (1 << 256) - 1]
    k_l = synth.ints_to_limbs(K, 8)
    out = torch.zeros((n, 2 * C.limbs), dtype=torch.int32, device="cuda")
    gpu_lib.ecc_fixed_base_mul(cid, n, to_cuda(k_l), out)
    torch.cuda.synchronize()
    got = limbs_to_points(C, from_cuda(out).view(np.uint32))
    G = np.tile(np.concatenate([synth.ints_to_limbs([C.gx], C.limbs),
                                synth.ints_to_limbs([C.gy], C.limbs)], axis=1), (n, 1))
    want = limbs_to_points(C, cpp_oracle.scalar_mul(cid, k_l, G))
    assert got == want
    assert got[0] is None and got[1] == C.G and got[3] is None
    assert got[2] == ec.neg(C, C.G)


@pytest.mark.parametrize("cid", [0, 1, 4])
def test_sign_batch(gpu_lib, cid):
    import torch

    C = curves.BY_ID[cid]
    n = 1000
    raw = synth.ecdsa_raw(0x6ECC0900 + cid, n, C.n, 0)
    d, e, k = raw["d"].copy(), raw["e"], raw["k"].copy()
    d[0] = 0                                       # invalid private key
    k[1] = synth.limbs_to_be32(synth.ints_to_limbs([C.n], 8))[0]  # nonce = n
    r = torch.zeros((n, 32), dtype=torch.uint8, device="cuda")
    s = torch.zeros_like(r)
    pub = torch.zeros((n, 64), dtype=torch.uint8, device="cuda")
    gpu_lib.ecc_sign_batch(cid, n, to_cuda(d), to_cuda(e), to_cuda(k), r, s, pub)
    torch.cuda.synchronize()
    r_w, s_w, pub_w = cpp_oracle.sign(cid, d[2:], e[2:], k[2:])
    assert np.array_equal(from_cuda(r)[2:], r_w)
    assert np.array_equal(from_cuda(s)[2:], s_w)
    assert np.array_equal(from_cuda(pub)[2:], pub_w)
    assert from_cuda(r)[:2].sum() == 0 and from_cuda(s)[:2].sum() == 0
