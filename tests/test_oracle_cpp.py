"""Pins for the plain C++ oracle against the Python oracle (two independent
implementations: Barrett + Jacobian + MSB-first vs Python ints + affine + Algorithm 1)."""
import random

import numpy as np
import pytest

from oracle import curves, ec, ecdsa
from paper_2501_03245_gb300 import synth


@pytest.mark.parametrize("cid", [0, 1, 2, 3, 4])
def test_field_mul_inv(cpp_oracle, cid):
    C = curves.BY_ID[cid]
    rng = random.Random(cid)
    for which, mod in ((0, C.p), (1, C.n)):
        m = C.limbs if which == 0 else 8
        vals_a = [0, 1, mod - 1, (1 << (32 * m - 1)) % mod] + [rng.randrange(mod) for _ in range(60)]
        vals_b = [mod - 1, mod - 1, mod - 1, 2] + [rng.randrange(mod) for _ in range(60)]
        got = synth.limbs_to_ints(cpp_oracle.fe_mul(cid, which, synth.ints_to_limbs(vals_a, m),
                                                    synth.ints_to_limbs(vals_b, m)))
        assert got == [a * b % mod for a, b in zip(vals_a, vals_b)]
        inv = synth.limbs_to_ints(cpp_oracle.fe_inv(cid, which, synth.ints_to_limbs(vals_a, m)))
        assert inv == [pow(a, -1, mod) if a else 0 for a in vals_a]


@pytest.mark.parametrize("cid", [0, 1, 2, 3, 4])
def test_scalar_mul_and_msm(cpp_oracle, cid):
    C = curves.BY_ID[cid]
    m = C.limbs
    a, ks = synth.msm_raw(0x6ECC0100 + cid, 12, C.n, 1)
    A, K = synth.limbs_to_ints(a), synth.limbs_to_ints(ks[0])
    K[0] = 0
    K[1] = C.n  # n * P = O
    k_l = synth.ints_to_limbs(K, 8)
    P = [ec.mul(C, x, C.G) for x in A]
    P[2] = None  # O input encoded (0, 0)
    pts = np.concatenate([synth.ints_to_limbs([ec.encode(q)[0] for q in P], m),
                          synth.ints_to_limbs([ec.encode(q)[1] for q in P], m)], axis=1)
    out = cpp_oracle.scalar_mul(cid, k_l, pts)
    for i in range(12):
        want = ec.encode(ec.mul(C, K[i], P[i]) if P[i] else None)
        assert (synth.limbs_to_int(out[i, :m]), synth.limbs_to_int(out[i, m:])) == want
    o = cpp_oracle.msm(cid, pts, k_l)
    want = ec.encode(ec.msm(C, K, [q for q in P]) if True else None)
    assert (synth.limbs_to_int(o[:m]), synth.limbs_to_int(o[m:])) == want


@pytest.mark.parametrize("cid", [0, 1, 4])
def test_sign_verify_agree(cpp_oracle, cid):
    C = curves.BY_ID[cid]
    raw = synth.ecdsa_raw(0x6ECC0200 + cid, 48, C.n, 3)
    r, s, pub = cpp_oracle.sign(cid, raw["d"], raw["e"], raw["k"])
    r2, s2 = synth.apply_corruption(r, s, raw["corrupt_idx"], raw["corrupt_kind"], raw["corrupt_bit"])
    # extra malformed rows: r = 0, s = n, Q off-curve, Q = (0, 0)
    r2[0] = 0
    s2[1] = synth.limbs_to_be32(synth.ints_to_limbs([C.n], 8))[0]
    pub = pub.copy()
    pub[2, 63] ^= 1
    pub[3] = 0
    ok = cpp_oracle.verify(cid, raw["e"], r2, s2, pub)
    for i in range(48):
        d = int.from_bytes(bytes(raw["d"][i]), "big")
        k = int.from_bytes(bytes(raw["k"][i]), "big")
        e = int.from_bytes(bytes(raw["e"][i]), "big")
        assert (int.from_bytes(bytes(r[i]), "big"), int.from_bytes(bytes(s[i]), "big")) == ecdsa.sign(C, d, e, k)
        Q = (int.from_bytes(bytes(pub[i, :32]), "big"), int.from_bytes(bytes(pub[i, 32:]), "big"))
        want = ecdsa.verify(C, e, int.from_bytes(bytes(r2[i]), "big"), int.from_bytes(bytes(s2[i]), "big"),
                            ec.decode(Q))
        assert bool(ok[i]) == want, i
    assert ok[:4].sum() == 0 and ok[4:].sum() > 20
