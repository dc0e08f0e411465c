"""Pins for the oracle's ECDSA: round trips, corruption, and OpenSSL agreement."""
import numpy as np
import pytest

from oracle import curves, ecdsa
from paper_2501_03245_gb300 import synth

crypto_ec = pytest.importorskip("cryptography.hazmat.primitives.asymmetric.ec")
from cryptography.exceptions import InvalidSignature  # noqa: E402
from cryptography.hazmat.primitives import hashes  # noqa: E402
from cryptography.hazmat.primitives.asymmetric import utils  # noqa: E402

CASES = [(curves.SECP256K1, "SECP256K1"), (curves.P256, "SECP256R1")]


def _ossl_verify(cname, Q, e_bytes, r, s):
    pub = crypto_ec.EllipticCurvePublicNumbers(Q[0], Q[1], getattr(crypto_ec, cname)()).public_key()
    sig = utils.encode_dss_signature(r, s)
    try:
        pub.verify(sig, e_bytes, crypto_ec.ECDSA(utils.Prehashed(hashes.SHA256())))
        return True
    except InvalidSignature:
        return False


@pytest.mark.parametrize("C,cname", CASES, ids=["secp256k1", "P-256"])
def test_oracle_signatures_accepted_by_openssl(C, cname):
    raw = synth.ecdsa_raw(0x6ECC0000, 24, C.n, 4)
    for i in range(24):
        d = int.from_bytes(bytes(raw["d"][i]), "big")
        k = int.from_bytes(bytes(raw["k"][i]), "big")
        e_b = bytes(raw["e"][i])
        e = ecdsa.hash_to_int(e_b)
        r, s = ecdsa.sign(C, d, e, k)
        Q = ecdsa.public_key(C, d)
        assert ecdsa.verify(C, e, r, s, Q)
        assert _ossl_verify(cname, Q, e_b, r, s)


@pytest.mark.parametrize("C,cname", CASES, ids=["secp256k1", "P-256"])
def test_openssl_signatures_and_corruptions(C, cname):
    curve = getattr(crypto_ec, cname)()
    raw = synth.ecdsa_raw(0x6ECC0001, 16, C.n, 1)
    for i in range(16):
        d = int.from_bytes(bytes(raw["d"][i]), "big")
        key = crypto_ec.derive_private_key(d, curve)
        e_b = bytes(raw["e"][i])
        sig = key.sign(e_b, crypto_ec.ECDSA(utils.Prehashed(hashes.SHA256())))
        r, s = utils.decode_dss_signature(sig)
        pn = key.public_key().public_numbers()
        Q = (pn.x, pn.y)
        e = ecdsa.hash_to_int(e_b)
        assert ecdsa.verify(C, e, r, s, Q)
        # corrupt one bit of r or s; oracle and OpenSSL must agree
        bit = int(raw["corrupt_bit"][i])
        if raw["corrupt_kind"][i] == 0:
            r2, s2 = r ^ (1 << bit), s
        else:
            r2, s2 = r, s ^ (1 << bit)
        want = _ossl_verify(cname, Q, e_b, r2, s2) if (0 < r2 < C.n and 0 < s2 < C.n) else False
        assert ecdsa.verify(C, e, r2, s2, Q) == want
        assert want is False
        # other malformed inputs
        assert not ecdsa.verify(C, e, 0, s, Q)
        assert not ecdsa.verify(C, e, r, C.n, Q)
        assert not ecdsa.verify(C, e, r, s, None)
        assert not ecdsa.verify(C, e, r, s, (Q[0], (Q[1] + 1) % C.p))
        # hash not reduced before use: e and e + n sign the same way only mod n
        assert ecdsa.verify(C, e, r, s, Q) == ecdsa.verify(C, e % C.n, r, s, Q)


def test_corruption_recipe_is_deterministic():
    a = synth.ecdsa_raw(0x6ECC0000, 4096, curves.SECP256K1.n, 8)
    b = synth.ecdsa_raw(0x6ECC0000, 4096, curves.SECP256K1.n, 8)
    assert len(a["corrupt_idx"]) == 512 and len(set(a["corrupt_idx"].tolist())) == 512
    for key in a:
        assert np.array_equal(a[key], b[key])
