"""ECDSA signing and verification (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper only states that a verification is one fixed-point multiplication
(u1*G) plus one unknown-point multiplication (u2*Q) (Section 5.2).  The full
procedure is the standard one (SEC 1 v2 section 4.1.4, FIPS 186-4 section 6.4):

verify(e, r, s, Q):
  1. r, s must lie in [1, n-1];
  2. Q must be a point of the curve other than O (both curves have cofactor 1);
  3. e is the 32-byte hash read as a big-endian integer (both orders are
     256-bit, so no truncation; e is not reduced before use);
  4. w = s^-1 mod n, u1 = e w mod n, u2 = r w mod n;
  5. R = u1 G + u2 Q, rejected when R = O;
  6. accept iff x_R mod n == r.

sign(d, e, k): r = x(k G) mod n, s = k^-1 (e + r d) mod n.  Plain ECDSA (no
low-s normalisation).  The nonce k is an input: the caller draws it.

Parity pins (``tests/test_oracle_ecdsa.py``): sign-then-verify round trips,
corrupted signatures rejected, and agreement with OpenSSL (through the
``cryptography`` package, prehashed SHA-256 digests) in both directions on
secp256k1 and P-256.
"""
from . import ec


def hash_to_int(h: bytes) -> int:
    if len(h) != 32:
        raise ValueError("hash must be 32 bytes")
    return int.from_bytes(h, "big")


def public_key(C, d):
    return ec.mul(C, d, C.G)


def sign(C, d, e, k):
    """Returns (r, s).  Raises if the nonce gives r = 0 or s = 0 (probability
    about 2^-256 for a uniform k; the caller then draws another nonce)."""
    n = C.n
    if not (1 <= d < n and 1 <= k < n):
        raise ValueError("d and k must lie in [1, n-1]")
    R = ec.mul(C, k, C.G)
    r = R[0] % n
    s = pow(k, -1, n) * (e + r * d) % n
    if r == 0 or s == 0:
        raise ValueError("degenerate nonce")
    return r, s


def verify(C, e, r, s, Q):
    """Returns True iff (r, s) is a valid signature of hash value e under Q.
    Q is a tuple (x, y) or None; malformed inputs give False, never an error."""
    n = C.n
    if not (1 <= r < n and 1 <= s < n):
        return False
    if Q is None or not ec.on_curve(C, Q):
        return False
    w = pow(s, -1, n)
    u1 = e * w % n
    u2 = r * w % n
    R = ec.add(C, ec.mul(C, u1, C.G), ec.mul(C, u2, Q))
    if R is None:
        return False
    return R[0] % n == r
