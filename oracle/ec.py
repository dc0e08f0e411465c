"""Affine elliptic-curve group law, scalar multiplication and naive MSM (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Points are ``(x, y)`` tuples of canonical integers in [0, p); the point at
infinity O is ``None``.  Every function works for any odd prime p and any curve
y^2 = x^3 + a x + b (Eqn 1), so the same code serves the four standard curves
and the tiny curves enumerated by ``oracle.tiny``.

Parity pins (``tests/test_oracle_group.py``, ``tests/test_oracle_curves.py``):
exhaustive group axioms on tiny curves (closure, identity, inverse,
commutativity, associativity), Hasse bound and Lagrange on tiny curves,
collinearity of P, T and -(P+T), n*G = O on the standard curves, and agreement
with OpenSSL's public-key derivation d*G for secp256k1 and P-256.
"""


def on_curve(C, P):
    """True when P is O or satisfies y^2 = x^3 + a x + b mod p (Eqn 1)."""
    if P is None:
        return True
    x, y = P
    if not (0 <= x < C.p and 0 <= y < C.p):
        return False
    return (y * y - (x * x * x + C.a * x + C.b)) % C.p == 0


def neg(C, P):
    """-P = (x, -y); -O = O."""
    if P is None:
        return None
    x, y = P
    return (x, (-y) % C.p)


def dbl(C, P):
    """PDBL (Section 2.1.1): lambda = (3 x^2 + a) / (2 y), then as PADD.

    2O = O, and a point with y = 0 has order 2, so its double is O.
    """
    if P is None:
        return None
    x, y = P
    p = C.p
    if y % p == 0:
        return None
    lam = (3 * x * x + C.a) * pow(2 * y, -1, p) % p
    xr = (lam * lam - 2 * x) % p
    yr = (lam * (x - xr) - y) % p
    return (xr, yr)


def add(C, P, T):
    """PADD (Eqn 2-3): lambda = (y_p - y_t) / (x_p - x_t),
    x_r = lambda^2 - x_p - x_t, y_r = lambda (x_p - x_r) - y_p.

    The exceptional inputs the equations leave out are resolved by the group law:
    O is the identity, P + P is PDBL, and P + (-P) = O.
    """
    if P is None:
        return T
    if T is None:
        return P
    p = C.p
    xp, yp = P
    xt, yt = T
    if xp == xt:
        if (yp + yt) % p == 0:
            return None
        return dbl(C, P)
    lam = (yp - yt) * pow(xp - xt, -1, p) % p
    xr = (lam * lam - xp - xt) % p
    yr = (lam * (xp - xr) - yp) % p
    return (xr, yr)


def mul(C, s, P):
    """Double-and-add, least-significant bit first (Algorithm 1).

    Q starts at O; for each bit s_i (i = 0 .. l-1): if s_i = 1 then Q = Q + P;
    then P = P + P.  Any integer s >= 0 is accepted (no reduction mod n).
    """
    if s < 0:
        raise ValueError("scalar must be non-negative")
    Q = None
    for i in range(s.bit_length()):
        if (s >> i) & 1:
            Q = add(C, Q, P)
        P = dbl(C, P)
    return Q


def msm(C, scalars, points):
    """Multi-scalar multiplication by its definition: sum_i k_i * P_i, each term
    by double-and-add (Algorithm 1), summed with the group law."""
    acc = None
    for k, P in zip(scalars, points):
        acc = add(C, acc, mul(C, k, P))
    return acc


def encode(P):
    """Affine encoding used at the library boundary: O is written as (0, 0)
    (not on any curve here, since b != 0)."""
    return (0, 0) if P is None else P


def decode(P):
    return None if P == (0, 0) else P
