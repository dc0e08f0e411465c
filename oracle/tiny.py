"""Tiny prime-field curves, enumerated by brute force (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

For a small odd prime p every pair (x, y) in F_p^2 is tested against Eqn 1, so
the point set is known without any group-law code; the group law of
``oracle.ec`` is then checked against the axioms on the complete addition table.
"""
from .curves import Curve


def make(p, a, b):
    """A tiny curve (no generator or order attached)."""
    if (4 * a**3 + 27 * b**2) % p == 0:
        raise ValueError("singular curve")
    return Curve(name=f"tiny-{p}-{a}-{b}", p=p, a=a % p, b=b % p, gx=0, gy=0, n=0, h=0)


def points(C):
    """All affine points of C, by checking every (x, y) against Eqn 1."""
    p = C.p
    out = []
    for x in range(p):
        rhs = (x * x * x + C.a * x + C.b) % p
        for y in range(p):
            if (y * y - rhs) % p == 0:
                out.append((x, y))
    return out


def order(C, P, add):
    """Order of P by repeated addition (brute force)."""
    k, Q = 1, P
    while Q is not None:
        Q = add(C, Q, P)
        k += 1
    return k
