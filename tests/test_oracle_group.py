"""Pins for the oracle's group law (Eqn 2-3, PDBL) and double-and-add (Algorithm 1).

Tiny curves are enumerated by brute force (every (x, y) tested against Eqn 1),
so the point set is known independently of the addition formulas.  A dropped
term, a wrong sign or a swapped operand in PADD / PDBL breaks closure,
associativity or collinearity on these tables.
"""
import itertools
import random

import pytest

from oracle import curves, ec, tiny

TINY_PRIMES = [11, 13, 17, 23, 31, 43, 47, 101, 103]


def tiny_curves():
    rng = random.Random(0x6ECC)
    out = []
    for p in TINY_PRIMES:
        for a in (0, p - 3, rng.randrange(1, p)):
            for b in range(1, p):
                if (4 * a**3 + 27 * b**2) % p:
                    out.append(tiny.make(p, a, b))
                    break
    return out


TINY = tiny_curves()


@pytest.mark.parametrize("C", TINY, ids=lambda c: c.name)
def test_tiny_axioms(C):
    pts = tiny.points(C)
    allp = [None] + pts
    n_e = len(allp)
    # Hasse bound
    assert (n_e - (C.p + 1)) ** 2 <= 4 * C.p
    S = set(allp)
    table = {}
    for P in allp:
        assert ec.add(C, P, None) == P and ec.add(C, None, P) == P
        assert ec.add(C, P, ec.neg(C, P)) is None
        assert ec.dbl(C, P) == ec.add(C, P, P)
        for T in allp:
            R = ec.add(C, P, T)
            assert R in S  # closure
            table[(P, T)] = R
    for P, T in itertools.product(allp, allp):
        assert table[(P, T)] == table[(T, P)]  # commutativity
    # collinearity: P, T and -(P + T) lie on one line when P != +-T
    for P, T in itertools.product(pts, pts):
        if P[0] == T[0]:
            continue
        R = table[(P, T)]
        mR = ec.neg(C, R)
        lhs = (T[1] - P[1]) * (mR[0] - P[0]) - (mR[1] - P[1]) * (T[0] - P[0])
        assert lhs % C.p == 0
    # associativity: exhaustive for p <= 31, sampled above
    triples = itertools.product(allp, allp, allp)
    if C.p > 31:
        rng = random.Random(C.p)
        triples = [(rng.choice(allp), rng.choice(allp), rng.choice(allp)) for _ in range(20000)]
    for P, T, U in triples:
        assert table[(table[(P, T)], U)] == table[(P, table[(T, U)])]
    # Lagrange: every point order divides #E; scalar multiplication agrees
    for P in pts:
        k = tiny.order(C, P, ec.add)
        assert n_e % k == 0
        assert ec.mul(C, k, P) is None
        assert ec.mul(C, k + 1, P) == P
        for s in range(0, 2 * k + 3):
            Q = None
            for _ in range(s):
                Q = ec.add(C, Q, P)
            assert ec.mul(C, s, P) == Q


@pytest.mark.parametrize("C", list(curves.BY_ID.values()), ids=lambda c: c.name)
def test_large_curve_laws(C):
    rng = random.Random(C.p & 0xFFFF)
    pts = [ec.mul(C, rng.randrange(1, C.n), C.G) for _ in range(6)]
    for P in pts:
        assert ec.on_curve(C, P)
        assert ec.add(C, P, ec.neg(C, P)) is None
        assert ec.dbl(C, P) == ec.add(C, P, P)
    for P, T, U in itertools.combinations(pts, 3):
        assert ec.add(C, ec.add(C, P, T), U) == ec.add(C, P, ec.add(C, T, U))
    # scalar linearity: (a + b) P = a P + b P, (a b) G = a (b G)
    a, b = rng.randrange(C.n), rng.randrange(C.n)
    assert ec.mul(C, a + b, C.G) == ec.add(C, ec.mul(C, a, C.G), ec.mul(C, b, C.G))
    assert ec.mul(C, a * b % C.n, C.G) == ec.mul(C, a, ec.mul(C, b, C.G))


def test_msm_definition_and_closed_form():
    C = curves.BN254
    rng = random.Random(7)
    a = [rng.randrange(1, C.n) for _ in range(9)]
    k = [rng.randrange(C.n) for _ in range(9)] + [0]
    a.append(5)
    P = [ec.mul(C, x, C.G) for x in a]
    # closed form: sum k_i (a_i G) = (sum k_i a_i mod n) G
    assert ec.msm(C, k, P) == ec.mul(C, sum(x * y for x, y in zip(k, a)) % C.n, C.G)
    # linearity in the scalars
    k2 = [rng.randrange(C.n) for _ in range(10)]
    assert ec.add(C, ec.msm(C, k, P), ec.msm(C, k2, P)) == ec.msm(C, [x + y for x, y in zip(k, k2)], P)
    assert ec.msm(C, [0] * 10, P) is None
    assert ec.msm(C, [], []) is None


@pytest.mark.parametrize("C", list(curves.BY_ID.values()), ids=lambda c: c.name)
def test_large_curve_associativity_random_triples(C):
    # 2500 triples per curve (12,500 over the five curves) from a pool of random
    # multiples of G, its negatives, O and repeated points, so the exceptional
    # branches (P = T doubles, P = -T cancels, O passes through) meet the
    # regular ones in every position of (P + T) + U = P + (T + U)
    rng = random.Random(C.n & 0xFFFFFF)
    base = [ec.mul(C, rng.randrange(1, C.n), C.G) for _ in range(24)]
    pool = base + [ec.neg(C, P) for P in base[:6]] + [None]
    for _ in range(2500):
        P, T, U = rng.choice(pool), rng.choice(pool), rng.choice(pool)
        if rng.random() < 0.1:
            T = P
        assert ec.add(C, ec.add(C, P, T), U) == ec.add(C, P, ec.add(C, T, U))
