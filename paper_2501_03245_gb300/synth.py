"""Seeded synthetic inputs shared by the tests, the oracle and the benchmark.

This module only draws random numbers and reshapes bytes; it holds none of the
elliptic-curve arithmetic (no field, group or ECDSA operation), so the CPU
oracle and the CUDA path can both consume its output without sharing code.

Generator: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) in counter form: output i of stream ``s`` under seed
``seed`` is mix64(key(seed, s) + (i + 1) * 0x9E3779B97F4A7C15) with the
published mix64 finaliser.  Big integers are drawn as little-endian 32-bit limbs
and accepted by rejection (uniform in [lo, hi)), so no modular bias is added.

Workload seeds: workload k uses seed 0x6ECC0000 + k.
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

SEED_BASE = 0x6ECC0000

# stream identifiers (one independent stream per purpose)
S_PRIV, S_HASH, S_NONCE, S_CORRUPT, S_CORRUPT_KIND, S_BASE_MULT, S_SCALAR = 1, 2, 3, 4, 5, 6, 7
S_SIZES, S_ARRIVAL, S_KIND, S_REQSIZE = 8, 9, 10, 11


def _mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed, stream):
    with np.errstate(over="ignore"):
        k = _mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) ^ _mix64(np.uint64(stream) * GAMMA + GAMMA))
    return np.uint64(k)


def splitmix64(seed, stream, start, count):
    """``count`` 64-bit outputs starting at counter ``start``."""
    key = stream_key(seed, stream)
    ctr = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(key + ctr * GAMMA)


def int_to_limbs(v, nlimbs):
    return np.array([(v >> (32 * j)) & 0xFFFFFFFF for j in range(nlimbs)], dtype=np.uint32)


def limbs_to_int(row):
    v = 0
    for j in range(len(row) - 1, -1, -1):
        v = (v << 32) | int(row[j])
    return v


def limbs_to_ints(arr):
    return [limbs_to_int(r) for r in np.asarray(arr)]


def ints_to_limbs(vals, nlimbs):
    out = np.zeros((len(vals), nlimbs), dtype=np.uint32)
    for i, v in enumerate(vals):
        for j in range(nlimbs):
            out[i, j] = (v >> (32 * j)) & 0xFFFFFFFF
    return out


def _less_than(x, bound_limbs):
    """Row-wise x < bound for (count, nlimbs) little-endian limb arrays."""
    lt = np.zeros(x.shape[0], dtype=bool)
    eq = np.ones(x.shape[0], dtype=bool)
    for j in range(x.shape[1] - 1, -1, -1):
        b = bound_limbs[j]
        lt |= eq & (x[:, j] < b)
        eq &= x[:, j] == b
    return lt


def uniform_limbs(seed, stream, count, hi, lo=0, nlimbs=8):
    """``count`` integers uniform in [lo, hi) as (count, nlimbs) uint32 limbs,
    drawn by rejection from bitlen(hi)-bit candidates (2 limbs per 64-bit word)."""
    if hi <= lo:
        raise ValueError("empty range")
    full = hi == 1 << (32 * nlimbs)  # whole limb range: every candidate is < hi
    if hi > 1 << (32 * nlimbs):
        raise ValueError("bound does not fit the limb count")
    bits = (hi - 1).bit_length() if full else hi.bit_length()
    hi_l = None if full else int_to_limbs(hi, nlimbs)
    lo_l = int_to_limbs(lo, nlimbs)
    top = max(bits - 1, 0) // 32
    mask = np.uint32((1 << (bits - 32 * top)) - 1) if bits % 32 else np.uint32(0xFFFFFFFF)
    words_per = (nlimbs + 1) // 2
    out = np.zeros((0, nlimbs), dtype=np.uint32)
    start = 0
    while out.shape[0] < count:
        need = count - out.shape[0]
        batch = need + need // 4 + 16
        w = splitmix64(seed, stream, start, batch * words_per)
        start += batch * words_per
        cand = w.view(np.uint32).reshape(batch, 2 * words_per)[:, :nlimbs].copy()
        cand[:, top] &= mask
        cand[:, top + 1:] = 0
        ok = ~_less_than(cand, lo_l)
        if hi_l is not None:
            ok &= _less_than(cand, hi_l)
        out = np.concatenate([out, cand[ok][:need]])
    return out


def uniform_bytes(seed, stream, count, nbytes):
    w = splitmix64(seed, stream, 0, (count * nbytes + 7) // 8)
    return w.view(np.uint8)[: count * nbytes].reshape(count, nbytes).copy()


def uniform_unit(seed, stream, count, start=0):
    """Doubles uniform in [0, 1) from the top 53 bits of each output."""
    w = splitmix64(seed, stream, start, count)
    return (w >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def limbs_to_be32(arr):
    """(n, 8) little-endian u32 limbs -> (n, 32) big-endian bytes."""
    a = np.ascontiguousarray(np.asarray(arr, dtype=np.uint32)[:, ::-1])
    return a.astype(">u4").view(np.uint8).reshape(a.shape[0], 32)


def be32_to_limbs(b):
    """(n, 32) big-endian bytes -> (n, 8) little-endian u32 limbs."""
    b = np.ascontiguousarray(np.asarray(b, dtype=np.uint8))
    a = b.view(">u4").reshape(b.shape[0], 8).astype(np.uint32)
    return np.ascontiguousarray(a[:, ::-1])


def partial_shuffle(seed, stream, n, count):
    """``count`` distinct indices of range(n) by a seeded partial Fisher-Yates
    shuffle (index j drawn by rejection, no modulo bias)."""
    perm = np.arange(n, dtype=np.int64)
    pos = 0
    draws = splitmix64(seed, stream, 0, 4 * count + 64)
    di = 0
    for i in range(count):
        span = n - i
        limit = (1 << 64) - ((1 << 64) % span)
        while True:
            if di >= draws.shape[0]:
                draws = splitmix64(seed, stream, pos + di, 4 * count + 64)
                pos += di
                di = 0
            v = int(draws[di])
            di += 1
            if v < limit:
                break
        j = i + v % span
        perm[i], perm[j] = perm[j], perm[i]
    return np.sort(perm[:count])


def ecdsa_raw(seed, n_items, order, corrupt_den):
    """Random draws of an ECDSA verification workload.

    d: private keys uniform in [1, order-1] (distinct); e: 32-byte hashes;
    k: nonces uniform in [1, order-1]; ``n_items // corrupt_den`` distinct
    corrupted indices, each flipping one uniform bit (0 = least significant) of
    r (kind 0) or s (kind 1) with a fair coin.
    """
    d = uniform_limbs(seed, S_PRIV, n_items, order, lo=1)
    if n_items > 1 and np.unique(d, axis=0).shape[0] != n_items:
        raise RuntimeError("private-key collision")  # probability ~2^-200
    e = uniform_bytes(seed, S_HASH, n_items, 32)
    k = uniform_limbs(seed, S_NONCE, n_items, order, lo=1)
    n_bad = n_items // corrupt_den if corrupt_den else 0
    idx = partial_shuffle(seed, S_CORRUPT, n_items, n_bad) if n_bad else np.zeros(0, np.int64)
    kw = splitmix64(seed, S_CORRUPT_KIND, 0, max(n_bad, 1))[:n_bad]
    kind = (kw & np.uint64(1)).astype(np.uint8)
    bit = ((kw >> np.uint64(8)) & np.uint64(255)).astype(np.int64)
    return {
        "d": limbs_to_be32(d), "e": e, "k": limbs_to_be32(k),
        "corrupt_idx": idx, "corrupt_kind": kind, "corrupt_bit": bit,
    }


def apply_corruption(r_be, s_be, idx, kind, bit):
    """Flip bit ``bit`` (0 = least significant of the big-endian integer) of r or
    s at each corrupted index; returns new arrays."""
    r2, s2 = r_be.copy(), s_be.copy()
    for i, kd, b in zip(idx, kind, bit):
        tgt = r2 if kd == 0 else s2
        tgt[i, 31 - (b // 8)] ^= np.uint8(1 << (b % 8))
    return r2, s2


def msm_raw(seed, n_points, order, n_vectors=1):
    """Base multipliers a_i uniform in [1, order-1] (bases are a_i * G) and
    ``n_vectors`` scalar vectors uniform in [0, order)."""
    a = uniform_limbs(seed, S_BASE_MULT, n_points, order, lo=1)
    ks = [uniform_limbs(seed, S_SCALAR + 100 * v, n_points, order) for v in range(n_vectors)]
    return a, ks


def ragged_sizes(seed, count, lo_log2=10, hi_log2=18):
    """Sizes floor(2^(lo + (hi - lo) U)), U uniform in [0, 1)."""
    u = uniform_unit(seed, S_SIZES, count)
    return np.floor(np.exp2(lo_log2 + (hi_log2 - lo_log2) * u)).astype(np.int64)
