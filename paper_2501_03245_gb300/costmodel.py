"""Algorithmic work counts used for the roofline (no GPU code, no arithmetic of
the method itself -- only operation counts).

Basis (fixed, whatever reduction a kernel uses):
  * one modmul or modsqr of an m-limb field costs 2 m^2 + m 32-bit wide
    multiply-adds (m^2 for the product, m^2 + m for the Montgomery reduction;
    Section 4.1: 136 for m = 8);
  * affine PADD = 1 modinv + 3 modmul and PDBL = 1 modinv + 4 modmul (Table 1);
    inside a batch Montgomery's trick replaces the modinv by 3 modmul
    (Section 2.2.1), so a batched PADD costs 6 and a batched PDBL 7 modmul
    (Section 3.1: "6N modmul" for N PADDs).  The per-batch modinv and the
    gather tree are overhead, not counted.
"""

# Table 1 (affine column) and Section 2.2.1
PADD_FORMULA_MODMUL = 3
PDBL_FORMULA_MODMUL = 4
TRICK_MODMUL_PER_ELEMENT = 3
BATCH_PADD_MODMUL = PADD_FORMULA_MODMUL + TRICK_MODMUL_PER_ELEMENT   # 6
BATCH_PDBL_MODMUL = PDBL_FORMULA_MODMUL + TRICK_MODMUL_PER_ELEMENT   # 7

# ECDSA verification schedule of the verification kernel: signed windows of
# Q_WINDOW_BITS bits for u2 (the kernel's kQW), a table {Q .. 2^(w-1) Q} whose
# powers of two are doublings and the rest additions, 8-bit fixed-base comb.
Q_WINDOW_BITS = 5
G_COMB_ADDS = 32        # fixed-base comb, 8-bit windows
FINAL_ADDS = 1          # R = u1 G + u2 Q
SCALAR_MODMUL = 3 + 2 + 2   # batched s^-1 (trick), u1 and u2, two conversions out
PREP_MODMUL = 5 + 4         # five conversions into Montgomery form, on-curve check


def imad_per_modmul(limbs):
    """Wide multiply-adds of one Montgomery multiplication (Section 4.1)."""
    return 2 * limbs * limbs + limbs


def q_digits(w=Q_WINDOW_BITS):
    """Signed radix-2^w digits of a 256-bit scalar: ceil(256 / w), plus a carry
    digit when the top digit holds at least w - 1 bits."""
    top_bits = 256 - w * ((256 - 1) // w)
    return -(-256 // w) + (1 if top_bits >= w - 1 else 0)


def verify_schedule(w=Q_WINDOW_BITS):
    """(batched PDBL, batched PADD) per verification."""
    digits = q_digits(w)
    table = 1 << (w - 1)
    dbl = (digits - 1) * w + (w - 1)            # ladder + table powers of two
    add = digits + G_COMB_ADDS + (table - 1 - (w - 1)) + FINAL_ADDS
    return dbl, add


def verify_modmul(w=Q_WINDOW_BITS):
    """Algorithmic modmul per ECDSA verification (256-bit curves)."""
    dbl, add = verify_schedule(w)
    return dbl * BATCH_PDBL_MODMUL + add * BATCH_PADD_MODMUL + SCALAR_MODMUL + PREP_MODMUL


def verify_imad():
    return verify_modmul() * imad_per_modmul(8)


def fpmul_modmul():
    """Algorithmic modmul per fixed-base multiplication k G (32 comb additions)."""
    return G_COMB_ADDS * BATCH_PADD_MODMUL


# s = k^-1 (e + r d) mod n per signature: the batched inversion of k (3 modmul
# per item) and the products r d and (e + r d) k^-1, plus r into Montgomery form
SIGN_SCALAR_MODMUL = 7


def sign_modmul():
    """Algorithmic modmul per ECDSA signature: k G and the public key d G share
    the 32 comb rounds (two additions per round), then s = k^-1 (e + r d)."""
    return 2 * G_COMB_ADDS * BATCH_PADD_MODMUL + SIGN_SCALAR_MODMUL


def break_even_batch(inv_over_mul=100):
    """Smallest batch N for which 1 modinv + 6N modmul < 11N modmul
    (affine batch vs Jacobian PADD, Section 3.1) with modinv = inv_over_mul modmul."""
    n = 1
    while inv_over_mul + 6 * n >= 11 * n:
        n += 1
    return n


def msm_windows(scalar_bits, c):
    """Signed c-bit windows (c >= 2) of a scalar below 2^scalar_bits: the digits
    reach one bit past the scalar, since a top digit above 2^(c-1) carries out."""
    return -(-(scalar_bits + 1) // c)


def msm_modmul(n_points, windows, c, buckets_touched=None):
    """Algorithmic modmul of one Pippenger MSM with batch-affine bucket
    accumulation: one batched PADD per (point, window) digit, the bucket
    reduction (two additions per bucket) and the window combination
    (c doublings + 1 addition per window)."""
    buckets = windows * (1 << (c - 1)) if buckets_touched is None else buckets_touched
    return (n_points * windows * BATCH_PADD_MODMUL + 2 * buckets * BATCH_PADD_MODMUL
            + windows * (c * BATCH_PDBL_MODMUL + BATCH_PADD_MODMUL))


def msm_modmul_precomputed(n_points, windows, c):
    """The same MSM over bases that carry their window multiples 2^(c w) P_i:
    one batched PADD per (point, window) digit into a single set of 2^(c-1)
    buckets, whose reduction takes two additions per bucket; no window
    combination.  The table itself (c doublings per base and window) is built
    once per set of bases and not counted per call."""
    return n_points * windows * BATCH_PADD_MODMUL + 2 * (1 << (c - 1)) * BATCH_PADD_MODMUL
