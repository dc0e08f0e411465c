"""The roofline's work counts against the counts the paper prints
(tests/golden/paper_counts.json, each entry cited there)."""
import json
import os

from paper_2501_03245_gb300 import costmodel

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_counts.json")))


def test_table1_and_trick():
    assert costmodel.PADD_FORMULA_MODMUL == GOLDEN["affine_padd"]["modmul"]
    assert costmodel.PDBL_FORMULA_MODMUL == GOLDEN["affine_pdbl"]["modmul"]
    assert costmodel.TRICK_MODMUL_PER_ELEMENT == GOLDEN["montgomery_trick"]["modmul_per_element"]
    assert costmodel.BATCH_PADD_MODMUL == GOLDEN["batch_padd_modmul_per_op"]["value"]


def test_imad_count_per_modmul():
    g = GOLDEN["imad_modmul_256"]
    assert costmodel.imad_per_modmul(8) == g["total"] == g["product"] + g["reduction"]
    assert costmodel.imad_per_modmul(12) == 300


def test_break_even():
    ratio = GOLDEN["modinv_over_modadd"]["value"] // GOLDEN["modmul_over_modadd"]["value"]
    jac = GOLDEN["jacobian_padd"]["modmul"]
    assert ratio == 100 and jac == 11
    assert costmodel.break_even_batch(ratio) == GOLDEN["break_even_batch_exclusive"]["value"] + 1


def test_verify_count_structure():
    # w = 5: 52 digits (51 x 5 ladder doublings), table {Q..16Q}: 4 doublings,
    # 11 additions; 52 + 32 + 11 + 1 additions in all
    assert [costmodel.q_digits(w) for w in (4, 5, 6)] == [65, 52, 43]
    assert costmodel.verify_schedule(5) == (259, 96)
    assert costmodel.verify_schedule(4) == (259, 102)
    m = costmodel.verify_modmul()
    assert m == 259 * 7 + 96 * 6 + 7 + 9
    assert costmodel.verify_imad() == m * 136
    assert costmodel.fpmul_modmul() == 32 * 6
    # signing: k G and d G ride the same 32 comb rounds, then s = k^-1 (e + r d)
    assert costmodel.sign_modmul() == 2 * costmodel.fpmul_modmul() + costmodel.SIGN_SCALAR_MODMUL


def test_verify_schedule_matches_the_kernel():
    """The cost model's window width is the verification kernel's (read from
    the CUDA source, whose digit count the same rule gives)."""
    import os
    import re

    src = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "paper_2501_03245_gb300", "csrc", "verify.cuh")
    text = open(src).read()
    assert int(re.search(r"constexpr int kQW = (\d+);", text).group(1)) == costmodel.Q_WINDOW_BITS


def test_msm_precomputed_count():
    # one bucket set instead of W, no window combination
    n, c = 1 << 20, 16
    W = -(-256 // c)
    assert costmodel.msm_modmul_precomputed(n, W, c) == 6 * n * W + 2 * 6 * (1 << (c - 1))
    assert costmodel.msm_modmul(n, W, c) - costmodel.msm_modmul_precomputed(n, W, c) == \
        2 * 6 * (W - 1) * (1 << (c - 1)) + W * (7 * c + 6)


def _signed_digits(k, c):
    """Signed radix-2^c recoding with digits in [-2^(c-1)+1, 2^(c-1)]."""
    out = []
    while k:
        d = k & ((1 << c) - 1)
        if d > (1 << (c - 1)):
            d -= 1 << c
        out.append(d)
        k = (k - d) >> c
    return out


def test_msm_windows_by_brute_force():
    # every scalar below 2^b recodes into msm_windows(b, c) signed digits, and
    # some scalar needs all of them (c >= 2, the library's range: at c = 1 the
    # digit set is {0, 1} and never carries)
    for b in range(1, 11):
        for c in range(2, 8):
            need = max(len(_signed_digits(k, c)) for k in range(1 << b))
            assert need == costmodel.msm_windows(b, c), (b, c)
    assert costmodel.msm_windows(255, 16) == 16   # BLS12-381 r
    assert costmodel.msm_windows(254, 13) == 20   # BN254 r
