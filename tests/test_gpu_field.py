"""GPU parity of the field layer (a2 modmul, a3 modadd/modsub, a4 modinv,
a5 batch inversion) against the oracle's plain definitions, bit-exact."""
import random

import numpy as np
import pytest

from oracle import curves, field
from paper_2501_03245_gb300 import synth
from tests.helpers import from_cuda, to_cuda

pytestmark = pytest.mark.gpu

CASES = [(cid, f) for cid in range(5) for f in (0, 1)]


def _modulus(cid, f):
    C = curves.BY_ID[cid]
    return (C.p if f == 0 else C.n), (C.limbs if f == 0 else 8)


def _values(q, n, seed):
    rng = random.Random(seed)
    edge = [0, 1, 2, q - 1, q - 2, q // 2, (1 << (q.bit_length() - 1)) % q]
    return (edge + [rng.randrange(q) for _ in range(n)])[:n]


@pytest.mark.parametrize("cid,f", CASES)
def test_fp_mul_add_sub(gpu_lib, cid, f):
    import torch

    q, m = _modulus(cid, f)
    n = 2 * 256 + 37  # several blocks and a ragged tail
    A = _values(q, n, cid * 10 + f)
    B = list(reversed(_values(q, n, cid * 10 + f + 5)))
    a, b = to_cuda(synth.ints_to_limbs(A, m)), to_cuda(synth.ints_to_limbs(B, m))
    out = torch.zeros_like(a)
    for op, ref in ((gpu_lib.ecc_fp_mul, field.mul), (gpu_lib.ecc_fp_add, field.add),
                    (gpu_lib.ecc_fp_sub, field.sub)):
        op(cid, f, n, a, b, out)
        torch.cuda.synchronize()
        got = synth.limbs_to_ints(from_cuda(out))
        assert got == [ref(q, x, y) for x, y in zip(A, B)], op.__name__


@pytest.mark.parametrize("cid,f", CASES)
def test_fp_inverse_single_and_batch(gpu_lib, cid, f):
    import torch

    q, m = _modulus(cid, f)
    for n in (1, 255, 3 * 512 + 7):
        X = _values(q, n, n + cid)
        if n > 10:
            X[3] = 0
            X[n // 2] = 0
        x = to_cuda(synth.ints_to_limbs(X, m))
        out = torch.zeros_like(x)
        want = field.batch_inverse(q, X)
        gpu_lib.ecc_fp_inv_batch(cid, f, n, x, out)
        torch.cuda.synchronize()
        assert synth.limbs_to_ints(from_cuda(out)) == want
        if n <= 255:
            gpu_lib.ecc_fp_inv(cid, f, n, x, out)
            torch.cuda.synchronize()
            assert synth.limbs_to_ints(from_cuda(out)) == [field.inv(q, v) for v in X]


def test_host_memory_staging(gpu_lib):
    """The same call with host (numpy) buffers stages through the device."""
    q, m = _modulus(1, 0)
    A, B = _values(q, 300, 1), _values(q, 300, 2)
    a, b = synth.ints_to_limbs(A, m), synth.ints_to_limbs(B, m)
    out = np.zeros_like(a)
    gpu_lib.ecc_fp_mul(1, 0, 300, a, b, out)
    assert synth.limbs_to_ints(out) == [x * y % q for x, y in zip(A, B)]


def test_argument_errors(gpu_lib):
    import torch

    a = torch.zeros((4, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(gpu_lib.EccError) as e:
        gpu_lib.ecc_fp_mul(9, 0, 4, a, a, a)
    assert e.value.code == gpu_lib.ECC_EINVAL
    with pytest.raises(gpu_lib.EccError):
        gpu_lib.ecc_fp_mul(0, 0, 4, None, a, a)
    gpu_lib.ecc_fp_mul(0, 0, 0, None, None, None)  # n = 0 is a no-op
    with pytest.raises(gpu_lib.EccError) as e:
        gpu_lib.ecc_verify_batch(2, 4, a, a, a, a, a)
    assert e.value.code == gpu_lib.ECC_EUNSUPPORTED


def _carry_heavy(q, n, seed):
    """Operands whose limbs are mostly 0, 1, 2^31 and 2^32 - 1, values next to q
    and to powers of two: they drive long carry runs and zero Montgomery digits
    through a reduction that replaces multiply-adds by additions."""
    rng = random.Random(seed)
    out = []
    while len(out) < n:
        k = rng.randrange(5)
        if k == 0:
            v = sum(rng.choice([0, 1, 0x80000000, 0xFFFFFFFF, rng.randrange(1 << 32)]) << (32 * i)
                    for i in range(8))
        elif k == 1:
            v = q - 1 - rng.randrange(1 << rng.randrange(1, 200))
        elif k == 2:
            v = 1 << rng.randrange(256)
        elif k == 3:
            v = q - (1 << rng.randrange(256))
        else:
            v = rng.randrange(1 << rng.randrange(1, 257))
        out.append(v % q)
    return out


@pytest.mark.parametrize("cid", [1, 0], ids=["P-256", "secp256k1"])
def test_fp_mul_special_form(gpu_lib, cid):
    """The P-256 and secp256k1 base-field unit operations use the special-form
    reductions of Section 4.2 (P-256: u = T_0, u q by additions; secp256k1:
    u q = u 2^256 - u (2^32 + 977)): every product against the oracle on
    operands chosen to stress their carries and borrows."""
    import torch

    q = curves.BY_ID[cid].p
    n = 8192
    A, B = _carry_heavy(q, n, 11), _carry_heavy(q, n, 12)
    a, b = to_cuda(synth.ints_to_limbs(A, 8)), to_cuda(synth.ints_to_limbs(B, 8))
    out = torch.zeros_like(a)
    gpu_lib.ecc_fp_mul(cid, 0, n, a, b, out)
    torch.cuda.synchronize()
    assert synth.limbs_to_ints(from_cuda(out)) == [field.mul(q, x, y) for x, y in zip(A, B)]


def test_bench_modmul_reductions(gpu_lib):
    import torch

    from paper_2501_03245_gb300 import ecc

    sink = torch.zeros(512, dtype=torch.int32, device="cuda")
    gpu_lib.ecc_bench_modmul(1, 1, 512, 4, sink)
    gpu_lib.ecc_bench_modmul(0, 1, 512, 4, sink)
    gpu_lib.ecc_bench_modmul(3, 0, 512, 4, sink)
    torch.cuda.synchronize()
    with pytest.raises(ecc.EccError):
        gpu_lib.ecc_bench_modmul(3, 1, 512, 4, sink)


@pytest.mark.parametrize("cid", [0, 1, 2, 3, 4])
def test_bench_inv_methods_match_the_oracle(gpu_lib, cid):
    """The inversion probe runs a chain of dependent inversions in Montgomery
    form (a = xR -> x^-1 R, then flip bit 0) per thread: Fermat, the 30-bit
    divsteps of the GAS apply step and the 62-bit divsteps end on the oracle's
    chain, folded to one word per thread."""
    import torch

    C = curves.BY_ID[cid]
    q, N = C.p, C.limbs
    R = 1 << (32 * N)
    threads, iters = 70, 9
    one = synth.ints_to_limbs([R % q], N)[0]
    want = []
    for t in range(threads):
        w = [int(one[k]) ^ ((t * 2654435761 + k) & 0xFFFFFFFF) for k in range(N)]
        w[N - 1] &= 0x0FFFFFFF
        a = sum(v << (32 * k) for k, v in enumerate(w))
        for _ in range(iters):
            a = field.mul(q, R * R % q, field.inv(q, a)) if a % q else 0
            a ^= 1
        fold = 0
        for k in range(N):
            fold ^= (a >> (32 * k)) & 0xFFFFFFFF
        want.append(fold)
    for method in (0, 1, 2, 3):
        sink = torch.zeros(threads, dtype=torch.int32, device="cuda")
        gpu_lib.ecc_bench_inv(cid, method, threads, iters, sink)
        torch.cuda.synchronize()
        got = [int(v) & 0xFFFFFFFF for v in sink.cpu().tolist()]
        assert got == want, method
