"""The allocation-free batch inversion entry point (ecc_fp_inv_batch_noalloc).

Some callers may not allocate device memory while a call runs (a fixed memory
budget set at start-up, loops that cannot take the synchronisation cudaMalloc
implies, hosts without an allocator).  This entry point keeps its scratch in a
fixed device array inside the library.  The test calls it through the C ABI and
checks, on two calls in a row, that it returns exactly what ecc_fp_inv_batch
returns for the same input and what the oracle's inverse x^-1 mod q gives for
every element (exact integers: the tolerance is zero), in a base field and a
scalar field.  It runs last so that a failure here leaves every other test
already run.
"""
import numpy as np
import pytest

from paper_2501_03245_gb300 import synth

pytestmark = pytest.mark.gpu

P256_P = 0xFFFFFFFF00000001000000000000000000000000FFFFFFFFFFFFFFFFFFFFFFFF
BLS_P = 0x1A0111EA397FE69A4B1BA7B6434BACD764774B84F38512BF6730D2A0F6B0F6241EABFFFEB153FFFFB9FEFFFFFFFFAAAB
BN_R = 0x30644E72E131A029B85045B68181585D2833E84879B9709143E1F593F0000001


@pytest.mark.parametrize("curve,field,modulus,limbs,n", [
    (1, 0, P256_P, 8, 65536),     # the maximum size
    (3, 0, BLS_P, 12, 5000),
    (2, 1, BN_R, 8, 65536),       # a scalar field (BN254 r), the maximum size
], ids=["P-256-max", "BLS12-381", "BN254-Fr-max"])
def test_noalloc_matches_allocating_entry_point(gpu_lib, curve, field, modulus, limbs, n):
    import torch

    from oracle import field as ofield

    for call in range(2):  # two calls in a row share the same scratch
        vals = synth.uniform_limbs(0x6ECC9000 + 10 * call + curve, 1, n, modulus, nlimbs=limbs)
        vals[7] = 0  # a zero element maps to zero and leaves the others intact
        a = torch.from_numpy(vals.view(np.int32)).cuda()
        want = torch.empty_like(a)
        got = torch.empty_like(a)
        gpu_lib.ecc_fp_inv_batch(curve, field, n, a, want)
        gpu_lib.ecc_fp_inv_batch_noalloc(curve, field, n, a, got)
        torch.cuda.synchronize()
        assert torch.equal(got, want), call
        xs = synth.limbs_to_ints(vals)
        inv = synth.limbs_to_ints(got.cpu().numpy().view(np.uint32))
        assert inv == [ofield.inv(modulus, x) for x in xs], call


def test_noalloc_rejects_oversize_and_host_buffers(gpu_lib):
    import torch

    a = torch.zeros((65537, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(gpu_lib.EccError) as e:
        gpu_lib.ecc_fp_inv_batch_noalloc(1, 0, 65537, a, a)
    assert e.value.code == gpu_lib.ECC_EINVAL and "capacity" in str(e.value)
    h = np.zeros((4, 8), np.uint32)
    with pytest.raises(gpu_lib.EccError):
        gpu_lib.ecc_fp_inv_batch_noalloc(1, 0, 4, h, h)
