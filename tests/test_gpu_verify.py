"""GPU parity of batched ECDSA verification (a10) against the oracle.

Inputs are oracle-signed triples from the seeded generator, with the corruption
recipe of the workload (one bit of r or s flipped in 1/8 or 1/16 of the items)
and extra malformed rows.  Expected bits come from the oracle only."""
import numpy as np
import pytest

from oracle import cpp_oracle, curves
from paper_2501_03245_gb300 import synth
from tests.helpers import from_cuda, to_cuda

pytestmark = pytest.mark.gpu


def make_triples(cid, n, seed, den):
    C = curves.BY_ID[cid]
    raw = synth.ecdsa_raw(seed, n, C.n, den)
    r, s, pub = cpp_oracle.sign(cid, raw["d"], raw["e"], raw["k"])
    r, s = synth.apply_corruption(r, s, raw["corrupt_idx"], raw["corrupt_kind"], raw["corrupt_bit"])
    return raw["e"], r, s, pub


def add_malformed(cid, e, r, s, pub):
    C = curves.BY_ID[cid]
    e, r, s, pub = e.copy(), r.copy(), s.copy(), pub.copy()
    n_be = synth.limbs_to_be32(synth.ints_to_limbs([C.n], 8))[0]
    p_be = synth.limbs_to_be32(synth.ints_to_limbs([C.p], 8))[0]
    r[0] = 0                       # r = 0
    s[1] = n_be                    # s = n
    pub[2, 63] ^= 1                # Q off the curve
    pub[3] = 0                     # Q = (0, 0)
    pub[4, :32] = p_be             # x_Q = p (not canonical)
    r[5] = 0xFF                    # r > n
    e[6] = 0xFF                    # e = 2^256 - 1 (>= n, reduced mod n)
    return e, r, s, pub


def run_gpu(gpu_lib, cid, e, r, s, pub):
    import torch

    n = e.shape[0]
    ok = torch.zeros(n, dtype=torch.uint8, device="cuda")
    gpu_lib.ecc_verify_batch(cid, n, to_cuda(e), to_cuda(r), to_cuda(s), to_cuda(pub), ok)
    torch.cuda.synchronize()
    return from_cuda(ok)


@pytest.mark.parametrize("cid", [0, 1, 4])
def test_verify_small_with_malformed(gpu_lib, cid):
    e, r, s, pub = make_triples(cid, 700, 0x6ECC0500 + cid, 8)
    e, r, s, pub = add_malformed(cid, e, r, s, pub)
    want = cpp_oracle.verify(cid, e, r, s, pub)
    got = run_gpu(gpu_lib, cid, e, r, s, pub)
    assert np.array_equal(got, want)
    assert want[:6].sum() == 0 and want[6:].sum() > 500


def test_verify_secp256k1_4096(gpu_lib):
    """The secp256k1 workload: 4096 seeded triples, 512 corrupted."""
    e, r, s, pub = make_triples(0, 4096, synth.SEED_BASE + 0, 8)
    want = cpp_oracle.verify(0, e, r, s, pub)
    got = run_gpu(gpu_lib, 0, e, r, s, pub)
    assert np.array_equal(got, want)
    assert 4096 - 512 <= want.sum() < 4096


def test_verify_host_buffers(gpu_lib):
    e, r, s, pub = make_triples(1, 300, 0x6ECC0600, 16)
    ok = np.zeros(300, np.uint8)
    gpu_lib.ecc_verify_batch(1, 300, e, r, s, pub, ok)
    assert np.array_equal(ok, cpp_oracle.verify(1, e, r, s, pub))


@pytest.mark.parametrize("n", [1, 33])
def test_verify_tiny_batches(gpu_lib, n):
    e, r, s, pub = make_triples(1, n, 0x6ECC0700 + n, 0)
    assert run_gpu(gpu_lib, 1, e, r, s, pub).sum() == n


def test_verify_ragged_sets_in_a_cuda_graph(gpu_lib):
    """Verification requests of uneven sizes concatenated into one call,
    captured once in a CUDA graph and replayed on new inputs in the same
    buffers: every replay bit-exact against the oracle."""
    import torch

    cid = 4
    sizes = [1, 17, 300, 2048, 64, 5]
    n = sum(sizes)
    sets = [make_triples(cid, n, 0x6ECC1800 + k, 8) for k in range(2)]
    bufs = [torch.zeros(x.shape, dtype=torch.uint8, device="cuda") for x in sets[0]]
    ok = torch.zeros(n, dtype=torch.uint8, device="cuda")
    for b, x in zip(bufs, sets[0]):
        b.copy_(torch.from_numpy(x))
    gpu_lib.ecc_verify_batch(cid, n, *bufs, ok)  # builds the fixed-base table outside the capture
    torch.cuda.synchronize()
    st = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        gpu_lib.ecc_verify_batch(cid, n, *bufs, ok, st)
    for x in sets:
        for b, arr in zip(bufs, x):
            b.copy_(torch.from_numpy(arr))
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(from_cuda(ok), cpp_oracle.verify(cid, *x))


@pytest.mark.parametrize("cid", [0, 1, 4])
@pytest.mark.parametrize("ctas", [1, 2])
@pytest.mark.parametrize("n", [5000, 77])
def test_verify_cluster_gas(gpu_lib, n, ctas, cid):
    """Verification with one inversion per CTA and with the two CTAs of a
    cluster sharing each round's inversion (ecc_set_gas_cluster) gives the
    oracle's bits; 77 triples leave the second CTA of the pair without items."""
    e, r, s, pub = make_triples(cid, n, 0x6ECC4100 + n + cid, 16)
    e, r, s, pub = add_malformed(cid, e, r, s, pub)
    want = cpp_oracle.verify(cid, e, r, s, pub)
    from paper_2501_03245_gb300 import ecc

    gpu_lib.ecc_set_gas_cluster(ctas)
    try:
        got = run_gpu(gpu_lib, cid, e, r, s, pub)
    finally:
        gpu_lib.ecc_set_gas_cluster(DEFAULT_GAS_CLUSTER)
    assert np.array_equal(got, want)
    with pytest.raises(ecc.EccError):
        gpu_lib.ecc_set_gas_cluster(4)


# the library's default cluster size for verification
DEFAULT_GAS_CLUSTER = 2
