"""GPU parity of the batched affine PADD / PDBL (a6, a7) against the oracle's
group law, bit-exact, including every exceptional case and tiny-curve-free
edge inputs (O, P = T, P = -T)."""
import pytest

from oracle import curves, ec
from tests.helpers import from_cuda, limbs_to_points, points_to_limbs, random_points, to_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cid", [0, 1, 2, 3, 4])
def test_point_add_dbl(gpu_lib, cid):
    import torch

    C = curves.BY_ID[cid]
    pts, _ = random_points(C, 600, 0x6ECC0300 + cid)
    P = pts[:300]
    T = pts[300:]
    # exceptional pairs
    T[0] = P[0]                      # P + P -> doubling
    T[1] = ec.neg(C, P[1])           # P + (-P) -> O
    P[2] = None                      # O + T
    T[3] = None                      # P + O
    P[4], T[4] = None, None          # O + O
    T[5] = ec.dbl(C, P[5])           # P + 2P
    n = len(P)
    p_l, t_l = to_cuda(points_to_limbs(C, P)), to_cuda(points_to_limbs(C, T))
    out = torch.zeros_like(p_l)
    gpu_lib.ecc_point_add_batch(cid, n, p_l, t_l, out)
    torch.cuda.synchronize()
    assert limbs_to_points(C, from_cuda(out)) == [ec.add(C, a, b) for a, b in zip(P, T)]
    gpu_lib.ecc_point_dbl_batch(cid, n, p_l, out)
    torch.cuda.synchronize()
    assert limbs_to_points(C, from_cuda(out)) == [ec.dbl(C, a) for a in P]


@pytest.mark.parametrize("n", [1, 31, 257, 2 * 256 * 152 + 3])
def test_point_add_sizes(gpu_lib, n):
    """Slices spanning many CTAs and a ragged tail (P-256)."""
    import torch

    C = curves.P256
    base, _ = random_points(C, 64, 0x6ECC0400)
    P = [base[i % 64] for i in range(n)]
    T = [base[(7 * i + 3) % 64] for i in range(n)]
    p_l, t_l = to_cuda(points_to_limbs(C, P)), to_cuda(points_to_limbs(C, T))
    out = torch.zeros_like(p_l)
    gpu_lib.ecc_point_add_batch(1, n, p_l, t_l, out)
    torch.cuda.synchronize()
    table = {}
    got = limbs_to_points(C, from_cuda(out))
    for i in range(n):
        key = (i % 64, (7 * i + 3) % 64)
        if key not in table:
            table[key] = ec.add(C, P[i], T[i])
        assert got[i] == table[key], i
