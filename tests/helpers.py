"""Shared test helpers: oracle-side input construction and limb conversions."""
import numpy as np

from oracle import curves, ec
from paper_2501_03245_gb300 import synth


def points_to_limbs(C, pts):
    """List of oracle points (None = O) -> (n, 2m) uint32 limbs, O as (0, 0)."""
    m = C.limbs
    enc = [ec.encode(P) for P in pts]
    return np.concatenate([synth.ints_to_limbs([p[0] for p in enc], m),
                           synth.ints_to_limbs([p[1] for p in enc], m)], axis=1)


def limbs_to_points(C, arr):
    m = C.limbs
    out = []
    for row in np.asarray(arr):
        out.append(ec.decode((synth.limbs_to_int(row[:m]), synth.limbs_to_int(row[m:]))))
    return out


def random_points(C, count, seed):
    """count oracle points k_i G with seeded k_i (via the C++ oracle for speed)."""
    from oracle import cpp_oracle

    cid = [k for k, v in curves.BY_ID.items() if v is C][0]
    a, _ = synth.msm_raw(seed, count, C.n, 0)
    G = np.tile(points_to_limbs(C, [C.G]), (count, 1))
    out = cpp_oracle.scalar_mul(cid, a, G)
    return limbs_to_points(C, out), synth.limbs_to_ints(a)


def to_cuda(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def from_cuda(t):
    return t.cpu().numpy()
