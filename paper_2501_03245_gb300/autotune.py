"""Measured window-width autotuner for MSM size classes.

For every size class floor(log2 n) the tuner times ``ecc_msm`` on seeded
synthetic inputs for the cost model's window width and its neighbours, keeps the
fastest, installs it with ``ecc_msm_set_window`` and can persist the table as
JSON (keyed by GPU name and curve) so a later process reloads it instead of
measuring again.  Inputs are made on the device by the library itself
(``ecc_fixed_base_mul`` for the bases), so tuning needs no CPU arithmetic.
``tune_precomputed`` picks the width of a resident base set's window-multiple
table; ``tune_batch`` tunes, on a caller's ragged batch itself, the knobs its
instances share (a common width shift, the first-level reduction chunk, one
width step per group of classes).
"""
import json
import os

from . import ecc, synth


def _curve_order(curve):
    # group orders of the MSM curves (BN254 r, BLS12-381 r)
    return {
        ecc.ECC_BN254: 0x30644E72E131A029B85045B68181585D2833E84879B9709143E1F593F0000001,
        ecc.ECC_BLS12_381: 0x73EDA753299D7D483339D80809A1D80553BDA402FFFE5BFEFFFFFFFF00000001,
    }[curve]


def make_bases(curve, n, seed, torch):
    """n bases a_i G (a_i seeded, uniform in [1, r-1]) as a device tensor."""
    a = synth.uniform_limbs(seed, synth.S_BASE_MULT, n, _curve_order(curve), lo=1)
    limbs = ecc.ecc_limbs(curve)
    out = torch.empty((n, 2 * limbs), dtype=torch.int32, device="cuda")
    ecc.ecc_fixed_base_mul(curve, n, torch.from_numpy(a.view("int32")).cuda(), out)
    return out


def time_msm(curve, bases, scalars, n, torch, reps=3):
    out = torch.empty((1, 2 * ecc.ecc_limbs(curve)), dtype=torch.int32, device="cuda")
    ecc.ecc_msm(curve, n, bases, scalars, out)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        ecc.ecc_msm(curve, n, bases, scalars, out)
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps / 1e3


def time_msm_bases(curve, bases, scalars, n, vectors, torch, reps=3):
    """Time of one ecc_msm_bases call over `vectors` scalar vectors of n."""
    h = ecc.ecc_bases_create(curve, n, bases)
    try:
        out = torch.empty((vectors, 2 * ecc.ecc_limbs(curve)), dtype=torch.int32, device="cuda")
        ecc.ecc_msm_bases(h, vectors, scalars, out)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            ecc.ecc_msm_bases(h, vectors, scalars, out)
        b.record()
        torch.cuda.synchronize()
    finally:
        ecc.ecc_bases_destroy(h)
    return a.elapsed_time(b) / reps / 1e3


def tune_precomputed(handle, vectors, scalars, torch, candidates, reps=3):
    """Window width for a resident-bases handle with window multiples: builds
    the table for every candidate width, times ecc_msm_bases on `vectors`
    scalar vectors, and leaves the handle with the fastest.  Returns (c, times)
    with times[c] = (table build s, call s)."""
    import time

    times = {}
    for c in candidates:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ecc.ecc_bases_precompute(handle, c)
        build = time.perf_counter() - t0
        out = torch.empty((vectors, 24), dtype=torch.int32, device="cuda")  # 2 x 12 limbs covers every curve
        ecc.ecc_msm_bases(handle, vectors, scalars, out)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            ecc.ecc_msm_bases(handle, vectors, scalars, out)
        b.record()
        torch.cuda.synchronize()
        times[c] = (build, a.elapsed_time(b) / reps / 1e3)
    best = min(times, key=lambda c: times[c][1])
    ecc.ecc_bases_precompute(handle, best)
    return best, times


def tune(curve, log2_sizes, torch, spread=2, seed=0x6ECC7777, cache=None, vectors=1):
    """Returns {log2_n: c} and installs it in the library.  With vectors > 1
    every candidate is timed on the resident-bases form with that many scalar
    vectors per call (the best window grows with the vectors sharing a call)."""
    key = None
    table = {}
    if cache and os.path.exists(cache):
        key = f"{torch.cuda.get_device_name()}|{curve}|{vectors}"
        saved = json.load(open(cache)).get(key, {})
        table = {int(k): int(v) for k, v in saved.items()}
    missing = [l for l in log2_sizes if l not in table]
    if missing:
        n_max = 1 << max(missing)
        bases = make_bases(curve, n_max, seed, torch)
        ks = synth.uniform_limbs(seed, synth.S_SCALAR, n_max * vectors, _curve_order(curve))
        scalars = torch.from_numpy(ks.view("int32")).cuda()
        for l in missing:
            n = 1 << l
            ecc.ecc_msm_set_window(curve, l, 0)
            c0 = ecc.ecc_msm_window(curve, n)
            best = None
            for c in range(max(2, c0 - spread), min(20, c0 + spread) + 1):
                ecc.ecc_msm_set_window(curve, l, c)
                if vectors > 1:
                    t = time_msm_bases(curve, bases, scalars[:n * vectors].contiguous(), n, vectors, torch)
                else:
                    t = time_msm(curve, bases, scalars, n, torch)
                if best is None or t < best[0]:
                    best = (t, c)
            table[l] = best[1]
    for l, c in table.items():
        ecc.ecc_msm_set_window(curve, l, c)
    if cache:
        key = key or f"{torch.cuda.get_device_name()}|{curve}|{vectors}"
        data = json.load(open(cache)) if os.path.exists(cache) else {}
        data[key] = {str(k): v for k, v in sorted(table.items())}
        with open(cache, "w") as f:
            json.dump(data, f, indent=1)
    return table


def tune_batch(curve, log2_sizes, run, torch, shifts=(-1, 0, 1), chunks=(3, 4, 5), reps=3, min_gain=0.005):
    """Tunes the knobs that one ragged launch sequence shares across its
    instances on the batch itself: run() makes the caller's ecc_msm_ragged call.

    The first-level reduction of all instances runs in one launch whose round
    count is set by the largest chunk in it, so a per-class chunk choice made
    on batches of one size does not transfer to a mix; likewise the window
    widths of the classes interact through the shared launches.  So, starting
    from the per-class widths already installed (tune), every width is shifted
    by the same s (each in [2, 20]) for each s in shifts, then one chunk 2^k
    (capped at c - 1 per class) is set for every class for each k in chunks;
    each candidate is timed as reps calls of run(), the fastest is installed.
    Last, each group of classes that share a width tries that width - 1 and
    + 1 on the batch (the others fixed); a change stays when it is faster by
    more than min_gain.  Returns {"shift": s, "chunk_log2": k, "widths":
    {log2_n: c}, "ms": {...}}."""
    base = {l: ecc.ecc_msm_window(curve, 1 << l) for l in log2_sizes}

    def timed():
        run()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            run()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    def set_shift(s):
        for l, c in base.items():
            ecc.ecc_msm_set_window(curve, l, min(20, max(2, c + s)))

    def set_chunk(k):
        for l in log2_sizes:
            c = ecc.ecc_msm_window(curve, 1 << l)
            ecc.ecc_msm_set_reduce_chunk(curve, l, max(1, min(k, c - 1)))

    ms = {}
    set_chunk(chunks[len(chunks) // 2])
    for s in shifts:
        set_shift(s)
        ms[f"shift {s}"] = timed()
    shift = min(shifts, key=lambda s: ms[f"shift {s}"])
    set_shift(shift)
    for k in chunks:
        set_chunk(k)
        ms[f"chunk {k}"] = timed()
    chunk = min(chunks, key=lambda k: ms[f"chunk {k}"])
    set_chunk(chunk)
    best = ms[f"chunk {chunk}"]
    groups = {}
    for l in log2_sizes:
        groups.setdefault(ecc.ecc_msm_window(curve, 1 << l), []).append(l)
    for c, ls in sorted(groups.items()):
        for cc in (c - 1, c + 1):
            if not 2 <= cc <= 20:
                continue
            for l in ls:
                ecc.ecc_msm_set_window(curve, l, cc)
            set_chunk(chunk)
            t = timed()
            ms[f"width {c} -> {cc}"] = t
            if t < best * (1 - min_gain):
                best = t
                break
            for l in ls:
                ecc.ecc_msm_set_window(curve, l, c)
            set_chunk(chunk)
    widths = {l: ecc.ecc_msm_window(curve, 1 << l) for l in log2_sizes}
    return {"shift": shift, "chunk_log2": chunk, "widths": widths,
            "ms": {k: round(v, 3) for k, v in ms.items()}}
