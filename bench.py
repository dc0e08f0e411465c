#!/usr/bin/env python3
"""Benchmark: batched ECDSA verification on NIST P-256 (2^20 seeded triples,
1/16 corrupted) on GB300, one JSON line on stdout.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one batched verification of the whole 2^20-triple workload with the
inputs resident in HBM.  `value` is verifies/s over the timed steps (whole job:
the units all ranks processed / max time over ranks).  With N > 1 each rank
verifies its own independent 2^20-triple batch (weak scaling, no collective on
the data path).  Extra keys: roofline (dominant kernel against the measured
IMAD-pipe rate), e2e (same metric through the C ABI with host buffers, copies
inside the timed region), plain (one verification per launch), clocks,
cpu_baseline (the plain C++ oracle on the host cores, a bounded sample), msm
(BLS12-381, 2^20 resident bases x 16 scalar vectors), ragged (256 BN254 MSMs
in one captured launch sequence) and sm2 (the same verification workload on
the paper's SM2 curve, beside the paper's own A100 figure).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ECDSA verifies/sec and MSM points/sec on 1 GB300, batched vs plain, bit-exact"
N_VERIFY = 1 << 20
CURVE_P256 = 1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=N_VERIFY, help="triples per rank (default 2^20)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-msm", action="store_true", help="skip the MSM and ragged-MSM lines")
    ap.add_argument("--no-ragged", action="store_true", help="skip the ragged-MSM line")
    ap.add_argument("--no-table-msm", action="store_true",
                    help="skip the BLS12-381 resident-bases MSM line (keep the ragged line)")
    ap.add_argument("--no-sm2", action="store_true", help="skip the SM2 verification line")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the secp256k1 4096-triple and the SM2 signing / FPMUL lines")
    ap.add_argument("--msm-n", type=int, default=1 << 20, help="BLS12-381 MSM bases (default 2^20)")
    ap.add_argument("--msm-vectors", type=int, default=16, help="scalar vectors per MSM step")
    return ap.parse_args()


def max_over_ranks(x):
    """The largest of every rank's x (x itself when not distributed).  The
    tensor lives where the process group's backend expects it."""
    import torch

    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return float(x)
    dev = "cuda" if torch.distributed.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, seconds, world):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (weak scaling: every rank does the same units)."""
    return units_per_rank * world / max_over_ranks(seconds)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _nvtx(name):
    """Each line's timed region is an NVTX range named after the line (ncu
    --nvtx --nvtx-include "<name>/" profiles only launches inside it)."""
    try:
        import torch

        if name is None:
            torch.cuda.nvtx.range_pop()
        else:
            torch.cuda.nvtx.range_push(name)
    except Exception:
        pass


class ClockSampler:
    """SM clocks and throttle reasons during timed regions: one background
    `nvidia-smi -lms 200` for the whole run (started once, before the first
    timed region); each line's timed region is a named window, and a window's
    summary keeps only the samples stamped inside it."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.windows = {}
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(1.0)

    def begin(self, name):
        self.windows[name] = [time.time(), None]
        _nvtx(name)

    def end(self, name):
        self.windows[name][1] = time.time()
        _nvtx(None)

    def stop(self):
        time.sleep(0.3)
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=10)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in (out or "").splitlines() if l.strip()]

    def summary(self, name):
        import datetime

        t0, t1 = self.windows.get(name, (None, None))
        rows = []
        for line in self.lines:
            c = [x.strip() for x in line.split(",")]
            if len(c) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(c[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                continue
            if t0 is not None and t1 is not None and not (t0 - 0.25 <= ts <= t1 + 0.25):
                continue
            rows.append(c)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        num = lambda v: float(v) if v.replace(".", "", 1).isdigit() else None  # noqa: E731
        sm = [num(r[2]) for r in rows if num(r[2]) is not None]
        smax = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


class _NoClock:
    def begin(self, name):
        _nvtx(name)

    def end(self, name):
        _nvtx(None)

    def summary(self, name):
        return None


def hbm_peak():
    """Measured copy bandwidth (GB/s) of the GB300s, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


ORDERS = {1: 0xFFFFFFFF00000000FFFFFFFFFFFFFFFFBCE6FAADA7179E84F3B9CAC2FC632551,   # P-256 n
          4: 0xFFFFFFFEFFFFFFFFFFFFFFFFFFFFFFFF7203DF6B21C6052B53BBF40939D54123}   # SM2 n


def gen_inputs(ecc, synth, torch, n, seed, curve=CURVE_P256):
    import numpy as np

    raw = synth.ecdsa_raw(seed, n, ORDERS[curve], 16)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    d, e, k = dev(raw["d"]), dev(raw["e"]), dev(raw["k"])
    r = torch.empty((n, 32), dtype=torch.uint8, device="cuda")
    s = torch.empty_like(r)
    pub = torch.empty((n, 64), dtype=torch.uint8, device="cuda")
    ecc.ecc_sign_batch(curve, n, d, e, k, r, s, pub)
    torch.cuda.synchronize()
    r_h, s_h = r.cpu().numpy(), s.cpu().numpy()
    r_h, s_h = synth.apply_corruption(r_h, s_h, raw["corrupt_idx"], raw["corrupt_kind"], raw["corrupt_bit"])
    return e, dev(r_h), dev(s_h), pub


# DRAM traffic of one k_verify launch over 2^20 P-256 triples (dram__bytes_read.sum +
# dram__bytes_write.sum, from one ncu capture), valid only for the kernel sources
# it was taken on: the digest of those sources must match, else it is null.
VERIFY_TRAFFIC = {"bytes": 79369814528 + 33884342528, "batch": 1 << 20, "digest": "d56ffe9d83e1591f",
                  "sources": ["verify.cuh", "verify_host.cuh", "ops.cuh", "ec.cuh", "fp.cuh", "inv.cuh",
                              "ptx.cuh", "curves_gen.cuh", "internal.h", "k_verify_p256_c2.cu", "k_verify.cu"]}


def verify_traffic(n):
    import hashlib

    h = hashlib.sha256()
    for f in VERIFY_TRAFFIC["sources"]:
        with open(os.path.join(ROOT, "paper_2501_03245_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest()[:16] != VERIFY_TRAFFIC["digest"] or n != VERIFY_TRAFFIC["batch"]:
        return None
    return VERIFY_TRAFFIC["bytes"]


def imad_peak(ecc, torch, sms):
    """Measured wide multiply-add rate (pairs/s) of the integer pipe."""
    threads = sms * 2048
    sink = torch.zeros(threads, dtype=torch.int32, device="cuda")
    iters = 4096
    ecc.ecc_bench_imad(threads, 64, sink)
    torch.cuda.synchronize()
    best = 0.0
    for _ in range(3):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ecc.ecc_bench_imad(threads, iters, sink)
        b.record()
        torch.cuda.synchronize()
        best = max(best, threads * iters * 8 / (a.elapsed_time(b) / 1e3))
    return best


def cpu_baseline_verify(e, r, s, pub, sample):
    """The C++ oracle on the host cores over a bounded sample of the workload."""
    from oracle import cpp_oracle

    cpp_oracle.load()
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    cpp_oracle.verify(CURVE_P256, e[:sample], r[:sample], s[:sample], pub[:sample], threads=threads)
    dt = time.perf_counter() - t0
    one = max(1, sample // 16)  # the same oracle on one core, a 16th of the sample
    t1 = time.perf_counter()
    cpp_oracle.verify(CURVE_P256, e[:one], r[:one], s[:one], pub[:one], threads=1)
    dt1 = time.perf_counter() - t1
    return {"value": sample / dt, "unit": "verifies/s", "cores": threads, "kind": "oracle",
            "sample": f"first {sample} of the 2^20 P-256 triples, plain C++ bigint oracle "
                      f"(Barrett + Jacobian), {threads} threads, {dt:.2f} s",
            "single_core": {"value": one / dt1, "unit": "verifies/s",
                            "sample": f"first {one} triples, 1 thread, {dt1:.2f} s"}}


BLS_R = 0x73EDA753299D7D483339D80809A1D80553BDA402FFFE5BFEFFFFFFFF00000001
BN_R = 0x30644E72E131A029B85045B68181585D2833E84879B9709143E1F593F0000001


def _event_time(torch, fn, reps):
    """Mean device seconds per call of fn over reps back-to-back calls."""
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3 / reps


def _phases(ecc, torch, fn):
    """Per-phase device milliseconds of one MSM call (library phase timers)."""
    ecc.ecc_set_phase_timing(1)
    try:
        fn()
        torch.cuda.synchronize()
        return ecc.ecc_msm_phase_times()
    finally:
        ecc.ecc_set_phase_timing(0)


def _sort_line(phases, points, digits):
    """Achieved HBM rate of the counting sort (histogram + scatter): its
    algorithmic bytes are two reads of every 32-byte scalar and, per (point,
    window) digit, one 4-byte histogram update and one 4-byte entry write."""
    peak, kind = hbm_peak()
    b = 64 * points + 8 * digits
    ms = phases.get("sort")
    if not ms:
        return None
    gbs = b / (ms / 1e3) / 1e9
    return {"ms": ms, "bytes": b, "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
            "peak_kind": kind}


def bench_msm(ecc, costmodel, synth, torch, peak, rank, n=1 << 20, V=16, world=1, clk=None, reps=10):
    """BLS12-381 MSM: n resident bases a_i G (2^20 by default), V scalar vectors
    per step (16 by default; one ecc_msm_bases call), against the plain form (one
    MSM launch sequence per vector).  The bases are reused across calls, so they
    carry their window multiples 2^(c w) P_i (built once, like the verifier's
    fixed-base table); c is tuned over candidate widths on this call's shape.
    The same handle without the table (window width from the size-class tuner)
    is reported beside it."""
    from paper_2501_03245_gb300 import autotune

    curve = ecc.ECC_BLS12_381
    log2n = n.bit_length() - 1
    tuned = autotune.tune(curve, [log2n], torch, vectors=V)
    seed = synth.SEED_BASE + 2 + 1000 * rank
    a, ks = synth.msm_raw(seed, n, BLS_R, V)
    pts = torch.empty((n, 24), dtype=torch.int32, device="cuda")
    ecc.ecc_fixed_base_mul(curve, n, torch.from_numpy(a.view("int32")).cuda(), pts)
    sc = torch.from_numpy(np.concatenate(ks).view("int32")).cuda()
    h = ecc.ecc_bases_create(curve, n, pts)
    out = torch.empty((V, 24), dtype=torch.int32, device="cuda")
    try:
        clk = clk or _NoClock()
        ecc.ecc_msm_bases(h, V, sc, out)
        t_tab = _event_time(torch, lambda: ecc.ecc_msm_bases(h, V, sc, out), 3)
        ref = out.clone()
        c, sweep = autotune.tune_precomputed(h, V, sc, torch, range(14, 23))
        ecc.ecc_msm_bases(h, V, sc, out)
        clk.begin("msm")
        t = _event_time(torch, lambda: ecc.ecc_msm_bases(h, V, sc, out), reps)
        clk.end("msm")
        same = bool(torch.equal(out, ref))
        phases = _phases(ecc, torch, lambda: ecc.ecc_msm_bases(h, V, sc, out))
        one = out[:1]
        t1 = _event_time(torch, lambda: [ecc.ecc_msm_bases(h, 1, sc[v * n:(v + 1) * n], one)
                                         for v in range(V)], 1)
    finally:
        ecc.ecc_bases_destroy(h)
    W = costmodel.msm_windows(255, c)
    alg = costmodel.msm_modmul_precomputed(n, W, c) * V * costmodel.imad_per_modmul(12)
    c_tab = ecc.ecc_msm_window(curve, n)
    W_tab = costmodel.msm_windows(255, c_tab)
    alg_tab = costmodel.msm_modmul(n, W_tab, c_tab) * V * costmodel.imad_per_modmul(12)
    shape = f"2^{log2n}" if n & (n - 1) == 0 else str(n)
    return {"workload": f"MSM BLS12-381 G1, {shape} resident bases, {V} scalar vectors per step",
            "value": job_rate(n * V, t, world), "unit": "points/s", "ms_per_step": t * 1e3, "window_c": c,
            "timed_calls": reps, "clocks": clk.summary("msm"),
            "phases_ms": phases, "sort": _sort_line(phases, n * V, n * V * W),
            "form": "resident bases with window multiples 2^(c w) P_i, one bucket set",
            "table": {"build_ms": sweep[c][0] * 1e3, "bytes": W * n * 96,
                      "sweep_ms": {str(k): round(v[1] * 1e3, 2) for k, v in sweep.items()}},
            "bit_equal_to_no_table": same,
            "no_table": {"value": job_rate(n * V, t_tab, world), "ms_per_step": t_tab * 1e3, "window_c": c_tab,
                         "autotuned": {str(k): v for k, v in tuned.items()},
                         "frac": alg_tab / t_tab / peak},
            "plain": {"value": job_rate(n * V, t1, world), "unit": "points/s",
                      "form": "one MSM launch sequence per scalar vector (same table)"},
            "roofline": {"bound": "alu", "achieved": alg / t / 1e12, "peak": peak / 1e12,
                         "unit": "T IMAD.WIDE/s", "frac": alg / t / peak,
                         "basis": "6 modmul per (point, window) digit + 2 PADD per bucket of the "
                                  "single bucket set, 300 wide mul-adds per modmul"}}


# The paper's verification throughput on its own curve (Table 4: SM2, NVIDIA
# A100 40 GB, batch size not stated), quoted for context beside the same
# workload here.
PAPER_SM2_VERIFY_A100 = 4372853.0


def bench_sm2(ecc, costmodel, synth, torch, peak, rank, n, steps, world=1, clk=None):
    """ECDSA verification on the SM2 curve, the paper's curve: 2^20 triples with
    the same recipe as the P-256 line (1/16 corrupted), inputs resident.  The
    schedule and the limb count are the P-256 kernel's, so is the work basis."""
    curve = ecc.ECC_SM2
    e, r, s, pub = gen_inputs(ecc, synth, torch, n, synth.SEED_BASE + 5 + 1000 * rank, curve)
    ok = torch.zeros(n, dtype=torch.uint8, device="cuda")
    clk = clk or _NoClock()
    for _ in range(3):
        ecc.ecc_verify_batch(curve, n, e, r, s, pub, ok)
    clk.begin("sm2")
    t = _event_time(torch, lambda: ecc.ecc_verify_batch(curve, n, e, r, s, pub, ok), max(steps, 5))
    clk.end("sm2")
    value = job_rate(n, t, world)
    alg = costmodel.verify_imad() * n
    return {"workload": "ECDSA verify, SM2, 2^20 seeded triples, 1/16 corrupted", "value": value,
            "unit": "verifies/s", "ms_per_step": t * 1e3, "valid_signatures": int(ok.sum().item()),
            "timed_calls": max(steps, 5), "clocks": clk.summary("sm2"),
            "paper": {"value": PAPER_SM2_VERIFY_A100, "hardware": "NVIDIA A100 40 GB",
                      "source": "Table 4"},
            "ratio_to_paper": value / world / PAPER_SM2_VERIFY_A100,
            "roofline": {"bound": "alu", "kernel": "k_verify<SM2>", "achieved": alg / t / 1e12,
                         "peak": peak / 1e12, "unit": "T IMAD.WIDE/s", "frac": alg / t / peak}}


def bench_ragged(ecc, costmodel, synth, torch, peak, rank, world=1, clk=None, reps=10):
    """BN254 ragged batch: 256 MSMs with log-uniform sizes 2^10..2^18, all in one
    launch sequence captured once in a CUDA graph and replayed, against one
    launch sequence per MSM.  Window widths are autotuned per size class, then
    a common width shift and the reduction's bucket layout on this batch.  The
    algorithmic work is the sum of every instance's Pippenger count at the
    window width the library picks for its size."""
    from paper_2501_03245_gb300 import autotune

    clk = clk or _NoClock()
    curve = ecc.ECC_BN254
    classes = list(range(10, 19))
    tuned = autotune.tune(curve, classes, torch)  # one window width per size class
    seed = synth.SEED_BASE + 3 + 1000 * rank
    sizes = synth.ragged_sizes(seed, 256)
    total = int(sizes.sum())
    a, ks = synth.msm_raw(seed, total, BN_R, 1)
    pts = torch.empty((total, 16), dtype=torch.int32, device="cuda")
    ecc.ecc_fixed_base_mul(curve, total, torch.from_numpy(a.view("int32")).cuda(), pts)
    sc = torch.from_numpy(ks[0].view("int32")).cuda()
    offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.uint64)
    out = torch.empty((256, 16), dtype=torch.int32, device="cuda")
    # the knobs the instances share (a common width shift, the reduction
    # chunk) tuned on this batch, untimed
    layout = autotune.tune_batch(curve, classes, lambda: ecc.ecc_msm_ragged(curve, 256, offs, pts, sc, out), torch)
    ecc.ecc_msm_ragged(curve, 256, offs, pts, sc, out)
    torch.cuda.synchronize()
    ref = out.clone()
    clk.begin("ragged")
    eager = _event_time(torch, lambda: ecc.ecc_msm_ragged(curve, 256, offs, pts, sc, out), reps)
    graph = None
    try:
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            ecc.ecc_msm_ragged(curve, 256, offs, pts, sc, out, s)  # warm inside the side stream
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            ecc.ecc_msm_ragged(curve, 256, offs, pts, sc, out, s)
        out.zero_()
        graph = _event_time(torch, g.replay, reps)
        graph_ok = bool(torch.equal(out, ref))
    except Exception as ex:  # report, keep the eager number
        graph_ok = f"capture failed: {ex}"
    clk.end("ragged")
    phases = _phases(ecc, torch, lambda: ecc.ecc_msm_ragged(curve, 256, offs, pts, sc, out))
    one = torch.empty((1, 16), dtype=torch.int32, device="cuda")
    per = _event_time(torch, lambda: [ecc.ecc_msm(curve, int(sizes[i]), pts[int(offs[i]):int(offs[i + 1])],
                                                  sc[int(offs[i]):int(offs[i + 1])], one)
                                      for i in range(256)], 1)
    # the faster of the two forms; the graph's only when its replay reproduced
    # the eager result
    best = graph if (graph and graph_ok is True and graph <= eager) else eager
    widths = [ecc.ecc_msm_window(curve, int(k)) for k in sizes]
    alg = sum(costmodel.msm_modmul(int(k), costmodel.msm_windows(254, c), c) for k, c in zip(sizes, widths))
    alg *= costmodel.imad_per_modmul(8)
    digits = sum(int(k) * costmodel.msm_windows(254, c) for k, c in zip(sizes, widths))
    return {"workload": "256 BN254 MSMs, sizes log-uniform 2^10..2^18, one launch sequence",
            "points": total, "value": job_rate(total, best, world), "unit": "points/s",
            "form": "graph replay" if best is graph else "eager",
            "graph_replay_ms": graph * 1e3 if graph else None, "eager_ms": eager * 1e3,
            "graph_bit_equal": graph_ok, "timed_calls": reps, "clocks": clk.summary("ragged"),
            "autotuned": {"c": {str(k): ecc.ecc_msm_window(curve, 1 << k) for k in sorted(tuned)},
                          "batch": layout},
            "phases_ms": phases, "sort": _sort_line(phases, total, digits),
            "plain": {"value": job_rate(total, per, world), "unit": "points/s",
                      "form": "one launch sequence per MSM", "frac": alg / per / peak},
            "roofline": {"bound": "alu", "achieved": alg / best / 1e12, "peak": peak / 1e12,
                         "unit": "T IMAD.WIDE/s", "frac": alg / best / peak,
                         "basis": "per instance: 6 modmul per (point, window) digit + 2 PADD per bucket "
                                  "+ c PDBL and 1 PADD per window, 136 wide mul-adds per modmul"}}


SECP256K1_N = 0xFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFEBAAEDCE6AF48A03BBFD25E8CD0364141


def bench_k1(ecc, costmodel, synth, torch, peak, rank, world=1, clk=None, reps=20, plain_n=64):
    """ECDSA verification on secp256k1, 4096 triples (1/8 corrupted, the small
    workload), batched (one launch for all 4096) against the plain form (one
    triple per launch, timed on the first plain_n triples)."""
    clk = clk or _NoClock()
    curve, n = ecc.ECC_SECP256K1, 4096
    raw = synth.ecdsa_raw(synth.SEED_BASE + 1000 * rank, n, SECP256K1_N, 8)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    d, e, k = dev(raw["d"]), dev(raw["e"]), dev(raw["k"])
    r = torch.empty((n, 32), dtype=torch.uint8, device="cuda")
    s = torch.empty_like(r)
    pub = torch.empty((n, 64), dtype=torch.uint8, device="cuda")
    ecc.ecc_sign_batch(curve, n, d, e, k, r, s, pub)
    torch.cuda.synchronize()
    r_h, s_h = synth.apply_corruption(r.cpu().numpy(), s.cpu().numpy(), raw["corrupt_idx"],
                                      raw["corrupt_kind"], raw["corrupt_bit"])
    r, s = dev(r_h), dev(s_h)
    ok = torch.zeros(n, dtype=torch.uint8, device="cuda")
    for _ in range(3):
        ecc.ecc_verify_batch(curve, n, e, r, s, pub, ok)
    clk.begin("secp256k1")
    t = _event_time(torch, lambda: ecc.ecc_verify_batch(curve, n, e, r, s, pub, ok), reps)
    clk.end("secp256k1")
    ok1 = torch.zeros(1, dtype=torch.uint8, device="cuda")
    t1 = _event_time(torch, lambda: [ecc.ecc_verify_batch(curve, 1, e[i:i + 1], r[i:i + 1], s[i:i + 1],
                                                          pub[i:i + 1], ok1) for i in range(plain_n)], 1)
    alg = costmodel.verify_imad() * n
    return {"workload": "ECDSA verify, secp256k1, 4096 seeded triples, 1/8 corrupted",
            "value": job_rate(n, t, world), "unit": "verifies/s", "ms_per_step": t * 1e3,
            "timed_calls": reps, "valid_signatures": int(ok.sum().item()), "clocks": clk.summary("secp256k1"),
            "plain": {"value": job_rate(plain_n, t1, world), "unit": "verifies/s",
                      "form": f"one triple per launch, first {plain_n} triples"},
            "roofline": {"bound": "alu", "kernel": "k_verify<Secp256k1>", "achieved": alg / t / 1e12,
                         "peak": peak / 1e12, "unit": "T IMAD.WIDE/s", "frac": alg / t / peak,
                         "note": "4096 triples fill 16 of 304 resident CTAs: latency, not the pipe, "
                                 "bounds this size"}}


# The paper's ECDSA signing and fixed-point multiplication throughputs on its
# own curve (SM2, NVIDIA A100 40 GB): Table 4 (signing) and Table 5 (FPMUL at
# 2^11 and 2^14 operations per SP, 432 SPs), quoted for context.
PAPER_SM2_SIGN_A100 = 14141978.0
PAPER_SM2_FPMUL_A100 = {"2^11 per SP": 11723016.0, "2^14 per SP": 14389168.0}


def bench_sign_fpmul(ecc, costmodel, synth, torch, peak, rank, n, world=1, clk=None, reps=5):
    """Batched ECDSA signing and FPMUL k G on SM2 (the paper's curve), 2^20
    items each, inputs resident; the fixed-base table is built before timing."""
    clk = clk or _NoClock()
    curve = ecc.ECC_SM2
    raw = synth.ecdsa_raw(synth.SEED_BASE + 6 + 1000 * rank, n, ORDERS[curve], 16)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    d, e, k = dev(raw["d"]), dev(raw["e"]), dev(raw["k"])
    r = torch.empty((n, 32), dtype=torch.uint8, device="cuda")
    s = torch.empty_like(r)
    pub = torch.empty((n, 64), dtype=torch.uint8, device="cuda")
    kl = dev(synth.uniform_limbs(synth.SEED_BASE + 7 + 1000 * rank, 1, n, ORDERS[curve]).view(np.int32))
    pts = torch.empty((n, 16), dtype=torch.int32, device="cuda")
    for _ in range(3):
        ecc.ecc_sign_batch(curve, n, d, e, k, r, s, pub)
        ecc.ecc_fixed_base_mul(curve, n, kl, pts)
    clk.begin("sign_fpmul")
    t_sign = _event_time(torch, lambda: ecc.ecc_sign_batch(curve, n, d, e, k, r, s, pub), reps)
    t_fp = _event_time(torch, lambda: ecc.ecc_fixed_base_mul(curve, n, kl, pts), reps)
    clk.end("sign_fpmul")
    m8 = costmodel.imad_per_modmul(8)
    a_sign = costmodel.sign_modmul() * m8 * n
    a_fp = costmodel.fpmul_modmul() * m8 * n
    shape = "2^20" if n == 1 << 20 else str(n)
    return {"workload": f"ECDSA sign and FPMUL, SM2, {shape} items each", "timed_calls": reps,
            "clocks": clk.summary("sign_fpmul"),
            "sign": {"value": job_rate(n, t_sign, world), "unit": "signs/s", "ms_per_step": t_sign * 1e3,
                     "paper": {"value": PAPER_SM2_SIGN_A100, "hardware": "NVIDIA A100 40 GB",
                               "source": "Table 4"},
                     "roofline": {"bound": "alu", "kernel": "k_fixed_base<SM2> (signing mode)", "achieved": a_sign / t_sign / 1e12,
                                  "peak": peak / 1e12, "unit": "T IMAD.WIDE/s", "frac": a_sign / t_sign / peak}},
            "fpmul": {"value": job_rate(n, t_fp, world), "unit": "kG/s", "ms_per_step": t_fp * 1e3,
                      "paper": {"value": PAPER_SM2_FPMUL_A100, "hardware": "NVIDIA A100 40 GB",
                                "source": "Table 5"},
                      "roofline": {"bound": "alu", "kernel": "k_fixed_base<SM2> (FPMUL mode)", "achieved": a_fp / t_fp / 1e12,
                                   "peak": peak / 1e12, "unit": "T IMAD.WIDE/s", "frac": a_fp / t_fp / peak}}}


def verify_config(n):
    """The verification workload's config, shared by both arms."""
    shape = "2^20" if n == N_VERIFY else str(n)
    return {"workload": f"ECDSA verify, NIST P-256, {shape} seeded triples per GPU, 1/16 corrupted",
            "curve": "P-256", "batch": n, "l2": "working set > L2 (inputs 160 MiB + "
            "per-item state ~0.8 GiB per step)"}


def run_reference(args):
    """--impl reference: the oracle as it stands on the host cores, on the same
    workload (bounded samples per step); rank 0 only."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import cpp_oracle
    from paper_2501_03245_gb300 import synth

    cpp_oracle.load()
    order = 0xFFFFFFFF00000000FFFFFFFFFFFFFFFFBCE6FAADA7179E84F3B9CAC2FC632551
    sample = 4096
    raw = synth.ecdsa_raw(synth.SEED_BASE + 1, sample, order, 16)
    r, s, pub = cpp_oracle.sign(CURVE_P256, raw["d"], raw["e"], raw["k"])
    r, s = synth.apply_corruption(r, s, raw["corrupt_idx"], raw["corrupt_kind"], raw["corrupt_bit"])
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        cpp_oracle.verify(CURVE_P256, raw["e"][:256], r[:256], s[:256], pub[:256], threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cpp_oracle.verify(CURVE_P256, raw["e"], r, s, pub, threads=threads)
    dt = time.perf_counter() - t0
    value = sample * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "verifies/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": verify_config(N_VERIFY),
        "cpu_baseline": {"value": value, "unit": "verifies/s", "cores": threads, "kind": "oracle",
                         "sample": f"{sample} triples per step by the workload's recipe (seed "
                                   f"{synth.SEED_BASE + 1:#x}, 1/16 corrupted), plain C++ bigint "
                                   f"oracle (Barrett + Jacobian), {threads} threads"},
        "e2e": {"value": value, "unit": "verifies/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    from paper_2501_03245_gb300 import build as pkg_build
    from paper_2501_03245_gb300 import costmodel, ecc, synth

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pkg_build.build()
    ecc.load()
    n = args.n
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    e, r, s, pub = gen_inputs(ecc, synth, torch, n, synth.SEED_BASE + 1 + 1000 * rank)
    ok = torch.zeros(n, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        ecc.ecc_verify_batch(CURVE_P256, n, e, r, s, pub, ok, stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    n_valid = int(ok.sum().item())

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    events = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
    clk = ClockSampler(local)
    clk.start()
    barrier()
    clk.begin("verify")
    t_all0 = torch.cuda.Event(enable_timing=True)
    t_all1 = torch.cuda.Event(enable_timing=True)
    t_all0.record(stream)
    for a, b in events:
        a.record(stream)
        step()
        b.record(stream)
    t_all1.record(stream)
    barrier()
    clk.end("verify")
    total_s = t_all0.elapsed_time(t_all1) / 1e3
    per_launch = [a.elapsed_time(b) / 1e3 for a, b in events]
    value = job_rate(n * args.steps, total_s, world)
    total_s = max_over_ranks(total_s)

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    e_h = e.cpu().pin_memory()
    r_h = r.cpu().pin_memory()
    s_h = s.cpu().pin_memory()
    p_h = pub.cpu().pin_memory()
    ok_h = torch.zeros(n, dtype=torch.uint8).pin_memory()
    ecc.ecc_verify_batch(CURVE_P256, n, e_h, r_h, s_h, p_h, ok_h, stream)
    barrier()
    e2e_steps = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ecc.ecc_verify_batch(CURVE_P256, n, e_h, r_h, s_h, p_h, ok_h, stream)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_value = job_rate(n * e2e_steps, e2e_s, world)
    e2e_ok = bool(torch.equal(ok_h, ok.cpu()))

    # plain form: one verification per launch
    plain_n = 64
    ok1 = torch.zeros(1, dtype=torch.uint8, device="cuda")
    ecc.ecc_verify_batch(CURVE_P256, 1, e[:1], r[:1], s[:1], pub[:1], ok1, stream)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for i in range(plain_n):
        ecc.ecc_verify_batch(CURVE_P256, 1, e[i:i + 1], r[i:i + 1], s[i:i + 1], pub[i:i + 1],
                             ok1, stream)
    b.record(stream)
    torch.cuda.synchronize()
    plain = plain_n / (a.elapsed_time(b) / 1e3)

    cpu_baseline = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_baseline = cpu_baseline_verify(e.cpu().numpy(), r.cpu().numpy(), s.cpu().numpy(),
                                           pub.cpu().numpy(), 16384)
    peak = imad_peak(ecc, torch, sms)
    alg = costmodel.verify_imad() * n
    launch_s = statistics.median(per_launch)
    achieved = alg / launch_s
    line = {
        "metric": METRIC, "value": value, "unit": "verifies/s", "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": total_s / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": verify_config(n), "valid_signatures": n_valid,
        "roofline": {"bound": "alu", "kernel": "k_verify<P256, 256, 2>", "achieved": achieved / 1e12,
                     "peak": peak / 1e12, "unit": "T IMAD.WIDE/s", "frac": achieved / peak,
                     "traffic": verify_traffic(n), "traffic_unit": "DRAM bytes per launch",
                     "basis": f"{costmodel.verify_modmul()} modmul x 136 wide mul-adds per verify; "
                              "peak = measured mad.lo/madc.hi pair rate (ecc_bench_imad, same run)"},
        "plain": {"value": plain, "unit": "verifies/s", "form": "one verification per launch"},
        "e2e": {"value": e2e_value, "unit": "verifies/s",
                "h2d_bytes_per_step": 160 * n, "d2h_bytes_per_step": n, "bit_equal": e2e_ok},
        "gpu_launches": args.steps,
    }
    del e, r, s, pub, ok, e_h, r_h, s_h, p_h, ok_h
    if not args.no_msm:
        if not args.no_table_msm:
            line["msm"] = bench_msm(ecc, costmodel, synth, torch, peak, rank, args.msm_n, args.msm_vectors,
                                    world, clk)
        if not args.no_ragged:
            line["ragged"] = bench_ragged(ecc, costmodel, synth, torch, peak, rank, world, clk)
    if not args.no_sm2:
        line["sm2"] = bench_sm2(ecc, costmodel, synth, torch, peak, rank, n, args.steps, world, clk)
    if not args.no_extra:
        line["secp256k1"] = bench_k1(ecc, costmodel, synth, torch, peak, rank, world, clk)
        line["sign_fpmul"] = bench_sign_fpmul(ecc, costmodel, synth, torch, peak, rank, n, world, clk)
    clk.stop()
    line["clocks"] = clk.summary("verify")
    for key in ("msm", "ragged", "sm2", "secp256k1", "sign_fpmul"):
        if key in line:
            line[key]["clocks"] = clk.summary({"sign_fpmul": "sign_fpmul"}.get(key, key))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
