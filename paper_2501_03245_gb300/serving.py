"""Continuous-batching serving loop for ECDSA verification and MSM requests.

Requests of two kinds arrive over time: verification of a batch of secp256k1
triples, and a BN254 MSM of n points over device-resident bases (the same
bases for every request; a request uses the first n of them with its own
scalars).  The resident bases carry their window multiples (one bucket set per
MSM, width --table-c).

Ingest.  Request payloads land in device ring buffers in arrival order (one
ring per kind: the ECDSA triples, the MSM scalar rows), wrapping to the start
when a payload would pass the end.  A round is a run of consecutive waiting
requests of one kind whose payloads are contiguous in the ring, so its inputs
are one slice of the ring and are never copied.

Rounds.  The server keeps one CUDA stream per kind.  Whenever a kind's previous
round has finished on the device and requests of that kind are waiting, it
forms the next round from them in arrival order, as many as fit the round
limits and the device-memory budget, and launches it: one ecc_verify_batch, or
one ecc_msm_bases_ragged.  Rounds of the two kinds run concurrently on the GPU;
requests that arrive while a round is running join a later one.

Admission by device memory.  At start-up, after the bases, tables and rings are
resident, the server reads the free device memory (cudaMemGetInfo) and keeps a
reserve; the rest is the workspace budget.  Each kind's workspace is measured
from the library itself: a calibration round of two sizes runs with a counting
workspace allocator installed (ecc_set_allocator), giving bytes = fixed + per
item.  A round is admitted only while the workspaces of the rounds in flight
plus its own fit the budget; a request larger than the whole budget is
refused.

Clock.  Arrival times follow the offered-load schedule; a round's completion
is the host time at which its CUDA event is first seen complete (polled every
50 microseconds).  Both are perf_counter readings against the same start, so
latency = completion - arrival on one clock.

Load.  The work of a request is its algorithmic multiply-add count (the
verification kernel's count per triple; the Pippenger count at the table
width for an MSM).  The peak work rate is that of the saturated run (the whole
trace offered at once); offered load x means Poisson arrivals at x times the
peak work rate.

Run as a module for the load sweep:
  python -m paper_2501_03245_gb300.serving --loads 0.1,0.3,0.5,0.7,0.9 --requests 2000
"""
import argparse
import collections
import json
import math
import statistics
import time

import numpy as np

from . import costmodel, ecc, synth

SECP256K1_N = 0xFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFEBAAEDCE6AF48A03BBFD25E8CD0364141
BN254_R = 0x30644E72E131A029B85045B68181585D2833E84879B9709143E1F593F0000001


class Request:
    __slots__ = ("rid", "kind", "size", "arrival", "offset", "launched", "done", "result")

    def __init__(self, rid, kind, size, arrival, offset):
        self.rid, self.kind, self.size, self.arrival, self.offset = rid, kind, size, arrival, offset
        self.launched = self.done = None
        self.result = None


def make_trace(seed, count, rate, mix=0.5, verify_max_log2=12, msm_lo_log2=12, msm_hi_log2=20,
               pool_triples=1 << 16, pool_scalars=1 << 22):
    """Seeded request trace: Poisson arrivals at `rate` requests/s (rate = inf:
    everything at t = 0), kind by a biased coin, sizes log-uniform
    (verify floor(2^(12 U)) in 1..4096, MSM floor(2^(12 + 8 U)) in 2^12..2^20).
    Payloads take the next free place of their kind's ring, in arrival order,
    wrapping to 0 when they would pass its end."""
    u_gap = synth.uniform_unit(seed, synth.S_ARRIVAL, count)
    u_kind = synth.uniform_unit(seed, synth.S_KIND, count)
    u_size = synth.uniform_unit(seed, synth.S_REQSIZE, count)
    t = 0.0
    reqs = []
    v_off = m_off = 0
    for i in range(count):
        if math.isfinite(rate):
            t += -math.log(1.0 - u_gap[i]) / rate
        if u_kind[i] < mix:
            size = max(1, int(math.floor(2.0 ** (verify_max_log2 * u_size[i]))))
            off = v_off if v_off + size <= pool_triples else 0
            v_off = off + size
            reqs.append(Request(i, "verify", size, t, off))
        else:
            size = int(math.floor(2.0 ** (msm_lo_log2 + (msm_hi_log2 - msm_lo_log2) * u_size[i])))
            off = m_off if m_off + size <= pool_scalars else 0
            m_off = off + size
            reqs.append(Request(i, "msm", size, t, off))
    return reqs


def take_round(pending, limit, budget_left, cost):
    """The next round of one kind: the longest run of waiting requests (in
    arrival order) whose payloads are contiguous in the ring, at most `limit`
    items, and whose workspace cost(items) fits budget_left.  Returns (batch,
    items); an empty batch when even the first request does not fit."""
    batch, items = [], 0
    for q in pending:
        if batch and q.offset != batch[-1].offset + batch[-1].size:
            break  # the ring wrapped
        if batch and items + q.size > limit:
            break
        if cost(items + q.size) > budget_left:
            break
        batch.append(q)
        items += q.size
    return batch, items


def request_work(kind, size, table_c):
    """Algorithmic wide multiply-adds of one request."""
    if kind == "verify":
        return size * costmodel.verify_imad()
    W = costmodel.msm_windows(254, table_c)
    return costmodel.msm_modmul_precomputed(size, W, table_c) * costmodel.imad_per_modmul(8)


class Server:
    def __init__(self, torch, pool_triples=1 << 16, n_bases=1 << 20, pool_scalars=1 << 22,
                 max_verify_round=1 << 18, max_msm_round_points=1 << 22, reserve_frac=0.1,
                 seed=synth.SEED_BASE + 4, table_c=16, hbm_budget=None):
        self.torch = torch
        self.max_verify_round = max_verify_round
        self.max_msm_round_points = max_msm_round_points
        self.table_c = table_c
        dev = torch.device("cuda")
        ecc.load()
        # verification ring: seeded keys, hashes, nonces, signed on the device, 1/8 corrupted
        raw = synth.ecdsa_raw(seed, pool_triples, SECP256K1_N, 8)
        to = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)  # noqa: E731
        d, e, k = to(raw["d"]), to(raw["e"]), to(raw["k"])
        r = torch.empty((pool_triples, 32), dtype=torch.uint8, device=dev)
        s = torch.empty_like(r)
        pub = torch.empty((pool_triples, 64), dtype=torch.uint8, device=dev)
        ecc.ecc_sign_batch(ecc.ECC_SECP256K1, pool_triples, d, e, k, r, s, pub)
        torch.cuda.synchronize()
        r_h, s_h = synth.apply_corruption(r.cpu().numpy(), s.cpu().numpy(), raw["corrupt_idx"],
                                          raw["corrupt_kind"], raw["corrupt_bit"])
        self.e, self.r, self.s, self.pub = e, to(r_h), to(s_h), pub
        # MSM: resident bases a_i G and the ring of scalar rows
        a = synth.uniform_limbs(seed, synth.S_BASE_MULT, n_bases, BN254_R, lo=1)
        self.bases_pts = torch.empty((n_bases, 16), dtype=torch.int32, device=dev)
        ecc.ecc_fixed_base_mul(ecc.ECC_BN254, n_bases, to(a.view(np.int32)), self.bases_pts)
        self.bases = ecc.ecc_bases_create(ecc.ECC_BN254, n_bases, self.bases_pts)
        if table_c:
            # resident window multiples: every MSM round uses one bucket set
            ecc.ecc_bases_precompute(self.bases, table_c)
        self.n_bases = n_bases
        ks = synth.uniform_limbs(seed, synth.S_SCALAR, pool_scalars, BN254_R)
        self.scalars = to(ks.view(np.int32))
        torch.cuda.synchronize()
        self.streams = {"verify": torch.cuda.Stream(), "msm": torch.cuda.Stream()}
        self.model = self._calibrate()
        free, _ = torch.cuda.mem_get_info()
        self.budget = hbm_budget if hbm_budget is not None else int(free * (1.0 - reserve_frac))

    def close(self):
        if self.bases is not None:
            ecc.ecc_bases_destroy(self.bases)
            self.bases = None

    # -------------------------------------------------------------- admission
    def _calibrate(self):
        """Workspace bytes of a round as fixed + per-item, per kind, measured by
        running rounds of two sizes with a counting workspace allocator."""
        torch = self.torch
        live = {"now": 0, "peak": 0}
        sizes_of = {}

        def alloc(nbytes, stream):
            p = torch.cuda.caching_allocator_alloc(nbytes, torch.cuda.current_device(), stream)
            sizes_of[p] = nbytes
            live["now"] += nbytes
            live["peak"] = max(live["peak"], live["now"])
            return p

        def release(p, stream):
            live["now"] -= sizes_of.pop(p, 0)
            torch.cuda.caching_allocator_delete(p)

        model = {}
        ecc.ecc_set_allocator(alloc, release)
        try:
            v2 = min(4096, self.e.shape[0])
            m2 = min(1 << 15, self.n_bases, self.scalars.shape[0])
            for kind, (n1, n2) in (("verify", (max(1, v2 // 16), v2)), ("msm", (max(1, m2 // 8), m2))):
                peaks = []
                for n in (n1, n2):
                    live["peak"] = live["now"] = 0
                    q = Request(-1, kind, n, 0.0, 0)
                    rnd = self._launch(kind, [q])
                    rnd["event"].synchronize()
                    peaks.append(live["peak"])
                per = max(0.0, (peaks[1] - peaks[0]) / (n2 - n1))
                fixed = max(0.0, peaks[0] - per * n1)
                model[kind] = (fixed, per)
        finally:
            ecc.ecc_set_allocator(None, None)
        return model

    def cost(self, kind, items):
        """Workspace bytes of a round of `items` items of `kind` (with 25% slack)."""
        fixed, per = self.model[kind]
        return int(1.25 * (fixed + per * items)) + (1 << 20)

    # -------------------------------------------------------------- rounds
    def _launch(self, kind, batch):
        torch = self.torch
        st = self.streams[kind]
        lo = batch[0].offset
        n = sum(q.size for q in batch)
        with torch.cuda.stream(st):
            if kind == "verify":
                ok = torch.empty(n, dtype=torch.uint8, device="cuda")
                ecc.ecc_verify_batch(ecc.ECC_SECP256K1, n, self.e[lo:lo + n], self.r[lo:lo + n],
                                     self.s[lo:lo + n], self.pub[lo:lo + n], ok, st)
                out = ok
            else:
                sizes = np.array([q.size for q in batch], dtype=np.uint64)
                out = torch.empty((len(batch), 16), dtype=torch.int32, device="cuda")
                ecc.ecc_msm_bases_ragged(self.bases, len(batch), sizes, self.scalars[lo:lo + n], out, st)
            ev = torch.cuda.Event()
            ev.record(st)
        return {"kind": kind, "reqs": batch, "out": out, "event": ev,
                "bytes": self.cost(kind, n) if kind in getattr(self, "model", {}) else 0}

    @staticmethod
    def _finish(rnd, done):
        if rnd["kind"] == "verify":
            ok = rnd["out"].cpu().numpy()
            pos = 0
            for q in rnd["reqs"]:
                q.result = ok[pos:pos + q.size].copy()
                pos += q.size
                q.done = done
        else:
            pts = rnd["out"].cpu().numpy().view(np.uint32)
            for i, q in enumerate(rnd["reqs"]):
                q.result = pts[i].copy()
                q.done = done

    def run(self, reqs, poll_s=50e-6):
        """Serves a trace (arrival times relative to the start); returns it."""
        torch = self.torch
        pending = {"verify": collections.deque(), "msm": collections.deque()}
        inflight = {"verify": None, "msm": None}
        limits = {"verify": self.max_verify_round, "msm": self.max_msm_round_points}
        in_use = 0
        reqs = sorted(reqs, key=lambda q: q.arrival)
        for q in reqs:
            if self.cost(q.kind, q.size) > self.budget:
                raise ValueError(f"request {q.rid} needs more device memory than the whole budget")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nxt = 0
        remaining = len(reqs)
        while remaining:
            now = time.perf_counter() - t0
            while nxt < len(reqs) and reqs[nxt].arrival <= now:
                pending[reqs[nxt].kind].append(reqs[nxt])
                nxt += 1
            progressed = False
            for kind in ("verify", "msm"):
                rnd = inflight[kind]
                if rnd is not None and rnd["event"].query():
                    self._finish(rnd, time.perf_counter() - t0)
                    in_use -= rnd["bytes"]
                    remaining -= len(rnd["reqs"])
                    inflight[kind] = None
                    progressed = True
                if inflight[kind] is None and pending[kind]:
                    batch, _ = take_round(pending[kind], limits[kind], self.budget - in_use,
                                          lambda items, k=kind: self.cost(k, items))
                    if batch:
                        for _ in batch:
                            pending[kind].popleft()
                        for q in batch:
                            q.launched = now
                        rnd = self._launch(kind, batch)
                        in_use += rnd["bytes"]
                        inflight[kind] = rnd
                        progressed = True
            if not progressed:
                if nxt < len(reqs) and all(v is None for v in inflight.values()):
                    time.sleep(max(0.0, min(reqs[nxt].arrival - (time.perf_counter() - t0), 0.01)))
                else:
                    time.sleep(poll_s)
        torch.cuda.synchronize()
        return reqs

    # -------------------------------------------------------------- single requests
    def run_alone(self, q):
        """The same request served alone (one round of its own), for the
        alone-versus-in-the-mix check."""
        rnd = self._launch(q.kind, [q])
        rnd["event"].synchronize()
        if q.kind == "verify":
            return rnd["out"].cpu().numpy().copy()
        return rnd["out"].cpu().numpy().view(np.uint32)[0].copy()


def summarise(reqs, span=None, table_c=16):
    lat = [q.done - q.arrival for q in reqs]
    end = max(q.done for q in reqs)
    begin = min(q.arrival for q in reqs)
    span = span or max(end - begin, 1e-9)
    lat_ms = sorted(x * 1e3 for x in lat)

    def pct(p):
        return lat_ms[min(len(lat_ms) - 1, int(math.ceil(p / 100.0 * len(lat_ms))) - 1)]

    work = sum(request_work(q.kind, q.size, table_c) for q in reqs) if table_c else None
    return {"requests": len(reqs), "p50_ms": pct(50), "p99_ms": pct(99),
            "mean_ms": statistics.fmean(lat_ms), "throughput_req_s": len(reqs) / span,
            "verify_triples_s": sum(q.size for q in reqs if q.kind == "verify") / span,
            "msm_points_s": sum(q.size for q in reqs if q.kind == "msm") / span,
            "work_imad_s": work / span if work is not None else None}


def main():
    import torch

    ap = argparse.ArgumentParser()
    ap.add_argument("--loads", default="0.1,0.3,0.5,0.7,0.9")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--seed", type=int, default=synth.SEED_BASE + 4)
    ap.add_argument("--table-c", type=int, default=16,
                    help="window width of the resident bases' window multiples")
    ap.add_argument("--out", default=None, help="also write the sweep's JSON to this file")
    args = ap.parse_args()
    srv = Server(torch, seed=args.seed, table_c=args.table_c)
    try:
        # peak: the whole trace offered at once (saturation), in work per second
        sat = make_trace(args.seed, args.requests, float("inf"))
        srv.run(make_trace(args.seed, 16, float("inf")))  # warm-up
        srv.run(sat)
        peak = summarise(sat, table_c=args.table_c)
        mean_work = statistics.fmean(request_work(q.kind, q.size, args.table_c) for q in sat)
        out = {"peak": peak, "workspace_model": srv.model, "budget_bytes": srv.budget,
               "mean_request_work_imad": mean_work, "loads": []}
        for load in [float(x) for x in args.loads.split(",")]:
            rate = load * peak["work_imad_s"] / mean_work
            tr = make_trace(args.seed + 17, args.requests, rate)
            srv.run(tr)
            row = summarise(tr, table_c=args.table_c)
            row.update({"offered_load": load, "offered_req_s": rate,
                        "offered_work_imad_s": rate * mean_work,
                        "work_frac_of_peak": row["work_imad_s"] / peak["work_imad_s"]})
            out["loads"].append(row)
            print(json.dumps(row), flush=True)
        print(json.dumps({"serving": out}))
        if args.out:
            with open(args.out, "w") as f:
                json.dump({"serving": out}, f, indent=1)
    finally:
        srv.close()


if __name__ == "__main__":
    main()
