"""Continuous-batching serving loop for ECDSA verification and MSM requests.

Requests of two kinds arrive over time: verification of a batch of secp256k1
triples, and a BN254 MSM of n points over device-resident bases (the same
bases for every request; a request uses the first n of them with its own
scalars).  The resident bases carry their window multiples (one bucket set per
MSM, width --table-c).  The server keeps one CUDA stream per kind.  Whenever a kind's
previous round has finished on the device and requests of that kind are
waiting, it forms the next round from the waiting requests in arrival order --
as many as fit the round limits and the free part of the device-memory budget
-- and launches it: one ``ecc_verify_batch`` over the concatenated triples, or
one ``ecc_msm_bases_ragged`` over the concatenated scalar vectors.  Rounds of
the two kinds run concurrently on the GPU; requests that arrive while a round
is running join the next one.  Completion times are read from CUDA events
(device clock), arrival times follow the offered-load schedule, and latency is
completion minus arrival.

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

from . import ecc, synth

SECP256K1_N = 0xFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFFEBAAEDCE6AF48A03BBFD25E8CD0364141
BN254_R = 0x30644E72E131A029B85045B68181585D2833E84879B9709143E1F593F0000001
VERIFY_BYTES_PER_TRIPLE = 1100      # inputs + per-item verification state
MSM_BYTES_PER_POINT = 1600          # digits, sorted pairs, running sums, partial sums


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
    (verify floor(2^(12 U)) in 1..4096, MSM floor(2^(12 + 8 U)) in 2^12..2^20)."""
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
            off = v_off % max(1, pool_triples - size)
            v_off += size
            reqs.append(Request(i, "verify", size, t, off))
        else:
            size = int(math.floor(2.0 ** (msm_lo_log2 + (msm_hi_log2 - msm_lo_log2) * u_size[i])))
            off = m_off % max(1, pool_scalars - size)
            m_off += size
            reqs.append(Request(i, "msm", size, t, off))
    return reqs


class Server:
    def __init__(self, torch, pool_triples=1 << 16, n_bases=1 << 20, pool_scalars=1 << 22,
                 hbm_budget=8 << 30, max_verify_round=1 << 18, max_msm_round_points=1 << 22,
                 seed=synth.SEED_BASE + 4, table_c=16):
        self.torch = torch
        self.budget = hbm_budget
        self.max_verify_round = max_verify_round
        self.max_msm_round_points = max_msm_round_points
        dev = torch.device("cuda")
        ecc.load()
        # verification pool: seeded keys, hashes, nonces, signed on the device, 1/8 corrupted
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
        # MSM: resident bases a_i G and a pool of scalar rows
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

    def close(self):
        if self.bases is not None:
            ecc.ecc_bases_destroy(self.bases)
            self.bases = None

    @staticmethod
    def cost(req):
        return req.size * (VERIFY_BYTES_PER_TRIPLE if req.kind == "verify" else MSM_BYTES_PER_POINT)

    # -------------------------------------------------------------- rounds
    def _launch(self, kind, batch):
        torch = self.torch
        st = self.streams[kind]
        with torch.cuda.stream(st):
            if kind == "verify":
                n = sum(q.size for q in batch)
                sl = lambda t, q: t[q.offset:q.offset + q.size]  # noqa: E731
                e = torch.cat([sl(self.e, q) for q in batch])
                r = torch.cat([sl(self.r, q) for q in batch])
                s = torch.cat([sl(self.s, q) for q in batch])
                pub = torch.cat([sl(self.pub, q) for q in batch])
                ok = torch.empty(n, dtype=torch.uint8, device="cuda")
                ecc.ecc_verify_batch(ecc.ECC_SECP256K1, n, e, r, s, pub, ok, st)
                out = ok
            else:
                sizes = np.array([q.size for q in batch], dtype=np.uint64)
                sc = torch.cat([self.scalars[q.offset:q.offset + q.size] for q in batch])
                out = torch.empty((len(batch), 16), dtype=torch.int32, device="cuda")
                ecc.ecc_msm_bases_ragged(self.bases, len(batch), sizes, sc, out, st)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(st)
        return {"kind": kind, "reqs": batch, "out": out, "event": ev,
                "bytes": sum(self.cost(q) for q in batch)}

    def _finish(self, rnd, t_start_event):
        done = t_start_event.elapsed_time(rnd["event"]) / 1e3
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
        in_use = 0
        reqs = sorted(reqs, key=lambda q: q.arrival)
        start = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        start.record()
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
                    self._finish(rnd, start)
                    in_use -= rnd["bytes"]
                    remaining -= len(rnd["reqs"])
                    inflight[kind] = None
                    progressed = True
                if inflight[kind] is None and pending[kind]:
                    batch, items = [], 0
                    limit = self.max_verify_round if kind == "verify" else self.max_msm_round_points
                    while pending[kind]:
                        q = pending[kind][0]
                        c = self.cost(q)
                        if batch and (items + q.size > limit or in_use + c > self.budget):
                            break
                        if not batch and in_use + c > self.budget and in_use > 0:
                            break  # wait for memory to free up
                        batch.append(pending[kind].popleft())
                        items += q.size
                        in_use += c
                        q.launched = now
                    if batch:
                        inflight[kind] = self._launch(kind, batch)
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


def summarise(reqs, span=None):
    lat = [q.done - q.arrival for q in reqs]
    end = max(q.done for q in reqs)
    begin = min(q.arrival for q in reqs)
    span = span or max(end - begin, 1e-9)
    lat_ms = sorted(x * 1e3 for x in lat)

    def pct(p):
        return lat_ms[min(len(lat_ms) - 1, int(math.ceil(p / 100.0 * len(lat_ms))) - 1)]

    return {"requests": len(reqs), "p50_ms": pct(50), "p99_ms": pct(99),
            "mean_ms": statistics.fmean(lat_ms), "throughput_req_s": len(reqs) / span,
            "verify_triples_s": sum(q.size for q in reqs if q.kind == "verify") / span,
            "msm_points_s": sum(q.size for q in reqs if q.kind == "msm") / span}


def main():
    import torch

    ap = argparse.ArgumentParser()
    ap.add_argument("--loads", default="0.1,0.3,0.5,0.7,0.9")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--seed", type=int, default=synth.SEED_BASE + 4)
    ap.add_argument("--table-c", type=int, default=16,
                    help="window width of the resident bases' window multiples (0: none)")
    args = ap.parse_args()
    srv = Server(torch, seed=args.seed, table_c=args.table_c)
    try:
        # peak: the whole trace offered at once (saturation)
        sat = make_trace(args.seed, args.requests, float("inf"))
        srv.run(make_trace(args.seed, 16, float("inf")))  # warm-up
        srv.run(sat)
        peak = summarise(sat)
        out = {"peak": peak, "loads": []}
        for load in [float(x) for x in args.loads.split(",")]:
            rate = load * peak["throughput_req_s"]
            tr = make_trace(args.seed + 17, args.requests, rate)
            srv.run(tr)
            row = summarise(tr)
            row.update({"offered_load": load, "offered_req_s": rate})
            out["loads"].append(row)
            print(json.dumps(row), flush=True)
        print(json.dumps({"serving": out}))
    finally:
        srv.close()


if __name__ == "__main__":
    main()
