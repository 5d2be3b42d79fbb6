"""Benchmark of the SVT track-fitting chain on one GB300 (or N replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--workload stress] [--no-cpu] [--no-plain] [--no-serve] [--no-sweep]
                    [--no-tune] [--no-subs]

One step = one batch of the headline workload through the whole chain:
unpack, combine, fit, chi-square cut, hit-warrior, ordered output.  The
headline workload is the largest single-GPU configuration: 200 events x 128
roads x 8 hits on each of 5 layers (838,860,800 combinations).

  value  track fits (combinations) per second with the words resident in
         HBM: the persistent kernel, replayed from a CUDA graph, autotuned;
         each step timed with CUDA events on its stream, a 256 MB buffer
         written between steps to flush L2.
  e2e    the same metric through the public C ABI from pinned host memory:
         per batch H2D of the words, svt_unpack, svt_fit_events,
         svt_get_tracks (D2H of the status block and the tracks), host wall
         clock; two contexts take batches in turn (one batch's copies overlap
         the other's kernel).  p50 / p99 are one batch at a time.
  roofline  integer multiply-adds: 36 per distinct fit (the fit of one input
         vector x, Sec. II: 18 for p = F x + q, 18 for the chi-square rows;
         combinations that differ only in the excluded layer's hit share x),
         against the device's multiply-add rate (SMs x 64 lanes x clock; the
         in-tree measurement beside it).
  scaled / uneven  the 3000 x 64 and 10,000-event uneven batches: the
         persistent form against the plain per-stage launch (fits/s, p50,
         p99 per batch, device and end to end).
  serving  the serving runtime under Poisson arrivals at five offered event
         rates, p50 / p99 from arrival to tracks in host memory.
  packet_sweep  end-to-end latency of one batch from 600 kB of words up,
         with pageable, page-locked, and in-place (kernels read and write
         page-locked host memory) buffers, and the transfer share of each.
  loopback  a transmitter process sends packets over loopback TCP to a
         receiver process that runs the chain; round trip timed at the
         transmitter (the paper's latency set-up, without a NIC).
  cpu_baseline  the oracle (test infrastructure) on the machine's host cores:
         its event-parallel driver on a bounded sample, per-stage times.
  --impl reference  the oracle as it stands, timed on the host cores.

Multi-GPU: the chain shards by events with no exchange, so N ranks run
independent replicas (weak scaling); value = all ranks' fits / max time.
"""
from __future__ import annotations

import argparse
import atexit
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

# multiply-add lanes of one GB300 SM (the IMAD rate: half the FP32 lanes)
IMAD_LANES_PER_SM = 64
MACS_PER_FIT = 36   # 6 inputs x (3 track parameters + 3 chi-square components)
HEADLINE = "stress"


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="svt", choices=["svt", "reference"])
    ap.add_argument("--workload", default=HEADLINE)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-mode comparisons")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving-loop measurement")
    ap.add_argument("--no-sweep", action="store_true", help="skip the packet-size sweep")
    ap.add_argument("--launch", default="", help="block,blocks_per_sm,small_n4,run_roads of the headline's "
                    "persistent kernel instead of the autotuner's choice (for profiler runs)")
    ap.add_argument("--no-subs", action="store_true", help="skip the scaled and uneven sub-workloads")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner (default launch settings; for profiler runs)")
    ap.add_argument("--serve-requests", type=int, default=2000, help="requests per offered rate")
    return ap.parse_args(argv)


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def load_cut(workload):
    with open(os.path.join(ROOT, "tests", "golden", "chi2_cuts.json")) as f:
        return int(json.load(f)[workload]["cut"])


def distinct_fits(batch) -> int:
    """Combinations of the four fitted layers summed over roads: the fits
    with distinct inputs (the excluded layer's hit is not an input)."""
    n = batch.roads["n"].astype(np.int64)
    ex = batch.roads["excl"].astype(np.int64)
    per = np.prod(n, axis=1)
    ne = n[np.arange(len(n)), ex]
    return int(np.sum(np.where(ne > 0, per // np.maximum(ne, 1), 0)))


def workload_desc(cfg, n_fits, n_words):
    return "%s: %s (%d combinations, %d words)" % (cfg.name, cfg.description, n_fits, n_words)


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.monotonic(), [x.strip() for x in line.split(",")]))

    def __exit__(self, *a):
        proc, self.proc = self.proc, None
        if proc:
            proc.terminate()
            try:
                proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                proc.kill()

    def summary(self, t0=None, t1=None):
        """Median SM clock, maximum clock and throttle reasons of the samples
        taken between monotonic times t0 and t1 (all samples by default)."""
        mhz, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for t, r in self.rows:
            if (t0 is not None and t < t0) or (t1 is not None and t > t1):
                continue
            try:
                mhz.append(float(r[1]))
                mx = float(r[2])
                for n, v in zip(names, r[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
            except (ValueError, IndexError):
                pass
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(mhz)}


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------

def run_device_steps(ctx, B, torch, d_words, n_words, mode, steps, warmup, stream):
    """Per-step device time (ms) of unpack + fit with an L2 flush between."""
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    with torch.cuda.stream(stream):
        for i in range(warmup + steps):
            flush.fill_(i & 0xFF)
            if i >= warmup:
                starts[i - warmup].record(stream)
            B.check(ctx.unpack(d_words, n_words, stream), "svt_unpack")
            B.check(ctx.fit_events(mode, stream), "svt_fit_events")
            if i >= warmup:
                ends[i - warmup].record(stream)
    stream.synchronize()
    st, _ = ctx.get_tracks(out=None, stream=stream)
    B.check(st, "svt_get_tracks")
    return [s.elapsed_time(e) for s, e in zip(starts, ends)]


def run_e2e(ctx, B, torch, h_words, d_words, h_out, mode, steps, warmup, stream):
    """Per-batch host wall time (s) through the public API, pinned host I/O,
    one batch at a time."""
    n_words = h_words.numel()
    lat, d2h = [], []
    for i in range(warmup + steps):
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            d_words.copy_(h_words, non_blocking=True)
        B.check(ctx.unpack(d_words, n_words, stream), "svt_unpack")
        B.check(ctx.fit_events(mode, stream), "svt_fit_events")
        st, n = ctx.get_tracks(out=h_out, cap=h_out.numel() // 40, stream=stream)
        B.check(st, "svt_get_tracks")
        t1 = time.perf_counter()
        if i >= warmup:
            lat.append(t1 - t0)
            d2h.append(n * 40)
    return lat, d2h


def run_e2e_pipelined(ctxs, B, torch, h_words, d_words, h_outs, mode, steps, warmup, streams):
    """Throughput through the public API with two contexts on two streams
    taking batches in turn: batch i + 1's H2D copy and kernel are enqueued
    before batch i's tracks are read back (svt_get_tracks waits for them), so
    one batch's copies overlap the other's kernel.  Every batch still copies
    its words in from pinned host memory and its tracks out.  Returns the
    host wall time (s) of `steps` batches started and finished inside the
    timed region (warm-up batches drained first) and the D2H bytes."""
    n_words = h_words.numel()

    def submit(k):
        with torch.cuda.stream(streams[k]):
            d_words[k].copy_(h_words, non_blocking=True)
        B.check(ctxs[k].unpack(d_words[k], n_words, streams[k]), "svt_unpack")
        B.check(ctxs[k].fit_events(mode, streams[k]), "svt_fit_events")

    def run(count):
        d2h = []
        submit(0)
        for i in range(count):
            k = i % 2
            if i + 1 < count:
                submit((i + 1) % 2)
            st, n = ctxs[k].get_tracks(out=h_outs[k], cap=h_outs[k].numel() // 40, stream=streams[k])
            B.check(st, "svt_get_tracks")
            d2h.append(n * 40)
        return d2h

    run(max(2, warmup))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d2h = run(steps)
    t1 = time.perf_counter()
    return t1 - t0, d2h


def cpu_baseline(batch, consts, cut, target_s=12.0):
    """The oracle as it stands on the host cores: its event-parallel driver
    (one event per core at a time) on the first events of the batch, grown
    until a run takes about target_s / 2 seconds; per-stage host times."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    n_ev = min(batch.n_events, cores)
    while True:
        words = batch.event_slice(0, n_ev)
        t0 = time.perf_counter()
        rc, out, times = oracle.run_mt(words, consts, cut)
        dt = time.perf_counter() - t0
        assert rc == 0
        if dt > target_s / 2 or n_ev >= batch.n_events:
            break
        n_ev = min(batch.n_events, max(n_ev + cores, int(n_ev * 1.1 * target_s / 2 / max(dt, 1e-3))))
    sel = batch.roads["event"] < n_ev
    fits = int(np.prod(batch.roads["n"][sel], axis=1).sum())
    return {"value": fits / dt, "unit": "fits/s", "cores": times["threads"], "kind": "oracle",
            "sample": "first %d events of the batch (%d combinations), one run, %.1f s wall"
                      % (n_ev, fits, dt),
            "stage_s": {"unpack": round(times["unpack_s"], 3), "combine_fit_cut": round(times["fit_s"], 3),
                        "hit_warrior": round(times["warrior_s"], 3),
                        "note": "unpack serial; the others summed over threads"}}


def run_serving(B, synth, consts, cut, rates, n_requests, n_slots=8, seed=0, **server_cfg):
    """Serving loop (svt_server) under Poisson arrivals of requests whose
    event counts are log-uniform in [1, 512) (scaled-shaped events), at each
    offered event rate.  Latency of a request: from its scheduled arrival to
    its tracks in host memory (admission wait, copies and kernel included)."""
    sizes = synth.request_sizes(seed, 64)
    pool = [synth.make_batch("scaled", seed=500 + i, n_events=int(k)).words for i, k in enumerate(sizes)]
    srv = B.Server(consts, cut, n_slots=n_slots, **server_cfg)
    try:
        for w in pool[:16]:                      # warm-up
            srv.submit(w)
            r = srv.wait(10_000_000)
            srv.take(r["request_id"], r["n_tracks"])
        rng = np.random.default_rng(seed)
        out = []
        for rate in rates:
            req_rate = rate / float(np.mean(sizes))
            n_req = int(n_requests)
            arrivals = np.cumsum(rng.exponential(1.0 / req_rate, n_req))
            done, sched = {}, {}

            def collect():
                while len(done) < n_req:
                    r = srv.wait(5_000_000)
                    if r is None:
                        break
                    srv.take(r["request_id"], r["n_tracks"])
                    done[r["request_id"]] = (r, time.perf_counter())

            th = threading.Thread(target=collect)
            th.start()
            t0 = time.perf_counter()
            n_ev = 0
            for i in range(n_req):
                target = t0 + arrivals[i]
                while True:
                    now = time.perf_counter()
                    if now >= target:
                        break
                    if target - now > 3e-4:
                        time.sleep(target - now - 2e-4)
                w = pool[i % len(pool)]
                t_sub = time.perf_counter()
                sched[srv.submit(w)] = (target, t_sub)
                n_ev += int(sizes[i % len(pool)])
            th.join()
            lat, wait, bad, t_end = [], [], 0, t0
            for rid, (r, t_done) in done.items():
                target, t_sub = sched[rid]
                lat.append((t_sub - target) + r["latency_ns"] * 1e-9)
                wait.append(t_sub - target)
                bad += r["status"] != B.OK
                t_end = max(t_end, t_done)
            lat = np.array(lat) * 1e6
            out.append({"offered_events_per_s": rate, "requests": n_req, "completed": len(done),
                        "errors": bad, "sustained_events_per_s": n_ev / (t_end - t0),
                        "p50_us": float(np.percentile(lat, 50)), "p99_us": float(np.percentile(lat, 99)),
                        "p99_submit_wait_us": float(np.percentile(np.array(wait) * 1e6, 99))})
        return {"slots": srv.config()["n_slots"], "request_events": "log-uniform in [1, 512)",
                "arrivals": "Poisson", "rates": out}
    finally:
        srv.close()


# DRAM bytes (read + write) of one persistent-kernel launch per workload, from
# the ncu captures summarised under profiles/, with the SHA-256 of the kernel sources
# (kernels and their header) they were taken on: the bench line reports a
# figure only while the sources are unchanged.
NCU_TRAFFIC = {
    "stress": {"kernels_sha256": "0534c74cb0ab5f09209c952563eeee5892be75a4d1c9d099ab65f7b7abb143bf", "bytes": 5278720},    # 5.279 MB read, 0 B written
    "scaled": {"kernels_sha256": "0534c74cb0ab5f09209c952563eeee5892be75a4d1c9d099ab65f7b7abb143bf", "bytes": 12697600},   # 12.626 MB read + 71.7 KB written
    "uneven": {"kernels_sha256": "0534c74cb0ab5f09209c952563eeee5892be75a4d1c9d099ab65f7b7abb143bf", "bytes": 20996096},   # 17.692 MB read + 3.304 MB written
}


def measured_traffic(workload: str):
    import hashlib
    h = hashlib.sha256()
    for name in ("svt_kernels.cu", "svt_internal.h"):
        with open(os.path.join(ROOT, "paper_1312_0917_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    rec = NCU_TRAFFIC.get(workload)
    if rec and rec["kernels_sha256"] == h.hexdigest():
        return rec["bytes"]
    return None


# The plain pipeline stores every combination's key (8 bytes) and track
# parameters (12 bytes) and its warrior reads the keys back: 28 bytes of HBM
# traffic per combination that the persistent kernel never makes.
PLAIN_BYTES_PER_COMB = 28


def measured_hbm_gbs() -> float:
    """The measured copy bandwidth of the GB300s (MEASURED_PEAKS.json,
    written by the benchmark's driver), else the earlier measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return 6800.0


def plain_hbm(n_fits: int, ms: float) -> dict:
    """HBM roofline of the plain pipeline (bound by its per-combination stores)."""
    gbs = PLAIN_BYTES_PER_COMB * n_fits / (ms / 1e3) / 1e9
    peak = measured_hbm_gbs()
    return {"bytes_per_batch": PLAIN_BYTES_PER_COMB * n_fits, "achieved_gbs": round(gbs, 1),
            "peak_gbs": peak, "frac": round(gbs / peak, 3),
            "note": "28 B per combination: key and track parameters stored, keys read back"}


def max_over_ranks(x: float, world: int) -> float:
    """The largest x over all ranks (the job's time is its slowest rank's)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t[0])


def whole_job_rate(units_per_rank: int, world: int, seconds: float) -> float:
    """Units every rank processed (replicas: the same per rank) per second of
    the slowest rank."""
    return units_per_rank * world / seconds


def tune(ctx, B, d_words, n_words, stream):
    assert ctx.unpack(d_words, n_words, stream) == B.OK
    pts = ctx.autotune(reps=5, stream=stream)
    best = ctx.get_launch()
    keys = ("block", "blocks_per_sm", "small_n4", "run_roads")
    return dict(best, axes=list(keys) + ["us"],
                points=[[p[0][k] for k in keys] + [round(p[1] * 1e3, 1)] for p in pts])


def sub_workload(B, torch, synth, name, consts, local, args):
    """One sub-workload: the persistent form (autotuned, graph) against the
    plain per-stage launch, device time per batch and end to end (one batch
    at a time, pinned host I/O)."""
    cfg = synth.CONFIGS[name]
    batch = synth.make_batch(cfg, seed=0)
    cut = load_cut(name)
    n_fits, n_words = batch.n_fits, len(batch.words)
    ctx = B.Context(local, max_combinations=n_fits if not args.no_plain else 1 << 10)
    ctx.load_constants(consts, cut)
    stream = torch.cuda.Stream()
    h_words = torch.from_numpy(batch.words.view(np.int32)).pin_memory()
    d_words = torch.empty_like(h_words, device="cuda")
    d_words.copy_(h_words)
    torch.cuda.synchronize()
    out = {"workload": workload_desc(cfg, n_fits, n_words)}
    if not args.no_tune:
        out["autotuned"] = tune(ctx, B, d_words, n_words, stream)
    steps = max(10, args.steps)
    modes = [("persistent", B.PERSISTENT)] + ([] if args.no_plain else [("plain", B.PLAIN)])
    for label, mode in modes:
        ctx.use_graph(mode == B.PERSISTENT)
        t = run_device_steps(ctx, B, torch, d_words, n_words, mode, steps, args.warmup, stream)
        stats = ctx.get_stats(stream)
        h_out = torch.empty(max(1, stats["n_tracks"]) * 40, dtype=torch.uint8).pin_memory()
        lat, _ = run_e2e(ctx, B, torch, h_words, d_words, h_out, mode, steps, args.warmup, stream)
        out[label] = {"fits_per_s": n_fits / (statistics.mean(t) / 1e3),
                      "ms_per_batch": statistics.mean(t),
                      "p50_us": 1e3 * float(np.percentile(t, 50)), "p99_us": 1e3 * float(np.percentile(t, 99)),
                      "e2e_p50_us": 1e6 * float(np.percentile(lat, 50)),
                      "e2e_p99_us": 1e6 * float(np.percentile(lat, 99)),
                      "gpu_launches_per_batch": ctx.last_launch_count(),
                      "tracks": stats["n_tracks"]}
        if mode == B.PERSISTENT:
            out[label]["dram_bytes_per_batch"] = measured_traffic(name)
            out[label]["phase_us"] = dict(zip(
                ["word_scan", "road_decode", "cross_road_flags", "fit_cut_local_warrior",
                 "cross_road_warrior", "output"], [round(x / 1e3, 1) for x in stats["phase_ns"]]))
        else:
            out[label]["hbm_roofline"] = plain_hbm(n_fits, statistics.mean(t))
    ctx.close()
    return out


def packet_sweep(B, torch, synth, consts, local, sizes_kb=(600, 1200, 2400, 4800, 9600, 19200), reps=30):
    """End-to-end latency of one batch against its size (kB of input words;
    events shaped as the scaled workload, Sec. IV-C's packet sizes from 600 kB
    up), with the host buffers in three kinds of memory: pageable (the copies
    are staged by the CUDA runtime), page-locked (DMA copies in and out), and
    page-locked memory that the kernels read and write in place (no copies).
    The transfer share is 1 - device time / end-to-end time."""
    cut = load_cut("scaled")
    per_event = 4 * (len(synth.make_batch("scaled", seed=0, n_events=64).words) / 64)
    sizes = [(kb, max(1, int(round(kb * 1000 / per_event)))) for kb in sizes_kb]
    n_max = max(e for _, e in sizes)
    ctx = B.Context(local, max_words=int(n_max * per_event / 4) + 4096, max_events=n_max + 1,
                    max_roads=64 * (n_max + 1), max_tracks=256 * (n_max + 1), max_combinations=1 << 10)
    ctx.load_constants(consts, cut)
    stream = torch.cuda.Stream()
    rows = []
    for i, (kb, n_ev) in enumerate(sizes):
        batch = synth.make_batch("scaled", seed=500 + i, n_events=n_ev)
        n_words = len(batch.words)
        h_page = batch.words.view(np.int32).copy()
        h_pin = torch.from_numpy(h_page).pin_memory()
        d_words = torch.empty_like(h_pin, device="cuda")
        d_words.copy_(h_pin)
        torch.cuda.synchronize()
        dev = run_device_steps(ctx, B, torch, d_words, n_words, B.PERSISTENT, reps, 3, stream)
        n_tr = ctx.get_stats(stream)["n_tracks"]
        out_page = np.empty(max(1, n_tr), dtype=B.TRACK_DTYPE)
        out_pin = torch.empty(max(1, n_tr) * 40, dtype=torch.uint8).pin_memory()
        out_map = torch.empty(max(1, n_tr) * 40, dtype=torch.uint8).pin_memory()
        cap = max(1, n_tr)
        row = {"kB": round(4 * n_words / 1e3, 1), "events": n_ev, "tracks": n_tr,
               "device_p50_us": round(1e3 * float(np.percentile(dev, 50)), 1)}
        for kind in ("pageable", "pinned", "in_place", "pinned_in_tracks_out_in_place"):
            if kind in ("in_place", "pinned_in_tracks_out_in_place"):
                ctx.set_track_output(out_map, cap)
            lat = []
            for r in range(3 + reps):
                t0 = time.perf_counter()
                if kind == "in_place":
                    src = h_pin
                else:
                    with torch.cuda.stream(stream):
                        d_words.copy_(torch.from_numpy(h_page) if kind == "pageable" else h_pin,
                                      non_blocking=True)
                    src = d_words
                B.check(ctx.unpack(src, n_words, stream), "svt_unpack")
                B.check(ctx.fit_events(B.PERSISTENT, stream), "svt_fit_events")
                out = out_page if kind == "pageable" else out_pin if kind == "pinned" else out_map
                st, n = ctx.get_tracks(out=out, cap=cap, stream=stream)
                B.check(st, "svt_get_tracks")
                if r >= 3:
                    lat.append(time.perf_counter() - t0)
            if kind in ("in_place", "pinned_in_tracks_out_in_place"):
                ctx.set_track_output(None)
            p50 = 1e6 * float(np.percentile(lat, 50))
            row[kind] = {"p50_us": round(p50, 1), "p99_us": round(1e6 * float(np.percentile(lat, 99)), 1),
                         "transfer_share": round(max(0.0, 1 - row["device_p50_us"] / p50), 3)}
        rows.append(row)
    ctx.close()
    return {"events": "scaled-shaped (64 roads, 1-4 hits per layer)", "reps": reps,
            "latency": "host wall time of one batch: words in, kernel, tracks out", "sizes": rows}


def _recv_exact(sock, view):
    """Fill the writable memoryview `view` from the socket."""
    got = 0
    while got < len(view):
        n = sock.recv_into(view[got:])
        if n == 0:
            raise ConnectionError("peer closed")
        got += n


def loopback_receiver(pipe, device, consts, cut, max_words):
    """The receiving process of the loopback loop (a separate process, as in
    Sec. III's transmitter/receiver set-up, Fig. 1): accepts one TCP
    connection on 127.0.0.1, then for every packet (8-byte word count, then
    the words) copies the words to the device, runs the chain and sends back
    a 24-byte header (status, track count, its own processing time in ns) and
    the tracks.  A word count of 0 ends it."""
    import socket
    import struct
    import torch
    from paper_1312_0917_gb300 import binding as B
    torch.cuda.set_device(device)
    max_tracks = max_words
    ctx = B.Context(device, max_words=max_words, max_events=max_words // 3 + 1, max_roads=max_words // 3 + 1,
                    max_tracks=max_tracks, max_combinations=1 << 10)
    ctx.load_constants(consts, cut)
    stream = torch.cuda.Stream()
    h_words = torch.empty(max_words, dtype=torch.int32).pin_memory()
    d_words = torch.empty(max_words, dtype=torch.int32, device="cuda")
    h_out = torch.empty(max_tracks * 40, dtype=torch.uint8).pin_memory()
    wview = memoryview(h_words.numpy()).cast("B")
    oview = memoryview(h_out.numpy())
    srv = socket.socket(socket.AF_INET, socket.SOCK_STREAM)
    srv.bind(("127.0.0.1", 0))
    srv.listen(1)
    pipe.send(srv.getsockname()[1])
    sock, _ = srv.accept()
    sock.setsockopt(socket.IPPROTO_TCP, socket.TCP_NODELAY, 1)
    hdr = bytearray(8)
    try:
        while True:
            _recv_exact(sock, memoryview(hdr))
            (n_words,) = struct.unpack("<Q", hdr)
            if n_words == 0:
                break
            _recv_exact(sock, wview[:4 * n_words])
            t0 = time.perf_counter_ns()
            with torch.cuda.stream(stream):
                d_words[:n_words].copy_(h_words[:n_words], non_blocking=True)
            B.check(ctx.unpack(d_words, n_words, stream), "svt_unpack")
            B.check(ctx.fit_events(B.PERSISTENT, stream), "svt_fit_events")
            st, n = ctx.get_tracks(out=h_out, cap=max_tracks, stream=stream)
            dt = time.perf_counter_ns() - t0
            sock.sendall(struct.pack("<qqq", st, n if st == B.OK else 0, dt))
            if st == B.OK and n:
                sock.sendall(oview[:40 * n])
    finally:
        sock.close()
        srv.close()
        ctx.close()


def loopback_loop(synth, consts, local, sizes_kb=(600, 2400, 9600), reps=20):
    """NEXT-3 of the hot-path plan: a transmitter (this process) sends packets
    of words over host loopback TCP to a receiver process that runs the chain
    on the GPU and sends the tracks back; the round trip is timed at the
    transmitter (Sec. III, Fig. 1).  Reports per packet size the round trip
    (p50 / p99), the receiver's own time (H2D, kernel, D2H), and the share of
    the round trip spent outside it (socket transfers both ways)."""
    import multiprocessing as mp
    import socket
    import struct
    cut = load_cut("scaled")
    per_event = 4 * (len(synth.make_batch("scaled", seed=0, n_events=64).words) / 64)
    sizes = [(kb, max(1, int(round(kb * 1000 / per_event)))) for kb in sizes_kb]
    max_words = int(max(e for _, e in sizes) * per_event / 4) + 4096
    ctx_mp = mp.get_context("spawn")
    parent, child = ctx_mp.Pipe()
    proc = ctx_mp.Process(target=loopback_receiver, args=(child, local, consts, cut, max_words), daemon=True)
    proc.start()
    rows = []
    try:
        if not parent.poll(300):
            raise RuntimeError("the loopback receiver did not start")
        port = parent.recv()
        sock = socket.create_connection(("127.0.0.1", port))
        sock.setsockopt(socket.IPPROTO_TCP, socket.TCP_NODELAY, 1)
        hdr = bytearray(24)
        for i, (kb, n_ev) in enumerate(sizes):
            words = synth.make_batch("scaled", seed=700 + i, n_events=n_ev).words
            out = bytearray(40 * max_words)
            rtt, proc_ns, n_tr = [], [], 0
            for r in range(3 + reps):
                t0 = time.perf_counter()
                sock.sendall(struct.pack("<Q", len(words)))
                sock.sendall(memoryview(words).cast("B"))
                _recv_exact(sock, memoryview(hdr))
                st, n_tr, dt = struct.unpack("<qqq", hdr)
                if st != 0:
                    raise RuntimeError("receiver status %d" % st)
                _recv_exact(sock, memoryview(out)[:40 * n_tr])
                t1 = time.perf_counter()
                if r >= 3:
                    rtt.append(t1 - t0)
                    proc_ns.append(dt)
            p50 = 1e6 * float(np.percentile(rtt, 50))
            pr = float(np.percentile(proc_ns, 50)) / 1e3
            rows.append({"kB": round(4 * len(words) / 1e3, 1), "events": n_ev, "tracks": n_tr,
                         "round_trip_p50_us": round(p50, 1),
                         "round_trip_p99_us": round(1e6 * float(np.percentile(rtt, 99)), 1),
                         "receiver_p50_us": round(pr, 1), "socket_share": round(max(0.0, 1 - pr / p50), 3)})
        sock.sendall(struct.pack("<Q", 0))
        sock.close()
    finally:
        proc.join(timeout=30)
        if proc.is_alive():
            proc.terminate()
    return {"transport": "TCP over 127.0.0.1, one connection, TCP_NODELAY", "reps": reps,
            "receiver": "separate process: pinned H2D, persistent kernel, D2H of the tracks", "sizes": rows}


def gpu_arm(args):
    import torch
    from paper_1312_0917_gb300 import binding as B, synth, build as nvbuild

    rank, local, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    nvbuild.build()
    peak = B.measure_int_peak(local)
    cfg = synth.CONFIGS[args.workload]
    batch = synth.make_batch(cfg, seed=0)
    consts = synth.make_constants(0)
    cut = load_cut(args.workload)
    n_fits, n_words, n_events = batch.n_fits, len(batch.words), batch.n_events
    n_fit4 = distinct_fits(batch)
    mode = B.PERSISTENT

    ctx = B.Context(local, max_combinations=n_fits if not args.no_plain else 1 << 10)
    ctx.load_constants(consts, cut)
    stream = torch.cuda.Stream()
    h_words = torch.from_numpy(batch.words.view(np.int32)).pin_memory()
    d_words = torch.empty_like(h_words, device="cuda")
    d_words.copy_(h_words)
    torch.cuda.synchronize()

    # correctness of the timed configuration is checked by the tests (every
    # workload against the oracle); here the track count is recorded
    tuned = None if args.no_tune or args.launch else tune(ctx, B, d_words, n_words, stream)
    if args.launch:
        blk, bps, small, run = (int(x) for x in args.launch.split(","))
        ctx.set_launch(block=blk, blocks_per_sm=bps, small_n4=small, run_roads=run)
        tuned = dict(ctx.get_launch(), note="set by --launch, not tuned")
    ctx.use_graph(True)
    clocks = ClockSampler(local).__enter__()
    atexit.register(clocks.__exit__)   # the sampler stops on an early exit too
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_timed0 = time.monotonic()
    times = run_device_steps(ctx, B, torch, d_words, n_words, mode, args.steps, args.warmup, stream)
    torch.cuda.synchronize()
    t_timed1 = time.monotonic()
    if world > 1:
        dist.barrier()
    launches = ctx.last_launch_count()
    stats = ctx.get_stats(stream)
    total_ms = max_over_ranks(sum(times), world)
    step_ms = total_ms / len(times)
    value = whole_job_rate(n_fits, world, step_ms / 1e3)

    # the plain per-stage pipeline on the same batch, for comparison
    plain = None
    if not args.no_plain:
        ctx.use_graph(False)
        pt = run_device_steps(ctx, B, torch, d_words, n_words, B.PLAIN, max(5, args.steps // 3), 3, stream)
        plain = {"ms_per_step": statistics.mean(pt), "fits_per_s": n_fits / (statistics.mean(pt) / 1e3),
                 "p50_us": 1e3 * float(np.percentile(pt, 50)), "p99_us": 1e3 * float(np.percentile(pt, 99)),
                 "gpu_launches_per_step": ctx.last_launch_count(),
                 "hbm_roofline": plain_hbm(n_fits, statistics.mean(pt))}
        ctx.use_graph(True)

    # end to end through the public API: the latency of one batch at a time,
    # then the throughput of two contexts taking batches in turn (the value)
    h_out = torch.empty(max(1, stats["n_tracks"]) * 40, dtype=torch.uint8).pin_memory()
    lat, d2h = run_e2e(ctx, B, torch, h_words, d_words, h_out, mode, args.steps, args.warmup, stream)
    ctx2 = B.Context(local, max_combinations=1 << 10)
    ctx2.load_constants(consts, cut)
    if tuned:
        ctx2.set_launch(**{k: tuned[k] for k in ("block", "blocks_per_sm", "small_n4", "run_roads")})
    ctx2.use_graph(True)
    stream2 = torch.cuda.Stream()
    d_words2 = torch.empty_like(d_words)
    h_out2 = torch.empty_like(h_out).pin_memory()
    if world > 1:
        dist.barrier()
    pipe_s, pipe_d2h = run_e2e_pipelined([ctx, ctx2], B, torch, h_words, [d_words, d_words2],
                                         [h_out, h_out2], mode, args.steps, args.warmup, [stream, stream2])
    ctx2.close()
    e2e_s = max_over_ranks(pipe_s, world)
    e2e = {"value": whole_job_rate(n_fits * args.steps, world, e2e_s), "unit": "fits/s",
           "h2d_bytes_per_step": n_words * 4, "d2h_bytes_per_step": int(statistics.mean(pipe_d2h)) + 200,
           "pipelined": "two contexts taking batches in turn (copies of one overlap the other's kernel)",
           "p50_us": 1e6 * float(np.percentile(lat, 50)), "p99_us": 1e6 * float(np.percentile(lat, 99)),
           "latency": "one batch at a time: H2D, kernel, D2H",
           "serial_value": whole_job_rate(n_fits * len(lat), world, max_over_ranks(sum(lat), world)),
           "events_per_s": n_events * world * args.steps / e2e_s}
    ctx.close()
    clocks.__exit__()

    if rank != 0:
        dist.barrier()
        return
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    # the timed region is short (tens of ms): its samples, and those of the
    # whole GPU section (timed steps, plain, end-to-end runs) beside them
    clk = clocks.summary(t_timed0 - 0.02, t_timed1 + 0.02)
    clk["gpu_section"] = clocks.summary()
    mhz = clk["sm_max_mhz"] or 2070.0
    peak_macs = sms * IMAD_LANES_PER_SM * mhz * 1e6 / 1e12
    achieved = MACS_PER_FIT * n_fit4 / (step_ms / 1e3) / 1e12
    line = {
        "metric": "track fits/s", "value": value, "unit": "fits/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32/int64", "data": "synthetic (seeded generator, workload shape of the config)",
        "config": {"workload": workload_desc(cfg, n_fits, n_words), "mode": "persistent",
                   "graph": True, "autotuned": tuned, "l2": "256 MB flush written between steps",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "events_per_s": n_events * world / (step_ms / 1e3),
        "latency_us": {"p50": 1e3 * float(np.percentile(times, 50)),
                       "p99": 1e3 * float(np.percentile(times, 99))},
        "tracks_per_step": stats["n_tracks"], "status": stats["status"],
        "phase_us": dict(zip(["word_scan", "road_decode", "cross_road_flags", "fit_cut_local_warrior",
                              "cross_road_warrior", "output"],
                             [round(x / 1e3, 1) for x in stats["phase_ns"]])),
        "e2e": e2e,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak_macs, "unit": "T int32 MAC/s",
                     "frac": achieved / peak_macs, "traffic": measured_traffic(args.workload),
                     "peak_measured": peak["imad"] / 1e12,
                     "units": "%d distinct fits x %d multiply-adds per launch" % (n_fit4, MACS_PER_FIT),
                     "note": "peak = SMs x 64 multiply-add lanes x max clock; peak_measured: "
                             "svt_measure_int_peak (mad.lo.u32 chains on every SM); "
                             "per combination the same time is %.2f T MAC/s"
                             % (MACS_PER_FIT * n_fits / (step_ms / 1e3) / 1e12)},
        "int_peak_tops": {k: round(v / 1e12, 2) for k, v in peak.items()},
        "gpu_launches": launches * args.steps,
        "clocks": clk,
    }
    if plain:
        line["plain"] = plain
    if world == 1 and not args.no_subs:
        for name in ("scaled", "uneven"):
            if name != args.workload:
                line[name] = sub_workload(B, torch, synth, name, consts, local, args)
    if not args.no_sweep and world == 1:
        line["packet_sweep"] = packet_sweep(B, torch, synth, consts, local)
        line["loopback"] = loopback_loop(synth, consts, local)
    if not args.no_serve and world == 1:
        line["serving"] = run_serving(B, synth, consts, load_cut("serving"),
                                      (1e4, 3e4, 1e5, 3e5, 1e6), args.serve_requests)
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(batch, consts, cut)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()


# --------------------------------------------------------------------------
# reference arm: the CPU oracle as it stands
# --------------------------------------------------------------------------

def reference_arm(args):
    rank, local, world = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1312_0917_gb300 import synth
    oracle.build()
    cfg = synth.CONFIGS[args.workload]
    batch = synth.make_batch(cfg, seed=0)
    consts = synth.make_constants(0)
    cut = load_cut(args.workload)
    # bounded sample per step: one event per host core (the oracle's
    # event-parallel driver), at least enough events for about a second
    cores = os.cpu_count() or 1
    per_ev = batch.n_fits / batch.n_events
    n_ev = max(1, min(batch.n_events, max(cores, int(cores * 2e6 / per_ev))))
    words = batch.event_slice(0, n_ev)
    fits = int(np.prod(batch.roads["n"][batch.roads["event"] < n_ev], axis=1).sum())
    for _ in range(args.warmup):
        oracle.run_mt(words, consts, cut)
    t, threads = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        rc, out, times = oracle.run_mt(words, consts, cut)
        t.append(time.perf_counter() - t0)
        threads = times["threads"]
        assert rc == 0
    value = fits * len(t) / sum(t)
    sample = ("first %d events of the %s batch (%d combinations) per step, the oracle's "
              "event-parallel driver" % (n_ev, cfg.name, fits))
    line = {"impl": "reference", "metric": "track fits/s", "value": value, "unit": "fits/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(t) / len(t), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32/int64", "data": "synthetic",
            "config": {"workload": workload_desc(cfg, batch.n_fits, len(batch.words)),
                       "mode": "cpu oracle, events over host cores"},
            "cpu_baseline": {"value": value, "unit": "fits/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "fits/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        reference_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
