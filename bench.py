"""Benchmark of the triplet merge tree path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step is one pass of the whole hot path over the 1024^3 lognormal field
exp(0.8 g) (g a Gaussian random field with P(k) ~ k^-2, float32, seed 1+rank):
  mt_build_triplets    (validate, init, descent jumping, merge, repair)
  mt_persistence_pairs (ordered pair compaction; synchronises)
  mt_components_at     (labels of G_t at the field's median value)
The field (4 GiB) and triplets (8 GiB) are far larger than the 129 MB L2, so
no flush is needed between steps. Timing uses CUDA events on the launching
stream, W untimed warm-up steps, barrier + synchronize on both sides, max over
ranks. One JSON line is printed by rank 0.

Multi-GPU: the single-field path does not shard; N ranks run N independent
replicas (one field each, no collective on the data path) and `value` is the
vertices of all ranks / the slowest rank's time ("scaling": "weak").

--impl reference times the CPU oracle (the plain sort + union-find sweep of
Section 2.1) on a bounded crop of the same field on the host cores.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "merge-tree Mvertices/s at 1024^3 f32 (exact); batched fields/s; serve p50/p99 ms"
UNIT = "Mvertices/s"
WORKLOAD = "lognorm1024"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--side", type=int, default=1024, help="cube side (1024 = the benchmark workload)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-side", type=int, default=256, help="side of the crop the CPU oracle times")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=5.0)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.t: threading.Thread | None = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, val in zip(names, p[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ algorithmic bytes
def algorithmic_bytes(n: int, shape, npairs: int, tile=(16, 16, 32)) -> dict:
    """Bytes the method must move per step, by kernel:
      tile    init: read f (4n) + write W (8n); plus two triplet reads per
              merged edge inside the tiles, 16 (E' - C)
      merge   (k_cross) two triplet reads per edge between tiles: 16 C
      repair  read + write W (16n)
      pairs   scan W (8n) + write pairs (8 npairs)
      labels  read f (4n) + W (8n), write labels (4n)
    E' = E - (n - #minima) (edges that are not steepest-descent seeds: the
    per-edge cost of the edge loop of Algorithm 1) and C the edges between
    tiles; tile + merge together are 12n + 16E'.
    """
    nz, ny, nx = shape
    tz, ty, tx = tile
    E = 3 * n - (nx * ny + ny * nz + nz * nx)
    nmin = npairs + 1
    Ep = E - (n - nmin)
    C = ((nx - 1) // tx) * ny * nz + ((ny - 1) // ty) * nx * nz + ((nz - 1) // tz) * nx * ny
    return {"tile": 12 * n + 16 * (Ep - C), "merge": 16 * C, "repair": 16 * n, "pairs": 8 * n + 8 * npairs,
            "labels": 16 * n, "E": E, "E_prime": Ep, "cross_edges": C}


def traffic_record(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or
    None if there is none or the kernel source changed since it was taken."""
    import hashlib

    prof = os.path.join(ROOT, "profiles", f"traffic_{kernel}_{WORKLOAD}.json")
    src = os.path.join(ROOT, "paper_2301_10838_gb300", "csrc", "mt_build.cu")
    try:
        with open(prof) as fh:
            rec = json.load(fh)
        with open(src, "rb") as fh:
            h = hashlib.sha256(fh.read()).hexdigest()[:16]
    except (OSError, ValueError):
        return None
    return rec.get("dram_bytes_per_launch") if rec.get("mt_build_cu_sha256_16") == h else None


def max_over_ranks(value: float, world: int, device) -> float:
    """The slowest rank's time (replicas: the job ends with the last one)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist

    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: int, steps: int, ms_total: float) -> float:
    """Whole-job throughput in millions of units per second: every rank
    processes its own units each step; the job time is the slowest rank's."""
    return world * units_per_rank * steps / (ms_total / 1e3) / 1e6


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ------------------------------------------------------------------ ours
def field_digest(f) -> str:
    """sha256 of the field's bytes (rank 0's field), so that a run can be
    tied to the exact input; read back in 256 MiB slices."""
    import hashlib

    h = hashlib.sha256()
    flat = f.reshape(-1)
    step = 1 << 26
    for i in range(0, flat.numel(), step):
        h.update(flat[i:i + step].cpu().numpy().tobytes())
    return h.hexdigest()


def run_ours(args):
    import numpy as np
    import torch

    import paper_2301_10838_gb300 as mt
    from paper_2301_10838_gb300 import fields

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    side = args.side
    f = fields.named_field(WORKLOAD, seed=1 + rank, side=side, device=str(dev))
    f = f.contiguous()
    n = f.numel()
    shape = tuple(f.shape)
    t_thr = float(f.reshape(-1)[:: 4099].float().median())
    field_sha = field_digest(f)
    W = torch.empty(n, dtype=torch.int64, device=dev)
    ws = mt.workspace(mt.grid_of(f), device=dev)
    labels = torch.empty(n, dtype=torch.int32, device=dev)
    # pair capacity: the number of local minima minus one, known after one build
    mt.mt_build_triplets(f, W, ws)
    probe = torch.empty((0, 2), dtype=torch.int32, device=dev)
    npairs, _ = mt.mt_persistence_pairs(f, W, probe, ws, allow_partial=True)
    pairs = torch.empty((npairs, 2), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        mt.mt_build_triplets(f, W, ws)
        np_, root = mt.mt_persistence_pairs(f, W, pairs, ws)
        mt.mt_components_at(f, W, t_thr, labels, ws)
        return np_

    for _ in range(args.warmup):
        step()
    mt.mt_sync_status(ws)

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize(dev)

    clocks = ClockSampler(dev.index if dev.index is not None else 0)
    mt.mt_trace_enable(True)
    mt.mt_trace_read(reset=True)
    launches0 = mt.mt_kernel_launches()
    barrier()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    barrier()
    clk = clocks.stop()
    launches = mt.mt_kernel_launches() - launches0
    phases = mt.mt_trace_read(reset=True)
    mt.mt_trace_enable(False)
    mt.mt_sync_status(ws)
    ms_total = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    ms_step = ms_total / args.steps
    value = job_rate(world, n, args.steps, ms_total)

    # roofline of the dominant kernel family from the live phase timing
    peak, peak_kind = measured_peaks()
    ab = algorithmic_bytes(n, shape, npairs)
    dom = max((k for k in phases if k in ab), key=lambda k: phases[k][1])
    calls, tot = phases[dom]
    achieved = ab[dom] / (tot / calls / 1e3) / 1e9
    traffic = traffic_record(dom) if side == 1024 else None
    step_bytes = sum(ab[k] for k in ("tile", "merge", "repair", "pairs", "labels"))

    # end to end through the public API with pinned host buffers: every step
    # copies its field in and its triplets, pairs and labels out. Three sets of
    # device buffers and separate copy streams let step k's copies out overlap
    # step k+1's kernels, and step k+1's copy in start before step k-1's
    # copies out have finished.
    e2e = None
    if not args.no_e2e:
        h_f = torch.empty(shape, dtype=torch.float32, pin_memory=True)
        h_f.copy_(f)
        h_W = torch.empty(n, dtype=torch.int64, pin_memory=True)
        h_lab = torch.empty(n, dtype=torch.int32, pin_memory=True)
        h_pairs = torch.empty((npairs, 2), dtype=torch.int32, pin_memory=True)
        depth = 3
        bufs = [(f, W, labels, pairs, ws)]
        for _ in range(depth - 1):
            bufs.append((torch.empty_like(f), torch.empty_like(W), torch.empty_like(labels),
                         torch.empty_like(pairs), torch.empty_like(ws)))
        s_in, s_cmp, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev), torch.cuda.Stream(dev)
        done = [torch.cuda.Event() for _ in range(depth)]  # buffers of slot i free again
        for ev in done:
            ev.record(s_out)
        k_e2e = max(3, args.steps)

        loaded = [None] * depth

        def prefetch(k):
            df = bufs[k % depth][0]
            s_in.wait_event(done[k % depth])
            with torch.cuda.stream(s_in):
                df.copy_(h_f, non_blocking=True)
                ev = torch.cuda.Event()
                ev.record(s_in)
            loaded[k % depth] = ev

        def e2e_step(k, last):
            df, dW, dl, dp, dws = bufs[k % depth]
            s_cmp.wait_event(loaded[k % depth])
            mt.mt_build_triplets(df, dW, dws, stream=s_cmp)
            mt.mt_components_at(df, dW, t_thr, dl, dws, stream=s_cmp)
            built = torch.cuda.Event()
            built.record(s_cmp)
            s_out.wait_event(built)
            with torch.cuda.stream(s_out):
                h_W.copy_(dW, non_blocking=True)
                h_lab.copy_(dl, non_blocking=True)
            if not last:
                prefetch(k + 1)  # the next field's upload overlaps this step
            np_, _ = mt.mt_persistence_pairs(df, dW, dp, dws, stream=s_cmp)
            paired = torch.cuda.Event()
            paired.record(s_cmp)
            s_out.wait_event(paired)
            with torch.cuda.stream(s_out):
                h_pairs[:np_].copy_(dp[:np_], non_blocking=True)
                done[k % depth].record(s_out)

        prefetch(0)
        e2e_step(0, True)
        torch.cuda.synchronize(dev)
        barrier()
        t0 = time.perf_counter()
        prefetch(0)
        for k in range(k_e2e):
            e2e_step(k, k + 1 == k_e2e)
        torch.cuda.synchronize(dev)
        e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3, world, dev)
        e2e = {"value": round(job_rate(world, n, k_e2e, e_ms), 1), "unit": UNIT,
               "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 8 * n + 8 * npairs + 4 * n,
               "ms_per_step": round(e_ms / k_e2e, 3), "steps": k_e2e,
               "timing": "host wall clock around K pipelined steps (copies on their own streams), synchronised"}
        del h_f, h_W, h_lab, h_pairs, bufs

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(f, args.cpu_side)
    del W, labels, pairs, ws
    f = None
    torch.cuda.empty_cache()
    batch = None if args.no_batch else bench_batch(args, dev)
    serve = None if args.no_serve else bench_serve(args, dev)

    if rank == 0:
        out = {
            "metric": METRIC,
            "value": round(value, 1),
            "unit": UNIT,
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": round(ms_step, 3),
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic",
            "config": {
                "workload": WORKLOAD if side == 1024 else f"{WORKLOAD}@{side}^3",
                "grid": [shape[2], shape[1], shape[0]],
                "field": "exp(0.8 g), g unit-variance GRF P(k)~k^-2, float32, seed 1+rank",
                "field_sha256": field_sha,
                "step": "mt_build_triplets + mt_persistence_pairs + mt_components_at(median)",
                "threshold": t_thr,
                "npairs": npairs,
                "l2": "inputs larger than L2 (4 GiB field, 8 GiB triplets); no flush",
                "parallelism": f"replicas{world}" if world > 1 else "single",
            },
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "traffic": traffic, "algorithmic_bytes_per_launch": ab[dom],
                         "ms_per_launch": round(tot / calls, 3)},
            "step_roofline": {"algorithmic_bytes": step_bytes,
                              "frac": round(step_bytes / (ms_step / 1e3) / 1e9 / peak, 4)},
            "phases_ms_per_step": {k: round(v[1] / args.steps, 3) for k, v in phases.items()},
            "clocks": clk,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "cpu_baseline": cpu,
            "batch": batch,
            "serve": serve,
        }
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def bench_batch(args, dev):
    """512 fields of uneven sizes (sides log-uniform in [16, 128] per axis,
    half white noise, half GRF P(k)~k^-3): one CUDA-graph replay of the
    batched build + pairs against 512 plain per-field calls on one stream,
    same outputs."""
    import numpy as np
    import torch

    import paper_2301_10838_gb300 as mt
    from paper_2301_10838_gb300 import fields
    from paper_2301_10838_gb300.batch import Batch

    shapes = fields.batch_shapes(512, 16, 128, seed=7)
    flds = [fields.batch_field(i, s) for i, s in enumerate(shapes)]
    b = Batch(shapes, device=dev)
    b.load(flds)
    variant = b.tune()
    b.capture()
    st = torch.cuda.current_stream(dev)
    for _ in range(max(3, args.warmup)):
        b.launch()
    torch.cuda.synchronize(dev)
    reps = max(5, args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        b.launch()
    e1.record(st)
    torch.cuda.synchronize(dev)
    ms_batch = e0.elapsed_time(e1) / reps
    # plain: one field at a time through the single-field calls
    ins, outs = [], []
    for i, s in enumerate(shapes):
        fi = b.field(i)
        W = torch.empty(fi.numel(), dtype=torch.int64, device=dev)
        P = torch.empty((fi.numel(), 2), dtype=torch.int32, device=dev)
        ws = mt.workspace(mt.grid_of(fi), device=dev)
        ins.append(fi)
        outs.append((W, P, ws))

    def plain():
        ks = []
        for fi, (W, P, ws) in zip(ins, outs):
            mt.mt_build_triplets(fi, W, ws)
            ks.append(mt.mt_persistence_pairs(fi, W, P, ws)[0])
        return ks

    plain()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    prep = max(2, args.steps // 2)
    for _ in range(prep):
        ks = plain()
    torch.cuda.synchronize(dev)
    ms_plain = (time.perf_counter() - t0) * 1e3 / prep
    same = all(int(b.npairs[i]) == ks[i] and torch.equal(b.results(i)[0], outs[i][0]) for i in range(len(shapes)))
    nv = sum(int(np.prod(s)) for s in shapes)
    return {"fields": len(shapes), "vertices": nv, "variant": variant,
            "fields_per_s_batched": round(len(shapes) / (ms_batch / 1e3), 1),
            "fields_per_s_plain": round(len(shapes) / (ms_plain / 1e3), 1),
            "ms_per_batch": round(ms_batch, 3), "ms_plain_512": round(ms_plain, 3),
            "speedup": round(ms_plain / ms_batch, 2), "identical_outputs": bool(same),
            "timing": "batched: CUDA-graph replays timed with CUDA events; plain: 512 x (mt_build_triplets + "
                      "mt_persistence_pairs), host wall clock (each pairs call synchronises)"}


def bench_serve(args, dev):
    """Poisson request stream (200 req/s) of GRF fields (P(k)~k^-2.5, unit
    variance, cubic sides log-uniform in [32, 384]), each asking for pairs and
    labels at a random threshold; p50/p99 latency from submission to results
    in host memory. A pool of 24 distinct fields is reused cyclically (each
    request has its own threshold and output buffers). Also: the same request
    list submitted at once (saturated throughput) against the plain
    single-field path run back to back on one stream."""
    import numpy as np
    import torch

    import paper_2301_10838_gb300 as mt
    from paper_2301_10838_gb300 import fields
    from paper_2301_10838_gb300.serve import Server

    stream = fields.serve_stream(200.0, args.serve_seconds, 32, 384, seed=11)
    pool_sides = [r.side for r in stream[:24]]
    pool = []
    for k, side in enumerate(pool_sides):
        g = fields.grf((side, side, side), -2.5, 7000 + k, device=str(dev))
        pool.append(g.cpu().pin_memory())
        del g
    torch.cuda.empty_cache()
    maxn = max(p.numel() for p in pool)
    R = 48
    ring = [(torch.empty((maxn // 2 + 1, 2), dtype=torch.int32, pin_memory=True),
             torch.empty(maxn, dtype=torch.int32, pin_memory=True)) for _ in range(R)]
    srv = Server(hbm_budget_bytes=24 << 30, max_slots=6, device=dev.index or 0)
    try:
        # warm-up
        for k in range(4):
            P, L = ring[k]
            srv.wait(srv.submit(pool[k], 0.0, pairs=P, labels=L))
        # open-loop Poisson arrivals
        import threading

        results = [None] * len(stream)
        tickets = [None] * len(stream)
        t_start = time.perf_counter()

        def submitter():
            for i, r in enumerate(stream):
                delay = t_start + r.arrival_s - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                P, L = ring[i % R]
                tickets[i] = srv.submit(pool[i % len(pool)], r.threshold, pairs=P, labels=L)

        th = threading.Thread(target=submitter)
        th.start()
        for i in range(len(stream)):
            while tickets[i] is None:
                time.sleep(0.0002)
            results[i] = srv.wait(tickets[i])
        th.join()
        wall = time.perf_counter() - t_start
        lat = np.array([r["latency_s"] for r in results]) * 1e3
        nvert = sum(pool[i % len(pool)].numel() for i in range(len(stream)))
        # saturated: every request of the list submitted at once
        nsat = min(len(stream), 240)
        t0 = time.perf_counter()
        tks = []
        for i in range(nsat):
            P, L = ring[i % R]
            tks.append(srv.submit(pool[i % len(pool)], stream[i].threshold, pairs=P, labels=L))
            if len(tks) > R - 8:  # keep ring buffers unshared
                srv.wait(tks.pop(0))
        for tk in tks:
            srv.wait(tk)
        sat = nsat / (time.perf_counter() - t0)
    finally:
        srv.close()
    # plain single-field path, back to back on one stream, same work
    ws_cache = {}
    t0 = time.perf_counter()
    nplain = min(len(stream), 120)
    for i in range(nplain):
        h = pool[i % len(pool)]
        fd = h.to(dev, non_blocking=True)
        n = fd.numel()
        if n not in ws_cache:
            ws_cache[n] = (torch.empty(n, dtype=torch.int64, device=dev),
                           torch.empty((n // 2 + 1, 2), dtype=torch.int32, device=dev),
                           torch.empty(n, dtype=torch.int32, device=dev), mt.workspace(mt.grid_of(fd), device=dev))
        W, Pd, Ld, ws = ws_cache[n]
        mt.mt_build_triplets(fd, W, ws)
        k, _ = mt.mt_persistence_pairs(fd, W, Pd, ws)
        mt.mt_components_at(fd, W, stream[i].threshold, Ld, ws)
        P, L = ring[i % R]
        P[:k].copy_(Pd[:k])
        L[:n].copy_(Ld)
    torch.cuda.synchronize(dev)
    plain = nplain / (time.perf_counter() - t0)
    return {"requests": len(stream), "rate_hz": 200.0, "seconds": args.serve_seconds,
            "p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
            "throughput_req_s": round(len(stream) / wall, 1),
            "mvertices_s_offered": round(nvert / wall / 1e6, 1),
            "saturated_fields_per_s": round(sat, 1), "plain_fields_per_s": round(plain, 1),
            "speedup_saturated_vs_plain": round(sat / plain, 2), "slots": 6, "pool_fields": len(pool)}


def cpu_baseline(f_dev, side: int):
    """The CPU oracle, as it stands, on a side^3 crop of the same field: one
    host thread runs sort + sweep, pairs and labels."""
    import numpy as np

    import oracle

    crop = f_dev[:side, :side, :side].contiguous().cpu().numpy()
    t_thr = float(np.median(crop[::7, ::7, ::7]))
    t0 = time.perf_counter()
    W = oracle.merge_tree(crop)
    oracle.pairs(W)
    oracle.components(crop, t_thr)
    dt = time.perf_counter() - t0
    return {"value": round(crop.size / dt / 1e6, 3), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{side}^3 corner crop of the benchmark field ({crop.size} vertices), "
                      f"sort+sweep+pairs+labels, {dt:.2f} s"}


# ------------------------------------------------------------- reference
def run_reference(args):
    """The CPU oracle timed on the host cores on a bounded crop of the same
    workload, with our arm's metric, unit and direction."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    import numpy as np

    import oracle
    from paper_2301_10838_gb300 import fields

    side = min(args.cpu_side, args.side)
    # the same generator and seed as our arm's rank 0; on a GPU machine the field
    # is synthesised on the device exactly as our arm does (input generation
    # only) and a corner crop is copied to the host
    import torch

    if torch.cuda.is_available():
        full = fields.named_field(WORKLOAD, seed=1, side=args.side, device="cuda")
        crop = full[:side, :side, :side].contiguous().cpu().numpy()
        gen = f"generated at {args.side}^3 on the device"
        del full
        torch.cuda.empty_cache()
    else:
        full = fields.named_field(WORKLOAD, seed=1, side=min(args.side, 2 * side), device="cpu")
        crop = np.ascontiguousarray(full[:side, :side, :side])
        gen = f"generated at {full.shape[0]}^3 on the host"
    t_thr = float(np.median(crop[::7, ::7, ::7]))

    def step():
        W = oracle.merge_tree(crop)
        oracle.pairs(W)
        oracle.components(crop, t_thr)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = crop.size * args.steps / dt / 1e6
    sample = f"{side}^3 corner crop of the {WORKLOAD} field ({gen}), one host thread"
    out = {
        "impl": "reference",
        "metric": METRIC,
        "value": round(value, 3),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample,
                   "step": "oracle merge_tree + pairs + components(median)"},
        "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
