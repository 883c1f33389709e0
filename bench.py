"""Benchmark of the MNS fractal coder on GB300.

Default workload (batch40x512): one step = the whole hot path over one batch: the
MNS quadtree encode (moments, phase 1, phase 2, split, stream packing) of the
ten 512x512 synthetic images shaped like the paper's test images (8 scenes +
2 Voronoi images) at each RMS threshold of the sweep {4, 8, 12, 16} -- 40
encodes in one persistent launch -- followed by the 10-iteration decode of
all 40 streams.  The step is captured in CUDA graphs and replayed; L2 is
flushed (a 256 MiB write) before every timed step because the inputs
(10.5 MB) are far smaller than L2.

Other workloads (`--workload`), one JSON line each:
  one256      one 256x256 image, MNS 16->4, RMS 8, decode 10 iterations
  exhaustive  exhaustive search (8 isometries, domain step 4, 8x8 ranges) of a
              512x512 and a 1024x1024 image: tensor-core and CUDA-core engines
  mixed512    512 images of mixed sides {256..2048} in one persistent launch per
              pass (CUDA graphs, autotuned launch mapping), MNS 32->4, RMS 8,
              decode 8 iterations; against per-image launches with the same output
  serving     serving: Poisson arrivals (2000/s), 80 % encode / 20 % decode,
              sides log-uniform in [128, 4096], through the library's request
              server; p50/p99 latency and Mpixel/s against a per-request loop

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload batch40x512|one256|exhaustive|mixed512|serving]

With N > 1 (torchrun) every rank runs the same workload on its own GPU
(replicas, weak scaling); rank 0 prints one JSON line.  `--impl reference`
times the CPU oracle (the plain restatement of the paper's algorithm) on the
host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

THRESHOLDS = [4.0, 8.0, 12.0, 16.0]
METRIC = "MNS encode Mpixel/s & range-domain fits/s (bit-exact); served p50/p99 latency"
L2_BYTES = 129 << 20


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# --------------------------------------------------------------------------
# Workloads

class Spec:
    """A batched workload: items (image, mode, bmax, bmin, thr), decode iterations."""

    def __init__(self, name, desc, items, iters, autotune=False, plain=False):
        self.name, self.desc, self.items, self.iters = name, desc, items, iters
        self.autotune, self.plain = autotune, plain

    @property
    def pixels(self):
        return sum(im.size for im, *_ in self.items)


def _gen(args):
    kind, n, seed = args
    return synth.gaussian_scene(n, seed) if kind == "g" else synth.voronoi(n, seed)


def gen_images(specs, workers=None):
    """Generate synthetic images in a process pool (spawned: safe before or
    after CUDA initialisation)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    if len(specs) < 8:
        return [_gen(s) for s in specs]
    workers = workers or min(16, os.cpu_count() or 1)
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_gen, specs, chunksize=4))


def make_spec(name):
    if name == "one256":
        return Spec(name, "one256: 256x256 scene seed 0, MNS 16->8->4, RMS 8 + decode 10 it",
                    [(synth.scene256_image(), "mns", 16, 4, 8.0)], 10, autotune=True)
    if name == "batch40x512":
        imgs = [im for _, im in synth.scenes512_images()]
        return Spec(name, "batch40x512: 10 x 512x512 (8 scenes seeds 1-8 + 2 Voronoi 101/102) x RMS {4,8,12,16}, "
                          "MNS 32->4 + decode 10 it",
                    [(im, "mns", 32, 4, t) for t in THRESHOLDS for im in imgs], 10)
    if name == "mixed512":
        sides = synth.mixed_sides()
        imgs = gen_images([("g", int(s), 1000 + i) for i, s in enumerate(sides)])
        return Spec(name, "mixed512: 512 scenes, sides {256,512,1024,2048} w .4/.3/.2/.1 (rng 4, seed 1000+i), "
                          "MNS 32->4, RMS 8 + decode 8 it, one persistent launch per pass",
                    [(im, "mns", 32, 4, 8.0) for im in imgs], 8, autotune=True, plain=True)
    raise ValueError(name)


# --------------------------------------------------------------------------
# Measurement helpers

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")

    def __init__(self, gpu_id: str):
        self.gpu = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons, busy = [], [], set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 10:
                continue
            try:
                util = float(parts[9])
                smax.append(float(parts[2]))
                if util <= 0:
                    continue
                sm.append(float(parts[1]))
            except ValueError:
                continue
            busy += 1
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples_under_load": busy, "samples": len(self.lines)}


def profile_record(kernel_key: str):
    """A kernel's record from its committed ncu summary (DRAM bytes and warp
    instructions per launch), valid only while the kernel's sources are
    unchanged (their hashes are recorded beside it); None otherwise."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            prof = json.load(f)
        ent = prof[kernel_key]
        for src, h0 in ent["sources"].items():
            h = hashlib.sha256(open(os.path.join(ROOT, src), "rb").read()).hexdigest()[:16]
            if h != h0:
                return None
        return ent
    except Exception:
        return None


def traffic_from_profile(kernel_key: str):
    """DRAM bytes per launch of a kernel (profile_record)."""
    ent = profile_record(kernel_key)
    return float(ent["bytes_per_launch"]) if ent else None


def issue_from_profile(kernel_key: str, dur_ms: float, clocks: dict, sms: int):
    """The kernel's instruction issue rate against the GPU's: warp
    instructions per launch (ncu, profile_record) / the launch's duration,
    over one warp instruction per scheduler per clock (4 per SM) at the SM
    clock sampled during the timed region."""
    ent = profile_record(kernel_key)
    if not ent or not ent.get("inst_per_launch") or not dur_ms:
        return None
    mhz = (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz")
    if not mhz:
        return None
    inst = float(ent["inst_per_launch"])
    ach = inst / (dur_ms * 1e-3)
    peak = 4.0 * sms * mhz * 1e6
    return {"warp_instructions_per_launch": inst, "achieved_per_s": round(ach, 1), "peak_per_s": round(peak, 1),
            "frac": round(ach / peak, 4),
            "source": "smsp__inst_executed.sum of the kernel's committed ncu capture (valid while its sources are "
                      "unchanged); peak = SMs x 4 schedulers x the SM clock sampled under load"}


def gpu_uuid(torch, dev):
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        return str(dev.index or 0)


def kernel_table(rows_per_step):
    """[(name, ms)] lists of several steps -> per-kernel launches/step, mean ms per launch, share."""
    agg = {}
    for rows in rows_per_step:
        for name, ms in rows:
            a = agg.setdefault(name, [0, 0.0])
            a[0] += 1
            a[1] += ms
    steps = max(1, len(rows_per_step))
    total = sum(v[1] for v in agg.values()) or 1.0
    return {k: {"launches_per_step": v[0] // steps, "ms_per_launch": round(v[1] / v[0], 5),
                "share": round(v[1] / total, 4)} for k, v in sorted(agg.items(), key=lambda kv: -kv[1][1])}


def dist_setup():
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    return world, rank, torch.device("cuda", local)


def max_over_ranks(world, dev, v):
    """The slowest rank's value (replicas: the job ends with the last rank)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    t = torch.tensor([v], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, dev, ms_per_step_local, units_per_rank_step):
    """Whole-job throughput of `world` replicas: every rank processes the same
    units per step; the job's step time is the slowest rank's."""
    ms = max_over_ranks(world, dev, ms_per_step_local)
    return ms, world * units_per_rank_step / (ms * 1e-3)


def dist_finish(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()


# --------------------------------------------------------------------------
# CPU oracle (the reference arm and the cpu_baseline object)

def time_oracle(items, iters, budget_s: float, threads: int):
    """Encode + decode as many items as fit in the budget, spread over
    `threads` host threads.  Returns (Mpixel/s, items done, seconds)."""
    from concurrent.futures import ThreadPoolExecutor

    from oracle import oracle as O

    O.lib()

    def one(item):
        im, mode, bmax, bmin, t = item
        p = O.make_params(mode, bmax, bmin, t)
        leaves, _, _ = O.encode(im, p)
        O.decode(leaves, im.shape[1], im.shape[0], p, iters)
        return im.size

    t0 = time.perf_counter()
    done_px = done = i = 0
    with ThreadPoolExecutor(max_workers=threads) as ex:
        while time.perf_counter() - t0 < budget_s:
            chunk = [items[(i + j) % len(items)] for j in range(threads)]
            i += threads
            for px in ex.map(one, chunk):
                done_px += px
                done += 1
    dt = time.perf_counter() - t0
    return done_px / dt / 1e6, done, dt


def time_oracle_exhaustive(img, budget_s: float, threads: int, dom_step=4, isos=8):
    """Exhaustive search of sampled 8x8 ranges of `img` for `budget_s`
    seconds.  Returns (fits/s, ranges done, seconds)."""
    from concurrent.futures import ThreadPoolExecutor

    from oracle import oracle as O

    O.lib()
    p = O.make_params("exhaustive", 8, 8, 8.0, dom_step=dom_step, isometries=isos)
    H, W = img.shape
    nd = ((W - 16) // dom_step + 1) * ((H - 16) // dom_step + 1)
    rng = np.random.default_rng(7)

    def one(k):
        xs = rng.integers(0, W // 8, size=4) * 8
        ys = rng.integers(0, H // 8, size=4) * 8
        O.search_ranges(img, p, xs, ys, np.full(4, 8))
        return 4

    t0 = time.perf_counter()
    done = 0
    with ThreadPoolExecutor(max_workers=threads) as ex:
        while time.perf_counter() - t0 < budget_s:
            done += sum(ex.map(one, range(threads)))
    dt = time.perf_counter() - t0
    return done * nd * isos / dt, done, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    threads = os.cpu_count() or 1
    step_s = max(0.5, min(args.ref_step_s, 150.0 / max(1, args.steps + args.warmup)))
    if args.workload == "exhaustive":
        img = synth.exhaustive_images()[1][1]
        for _ in range(args.warmup):
            time_oracle_exhaustive(img, min(0.5, step_s), threads)
        vals = [time_oracle_exhaustive(img, step_s, threads)[0] for _ in range(args.steps)]
        value, unit, desc = statistics.mean(vals), "fits/s", "exhaustive search, sampled 8x8 ranges of the 1024x1024 image"
        ms, metric = None, "exhaustive-search range-domain fits/s (bit-exact)"
    elif args.workload == "serving":
        print(json.dumps({"impl": "reference", "unavailable": "the serving workload has no CPU counterpart; "
                                                              "the oracle arm covers one256-mixed512"}), flush=True)
        return 0
    else:
        spec = make_spec(args.workload)
        for _ in range(args.warmup):
            time_oracle(spec.items, spec.iters, min(0.5, step_s), threads)
        vals = [time_oracle(spec.items, spec.iters, step_s, threads)[0] for _ in range(args.steps)]
        value, unit, desc = statistics.mean(vals), "Mpixel/s", spec.desc
        ms, metric = round(spec.pixels / (value * 1e6) * 1e3, 3), METRIC
    line = {
        "impl": "reference", "metric": metric, "value": round(value, 3), "unit": unit,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": desc, "sample": f"{step_s:g} s of oracle work per step"},
        "cpu_baseline": {"value": round(value, 3), "unit": unit, "cores": threads, "kind": "oracle",
                         "sample": f"items of the workload, {step_s:g} s per step on {threads} threads"},
        "e2e": {"value": round(value, 3), "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# GPU arm: batched encode + decode (one256, batch40x512, mixed512)

def run_batched(args, spec: Spec):
    import torch

    world, rank, dev = dist_setup()
    import paper_1501_02894_gb300 as fic

    fic.lib()
    items = spec.items
    n = len(items)
    pixels = spec.pixels
    iters = spec.iters
    plist = [fic.params(m, bmax, bmin, t) for _, m, bmax, bmin, t in items]
    # one pinned host arena and one device arena for the batch's images, one
    # device arena for all streams' records and info blocks, one for the
    # decoded images: the end-to-end pass moves each with a single copy
    offs = np.cumsum([0] + [it[0].size for it in items])
    host_in = torch.empty(int(offs[-1]), dtype=torch.uint8).pin_memory()
    for it, o in zip(items, offs):
        host_in[int(o): int(o) + it[0].size].copy_(torch.from_numpy(it[0].reshape(-1)))
    dev_in = host_in.to(dev)
    dimgs = [dev_in[int(o): int(o) + it[0].size].view(it[0].shape) for it, o in zip(items, offs)]
    caps = [fic.stream_sizes(it[0].shape[1], it[0].shape[0], p)[1] for it, p in zip(items, plist)]
    roffs = np.cumsum([0] + [16 * c for c in caps])
    rec_arena = torch.empty(int(roffs[-1]), dtype=torch.uint8, device=dev)
    info_arena = torch.zeros((n, fic.INFO_WORDS), dtype=torch.int32, device=dev)
    outs_s = [fic.Stream(it[0].shape[1], it[0].shape[0], p, dev, records=rec_arena[int(a): int(b)], info=info_arena[i])
              for i, (it, p, a, b) in enumerate(zip(items, plist, roffs[:-1], roffs[1:]))]
    dec_arena = torch.empty(int(offs[-1]), dtype=torch.uint8, device=dev)
    dec_outs = [dec_arena[int(o): int(o) + it[0].size].view(it[0].shape) for it, o in zip(items, offs)]
    stream = torch.cuda.Stream(dev)
    flush_l2 = pixels < 2 * L2_BYTES
    flush = torch.empty(256 << 20 if flush_l2 else 1, dtype=torch.uint8, device=dev)

    with torch.cuda.stream(stream):
        enc = fic.EncodePlan(dimgs, plist, outs=outs_s, stream=stream)
        enc.run(stream)
        dec = fic.DecodePlan(enc.outs, outs=dec_outs, stream=stream)
        dec.run(iters, stream)
    stream.synchronize()
    tuning = None
    if spec.autotune:
        with torch.cuda.stream(stream):
            te = enc.autotune(reps=3, stream=stream)
            td = dec.autotune(iters, reps=3, stream=stream)
        tuning = {"encode": te, "decode": td}
    nrec, fits = [], 0
    for st in enc.outs:
        r, f = st.info_host(stream)
        nrec.append(r)
        fits += f
    ntops = [st.ntop for st in enc.outs]

    # the step as one graph (the decoder's setup kernel is a programmatic
    # dependent of the stream packer, so its launch overlaps the encode's
    # tail), and the encode and the decode alone for the breakdown
    g_step, g_enc, g_dec = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g_step, stream=stream):
            enc.run(stream)
            dec.run(iters, stream)
        with torch.cuda.graph(g_enc, stream=stream):
            enc.run(stream)
        with torch.cuda.graph(g_dec, stream=stream):
            dec.run(iters, stream)
    stream.synchronize()
    with torch.cuda.stream(stream):
        launches_per_step = len(enc.run_timed(stream)) + len(dec.run_timed(iters, stream))

    sampler = ClockSampler(gpu_uuid(torch, dev))
    sampler.start()
    time.sleep(0.2)
    warm = max(args.warmup, 3)
    with torch.cuda.stream(stream):
        for _ in range(warm):
            flush.fill_(1)
            g_step.replay()
    stream.synchronize()
    t_heat = time.perf_counter()
    while time.perf_counter() - t_heat < args.heat_s:
        with torch.cuda.stream(stream):
            for _ in range(5 if pixels > 64 << 20 else 20):
                flush.fill_(1)
                g_step.replay()
        stream.synchronize()
    ref0 = enc.outs[0].to_host(stream)

    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    t_wall0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.fill_(i & 0xff)
            a, c = ev[i]
            a.record(stream)
            g_step.replay()
            c.record(stream)
    stream.synchronize()
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter() - t_wall0
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(c) for a, c in ev]
    ms_per_step, px_s = replica_throughput(world, dev, statistics.mean(step_ms), pixels)
    value = px_s / 1e6

    # ---- the encode and the decode alone, timed the same way (breakdown)
    def time_graph(g, before=None):
        out = []
        with torch.cuda.stream(stream):
            for i in range(warm + args.steps):
                flush.fill_(i & 0xff)
                if before is not None:
                    before.replay()
                x, y = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                x.record(stream)
                g.replay()
                y.record(stream)
                out.append((x, y))
        stream.synchronize()
        return [x.elapsed_time(y) for x, y in out[warm:]]

    enc_ms = time_graph(g_enc)
    dec_ms = time_graph(g_dec, before=g_enc)
    chk = enc.outs[0].to_host(stream)
    assert np.array_equal(chk["records"].view(np.uint8), ref0["records"].view(np.uint8)), "graph replay changed output"

    # ---- per-kernel durations: the same step with an event after every kernel
    krows = []
    with torch.cuda.stream(stream):
        for i in range(min(args.steps, 20)):
            flush.fill_(i & 0xff)
            krows.append(enc.run_timed(stream) + dec.run_timed(iters, stream))
    ktab = kernel_table(krows)

    # ---- per-iteration decoder time inside the graph: the iteration kernels
    # are programmatic dependents of one another (each one's ramp overlaps the
    # previous one's tail), so events between them would serialise what the
    # step overlaps.  Time a one-iteration decode graph (the setup kernel
    # alone) the same way as the timed region; the difference to the full
    # decode graph, divided by the iteration launches, is the in-graph
    # duration of one iteration launch.
    iter_graph_ms = None
    if iters > 1:
        g_dec1 = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            with torch.cuda.graph(g_dec1, stream=stream):
                dec.run(1, stream)
        stream.synchronize()
        ev1 = []
        with torch.cuda.stream(stream):
            for i in range(warm + args.steps):
                flush.fill_(i & 0xff)
                g_enc.replay()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                g_dec1.replay()
                b.record(stream)
                ev1.append((a, b))
        stream.synchronize()
        dec1_ms = statistics.mean(a.elapsed_time(b) for a, b in ev1[warm:])
        iter_graph_ms = (statistics.mean(dec_ms) - dec1_ms) / (iters - 1)
        with torch.cuda.stream(stream):
            g_dec.replay()  # the full decode again (later checks read its output)
        stream.synchronize()

    # ---- end to end through the public API: the pinned host images in, every
    # stream's records (those it holds: fic_records_to_host reads the counts
    # on the device) and info block and the decoded images out, the copies
    # inside the timed region
    out_host = torch.empty(int(offs[-1]), dtype=torch.uint8).pin_memory()
    rec_host = torch.empty(rec_arena.numel(), dtype=torch.uint8).pin_memory()
    info_host = torch.empty((n, fic.INFO_WORDS), dtype=torch.int32).pin_memory()

    def host_views(rec_h, info_h):
        return [rec_h[int(a): int(b)] for a, b in zip(roffs[:-1], roffs[1:])], [info_h[i] for i in range(n)]

    rec_views, info_views = host_views(rec_host, info_host)

    def out_graph(streams, rec_v, info_v, out_h, dec):
        """The step's results out (records by fic_records_to_host, decoded
        images by copy), captured once: a step then enqueues one graph instead
        of marshalling 40 stream descriptors on the host."""
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            with torch.cuda.graph(g, stream=stream):
                fic.records_to_host(streams, rec_v, info_v, stream)
                out_h.copy_(dec, non_blocking=True)
        stream.synchronize()
        return g

    g_out = out_graph(enc.outs, rec_views, info_views, out_host, dec_arena)
    h2d = host_in.numel()
    d2h = out_host.numel() + 16 * int(sum(nrec)) + 4 * info_host.numel()
    e2e_ev = []
    with torch.cuda.stream(stream):
        for i in range(warm + args.steps):
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.fill_(i & 0xff)
            s0.record(stream)
            dev_in.copy_(host_in, non_blocking=True)
            g_step.replay()
            g_out.replay()
            s1.record(stream)
            e2e_ev.append((s0, s1))
    stream.synchronize()
    assert np.array_equal(rec_host[: 16 * nrec[0]].numpy(), ref0["records"].view(np.uint8)), "e2e copy differs"
    e2e_serial_ms, e2e_serial_px_s = replica_throughput(
        world, dev, statistics.mean(a.elapsed_time(b) for a, b in e2e_ev[warm:]), pixels)

    # ---- end to end, pipelined: a second set of device buffers, plans and
    # graphs; step i copies its inputs in on one stream, encodes and decodes
    # on a second and copies its results out on a third, so that the copies
    # of neighbouring steps overlap the compute.  Every step still moves its
    # own inputs in and its own results out inside the timed region.
    class Slot:
        pass

    def make_slot():
        sl = Slot()
        sl.dev_in = torch.empty_like(dev_in)
        imgs_s = [sl.dev_in[int(o): int(o) + it[0].size].view(it[0].shape) for it, o in zip(items, offs)]
        sl.rec = torch.empty_like(rec_arena)
        sl.info = torch.zeros_like(info_arena)
        outs_ss = [fic.Stream(it[0].shape[1], it[0].shape[0], p, dev, records=sl.rec[int(a): int(b)], info=sl.info[i])
                   for i, (it, p, a, b) in enumerate(zip(items, plist, roffs[:-1], roffs[1:]))]
        sl.dec = torch.empty_like(dec_arena)
        dec_outs_s = [sl.dec[int(o): int(o) + it[0].size].view(it[0].shape) for it, o in zip(items, offs)]
        with torch.cuda.stream(stream):
            sl.enc_plan = fic.EncodePlan(imgs_s, plist, outs=outs_ss, stream=stream)
            sl.enc_plan.set_tuning(**enc.tuning)
            sl.enc_plan.run(stream)
            sl.dec_plan = fic.DecodePlan(sl.enc_plan.outs, outs=dec_outs_s, stream=stream)
            sl.dec_plan.set_tuning(**dec.tuning)
        sl.g_step = torch.cuda.CUDAGraph()
        with torch.cuda.stream(stream):
            with torch.cuda.graph(sl.g_step, stream=stream):
                sl.enc_plan.run(stream)
                sl.dec_plan.run(iters, stream)
        stream.synchronize()
        sl.out_host = torch.empty(int(offs[-1]), dtype=torch.uint8).pin_memory()
        sl.rec_host = torch.empty(rec_arena.numel(), dtype=torch.uint8).pin_memory()
        sl.info_host = torch.empty((n, fic.INFO_WORDS), dtype=torch.int32).pin_memory()
        sl.rec_views, sl.info_views = host_views(sl.rec_host, sl.info_host)
        sl.g_out = out_graph(sl.enc_plan.outs, sl.rec_views, sl.info_views, sl.out_host, sl.dec)
        return sl

    slot0 = Slot()
    slot0.dev_in, slot0.rec, slot0.info, slot0.dec = dev_in, rec_arena, info_arena, dec_arena
    slot0.g_step = g_step
    slot0.out_host, slot0.rec_host, slot0.info_host = out_host, rec_host, info_host
    slot0.g_out = g_out
    slots = [slot0, make_slot()]
    s_in, s_cmp, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_cmp = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]

    def pipe(steps):
        for i in range(steps):
            k = i & 1
            sl = slots[k]
            with torch.cuda.stream(s_in):
                if i >= 2:
                    s_in.wait_event(ev_cmp[k])  # the slot's previous inputs are consumed
                sl.dev_in.copy_(host_in, non_blocking=True)
                ev_in[k].record(s_in)
            with torch.cuda.stream(s_cmp):
                s_cmp.wait_event(ev_in[k])
                if i >= 2:
                    s_cmp.wait_event(ev_out[k])  # the slot's previous results are out
                sl.g_step.replay()
                ev_cmp[k].record(s_cmp)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_cmp[k])
                sl.g_out.replay()
                ev_out[k].record(s_out)

    torch.cuda.synchronize(dev)
    pipe(warm)
    torch.cuda.synchronize(dev)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    p0.record(s_in)
    pipe(args.steps)
    p1.record(s_out)  # the last step's last copy depends on all earlier work
    torch.cuda.synchronize(dev)
    for sl in slots:
        assert np.array_equal(sl.rec_host[: 16 * nrec[0]].numpy(), ref0["records"].view(np.uint8)), \
            "pipelined e2e copy differs"
        assert torch.equal(sl.out_host, slots[0].out_host), "pipelined decodes differ between slots"
    e2e_ms, e2e_px_s = replica_throughput(world, dev, p0.elapsed_time(p1) / args.steps, pixels)
    e2e_value = e2e_px_s / 1e6

    # ---- roofline of the dominant kernel (HBM bound): algorithmic bytes per launch
    peaks, peak_kind = load_peaks()
    peak = float(peaks["hbm_gbs"])
    enc_bytes = pixels + sum(16 * r for r in nrec) + sum(8 * t + 4 for t in ntops)
    dec_bytes_iter = 2 * pixels + sum(16 * r for r in nrec) + sum(4 * (t + 1) for t in ntops)
    alg = {"mns_encode_kernel": enc_bytes, "decode_iter_kernel": dec_bytes_iter, "decode_d4_iter_kernel": dec_bytes_iter,
           # the cooperative single launch runs every iteration after the first
           "decode_d4_loop_kernel": max(iters - 1, 0) * dec_bytes_iter}
    dom = max((k for k in ktab if k in alg), key=lambda k: ktab[k]["share"])
    dur_ms, dur_src = ktab[dom]["ms_per_launch"], "CUDA events around every launch (serialised)"
    if dom in ("decode_d4_iter_kernel", "decode_iter_kernel") and iter_graph_ms:
        dur_ms = iter_graph_ms
        dur_src = ("in the timed graph: (decode graph - one-iteration decode graph) / iteration launches, "
                   "CUDA events over the timed region")
    ach = alg[dom] / (dur_ms * 1e-3) / 1e9
    key = f"{dom}_{spec.name}"
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4), "peak_kind": peak_kind, "traffic": traffic_from_profile(key),
                "alg_bytes_per_launch": alg[dom], "ms_per_launch": round(dur_ms, 5), "duration": dur_src,
                "kernels": {k: dict(v, GB_s=round(alg[k] / (v["ms_per_launch"] * 1e-3) / 1e9, 1)) if k in alg else v
                            for k, v in ktab.items()}}

    # the MNS fit kernel (the quadtree encoder, Section 3) on its own: the
    # kernel the throughput target is about, whatever its share of the step
    roofline_fit = None
    fit_k = next((k for k in ktab if k == "mns_encode_kernel"), None)
    if fit_k:
        f_ms = ktab[fit_k]["ms_per_launch"]
        f_ach = enc_bytes / (f_ms * 1e-3) / 1e9
        roofline_fit = {"bound": "hbm", "kernel": fit_k, "achieved": round(f_ach, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(f_ach / peak, 4), "peak_kind": peak_kind,
                        "traffic": traffic_from_profile(f"{fit_k}_{spec.name}"),
                        "alg_bytes_per_launch": enc_bytes, "ms_per_launch": round(f_ms, 5),
                        "duration": "CUDA events around the launch on its stream, mean over the timed steps",
                        "fits_per_s": round(fits / (f_ms * 1e-3), 1),
                        "mpix_s": round(pixels / (f_ms * 1e-3) / 1e6, 1)}
    if dom in ("decode_d4_iter_kernel", "decode_iter_kernel"):
        roofline["working_set"] = ("L2-resident within the step (the two 2x2-sum images and the tables stay in L2 "
                                   "between iterations; L2 is flushed only before each step)"
                                   if 2 * pixels < L2_BYTES else "larger than L2")
        ev_ms = ktab[dom]["ms_per_launch"]
        roofline["frac_event_serialised"] = round(alg[dom] / (ev_ms * 1e-3) / 1e9 / peak, 4)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    roofline["issue"] = issue_from_profile(key, dur_ms, clocks, sms)
    if roofline_fit:
        roofline_fit["issue"] = issue_from_profile(f"{fit_k}_{spec.name}", roofline_fit["ms_per_launch"], clocks, sms)

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "Mpixel/s", "n_gpus": world, "steps": args.steps,
        "warmup": warm, "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": spec.desc, "images": n, "pixels_per_step": pixels,
                   "l2": "flushed (256 MiB write) before every step" if flush_l2 else
                         f"not flushed: inputs ({pixels / 2**20:.0f} MiB) larger than L2",
                   "parallelism": f"replicas x{world}",
                   "graph": "one CUDA graph per step (encode, pack, decoder setup and iterations)"},
        "encode_mpix_s": round(world * pixels / (statistics.mean(enc_ms) * 1e-3) / 1e6, 3),
        "fits_per_s": round(world * fits / (ms_per_step * 1e-3), 1),
        "fits_per_step": fits,
        "records_per_step": int(sum(nrec)),
        "wall_s_timed": round(t_wall, 3),
        "roofline": roofline,
        "roofline_fit": roofline_fit,
        "e2e": {"value": round(e2e_value, 3), "unit": "Mpixel/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms, 5),
                "mode": "pipelined over steps: inputs in, encode + decode, results out on three streams "
                        "with two buffer sets; no L2 flush (every step's inputs arrive by copy)",
                "out": "decoded images by copy engine; each stream's records (the ones it holds) and info block "
                       "by fic_records_to_host, which reads the counts on the device (both captured in one graph "
                       "per buffer set)",
                "serial": {"value": round(e2e_serial_px_s / 1e6, 3), "ms_per_step": round(e2e_serial_ms, 5),
                           "mode": "one step at a time on one stream, L2 flushed before each step"}},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
    }
    if spec.name in ("one256", "batch40x512"):
        line["rate_distortion"], line["bitstream"] = rate_distortion(fic, torch, stream, items, enc, dec, nrec)
    if spec.name == "batch40x512":
        line["fig6"] = fig6_curves(fic, torch, stream, dimgs[:10], flush)
    if tuning:
        line["autotune"] = {"encode_best": tuning["encode"]["best"], "encode_best_ms": round(tuning["encode"]["best_ms"], 4),
                            "encode_trials": tuning["encode"]["trials"],
                            "decode_best": tuning["decode"]["best"], "decode_best_ms": round(tuning["decode"]["best_ms"], 4),
                            "decode_trials": tuning["decode"]["trials"]}
    if spec.plain:
        line["plain_per_image"] = plain_per_image(fic, torch, stream, dimgs, plist, iters, enc, dec, pixels, value)
    if spec.name == "batch40x512" and world == 1 and args.line_serve_s > 0:
        # the metric's served p50/p99: a bounded replay of the serving trace
        # (config 5) after the timed steps, with the per-request loop beside it
        line["serving"] = serving_phase(torch, fic, dev, args.rate, args.line_serve_s, args.hbm_budget_gb)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        v, done, dt = time_oracle(items, iters, args.cpu_s, threads)
        v1, done1, dt1 = time_oracle(items, iters, args.cpu_s / 3, 1)
        line["cpu_baseline"] = {"value": round(v, 3), "unit": "Mpixel/s", "cores": threads, "kind": "oracle",
                                "sample": f"{done} images of the batch, encode + {iters}-iteration decode, "
                                          f"{dt:.1f} s on {threads} threads",
                                "single_thread": {"value": round(v1, 3), "unit": "Mpixel/s", "cores": 1,
                                                  "sample": f"{done1} images, {dt1:.1f} s on one thread"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    dist_finish(world)
    return 0


def rate_distortion(fic, torch, stream, items, enc, dec, nrec):
    """Bits per pixel of each stream's bitstream (Sections 3.3-3.4, with
    Technique 2) and PSNR of its decode (Section 4), per threshold; plus the
    device time of writing and reading all the bitstreams."""
    from oracle import oracle as O  # PSNR definition only

    per = {}
    with torch.cuda.stream(stream):
        bits = fic.serialize_batch(enc.outs, True, stream)
        pitems = [(w, ix, st.width, st.height, st.params) for (w, ix), st in zip(bits, enc.outs)]
        back = fic.parse_batch(pitems, True, stream)
        ws = torch.empty(max(int(fic.lib().fic_bitstream_batch_workspace_bytes(
            (fic.fic.StreamC * len(back))(*[b.c for b in back]), len(back))), 1), dtype=torch.uint8,
            device=back[0].records.device)
        # timing: every stream written in one batched call, then every stream
        # read back in one, into the buffers above (best of a few).  Device
        # time: a spin kernel keeps the stream busy while the host prepares
        # the calls, so the events bracket the kernels only; call time: the
        # same calls back to back on an idle stream (the binding's argument
        # marshalling included).
        times, calls = [], []
        for spin in (True, False):
            for _ in range(5):
                if spin:
                    torch.cuda._sleep(2_000_000)
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
                ev[0].record(stream)
                fic.serialize_batch(enc.outs, True, stream, outs=bits, workspace=ws)
                ev[1].record(stream)
                fic.parse_batch(pitems, True, stream, outs=back, workspace=ws)
                ev[2].record(stream)
                (times if spin else calls).append(ev)
                stream.synchronize()
    ev = min(times, key=lambda e: e[0].elapsed_time(e[2]))
    evc = min(calls, key=lambda e: e[0].elapsed_time(e[2]))
    total_bits = 0
    for (im, mode, bmax, bmin, t), (w, ix), d in zip(items, bits, dec.outs):
        nb = int(ix[-1].item())
        total_bits += nb
        e = per.setdefault(t, {"bpp": [], "psnr": []})
        e["bpp"].append(nb / im.size)
        e["psnr"].append(O.psnr(im, d.cpu().numpy()))
    same = all(np.array_equal(b.to_host(stream)["records"].view(np.uint8), st.to_host(stream)["records"].view(np.uint8))
               for b, st in zip(back[:4], enc.outs[:4]))
    rd = [{"rms_threshold": t, "bpp": round(float(np.mean(v["bpp"])), 4), "psnr_db": round(float(np.mean(v["psnr"])), 3)}
          for t, v in sorted(per.items())]
    return rd, {"streams": len(items), "records": int(sum(nrec)), "bits": total_bits,
                "serialize_ms": round(ev[0].elapsed_time(ev[1]), 4), "parse_ms": round(ev[1].elapsed_time(ev[2]), 4),
                "call_ms": {"serialize": round(evc[0].elapsed_time(evc[1]), 4),
                            "parse": round(evc[1].elapsed_time(evc[2]), 4)},
                "round_trip_identical": bool(same),
                "note": "all streams in one batched serialize call and one batched parse call (three kernels "
                        "each, into preallocated buffers); technique 2 on; serialize_ms / parse_ms: device time "
                        "(a spin kernel keeps the stream busy while the host enqueues); call_ms: on an idle "
                        "stream, the binding's argument marshalling included"}


def fig6_curves(fic, torch, stream, dimgs, flush, reps=10, iters=10):
    """Section 4 (Fig. 6) on the synthetic stand-ins for the paper's 512x512
    test images: no-search against MNS over the RMS threshold sweep, in the
    paper's own configuration (quadtree 16 -> 2, 3-bit contrast, 8-bit
    luminance, Technique 2).  Per point: bits per pixel of the bitstream,
    PSNR of the decode, and the device time of encoding the ten images in
    one launch (CUDA events, L2 flushed before each run)."""
    from oracle import oracle as O  # PSNR definition only

    imgs_h = [d.cpu().numpy() for d in dimgs]
    px = sum(im.size for im in imgs_h)
    points = []
    for mode in ("nosearch", "mns"):
        for t in THRESHOLDS:
            p = fic.params(mode, 16, 2, t, s_bits=3, o_bits=8)
            with torch.cuda.stream(stream):
                plan = fic.EncodePlan(dimgs, p, stream=stream)
                plan.run(stream)
                ms = []
                for r in range(reps + 2):
                    flush.fill_(r & 0xff)
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    plan.run(stream)
                    b.record(stream)
                    ms.append((a, b))
                dplan = fic.DecodePlan(plan.outs, stream=stream)
                dplan.run(iters, stream)
                bits = [fic.serialize(st, True, stream)[1] for st in plan.outs]
            stream.synchronize()
            enc_ms = statistics.mean(a.elapsed_time(b) for a, b in ms[2:])
            nbits = sum(int(ix[-1].item()) for ix in bits)
            ps = [O.psnr(im, d.cpu().numpy()) for im, d in zip(imgs_h, dplan.outs)]
            points.append({"mode": mode, "rms_threshold": t, "bpp": round(nbits / px, 4),
                           "psnr_db": round(float(np.mean(ps)), 3), "encode_us": round(enc_ms * 1e3, 2),
                           "encode_mpix_s": round(px / (enc_ms * 1e-3) / 1e6, 1)})
    return {"config": "ten 512x512 images (8 scenes seeds 1-8 + 2 Voronoi 101/102), quadtree 16->2, s 3 bits, "
                      "o 8 bits, Technique 2, decode 10 iterations from mid-grey", "points": points}


def plain_per_image(fic, torch, stream, dimgs, plist, iters, enc, dec, pixels, batched_value):
    """The same encode + decode, one image at a time: (a) the plain API calls
    fic_encode + fic_decode per image, (b) one prepared plan per image
    launched in turn.  Outputs are checked equal to the batched launch."""
    out = {}
    with torch.cuda.stream(stream):
        # (b) per-image plans
        plans = []
        for d, p in zip(dimgs, plist):
            e = fic.EncodePlan([d], p, stream=stream)
            e.run(stream)
            plans.append((e, fic.DecodePlan(e.outs, stream=stream)))
        stream.synchronize()
        ms = []
        for rep in range(4):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for e, dp in plans:
                e.run(stream)
                dp.run(iters, stream)
            b.record(stream)
            stream.synchronize()
            if rep:
                ms.append(a.elapsed_time(b))
        v_plans = pixels / (statistics.mean(ms) * 1e-3) / 1e6
        # (a) plain API calls
        ms = []
        for rep in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            outs = []
            a.record(stream)
            for d, p in zip(dimgs, plist):
                st = fic.fic_encode(d, p, stream=stream)
                outs.append((st, fic.fic_decode(st, iters, stream=stream)))
            b.record(stream)
            stream.synchronize()
            if rep:
                ms.append(a.elapsed_time(b))
        v_api = pixels / (statistics.mean(ms) * 1e-3) / 1e6
    # identical output: every stream and decoded image of a sample of images
    same = True
    for i in range(0, len(dimgs), max(1, len(dimgs) // 16)):
        ga, gb = enc.outs[i].to_host(stream), outs[i][0].to_host(stream)
        gc = plans[i][0].outs[0].to_host(stream)
        same &= np.array_equal(ga["records"].view(np.uint8), gb["records"].view(np.uint8))
        same &= np.array_equal(ga["records"].view(np.uint8), gc["records"].view(np.uint8))
        same &= bool(torch.equal(dec.outs[i], outs[i][1])) and bool(torch.equal(dec.outs[i], plans[i][1].outs[0]))
    return {"api_calls_mpix_s": round(v_api, 3), "per_image_plans_mpix_s": round(v_plans, 3),
            "batched_over_api_calls": round(batched_value / v_api, 3),
            "batched_over_per_image_plans": round(batched_value / v_plans, 3),
            "identical_output": bool(same),
            "note": "same images and parameters, one image per launch, no graphs; output compared on a sample "
                    "of 1/16 of the images"}


# --------------------------------------------------------------------------
# GPU arm: exhaustive search (exhaustive)

def run_exhaustive(args):
    import torch

    world, rank, dev = dist_setup()
    import paper_1501_02894_gb300 as fic

    fic.lib()
    imgs = synth.exhaustive_images()
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    peaks, peak_kind = load_peaks()
    res = {}
    sampler = ClockSampler(gpu_uuid(torch, dev))
    sampler.start()
    time.sleep(0.2)
    outs = {}
    for engine, ename in ((0, "tcgen05"), (1, "cuda_cores")):
        plans, work = [], []
        with torch.cuda.stream(stream):
            for name, im in imgs:
                p = fic.params("exhaustive", 8, 8, 8.0, dom_step=4, isometries=8, engine=engine)
                d = torch.from_numpy(im).to(dev)
                plan = fic.EncodePlan([d], p, stream=stream)
                plan.run(stream)
                plans.append((name, im, d, plan))
            stream.synchronize()
            for name, im, d, plan in plans:
                H, W = im.shape
                nr = (W // 8) * (H // 8)
                nd = ((W - 16) // 4 + 1) * ((H - 16) // 4 + 1)
                work.append((name, nr, nd, W * H))
                _, f = plan.outs[0].info_host(stream)
                assert f == nr * nd * 8
            for _ in range(max(args.warmup, 3)):
                flush.fill_(1)
                for _, _, _, plan in plans:
                    plan.run(stream)
            stream.synchronize()
            rows = {name: [] for name, *_ in plans}
            steps = max(1, min(args.steps, 20))
            for i in range(steps):
                flush.fill_(i & 0xff)
                for name, _, _, plan in plans:
                    rows[name].append(plan.run_timed(stream))
        outs[ename] = [plan.outs[0].to_host(stream) for *_, plan in plans]
        per = {}
        for (name, nr, nd, px) in work:
            tab = kernel_table(rows[name])
            total_ms = sum(v["ms_per_launch"] * v["launches_per_step"] for v in tab.values())
            search = "exh_tc_kernel" if engine == 0 else "exh_cuda_kernel"
            flops = 2.0 * nr * 8 * nd * 64
            s_ms = tab[search]["ms_per_launch"]
            per[name] = {"ranges": nr, "domains": nd, "fits": nr * nd * 8, "ms": round(total_ms, 4),
                         "fits_per_s": round(nr * nd * 8 / (total_ms * 1e-3), 1),
                         "mpix_s": round(px / (total_ms * 1e-3) / 1e6, 3),
                         "search_kernel": search, "search_ms": s_ms,
                         "search_tflops": round(flops / (s_ms * 1e-3) / 1e12, 2), "kernels": tab}
        res[ename] = per
    clocks = sampler.stop()
    same = all(np.array_equal(a["records"].view(np.uint8), b["records"].view(np.uint8))
               for a, b in zip(outs["tcgen05"], outs["cuda_cores"]))
    # Section 2 (Figs. 2, 3): distribution of x_d - x_r, y_d - y_r of the
    # exhaustive search, against two uniform random points (p(u) = 1 - |u|)
    offset_stats = {}
    for (name, im, d, plan) in plans:
        H, W = im.shape
        with torch.cuda.stream(stream):
            hx, hy = fic.offset_histogram(plan.outs[0], stream)
        stream.synchronize()
        st = {}
        for axis, h, n in (("x", hx, W), ("y", hy, H)):
            c = h.cpu().numpy().astype(np.float64)
            u = (np.arange(2 * n) - n) / n
            tot = c.sum()
            st[f"mean_abs_d{axis}_over_side"] = round(float((c * np.abs(u)).sum() / tot), 4)
            st[f"frac_abs_d{axis}_le_side_over_8"] = round(float(c[np.abs(u) <= 0.125].sum() / tot), 4)
        st["uniform_model"] = {"mean_abs": round(1 / 3, 4), "frac_le_1_8": round(2 * 0.125 - 0.125 ** 2, 4)}
        offset_stats[name] = st
    tot_fits = sum(v["fits"] for v in res["tcgen05"].values())
    tot_ms = sum(v["ms"] for v in res["tcgen05"].values())
    value = world * tot_fits / (tot_ms * 1e-3)
    big = res["tcgen05"]["scene9_1024"]
    peak = float(peaks["bf16_tflops"])
    roofline = {"bound": "tensor", "kernel": "exh_tc_kernel (1024x1024)", "achieved": big["search_tflops"],
                "peak": peak, "unit": "TFLOP/s", "frac": round(big["search_tflops"] / peak, 4),
                "peak_kind": f"{peak_kind} bf16 burst x 1 (fp16 operands, same nominal rate)",
                "traffic": None,
                "flops_per_launch": 2.0 * big["ranges"] * 8 * big["domains"] * 64,
                "note": "algorithmic FLOPs = 2 x (ranges x 8 isometries) x domains x 64 decimated values"}
    line = {
        "metric": "exhaustive-search range-domain fits/s (bit-exact)", "value": round(value, 1), "unit": "fits/s",
        "n_gpus": world, "steps": max(1, min(args.steps, 20)), "warmup": max(args.warmup, 3),
        "ms_per_step": round(tot_ms, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f16 operands, f32 accumulate (exact integers), int64 decisions", "data": "synthetic",
        "config": {"workload": "exhaustive: 512x512 seed 1 + 1024x1024 seed 9, 8x8 ranges, domain step 4, 8 isometries",
                   "l2": "flushed (256 MiB write) before every step", "parallelism": f"replicas x{world}"},
        "engines": res, "engines_identical_output": bool(same), "offset_stats": offset_stats,
        "cuda_core_over_tensor_time": round(sum(v["ms"] for v in res["cuda_cores"].values()) / tot_ms, 3),
        "roofline": roofline, "gpu_launches": 4 * len(imgs) * max(1, min(args.steps, 20)), "clocks": clocks,
        "e2e": None,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        v, done, dt = time_oracle_exhaustive(imgs[1][1], args.cpu_s, threads)
        line["cpu_baseline"] = {"value": round(v, 1), "unit": "fits/s", "cores": threads, "kind": "oracle",
                                "sample": f"{done} random 8x8 ranges of the 1024x1024 image, full search, "
                                          f"{dt:.1f} s on {threads} threads"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    dist_finish(world)
    return 0


# --------------------------------------------------------------------------
# GPU arm: serving (serving)

def serving_phase(torch, fic, dev, rate, seconds, hbm_budget_gb, plain=True):
    """Replay a Poisson trace of encode and decode requests (config 5) through
    the request server, and (with `plain`) the same trace one request at a
    time.  Returns a dict of the measurements."""
    t_setup = time.perf_counter()
    t_arr, is_enc, side, seeds = synth.serving_requests(rate=rate, seconds=seconds)
    nreq = len(t_arr)
    # image pool: one image per distinct side, from the seed of the first
    # request of that side (generating every request's own image is
    # hours of host work at this rate)
    sides = sorted(set(int(s) for s in side))
    first = {}
    for i, s in enumerate(side):
        first.setdefault(int(s), i)
    pool_imgs = gen_images([("g", s, int(seeds[first[s]])) for s in sides])
    pool = dict(zip(sides, pool_imgs))
    P = fic.params("mns", 32, 4, 8.0)
    iters = 8
    # decode inputs: the stream of each pool image, encoded once at setup
    streams, offsets = {}, {}
    for s, im in pool.items():
        st = fic.fic_encode(torch.from_numpy(im).to(dev), P)
        h = st.to_host()
        streams[s] = h["records"].copy()
        offsets[s] = h["tile_offsets"].astype(np.int32)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup

    class Buffers:
        def __init__(self):
            self.free = {}

        def get(self, key, make):
            lst = self.free.setdefault(key, [])
            return lst.pop() if lst else make()

        def put(self, key, buf):
            self.free[key].append(buf)

    def serve_with_server():
        srv = fic.Server(hbm_budget_bytes=int(hbm_budget_gb * (1 << 30)), streams=4, max_batch=64,
                         queue_capacity=1 << 20, host_staging_bytes=4 << 30)
        bufs = Buffers()
        live = {}  # ticket -> (i, key, bufs, submit lag)
        lat = np.zeros(nreq)
        qms = np.zeros(nreq)
        px_done = 0
        order = []
        t0 = time.perf_counter() + 0.05

        def reap(block=False):
            nonlocal px_done
            while order:
                tk = order[0]
                r = srv.wait(tk, -1) if block else srv.poll(tk)
                if r is None:
                    return
                order.pop(0)
                i, key, b, lag = live.pop(tk)
                lat[i] = lag + r["latency_ms"]
                qms[i] = lag + r["queue_ms"]
                px_done += int(side[i]) ** 2
                for k2, v in zip(key, b):
                    bufs.put(k2, v)

        for i in range(nreq):
            s = int(side[i])
            now = time.perf_counter() - t0
            if now < t_arr[i]:
                reap()
                while time.perf_counter() - t0 < t_arr[i]:
                    pass
            lag = max(0.0, (time.perf_counter() - t0) - t_arr[i]) * 1e3
            if is_enc[i]:
                cap, ntop = (s // 4) ** 2, (s // 32) ** 2
                rb = bufs.get(("r", s), lambda: np.zeros(cap, dtype=fic.RECORD_DTYPE))
                sb = bufs.get(("s", s), lambda: np.zeros(ntop, dtype=np.uint32))
                tk = srv.submit_encode(pool[s], P, out_records=rb, out_split=sb)
                live[tk] = (i, (("r", s), ("s", s)), (rb, sb), lag)
            else:
                ob = bufs.get(("o", s), lambda: np.zeros((s, s), dtype=np.uint8))
                tk = srv.submit_decode(streams[s], s, s, P, iters, out=ob)
                live[tk] = (i, (("o", s),), (ob,), lag)
            order.append(tk)
        reap(block=True)
        t_end = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        return lat, px_done, t_end, st, qms

    def serve_plain():
        """One request at a time in arrival order: copy in, fic_encode or
        fic_decode, copy out, synchronise.  The inputs come from the same
        pageable host arrays the server receives."""
        lat = np.zeros(nreq)
        px_done = 0
        stream = torch.cuda.current_stream()
        pinned = {s: torch.from_numpy(im) for s, im in pool.items()}
        t0 = time.perf_counter() + 0.05
        deadline = seconds * 2 + 30
        served = 0
        for i in range(nreq):
            s = int(side[i])
            while time.perf_counter() - t0 < t_arr[i]:
                pass
            if is_enc[i]:
                d = pinned[s].to(dev)
                stv = fic.fic_encode(d, P)
                stv.to_host()
            else:
                rec = torch.from_numpy(streams[s].view(np.uint8)).to(dev)
                stv = fic.Stream(s, s, P, dev)
                stv.records[: rec.numel()].copy_(rec)
                stv.tile_offsets.copy_(torch.from_numpy(offsets[s]))
                fic.fic_decode(stv, iters).cpu()
            stream.synchronize()
            lat[i] = (time.perf_counter() - t0 - t_arr[i]) * 1e3
            px_done += s * s
            served += 1
            if time.perf_counter() - t0 > deadline:
                break
        t_end = time.perf_counter() - t0
        return lat[:served], px_done, t_end, served

    # the client's own pauses would count as request latency: no cyclic
    # garbage collection while a trace is replayed
    import gc
    gc.collect()
    gc.disable()
    try:
        sampler = ClockSampler(gpu_uuid(torch, dev))
        sampler.start()
        lat_s, px_s, t_s, stats, q_s = serve_with_server()
        clocks = sampler.stop()
        gc.collect()
        lat_p, px_p, t_p, served_p = serve_plain() if plain else (np.zeros(0), 0, 1.0, 0)
    finally:
        gc.enable()

    def pct(a, q):
        return round(float(np.percentile(a, q)), 3) if len(a) else None

    offered = float(np.sum(side.astype(np.float64) ** 2)) / seconds / 1e6
    out = {
        "served_mpix_s": round(px_s / t_s / 1e6, 3), "offered_mpix_s": round(offered, 3), "requests": nreq,
        "seconds": round(t_s, 3), "distinct_sides": len(sides),
        "latency_ms": {"p50": pct(lat_s, 50), "p99": pct(lat_s, 99), "mean": round(float(np.mean(lat_s)), 3),
                       "max": round(float(np.max(lat_s)), 3), "from": "arrival to result in the caller's buffer"},
        "server_stats": stats,
        "by_side": {name: {"requests": int(m.sum()), "p50_ms": pct(lat_s[m], 50), "p99_ms": pct(lat_s[m], 99),
                           "queue_p50_ms": pct(q_s[m], 50), "plain_p50_ms": pct(lat_p[m[:len(lat_p)]], 50),
                           "plain_p99_ms": pct(lat_p[m[:len(lat_p)]], 99)}
                    for name, m in (("side<512", side < 512), ("512<=side<1536", (side >= 512) & (side < 1536)),
                                    ("side>=1536", side >= 1536))},
        "setup_s": round(setup_s, 1), "clocks": clocks,
        "workload": f"Poisson {rate:.0f} req/s for {seconds:g} s, 80% encode / 20% decode (8 it), sides "
                    f"log-uniform [128,4096] step 32, MNS 32->4 RMS 8; one pool image per side; "
                    f"{hbm_budget_gb:g} GB budget, 4 streams, batches of <= 64 jobs",
    }
    if plain:
        out["plain_per_request"] = {
            "mpix_s": round(px_p / t_p / 1e6, 3), "served": int(served_p),
            "latency_ms": {"p50": pct(lat_p, 50), "p99": pct(lat_p, 99),
                           "mean": round(float(np.mean(lat_p)), 3) if len(lat_p) else None},
            "how": "one request at a time in arrival order: H2D from the same pageable host arrays the server "
                   "receives, fic_encode / fic_decode, D2H, synchronise"}
    return out


def run_serving(args):
    import torch

    world, rank, dev = dist_setup()
    import paper_1501_02894_gb300 as fic

    fic.lib()
    m = serving_phase(torch, fic, dev, args.rate, args.serve_s, args.hbm_budget_gb)
    value = m["served_mpix_s"]
    line = {
        "metric": "served MNS encode/decode Mpixel/s with p50/p99 latency (bit-exact)", "value": value,
        "unit": "Mpixel/s", "n_gpus": world, "steps": 1, "warmup": 0, "ms_per_step": round(m["seconds"] * 1e3, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": "serving: " + m["workload"], "requests": m["requests"],
                   "distinct_sides": m["distinct_sides"], "hbm_budget_gb": args.hbm_budget_gb,
                   "server": "4 streams, batches of <= 64 jobs"},
        "offered_mpix_s": m["offered_mpix_s"], "latency_ms": m["latency_ms"], "server_stats": m["server_stats"],
        "by_side": m["by_side"], "plain_per_request": m["plain_per_request"],
        "setup_s": m["setup_s"], "clocks": m["clocks"], "roofline": None, "gpu_launches": None,
        "e2e": {"value": value, "unit": "Mpixel/s", "h2d_bytes_per_step": None, "d2h_bytes_per_step": None,
                "note": "the served rate is end to end: host buffers in and out"},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    dist_finish(world)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch40x512", choices=["one256", "batch40x512", "exhaustive", "mixed512", "serving"])
    ap.add_argument("--cpu-s", type=float, default=15.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--ref-step-s", type=float, default=10.0, help="oracle seconds per reference step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--heat-s", type=float, default=2.0, help="busy seconds before the timed steps (clock sampling)")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: arrivals per second")
    ap.add_argument("--serve-s", type=float, default=60.0, help="serving: seconds of arrivals")
    ap.add_argument("--hbm-budget-gb", type=float, default=40.0, help="serving: server device memory")
    ap.add_argument("--line-serve-s", type=float, default=10.0,
                    help="default workload: seconds of the serving trace replayed after the timed steps (0: none)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "exhaustive":
        return run_exhaustive(args)
    if args.workload == "serving":
        return run_serving(args)
    return run_batched(args, make_spec(args.workload))


if __name__ == "__main__":
    sys.exit(main())
