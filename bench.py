"""Benchmark of the MNS fractal coder on GB300.

One step = the whole hot path over one batch: the MNS quadtree encode
(moments, phase 1, phase 2, split, stream packing) of the ten 512x512
synthetic images shaped like the paper's test images (8 scenes + 2 Voronoi
images) at each RMS threshold of the sweep {4, 8, 12, 16} -- 40 encodes in
one persistent launch -- followed by the 10-iteration decode of all 40
streams.  The step is captured in CUDA graphs and replayed; L2 is flushed
(a 256 MiB write) before every timed step because the inputs (2.6 MB) are
far smaller than L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

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
DECODE_ITERS = 10
METRIC = "MNS encode Mpixel/s & range-domain fits/s (bit-exact); served p50/p99 latency"
WORKLOAD = "cfg2: 10 x 512x512 (8 scenes seeds 1-8 + 2 Voronoi 101/102) x RMS {4,8,12,16}, MNS 32->4 + decode 10 it"


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def workload():
    imgs = [im for _, im in synth.cfg2_images()]
    batch = [(im, t) for t in THRESHOLDS for im in imgs]
    return batch


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


def traffic_from_profile(kernel_key: str):
    """DRAM bytes per launch of a kernel from the committed ncu summary, valid
    only while the kernel source is unchanged (hash recorded beside it)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            prof = json.load(f)
        ent = prof[kernel_key]
        src = os.path.join(ROOT, ent["source"])
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        if h != ent["source_sha256_16"]:
            return None
        return float(ent["bytes_per_launch"])
    except Exception:
        return None


# --------------------------------------------------------------------------
# CPU oracle (the reference arm and the cpu_baseline object)

def time_oracle(batch, budget_s: float, threads: int):
    """Encode + decode as many (image, threshold) pairs as fit in the budget,
    spread over `threads` host threads.  Returns (Mpixel/s, pairs done)."""
    from concurrent.futures import ThreadPoolExecutor

    from oracle import oracle as O

    O.lib()

    def one(item):
        im, t = item
        p = O.make_params("mns", 32, 4, t)
        leaves, _, _ = O.encode(im, p)
        O.decode(leaves, im.shape[1], im.shape[0], p, DECODE_ITERS)
        return im.size

    t0 = time.perf_counter()
    done_px = 0
    done = 0
    i = 0
    with ThreadPoolExecutor(max_workers=threads) as ex:
        while time.perf_counter() - t0 < budget_s:
            chunk = [batch[(i + j) % len(batch)] for j in range(threads)]
            i += threads
            for px in ex.map(one, chunk):
                done_px += px
                done += 1
    dt = time.perf_counter() - t0
    return done_px / dt / 1e6, done, dt


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    batch = workload()
    threads = os.cpu_count() or 1
    vals = []
    total_px = sum(im.size for im, _ in batch)
    # each step is a bounded sample so that the whole run stays within minutes
    step_s = max(0.5, min(args.ref_step_s, 150.0 / max(1, args.steps + args.warmup)))
    args.ref_step_s = step_s
    for _ in range(args.warmup):
        time_oracle(batch, min(0.5, step_s), threads)
    for _ in range(args.steps):
        v, n, dt = time_oracle(batch, step_s, threads)
        vals.append(v)
    value = statistics.mean(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "Mpixel/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total_px / (value * 1e6) * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "mode": "mns", "sample": f"{args.ref_step_s:.0f} s of oracle work per step"},
        "cpu_baseline": {"value": round(value, 3), "unit": "Mpixel/s", "cores": threads, "kind": "oracle",
                         "sample": f"(image, threshold) pairs of the batch, encode + {DECODE_ITERS}-iteration decode, "
                                   f"{args.ref_step_s:.0f} s per step on {threads} threads"},
        "e2e": {"value": round(value, 3), "unit": "Mpixel/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# GPU arm

def run_ours(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_1501_02894_gb300 as fic

    fic.lib()
    batch = workload()
    n = len(batch)
    pixels = sum(im.size for im, _ in batch)
    plist = [fic.params("mns", 32, 4, t) for _, t in batch]
    host = [torch.from_numpy(im).pin_memory() for im, _ in batch]
    dimgs = [h.to(dev) for h in host]
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    with torch.cuda.stream(stream):
        enc = fic.EncodePlan(dimgs, plist, stream=stream)
        enc.run(stream)
        dec = fic.DecodePlan(enc.outs, stream=stream)
        dec.run(DECODE_ITERS, stream)
    stream.synchronize()
    nrec = []
    fits = 0
    for st in enc.outs:
        r, f = st.info_host(stream)
        nrec.append(r)
        fits += f
    ntops = [st.ntop for st in enc.outs]

    # CUDA graphs: one for the encode launch, one for the decode iterations
    g_enc, g_dec = torch.cuda.CUDAGraph(), torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g_enc, stream=stream):
            enc.run(stream)
        with torch.cuda.graph(g_dec, stream=stream):
            dec.run(DECODE_ITERS, stream)
    stream.synchronize()
    launches_per_step = 2 + 1 + DECODE_ITERS  # encoder + pack, decode setup + one launch per iteration

    def step():
        g_enc.replay()
        g_dec.replay()

    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = str(local)
    sampler = ClockSampler(gpu_id)
    sampler.start()
    time.sleep(0.2)
    # warm-up steps, then keep the GPU busy for --heat-s seconds (clock sampling)
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            flush.fill_(1)
            step()
    stream.synchronize()
    t_heat = time.perf_counter()
    while time.perf_counter() - t_heat < args.heat_s:
        with torch.cuda.stream(stream):
            for _ in range(20):
                flush.fill_(1)
                step()
        stream.synchronize()
    # outputs of the graphs must equal those of the direct launch
    ref0 = enc.outs[0].to_host(stream)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t_wall0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.fill_(i & 0xff)
            a, b, c = ev[i]
            a.record(stream)
            g_enc.replay()
            b.record(stream)
            g_dec.replay()
            c.record(stream)
    stream.synchronize()
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter() - t_wall0
    clocks = sampler.stop()
    enc_ms = [a.elapsed_time(b) for a, b, _ in ev]
    dec_ms = [b.elapsed_time(c) for _, b, c in ev]
    step_ms = [e + d for e, d in zip(enc_ms, dec_ms)]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = world * pixels / (ms_per_step * 1e-3) / 1e6

    chk = enc.outs[0].to_host(stream)
    assert np.array_equal(chk["records"].view(np.uint8), ref0["records"].view(np.uint8)), "graph replay changed output"

    # ---- end to end through the public API: pinned host images in, streams and
    # decoded images out, copies inside the timed region
    out_host = [torch.empty((512, 512), dtype=torch.uint8).pin_memory() for _ in range(n)]
    rec_host = [torch.empty(st.records.numel(), dtype=torch.uint8).pin_memory() for st in enc.outs]
    info_host = torch.empty((n, 16), dtype=torch.int32).pin_memory()
    h2d = pixels
    d2h = pixels + sum(16 * r for r in nrec) + 64 * n
    e2e_ev = []
    with torch.cuda.stream(stream):
        for i in range(max(args.warmup, 3) + args.steps):
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.fill_(i & 0xff)
            s0.record(stream)
            for h, d in zip(host, dimgs):
                d.copy_(h, non_blocking=True)
            g_enc.replay()
            g_dec.replay()
            for j, st in enumerate(enc.outs):
                info_host[j].copy_(st.info, non_blocking=True)
                rec_host[j][: 16 * nrec[j]].copy_(st.records[: 16 * nrec[j]], non_blocking=True)
                out_host[j].copy_(dec.outs[j], non_blocking=True)
            s1.record(stream)
            e2e_ev.append((s0, s1))
    stream.synchronize()
    e2e_ms = [a.elapsed_time(b) for a, b in e2e_ev[max(args.warmup, 3):]]
    e2e_ms_mean = sum(e2e_ms) / len(e2e_ms)
    if world > 1:
        t = torch.tensor([e2e_ms_mean], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms_mean = float(t.item())
    e2e_value = world * pixels / (e2e_ms_mean * 1e-3) / 1e6

    # ---- roofline of the dominant kernel (HBM bound): algorithmic bytes per launch
    peak, peak_kind = load_peaks()
    enc_bytes = sum(im.size for im, _ in batch) + sum(16 * r for r in nrec) + sum(8 * t + 4 for t in ntops)
    dec_bytes_iter = 2 * pixels + sum(16 * r for r in nrec) + sum(4 * (t + 1) for t in ntops)
    enc_launch_ms = sum(enc_ms) / len(enc_ms)
    dec_launch_ms = sum(dec_ms) / len(dec_ms) / DECODE_ITERS
    enc_gbs = enc_bytes / (enc_launch_ms * 1e-3) / 1e9
    dec_gbs = dec_bytes_iter / (dec_launch_ms * 1e-3) / 1e9
    if sum(enc_ms) >= sum(dec_ms):
        dom, ach, key = "mns_encode_kernel", enc_gbs, "mns_encode_kernel_cfg2"
    else:
        dom, ach, key = "decode_iter_kernel", dec_gbs, "decode_iter_kernel_cfg2"
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4), "peak_kind": peak_kind, "traffic": traffic_from_profile(key),
                "kernels": {"mns_encode": {"ms_per_launch": round(enc_launch_ms, 5), "alg_bytes": enc_bytes,
                                           "GB_s": round(enc_gbs, 1)},
                            "decode_iter": {"ms_per_launch": round(dec_launch_ms, 5), "alg_bytes": dec_bytes_iter,
                                            "GB_s": round(dec_gbs, 1)}}}

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "Mpixel/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "images": n, "pixels_per_step": pixels, "l2": "flushed (256 MiB write) before every step",
                   "parallelism": f"replicas x{world}", "graph": "CUDA graphs (encode, decode)"},
        "encode_mpix_s": round(world * pixels / (sum(enc_ms) / len(enc_ms) * 1e-3) / 1e6, 3),
        "fits_per_s": round(world * fits / (ms_per_step * 1e-3), 1),
        "fits_per_step": fits,
        "records_per_step": int(sum(nrec)),
        "wall_s_timed": round(t_wall, 3),
        "roofline": roofline,
        "e2e": {"value": round(e2e_value, 3), "unit": "Mpixel/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        v, done, dt = time_oracle(batch, args.cpu_s, threads)
        line["cpu_baseline"] = {"value": round(v, 3), "unit": "Mpixel/s", "cores": threads, "kind": "oracle",
                                "sample": f"{done} (image, threshold) pairs of the batch, encode + "
                                          f"{DECODE_ITERS}-iteration decode, {dt:.1f} s on {threads} threads"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-s", type=float, default=15.0, help="seconds of oracle work for cpu_baseline")
    ap.add_argument("--ref-step-s", type=float, default=10.0, help="oracle seconds per reference step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--heat-s", type=float, default=2.0, help="busy seconds before the timed steps (clock sampling)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
