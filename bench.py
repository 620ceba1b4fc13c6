"""Benchmark: encode + two-erasure recovery throughput of the cyclic-group
RAID-6 code on GB300, in user-data GB/s, with the HBM roofline of the tile
engine kernel.

Workload (one step): 8192 stripes of p = 13, N = 12 data strips, rows of
4 KiB (4.5 GiB of user data, 5.25 GiB moved per operation), seeded random
bytes generated on the device.  A step runs, each as ONE launch over all
stripes: encode (P and Q), then recovery of a uniformly drawn erasure pair
per stripe for each class of Lemma 3.1.2 -- two data strips, data + P,
data + Q, P + Q.  User bytes per step = 5 x N x (p-1) x C x stripes.  Every
operation moves (N+2)(p-1)C bytes per stripe; each operation's inputs (5.25
GiB) are far larger than the 129 MB L2, so no flush is needed.

At N = 1 the line also carries the two other forms of the same code, each
with its own clock record: `batched` -- the uneven 50k-stripe workload in
waves, one persistent launch per wave against one launch per stripe on the
same bytes (and a per-prime split) -- and `serve` -- a Poisson request stream
swept from 0.1x to 2x of saturation, continuous batching against one launch
per request (p50/p99 latency, user GB/s, kernel launches).

Multi-GPU: stripes are independent codes, so each rank runs the same
workload on its own stripes (weak scaling, no collective on the data path);
the timing is the max over ranks.

--impl reference times the CPU oracle on a bounded sample of the same
workload (the reference arm: the paper ships no code to run).
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

P, N, C, S = 13, 12, 4096, 8192
SEED = 1
CLASSES = ("dd", "dp", "dq", "pq")
METRIC = "encode & 2-erasure recovery user GB/s vs HBM roofline"
WORKLOAD = "p=13, N=12 data strips + P + Q, 12 rows x 4 KiB per strip, 8192 stripes; " \
           "encode + per-stripe random DD/DP/DQ/PQ recovery, one launch per op"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="leave the batched sub-object out of the line")
    ap.add_argument("--no-serve", action="store_true", help="leave the serving sub-object out of the line")
    ap.add_argument("--stripes", type=int, default=None,
                    help="stripes per GPU (default: the workload's own, 8192 for p13n12; other values are "
                         "profiling cases, not bench lines)")
    ap.add_argument("--workload", default="p13n12",
                    choices=["p13n12", "p5n4", "p59n58", "qext", "h17", "h257", "h257n16", "p13n12_ops",
                             "batched", "serve"],
                    help="p13n12: the bench line; p5n4 / p59n58: the p=5 and p=59 plain geometries; "
                         "qext: extended Q-parity, p=59 with 117 data strips; "
                         "h17: the horizontal Z_17 representation (one element per 16-bit word); "
                         "h257 / h257n16: Z_257 (256-bit elements), N=256 / N=16; "
                         "p13n12_ops: degraded read and small write on the bench line's geometry; "
                         "batched: the uneven 50k-stripe batch vs per-stripe launches; "
                         "serve: Poisson request stream, continuous batching vs per-job launches")
    ap.add_argument("--serve-requests", type=int, default=20000)
    ap.add_argument("--pool-gb", type=float, default=40.0)
    ap.add_argument("--batch-jobs", type=int, default=50000)
    ap.add_argument("--arena-gb", type=float, default=100.0)
    ap.add_argument("--schedule", default="dynamic", choices=["static", "dynamic"])
    ap.add_argument("--tuning", default="autotune", choices=["autotune", "default"],
                    help="batched: autotune the layout on the first wave (the bench line), or keep the default "
                         "layout (profiling captures)")
    ap.add_argument("--row-align", type=int, default=16,
                    help="batched: bytes each row stride is rounded up to (16 = packed rows, the workload as "
                         "specified; 128 = rows padded to whole L2 lines)")
    return ap.parse_args()


def user_bytes_per_op(stripes):
    return N * (P - 1) * C * stripes


def moved_bytes_per_op(stripes):
    return (N + 2) * (P - 1) * C * stripes


def max_over_ranks(ms, device=None):
    """The timed region's duration as the slowest rank saw it (all ranks get it)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(user_bytes_per_rank_step, steps, world, ms):
    """Whole-job throughput: the user bytes every rank processed over the slowest
    rank's time (weak scaling: each rank encodes and recovers its own stripes)."""
    return user_bytes_per_rank_step * steps * world / (ms * 1e-3) / 1e9


def peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples taken while the timed region runs."""

    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sms, maxs, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                maxs.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sms) if sms else None,
                "sm_max_mhz": max(maxs) if maxs else None,
                "reasons": sorted(reasons), "samples": len(sms)}


# --------------------------------------------------------------- GPU arm

def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_cs_0611109_gb300 import build, inputs
    build.build()
    from paper_cs_0611109_gb300 import rcg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    ctx = rcg.Context(local)
    S = args.stripes or globals()["S"]
    sb = inputs.stripe_bytes(P, N, C)
    buf = torch.empty((S, N + 2, P - 1, C), dtype=torch.uint8, device=dev)
    rcg.rcg_fill_random(buf, S * sb, SEED + 100 * rank)
    L = rcg.make_layout(buf, P, N, C)
    ctx.encode(L, 0, S)
    pairs = {k: torch.from_numpy(inputs.random_pairs(20 + n + 100 * rank, N, S, k)).to(dev)
             for n, k in enumerate(CLASSES)}

    def step(evs=None):
        ops = [lambda: ctx.encode(L, 0, S)] + [
            (lambda k=k: ctx.recover_many(L, 0, S, pairs[k])) for k in CLASSES]
        for n, op in enumerate(ops):
            if evs is not None:
                evs[n][0].record(stream)
            op()
            if evs is not None:
                evs[n][1].record(stream)
        return len(ops)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ctx.last_device_status() != 0:
        raise RuntimeError("device status word set during warm-up")

    launch_evs = [[[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(5)]
                  for _ in range(args.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    t0.record(stream)
    launches = 0
    for k in range(args.steps):
        launches += step(launch_evs[k])
    t1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    ms = max_over_ranks(t0.elapsed_time(t1), dev)
    status = ctx.last_device_status()
    if status != 0:
        raise RuntimeError("device status word %#x after the timed region" % status)

    per_launch = [[launch_evs[k][n][0].elapsed_time(launch_evs[k][n][1]) for k in range(args.steps)]
                  for n in range(5)]
    all_launch = [x for row in per_launch for x in row]
    avg_launch_ms = sum(all_launch) / len(all_launch)
    peak, peak_kind = peak_hbm()
    achieved = moved_bytes_per_op(S) / (avg_launch_ms * 1e-3) / 1e9

    user_step = 5 * user_bytes_per_op(S)
    value = whole_job_gbs(user_step, args.steps, world, ms)
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (SplitMix64 bytes generated on the device, seed %d)" % SEED,
        "config": {"workload": WORKLOAD if S == 8192 else "profiling case: %d stripes" % S,
                   "p": P, "n_data": N, "row_bytes": C, "stripes_per_gpu": S,
                   "ops_per_step": ["encode", "recover_dd", "recover_dp", "recover_dq", "recover_pq"],
                   "user_bytes_per_step_per_gpu": user_step,
                   "hbm_bytes_per_op_per_gpu": moved_bytes_per_op(S),
                   "l2": "inputs (5.25 GiB per op) far larger than the 129 MB L2; no flush",
                   "parallelism": "stripe-sharded x%d, no collective" % world},
        "roofline": {"bound": "hbm", "kernel": "rcg_tile_engine<wide>",
                     "achieved": round(achieved, 1), "peak": peak, "peak_kind": peak_kind,
                     "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
                     "avg_launch_ms": round(avg_launch_ms, 4),
                     "bytes_per_launch": moved_bytes_per_op(S)},
        "per_op": {name: {"ms": round(sum(row) / len(row), 4),
                          "user_gbs": round(user_bytes_per_op(S) / (sum(row) / len(row) * 1e-3) / 1e9, 1),
                          "hbm_frac": round(moved_bytes_per_op(S) / (sum(row) / len(row) * 1e-3) / 1e9 / peak, 4)}
                   for name, row in zip(["encode", "dd", "dp", "dq", "pq"], per_launch)},
        "gpu_launches": launches,
        "clocks": clk,
    }
    out["roofline"]["traffic"] = measured_traffic(S)

    if not args.no_e2e:
        out["e2e"] = e2e_ours(ctx, rcg, torch, dev, stream, pairs, args, world, S)
    del buf
    torch.cuda.empty_cache()
    if world == 1:
        # the batched and served forms of the same code, each measured against
        # one launch per stripe / per request on the same GPU (single-GPU forms)
        if not args.no_batched:
            out["batched"] = measure_batched(args, ctx, rcg, torch)
        if not args.no_serve:
            out["serve"] = measure_serve(args, ctx, rcg, torch)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(budget_s=15.0)
        out["cpu_word_level"] = cpu_word_level()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return out if rank == 0 else None


def kernel_hash():
    """Hash of the tile engine's source file: DRAM counters taken on another
    version of the kernel are not reported."""
    import hashlib
    h = hashlib.sha256()
    h.update(open(os.path.join(ROOT, "paper_cs_0611109_gb300", "csrc", "rcg_engine.cu"), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(stripes):
    """dram__bytes_read.sum + dram__bytes_write.sum per launch from the
    committed ncu summary, scaled to `stripes` by the stripes it captured;
    None when the summary is missing or was taken on other kernel sources."""
    import re
    path = os.path.join(ROOT, "profiles", "rcg_tile_engine_p13n12_traffic.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    h = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    b = re.search(r"dram_bytes_per_launch:\s*([0-9]+)", text)
    n = re.search(r"captured_stripes:\s*([0-9]+)", text)
    if not (h and b and n) or h.group(1) != kernel_hash():
        return None
    return int(int(b.group(1)) * stripes / int(n.group(1)))


def e2e_ours(ctx, rcg, torch, dev, stream, pairs, args, world, S):
    """The same step through the public API with the stripes in pinned HOST
    memory (rcg_encode_host / rcg_recover_many_host): every step uploads what
    each operation reads and brings its results back to the host stripes."""
    from paper_cs_0611109_gb300 import inputs
    host = torch.empty((S, N + 2, P - 1, C), dtype=torch.uint8).pin_memory()
    dbuf = torch.empty((S, N + 2, P - 1, C), dtype=torch.uint8, device=dev)
    rcg.rcg_fill_random(dbuf, S * inputs.stripe_bytes(P, N, C), SEED)
    ctx.encode(rcg.make_layout(dbuf, P, N, C), 0, S)
    host.copy_(dbuf)
    torch.cuda.synchronize()
    del dbuf
    torch.cuda.empty_cache()
    HL = rcg.make_layout(host, P, N, C)
    pairs_host = {k: pairs[k].cpu().numpy() for k in CLASSES}
    strip = (P - 1) * C

    marks = []

    def step(record=False):
        def mark():
            if record:
                e = torch.cuda.Event(enable_timing=True)
                e.record(stream)
                marks.append(e)
        mark()
        ctx.encode_host(HL, 0, S, stream)
        mark()
        for k in CLASSES:
            ctx.recover_many_host(HL, 0, S, pairs_host[k], stream)
        mark()

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    steps = max(2, args.steps // 4)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        step(record=True)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    enc_each = [marks[3 * i].elapsed_time(marks[3 * i + 1]) for i in range(steps)]
    rec_each = [marks[3 * i + 1].elapsed_time(marks[3 * i + 2]) / len(CLASSES) for i in range(steps)]
    enc_ms, rec_ms = statistics.median(enc_each), statistics.median(rec_each)
    if ctx.last_device_status() != 0:
        raise RuntimeError("device status word set in the end-to-end run")
    value = 5 * user_bytes_per_op(S) * steps * world / (ms * 1e-3) / 1e9
    link = pinned_link_gbs(torch, dev, stream)
    del host
    # encode: N strips in, P and Q out; recovery: the N surviving strips and the pair in,
    # the two rebuilt strips out
    h2d = S * N * strip + len(CLASSES) * S * (N * strip + 2)
    d2h = S * 2 * strip * (1 + len(CLASSES))
    return {"value": round(value, 2), "unit": "GB/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h,
            "api": "rcg_encode_host + rcg_recover_many_host (pinned host stripes)",
            "link_gbs": link,
            "per_op_ms": {"encode_host": round(enc_ms, 3), "recover_many_host": round(rec_ms, 3),
                          "encode_host_each": [round(x, 2) for x in enc_each],
                          "recover_many_host_each": [round(x, 2) for x in rec_each]},
            # the copies of one direction cannot beat the link: an upper bound
            "ceiling_gbs": round(5 * user_bytes_per_op(S) / max(h2d / link["h2d"], d2h / link["d2h"]) * world, 1)
            if link["h2d"] and link["d2h"] else None}


def pinned_link_gbs(torch, dev, stream, nbytes=1 << 30):
    """Plain pinned host<->device copy speed on this machine (one 1 GiB copy each
    way, best of 3): the ceiling of the end-to-end number."""
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    out = {}
    for name, fn in (("h2d", lambda: d.copy_(h, non_blocking=True)), ("d2h", lambda: h.copy_(d, non_blocking=True))):
        best = None
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        out[name] = round(nbytes / (best * 1e-3) / 1e9, 1)
    del h, d
    return out


# --------------------------------------------------------------- CPU oracle

def oracle_step(stripes, seed=SEED):
    """One step of the workload on `stripes` stripes with the CPU oracle;
    returns (seconds, user bytes)."""
    import numpy as np

    import oracle
    from paper_cs_0611109_gb300 import inputs
    host = np.ascontiguousarray(inputs.random_stripes(seed, P, N, C, stripes))
    t = time.perf_counter()
    oracle.encode(P, N, C, host, stripes)
    for n, k in enumerate(CLASSES):
        pairs = inputs.random_pairs(20 + n, N, stripes, k)
        oracle.recover(P, N, C, host, stripes, pairs=pairs)
    return time.perf_counter() - t, 5 * user_bytes_per_op(stripes)


def cpu_baseline(budget_s=15.0):
    import oracle
    oracle.build()
    t1, _ = oracle_step(1)
    n = max(1, int(budget_s / max(t1, 1e-3)))
    t, ub = oracle_step(n)
    return {"value": round(ub / t / 1e9, 6), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": "%d of the 8192 stripes, the full 5-op step (encode + DD/DP/DQ/PQ), "
                      "single-threaded bit-level C oracle, %.1f s" % (n, t)}


def cpu_word_level(stripes=512):
    """O2, the word-level multi-threaded CPU implementation of the oracle/
    directory, on all host cores: the full 5-op step on a sample of stripes."""
    import numpy as np

    import oracle
    from paper_cs_0611109_gb300 import inputs
    oracle.build_o2()
    host = np.ascontiguousarray(inputs.random_stripes(SEED, P, N, C, stripes))
    cores = os.cpu_count() or 1
    t = time.perf_counter()
    oracle.o2_encode(P, N, C, host, stripes, threads=cores)
    for n, k in enumerate(CLASSES):
        oracle.o2_recover(P, N, C, host, stripes, pairs=inputs.random_pairs(20 + n, N, stripes, k), threads=cores)
    dt = time.perf_counter() - t
    return {"value": round(5 * user_bytes_per_op(stripes) / dt / 1e9, 3), "unit": "GB/s", "cores": cores,
            "kind": "word-level C (oracle/rcg_o2.c, pthreads), context only",
            "sample": "%d of the 8192 stripes, the full 5-op step, %.2f s" % (stripes, dt)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    import oracle
    oracle.build()
    stripes = 2
    for _ in range(args.warmup):
        oracle_step(stripes)
    total_t = total_b = 0.0
    for _ in range(args.steps):
        t, b = oracle_step(stripes)
        total_t += t
        total_b += b
    value = total_b / total_t / 1e9
    return {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "GB/s",
            "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * total_t / args.steps, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic (SplitMix64 bytes, seed %d)" % SEED,
            "config": {"workload": WORKLOAD, "p": P, "n_data": N, "row_bytes": C,
                       "stripes_per_step": stripes},
            "cpu_baseline": {"value": round(value, 6), "unit": "GB/s", "cores": 1, "kind": "oracle",
                             "sample": "%d stripes per step of the 8192, full 5-op step" % stripes},
            "e2e": {"value": round(value, 6), "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


# ------------------------------------------------------ other geometries

GEOMETRIES = {
    # name: (p, N, C, stripes, seed, description)
    "p5n4": (5, 4, 1024, 1024, 0, "p=5, N=4 data strips + P + Q, 4 rows x 1 KiB per strip, 1024 stripes; "
                                "encode, then each of the 15 erasure pairs over all stripes, one launch per op"),
    "p59n58": (59, 58, 2048, 1024, 2, "p=59, N=58 data strips + P + Q, 58 rows x 2 KiB per strip, 1024 stripes; "
                                  "two-data recovery with a uniformly drawn pair per stripe, one launch per op"),
    "qext": (59, 117, 2048, 512, 6, "extended Q-parity (Section 3.3, equation qext): p=59, N=117 data strips "
                                    "+ P + Q, 58 rows x 2 KiB per strip, 512 stripes; encode and each recovery "
                                    "class, one launch per op"),
}


def geometry_ops(name, N, S, dev, torch):
    """(op name, per-stripe pair tensor or None for encode) of one step."""
    import numpy as np

    from paper_cs_0611109_gb300 import inputs
    P_ = GEOMETRIES[name][0]
    if name == "p5n4":
        return [("encode", None)] + [("pair_%d_%d" % (i, j), torch.from_numpy(
            np.tile(np.array([[i, j]], dtype=np.uint8), (S, 1))).to(dev))
            for i in range(N + 2) for j in range(i + 1, N + 2)]
    if name == "p59n58":
        return [("dd", torch.from_numpy(inputs.random_pairs(22, N, S, "dd")).to(dev))]
    # qext: encode, and one launch per recovery class; pairs drawn uniformly within the class
    rng = np.random.Generator(np.random.PCG64(61))

    def draw(lo_i, hi_i, lo_j, hi_j):
        out = np.empty((S, 2), dtype=np.uint8)
        for s in range(S):
            while True:
                i, j = int(rng.integers(lo_i, hi_i)), int(rng.integers(lo_j, hi_j))
                if i < j:
                    break
            out[s] = (i, j)
        return torch.from_numpy(out).to(dev)

    return [("encode", None),
            ("dd_regular", draw(0, P_, 0, P_)),          # (1 + x^z)
            ("dd_mixed", draw(0, P_, P_, N)),            # trinomial inverse
            ("dd_extended", draw(P_, N, P_, N)),         # (1 + x^z) after x^(-m_i)
            ("dp_extended", draw(P_, N, N, N + 1)),      # (1 + x^m) D = dQ
            ("dq_extended", draw(P_, N, N + 1, N + 2)),
            ("dd_any", torch.from_numpy(inputs.random_pairs(23, N, S, "dd")).to(dev)),
            ("any", torch.from_numpy(inputs.random_pairs(24, N, S, "any")).to(dev))]


def run_geometry(args):
    """One plain (one launch per op over all stripes) geometry: every op timed
    with CUDA events on the launching stream; HBM fraction per op against the
    measured copy peak."""
    import torch

    from paper_cs_0611109_gb300 import build, inputs
    build.build()
    from paper_cs_0611109_gb300 import rcg

    p, n, c, S, seed, desc = GEOMETRIES[args.workload]
    if args.stripes and args.stripes != S:
        S, desc = args.stripes, "profiling case: %d stripes of %s" % (args.stripes, desc)
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    ctx = rcg.Context(0)
    buf = torch.empty((S, n + 2, p - 1, c), dtype=torch.uint8, device=dev)
    rcg.rcg_fill_random(buf, S * inputs.stripe_bytes(p, n, c), seed)
    L = rcg.make_layout(buf, p, n, c)
    ctx.encode(L, 0, S)
    ops = geometry_ops(args.workload, n, S, dev, torch)
    # an L2 flush between launches when one op's traffic fits in L2: a READ of
    # 256 MB, so L2 holds clean unrelated lines (a write would leave dirty
    # lines that the timed kernel then pays to write back)
    moved = (n + 2) * (p - 1) * c * S
    flush = torch.ones(256 << 20 >> 3, dtype=torch.int64, device=dev) if moved < (512 << 20) else None

    def run(name, pairs):
        if pairs is None:
            ctx.encode(L, 0, S)
        else:
            ctx.recover_many(L, 0, S, pairs)

    for _ in range(args.warmup):
        for name, pairs in ops:
            run(name, pairs)
    torch.cuda.synchronize()
    if ctx.last_device_status() != 0:
        raise RuntimeError("device status word set during warm-up")
    evs = {name: [] for name, _ in ops}
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    for _ in range(args.steps):
        for name, pairs in ops:
            if flush is not None:
                flush.sum()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run(name, pairs)
            e1.record(stream)
            evs[name].append((e0, e1))
    torch.cuda.synchronize()
    clk = clocks.stop()
    status = ctx.last_device_status()
    if status:
        raise RuntimeError("device status word %#x" % status)
    peak, kind = peak_hbm()
    user = n * (p - 1) * c * S
    per_op, total_ms = {}, 0.0
    for name, _ in ops:
        ms = sum(a.elapsed_time(b) for a, b in evs[name]) / len(evs[name])
        total_ms += ms
        per_op[name] = {"ms": round(ms, 4), "user_gbs": round(user / (ms * 1e-3) / 1e9, 1),
                        "hbm_gbs": round(moved / (ms * 1e-3) / 1e9, 1),
                        "hbm_frac": round(moved / (ms * 1e-3) / 1e9 / peak, 4)}
    achieved = moved * len(ops) / (total_ms * 1e-3) / 1e9
    ref = None
    if flush is not None:
        # what any single launch of this traffic achieves here: a plain
        # elementwise kernel that reads as many bytes as an op reads and writes
        # the 2 strips it writes, timed the same way (after the same L2 flush)
        wr = torch.empty(2 * (p - 1) * c * S, dtype=torch.uint8, device=dev)
        rd = torch.empty(max(n, 2) * (p - 1) * c * S, dtype=torch.uint8, device=dev)
        a_in, b_in = rd[:wr.numel()], rd[wr.numel():2 * wr.numel()]
        tot = 0.0
        for it in range(args.warmup + args.steps):
            flush.sum()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            torch.bitwise_xor(a_in, b_in, out=wr)
            e1.record(stream)
            torch.cuda.synchronize()
            if it >= args.warmup:
                tot += e0.elapsed_time(e1)
        ms_ref = tot / args.steps
        ref = {"what": "torch.bitwise_xor reading %d B and writing %d B, after the same L2 flush"
                       % (2 * wr.numel(), wr.numel()),
               "ms": round(ms_ref, 4), "hbm_frac": round(3 * wr.numel() / (ms_ref * 1e-3) / 1e9 / peak, 4),
               "note": "a launch this small is bound by launch and DRAM latency, not by bandwidth"}
        del rd, wr
    batched = None
    if args.workload == "p5n4":
        batched = p5n4_sixteen_in_one_batch(args, ctx, rcg, torch, buf, ops, flush, stream)
    ctx.close()
    line_gbs = user * len(ops) / (total_ms * 1e-3) / 1e9
    out = {"metric": METRIC, "value": round(line_gbs, 2), "unit": "GB/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms, 4),
            "higher_is_better": True, "dtype": "u8",
            "data": "synthetic (SplitMix64 bytes generated on the device, seed %d)" % seed,
            "config": {"workload": desc, "p": p, "n_data": n, "row_bytes": c, "stripes": S,
                       "hbm_bytes_per_op": moved,
                       "l2": "256 MB buffer read between launches" if flush is not None else
                             "inputs far larger than the 129 MB L2; no flush"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1),
                         # the launch's kernel: the column kernel for p <= 7, else the
                         # tile engine's shape for the launch's traffic (256 MB threshold)
                         "kernel": "rcg_column_kernel" if p <= 7 else
                                   "rcg_tile_engine<wide>" if moved >= (256 << 20) else "rcg_tile_engine<pair>",
                         "peak": peak, "peak_kind": kind, "unit": "GB/s", "frac": round(achieved / peak, 4)},
            "per_op": per_op, "gpu_launches": len(ops) * args.steps, "clocks": clk,
            "small_launch_reference": ref}
    if batched is not None:
        # the line's value and roofline: the 16 operations as one batch launch
        out["plain_one_launch_per_op"] = {"user_gbs": round(line_gbs, 2), "ms_per_step": round(total_ms, 4),
                                          "roofline": out["roofline"]}
        out["value"] = batched["user_gbs"]
        out["ms_per_step"] = batched["ms"]
        out["roofline"] = batched.pop("roofline")
        out["batched_16_ops"] = batched
        out["gpu_launches"] += batched["launches"]
        out["config"]["workload"] = desc + "; the line's value: the same 16 operations on 16 copies of the " \
                                           "stripes as ONE batch launch (column kernel, 384 MB)"
    return out


def p5n4_sixteen_in_one_batch(args, ctx, rcg, torch, buf, ops, flush, stream):
    """The p = 5 geometry's 16 operations (encode and the 15 erasure pairs),
    each on a copy of the 1024 stripes of its own, as ONE batch launch: 384 MB,
    about three times the L2, which a single 24 MB operation cannot fill.
    A 256 MB read flushes L2 between timed launches."""
    p, n, c, S = GEOMETRIES["p5n4"][:4]
    copies = torch.empty((len(ops),) + tuple(buf.shape), dtype=torch.uint8, device=buf.device)
    for k in range(len(ops)):
        copies[k].copy_(buf)  # encoded stripes: the recoveries rebuild the bytes they hold
    jobs = []
    for k, (name, pairs) in enumerate(ops):
        L = rcg.make_layout(copies[k], p, n, c)
        if pairs is None:
            jobs.append(rcg.make_job(L, 0, S, rcg.RCG_OP_ENCODE))
        else:
            i, j = (int(x) for x in pairs[0].tolist())
            jobs.append(rcg.make_job(L, 0, S, rcg.RCG_OP_RECOVER, i, j))
    prepared = ctx.batch_prepare(jobs)
    for _ in range(max(3, args.warmup)):
        ctx.batch_launch(prepared)
    torch.cuda.synchronize()
    evs = []
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    for _ in range(args.steps):
        flush.sum()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.batch_launch(prepared)
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    clk = clocks.stop()
    rcg.rcg_batch_free(prepared)
    if ctx.last_device_status():
        raise RuntimeError("device status word set by the 16-operation batch")
    ms = sum(a.elapsed_time(b) for a, b in evs) / len(evs)
    moved = len(ops) * (n + 2) * (p - 1) * c * S
    user = len(ops) * n * (p - 1) * c * S
    peak, kind = peak_hbm()
    achieved = moved / (ms * 1e-3) / 1e9
    del copies
    return {"ms": round(ms, 4), "user_gbs": round(user / (ms * 1e-3) / 1e9, 1), "hbm_gbs": round(achieved, 1),
            "hbm_frac": round(achieved / peak, 4), "bytes_per_launch": moved, "launches": args.steps,
            "l2": "256 MB buffer read between launches", "clocks": clk,
            "roofline": {"bound": "hbm", "kernel": "rcg_column_batch_param<5> (table in the parameter block)", "achieved": round(achieved, 1),
                         "peak": peak, "peak_kind": kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                         "avg_launch_ms": round(ms, 4), "bytes_per_launch": moved}}


# ---------------------------------------------- degraded read, small write

def run_ops(args):
    """The degraded read (rebuild one strip without touching the stripe) and
    the small write (replace a data strip, update P and Q) over the c2
    geometry: 8192 stripes, one launch per op (a batch of one job), each op
    under both engine shapes (wide: one CTA per SM; pair: two).
    Algorithmic bytes per stripe: degraded read (N+1)(p-1)C -- N strips read,
    one written; small write 7(p-1)C -- old strip, new strip, P, Q read; strip,
    P, Q written."""
    import torch

    from paper_cs_0611109_gb300 import build
    build.build()
    from paper_cs_0611109_gb300 import rcg

    S = args.stripes or globals()["S"]
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    ctx = rcg.Context(0)
    buf = torch.empty((S, N + 2, P - 1, C), dtype=torch.uint8, device=dev)
    rcg.rcg_fill_random(buf, buf.numel(), SEED)
    L = rcg.make_layout(buf, P, N, C)
    ctx.encode(L, 0, S)
    aux = torch.empty((S, P - 1, C), dtype=torch.uint8, device=dev)
    rcg.rcg_fill_random(aux, aux.numel(), SEED + 7)
    strip = (P - 1) * C
    ops = [("degraded_read_data", rcg.make_job(L, 0, S, rcg.RCG_OP_DEGRADED_READ, 0, 3, aux), (N + 1) * strip, N * strip),
           ("degraded_read_q", rcg.make_job(L, 0, S, rcg.RCG_OP_DEGRADED_READ, 0, N + 1, aux), (N + 1) * strip, N * strip),
           ("degraded_read_p", rcg.make_job(L, 0, S, rcg.RCG_OP_DEGRADED_READ, 0, N, aux), (N + 1) * strip, N * strip),
           ("small_write", rcg.make_job(L, 0, S, rcg.RCG_OP_UPDATE, 5, 0, aux), 7 * strip, strip)]
    shapes = {"wide": rcg.RCG_SHAPE_WIDE, "pair": rcg.RCG_SHAPE_PAIR}
    prepared = {}
    for sh, code in shapes.items():
        ctx.set_batch_tuning({"shape": code, "schedule": rcg.RCG_SCHED_DYNAMIC, "item_bytes": 0, "tile_div": 1,
                              "ring": rcg.RCG_RING_FIXED})
        for name, job, _, _ in ops:
            prepared[(sh, name)] = ctx.batch_prepare([job])
    ctx.set_batch_tuning(None)
    keys = list(prepared)
    evs = {k: [] for k in keys}
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    # one shape at a time: the batch slots' graphs are captured per shape, so
    # the warm-up launches of each shape recapture them outside the timing
    for sh in shapes:
        mine = [k for k in keys if k[0] == sh]
        for _ in range(args.warmup):
            for k in mine:
                ctx.batch_launch(prepared[k])
        torch.cuda.synchronize()
        for _ in range(args.steps):
            for k in mine:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.batch_launch(prepared[k])
                e1.record(stream)
                evs[k].append((e0, e1))
        torch.cuda.synchronize()
    clk = clocks.stop()
    status = ctx.last_device_status()
    if status:
        raise RuntimeError("device status word %#x" % status)
    peak, kind = peak_hbm()
    per_op, tot_ms, tot_moved = {}, 0.0, 0
    for (sh, name) in keys:
        moved1 = next(m for n_, _, m, _ in ops if n_ == name)
        ms = sum(a.elapsed_time(b) for a, b in evs[(sh, name)]) / len(evs[(sh, name)])
        moved = moved1 * S
        if sh == "wide":
            tot_ms += ms
            tot_moved += moved
        per_op.setdefault(name, {})[sh] = {"ms": round(ms, 4), "hbm_gbs": round(moved / (ms * 1e-3) / 1e9, 1),
                                           "hbm_frac": round(moved / (ms * 1e-3) / 1e9 / peak, 4), "bytes": moved}
    for b in prepared.values():
        rcg.rcg_batch_free(b)
    ctx.close()
    achieved = tot_moved / (tot_ms * 1e-3) / 1e9
    return {"metric": "degraded read and small write: HBM GB/s vs roofline", "value": round(achieved, 1),
            "unit": "GB/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(tot_ms, 4), "higher_is_better": True, "dtype": "u8",
            "data": "synthetic (SplitMix64 bytes generated on the device, seed %d)" % SEED,
            "config": {"workload": "p=13, N=12, 12 rows x 4 KiB per strip, %d stripes: degraded read of data "
                                   "strip 3, of Q and of P, small write of data strip 5; one launch each, "
                                   "under the wide and the pair engine shape (value: wide)" % S,
                       "l2": "inputs far larger than the 129 MB L2; no flush"},
            "roofline": {"bound": "hbm", "kernel": "rcg_tile_engine<wide>", "achieved": round(achieved, 1),
                         "peak": peak, "peak_kind": kind, "unit": "GB/s", "frac": round(achieved / peak, 4)},
            "per_op": per_op, "gpu_launches": len(keys) * args.steps, "clocks": clk}


# ------------------------------------------------ horizontal representation

# name: (p, N, strip bytes, stripes, seed, description)
HGEOMETRIES = {
    "h17": (17, 16, 65536, 4096, 5, "horizontal Z_17 (Section 4.5): p=17, N=16 data strips + P + Q of 64 KiB "
                                    "(32768 16-bit elements), %d stripes; encode + DD/DP/DQ/PQ, one launch per op"),
    "h257": (257, 256, 65536, 256, 8, "horizontal Z_257 (Section 3.4): p=257, N=256 data strips + P + Q of 64 KiB "
                                      "(2048 256-bit elements), %d stripes; encode + DD/DP/DQ/PQ, one launch per op"),
    "h257n16": (257, 16, 65536, 4096, 9, "horizontal Z_257: p=257, N=16 data strips + P + Q of 64 KiB, %d stripes; "
                                         "encode + DD/DP/DQ/PQ, one launch per op (recovery arithmetic per byte "
                                         "16x that of N=256)"),
}


def run_h(args):
    """The horizontal representation of Section 4.5 (one ring element per
    (p-1)-bit field): Z_17 (16-bit words) or Z_257 (256-bit elements); encode
    and one launch per recovery class with a uniformly drawn pair per stripe
    (16-bit pairs at p = 257)."""
    import numpy as np
    import torch

    from paper_cs_0611109_gb300 import build, inputs
    build.build()
    from paper_cs_0611109_gb300 import rcg

    p, n, B, S, seed, desc = HGEOMETRIES[args.workload]
    if args.stripes and args.stripes != S:
        S = args.stripes
        desc = "profiling case: " + desc
    desc = desc % S
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    ctx = rcg.Context(0)
    buf = torch.empty((S, n + 2, B), dtype=torch.uint8, device=dev)
    rcg.rcg_fill_random(buf, buf.numel(), seed)
    L = rcg.make_hlayout(buf, p, n, B)
    ctx.h_encode(L, 0, S)
    wide = np.uint16 if p == 257 else np.uint8

    def pairs_of(m, k):
        pr = inputs.random_pairs(3500 + m, n, S, k, dtype=wide)
        return torch.from_numpy(pr.view(np.int16) if p == 257 else pr).to(dev)

    ops = [("encode", None)] + [(k, pairs_of(m, k)) for m, k in enumerate(CLASSES)]
    moved = (n + 2) * B * S
    user = n * B * S

    def run(pairs):
        if pairs is None:
            ctx.h_encode(L, 0, S)
        else:
            ctx.h_recover_many(L, 0, S, pairs)

    for _ in range(args.warmup):
        for _, pr in ops:
            run(pr)
    torch.cuda.synchronize()
    if ctx.last_device_status() != 0:
        raise RuntimeError("device status word set during warm-up")
    evs = {name: [] for name, _ in ops}
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    for _ in range(args.steps):
        for name, pr in ops:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run(pr)
            e1.record(stream)
            evs[name].append((e0, e1))
    torch.cuda.synchronize()
    clk = clocks.stop()
    status = ctx.last_device_status()
    if status:
        raise RuntimeError("device status word %#x" % status)
    peak, kind = peak_hbm()
    per_op, total_ms = {}, 0.0
    for name, _ in ops:
        ms = sum(a.elapsed_time(b) for a, b in evs[name]) / len(evs[name])
        total_ms += ms
        per_op[name] = {"ms": round(ms, 4), "user_gbs": round(user / (ms * 1e-3) / 1e9, 1),
                        "hbm_gbs": round(moved / (ms * 1e-3) / 1e9, 1),
                        "hbm_frac": round(moved / (ms * 1e-3) / 1e9 / peak, 4)}
    achieved = moved * len(ops) / (total_ms * 1e-3) / 1e9
    ctx.close()
    return {"metric": METRIC, "value": round(user * len(ops) / (total_ms * 1e-3) / 1e9, 2), "unit": "GB/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms, 4),
            "higher_is_better": True, "dtype": "u16 lanes" if p == 17 else "u256 elements",
            "data": "synthetic (SplitMix64 bytes generated on the device, seed %d)" % seed,
            "config": {"workload": desc, "p": p, "n_data": n, "strip_bytes": B, "stripes": S,
                       "hbm_bytes_per_op": moved, "l2": "inputs far larger than the 129 MB L2; no flush"},
            "roofline": {"bound": "hbm", "kernel": "rcg_h_kernel<16>" if p == 17 else "rcg_h257_kernel",
                         "achieved": round(achieved, 1), "peak": peak, "peak_kind": kind, "unit": "GB/s",
                         "frac": round(achieved / peak, 4)},
            "per_op": per_op, "gpu_launches": len(ops) * args.steps, "clocks": clk}


# ----------------------------------------------------------- batched form

def gpu_busy(torch, seconds):
    """An untimed spin of about `seconds` on the current stream (about 2e9 SM
    cycles a second), so that a launch the host submits meanwhile is queued
    before the GPU gets to it."""
    torch.cuda._sleep(int(seconds * 2.0e9))


def batched_waves(jobs, arena_bytes, row_align):
    """Cut the job list into waves whose stripes fit the device arena; each
    entry is (job, byte offset in the arena)."""
    align = lambda x: (x + 255) // 256 * 256
    rs_of = lambda c: (c + row_align - 1) // row_align * row_align
    footprint = lambda j: (j["n"] + 2) * (j["p"] - 1) * rs_of(j["c"])
    waves, cur, used = [], [], 0
    for j in jobs:
        sz = align(footprint(j))
        if used + sz > arena_bytes and cur:
            waves.append(cur)
            cur, used = [], 0
        cur.append((j, used))
        used += sz
    if cur:
        waves.append(cur)
    return waves, rs_of, lambda w: w[-1][1] + align(footprint(w[-1][0]))


def measure_batched(args, ctx, rcg, torch):
    """The uneven batched workload: 50k single-stripe descriptors (p over
    {5,13,29,59}, N in [3,p-1], rows 512 B..64 KiB log-uniform, 60 % encode /
    40 % two-erasure recovery), 390 GiB with parity, so it runs in waves that
    fit the device arena.  Each wave is timed on the same bytes as ONE
    persistent batch launch (autotuned layout, and the default layout) and as
    one launch per stripe (rcg_encode / rcg_recover); each prime's jobs of the
    wave are also timed as a batch of their own (the per-prime split).
    Recovery stripes are encoded before the timed launches.  Clocks are
    sampled over the whole measurement."""
    from paper_cs_0611109_gb300 import inputs

    ctx.set_batch_schedule(rcg.RCG_SCHED_DYNAMIC if args.schedule == "dynamic" else rcg.RCG_SCHED_STATIC)
    stream = torch.cuda.current_stream()
    jobs = inputs.batched_jobs(3, args.batch_jobs)
    free = torch.cuda.mem_get_info()[0]
    arena_bytes = int(min(args.arena_gb * 1e9, 0.8 * free))
    arena = torch.empty(arena_bytes, dtype=torch.uint8, device="cuda")
    base = arena.data_ptr()
    if args.row_align < 16 or args.row_align % 16:
        raise SystemExit("--row-align must be a positive multiple of 16")
    waves, rs_of, wave_bytes = batched_waves(jobs, arena_bytes, args.row_align)

    tot = {"batched_ms": 0.0, "default_ms": 0.0, "per_stripe_ms": 0.0, "user": 0, "moved": 0,
           "launches_per_stripe": 0, "kernel_launches": 0}
    by_p = {}
    tuning = None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    for w in waves:
        rcg.rcg_fill_random(arena, wave_bytes(w), 3)
        lays = [rcg.make_layout(base + o, j["p"], j["n"], j["c"], rs_of(j["c"])) for j, o in w]
        pre = [rcg.make_job(L, 0, 1, rcg.RCG_OP_ENCODE) for L, (j, _) in zip(lays, w) if j["op"] == "recover"]
        if pre:
            assert ctx.batch_wait(ctx.batch_submit(pre))
        mix = [rcg.make_job(L, 0, 1, rcg.RCG_OP_ENCODE) if j["op"] == "encode" else
               rcg.make_job(L, 0, 1, rcg.RCG_OP_RECOVER, j["i"], j["j"]) for L, (j, _) in zip(lays, w)]
        if tuning is None and args.tuning == "autotune":
            # autotune the layout once, on the first wave (the batch itself runs
            # repeatedly: every op is idempotent on non-overlapping jobs)
            h0 = time.perf_counter()
            tuning = ctx.batch_autotune(mix)
            tot["autotune_s"] = round(time.perf_counter() - h0, 2)

        def time_batch(batch_jobs):
            # GPU time of one batch launch: the host submits it while the GPU
            # is still busy with an untimed spin, as it would be while a
            # previous batch runs, so the events time the GPU's work; the
            # host's part (prepare + the launch call) is returned beside it
            h0 = time.perf_counter()
            prepared = ctx.batch_prepare(batch_jobs)
            prep_ms = (time.perf_counter() - h0) * 1e3
            launch_ms = 0.0
            # warm-up: every batch slot of the context (16) holds this table
            # before the timed launch, so no slot grows or re-captures its
            # graph inside the timed region (a one-time cost per slot)
            for _ in range(17):
                h1 = time.perf_counter()
                t = ctx.batch_launch(prepared)
                launch_ms = max(launch_ms, (time.perf_counter() - h1) * 1e3)
                ctx.batch_wait(t)
            torch.cuda.synchronize()
            gpu_busy(torch, 2e-3 + 3e-3 * launch_ms)
            e0.record(stream)
            h1 = time.perf_counter()
            ctx.batch_launch(prepared)
            launch_ms = (time.perf_counter() - h1) * 1e3
            e1.record(stream)
            torch.cuda.synchronize()
            rcg.rcg_batch_free(prepared)
            tot["kernel_launches"] += 1
            return e0.elapsed_time(e1), prep_ms + launch_ms

        for mode in ("default", "tuned"):
            ctx.set_batch_tuning(None if mode == "default" else tuning)
            if mode == "default" and args.schedule == "static":
                ctx.set_batch_schedule(rcg.RCG_SCHED_STATIC)
            ms, prep_ms = time_batch(mix)
            tot["batched_ms" if mode == "tuned" else "default_ms"] += ms
            if mode == "tuned":
                # host part (validation, tiling, tensor maps, work items, and the
                # launch call: the table into pinned memory, the graph launch):
                # it can overlap the previous batch on the GPU; reported separately
                tot["host_ms"] = tot.get("host_ms", 0.0) + prep_ms
        # per-prime split: each prime's jobs of this wave as a batch of their own (tuned layout)
        for pr in sorted({j["p"] for j, _ in w}):
            sel = [job for job, (j, _) in zip(mix, w) if j["p"] == pr]
            ms, _ = time_batch(sel)
            d = by_p.setdefault(pr, {"ms": 0.0, "moved": 0, "user": 0, "jobs": 0})
            d["ms"] += ms
            d["jobs"] += len(sel)
            for j, _ in w:
                if j["p"] == pr:
                    d["moved"] += (j["n"] + 2) * (j["p"] - 1) * j["c"]
                    d["user"] += j["n"] * (j["p"] - 1) * j["c"]
        gpu_busy(torch, 2e-3)
        e0.record(stream)
        for L, (j, _) in zip(lays, w):
            if j["op"] == "encode":
                ctx.encode(L, 0, 1)
            else:
                ctx.recover(L, 0, j["i"], j["j"])
        e1.record(stream)
        torch.cuda.synchronize()
        tot["per_stripe_ms"] += e0.elapsed_time(e1)
        tot["launches_per_stripe"] += len(w)
        for j, _ in w:
            tot["user"] += j["n"] * (j["p"] - 1) * j["c"]
            tot["moved"] += (j["n"] + 2) * (j["p"] - 1) * j["c"]
    clk = clocks.stop()
    status = ctx.last_device_status()
    if status:
        raise RuntimeError("device status word %#x" % status)
    del arena
    torch.cuda.empty_cache()
    peak, kind = peak_hbm()
    gbs = lambda nbytes, ms: nbytes / (ms * 1e-3) / 1e9
    return {
        "workload": "batched uneven: %d single-stripe jobs, p in {5,13,29,59}, N in [3,p-1], rows 512 B..64 KiB "
                    "log-uniform, 60%% encode / 40%% two-erasure recovery; %d waves of <= %.0f GB, each one "
                    "persistent launch (CUDA graph) vs one launch per stripe on the same bytes"
                    % (len(jobs), len(waves), arena_bytes / 1e9),
        "row_stride": "packed (row stride = C)" if args.row_align == 16 else
                      "C rounded up to a multiple of %d bytes" % args.row_align,
        "user_bytes": tot["user"], "hbm_bytes": tot["moved"],
        "batched": {"ms": round(tot["batched_ms"], 3), "user_gbs": round(gbs(tot["user"], tot["batched_ms"]), 1),
                    "hbm_gbs": round(gbs(tot["moved"], tot["batched_ms"]), 1),
                    "hbm_frac": round(gbs(tot["moved"], tot["batched_ms"]) / peak, 4), "launches": len(waves),
                    "layout": "autotuned on the first wave" if args.tuning == "autotune" else "default",
                    "tuning": tuning,
                    "autotune_s": tot.get("autotune_s"),
                    "timing": "GPU time of each launch, submitted while the GPU is busy with an untimed spin",
                    "host_ms": round(tot.get("host_ms", 0.0), 3),
                    "user_gbs_with_host": round(gbs(tot["user"], tot["batched_ms"] + tot.get("host_ms", 0.0)), 1)},
        "batched_default_layout": {"ms": round(tot["default_ms"], 3),
                                   "user_gbs": round(gbs(tot["user"], tot["default_ms"]), 1),
                                   "hbm_frac": round(gbs(tot["moved"], tot["default_ms"]) / peak, 4)},
        "per_stripe": {"ms": round(tot["per_stripe_ms"], 3),
                       "user_gbs": round(gbs(tot["user"], tot["per_stripe_ms"]), 1),
                       "hbm_gbs": round(gbs(tot["moved"], tot["per_stripe_ms"]), 1),
                       "hbm_frac": round(gbs(tot["moved"], tot["per_stripe_ms"]) / peak, 4),
                       "launches": tot["launches_per_stripe"]},
        "speedup_batched_over_per_stripe": round(tot["per_stripe_ms"] / tot["batched_ms"], 2),
        "by_prime": {str(pr): {"jobs": d["jobs"], "ms": round(d["ms"], 3),
                               "user_gbs": round(gbs(d["user"], d["ms"]), 1),
                               "hbm_frac": round(gbs(d["moved"], d["ms"]) / peak, 4),
                               "share_of_bytes": round(d["moved"] / tot["moved"], 4)}
                     for pr, d in sorted(by_p.items())},
        "peak": peak, "peak_kind": kind,
        "gpu_launches": tot["kernel_launches"] + tot["launches_per_stripe"],
        "clocks": clk,
    }


def run_batched(args):
    """The batched workload on its own line."""
    import torch

    from paper_cs_0611109_gb300 import build
    build.build()
    from paper_cs_0611109_gb300 import rcg

    torch.cuda.set_device(0)
    ctx = rcg.Context(0)
    m = measure_batched(args, ctx, rcg, torch)
    ctx.close()
    return {"metric": "batched uneven stripes: user GB/s, one persistent launch per wave (autotuned layout) "
                      "vs the default layout vs one launch per stripe",
            "value": m["batched"]["user_gbs"], "unit": "GB/s", "n_gpus": 1, "higher_is_better": True,
            "dtype": "u8", "data": "synthetic (SplitMix64 bytes, seed 3)",
            "config": {"workload": m["workload"], "row_stride": m["row_stride"], "schedule": args.schedule},
            **{k: v for k, v in m.items() if k not in ("workload", "row_stride")}}


# ---------------------------------------------------------------- serving

SERVE_LOADS = (0.1, 0.25, 0.5, 0.75, 1.0, 1.5, 2.0)


def measure_serve(args, ctx, rcg, torch):
    """Serving: a pool of device-resident stripes with the batched workload's
    geometry (encoded before the run), and a Poisson stream of requests on
    uniformly drawn stripes -- 70 % encode, 20 % degraded read of one strip,
    10 % double-erasure rebuild.  The arrival rate is swept from 10 % to 200 %
    of the measured saturation rate; at each rate the same stream is served by
    the continuous-batching server and by one launch per request.  Latency is
    arrival to completion (as the host sees it).  Clocks are sampled over the
    whole sweep."""
    import numpy as np

    from paper_cs_0611109_gb300 import inputs

    geo = inputs.batched_jobs(4, 10 ** 6)
    align = lambda x: (x + 255) // 256 * 256
    pool_bytes = int(args.pool_gb * 1e9)
    stripes, used = [], 0
    for g in geo:
        sz = align(inputs.stripe_bytes(g["p"], g["n"], g["c"]))
        if used + sz > pool_bytes:
            break
        stripes.append((g, used))
        used += sz
    pool = torch.empty(used, dtype=torch.uint8, device="cuda")
    rcg.rcg_fill_random(pool, used, 4)
    lays = [rcg.make_layout(pool.data_ptr() + o, g["p"], g["n"], g["c"]) for g, o in stripes]
    b = ctx.batch_prepare([rcg.make_job(L, 0, 1, rcg.RCG_OP_ENCODE) for L in lays])
    assert ctx.batch_wait(ctx.batch_launch(b))
    rcg.rcg_batch_free(b)

    rng = np.random.Generator(np.random.PCG64(5))
    n = args.serve_requests
    pick = rng.integers(0, len(stripes), size=n)
    kinds = rng.choice(3, size=n, p=[0.7, 0.2, 0.1])  # encode, degraded read, rebuild
    out_sizes = [(stripes[s][0]["p"] - 1) * stripes[s][0]["c"] if k == 1 else 0 for s, k in zip(pick, kinds)]
    out_offs = np.cumsum([0] + [align(x) for x in out_sizes])
    outs = torch.empty(max(256, int(out_offs[-1])), dtype=torch.uint8, device="cuda")
    jobs, user = [], 0
    for r in range(n):
        g, _ = stripes[pick[r]]
        L = lays[pick[r]]
        if kinds[r] == 0:
            jobs.append(rcg.make_job(L, 0, 1, rcg.RCG_OP_ENCODE))
        elif kinds[r] == 1:
            jobs.append(rcg.make_job(L, 0, 1, rcg.RCG_OP_DEGRADED_READ, 0, int(rng.integers(0, g["n"] + 2)),
                                     outs.data_ptr() + int(out_offs[r])))
        else:
            a, c = sorted(rng.choice(g["n"] + 2, size=2, replace=False).tolist())
            jobs.append(rcg.make_job(L, 0, 1, rcg.RCG_OP_RECOVER, a, c))
        user += g["n"] * (g["p"] - 1) * g["c"]
    gaps = rng.exponential(1.0, size=n)

    def serve(rate, per_job):
        arrivals = (np.cumsum(gaps) * (1e9 / rate)).astype(np.int64) if rate else np.zeros(n, np.int64)
        srv = rcg.rcg_serve_create(ctx.handle, per_job_launches=per_job)
        rcg.rcg_serve_submit(srv, jobs, arrivals)
        rcg.rcg_serve_start(srv)
        rcg.rcg_serve_drain(srv, 600 * 10 ** 9)
        res = rcg.rcg_serve_results(srv, n)
        st = rcg.rcg_serve_get_stats(srv)
        rcg.rcg_serve_destroy(srv)
        lat = np.array([r["complete_ns"] - r["arrival_ns"] for r in res], dtype=np.float64) / 1e6
        span = (max(r["complete_ns"] for r in res) - min(r["arrival_ns"] for r in res)) / 1e9
        return {"p50_ms": round(float(np.percentile(lat, 50)), 3), "p99_ms": round(float(np.percentile(lat, 99)), 3),
                "user_gbs": round(user / span / 1e9, 1), "kernel_launches": st["kernel_launches"],
                "max_inflight_launches": st["max_inflight_launches"],
                "max_inflight_requests": st["max_inflight_jobs"]}

    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    serve(0, False)  # warm-up: graph capture, caches
    sat = serve(0, False)  # everything at t = 0: the saturation throughput
    sat_per_job = serve(0, True)
    sat_rate = sat["user_gbs"] * 1e9 / (user / n)
    points = []
    launches = 0
    for f in SERVE_LOADS:
        rate = f * sat_rate
        bt, pj = serve(rate, False), serve(rate, True)
        launches += bt["kernel_launches"] + pj["kernel_launches"]
        points.append({"load": f, "rate_req_per_s": round(rate), "batched": bt, "per_job": pj})
    clk = clocks.stop()
    status = ctx.last_device_status()
    if status:
        raise RuntimeError("device status word %#x" % status)
    del pool, outs
    torch.cuda.empty_cache()
    return {"workload": "serving: Poisson stream of %d requests on %d resident stripes (%.1f GB), batched-workload "
                        "geometry, 70%% encode / 20%% degraded read / 10%% rebuild; rate swept 0.1x..2x of the "
                        "saturation rate; continuous batching (up to 8 batches in flight, round-robin over "
                        "the server's 8 streams) vs one launch per request (round-robin over the same 8 streams)"
                        % (n, len(stripes), used / 1e9),
            "requests": n, "resident_stripes": len(stripes), "pool_bytes": used,
            "mean_user_bytes_per_request": user // n,
            "saturation": {"batched": sat, "per_job": sat_per_job}, "sweep": points,
            "gpu_launches": launches, "clocks": clk}


def run_serve(args):
    """The served workload on its own line."""
    import torch

    from paper_cs_0611109_gb300 import build
    build.build()
    from paper_cs_0611109_gb300 import rcg

    torch.cuda.set_device(0)
    ctx = rcg.Context(0)
    m = measure_serve(args, ctx, rcg, torch)
    ctx.close()
    return {"metric": "serving: p50/p99 latency and user GB/s vs arrival rate, continuous batching vs per-job launches",
            "value": m["saturation"]["batched"]["user_gbs"], "unit": "GB/s (saturation, batched)", "n_gpus": 1,
            "higher_is_better": True, "dtype": "u8", "data": "synthetic (SplitMix64 bytes, seed 4)",
            "config": {"workload": m["workload"]}, **{k: v for k, v in m.items() if k != "workload"}}


def main():
    args = parse()
    if args.workload == "batched" and args.impl == "ours":
        print(json.dumps(run_batched(args)), flush=True)
        return
    if args.workload == "serve" and args.impl == "ours":
        print(json.dumps(run_serve(args)), flush=True)
        return
    if args.workload == "p13n12_ops" and args.impl == "ours":
        print(json.dumps(run_ops(args)), flush=True)
        return
    if args.workload in HGEOMETRIES and args.impl == "ours":
        print(json.dumps(run_h(args)), flush=True)
        return
    if args.workload in GEOMETRIES and args.impl == "ours":
        print(json.dumps(run_geometry(args)), flush=True)
        return
    out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
