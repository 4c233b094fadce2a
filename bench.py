"""Benchmark: checkpoint + restore throughput of the CRAC device data pass.

Workload (config 2): 256 cudaMalloc-style allocations, log-uniform
4 KiB-64 MiB rescaled to 4 GiB, fp32 N(0,1) contents, 64 KiB chunks, 10% of
chunks rewritten between checkpoints (a fixed seeded hot set, XOR-toggled,
so every checkpoint sees exactly 10% dirty chunks).

One step = mutate the hot set + incremental checkpoint of every allocation
+ full restart from the resulting image chain.  Metric value = (tracked
bytes checkpointed + tracked bytes restored) / step time, in GB/s (1e9 B/s).

  value  inputs resident in HBM: images kept in device memory, no host copies
  e2e    the same step through the C ABI with host images: the checkpoint
         drains to pinned host memory, the restart copies host -> device

Also reported: the roofline of the dominant kernel (the fused checkpoint
pass), the batched-vs-per-allocation launch comparison, and the CPU oracle
timed on a bounded sample of the same workload on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl crac|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)


import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "ckpt+restore GB/s vs HBM peak; batched vs per-alloc speedup; p99 ckpt ms"
UNIT = "GB/s"
WORKLOAD = "c2: 256 allocs log-uniform 4KiB-64MiB = 4 GiB, fp32 N(0,1), 64 KiB chunks, 10% dirty"


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def restore_flags(args) -> int:
    """crac_config_t.flags for host images: restores in place (default) or
    staged; drains through staging (default) or direct."""
    import paper_2008_10596_gb300 as C
    f = C.CRAC_FLAG_STAGED_RESTORE if getattr(args, "staged_restore", False) else 0
    f |= C.CRAC_FLAG_WAIT_PASS if getattr(args, "wait_pass", False) else 0
    return f | (C.CRAC_FLAG_DIRECT_DRAIN if getattr(args, "direct_drain", False) else 0)


KERNEL_UNITS = ("crac_pass_split.cu", "crac_pass_fused.cu", "crac_pass_tma.cu", "crac_pass_per_alloc.cu",
                "crac_restore.cu", "crac_codec.cu", "crac_noalloc.cu", "crac_drain.cu")


def kernel_src_sha(unit: str | None = None, read=None) -> str:
    """sha256 prefix over device sources: with `unit` (a .cu file of the
    library), that file and the device headers it includes; without, every
    .cu and .cuh of the library in name order, the test mutators excepted.
    It is what an ncu summary was captured against.  `read(name)` returns a
    source file's bytes (default: the working tree)."""
    import glob
    import hashlib
    csrc = os.path.join(ROOT, "paper_2008_10596_gb300", "csrc")
    if read is None:
        def read(name):
            return open(os.path.join(csrc, name), "rb").read()
    if unit is None:
        names = sorted(os.path.basename(f) for f in glob.glob(os.path.join(csrc, "*.cu")) +
                       glob.glob(os.path.join(csrc, "*.cuh")))
        names = [f for f in names if f != "crac_testkit.cu"]
    else:
        names, todo = set(), [unit]
        while todo:
            f = todo.pop()
            if f in names:
                continue
            names.add(f)
            todo += [x.decode() for x in re.findall(rb'#include "([^"]+\.cuh)"', read(f))]
        names = sorted(names)
    h = hashlib.sha256()
    for f in names:
        h.update(f.encode())
        h.update(read(f))
    return h.hexdigest()[:16]


SHA_LINE = re.compile(r"Kernel source sha256 prefix at capture: `([0-9a-f]+)`(?: \(([\w.]+\.cu) and the device headers it includes\))?")


def summary_sha_ok(text: str):
    """(captured sha, current sha) of an ncu summary: per translation unit
    where the summary names one, else over every device source."""
    m = SHA_LINE.search(text)
    if not m:
        return None
    return m.group(1), kernel_src_sha(m.group(2))


def profile_traffic(kernel_tag: str):
    """Per-launch DRAM bytes from the committed ncu summary, if it matches the kernel source."""
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    shas = summary_sha_ok(text)
    if shas is None or shas[0] != shas[1]:
        return None
    fields = {}
    for line in text.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    try:
        return int(fields["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    FIELDS = ("pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus = (bus_id or "").lower()
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            if self.bus and not parts[0].lower().endswith(self.bus[-12:]):
                continue
            rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "sm_mhz_min": min(sm) if sm else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


def aggregate_over_ranks(t_ms: float, units: float, world: int, device=None):
    """Whole-job throughput of independent replicas: the slowest rank's time
    and the units of all ranks.  Works with NCCL (device tensors) and gloo."""
    if world <= 1:
        return t_ms, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([t_ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------

def _sample_prefix(sizes, budget):
    out, acc = [], 0
    for s in sizes:
        if acc + s > budget and out:
            break
        out.append(s)
        acc += s
    return out


def oracle_step_timer(host_bufs, S, seed, workers=1):
    """Returns step() for the oracle: step() = mutate 10% + incremental
    checkpoint + full restart of the chain, on host byte arrays; the
    fingerprint loop runs on `workers` threads.  Building the FULL base image
    is set-up, outside the steps."""
    from oracle import oracle as O
    sizes = [b.size for b in host_bufs]
    ctx = O.OracleContext(S, lineage=1, workers=workers)
    for i, n in enumerate(sizes):
        ctx.register((i + 1) << 36, n)
    first = W.chunk_layout(sizes, S)
    muts = W.choose_mutations(seed, int(first[-1]), 0.10)
    chain = [ctx.checkpoint(host_bufs)]

    def step():
        W.apply_mutations_host(host_bufs, first, S, muts)
        chain.append(ctx.checkpoint(host_bufs))
        ctx.restart(chain)
        return 2 * sum(sizes)

    return step


def cpu_baseline_measure(host_bufs, S, seed, label, target_s=10.0, max_steps=20, workers=1):
    step = oracle_step_timer(host_bufs, S, seed, workers)
    t0 = time.perf_counter()
    nbytes, steps = 0, 0
    while steps < max_steps and (steps == 0 or time.perf_counter() - t0 < target_s):
        nbytes += step()
        steps += 1
    dt = time.perf_counter() - t0
    return {"value": nbytes / dt / 1e9, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": f"{label}; {steps} steps", "seconds": round(dt, 3)}


def cpu_baseline_both(host_bufs, S, seed, label, same_config):
    """The oracle on one thread and with its per-chunk fingerprint loop split
    over every host core, on the same bytes.  The line's value is the
    all-cores one."""
    cores = os.cpu_count() or 1
    one = cpu_baseline_measure(host_bufs, S, seed, label + "; single thread", target_s=8.0, max_steps=3)
    allc = cpu_baseline_measure(host_bufs, S, seed, label + f"; fingerprint loop on {cores} threads",
                                target_s=8.0, max_steps=5, workers=cores)
    return {"value": allc["value"], "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": allc["sample"], "seconds": allc["seconds"], "same_config": same_config,
            "single_thread": {"value": one["value"], "cores": 1, "seconds": one["seconds"], "sample": one["sample"]},
            "all_cores": {"value": allc["value"], "cores": cores, "seconds": allc["seconds"]},
            "nproc": cores}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import build as ob
    ob.build()
    wl = W.config2()
    budget = int(os.environ.get("CRAC_REF_SAMPLE_BYTES", str(wl.total_bytes)))
    sizes = _sample_prefix(wl.sizes, budget)
    host = [W.host_contents("f32_normal", n, wl.seed + i) for i, n in enumerate(sizes)]
    cores = os.cpu_count() or 1
    step = oracle_step_timer(host, wl.chunk_bytes, wl.seed, workers=cores)
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    nbytes = 0
    for _ in range(args.steps):
        nbytes += step()
    dt = time.perf_counter() - t0
    v = nbytes / dt / 1e9
    whole = len(sizes) == len(wl.sizes)
    label = ((f"all 256 c2 allocations ({sum(sizes) / 2**20:.0f} MiB)" if whole else
              f"first {len(sizes)} of 256 c2 allocations ({sum(sizes) / 2**20:.0f} MiB)") +
             f", numpy N(0,1); per step: 10% mutate + incremental ckpt + full chain restart; "
             f"fingerprint loop on {cores} threads")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_bytes": sum(sizes), "same_config": whole},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": label},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# The CUDA path
# ---------------------------------------------------------------------------

def run_crac(args):
    import torch
    import torch.cuda.nvtx as nvtx
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import paper_2008_10596_gb300 as C
    from paper_2008_10596_gb300 import testkit

    def barrier():
        if world > 1:
            dist.barrier()

    wl = W.config2(total=args.total_mib << 20)
    S = wl.chunk_bytes
    sizes = wl.sizes
    B = wl.total_bytes
    workload = WORKLOAD if args.total_mib == 4096 else WORKLOAD.replace("= 4 GiB", f"= {args.total_mib} MiB")
    first = W.chunk_layout(sizes, S)
    n = int(first[-1])
    g = torch.Generator(device=dev)
    g.manual_seed(wl.seed + rank)
    bufs = []
    for s in sizes:
        t = torch.randn((s + 3) // 4, generator=g, device=dev, dtype=torch.float32)
        bufs.append(t.view(torch.uint8)[:s])
    muts = W.choose_mutations(wl.seed, n, wl.dirty_fraction)
    ent = np.zeros((len(muts), 3), dtype=np.uint64)
    for i, m in enumerate(muts):
        a = int(np.searchsorted(first, m.chunk, side="right") - 1)
        lo = (m.chunk - int(first[a])) * S
        ent[i] = (bufs[a].data_ptr() + lo, min(S, sizes[a] - lo), m.mask)
    ent_dev = torch.from_numpy(ent.view(np.int64)).to(dev)
    stream = torch.cuda.current_stream(dev)

    def mutate():
        testkit.mutate_xor(ent_dev.data_ptr(), len(muts), stream)

    def make_ctx(**kw):
        ctx = C.crac_ctx_create(C.crac_config_default(chunk_bytes=S, lineage=1000 + rank, device=local, **kw))
        for b in bufs:
            C.crac_ctx_register_alloc(ctx, b.data_ptr(), b.numel(), C.CRAC_KIND_DEVICE)
        return ctx

    # The device arena is process-wide: the reservation covers every device-
    # resident context of this run (their base images and the timed loop's
    # growing chain), so that no step allocates from CUDA.
    ctx_dev = make_ctx(image_residency=C.CRAC_RESIDENCY_DEVICE, reserve_device_bytes=16 * B)
    # The pinned arena is process-wide too: the reservation covers both host-
    # image contexts' chains (the e2e leg's and the rollback leg's).
    ctx_host = make_ctx(image_residency=C.CRAC_RESIDENCY_HOST, reserve_host_bytes=6 * B, flags=restore_flags(args))
    ctx_pa = make_ctx(image_residency=C.CRAC_RESIDENCY_DEVICE, launch_mode=C.CRAC_LAUNCH_PER_ALLOC)
    ctx_b = make_ctx(image_residency=C.CRAC_RESIDENCY_DEVICE)
    ctx_ldg = make_ctx(image_residency=C.CRAC_RESIDENCY_DEVICE, pass_kernel=C.CRAC_PASS_LDG)
    ctx_tma = make_ctx(image_residency=C.CRAC_RESIDENCY_DEVICE, pass_kernel=C.CRAC_PASS_TMA)
    ctx_sparse = make_ctx(image_residency=C.CRAC_RESIDENCY_DEVICE, pass_kernel=C.CRAC_PASS_SPARSE)
    ctx_inc = make_ctx(image_residency=C.CRAC_RESIDENCY_DEVICE, flags=C.CRAC_FLAG_INCREMENTAL_RESTORE)
    ctx_inc_host = make_ctx(image_residency=C.CRAC_RESIDENCY_HOST, flags=C.CRAC_FLAG_INCREMENTAL_RESTORE)

    def step(ctx, host=False, pass_ms=None, lat_ms=None, rst=None, phases=None):
        mutate()
        t0 = time.perf_counter()
        img = C.crac_ctx_checkpoint(ctx, stream)
        t1 = time.perf_counter()
        if host:
            C.crac_image_wait(img)
        t2 = time.perf_counter()
        if lat_ms is not None:
            lat_ms.append((t2 - t0) * 1e3)
        if pass_ms is not None:
            # filled in place (no per-field Python work inside the timed loop)
            pass_ms.append(C.crac_ctx_last_pass(ctx, C.CracPassInfo()))
        C.crac_ctx_restart(ctx, img, stream)
        if phases is not None:
            phases.append(((t1 - t0) * 1e3, (t2 - t1) * 1e3, (time.perf_counter() - t2) * 1e3))
        if rst is not None:
            rst.append(C.crac_ctx_last_restart(ctx, C.CracRestartInfo()))
        C.crac_image_release(img)

    def pass_rows(infos):
        return [(i.device_ms, i.k, i.payload_bytes, i.hash_ms, i.finalize_ms, i.gather_ms, i.in_place)
                for i in infos]

    # Base images (full) for each context.
    for ctx in (ctx_dev, ctx_host, ctx_pa, ctx_b, ctx_ldg, ctx_tma, ctx_sparse, ctx_inc, ctx_inc_host):
        img = C.crac_ctx_checkpoint(ctx, stream)
        C.crac_image_wait(img)
        C.crac_image_release(img)
    torch.cuda.synchronize()

    # ---- value: device-resident images --------------------------------------
    # Clocks are sampled every 50 ms from the first warm-up step to the end of
    # the last GPU leg (the device-resident timed loop alone is shorter than
    # one sampling period).
    sampler = ClockSampler(None)
    sampler.start()
    for _ in range(args.warmup):
        step(ctx_dev)
    torch.cuda.synchronize()
    barrier()
    launches0 = C.crac_kernel_launches()
    mem0 = C.crac_memory_stats()
    pass_ms, lat_ms, rst = [], [], []
    torch.cuda.synchronize()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    nvtx.range_push("timed")      # ncu captures select kernels by these ranges
    for _ in range(args.steps):
        step(ctx_dev, pass_ms=pass_ms, lat_ms=lat_ms, rst=rst)
    nvtx.range_pop()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    t_ms = ev0.elapsed_time(ev1)
    bytes_per_step = 2 * B
    t_ms, job_bytes = aggregate_over_ranks(t_ms, bytes_per_step * args.steps, world, dev)
    launches = C.crac_kernel_launches() - launches0 + args.steps   # + one mutator launch per step
    mem1 = C.crac_memory_stats()
    arena_growth = {"device_grow_events": mem1["device_grow_events"] - mem0["device_grow_events"],
                    "host_grow_events": mem1["host_grow_events"] - mem0["host_grow_events"]}
    value = job_bytes / (t_ms / 1e3) / 1e9

    # ---- roofline: the dominant kernel is the split pass's streaming hash ------
    pass_ms = pass_rows(pass_ms)
    rst = [C.restart_info_dict(r) for r in rst]
    dev_ms = statistics.mean(p[0] for p in pass_ms)
    k_avg = statistics.mean(p[1] for p in pass_ms)
    d_avg = statistics.mean(p[2] for p in pass_ms)
    hash_ms = statistics.mean(p[3] for p in pass_ms)
    fin_ms = statistics.mean(p[4] for p in pass_ms)
    gat_ms = statistics.mean(p[5] for p in pass_ms)
    in_place = statistics.mean(p[6] for p in pass_ms)
    spec_bytes = d_avg * in_place / k_avg if k_avg else 0.0   # chunks the hash kernel wrote as it read them
    peak, peak_src = load_peaks()
    psrc = f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)" if peak_src == "measured" else "fallback"
    # The step's dominant kernel is the restore scatter (every tracked byte read
    # from the image payloads and written back, plus 8 B idx + 8 B off + 2 B
    # owner per visited entry); its launches are timed by the library with
    # CUDA events on the launching stream.
    sc_ms = statistics.mean(r["device_ms"] for r in rst)
    sc_entries = statistics.mean(r["entries_scanned"] for r in rst)
    sc_bytes = statistics.mean(r["restored_bytes"] for r in rst)
    alg_sc = 2 * sc_bytes + 18 * sc_entries
    roofline = {"bound": "hbm", "achieved": alg_sc / (sc_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                "frac": alg_sc / (sc_ms / 1e3) / 1e9 / peak, "traffic": profile_traffic("scatter_c2_64KiB"),
                "kernel": "scatter_kernel (restore, all launches of a restart)",
                "alg_bytes_per_launch": int(alg_sc), "avg_launch_ms": sc_ms,
                "launches_per_restart": statistics.mean(r["scatter_launches"] for r in rst), "peak_source": psrc}
    # every tracked byte read once + one accumulator per chunk + the predicted
    # dirty chunks written to staging as they are read
    alg_hash = B + 8 * n + spec_bytes
    roofline_hash = {"bound": "hbm", "achieved": alg_hash / (hash_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": alg_hash / (hash_ms / 1e3) / 1e9 / peak,
                     "traffic": profile_traffic("split_hash_c2_64KiB"), "kernel": "split_hash_kernel",
                     "alg_bytes_per_launch": int(alg_hash), "avg_launch_ms": hash_ms, "peak_source": psrc}
    alg_pass = B + d_avg + 16 * n + 16 * k_avg    # read B, write D, fp old + new, idx + off
    pass_info = {"kernels": "split: hash (+ predicted write-through) -> finalize+compact -> gather (one graph)",
                 "device_ms": dev_ms, "hash_ms": hash_ms, "finalize_ms": fin_ms, "gather_ms": gat_ms,
                 "in_place_chunks": in_place, "dirty_chunks": k_avg,
                 "alg_bytes": int(alg_pass), "achieved_gbs": alg_pass / (dev_ms / 1e3) / 1e9,
                 "frac": alg_pass / (dev_ms / 1e3) / 1e9 / peak, "tracked_gbs": B / (dev_ms / 1e3) / 1e9}

    # ---- batched vs per-allocation launches, and the pass variants -------------
    cmp = {"per_alloc": ([], []), "split": ([], []), "ldg": ([], []), "tma": ([], []), "sparse": ([], [])}
    ctxs = {"per_alloc": ctx_pa, "split": ctx_b, "ldg": ctx_ldg, "tma": ctx_tma, "sparse": ctx_sparse}
    nvtx.range_push("variants")
    for _ in range(max(3, min(args.steps, 5))):
        mutate()
        for name, ctx in ctxs.items():
            t0 = time.perf_counter()
            img = C.crac_ctx_checkpoint(ctx, stream)
            cmp[name][1].append((time.perf_counter() - t0) * 1e3)
            cmp[name][0].append(C.crac_ctx_last_pass(ctx)["device_ms"])
            C.crac_image_release(img)
    nvtx.range_pop()
    med = {k: (statistics.median(v[0]), statistics.median(v[1])) for k, v in cmp.items()}
    batched = {"per_alloc_device_ms": med["per_alloc"][0], "batched_device_ms": med["split"][0],
               "speedup_device": med["per_alloc"][0] / med["split"][0],
               "per_alloc_wall_ms": med["per_alloc"][1], "batched_wall_ms": med["split"][1],
               "speedup_wall": med["per_alloc"][1] / med["split"][1],
               "per_alloc_launches": 3 * len(sizes), "batched_graph_launches": 1,
               "variants_device_ms": {k: v[0] for k, v in med.items()}}

    # ---- rollback: incremental restore of the last image after a 10% change ----
    def rollback_leg(ctx, host):
        rb, wall = [], []
        for _ in range(max(3, min(args.steps, 5))):
            mutate()
            img = C.crac_ctx_checkpoint(ctx, stream)
            if host:
                C.crac_image_wait(img)
            mutate()                                  # the state diverges from the image again
            t0 = time.perf_counter()
            C.crac_ctx_restart(ctx, img, stream)
            wall.append((time.perf_counter() - t0) * 1e3)
            rb.append(C.crac_ctx_last_restart(ctx))
            C.crac_image_release(img)
        return {"device_ms": statistics.median(r["device_ms"] for r in rb),
                "call_ms": statistics.median(wall),
                "chunks_rewritten": statistics.median(r["chunks_rewritten"] for r in rb),
                "chunks": n, "bytes_rewritten": statistics.median(r["restored_bytes"] for r in rb)}

    nvtx.range_push("rollback")
    rollback = rollback_leg(ctx_inc, False)
    rollback_host = rollback_leg(ctx_inc_host, True)
    nvtx.range_pop()
    rollback["full_restore_device_ms"] = statistics.median(r["device_ms"] for r in rst)
    rollback["speedup_vs_full"] = rollback["full_restore_device_ms"] / rollback["device_ms"]
    rollback["host_images"] = rollback_host
    rollback["how"] = ("CRAC_FLAG_INCREMENTAL_RESTORE: fingerprint the current memory against the image, "
                       "rewrite the chunks that differ; device-resident images, and host-resident ones "
                       "(host_images: only the differing chunks cross the host link; compare with the e2e "
                       "restart_call of a full restore)")

    # ---- host link probe: pinned 1 GiB copies, best of 10 each way ------------
    link = None
    if not args.no_e2e:
        hbuf = torch.empty(1 << 30, dtype=torch.uint8, pin_memory=True)
        dbuf = torch.empty(1 << 30, dtype=torch.uint8, device=dev)
        best = {"h2d": 1e9, "d2h": 1e9}
        for _ in range(10):
            for d, (dst, src) in (("h2d", (dbuf, hbuf)), ("d2h", (hbuf, dbuf))):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                dst.copy_(src, non_blocking=True)
                b.record(stream)
                b.synchronize()
                best[d] = min(best[d], a.elapsed_time(b))
        link = {"h2d_gbs": (1 << 30) / (best["h2d"] / 1e3) / 1e9, "d2h_gbs": (1 << 30) / (best["d2h"] / 1e3) / 1e9,
                "probe": "pinned 1 GiB cudaMemcpyAsync, best of 10"}
        del hbuf, dbuf

    # ---- e2e: host images through the C ABI ----------------------------------
    e2e_steps = 0 if args.no_e2e else max(1, min(args.steps, 10))
    e2e = None
    if e2e_steps:
        step(ctx_host, host=True)
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e_pass, e_phase, e_rst = [], [], []
        emem0 = C.crac_memory_stats()
        e0.record(stream)
        nvtx.range_push("e2e")
        for _ in range(e2e_steps):
            step(ctx_host, host=True, pass_ms=e_pass, phases=e_phase, rst=e_rst)
        nvtx.range_pop()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        te = e0.elapsed_time(e1)
        emem1 = C.crac_memory_stats()
        e_pass = pass_rows(e_pass)
        k_e = statistics.mean(p[1] for p in e_pass)
        d_e = statistics.mean(p[2] for p in e_pass)
        d2h = int(d_e + 8 * k_e + 8 * n + 64)
        # The restart reads every restored chunk once from the chain's pinned
        # images (in place), plus each visited entry's index and offset, and
        # uploads the fingerprint table and the descriptors.
        ent = statistics.mean(r.entries_scanned for r in e_rst)
        h2d = int(B + 16 * ent + 8 * n + 40 * len(sizes) * statistics.mean(r.chain_length for r in e_rst))
        e2e = {"value": bytes_per_step * e2e_steps * world / (te / 1e3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": e2e_steps,
               "ms_per_step": te / e2e_steps, "link": link,
               "arena_growth": {"host_grow_events": emem1["host_grow_events"] - emem0["host_grow_events"],
                                "device_grow_events": emem1["device_grow_events"] - emem0["device_grow_events"]},
               "phases_ms": {"checkpoint_call": statistics.median(p[0] for p in e_phase),
                             "drain_wait": statistics.median(p[1] for p in e_phase),
                             "restart_call": statistics.median(p[2] for p in e_phase)}}

    clocks = sampler.stop()
    clocks["window"] = "warm-up through the end of the e2e leg"

    # ---- CPU oracle on a bounded sample (rank 0, N=1 only) -------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        from oracle import build as ob
        ob.build()
        budget = int(os.environ.get("CRAC_CPU_SAMPLE_BYTES", str(B)))
        ssz = _sample_prefix(sizes, budget)
        host = [bufs[i].cpu().numpy().copy() for i in range(len(ssz))]
        whole = len(ssz) == len(sizes)
        cpu = cpu_baseline_both(host, S, wl.seed,
                                (f"all {len(ssz)} allocations" if whole else
                                 f"first {len(ssz)} of {len(sizes)} allocations") +
                                f" ({sum(ssz) / 2**20:.0f} MiB) of this workload read back to host; "
                                "10% mutate + incremental ckpt + full restart", whole)
        del host

    for ctx in (ctx_dev, ctx_host, ctx_pa, ctx_b, ctx_ldg, ctx_tma, ctx_sparse, ctx_inc, ctx_inc_host):
        C.crac_ctx_destroy(ctx)

    # ---- serving: config 5's request loop, short (N=1 only) -------------------
    serving = None
    if world == 1 and not args.no_serving:
        total5 = args.serving_gib * W.GIB
        sr = ServingRun(dev, total=total5)
        sr.base_images()
        sampler5 = ClockSampler(None)   # the loop is mostly idle: the clocks it runs at
        sampler5.start()
        serving = sr.run(args.serving_requests, args.rate)
        serving["clocks"] = sampler5.stop()
        serving["cuda_device_max_connections"] = os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS")
        sr.close()
        serving["workload"] = (f"c5 shape: 64 contexts, {args.serving_gib} GiB total (log-uniform 0.5-8 GiB scaled "
                               f"by {total5 / (173 * W.GIB):.3f}), {args.serving_requests} requests Poisson "
                               f"{args.rate}/s, 75% ckpt / 25% restart, 24 GiB staging budget, 8 slots, host images")

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
                "config": {"workload": workload, "allocs": len(sizes), "tracked_bytes": B, "chunk_bytes": S,
                           "dirty_fraction": wl.dirty_fraction, "n_chunks": n,
                           "l2": "inputs (4 GiB) larger than L2 (126 MB); no flush",
                           "step": "mutate 10% + incremental ckpt + full restart (device-resident images)",
                           "parallelism": f"replicas{world}"},
                "roofline": roofline, "roofline_ckpt_hash": roofline_hash, "pass": pass_info, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": launches, "arena_growth_in_timed_loop": arena_growth, "rollback": rollback,
                "batched_vs_per_alloc": batched,
                "ckpt_latency_ms": {"p50": statistics.median(lat_ms),
                                    "p99": float(np.percentile(lat_ms, 99))},
                "serving_latency_ms": None if serving is None else {
                    "checkpoint": serving["latency_ms"]["checkpoint"], "restart": serving["latency_ms"]["restart"],
                    "all": serving["latency_all_ms"]},
                "serving": serving,
                "ckpt_pass_gbs": B / (dev_ms / 1e3) / 1e9, "dirty_chunks": k_avg, "dirty_bytes": d_avg}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# Config 3: device + managed memory, 4-stream mutator, 3 checkpoints + restart
# ---------------------------------------------------------------------------

def run_config3(args):
    import torch
    import paper_2008_10596_gb300 as C
    from paper_2008_10596_gb300 import testkit
    from workloads.device import C3Memory, rows_tensor
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    scale = args.total_mib / 4096.0 if args.total_mib != 4096 else 1.0
    mem = C3Memory(dev, device_total=int(12 * W.GIB * scale), managed_total=int(4 * W.GIB * scale))
    wl, S, ptrs, sizes, kinds = mem.wl, mem.S, mem.ptrs, mem.sizes, mem.kinds
    main = torch.cuda.current_stream(dev)
    mutate = mem.mutate

    ctx = C.crac_ctx_create(C.crac_config_default(chunk_bytes=S, lineage=3, device=0,
                                                  reserve_host_bytes=int(2.2 * sum(sizes)), flags=restore_flags(args)))
    for ptr, n, k in zip(ptrs, sizes, kinds):
        C.crac_ctx_register_alloc(ctx, ptr, n, k)
    B = sum(sizes)
    ckpts = []
    imgs = []
    for i in range(3):
        if i:
            mutate(wl.seed + i)
        t0 = time.perf_counter()
        img = C.crac_ctx_checkpoint(ctx, main)
        t1 = time.perf_counter()
        C.crac_image_wait(img)
        t2 = time.perf_counter()
        info = C.crac_ctx_last_pass(ctx)
        ii = C.crac_image_info(img)
        imgs.append(img)
        ckpts.append({"epoch": ii["epoch"], "full": bool(ii["flags"] & 1), "dirty_bytes": ii["payload_bytes"],
                      "segments": info["segments"], "pass_ms": info["device_ms"], "prefetch_ms": info["prefetch_ms"],
                      "pass_tracked_gbs": B / (info["device_ms"] / 1e3) / 1e9,
                      "call_ms": (t1 - t0) * 1e3, "until_drained_ms": (t2 - t0) * 1e3,
                      "e2e_payload_gbs": ii["payload_bytes"] / max(t2 - t0, 1e-9) / 1e9})
    # restart from the third image into zeroed memory, compare with a copy
    keep = [torch.empty(n, dtype=torch.uint8, device=dev) for n in sizes]
    rows = mem.copy_rows([k.data_ptr() for k in keep])
    e = rows_tensor(rows, dev)
    testkit.rewrite(e.data_ptr(), len(rows), main)
    zero = torch.zeros(64 << 20, dtype=torch.uint8, device=dev)
    rows = [(p + o, zero.data_ptr(), min(64 << 20, n - o)) for p, n in zip(ptrs, sizes) for o in range(0, n, 64 << 20)]
    e = rows_tensor(rows, dev)
    testkit.rewrite(e.data_ptr(), len(rows), main)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    C.crac_ctx_restart(ctx, imgs[-1], main)
    torch.cuda.synchronize()
    t_restart = time.perf_counter() - t0
    back = [torch.empty(n, dtype=torch.uint8, device=dev) for n in sizes]
    rows = mem.copy_rows([b.data_ptr() for b in back])
    e = rows_tensor(rows, dev)
    testkit.rewrite(e.data_ptr(), len(rows), main)
    torch.cuda.synchronize()
    exact = all(torch.equal(a, b) for a, b in zip(keep, back))
    for img in imgs:
        C.crac_image_release(img)
    C.crac_ctx_destroy(ctx)
    mem.free()
    line = {"workload": f"c3: {len(wl.sizes)} device ({sum(wl.sizes) / 2**30:.1f} GiB) + {len(wl.managed_sizes)} "
                        f"managed ({sum(wl.managed_sizes) / 2**30:.1f} GiB) allocations, 64 KiB chunks, 25% of pages "
                        "rewritten (bf16) on 4 streams between checkpoints",
            "tracked_bytes": B, "checkpoints": ckpts, "restart_ms": t_restart * 1e3,
            "restart_gbs": B / t_restart / 1e9, "restart_chain": 3, "restored_exact": exact,
            "note": "host-resident images; restart copies the chain's surviving chunks host->device"}
    print(json.dumps(line), flush=True)
    return 0 if exact else 1


# ---------------------------------------------------------------------------
# Config 4: 120 GiB / 2048 allocations, dirty sweep, autotuned chunk size
# ---------------------------------------------------------------------------

def run_config4(args):
    import torch
    import paper_2008_10596_gb300 as C
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    total = (args.total_mib << 20) if args.total_mib != 4096 else 120 * W.GIB
    from workloads.device import c4_memory
    sizes, bufs, mutate = c4_memory(total, 2048, dev)
    B = sum(sizes)
    peak, _ = load_peaks()
    cands = [4 * W.KIB, 64 * W.KIB, 256 * W.KIB]
    stream = torch.cuda.current_stream(dev)
    points = []
    for frac in (0.0, 0.01, 0.10, 0.50, 1.00):
        ctx = C.crac_ctx_create(C.crac_config_default(chunk_bytes=64 * W.KIB, lineage=4, device=0,
                                                      staging_bytes=8 * W.GIB,
                                                      image_residency=C.CRAC_RESIDENCY_DEVICE))
        for b in bufs:
            C.crac_ctx_register_alloc(ctx, b.data_ptr(), b.numel())
        C.crac_ctx_tune_observe(ctx, cands, stream)
        for r in range(2):
            mutate(frac, int(1000 * frac) + r)
            obs = C.crac_ctx_tune_observe(ctx, cands, stream)
        res = C.crac_ctx_tune_apply(ctx, 190.0, stream)
        per = []
        for S, ms, d in zip(obs["chunk_bytes"], obs["last_pass_ms"], obs["last_dirty_bytes"]):
            nch = sum(-(-n // S) for n in sizes)
            kk = d // S
            alg = B + d + 16 * nch + 16 * kk
            per.append({"chunk_bytes": S, "pass_ms": ms, "dirty_bytes": d, "tracked_gbs": B / (ms / 1e3) / 1e9,
                        "hbm_frac": alg / (ms / 1e3) / 1e9 / peak})
        # the chosen size and kernel: its timed pass against B + D + 16n + 16k at that size
        Sc = res["chosen_chunk_bytes"]
        pc = next((q for q in per if q["chunk_bytes"] == Sc), None)
        ms_c = res["variant_ms"][res["chosen_pass_kernel"]] if res["chosen_pass_kernel"] < len(res["variant_ms"]) else 0
        chosen = None
        if pc is not None and ms_c > 0:
            nch = sum(-(-n // Sc) for n in sizes)
            alg = B + pc["dirty_bytes"] + 16 * nch + 16 * (pc["dirty_bytes"] // Sc)
            chosen = {"pass_ms": ms_c, "tracked_gbs": B / (ms_c / 1e3) / 1e9, "hbm_frac": alg / (ms_c / 1e3) / 1e9 / peak}
        points.append({"dirty_fraction_4k_pages": frac, "per_chunk_size": per, "chosen": chosen,
                       "chosen_chunk_bytes": res["chosen_chunk_bytes"],
                       "chosen_pass_kernel": res["chosen_pass_kernel"], "cost_ms": res["cost_ms"],
                       "variant_ms_at_chosen": res["variant_ms"],
                       "chosen_ldg_chunks_per_tile": res["chosen_chunks_per_tile"],
                       "ldg_tile_ms": dict(zip(res["ldg_tiles"], res["ldg_tile_ms"]))})
        C.crac_ctx_destroy(ctx)
    line = {"workload": f"c4: {len(sizes)} allocations, Zipf(1.1) sizes = {B / 2**30:.1f} GiB, uint8/fp32/int64",
            "tracked_bytes": B, "link_gbs_assumed": 190.0, "peak_gbs": peak, "points": points,
            "note": "per_chunk_size: the split graph (hash, finalize+compact, gather into 8 GiB staging segments) "
                    "at each candidate size, device time, dirty bytes measured by the pass against the previous "
                    "observation; chosen: the tuner's size and kernel, its timed pass at that size"}
    if not args.no_cpu:
        line["cpu_baseline"] = c4_oracle_subset(bufs, sizes, B)
    print(json.dumps(line), flush=True)
    return 0


def c4_oracle_subset(bufs, sizes, B, budget=4 * W.GIB):
    """The oracle's checkpoint pass on a 4 GiB subset of config 4's memory
    (its first allocations, read back to the host), 64 KiB chunks, 10% of
    the 4 KiB pages XOR-mutated before a delta checkpoint; single-threaded
    and with the fingerprint loop on every host core; scaled linearly to the
    whole tracked size, stated as such."""
    from oracle import build as ob
    from oracle import oracle as O
    ob.build()
    ssz = _sample_prefix(sizes, budget)
    host = [bufs[i].cpu().numpy().copy() for i in range(len(ssz))]
    sub = sum(ssz)
    rng = np.random.default_rng(W.SEED_BASE + 4)
    pages = [(a, o) for a, n in enumerate(ssz) for o in range(0, n - 4095, 4096)]
    pick = rng.choice(len(pages), size=len(pages) // 10, replace=False)
    out = {"kind": "oracle", "unit": "GB/s", "sample": f"first {len(ssz)} of {len(sizes)} allocations "
           f"({sub / 2**30:.2f} GiB), 64 KiB chunks, delta checkpoint after 10% of 4 KiB pages rewritten; "
           f"scaled_s = seconds x {B / sub:.2f} (tracked / sample bytes)"}
    for label, workers in (("single_thread", 1), ("all_cores", os.cpu_count() or 1)):
        ctx = O.OracleContext(64 * W.KIB, lineage=4, workers=workers)
        for i, n in enumerate(ssz):
            ctx.register((i + 1) << 40, n)
        ctx.checkpoint(host)
        for j in pick:   # XOR-mutate the chosen pages (toggled back on the second round)
            a, o = pages[j]
            v = host[a][o:o + 4096].view(np.uint32)
            v ^= np.uint32(0x9E3779B1)
        t0 = time.perf_counter()
        ctx.checkpoint(host)
        dt = time.perf_counter() - t0
        out[label] = {"cores": workers, "seconds": dt, "value": sub / dt / 1e9, "scaled_s": dt * B / sub}
    out["value"] = out["all_cores"]["value"]
    out["cores"] = out["all_cores"]["cores"]
    return out


# ---------------------------------------------------------------------------
# Pass kernels side by side: chunk size x dirty fraction x kernel
# ---------------------------------------------------------------------------

PASS_NAMES = {"split": 3, "ldg": 1, "tma": 2, "sparse": 4}


def run_passes(args):
    """Each pass kernel on the same config-4-shaped memory (default 32 GiB,
    512 allocations), at each chunk size and fraction of rewritten 4 KiB
    pages: device time of a delta pass (best of 3) against a baseline taken
    right before it, device-resident images."""
    import torch
    import paper_2008_10596_gb300 as C
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    total = (args.total_mib << 20) if args.total_mib != 4096 else 32 * W.GIB
    n_allocs = max(16, int(512 * total / (32 * W.GIB)))
    from workloads.device import c4_memory
    sizes, bufs, mutate = c4_memory(total, n_allocs, dev)
    B = sum(sizes)
    peak, _ = load_peaks()
    stream = torch.cuda.current_stream(dev)
    points = []
    for S in [int(x) * W.KIB for x in args.chunk_kib.split(",")]:
        n = sum(-(-b // S) for b in sizes)
        for frac in [float(x) for x in args.dirty.split(",")]:
            for name in args.kernels.split(","):
                ctx = C.crac_ctx_create(C.crac_config_default(
                    chunk_bytes=S, lineage=5, device=0, staging_bytes=8 * W.GIB,
                    image_residency=C.CRAC_RESIDENCY_DEVICE, pass_kernel=PASS_NAMES[name],
                    ctas_per_sm=args.ctas_per_sm if name == "ldg" else 0,
                    chunks_per_tile=args.chunks_per_tile if name == "ldg" else 0))
                for b in bufs:
                    C.crac_ctx_register_alloc(ctx, b.data_ptr(), b.numel())
                C.crac_image_release(C.crac_ctx_checkpoint(ctx, stream))
                best = None
                for r in range(3):
                    mutate(frac, 7 + r)
                    C.crac_image_release(C.crac_ctx_checkpoint(ctx, stream))
                    info = C.crac_ctx_last_pass(ctx)
                    if best is None or info["device_ms"] < best["device_ms"]:
                        best = info
                C.crac_ctx_destroy(ctx)
                ms, D, k = best["device_ms"], best["payload_bytes"], best["k"]
                alg = B + D + 16 * n + 16 * k
                points.append({"chunk_bytes": S, "dirty_fraction_4k_pages": frac, "kernel": name,
                               "grid": best["grid"], "chunks_per_tile": best["chunks_per_tile"],
                               "pass_ms": ms, "dirty_bytes": D, "k": k, "tracked_gbs": B / (ms / 1e3) / 1e9,
                               "hbm_frac": alg / (ms / 1e3) / 1e9 / peak})
    line = {"workload": f"passes: {len(sizes)} allocations, Zipf(1.1) sizes = {B / 2**30:.1f} GiB, "
                        "uint8/fp32/int64", "tracked_bytes": B, "peak_gbs": peak, "points": points,
            "note": "hbm_frac = (B + D + 16 n + 16 k) / device time / peak; the split pass moves B + 2D"}
    print(json.dumps(line), flush=True)
    return 0


N_FULL = 3   # codec: timed full checkpoints per variant


def run_codec(args):
    """Coded images (CRAC_FLAG_COMPRESS) against plain ones on the config-2
    layout (256 allocations, 4 GiB, 64 KiB chunks, the same 10% hot set),
    filled in turn with fp32 N(0,1) (config 2's contents), bf16 N(0,1)
    (config 3's rewritten pages), zeros and uniform bytes.  Per content and
    image kind: a full checkpoint, delta checkpoints after the 10% XOR
    mutation, and a restart of the resulting chain; calls are timed on the
    wall clock including the drain wait, and the library's CUDA-event times
    of the pass, encoder and restore kernels are reported beside them."""
    import torch
    import torch.cuda.nvtx as nvtx
    import paper_2008_10596_gb300 as C
    from paper_2008_10596_gb300 import testkit
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    wl = W.config2(total=args.total_mib << 20)
    S, sizes = wl.chunk_bytes, wl.sizes
    B = wl.total_bytes
    first = W.chunk_layout(sizes, S)
    n = int(first[-1])
    stream = torch.cuda.current_stream(dev)
    peak, peak_src = load_peaks()
    g = torch.Generator(device=dev)
    bufs = [torch.empty(s, dtype=torch.uint8, device=dev) for s in sizes]

    def fill(kind, seed):
        g.manual_seed(seed)
        for b in bufs:
            s = b.numel()
            if kind == "f32_normal":
                b.copy_(torch.randn((s + 3) // 4, generator=g, device=dev).view(torch.uint8)[:s])
            elif kind == "bf16_normal":
                b.copy_(torch.randn((s + 1) // 2, generator=g, device=dev).to(torch.bfloat16).view(torch.uint8)[:s])
            elif kind == "zeros":
                b.zero_()
            else:
                b.copy_(torch.randint(0, 256, (s,), generator=g, device=dev, dtype=torch.uint8))
        torch.cuda.synchronize()

    muts = W.choose_mutations(wl.seed, n, wl.dirty_fraction)
    ent = np.zeros((len(muts), 3), dtype=np.uint64)
    for i, m in enumerate(muts):
        a = int(np.searchsorted(first, m.chunk, side="right") - 1)
        lo = (m.chunk - int(first[a])) * S
        ent[i] = (bufs[a].data_ptr() + lo, min(S, sizes[a] - lo), m.mask)
    ent_dev = torch.from_numpy(ent.view(np.int64)).to(dev)

    variants = {
        "host": dict(image_residency=C.CRAC_RESIDENCY_HOST),
        "host_coded": dict(image_residency=C.CRAC_RESIDENCY_HOST, flags=C.CRAC_FLAG_COMPRESS),
        "host_coded_direct": dict(image_residency=C.CRAC_RESIDENCY_HOST,
                                  flags=C.CRAC_FLAG_COMPRESS | C.CRAC_FLAG_DIRECT_DRAIN),
        "device": dict(image_residency=C.CRAC_RESIDENCY_DEVICE),
        "device_coded": dict(image_residency=C.CRAC_RESIDENCY_DEVICE, flags=C.CRAC_FLAG_COMPRESS),
    }
    # Every variant's chain (a first image, a full one, the deltas: ~2.5 B)
    # must stay under the pinned arena's 80% mark, where its background
    # growth (pinning a new region while the timed copies run) would start.
    reserve = dict(reserve_host_bytes=5 * B, reserve_device_bytes=4 * B)
    steps = max(3, min(args.steps, 5))
    sampler = ClockSampler(None)
    sampler.start()
    launches0 = C.crac_kernel_launches()
    mem0 = None
    rows = []
    enc = []   # encoder launches into device images: (raw bytes, stored bytes, entries, ms)
    for kind in ("f32_normal", "bf16_normal", "zeros", "u8_uniform"):
        for name, cfg in variants.items():
            fill("u8_uniform", wl.seed + 7)   # the untimed first image: other bytes everywhere
            ctx = C.crac_ctx_create(C.crac_config_default(chunk_bytes=S, lineage=3000, device=0, **cfg, **reserve))
            reserve = {}
            if mem0 is None:
                mem0 = C.crac_memory_stats()   # after the reservation
            for b in bufs:
                C.crac_ctx_register_alloc(ctx, b.data_ptr(), b.numel())
            # A first full checkpoint (of other bytes) sizes the context's
            # scratch; the timed full one follows the fill with this content
            # (every chunk dirty, steady state), then the deltas of the 10%
            # hot set.
            imgs, fulls, deltas = [C.crac_ctx_checkpoint(ctx, stream)], [], []
            C.crac_image_wait(imgs[0])
            fill(kind, wl.seed)
            # three full checkpoints (the first finds every chunk rewritten, the
            # next two follow an invalidation: the same work), then the deltas
            for r in range(N_FULL + steps):
                if r >= N_FULL:
                    testkit.mutate_xor(ent_dev.data_ptr(), len(muts), stream)
                elif r:
                    C.crac_ctx_invalidate(ctx)
                torch.cuda.synchronize()
                nvtx.range_push(f"codec_{name}")
                t0 = time.perf_counter()
                img = C.crac_ctx_checkpoint(ctx, stream)
                C.crac_image_wait(img)
                wall = (time.perf_counter() - t0) * 1e3
                nvtx.range_pop()
                imgs.append(img)
                pi = C.crac_ctx_last_pass(ctx)
                rec = {"wall_ms": wall, "device_ms": pi["device_ms"], "codec_ms": pi["codec_ms"],
                       "raw_bytes": pi["payload_bytes"], "stored_bytes": pi["stored_bytes"], "k": pi["k"]}
                if r < N_FULL:
                    fulls.append(rec)
                    # a full image needs no earlier one: release them, so that
                    # the pinned arena stays under its 80% mark
                    for old in imgs[:-1]:
                        C.crac_image_release(old)
                    imgs = imgs[-1:]
                else:
                    deltas.append(rec)
                if pi["codec_ms"] > 0 and name == "device_coded":
                    enc.append((kind, r < N_FULL, pi["payload_bytes"], pi["stored_bytes"], pi["k"], pi["codec_ms"]))
            want = [bufs[i][:4096].clone() for i in (0, len(bufs) // 2, len(bufs) - 1)]
            for b in bufs[::17]:
                b.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            C.crac_ctx_restart(ctx, imgs[-1], stream)
            torch.cuda.synchronize()
            rwall = (time.perf_counter() - t0) * 1e3
            ri = C.crac_ctx_last_restart(ctx)
            ok = all(torch.equal(bufs[i][:4096], w) for i, w in zip((0, len(bufs) // 2, len(bufs) - 1), want))
            for img in imgs:
                C.crac_image_release(img)
            C.crac_ctx_destroy(ctx)
            med = lambda key: statistics.median(d[key] for d in deltas)   # noqa: E731
            fmed = lambda key: statistics.median(d[key] for d in fulls)   # noqa: E731
            rows.append({
                "content": kind, "images": name,
                "full": {"wall_ms": fmed("wall_ms"), "wall_ms_each": [d["wall_ms"] for d in fulls],
                         "device_ms": fmed("device_ms"), "codec_ms": fmed("codec_ms"),
                         "raw_bytes": fulls[0]["raw_bytes"], "stored_bytes": fulls[0]["stored_bytes"],
                         "k": fulls[0]["k"], "ratio": fulls[0]["stored_bytes"] / fulls[0]["raw_bytes"]},
                "delta": {"wall_ms": med("wall_ms"), "device_ms": med("device_ms"), "codec_ms": med("codec_ms"),
                          "raw_bytes": med("raw_bytes"), "stored_bytes": med("stored_bytes"),
                          "ratio": med("stored_bytes") / med("raw_bytes")},
                "restart": {"wall_ms": rwall, "device_ms": ri["device_ms"], "chain_length": ri["chain_length"],
                            "tracked_gbs": B / (rwall / 1e3) / 1e9, "sampled_restore_ok": ok}})
    launches = C.crac_kernel_launches() - launches0
    mem1 = C.crac_memory_stats()
    clocks = sampler.stop()
    # The oracle's CRZ1 code on the host cores, on a bounded sample of the
    # fp32 content (the first allocations, up to 64 MiB, 64 KiB chunks).
    cpu = None
    if not args.no_cpu:
        from oracle import crz
        fill("f32_normal", wl.seed)
        sample, got = [], 0
        for b in bufs:
            if got >= 64 << 20:
                break
            sample.append(b.cpu().numpy())
            got += b.numel()
        chunks = [a[i:i + S] for a in sample for i in range(0, a.size, S)]
        t0 = time.perf_counter()
        streams = [crz.encode(ch) for ch in chunks]
        t_enc = time.perf_counter() - t0
        nd = max(1, len(chunks) // 4)
        t0 = time.perf_counter()
        for ch, z in zip(chunks[:nd], streams[:nd]):
            crz.decode(z, ch.size)
        t_dec = time.perf_counter() - t0
        raw = sum(ch.size for ch in chunks)
        raw_d = sum(ch.size for ch in chunks[:nd])
        cpu = {"value": raw / t_enc / 1e9, "unit": "GB/s (raw bytes encoded)", "cores": 1, "kind": "oracle",
               "decode_gbs": raw_d / t_dec / 1e9, "ratio": sum(len(z) for z in streams) / raw,
               "sample": f"{len(sample)} allocations, {raw / 2**20:.0f} MiB of the fp32 content in 64 KiB chunks "
                         f"(decode: the first {raw_d / 2**20:.0f} MiB); numpy, single thread"}
    # The encoder's roofline (64 KiB chunks: the pass made the block headers):
    # crz_size_kernel reads every block's header word (8 B per 512 B) and
    # writes each stream's length and offset; crz_encode_sized_kernel reads
    # the raw payload from staging once, the header words again, and writes
    # the streams: alg = D + Z + 16 k + 2 D / 64 for the two launches, timed
    # together (the device time of both).
    full_f32 = [e for e in enc if e[0] == "f32_normal" and e[1]]
    kind, _, D, Z, k, _ = full_f32[0]
    ms = statistics.median(e[5] for e in full_f32)
    alg = D + Z + 16 * k + 2 * (D // 64)
    roofline = {"bound": "hbm", "kernel": "crz_size_kernel + crz_encode_sized_kernel (full checkpoint, fp32 "
                                          "N(0,1), device images)",
                "achieved": alg / (ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                "frac": alg / (ms / 1e3) / 1e9 / peak, "traffic": profile_traffic("crz_encode_c2_f32"),
                "alg_bytes_per_launch": int(alg), "avg_launch_ms": ms, "raw_gbs": D / (ms / 1e3) / 1e9,
                "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)" if peak_src == "measured" else "fallback"}
    encoder = [{"content": e[0], "checkpoint": "full" if e[1] else "delta", "raw_bytes": e[2],
                "stored_bytes": e[3], "k": e[4], "ms": e[5], "raw_gbs": e[2] / (e[5] / 1e3) / 1e9,
                "hbm_frac": (e[2] + e[3] + 16 * e[4] + 2 * (e[2] // 64)) / (e[5] / 1e3) / 1e9 / peak} for e in enc]
    line = {"workload": "codec: c2 layout (256 allocs = 4 GiB, 64 KiB chunks, 10% hot set), contents "
                        "fp32 N(0,1) / bf16 N(0,1) / zeros / uniform bytes; plain vs CRZ1-coded images",
            "tracked_bytes": B, "n_chunks": n, "steps": steps, "roofline": roofline, "rows": rows,
            "encoder_launches": encoder, "gpu_launches": launches, "clocks": clocks, "cpu_baseline": cpu,
            "arena_growth": {k: mem1[k] - mem0[k] for k in ("host_grow_events", "device_grow_events")},
            "note": "wall_ms includes the drain wait; full = the median of three full checkpoints (the first "
                    "finds every chunk rewritten after an untimed one of uniform bytes, the next two follow an "
                    "invalidation); delta rows are medians over the steps; the restart restores the chain of the "
                    "last full image + steps deltas after zeroing every 17th allocation"}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Config 5: serving loop over 64 simulated process contexts
# ---------------------------------------------------------------------------

class ServingRun:
    """Config 5's serving loop: n_ctx simulated process contexts (log-uniform
    0.5-8 GiB images scaled to `total`, 4-64 allocations each, fp32 N(0,1)),
    checkpoint / restart requests arriving Poisson at `rate` (75% / 25%),
    admitted by a request server with 8 worker slots and a 24 GiB staging
    budget.  Before each checkpoint the request's prepare callback XORs a
    seeded 10% of the context's chunks; every 4th checkpoint of a context is
    FULL (the baseline is dropped first).  A restart targets the context's
    newest committed image.  Latency runs from the scheduled arrival to the
    request's completion event.

    on_result(j, i, kind, result, plan), when given, is called in submission
    order (so in each context's own order) from the collecting thread, with
    plan = {"mut": index into procs[i]["mut_lists"], "full": bool} for a
    checkpoint and {"image": handle, "epoch": its epoch} for a restart (the
    handle may have been released by then; the epoch names the image).
    on_submit(j, i, kind, plan), when given, is called for each restart as it
    is submitted, from the submitting thread.  max_backlog > 0 holds a request
    back (past its arrival time) while that many earlier ones are not yet
    collected: a slow on_result then bounds the images waiting for it instead
    of letting them pile up in memory (latencies are then not the config's)."""

    def __init__(self, dev, n_ctx=64, total=32 * W.GIB, seed=W.SEED_BASE + 5, flags=0, host_reserve=2.0):
        import torch
        import paper_2008_10596_gb300 as C
        self.torch, self.C, self.dev = torch, C, dev
        self.seed = seed
        self.rng = np.random.default_rng(seed)
        self.n_ctx = n_ctx
        self.total = total
        self.S = S = 64 * W.KIB
        raw = W.log_uniform(self.rng, n_ctx, 0.5 * W.GIB, 8 * W.GIB)
        scale = total / (173 * W.GIB)
        ctx_bytes = W.water_fill(raw, total, int(0.5 * W.GIB * scale), int(8 * W.GIB * scale) + 1, 64 * W.KIB)
        g = torch.Generator(device=dev)
        g.manual_seed(seed)
        self.procs = []
        for i, cb in enumerate(ctx_bytes):
            na = int(round(np.exp(self.rng.uniform(np.log(4), np.log(64)))))
            w = self.rng.dirichlet(np.ones(na))
            sizes = [max(64 * W.KIB, int(x * cb) // (64 * W.KIB) * (64 * W.KIB)) for x in w]
            bufs = [torch.randn(n // 4, generator=g, device=dev).view(torch.uint8) for n in sizes]
            ctx = C.crac_ctx_create(C.crac_config_default(
                chunk_bytes=S, lineage=5000 + i, device=dev.index or 0,
                reserve_host_bytes=int(host_reserve * total) if i == 0 else 0, flags=flags))
            for b in bufs:
                C.crac_ctx_register_alloc(ctx, b.data_ptr(), b.numel())
            first = W.chunk_layout(sizes, S)
            mut_lists, muts = [], []
            for r in range(4):
                ms = W.choose_mutations(seed * 131 + i * 7 + r, int(first[-1]), 0.10)
                rows = []
                for m in ms:
                    a = int(np.searchsorted(first, m.chunk, side="right") - 1)
                    lo = (m.chunk - int(first[a])) * S
                    rows.append((bufs[a].data_ptr() + lo, min(S, sizes[a] - lo), m.mask))
                mut_lists.append(ms)
                muts.append(torch.from_numpy(np.array(rows, dtype=np.uint64).view(np.int64)).to(dev))
            self.procs.append({"ctx": ctx, "bufs": bufs, "sizes": sizes, "first": first,
                               "stream": torch.cuda.Stream(dev), "muts": muts, "mut_lists": mut_lists,
                               "bytes": sum(sizes), "ckpts": 0, "images": [], "latest": None})
        torch.cuda.synchronize(dev)

    def base_images(self, on_base=None):
        """The FULL base image of every context, before the measured loop."""
        for i, p in enumerate(self.procs):
            img = self.C.crac_ctx_checkpoint(p["ctx"], p["stream"])
            self.C.crac_image_wait(img)
            p["latest"] = img
            p["images"].append(img)
            if on_base is not None:
                on_base(i, img)
        self.torch.cuda.synchronize(self.dev)

    def run(self, n_req, rate, on_result=None, workers=8, budget=24 * W.GIB, max_lease=4 * W.GIB,
            on_submit=None, max_backlog=0):
        import queue as _q
        import threading
        C, torch = self.C, self.torch
        procs = self.procs
        server = C.crac_server_create(workers=workers, staging_budget=budget, max_lease=max_lease)
        rng = self.rng
        inter = rng.exponential(1.0 / rate, size=n_req)
        arrivals = np.cumsum(inter)
        targets = rng.integers(0, self.n_ctx, size=n_req)
        kinds = np.where(rng.uniform(size=n_req) < 0.75, C.CRAC_REQ_CHECKPOINT, C.CRAC_REQ_RESTART)
        lock = threading.Lock()
        callbacks = []
        results = {}
        errors = []

        def make_prep(p, k_mut, full):
            def prep(stream, arg):
                m = p["muts"][k_mut]
                from paper_2008_10596_gb300 import testkit
                testkit.mutate_xor(m.data_ptr(), m.shape[0], stream)
                if full:
                    C.crac_ctx_invalidate(p["ctx"])
            return C.PREPARE_FN(prep)

        qq = _q.Queue()
        collected = [0]

        def collect():
            for j, t, i, kind, plan in iter(qq.get, None):
                r = C.crac_server_wait(server, t)
                p = procs[i]
                with lock:
                    # under the lock: a restart is not submitted between the
                    # callback's look at this image and its publication below
                    if on_result is not None and not errors:
                        try:
                            on_result(j, i, int(kind), r, plan)
                        except Exception as e:   # reported after the loop
                            errors.append(e)
                    if kind == C.CRAC_REQ_CHECKPOINT and r["status"] == 0:
                        # the drain's own device time (settled: the request waited for it)
                        r["drain_ms"] = C.crac_image_info(r["image"])["drain_ms"]
                        # keep only the newest image: its chain holds what a
                        # restart needs, and each FULL image frees the history
                        for old in p["images"]:
                            C.crac_image_release(old)
                        p["images"] = [r["image"]]
                        p["latest"] = r["image"]
                    results[t] = (int(kind), r, p["bytes"])
                    collected[0] += 1

        m0 = C.crac_memory_stats()
        # The prepare callbacks (the application's mutator launches) run on the
        # server's worker threads and need the GIL: hand it over quickly.
        switch = sys.getswitchinterval()
        sys.setswitchinterval(0.0002)
        th = threading.Thread(target=collect)
        th.start()
        t0 = C.crac_time_now() + 0.05
        for j in range(n_req):
            i = int(targets[j])
            p = procs[i]
            t_arr = t0 + float(arrivals[j])
            while C.crac_time_now() < t_arr:
                time.sleep(min(0.002, max(0.0, t_arr - C.crac_time_now())))
            while max_backlog and j - collected[0] >= max_backlog and th.is_alive():
                time.sleep(0.001)
            if kinds[j] == C.CRAC_REQ_CHECKPOINT:
                p["ckpts"] += 1
                plan = {"mut": p["ckpts"] % 4, "full": p["ckpts"] % 4 == 0}
                cb = make_prep(p, plan["mut"], plan["full"])
                callbacks.append(cb)
                t = C.crac_server_submit(server, p["ctx"], C.CRAC_REQ_CHECKPOINT, None, p["stream"], cb, None, t_arr)
            else:
                with lock:   # the collector releases superseded images under the lock
                    img = p["latest"]
                    plan = {"image": img, "epoch": C.crac_image_info(img)["epoch"]}
                    if on_submit is not None:
                        on_submit(j, i, int(kinds[j]), plan)
                    t = C.crac_server_submit(server, p["ctx"], C.CRAC_REQ_RESTART, img, p["stream"], None, None,
                                             t_arr)
            qq.put((j, t, i, int(kinds[j]), plan))
        qq.put(None)
        th.join()
        sys.setswitchinterval(switch)
        t_end = max(r["t_done"] for _, r, _ in results.values())
        stats = C.crac_server_stats(server)
        C.crac_server_destroy(server)
        if errors:
            raise errors[0]
        m1 = C.crac_memory_stats()
        out = self._summary(results, stats, t0, t_end, arrivals, targets, n_req, rate, workers, budget)
        # CUDA allocations made inside the loop (each can stall the requests in flight)
        out["growth_in_loop"] = {k: m1[k] - m0[k] for k in ("host_grow_events", "device_grow_events",
                                                             "scratch_grow_events")}
        return out

    def _summary(self, results, stats, t0, t_end, arrivals, targets, n_req, rate, workers, budget):
        C = self.C
        lat = {"checkpoint": [], "restart": []}
        wait = {"checkpoint": [], "restart": []}
        serv = {"checkpoint": [], "restart": []}
        # service = prepare callback (the mutator launch, Python) + the
        # operation's call + (checkpoints) the wait for the image to settle
        parts = {k: {"prepare": [], "call": [], "settle": []} for k in ("checkpoint", "restart")}
        full_serv, full_wait = [], []
        drain_gbs, full_drain_gbs = [], []   # payload bytes / drain device time, per checkpoint
        scanned = payload = 0
        fails = 0
        slow = []
        for kind, r, nb in results.values():
            if r["status"] != 0:
                fails += 1
                continue
            ms3 = ((r["t_op"] - r["t_admit"]) * 1e3, (r["t_op_end"] - r["t_op"]) * 1e3,
                   (r["t_done"] - r["t_op_end"]) * 1e3)
            slow.append(((r["t_done"] - r["t_admit"]) * 1e3, kind, nb, r["payload_bytes"],
                         (r["t_admit"] - r["t_arrival"]) * 1e3, r["t_arrival"] - t0, ms3, r.get("drain_ms", 0.0)))
            key = "checkpoint" if kind == C.CRAC_REQ_CHECKPOINT else "restart"
            lat[key].append((r["t_done"] - r["t_arrival"]) * 1e3)
            wait[key].append((r["t_admit"] - r["t_arrival"]) * 1e3)
            serv[key].append((r["t_done"] - r["t_admit"]) * 1e3)
            for name, v in zip(("prepare", "call", "settle"), ms3):
                parts[key][name].append(v)
            if kind == C.CRAC_REQ_CHECKPOINT and r.get("drain_ms", 0) > 0 and r["payload_bytes"] >= (1 << 20):
                g = r["payload_bytes"] / (r["drain_ms"] / 1e3) / 1e9
                drain_gbs.append(g)
                if r["payload_bytes"] >= nb:
                    full_drain_gbs.append(g)
            if kind == C.CRAC_REQ_CHECKPOINT and r["payload_bytes"] >= nb:
                full_serv.append((r["t_done"] - r["t_admit"]) * 1e3)
                full_wait.append((r["t_admit"] - r["t_arrival"]) * 1e3)
            scanned += nb
            payload += r["payload_bytes"]
        wall = t_end - t0
        allv = lat["checkpoint"] + lat["restart"]

        def pct(v, q):
            return float(np.percentile(v, q)) if v else None

        def dist(v):
            return {"p50": pct(v, 50), "p99": pct(v, 99), "max": max(v) if v else None, "n": len(v)}

        return {"contexts": self.n_ctx, "tracked_bytes": sum(p["bytes"] for p in self.procs),
                "requests": n_req, "rate_per_s": rate, "workers": workers, "staging_budget": budget,
                "failed": fails, "wall_s": wall,
                "latency_ms": {k: dist(v) for k, v in lat.items()},
                "latency_all_ms": {"p50": pct(allv, 50), "p99": pct(allv, 99)},
                "queue_wait_ms": {k: dist(v) for k, v in wait.items()},
                "service_ms": {k: dist(v) for k, v in serv.items()},
                "service_parts_ms": {k: {n: dist(v) for n, v in d.items()} for k, d in parts.items()},
                "full_checkpoint_ms": {"service": dist(full_serv), "queue_wait": dist(full_wait)},
                # the drains' own rate (payload / device time of the drain on the
                # context's side stream, checkpoints of at least 1 MiB): a slow
                # tail here is the host link, not queueing or host code
                "drain_gbs": {"all": {"p50": pct(drain_gbs, 50), "p1": pct(drain_gbs, 1),
                                      "min": min(drain_gbs) if drain_gbs else None, "n": len(drain_gbs)},
                              "full": {"p50": pct(full_drain_gbs, 50), "p1": pct(full_drain_gbs, 1),
                                       "min": min(full_drain_gbs) if full_drain_gbs else None,
                                       "n": len(full_drain_gbs)}},
                # the five longest services: what the tail is made of
                "slowest": [{"service_ms": s, "kind": "checkpoint" if k == C.CRAC_REQ_CHECKPOINT else "restart",
                             "context_bytes": nb, "payload_bytes": pb, "queue_wait_ms": w, "arrival_s": a,
                             "prepare_ms": m3[0], "call_ms": m3[1], "settle_ms": m3[2], "drain_ms": dm}
                            for s, k, nb, pb, w, a, m3, dm in sorted(slow, key=lambda x: x[0], reverse=True)[:5]],
                "memory": C.crac_memory_stats(),
                "offered_gbs": sum(self.procs[int(t)]["bytes"] for t in targets) / (float(arrivals[-1]) or 1) / 1e9,
                "achieved_tracked_gbs": scanned / wall / 1e9, "achieved_payload_gbs": payload / wall / 1e9,
                "server": stats}

    def close(self):
        self.torch.cuda.synchronize(self.dev)
        for p in self.procs:
            for img in p["images"]:
                self.C.crac_image_release(img)
            p["images"] = []
            self.C.crac_ctx_destroy(p["ctx"])
        self.procs = []


def run_config5(args):
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    total = (args.total_mib << 20) if args.total_mib != 4096 else 32 * W.GIB
    sr = ServingRun(dev, total=total, flags=restore_flags(args))
    sr.base_images()
    sampler5 = ClockSampler(None)
    sampler5.start()
    out = sr.run(args.requests, args.rate, workers=args.workers)
    out["clocks"] = sampler5.stop()
    sr.close()
    line = {"workload": f"c5: 64 contexts, {total / 2**30:.0f} GiB total (log-uniform 0.5-8 GiB scaled by "
                        f"{total / (173 * W.GIB):.3f}), {args.requests} requests Poisson {args.rate}/s, "
                        "75% ckpt / 25% restart, 10% of chunks mutated before each checkpoint, "
                        f"24 GiB staging budget, {args.workers} slots"}
    line.update(out)
    print(json.dumps(line), flush=True)
    return 0 if out["failed"] == 0 else 1


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="crac", choices=["crac", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline leg")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end (host image) leg")
    ap.add_argument("--total-mib", type=int, default=4096,
                    help="tracked bytes of the config-2 workload (default 4096 = the full config)")
    ap.add_argument("--requests", type=int, default=1200, help="c5: requests in the serving loop")
    ap.add_argument("--rate", type=float, default=20.0, help="c5: Poisson arrival rate (requests/s)")
    ap.add_argument("--workers", type=int, default=8, help="c5: request server slots (requests in flight)")
    ap.add_argument("--no-serving", action="store_true", help="c2: skip the short serving leg")
    ap.add_argument("--serving-gib", type=int, default=8, help="c2: total context memory of the serving leg")
    ap.add_argument("--serving-requests", type=int, default=600, help="c2: requests of the serving leg")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c4", "c5", "passes", "codec"],
                    help="c2 (default): the headline line; c3/c4/c5/passes: their own JSON lines")
    ap.add_argument("--staged-restore", action="store_true",
                    help="c2 e2e, c3, c5: restore host images through staging (copy engine) instead of in place")
    ap.add_argument("--wait-pass", action="store_true",
                    help="host contexts: every checkpoint call waits for its pass (CRAC_FLAG_WAIT_PASS)")
    ap.add_argument("--direct-drain", action="store_true",
                    help="c2 e2e, c3, c5: write host images straight into pinned memory instead of staging + D2H")
    ap.add_argument("--chunk-kib", default="4,64", help="passes: chunk sizes in KiB")
    ap.add_argument("--dirty", default="0,0.1,0.5,1", help="passes: fractions of 4 KiB pages rewritten")
    ap.add_argument("--kernels", default="split,ldg,tma,sparse", help="passes: pass kernels")
    ap.add_argument("--ctas-per-sm", type=int, default=0, help="passes: LDG CTAs per SM (0 = occupancy)")
    ap.add_argument("--chunks-per-tile", type=int, default=0, help="passes: LDG tile in chunks (0 = default)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "crac":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "c3":
        return run_config3(args)
    if args.workload == "c4":
        return run_config4(args)
    if args.workload == "c5":
        return run_config5(args)
    if args.workload == "passes":
        return run_passes(args)
    if args.workload == "codec":
        return run_codec(args)
    return run_crac(args)


if __name__ == "__main__":
    # The serving leg runs 64 contexts, each with its own stream and the
    # library's side stream: with the default 8 hardware work queues, work of
    # unrelated streams shares a queue and waits behind it.  32 queues (the
    # maximum) is the setting a many-context server runs with; it must be set
    # before CUDA starts in this process (a value the caller set is kept), and
    # only when the benchmark itself runs, not when a test imports it.
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    sys.exit(main())
