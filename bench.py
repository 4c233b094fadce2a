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


def profile_traffic(kernel_tag: str):
    """Per-launch DRAM bytes from the committed ncu summary, if it matches the kernel source."""
    import hashlib
    src = os.path.join(ROOT, "paper_2008_10596_gb300", "csrc", "crac_kernels.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    path = os.path.join(ROOT, "profiles", f"{kernel_tag}.md")
    if not os.path.exists(path):
        return None
    fields = {}
    for line in open(path):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    if fields.get("kernel_src_sha") != sha:
        return None
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
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


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


def oracle_step_timer(host_bufs, S, seed):
    """Returns (setup, step) for the oracle: step() = mutate 10% + incremental
    checkpoint + full restart of the chain, on host byte arrays."""
    from oracle import oracle as O
    sizes = [b.size for b in host_bufs]
    ctx = O.OracleContext(S, lineage=1)
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


def cpu_baseline_measure(host_bufs, S, seed, label, target_s=10.0, max_steps=20):
    step = oracle_step_timer(host_bufs, S, seed)
    t0 = time.perf_counter()
    nbytes, steps = 0, 0
    while steps < max_steps and (steps == 0 or time.perf_counter() - t0 < target_s):
        nbytes += step()
        steps += 1
    dt = time.perf_counter() - t0
    return {"value": nbytes / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{label}; {steps} steps", "seconds": round(dt, 3)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import build as ob
    ob.build()
    wl = W.config2()
    budget = int(os.environ.get("CRAC_REF_SAMPLE_BYTES", str(1 << 30)))
    sizes = _sample_prefix(wl.sizes, budget)
    host = [W.host_contents("f32_normal", n, wl.seed + i) for i, n in enumerate(sizes)]
    step = oracle_step_timer(host, wl.chunk_bytes, wl.seed)
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    nbytes = 0
    for _ in range(args.steps):
        nbytes += step()
    dt = time.perf_counter() - t0
    v = nbytes / dt / 1e9
    label = (f"first {len(sizes)} of 256 c2 allocations ({sum(sizes) / 2**20:.0f} MiB), numpy N(0,1); "
             "per step: 10% mutate + incremental ckpt + full chain restart; single thread")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_bytes": sum(sizes)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": label},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# The CUDA path
# ---------------------------------------------------------------------------

def run_crac(args):
    import torch
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

    ctx_dev = make_ctx(image_residency=C.CRAC_RESIDENCY_DEVICE, reserve_device_bytes=8 * B)
    ctx_host = make_ctx(image_residency=C.CRAC_RESIDENCY_HOST, reserve_host_bytes=3 * B)
    ctx_pa = make_ctx(image_residency=C.CRAC_RESIDENCY_DEVICE, launch_mode=C.CRAC_LAUNCH_PER_ALLOC)
    ctx_b = make_ctx(image_residency=C.CRAC_RESIDENCY_DEVICE)
    ctx_ldg = make_ctx(image_residency=C.CRAC_RESIDENCY_DEVICE, pass_kernel=C.CRAC_PASS_LDG)
    ctx_tma = make_ctx(image_residency=C.CRAC_RESIDENCY_DEVICE, pass_kernel=C.CRAC_PASS_TMA)

    def step(ctx, host=False, pass_ms=None, lat_ms=None):
        mutate()
        t0 = time.perf_counter()
        img = C.crac_ctx_checkpoint(ctx, stream)
        if host:
            C.crac_image_wait(img)
        if lat_ms is not None:
            lat_ms.append((time.perf_counter() - t0) * 1e3)
        if pass_ms is not None:
            info = C.crac_ctx_last_pass(ctx)
            pass_ms.append((info["device_ms"], info["k"], info["payload_bytes"], info["hash_ms"],
                            info["finalize_ms"], info["gather_ms"]))
        C.crac_ctx_restart(ctx, img, stream)
        C.crac_image_release(img)

    # Base images (full) for each context.
    for ctx in (ctx_dev, ctx_host, ctx_pa, ctx_b, ctx_ldg, ctx_tma):
        img = C.crac_ctx_checkpoint(ctx, stream)
        C.crac_image_wait(img)
        C.crac_image_release(img)
    torch.cuda.synchronize()

    # ---- value: device-resident images --------------------------------------
    # Clocks are sampled from the start of the warm-up to the end of the timed
    # steps (the timed region alone is shorter than the sampling period).
    sampler = ClockSampler(None)
    sampler.start()
    for _ in range(args.warmup):
        step(ctx_dev)
    torch.cuda.synchronize()
    barrier()
    launches0 = C.crac_kernel_launches()
    pass_ms, lat_ms = [], []
    torch.cuda.synchronize()
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step(ctx_dev, pass_ms=pass_ms, lat_ms=lat_ms)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    t_ms = ev0.elapsed_time(ev1)
    if world > 1:
        tt = torch.tensor([t_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_ms = float(tt.item())
    launches = C.crac_kernel_launches() - launches0 + args.steps   # + one mutator launch per step
    bytes_per_step = 2 * B
    value = bytes_per_step * args.steps * world / (t_ms / 1e3) / 1e9

    # ---- roofline: the dominant kernel is the split pass's streaming hash ------
    dev_ms = statistics.mean(p[0] for p in pass_ms)
    k_avg = statistics.mean(p[1] for p in pass_ms)
    d_avg = statistics.mean(p[2] for p in pass_ms)
    hash_ms = statistics.mean(p[3] for p in pass_ms)
    fin_ms = statistics.mean(p[4] for p in pass_ms)
    gat_ms = statistics.mean(p[5] for p in pass_ms)
    peak, peak_src = load_peaks()
    alg_hash = B + 8 * n                          # every tracked byte read once + one accumulator per chunk
    achieved = alg_hash / (hash_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": profile_traffic("split_hash_c2_64KiB"), "kernel": "split_hash_kernel",
                "alg_bytes_per_launch": int(alg_hash), "avg_launch_ms": hash_ms,
                "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)" if peak_src == "measured" else "fallback"}
    alg_pass = B + d_avg + 16 * n + 16 * k_avg    # read B, write D, fp old + new, idx + off
    pass_info = {"kernels": "split: hash -> finalize+compact -> gather (one graph)", "device_ms": dev_ms,
                 "hash_ms": hash_ms, "finalize_ms": fin_ms, "gather_ms": gat_ms,
                 "alg_bytes": int(alg_pass), "achieved_gbs": alg_pass / (dev_ms / 1e3) / 1e9,
                 "frac": alg_pass / (dev_ms / 1e3) / 1e9 / peak, "tracked_gbs": B / (dev_ms / 1e3) / 1e9}

    # ---- batched vs per-allocation launches, and the pass variants -------------
    cmp = {"per_alloc": ([], []), "split": ([], []), "ldg": ([], []), "tma": ([], [])}
    ctxs = {"per_alloc": ctx_pa, "split": ctx_b, "ldg": ctx_ldg, "tma": ctx_tma}
    for _ in range(max(3, min(args.steps, 5))):
        mutate()
        for name, ctx in ctxs.items():
            t0 = time.perf_counter()
            img = C.crac_ctx_checkpoint(ctx, stream)
            cmp[name][1].append((time.perf_counter() - t0) * 1e3)
            cmp[name][0].append(C.crac_ctx_last_pass(ctx)["device_ms"])
            C.crac_image_release(img)
    med = {k: (statistics.median(v[0]), statistics.median(v[1])) for k, v in cmp.items()}
    batched = {"per_alloc_device_ms": med["per_alloc"][0], "batched_device_ms": med["split"][0],
               "speedup_device": med["per_alloc"][0] / med["split"][0],
               "per_alloc_wall_ms": med["per_alloc"][1], "batched_wall_ms": med["split"][1],
               "speedup_wall": med["per_alloc"][1] / med["split"][1],
               "per_alloc_launches": 3 * len(sizes), "batched_graph_launches": 1,
               "variants_device_ms": {k: v[0] for k, v in med.items()}}

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
    e2e_steps = 0 if args.no_e2e else max(1, min(args.steps, 5))
    e2e = None
    if e2e_steps:
        step(ctx_host, host=True)
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e_pass = []
        e0.record(stream)
        for _ in range(e2e_steps):
            step(ctx_host, host=True, pass_ms=e_pass)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        te = e0.elapsed_time(e1)
        k_e = statistics.mean(p[1] for p in e_pass)
        d_e = statistics.mean(p[2] for p in e_pass)
        d2h = int(d_e + 8 * k_e + 8 * n + 64)
        h2d = int(B + d_e + 16 * k_e + 8 * n + 2 * n + 32 * len(sizes))
        e2e = {"value": bytes_per_step * e2e_steps * world / (te / 1e3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": e2e_steps,
               "ms_per_step": te / e2e_steps, "link": link}

    # ---- CPU oracle on a bounded sample (rank 0, N=1 only) -------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        from oracle import build as ob
        ob.build()
        budget = int(os.environ.get("CRAC_CPU_SAMPLE_BYTES", str(1 << 30)))
        ssz = _sample_prefix(sizes, budget)
        host = [bufs[i].cpu().numpy().copy() for i in range(len(ssz))]
        cpu = cpu_baseline_measure(host, S, wl.seed,
                                   f"first {len(ssz)} of 256 allocations ({sum(ssz) / 2**20:.0f} MiB) of this "
                                   "workload read back to host; 10% mutate + incremental ckpt + full restart; "
                                   "single thread")
        cpu["nproc"] = os.cpu_count()

    for ctx in (ctx_dev, ctx_host, ctx_pa, ctx_b, ctx_ldg, ctx_tma):
        C.crac_ctx_destroy(ctx)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
                "config": {"workload": workload, "allocs": len(sizes), "tracked_bytes": B, "chunk_bytes": S,
                           "dirty_fraction": wl.dirty_fraction, "n_chunks": n,
                           "l2": "inputs (4 GiB) larger than L2 (126 MB); no flush",
                           "step": "mutate 10% + incremental ckpt + full restart (device-resident images)",
                           "parallelism": f"replicas{world}"},
                "roofline": roofline, "pass": pass_info, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                "gpu_launches": launches, "batched_vs_per_alloc": batched,
                "ckpt_latency_ms": {"p50": statistics.median(lat_ms),
                                    "p99": float(np.percentile(lat_ms, 99))},
                "ckpt_pass_gbs": B / (dev_ms / 1e3) / 1e9, "dirty_chunks": k_avg, "dirty_bytes": d_avg}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


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
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "crac":
        print("note: fewer than 3 warm-up steps", file=sys.stderr)
    return run_reference(args) if args.impl == "reference" else run_crac(args)


if __name__ == "__main__":
    sys.exit(main())
