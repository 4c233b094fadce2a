"""Configs 2, 3 and 4 at their stated sizes, every image byte against the oracle (GPU).

Each image the library writes is compared, section by section, with the
image the oracle computes from the same device memory (tests/image_check.py):
every fingerprint, every dirty chunk id and every payload byte.  Restores are
compared with a device copy of the memory they must reproduce.

* config 2: 256 allocations, 4 GiB, fp32 N(0,1), 64 KiB chunks, 10% of chunks
  XOR-mutated; FULL image, restore, delta, chain restore; host and device
  images.
* config 3: 12 GiB device + 4 GiB managed memory, bf16 contents, 25% of the
  64 KiB pages rewritten on four streams before each of three checkpoints
  (joined into the checkpoint's stream), restart from the third image.
* config 4 shape at 8 GiB (128 allocations, Zipf sizes, uint8/fp32/int64):
  for each dirty fraction 0/1/10/50/100% of the 4 KiB pages, the autotuner
  picks chunk size and kernel, then a FULL image and a delta with that
  choice are verified and the chain restored.  The staging capacity is set
  to 2 GiB, so the pass runs in several staging segments.  With
  CRAC_FULLSIZE_C4=1 the same test runs at config 4's 120 GiB and 2048
  allocations (images kept on the device, each released once verified).
"""
import os

import numpy as np
import pytest
import torch

import paper_2008_10596_gb300 as C
import workloads as W
from paper_2008_10596_gb300 import testkit
from tests.image_check import AllocReader, mirror, verify_image
from workloads.device import C3Memory, c2_memory, c4_memory, rows_tensor

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("oracle_lib")]


def _mut_rows(ptrs, sizes, first, S, muts):
    rows = []
    for m in muts:
        a = int(np.searchsorted(first, m.chunk, side="right") - 1)
        lo = (m.chunk - int(first[a])) * S
        rows.append((ptrs[a] + lo, min(S, sizes[a] - lo), m.mask))
    return rows


def _restore_matches(ctx, img, tensors, stream):
    """Restart `img` into zeroed memory; the memory must equal what it held."""
    saved = [t.clone() for t in tensors]
    for t in tensors:
        t.zero_()
    C.crac_ctx_restart(ctx, img, stream)
    torch.cuda.synchronize()
    ok = all(torch.equal(a, b) for a, b in zip(tensors, saved))
    del saved
    return ok


@pytest.mark.parametrize("residency", [C.CRAC_RESIDENCY_HOST, C.CRAC_RESIDENCY_DEVICE])
def test_config2_every_byte(residency):
    dev = torch.device("cuda", 0)
    wl, bufs = c2_memory(dev)
    S = wl.chunk_bytes
    ptrs = [b.data_ptr() for b in bufs]
    kinds = [C.CRAC_KIND_DEVICE] * len(bufs)
    first = W.chunk_layout(wl.sizes, S)
    n = int(first[-1])
    stream = torch.cuda.current_stream()
    ctx = C.crac_ctx_create(C.crac_config_default(chunk_bytes=S, lineage=2, image_residency=residency))
    ora = mirror(S, 2, ptrs, wl.sizes, kinds)
    reader = AllocReader(ptrs, wl.sizes, kinds)
    imgs = []
    try:
        for p, nb in zip(ptrs, wl.sizes):
            C.crac_ctx_register_alloc(ctx, p, nb, C.CRAC_KIND_DEVICE)
        img1 = C.crac_ctx_checkpoint(ctx, stream)
        imgs.append(img1)
        r1 = verify_image(img1, ora, reader)
        assert r1["k"] == n and r1["payload_bytes"] == wl.total_bytes
        assert _restore_matches(ctx, img1, bufs, stream)

        muts = W.choose_mutations(wl.seed, n, wl.dirty_fraction)
        ent = rows_tensor(_mut_rows(ptrs, wl.sizes, first, S, muts), dev)
        testkit.mutate_xor(ent.data_ptr(), len(muts), stream)
        img2 = C.crac_ctx_checkpoint(ctx, stream)
        imgs.append(img2)
        r2 = verify_image(img2, ora, reader)
        assert r2["k"] == len(muts)
        assert _restore_matches(ctx, img2, bufs, stream)
    finally:
        torch.cuda.synchronize()
        for i in imgs:
            C.crac_image_release(i)
        C.crac_ctx_destroy(ctx)


def test_config3_every_byte():
    dev = torch.device("cuda", 0)
    mem = C3Memory(dev)
    S = mem.S
    stream = torch.cuda.current_stream(dev)
    B = sum(mem.sizes)
    ctx = C.crac_ctx_create(C.crac_config_default(chunk_bytes=S, lineage=3, device=0,
                                                  reserve_host_bytes=int(1.6 * B)))
    ora = mirror(S, 3, mem.ptrs, mem.sizes, mem.kinds)
    reader = AllocReader(mem.ptrs, mem.sizes, mem.kinds)
    imgs = []
    try:
        assert sum(mem.wl.sizes) == 12 * W.GIB and sum(mem.wl.managed_sizes) == 4 * W.GIB
        for p, nb, kd in zip(mem.ptrs, mem.sizes, mem.kinds):
            C.crac_ctx_register_alloc(ctx, p, nb, kd)
        for i in range(3):
            if i:
                mem.mutate(mem.wl.seed + i)
            img = C.crac_ctx_checkpoint(ctx, stream)
            imgs.append(img)
            info = C.crac_ctx_last_pass(ctx)
            assert info["prefetch_ms"] >= 0
            r = verify_image(img, ora, reader)
            if i == 0:
                assert r["payload_bytes"] == B
            else:
                assert 0 < r["k"] < r["n_chunks"]
        # restart from the third image (FULL + two deltas) into zeroed memory
        keep = [torch.empty(nb, dtype=torch.uint8, device=dev) for nb in mem.sizes]
        e = rows_tensor(mem.copy_rows([t.data_ptr() for t in keep]), dev)
        testkit.rewrite(e.data_ptr(), len(keep), stream)
        zero = torch.zeros(64 << 20, dtype=torch.uint8, device=dev)
        rows = [(p + o, zero.data_ptr(), min(64 << 20, nb - o))
                for p, nb in zip(mem.ptrs, mem.sizes) for o in range(0, nb, 64 << 20)]
        e = rows_tensor(rows, dev)
        testkit.rewrite(e.data_ptr(), len(rows), stream)
        C.crac_ctx_restart(ctx, imgs[-1], stream)
        back = [torch.empty(nb, dtype=torch.uint8, device=dev) for nb in mem.sizes]
        e = rows_tensor(mem.copy_rows([t.data_ptr() for t in back]), dev)
        testkit.rewrite(e.data_ptr(), len(back), stream)
        torch.cuda.synchronize()
        assert all(torch.equal(a, b) for a, b in zip(keep, back))
    finally:
        torch.cuda.synchronize()
        for i in imgs:
            C.crac_image_release(i)
        C.crac_ctx_destroy(ctx)
        mem.free()


FULL_C4 = os.environ.get("CRAC_FULLSIZE_C4") == "1"


def test_config4_sweep_every_byte():
    dev = torch.device("cuda", 0)
    total, n_allocs = (120 * W.GIB, 2048) if FULL_C4 else (8 * W.GIB, 128)
    sizes, bufs, mutate = c4_memory(total, n_allocs, dev)
    ptrs = [b.data_ptr() for b in bufs]
    kinds = [C.CRAC_KIND_DEVICE] * len(bufs)
    stream = torch.cuda.current_stream(dev)
    reader = AllocReader(ptrs, sizes, kinds)
    cands = [4 * W.KIB, 64 * W.KIB, 256 * W.KIB]
    chosen = []
    for j, frac in enumerate((0.0, 0.01, 0.10, 0.50, 1.00)):
        ctx = C.crac_ctx_create(C.crac_config_default(
            chunk_bytes=64 * W.KIB, lineage=40 + j, device=0, staging_bytes=(8 if FULL_C4 else 2) * W.GIB,
            image_residency=C.CRAC_RESIDENCY_DEVICE))
        imgs = []
        try:
            for p, nb in zip(ptrs, sizes):
                C.crac_ctx_register_alloc(ctx, p, nb)
            C.crac_ctx_tune_observe(ctx, cands, stream)
            for r in range(2):
                mutate(frac, 100 * j + r)
                C.crac_ctx_tune_observe(ctx, cands, stream)
            res = C.crac_ctx_tune_apply(ctx, 190.0, stream)
            S, kern = res["chosen_chunk_bytes"], res["chosen_pass_kernel"]
            ora = mirror(S, 40 + j, ptrs, sizes, kinds)
            if FULL_C4:
                free, tot = torch.cuda.mem_get_info()
                print(f"c4 point {frac}: chunk {S}, kernel {kern}; device free {free / 2**30:.1f} of "
                      f"{tot / 2**30:.1f} GiB, torch reserved {torch.cuda.memory_reserved() / 2**30:.1f} GiB, "
                      f"arenas {C.crac_memory_stats()}", flush=True)
            a = C.crac_ctx_checkpoint(ctx, stream)
            imgs.append(a)
            ra = verify_image(a, ora, reader)
            assert ra["k"] == ra["n_chunks"]
            if FULL_C4:   # keep only the newest image in device memory
                C.crac_ctx_drop_history(ctx)
                C.crac_image_release(imgs.pop())
            mutate(frac, 100 * j + 7)
            b = C.crac_ctx_checkpoint(ctx, stream)
            imgs.append(b)
            info = C.crac_ctx_last_pass(ctx)
            rb = verify_image(b, ora, reader)
            chosen.append((frac, S, kern, info["pass_kernel"], rb["k"], rb["n_chunks"], info["segments"]))
            if frac == 0.0:
                assert rb["k"] == 0
            if not FULL_C4:
                assert _restore_matches(ctx, b, bufs, stream)
        finally:
            torch.cuda.synchronize()
            for i in imgs:
                C.crac_image_release(i)
            C.crac_ctx_destroy(ctx)
    print("c4 sweep (fraction, chunk, tuned kernel, kernel run, k, n, segments):", chosen)
