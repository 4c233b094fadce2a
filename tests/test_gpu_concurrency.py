"""Concurrent contexts (GPU): several host threads, each with its own
context, stream and allocations, checkpoint and restart at the same time,
sharing the process-wide arenas, the image table and the launch counter
(plain and coded images).
Every image must equal the oracle's and every restart must bring back its
memory exactly."""
import threading

import numpy as np
import pytest
import torch

import paper_2008_10596_gb300 as C
import workloads as W
from oracle import oracle as O
from paper_2008_10596_gb300 import testkit

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("oracle_lib")]

KIB = 1024


def _worker(idx, kern, residency, flags, out, errors):
    try:
        S = 4 * KIB
        stream = torch.cuda.Stream()
        rng = np.random.default_rng(idx)
        sizes = [int(x) // 16 * 16 + 16 for x in rng.integers(1, 200000, size=6)]
        with torch.cuda.stream(stream):
            kind = "f32_normal" if flags & C.CRAC_FLAG_COMPRESS else "u8"   # coded: content that shrinks
        bufs = [torch.from_numpy(W.host_contents(kind, n, 900 + 10 * idx + i)).to("cuda", non_blocking=False)
                    for i, n in enumerate(sizes)]
        stream.synchronize()
        ctx = C.crac_ctx_create(C.crac_config_default(chunk_bytes=S, lineage=8000 + idx, pass_kernel=kern,
                                                      image_residency=residency, flags=flags))
        ora = O.OracleContext(S, lineage=8000 + idx, coded=bool(flags & C.CRAC_FLAG_COMPRESS))
        imgs = []
        try:
            for b, n in zip(bufs, sizes):
                C.crac_ctx_register_alloc(ctx, b.data_ptr(), n)
                ora.register(b.data_ptr(), n)
            first = W.chunk_layout(sizes, S)
            for step in range(4):
                if step:
                    muts = W.choose_mutations(idx * 100 + step, int(first[-1]), 0.2)
                    rows = []
                    for m in muts:
                        a = int(np.searchsorted(first, m.chunk, side="right") - 1)
                        lo = (m.chunk - int(first[a])) * S
                        rows.append((bufs[a].data_ptr() + lo, min(S, sizes[a] - lo), m.mask))
                    ent = torch.from_numpy(np.array(rows, dtype=np.uint64).view(np.int64)).to("cuda")
                    testkit.mutate_xor(ent.data_ptr(), len(rows), stream)
                img = C.crac_ctx_checkpoint(ctx, stream)
                imgs.append(img)
                C.crac_image_wait(img)
                stream.synchronize()
                host = [b.cpu().numpy() for b in bufs]
                if C.crac_image_serialize(img) != ora.checkpoint(host):
                    raise AssertionError(f"worker {idx}: image {step} differs from the oracle")
            want = [b.cpu().numpy() for b in bufs]
            for b in bufs:
                b.zero_()
            torch.cuda.synchronize()
            C.crac_ctx_restart(ctx, imgs[-1], stream)
            stream.synchronize()
            for b, w in zip(bufs, want):
                if not np.array_equal(b.cpu().numpy(), w):
                    raise AssertionError(f"worker {idx}: restore differs")
            out[idx] = len(imgs)
        finally:
            torch.cuda.synchronize()
            for img in imgs:
                C.crac_image_release(img)
            C.crac_ctx_destroy(ctx)
    except Exception as e:   # reported by the main thread
        errors.append(e)


def test_concurrent_contexts():
    coded = C.CRAC_FLAG_COMPRESS
    plans = [(C.CRAC_PASS_AUTO, C.CRAC_RESIDENCY_HOST, 0), (C.CRAC_PASS_SPLIT, C.CRAC_RESIDENCY_DEVICE, 0),
             (C.CRAC_PASS_LDG, C.CRAC_RESIDENCY_HOST, 0), (C.CRAC_PASS_TMA, C.CRAC_RESIDENCY_DEVICE, 0),
             (C.CRAC_PASS_SPARSE, C.CRAC_RESIDENCY_DEVICE, 0), (C.CRAC_PASS_AUTO, C.CRAC_RESIDENCY_DEVICE, 0),
             (C.CRAC_PASS_SPLIT, C.CRAC_RESIDENCY_HOST, coded),
             (C.CRAC_PASS_AUTO, C.CRAC_RESIDENCY_HOST, coded | C.CRAC_FLAG_DIRECT_DRAIN),
             (C.CRAC_PASS_TMA, C.CRAC_RESIDENCY_DEVICE, coded)]
    out, errors = {}, []
    threads = [threading.Thread(target=_worker, args=(i, k, r, f, out, errors)) for i, (k, r, f) in enumerate(plans)]
    launches0 = C.crac_kernel_launches()
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errors:
        raise errors[0]
    assert sorted(out) == list(range(len(plans))) and all(v == 4 for v in out.values())
    assert C.crac_kernel_launches() > launches0
