"""The request server (GPU): continuous admission of checkpoint/restart
requests from several contexts under a staging budget.  Every context runs
the same request sequence twice -- once alone (each request waited for
before the next is submitted, one context at a time) and once in the mix
(all contexts at once, four workers, a staging budget that forces requests
to wait for leases) -- and every image and the restored memory must be
identical byte for byte, and equal to the oracle's.  Two of the contexts
make coded images (CRAC_FLAG_COMPRESS) of fp32 contents."""
import numpy as np
import pytest
import torch

import paper_2008_10596_gb300 as C
import workloads as W
from oracle import oracle as O
from paper_2008_10596_gb300 import testkit

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("oracle_lib")]

KIB = 1024
S = 64 * KIB
SIZES = [[3 * 1024 * KIB + 5, 700 * KIB], [8 * 1024 * KIB], [123457, 2 * 1024 * KIB, 64 * KIB],
         [5 * 1024 * KIB + 64 * KIB], [1024 * KIB, 1024 * KIB + 7, 300 * KIB, 4096]]
PLAN = ["c", "c", "c", "r", "c"]     # checkpoints, restart from the latest image, one more checkpoint
CODED = (1, 3)                       # contexts whose images are coded


class Proc:
    """One simulated process: allocations, a stream, a context and its oracle."""

    def __init__(self, i, sizes):
        self.i = i
        self.sizes = sizes
        coded = i in CODED
        kind = "f32_normal" if coded else "u32_xorshift"
        self.bufs = [torch.from_numpy(W.host_contents(kind, n, 700 + 10 * i + j)).to("cuda")
                     for j, n in enumerate(sizes)]
        self.stream = torch.cuda.Stream()
        self.ctx = C.crac_ctx_create(C.crac_config_default(chunk_bytes=S, lineage=600 + i,
                                                          flags=C.CRAC_FLAG_COMPRESS if coded else 0))
        self.ora = O.OracleContext(S, lineage=600 + i, coded=coded)
        for b, n in zip(self.bufs, sizes):
            C.crac_ctx_register_alloc(self.ctx, b.data_ptr(), n)
            self.ora.register(b.data_ptr(), n)
        first = W.chunk_layout(sizes, S)
        self.muts = []
        for step in range(len(PLAN)):
            ms = W.choose_mutations(1000 * i + step, int(first[-1]), 0.3)
            rows = []
            for m in ms:
                a = int(np.searchsorted(first, m.chunk, side="right") - 1)
                lo = (m.chunk - int(first[a])) * S
                rows.append((self.bufs[a].data_ptr() + lo, min(S, sizes[a] - lo), m.mask))
            self.muts.append(torch.from_numpy(np.array(rows, dtype=np.uint64).view(np.int64)).to("cuda"))
        self.step = 0
        self.images = []
        self.raw = []
        torch.cuda.synchronize()
        self.cb = C.PREPARE_FN(self._prepare)

    def _prepare(self, stream, arg):
        m = self.muts[self.step]
        testkit.mutate_xor(m.data_ptr(), m.shape[0], stream)

    def submit(self, server):
        kind = PLAN[self.step]
        if kind == "c":
            return C.crac_server_submit(server, self.ctx, C.CRAC_REQ_CHECKPOINT, None, self.stream, self.cb)
        return C.crac_server_submit(server, self.ctx, C.CRAC_REQ_RESTART, self.images[-1], self.stream)

    def finish(self, res):
        assert res["status"] == 0, C.crac_status_str(res["status"])
        if PLAN[self.step] == "c":
            self.images.append(res["image"])
            self.raw.append(C.crac_image_serialize(res["image"]))
        self.step += 1

    def close(self):
        for img in self.images:
            C.crac_image_release(img)
        C.crac_ctx_destroy(self.ctx)


def _run(mixed):
    procs = [Proc(i, s) for i, s in enumerate(SIZES)]
    budget = 2 * 8 * 1024 * KIB + 64 * KIB if mixed else 0
    server = C.crac_server_create(workers=4 if mixed else 1, staging_budget=budget or (64 << 20))
    try:
        if mixed:
            live = {p.submit(server): p for p in procs}
            while live:
                t = next(iter(live))
                p = live.pop(t)
                p.finish(C.crac_server_wait(server, t))
                if p.step < len(PLAN):
                    live[p.submit(server)] = p
        else:
            for p in procs:
                while p.step < len(PLAN):
                    p.finish(C.crac_server_wait(server, p.submit(server)))
        stats = C.crac_server_stats(server)
        torch.cuda.synchronize()
        mem = [[b.cpu().numpy() for b in p.bufs] for p in procs]
        raws = [p.raw for p in procs]
        return raws, mem, stats
    finally:
        C.crac_server_destroy(server)
        for p in procs:
            p.close()


def _without_ptrs(raw):
    """The image with its allocation table's orig_ptr fields zeroed (the two
    runs use different allocations; every other byte must match)."""
    b = bytearray(raw)
    n_allocs = int.from_bytes(b[48:56], "little")
    for a in range(n_allocs):
        o = 80 + 40 * a + 8
        b[o:o + 8] = bytes(8)
    return bytes(b)


def test_server_results_alone_equal_mixed_and_oracle():
    raw_a, mem_a, st_a = _run(False)
    raw_b, mem_b, st_b = _run(True)
    assert st_a["max_in_flight"] == 1
    assert st_b["max_in_flight"] > 1                     # requests really overlapped
    assert st_b["staging_high_water"] <= st_b["staging_budget"]
    for pa, pb in zip(raw_a, raw_b):
        assert len(pa) == len(pb) == len(PLAN) - 1
        assert [_without_ptrs(x) for x in pa] == [_without_ptrs(x) for x in pb]
    for ma, mb in zip(mem_a, mem_b):
        for x, y in zip(ma, mb):
            assert np.array_equal(x, y)
    # the images of the mixed run against the oracle, replaying the same plan
    for i, sizes in enumerate(SIZES):
        ora = O.OracleContext(S, lineage=600 + i, coded=i in CODED)
        kind_i = "f32_normal" if i in CODED else "u32_xorshift"
        host = [W.host_contents(kind_i, n, 700 + 10 * i + j) for j, n in enumerate(sizes)]
        for j, n in enumerate(sizes):
            ora.register((i + 1) << 40 | (j << 32), n)
        first = W.chunk_layout(sizes, S)
        imgs = []
        k = 0
        for step, kind in enumerate(PLAN):
            if kind == "c":
                W.apply_mutations_host(host, first, S, W.choose_mutations(1000 * i + step, int(first[-1]), 0.3))
                imgs.append(ora.checkpoint(host))
                got = O.parse_image(raw_b[i][k])
                want = O.parse_image(imgs[-1])
                assert got.fp.tolist() == want.fp.tolist() and got.idx.tolist() == want.idx.tolist()
                assert bytes(got.payload) == bytes(want.payload) and got.epoch == want.epoch
                assert got.coded == want.coded == (i in CODED)
                if got.coded:
                    assert got.zlen.tolist() == want.zlen.tolist()
                k += 1
            else:
                host = ora.restart(imgs)
        for x, y in zip(host, mem_b[i]):
            assert np.array_equal(x, y)
