"""Config 5's serving loop with every request checked against an oracle replay (GPU).

The benchmark's serving loop (bench.ServingRun: 64 contexts, Poisson
arrivals, 75% checkpoints / 25% restarts, admission by worker slots and a
staging budget, requests of different contexts overlapping on the device)
runs with a callback that replays each context's requests, in the order the
context saw them, on an oracle context holding a host copy of its memory:

* checkpoint: the same seeded 10% chunk XOR is applied to the host copy (and
  the baseline dropped where the request made a FULL image); the library's
  image must equal, byte for byte, the oracle's image of the host copy;
* restart: the oracle restores the same image's chain into the host copy
  (the next checkpoint of the context then checks the restored memory, and
  at the end every context's device memory is compared with its copy).

By default the contexts hold 1 GiB in all (the config's log-uniform
0.5-8 GiB sizes scaled down) and 200 requests arrive at 20/s; with
CRAC_FULLSIZE_C5=1 the loop runs at the benchmark's 32 GiB and 1200
requests.  The replay is slower than the arrivals, so a request is held back
while 16 earlier ones wait for it (the loop's images stay bounded in pinned
memory; the latencies are not the benchmark's).
"""
import os
import threading

import numpy as np
import pytest
import torch

import bench
import paper_2008_10596_gb300 as C
import workloads as W
from oracle import oracle as O
from tests.image_check import host_workers

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("oracle_lib")]

FULL_C5 = os.environ.get("CRAC_FULLSIZE_C5") == "1"


class Replay:
    def __init__(self, sr):
        self.sr = sr
        self.ora, self.host, self.raw = [], [], []
        for i, p in enumerate(sr.procs):
            o = O.OracleContext(sr.S, lineage=5000 + i, workers=host_workers())
            for b in p["bufs"]:
                o.register(b.data_ptr(), b.numel())
            self.ora.append(o)
            self.host.append([b.cpu().numpy().copy() for b in p["bufs"]])
            self.raw.append({})          # epoch -> serialized image, the newest image's chain
        self.checked = {"checkpoint": 0, "restart": 0, "full": 0}
        # epochs that submitted, not yet replayed restarts target, per context
        self.pinned = [dict() for _ in sr.procs]
        self.lock = threading.Lock()

    def on_submit(self, j, i, kind, plan):
        with self.lock:
            e = plan["epoch"]
            self.pinned[i][e] = self.pinned[i].get(e, 0) + 1

    def _keep(self, i, lib):
        """Store an image; keep the newest image's chain and the chains of the
        images that submitted restarts still target (a restart targets the
        newest image published when it was submitted, which may be older than
        the newest one stored by now; the serving loop runs this callback and
        publishes the image under one lock, so no restart is submitted in
        between)."""
        im = O.parse_image(lib)
        with self.lock:
            self.raw[i][im.epoch] = lib
            keep = set()
            for top in [im.epoch] + list(self.pinned[i]):
                e = top
                while e not in keep:
                    keep.add(e)
                    pe = O.parse_image(self.raw[i][e])
                    if pe.full:
                        break
                    e = pe.parent_epoch
            for old in [x for x in self.raw[i] if x not in keep]:
                del self.raw[i][old]
        return im

    def on_base(self, i, img):
        lib = C.crac_image_serialize(img)
        assert lib == self.ora[i].checkpoint(self.host[i]), f"context {i}: base image differs"
        self._keep(i, lib)

    def on_result(self, j, i, kind, r, plan):
        assert r["status"] == 0, f"request {j} failed: {r['status']}"
        p = self.sr.procs[i]
        if kind == C.CRAC_REQ_CHECKPOINT:
            W.apply_mutations_host(self.host[i], p["first"], self.sr.S, p["mut_lists"][plan["mut"]])
            if plan["full"]:
                self.ora[i].invalidate()
            lib = C.crac_image_serialize(r["image"])
            want = self.ora[i].checkpoint(self.host[i])
            assert lib == want, f"request {j}: context {i}'s image differs from the oracle's"
            im = self._keep(i, lib)
            self.checked["checkpoint"] += 1
            self.checked["full"] += int(im.full)
        else:
            chain, e = [], plan["epoch"]
            with self.lock:
                while True:
                    b = self.raw[i][e]
                    chain.append(b)
                    pe = O.parse_image(b)
                    if pe.full:
                        break
                    e = pe.parent_epoch
                left = self.pinned[i][plan["epoch"]] - 1
                if left:
                    self.pinned[i][plan["epoch"]] = left
                else:
                    del self.pinned[i][plan["epoch"]]
            mem = self.ora[i].restart(chain[::-1])
            self.host[i] = [m.copy() for m in mem]
            self.checked["restart"] += 1


def test_serving_loop_against_oracle_replay():
    dev = torch.device("cuda", 0)
    total, n_req = (32 * W.GIB, 1200) if FULL_C5 else (1 * W.GIB, 200)
    # host memory: the images' pinned memory (the newest chains, about 1.3x
    # the contexts), the replay's copy of every context and its serialized
    # chains (about 1.3x again) must fit the host together
    sr = bench.ServingRun(dev, total=total, host_reserve=1.5 if FULL_C5 else 2.0)
    try:
        rep = Replay(sr)
        sr.base_images(rep.on_base)
        # the replay is slower than the arrivals: at most 16 requests wait for
        # it, so that superseded images do not pile up in pinned memory
        out = sr.run(n_req, 20.0, on_result=rep.on_result, on_submit=rep.on_submit, max_backlog=16)
        assert out["failed"] == 0
        assert rep.checked["checkpoint"] + rep.checked["restart"] == n_req
        assert rep.checked["restart"] > 0 and rep.checked["full"] > 0
        # every context's memory equals its replayed copy
        torch.cuda.synchronize()
        for i, p in enumerate(sr.procs):
            for b, h in zip(p["bufs"], rep.host[i]):
                assert np.array_equal(b.cpu().numpy(), h), f"context {i}: memory differs from the replay"
        print("serving replay:", rep.checked, "overlap: max in flight", out["server"].get("max_in_flight"))
    finally:
        sr.close()
