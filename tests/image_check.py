"""Whole-image comparison of a library image with the oracle at any size (GPU).

At multi-GiB sizes neither the library's serialized image nor the oracle's
copy of it is built whole.  The oracle takes the checkpoint one allocation at
a time (OracleContext.checkpoint_by_alloc), reading each allocation's bytes
from device memory once; each part it hands out -- the allocation's
fingerprints, the global ids of its dirty chunks, (the stream lengths of a
coded image,) and its payload bytes -- is compared with the same bytes of the
library's serialized image, read by range through the C ABI
(crac_image_read).  Header and allocation table are compared last, and the
section sizes must add up to the image's size, so every byte of the image is
compared with the oracle's.
"""
from __future__ import annotations

import ctypes
import os
import time

import numpy as np
import torch

import paper_2008_10596_gb300 as C
from oracle import oracle as O
from workloads.device import raw_tensor

HEADER_BYTES = 80
ALLOC_BYTES = 40


def host_workers() -> int:
    return max(1, os.cpu_count() or 1)


class AllocReader:
    """read(i) -> host bytes of allocation i, through two pinned buffers: the
    copy of allocation i + 1 runs on a side stream while the oracle works on
    allocation i.  Device and managed memory are copied by the copy engine;
    page-locked host memory is read where it is."""

    def __init__(self, ptrs, sizes, kinds):
        self.ptrs, self.sizes, self.kinds = list(ptrs), list(sizes), list(kinds)
        cap = max([s for s, k in zip(self.sizes, self.kinds) if k != C.CRAC_KIND_HOST] + [1])
        self.buf = [torch.empty(cap, dtype=torch.uint8, pin_memory=True) for _ in range(2)]
        self.stream = torch.cuda.Stream()
        self.ev = [torch.cuda.Event(), torch.cuda.Event()]
        self.pending = {}

    def _start(self, i):
        if i >= len(self.ptrs) or i in self.pending or self.kinds[i] == C.CRAC_KIND_HOST:
            return
        slot = i % 2
        self.stream.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(self.stream):
            self.buf[slot][:self.sizes[i]].copy_(raw_tensor(self.ptrs[i], self.sizes[i]), non_blocking=True)
            self.ev[slot].record(self.stream)
        self.pending[i] = slot

    def read(self, i):
        n = self.sizes[i]
        if self.kinds[i] == C.CRAC_KIND_HOST:
            torch.cuda.synchronize()
            out = np.frombuffer(ctypes.string_at(self.ptrs[i], n), dtype=np.uint8)
            self._start(i + 1)
            return out
        self._start(i)
        slot = self.pending.pop(i)
        self.ev[slot].synchronize()
        out = self.buf[slot][:n].numpy()
        self._start(i + 1)   # lands in the other buffer, while the oracle reads this one
        return out


def verify_image(img: int, ora: O.OracleContext, reader: AllocReader) -> dict:
    """Compare every byte of library image `img` with the image the oracle
    context computes from the current contents of its registered
    allocations (which `reader` reads, in registration order).  Raises
    AssertionError at the first difference; returns sizes and timings."""
    t0 = time.perf_counter()
    C.crac_image_wait(img)
    info = C.crac_image_info(img)
    na = len(ora.allocs)
    assert info["n_allocs"] == na, (info["n_allocs"], na)
    first = ora.layout()
    n = int(first[-1])
    assert info["n_chunks"] == n, (info["n_chunks"], n)
    k = info["k"]
    coded = bool(info["flags"] & C.CRAC_IMAGE_CODED)
    fp_at = HEADER_BYTES + ALLOC_BYTES * na
    idx_at = fp_at + 8 * n
    zlen_at = idx_at + 8 * k
    pay_at = zlen_at + (8 * k if coded else 0)
    pos = {"k": 0, "d": 0}
    scratch = {}

    def lib_u64(offset, count):
        return np.frombuffer(C.crac_image_read(img, offset, 8 * count), dtype="<u8")

    def lib_bytes(offset, count):
        b = scratch.get("pay")
        if b is None or b.size < count:
            b = scratch["pay"] = np.empty(max(count, 1 << 20), dtype=np.uint8)
        C.crac_image_read(img, offset, count, out=b[:count])
        return b[:count]

    def visit(i, fa, ids, pieces, zlen):
        lo = int(first[i])
        got = lib_u64(fp_at + 8 * lo, fa.size)
        if not np.array_equal(got, fa):
            bad = np.flatnonzero(got != fa)[:4]
            raise AssertionError(f"allocation {i}: fingerprints differ at chunks {(lo + bad).tolist()}")
        kk = int(ids.size)
        assert pos["k"] + kk <= k, f"allocation {i}: more dirty chunks than the image lists"
        got = lib_u64(idx_at + 8 * pos["k"], kk)
        if not np.array_equal(got, ids):
            raise AssertionError(f"allocation {i}: dirty chunk ids differ")
        if coded:
            got = lib_u64(zlen_at + 8 * pos["k"], kk)
            assert np.array_equal(got, zlen), f"allocation {i}: stream lengths differ"
        blob = b"".join(pieces)
        assert pos["d"] + len(blob) <= info["payload_bytes"], f"allocation {i}: payload longer than the image's"
        got = lib_bytes(pay_at + pos["d"], len(blob))
        if not np.array_equal(got, np.frombuffer(blob, dtype=np.uint8)):
            raise AssertionError(f"allocation {i}: payload bytes differ")
        pos["k"] += kk
        pos["d"] += len(blob)

    head = ora.checkpoint_by_alloc(reader.read, visit)
    assert pos["k"] == k, (pos["k"], k)
    assert pos["d"] == info["payload_bytes"], (pos["d"], info["payload_bytes"])
    assert info["serialized_bytes"] == pay_at + pos["d"]
    assert C.crac_image_read(img, 0, len(head)) == head, "header or allocation table differs"
    return {"serialized_bytes": info["serialized_bytes"], "k": k, "payload_bytes": info["payload_bytes"],
            "n_chunks": n, "seconds": time.perf_counter() - t0}


def mirror(ctx_chunk: int, lineage: int, ptrs, sizes, kinds, coded=False) -> O.OracleContext:
    """An oracle context with the same registry, using every host core for
    the fingerprint loop."""
    ora = O.OracleContext(ctx_chunk, lineage=lineage, coded=coded, workers=host_workers())
    for p, nb, kd in zip(ptrs, sizes, kinds):
        ora.register(p, nb, kd)
    return ora
