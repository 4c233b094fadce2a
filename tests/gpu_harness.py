"""Test harness: device allocations, a libcrac context and an oracle context
kept in lockstep.  Inputs come from `workloads`; the oracle sees the device
bytes as copied back to the host; the library sees the device memory."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

import paper_2008_10596_gb300 as C
import workloads as W
from oracle import oracle as O
from paper_2008_10596_gb300 import testkit


class Buf:
    def __init__(self, nbytes: int, kind: int, tensor=None, ptr: int = 0):
        self.nbytes = nbytes
        self.kind = kind
        self.tensor = tensor
        self.ptr = tensor.data_ptr() if tensor is not None else ptr

    def read(self) -> np.ndarray:
        if self.tensor is not None:
            t = self.tensor[: self.nbytes]
            if t.device.type == "cpu":     # pinned host memory: copy, do not alias it
                torch.cuda.synchronize()
                return t.numpy().copy()
            return t.cpu().numpy()
        torch.cuda.synchronize()
        return np.frombuffer(ctypes.string_at(self.ptr, self.nbytes), dtype=np.uint8).copy()

    def write(self, data: np.ndarray) -> None:
        data = np.ascontiguousarray(data, dtype=np.uint8)
        assert data.size == self.nbytes
        if self.tensor is not None:
            self.tensor[: self.nbytes].copy_(torch.from_numpy(data))
        else:
            torch.cuda.synchronize()
            ctypes.memmove(self.ptr, data.ctypes.data, self.nbytes)

    def zero(self) -> None:
        self.write(np.zeros(self.nbytes, dtype=np.uint8))


class Harness:
    def __init__(self, chunk: int, lineage: int = 5, **cfg):
        self.S = chunk
        self.cfg = C.crac_config_default(chunk_bytes=chunk, lineage=lineage, **cfg)
        self.ctx = C.crac_ctx_create(self.cfg)
        self.oracle = O.OracleContext(chunk, lineage=lineage,
                                      coded=bool(cfg.get("flags", 0) & C.CRAC_FLAG_COMPRESS))
        self.bufs: list[Buf] = []
        self.images: list[int] = []
        self.stream = torch.cuda.current_stream()
        self._managed: list[int] = []

    # -- registry --------------------------------------------------------------
    def add(self, nbytes: int, kind: int = C.CRAC_KIND_DEVICE, data: np.ndarray | None = None,
            seed: int = 1) -> Buf:
        if kind == C.CRAC_KIND_DEVICE:
            b = Buf(nbytes, kind, tensor=torch.empty(nbytes, dtype=torch.uint8, device="cuda"))
        elif kind == C.CRAC_KIND_HOST:    # page-locked host memory (cudaHostAlloc)
            b = Buf(nbytes, kind, tensor=torch.empty(nbytes, dtype=torch.uint8, pin_memory=True))
        else:
            p = C.crac_alloc_managed(nbytes)
            self._managed.append(p)
            b = Buf(nbytes, kind, ptr=p)
        b.write(data if data is not None else W.host_contents("u32_xorshift", nbytes, seed))
        C.crac_ctx_register_alloc(self.ctx, b.ptr, nbytes, kind)
        self.oracle.register(b.ptr, nbytes, kind)
        self.bufs.append(b)
        return b

    def free(self, i: int) -> Buf:
        b = self.bufs.pop(i)
        C.crac_ctx_free(self.ctx, b.ptr)
        self.oracle.free(b.ptr)
        return b

    def host(self) -> list:
        return [b.read() for b in self.bufs]

    def first(self) -> np.ndarray:
        return W.chunk_layout([b.nbytes for b in self.bufs], self.S)

    # -- the pass --------------------------------------------------------------
    def checkpoint(self, compare: bool = True):
        """(image handle, library bytes, oracle bytes)."""
        img = C.crac_ctx_checkpoint(self.ctx, self.stream)
        self.images.append(img)
        C.crac_image_wait(img)
        lib = C.crac_image_serialize(img)
        ora = self.oracle.checkpoint(self.host()) if compare else None
        return img, lib, ora

    def restart(self, img: int, chain_bytes: list | None = None) -> None:
        C.crac_ctx_restart(self.ctx, img, self.stream)
        torch.cuda.synchronize()
        if chain_bytes is not None:
            self.oracle.restart(chain_bytes)

    # -- mutations -------------------------------------------------------------
    def mutate(self, muts: list) -> None:
        """Apply workloads.ChunkMutation list (global chunk ids) on the device."""
        if not muts:
            return
        first = self.first()
        rows = []
        for m in muts:
            a = int(np.searchsorted(first, m.chunk, side="right") - 1)
            local = m.chunk - int(first[a])
            lo = local * self.S
            ln = min(self.S, self.bufs[a].nbytes - lo)
            rows.append((self.bufs[a].ptr + lo, ln, m.mask))
        arr = np.zeros((len(rows), 3), dtype=np.uint64)
        for i, (p, ln, mk) in enumerate(rows):
            arr[i] = (p, ln, mk)
        dev = torch.from_numpy(arr.view(np.int64)).to("cuda")
        testkit.mutate_xor(dev.data_ptr(), len(rows), self.stream)
        torch.cuda.synchronize()

    def close(self) -> None:
        torch.cuda.synchronize()
        for img in self.images:
            C.crac_image_release(img)
        self.images = []
        C.crac_ctx_destroy(self.ctx)
        for p in self._managed:
            C.crac_free_managed(p)
        self._managed = []


def pattern_mutations(first: np.ndarray, sizes: list, S: int, pattern: str, seed: int = 3):
    """Chunk mutations for a named dirty pattern over the layout `first`."""
    n = int(first[-1])
    rng = W.XorShift64(seed)
    if pattern == "none":
        ids = []
    elif pattern == "all":
        ids = list(range(n))
    elif pattern == "first":
        ids = [int(first[a]) for a in range(len(sizes))]
    elif pattern == "last":
        ids = [int(first[a + 1]) - 1 for a in range(len(sizes))]
    elif pattern == "tail":
        ids = [int(first[a + 1]) - 1 for a in range(len(sizes)) if sizes[a] % S]
    elif pattern == "alternating":
        ids = list(range(0, n, 2))
    elif pattern == "random10":
        ids = W.choose_distinct(rng, n, max(1, n // 10))
    else:
        raise ValueError(pattern)
    return [W.ChunkMutation(c, rng.mask32()) for c in sorted(set(ids))]
