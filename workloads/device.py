"""Device-resident inputs of the benchmark configurations (torch + the test
mutators), shared by the GPU tests and the benchmark.

Like the rest of `workloads`, this holds input generators only: allocations,
their seeded contents, and the mutators that rewrite part of them between
checkpoints.  None of the method's arithmetic is here.  Contents come from
torch's CUDA generator (the oracle never regenerates them: it reads the
device bytes back).
"""
from __future__ import annotations

import numpy as np

from workloads import GIB, KIB, MIB, config2, config3, config4


class _RawDevice:
    """A device (or managed) address range seen through the CUDA array
    interface, so that torch can wrap memory it did not allocate."""

    def __init__(self, ptr: int, nbytes: int):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False),
                                         "version": 3, "strides": None}


def raw_tensor(ptr: int, nbytes: int):
    """uint8 tensor over nbytes of device or managed memory at ptr (no copy)."""
    import torch
    return torch.as_tensor(_RawDevice(ptr, nbytes), device="cuda")


def rows_tensor(rows, dev):
    """(ptr, ptr/len, len/mask) rows as the int64 device tensor the test
    mutators read."""
    import torch
    arr = np.asarray(rows, dtype=np.uint64).reshape(-1, 3)
    return torch.from_numpy(arr.view(np.int64)).to(dev)


def c2_memory(dev, total: int = 4 * GIB, n: int = 256):
    """Config 2: 256 allocations (log-uniform sizes water-filled to the
    total), fp32 N(0,1) contents.  Returns (workload, uint8 tensors)."""
    import torch
    wl = config2(total=total, n=n)
    g = torch.Generator(device=dev)
    g.manual_seed(wl.seed)
    bufs = []
    for nb in wl.sizes:
        t = torch.randn((nb + 3) // 4, generator=g, device=dev, dtype=torch.float32)
        bufs.append(t.view(torch.uint8)[:nb])
    return wl, bufs


class C3Memory:
    """Config 3: device allocations plus managed (UVM) ones, bf16 N(0,1)
    contents, and a mutator that rewrites 25% of the 64 KiB pages with bf16
    values on four streams (joined into the main stream afterwards, so that a
    checkpoint on the main stream is stream-synced)."""

    def __init__(self, dev, device_total: int = 12 * GIB, managed_total: int = 4 * GIB):
        import torch
        import paper_2008_10596_gb300 as C
        from paper_2008_10596_gb300 import testkit
        self.torch, self.C, self.testkit = torch, C, testkit
        self.dev = dev
        wl = config3(device_total=device_total // (64 * KIB) * (64 * KIB),
                     managed_total=managed_total // (64 * KIB) * (64 * KIB))
        self.wl = wl
        self.S = wl.chunk_bytes
        g = torch.Generator(device=dev)
        g.manual_seed(wl.seed)
        self.pool = torch.randn(64 << 20, generator=g, device=dev, dtype=torch.float32).to(torch.bfloat16)
        self.pool_u8 = self.pool.view(torch.uint8)   # 128 MiB of bf16 values
        self.tensors, self.kinds, self.managed = [], [], []
        self.ptrs, self.sizes = [], []
        for nb in wl.sizes:
            t = torch.empty(nb, dtype=torch.uint8, device=dev)
            self.tensors.append(t)
            self.ptrs.append(t.data_ptr())
            self.sizes.append(nb)
            self.kinds.append(C.CRAC_KIND_DEVICE)
        for nb in wl.managed_sizes:
            p = C.crac_alloc_managed(nb)
            self.managed.append(p)
            self.ptrs.append(p)
            self.sizes.append(nb)
            self.kinds.append(C.CRAC_KIND_MANAGED)
        rng = np.random.default_rng(wl.seed)
        rows = []
        for ptr, nb in zip(self.ptrs, self.sizes):   # initial contents: pool slices at random offsets
            for o in range(0, nb, 64 << 20):
                ln = min(64 << 20, nb - o)
                rows.append((ptr + o, self._pool_src(rng, ln), ln))
        e = rows_tensor(rows, dev)
        testkit.rewrite(e.data_ptr(), len(rows), torch.cuda.current_stream(dev))
        torch.cuda.synchronize(dev)
        self.pages = [(a, o) for a, nb in enumerate(self.sizes) for o in range(0, nb, self.S)]
        self.streams = [torch.cuda.Stream(dev) for _ in range(4)]

    def _pool_src(self, rng, ln):
        return self.pool_u8.data_ptr() + int(rng.integers(0, (self.pool_u8.numel() - ln) // 16 + 1)) * 16

    def mutate(self, seed: int) -> int:
        """Rewrite a seeded 25% of the pages on four streams; the main stream
        waits for all four."""
        torch = self.torch
        r = np.random.default_rng(seed)
        pick = r.choice(len(self.pages), size=len(self.pages) // 4, replace=False)
        rows = []
        for i in pick:
            a, o = self.pages[i]
            ln = min(self.S, self.sizes[a] - o)
            rows.append((self.ptrs[a] + o, self._pool_src(r, ln), ln))
        parts = np.array_split(np.asarray(rows, dtype=np.uint64), 4)
        ents = [torch.from_numpy(pp.view(np.int64)).to(self.dev) for pp in parts]
        torch.cuda.synchronize(self.dev)
        main = torch.cuda.current_stream(self.dev)
        for st, en, pp in zip(self.streams, ents, parts):
            self.testkit.rewrite(en.data_ptr(), len(pp), st)
        for st in self.streams:
            main.wait_stream(st)
        return len(rows)

    def copy_rows(self, dst_ptrs):
        """Rows copying every allocation to dst_ptrs (same sizes)."""
        return [(d, p, nb) for d, p, nb in zip(dst_ptrs, self.ptrs, self.sizes)]

    def free(self):
        self.torch.cuda.synchronize(self.dev)
        for p in self.managed:
            self.C.crac_free_managed(p)
        self.managed = []
        self.tensors = []


def c4_memory(total: int, n: int, dev):
    """Config-4-shaped device memory (Zipf sizes, uint8 / fp32 / int64
    contents cycling per allocation) and a mutator that rewrites a fraction of
    its 4 KiB pages (XOR with an odd mask, so every chosen page changes)."""
    import torch
    from paper_2008_10596_gb300 import testkit
    wl = config4(total=total, n=n)
    sizes = wl.sizes
    g = torch.Generator(device=dev)
    g.manual_seed(wl.seed)
    bufs = []
    for i, nb in enumerate(sizes):
        if i % 3 == 0:
            t = torch.randint(0, 256, (nb,), generator=g, device=dev, dtype=torch.uint8)
        elif i % 3 == 1:
            t = torch.randn(nb // 4, generator=g, device=dev, dtype=torch.float32).view(torch.uint8)
        else:
            t = torch.randint(-(1 << 62), 1 << 62, (nb // 8,), generator=g, device=dev,
                              dtype=torch.int64).view(torch.uint8)
        bufs.append(t)
    page_counts = torch.tensor([nb // 4096 for nb in sizes], device=dev, dtype=torch.int64)
    page_first = torch.cumsum(page_counts, 0) - page_counts
    bases = torch.tensor([b.data_ptr() for b in bufs], device=dev, dtype=torch.int64)
    n_pages = int(page_counts.sum().item())

    def mutate(frac, seed):
        k = int(round(frac * n_pages))
        if k == 0:
            return 0
        gg = torch.Generator(device=dev)
        gg.manual_seed(seed)
        pid = torch.randperm(n_pages, generator=gg, device=dev)[:k]
        a = torch.searchsorted(page_first, pid, right=True) - 1
        ptr = bases[a] + (pid - page_first[a]) * 4096
        mask = (torch.randint(0, 1 << 31, (k,), generator=gg, device=dev, dtype=torch.int64) * 2 + 1) & 0xFFFFFFFF
        ent = torch.stack([ptr, torch.full_like(ptr, 4096), mask], dim=1).contiguous()
        testkit.mutate_xor(ent.data_ptr(), k, torch.cuda.current_stream())
        torch.cuda.synchronize()
        return k

    return sizes, bufs, mutate


__all__ = ["raw_tensor", "rows_tensor", "c2_memory", "C3Memory", "c4_memory", "GIB", "KIB", "MIB"]
