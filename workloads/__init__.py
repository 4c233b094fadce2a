"""Seeded synthetic inputs for the checkpoint/restart data pass.

This module is the one piece both the CPU oracle's tests and the CUDA path's
tests share.  It holds input generators only: allocation size lists, buffer
contents, the choice of chunks a mutator rewrites, and the mutation masks.
It computes none of the method's arithmetic (no fingerprint, no dirty test,
no compaction, no image layout).

The workloads stand in for the applications the paper checkpoints (Rodinia,
LULESH, HPGMG-FV, HYPRE; Sec. 4, Tables 1-2): those programs and their
datasets are not available, so each configuration below reproduces the
shape of the work -- allocation count and size mix, total tracked bytes,
content type, and the fraction of memory rewritten between checkpoints.

Generators:
  * Marsaglia xorshift64 (shift triple 13, 7, 17; "Xorshift RNGs", J. Stat.
    Softw. 8(14), 2003).  One step per uint32, value = high 32 bits of the
    state after the step.  The sequence is produced in parallel lanes by
    jumping the state ahead with the step's 64x64 matrix over GF(2).
  * numpy's PCG64 Generator for size lists and normal/uniform contents.
  * torch's CUDA generator for full-size device-resident contents (the
    oracle never regenerates these; it reads the device bytes back).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

KIB = 1024
MIB = 1024 * KIB
GIB = 1024 * MIB

#: Config i uses seed SEED_BASE + i (configs numbered from 1).
SEED_BASE = 2008105960

_U64 = np.uint64
_MASK64 = (1 << 64) - 1


# ---------------------------------------------------------------------------
# xorshift64
# ---------------------------------------------------------------------------

def _xs_step(x: np.ndarray) -> np.ndarray:
    x = x ^ (x << _U64(13))
    x = x ^ (x >> _U64(7))
    x = x ^ (x << _U64(17))
    return x


def xorshift64_next(state: int) -> int:
    """One xorshift64 step on a Python int; returns the new state."""
    x = state & _MASK64
    x ^= (x << 13) & _MASK64
    x ^= x >> 7
    x ^= (x << 17) & _MASK64
    return x


def _jump_columns(steps: int) -> np.ndarray:
    """Columns of T^steps over GF(2): col[b] = T^steps(e_b)."""
    cols = np.array([1 << b for b in range(64)], dtype=_U64)
    for _ in range(steps):
        cols = _xs_step(cols)
    return cols


def _apply_cols(cols: np.ndarray, state: int) -> int:
    acc = 0
    b = 0
    s = state
    while s:
        if s & 1:
            acc ^= int(cols[b])
        s >>= 1
        b += 1
    return acc


def xorshift64_u32(seed: int, n: int, lane_steps: int = 1024) -> np.ndarray:
    """n uint32 values: value i = high 32 bits of the state after step i+1."""
    if seed & _MASK64 == 0:
        raise ValueError("xorshift64 seed must be non-zero")
    if n == 0:
        return np.zeros(0, dtype=np.uint32)
    m = max(1, min(lane_steps, n))
    lanes = -(-n // m)
    cols = _jump_columns(m)
    starts = np.empty(lanes, dtype=_U64)
    s = seed & _MASK64
    for lane in range(lanes):
        starts[lane] = s
        s = _apply_cols(cols, s)
    out = np.empty((m, lanes), dtype=np.uint32)
    x = starts
    for t in range(m):
        x = _xs_step(x)
        out[t] = (x >> _U64(32)).astype(np.uint32)
    return np.ascontiguousarray(out.T).reshape(-1)[:n]


class XorShift64:
    """Sequential xorshift64 stream for small draws (chunk choices, masks)."""

    def __init__(self, seed: int):
        if seed & _MASK64 == 0:
            raise ValueError("xorshift64 seed must be non-zero")
        self.state = seed & _MASK64

    def next64(self) -> int:
        self.state = xorshift64_next(self.state)
        return self.state

    def below(self, bound: int) -> int:
        return self.next64() % bound

    def mask32(self) -> int:
        """A non-zero uint32 XOR mask: high half of the next state, low bit set."""
        return ((self.next64() >> 32) | 1) & 0xFFFFFFFF


def choose_distinct(rng: XorShift64, n: int, k: int) -> list[int]:
    """k distinct indices of range(n) by a partial Fisher-Yates shuffle.

    Returned in draw order (not sorted).  Uses a sparse swap table so it
    runs in O(k) for any n.
    """
    if k > n:
        raise ValueError("k > n")
    swapped: dict[int, int] = {}
    out = []
    for i in range(k):
        j = i + rng.below(n - i)
        vi = swapped.get(i, i)
        vj = swapped.get(j, j)
        swapped[j] = vi
        swapped[i] = vj
        out.append(vj)
    return out


# ---------------------------------------------------------------------------
# Size lists
# ---------------------------------------------------------------------------

def log_uniform(rng: np.random.Generator, n: int, lo: float, hi: float) -> np.ndarray:
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=n))


def water_fill(raw: np.ndarray, total: int, lo: int, hi: int, align: int) -> np.ndarray:
    """Scale raw sizes by one factor f, clamped to [lo, hi], so they sum to total.

    The clamped sum is monotone in f, so f is found by bisection.  Sizes are
    then floored to `align`; the realized total is within len(raw)*align of
    the request.  Deterministic for a given raw vector.
    """
    raw = np.asarray(raw, dtype=np.float64)
    if lo * len(raw) > total or hi * len(raw) < total:
        raise ValueError("total not reachable under the clamp")

    def clamped_sum(f: float) -> float:
        return float(np.clip(raw * f, lo, hi).sum())

    f_lo, f_hi = 0.0, 1.0
    while clamped_sum(f_hi) < total:
        f_hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (f_lo + f_hi)
        if clamped_sum(mid) < total:
            f_lo = mid
        else:
            f_hi = mid
    sizes = np.clip(raw * f_hi, lo, hi)
    sizes = (np.floor(sizes / align) * align).astype(np.int64)
    return np.maximum(sizes, lo)


def zipf_truncated(rng: np.random.Generator, n: int, s: float, kmax: int) -> np.ndarray:
    """n draws of X ~ Zipf(s) truncated to [1, kmax] by inverse CDF."""
    k = np.arange(1, kmax + 1, dtype=np.float64)
    pmf = k ** (-s)
    cdf = np.cumsum(pmf)
    cdf /= cdf[-1]
    u = rng.uniform(0.0, 1.0, size=n)
    return np.searchsorted(cdf, u, side="left").astype(np.int64) + 1


# ---------------------------------------------------------------------------
# Workload configurations
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    seed: int
    chunk_bytes: int
    sizes: list[int]                      # device allocations, registration order
    managed_sizes: list[int] = field(default_factory=list)
    content: str = "u32_xorshift"         # u32_xorshift | f32_normal | mixed | bf16
    dirty_fraction: float = 0.0
    note: str = ""

    @property
    def total_bytes(self) -> int:
        return int(sum(self.sizes) + sum(self.managed_sizes))


def config1() -> Workload:
    """One 16 MiB buffer of xorshift64 uint32, 4 KiB chunks, 1% of chunks mutated."""
    return Workload(name="c1_16MiB_x1_4KiB", seed=SEED_BASE + 1, chunk_bytes=4 * KIB,
                    sizes=[16 * MIB], content="u32_xorshift", dirty_fraction=0.01)


def config2_sizes(seed: int = SEED_BASE + 2, n: int = 256, total: int = 4 * GIB) -> list[int]:
    rng = np.random.default_rng(seed)
    raw = log_uniform(rng, n, 4 * KIB, 64 * MIB)
    return [int(s) for s in water_fill(raw, total, 4 * KIB, 64 * MIB, 256)]


def config2(total: int = 4 * GIB, n: int = 256) -> Workload:
    """256 allocations, log-uniform 4 KiB-64 MiB rescaled to ~4 GiB, fp32 N(0,1), 64 KiB chunks."""
    return Workload(name=f"c2_{total // MIB}MiB_x{n}_64KiB", seed=SEED_BASE + 2,
                    chunk_bytes=64 * KIB, sizes=config2_sizes(total=total, n=n),
                    content="f32_normal", dirty_fraction=0.10)


def _draw_until(rng: np.random.Generator, total: int, lo: int, hi: int, align: int) -> list[int]:
    out: list[int] = []
    acc = 0
    while acc < total:
        s = int(log_uniform(rng, 1, lo, hi)[0]) // align * align
        s = max(s, lo)
        if acc + s > total:
            s = total - acc
        out.append(s)
        acc += s
    return out


def config3(device_total: int = 12 * GIB, managed_total: int = 4 * GIB) -> Workload:
    """Device + managed allocations, 64 KiB-512 MiB log-uniform, 25% of 64 KiB pages rewritten."""
    rng = np.random.default_rng(SEED_BASE + 3)
    dev = _draw_until(rng, device_total, 64 * KIB, 512 * MIB, 64 * KIB)
    man = _draw_until(rng, managed_total, 64 * KIB, 512 * MIB, 64 * KIB)
    return Workload(name=f"c3_{device_total // GIB}GiB_dev_{managed_total // GIB}GiB_managed",
                    seed=SEED_BASE + 3, chunk_bytes=64 * KIB, sizes=dev, managed_sizes=man,
                    content="bf16", dirty_fraction=0.25)


def config4(total: int = 120 * GIB, n: int = 2048) -> Workload:
    """2048 allocations, Zipf(1.1) sizes in 4 KiB units rescaled to 120 GiB, mixed contents."""
    rng = np.random.default_rng(SEED_BASE + 4)
    x = zipf_truncated(rng, n, 1.1, 1 << 20)
    sizes = water_fill(x.astype(np.float64) * 4 * KIB, total, 4 * KIB, 4 * GIB, 4 * KIB)
    return Workload(name=f"c4_{total // GIB}GiB_x{n}", seed=SEED_BASE + 4, chunk_bytes=64 * KIB,
                    sizes=[int(s) for s in sizes], content="mixed")


# ---------------------------------------------------------------------------
# Contents and mutations
# ---------------------------------------------------------------------------

def host_contents(kind: str, nbytes: int, seed: int) -> np.ndarray:
    """Host bytes (np.uint8, length nbytes) of the named content type."""
    if kind == "u32_xorshift":
        words = xorshift64_u32(seed, -(-nbytes // 4))
        return words.view(np.uint8)[:nbytes].copy()
    rng = np.random.default_rng(seed)
    if kind == "f32_normal":
        v = rng.standard_normal(-(-nbytes // 4), dtype=np.float32)
    elif kind == "u8":
        v = rng.integers(0, 256, size=nbytes, dtype=np.uint8)
    elif kind == "i64":
        v = rng.integers(-(1 << 63), (1 << 63) - 1, size=-(-nbytes // 8), dtype=np.int64)
    elif kind == "bf16":
        f = rng.standard_normal(-(-nbytes // 2), dtype=np.float32)
        v = f32_to_bf16_rne(f)
    else:
        raise ValueError(kind)
    return v.view(np.uint8)[:nbytes].copy()


def f32_to_bf16_rne(f: np.ndarray) -> np.ndarray:
    """fp32 -> bf16 bit patterns (uint16), round to nearest even (finite inputs)."""
    u = np.ascontiguousarray(f, dtype=np.float32).view(np.uint32).astype(np.uint64)
    rounding = ((u >> np.uint64(16)) & np.uint64(1)) + np.uint64(0x7FFF)
    return ((u + rounding) >> np.uint64(16)).astype(np.uint16)


@dataclass
class ChunkMutation:
    """XOR every uint32 of chunk `chunk` (global id) with `mask`."""
    chunk: int
    mask: int


def choose_mutations(seed: int, n_chunks: int, fraction: float) -> list[ChunkMutation]:
    """round(fraction*n_chunks) distinct chunks, each with a non-zero XOR mask."""
    k = int(round(fraction * n_chunks))
    rng = XorShift64(seed ^ 0xC4A5_0000_0000_0001)
    picks = choose_distinct(rng, n_chunks, k)
    return [ChunkMutation(c, rng.mask32()) for c in picks]


def chunk_layout(sizes: list[int], chunk_bytes: int) -> np.ndarray:
    """first-chunk offsets (len(sizes)+1) of allocations laid out in order."""
    counts = [-(-s // chunk_bytes) for s in sizes]
    return np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)


def apply_mutations_host(bufs: list[np.ndarray], first: np.ndarray, chunk_bytes: int,
                         muts: list[ChunkMutation]) -> None:
    """Apply chunk XOR mutations to host byte arrays in place.

    Only whole uint32 words are XORed; a trailing partial word (chunk length
    not a multiple of 4) gets its bytes XORed with the mask's low bytes.
    """
    for m in muts:
        a = int(np.searchsorted(first, m.chunk, side="right") - 1)
        local = m.chunk - int(first[a])
        lo = local * chunk_bytes
        hi = min(lo + chunk_bytes, len(bufs[a]))
        seg = bufs[a][lo:hi]
        nw = len(seg) // 4
        if nw:
            w = seg[: nw * 4].view(np.uint32)
            w ^= np.uint32(m.mask)
        for t in range(nw * 4, len(seg)):
            seg[t] ^= (m.mask >> (8 * (t % 4))) & 0xFF
