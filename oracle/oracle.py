"""CPU oracle for the device data pass of CRAC-style checkpoint-restart.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
benchmark's CPU-baseline / reference leg import this module.  It shares no
code with the CUDA library and never calls it: it works on plain host byte
arrays that the caller copied out of device memory.

What it computes, in the paper's terms:
  * Checkpoint saves the memory of the *active* allocations only -- those
    made by the cudaMalloc family and not yet freed (Sec. 3.2, "Saving the
    library-allocated arena"), in the order they were allocated (Sec. 3.1,
    log-and-replay restores regions "in the same order as when they were
    allocated").  Device (cudaMalloc), unified (cudaMallocManaged) and
    page-locked host (cudaMallocHost / cudaHostAlloc) regions are all
    saved (Sec. 3.2, "restoring the CUDA library-allocated regions"); the
    kind is recorded with each allocation.
  * Restart copies the saved bytes back into the allocations (same
    subsection), after which the device state equals the checkpointed one.
  * Before the copy, pending device work is drained (Sec. 2.2, CheCUDA
    step (a)); here the caller hands in bytes that already reflect it.

The incremental part is this project's design, not the paper's (the paper
copies every active allocation at every checkpoint): memory is cut into
fixed-size chunks, each chunk gets a CRAC-FP64 fingerprint, and an image
carries only the chunks whose fingerprint differs from the previous
checkpoint's.  The steps below follow that definition in order, with numpy
primitives for the bulk steps (nonzero, cumsum, concatenation).

Image byte layout (all integers little-endian):
  header, 80 bytes:
    0  magic "CRACIMG1"      8  u32 version (1)     12 u32 flags (bit0 FULL)
    16 u32 chunk_bytes       20 u32 hash_id (1)     24 u64 lineage
    32 u64 epoch             40 u64 parent_epoch (all ones if none)
    48 u64 n_allocs          56 u64 n_chunks        64 u64 k (chunks present)
    72 u64 payload_bytes
  alloc table: n_allocs x 40 bytes
    u64 id, u64 orig_ptr, u64 bytes, u32 kind, u32 zero, u64 first_chunk
  u64 fp[n_chunks]          fingerprints of every chunk at this epoch
  u64 idx[k]                ascending global ids of the chunks present
  payload                   those chunks' bytes, concatenated, tails unpadded
A coded image (flags bit1 CODED, chosen per context) stores each chunk as
its CRZ1 stream (crz.py): u64 zlen[k] follows idx, and the payload is the
streams in idx order, each zero-padded to a multiple of 16 bytes.
"""
from __future__ import annotations

import ctypes
import os
import struct
from dataclasses import dataclass

import numpy as np

from oracle import crz

MAGIC = b"CRACIMG1"
VERSION = 1
HASH_ID = 1
FLAG_FULL = 1
FLAG_CODED = 2
NO_PARENT = (1 << 64) - 1
KIND_DEVICE = 0
KIND_MANAGED = 1
KIND_HOST = 2     # page-locked host memory (Sec. 3.2 lists cudaMallocHost / cudaHostAlloc)

HEADER = struct.Struct("<8sIIIIQQQQQQQ")
ALLOC = struct.Struct("<QQQIIQ")
assert HEADER.size == 80 and ALLOC.size == 40


class OracleError(Exception):
    code = "ERROR"


class InvalidArg(OracleError):
    code = "INVALID_ARG"


class Overlap(OracleError):
    code = "OVERLAP"


class UnknownPtr(OracleError):
    code = "UNKNOWN_PTR"


class ImageMismatch(OracleError):
    code = "IMAGE_MISMATCH"


class Corrupt(OracleError):
    code = "CORRUPT"


# ---------------------------------------------------------------------------
# Fingerprints through the plain C transcription (crac_fp.c)
# ---------------------------------------------------------------------------

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_lib", "liboracle_fp.so")
_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            from oracle import build as _b
            _b.build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.oracle_fp64.restype = ctypes.c_uint64
        lib.oracle_fp64.argtypes = [ctypes.c_void_p, ctypes.c_uint64]
        lib.oracle_fp_chunks.restype = None
        lib.oracle_fp_chunks.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64,
                                         ctypes.c_void_p]
        _lib = lib
    return _lib


def fp64(chunk) -> int:
    """CRAC-FP64 of one chunk (bytes-like or uint8 array, length >= 1)."""
    a = np.ascontiguousarray(np.frombuffer(bytes(chunk), dtype=np.uint8)
                             if not isinstance(chunk, np.ndarray) else chunk, dtype=np.uint8)
    if a.size == 0:
        raise InvalidArg("empty chunk")
    return int(_load().oracle_fp64(a.ctypes.data, a.size))


def fp_chunks(buf: np.ndarray, chunk_bytes: int, workers: int = 1) -> np.ndarray:
    """Fingerprints of every chunk of one allocation's bytes.

    Chunks are independent, so with workers > 1 the chunk list is cut into
    that many contiguous runs of whole chunks and each run goes through the
    same C loop on its own thread (the C call releases the GIL); the result
    is the same array."""
    a = np.ascontiguousarray(buf, dtype=np.uint8)
    n = -(-a.size // chunk_bytes)
    out = np.empty(n, dtype=np.uint64)
    if n == 0:
        return out
    lib = _load()
    workers = max(1, min(int(workers), n))
    if workers == 1:
        lib.oracle_fp_chunks(a.ctypes.data, a.size, chunk_bytes, out.ctypes.data)
        return out
    bounds = [n * w // workers for w in range(workers + 1)]

    def run(w):
        c0, c1 = bounds[w], bounds[w + 1]
        lo, hi = c0 * chunk_bytes, min(c1 * chunk_bytes, a.size)
        if c1 > c0:
            lib.oracle_fp_chunks(a.ctypes.data + lo, hi - lo, chunk_bytes, out.ctypes.data + 8 * c0)

    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(workers) as ex:
        list(ex.map(run, range(workers)))
    return out


# ---------------------------------------------------------------------------
# Image parsing
# ---------------------------------------------------------------------------

@dataclass
class Image:
    flags: int
    chunk_bytes: int
    lineage: int
    epoch: int
    parent_epoch: int
    allocs: list            # list of (id, orig_ptr, bytes, kind, first_chunk)
    n_chunks: int
    fp: np.ndarray
    idx: np.ndarray
    payload: memoryview
    zlen: np.ndarray | None = None   # coded images: stream length of each chunk

    @property
    def full(self) -> bool:
        return bool(self.flags & FLAG_FULL)

    @property
    def k(self) -> int:
        return int(self.idx.size)

    @property
    def coded(self) -> bool:
        return bool(self.flags & FLAG_CODED)


def parse_image(buf: bytes) -> Image:
    mv = memoryview(bytes(buf))
    if len(mv) < HEADER.size:
        raise Corrupt("truncated header")
    (magic, version, flags, chunk, hash_id, lineage, epoch, parent, n_allocs, n_chunks, k,
     payload_bytes) = HEADER.unpack_from(mv, 0)
    if magic != MAGIC or version != VERSION or hash_id != HASH_ID:
        raise Corrupt("bad magic/version/hash id")
    coded = bool(flags & FLAG_CODED)
    need = HEADER.size + ALLOC.size * n_allocs + 8 * n_chunks + 8 * k * (2 if coded else 1) + payload_bytes
    if len(mv) != need:
        raise Corrupt(f"size {len(mv)} != {need}")
    allocs = []
    o = HEADER.size
    for _ in range(n_allocs):
        aid, ptr, nbytes, kind, _z, first = ALLOC.unpack_from(mv, o)
        allocs.append((aid, ptr, nbytes, kind, first))
        o += ALLOC.size
    fp = np.frombuffer(mv[o:o + 8 * n_chunks], dtype="<u8").astype(np.uint64)
    o += 8 * n_chunks
    idx = np.frombuffer(mv[o:o + 8 * k], dtype="<u8").astype(np.uint64)
    o += 8 * k
    zlen = None
    if coded:
        zlen = np.frombuffer(mv[o:o + 8 * k], dtype="<u8").astype(np.uint64)
        o += 8 * k
    return Image(flags, chunk, lineage, epoch, parent, allocs, n_chunks, fp, idx,
                 mv[o:o + payload_bytes], zlen)


def chunk_len(alloc_bytes: int, local: int, chunk_bytes: int) -> int:
    return min(chunk_bytes, alloc_bytes - local * chunk_bytes)


# ---------------------------------------------------------------------------
# The context: registry + fingerprint baseline + checkpoint/restart
# ---------------------------------------------------------------------------

@dataclass
class _Alloc:
    id: int
    ptr: int
    bytes: int
    kind: int


class OracleContext:
    """One simulated process: its active-allocation table and last fingerprints."""

    def __init__(self, chunk_bytes: int, lineage: int = 1, coded: bool = False, workers: int = 1):
        if chunk_bytes < 16 or chunk_bytes & (chunk_bytes - 1):
            raise InvalidArg("chunk_bytes must be a power of two >= 16")
        self.S = int(chunk_bytes)
        self.workers = int(workers)   # threads for the per-chunk fingerprint loop
        self.coded = bool(coded)   # images store CRZ1 streams (crz.py)
        self.lineage = int(lineage)
        self.allocs: list[_Alloc] = []
        self.next_id = 0
        self.fp_valid: dict[int, np.ndarray] = {}   # alloc id -> previous fingerprints
        self.epoch = 0                               # highest epoch seen
        self.last_epoch = NO_PARENT                  # parent for the next image

    # -- registry (the cudaMalloc-family log of active mallocs, Sec. 3.2) ---
    def register(self, ptr: int, nbytes: int, kind: int = KIND_DEVICE) -> int:
        if nbytes <= 0 or ptr == 0 or ptr % 16 or kind not in (KIND_DEVICE, KIND_MANAGED, KIND_HOST):
            raise InvalidArg("bad registration")
        for a in self.allocs:
            if ptr < a.ptr + a.bytes and a.ptr < ptr + nbytes:
                raise Overlap("overlapping registration")
        aid = self.next_id
        self.next_id += 1
        self.allocs.append(_Alloc(aid, int(ptr), int(nbytes), int(kind)))
        return aid

    def free(self, ptr: int) -> None:
        for i, a in enumerate(self.allocs):
            if a.ptr == ptr:
                del self.allocs[i]
                self.fp_valid.pop(a.id, None)
                return
        raise UnknownPtr("pointer not registered")

    def layout(self) -> np.ndarray:
        counts = [-(-a.bytes // self.S) for a in self.allocs]
        return np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)

    # -- checkpoint -------------------------------------------------------
    def checkpoint(self, contents: list) -> bytes:
        """Image of the active allocations; contents[i] = bytes of allocs[i]."""
        if len(contents) != len(self.allocs):
            raise InvalidArg("one content buffer per registered allocation")
        fps, idxs, zlens, pieces = [], [], [], []

        def keep(i, fa, ids, chunk_pieces, zlen):
            fps.append(fa)
            idxs.append(ids)
            pieces.extend(chunk_pieces)
            if zlen is not None:
                zlens.append(zlen)

        head = self.checkpoint_by_alloc(lambda i: contents[i], keep)
        # 6: header and allocation table, fingerprints, chunk list, (stream
        # lengths), payload.
        out = [head, np.concatenate(fps + [np.empty(0, np.uint64)]).astype("<u8").tobytes(),
               np.concatenate(idxs + [np.empty(0, np.uint64)]).astype("<u8").tobytes()]
        if self.coded:
            out.append(np.concatenate(zlens + [np.empty(0, np.uint64)]).astype("<u8").tobytes())
        out.append(b"".join(pieces))
        return b"".join(out)

    def checkpoint_by_alloc(self, read, visit) -> bytes:
        """The checkpoint, one allocation at a time, in registration order.

        read(i) returns the bytes of allocs[i]; each allocation is read once.
        For each one, visit(i, fp, ids, pieces, zlen) receives its
        fingerprints, the global ids of its dirty chunks (ascending), those
        chunks' payload pieces in that order, and (coded images) their
        stream lengths, else None.  The image is the header and allocation
        table this method returns, followed by the concatenation over
        allocations of every fp, then of every ids, (then of every zlen),
        then of every piece; checkpoint() assembles exactly that.  The new
        baseline is committed only after the last allocation.
        """
        S = self.S
        first = self.layout()
        n = int(first[-1])
        fp_next = {}
        k = 0
        payload_bytes = 0
        for i, a in enumerate(self.allocs):
            buf = np.ascontiguousarray(np.asarray(read(i)).view(np.uint8).reshape(-1))
            if buf.size != a.bytes:
                raise InvalidArg("content size differs from registered size")
            # 1-3: fingerprint every chunk, compare with the previous table of
            # the same allocation id; an allocation with no valid table is all
            # dirty.
            fa = fp_chunks(buf, S, self.workers)
            prev = self.fp_valid.get(a.id)
            dirty = np.ones(fa.size, dtype=bool) if prev is None else (fa != prev)
            # 4: ascending dirty ids (global ids are consecutive across
            # allocations); byte offsets are the running sum of the chunks'
            # actual (unpadded) lengths.
            local = np.flatnonzero(dirty)
            ids = (int(first[i]) + local).astype(np.uint64)
            # 5: payload = dirty chunk bytes in id order (coded: their CRZ1
            # streams, each zero-padded to 16 bytes).
            chunk_pieces = [buf[c * S:c * S + chunk_len(a.bytes, c, S)].tobytes() for c in local.tolist()]
            zlen = None
            if self.coded:
                streams = [crz.encode(np.frombuffer(c, dtype=np.uint8)) for c in chunk_pieces]
                zlen = np.array([len(z) for z in streams], dtype=np.uint64)
                chunk_pieces = [z + bytes(crz.padded(len(z)) - len(z)) for z in streams]
            visit(i, fa, ids, chunk_pieces, zlen)
            fp_next[a.id] = fa
            k += int(local.size)
            payload_bytes += sum(len(c) for c in chunk_pieces)
        flags = (FLAG_FULL if k == n else 0) | (FLAG_CODED if self.coded else 0)
        epoch = self.epoch + 1
        # 6: header and allocation table.
        out = [HEADER.pack(MAGIC, VERSION, flags, S, HASH_ID, self.lineage, epoch,
                           self.last_epoch, len(self.allocs), n, k, payload_bytes)]
        for i, a in enumerate(self.allocs):
            out.append(ALLOC.pack(a.id, a.ptr, a.bytes, a.kind, 0, int(first[i])))
        # 7: commit the new baseline.
        self.fp_valid = fp_next
        self.epoch = epoch
        self.last_epoch = epoch
        return b"".join(out)

    def invalidate(self) -> None:
        """Forget the baseline: the next image holds every chunk (FULL)."""
        self.fp_valid = {}

    def set_chunk_bytes(self, chunk_bytes: int) -> None:
        """Switch to another chunk size.  The previous fingerprints describe
        other chunks, so they are dropped: the next image is FULL."""
        if chunk_bytes < 16 or chunk_bytes & (chunk_bytes - 1):
            raise InvalidArg("chunk_bytes must be a power of two >= 16")
        self.S = int(chunk_bytes)
        self.fp_valid = {}

    # -- restart ------------------------------------------------------------
    def restart(self, chain: list) -> list:
        """Bytes of every registered allocation after restoring chain[-1].

        chain runs from an image with the FULL flag to the target, each entry
        the parent of the next.  The registry must match the target's
        allocation table (count, sizes, kinds, order).  Images are applied
        oldest first; each chunk goes to the allocation with the same id in
        the target's table.
        """
        imgs = [parse_image(b) for b in chain]
        if not imgs or not imgs[0].full:
            raise ImageMismatch("chain must start at a FULL image")
        for p, c in zip(imgs, imgs[1:]):
            if c.parent_epoch != p.epoch or c.lineage != p.lineage or c.chunk_bytes != p.chunk_bytes:
                raise ImageMismatch("broken chain")
        tgt = imgs[-1]
        if tgt.chunk_bytes != self.S:
            raise ImageMismatch("chunk size differs")
        if len(tgt.allocs) != len(self.allocs):
            raise ImageMismatch("allocation count differs")
        for a, (_id, _p, nbytes, kind, _f) in zip(self.allocs, tgt.allocs):
            if a.bytes != nbytes or a.kind != kind:
                raise ImageMismatch("allocation size/kind differs")
        S = self.S
        pos_of_id = {t[0]: i for i, t in enumerate(tgt.allocs)}
        mem = [np.zeros(a.bytes, dtype=np.uint8) for a in self.allocs]
        covered = [np.zeros(-(-a.bytes // S), dtype=bool) for a in self.allocs]
        for img in imgs:
            firsts = np.array([t[4] for t in img.allocs] + [img.n_chunks], dtype=np.int64)
            off = 0
            for e, c in enumerate(img.idx.tolist()):
                a = int(np.searchsorted(firsts, c, side="right") - 1)
                aid, _p, nbytes, _k, first = img.allocs[a]
                local = c - first
                ln = chunk_len(nbytes, local, S)
                # coded: the stream's length, and the 16-byte padded step
                zl = int(img.zlen[e]) if img.coded else ln
                step = crz.padded(zl) if img.coded else ln
                if off + step > len(img.payload):
                    raise Corrupt("payload shorter than its chunk list")
                pos = pos_of_id.get(aid)
                if pos is not None:
                    raw = img.payload[off:off + zl]
                    if img.coded:
                        try:
                            raw = crz.decode(raw, ln)
                        except crz.CodecError as err:
                            raise Corrupt(str(err)) from err
                    mem[pos][local * S:local * S + ln] = np.frombuffer(raw, dtype=np.uint8)
                    covered[pos][local] = True
                off += step
            if off != len(img.payload):
                raise Corrupt("payload length does not match the chunk list")
        if not all(cv.all() for cv in covered):
            raise ImageMismatch("chain does not cover every chunk of the target")
        # Re-bind the registry to the image's allocation identities and adopt
        # its fingerprints as the baseline for the next checkpoint.
        for i, a in enumerate(self.allocs):
            a.id = tgt.allocs[i][0]
        self.next_id = max([self.next_id] + [t[0] + 1 for t in tgt.allocs])
        self.fp_valid = {}
        for i, a in enumerate(self.allocs):
            lo = tgt.allocs[i][4]
            self.fp_valid[a.id] = tgt.fp[lo:lo + -(-a.bytes // S)].copy()
        self.lineage = tgt.lineage
        self.epoch = max(self.epoch, tgt.epoch)
        self.last_epoch = tgt.epoch
        return mem
