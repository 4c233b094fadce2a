"""Pins for the oracle's checkpoint/restart semantics (CPU only).

Each test checks the oracle against something other than itself:
  * the paper's problem statement: restart(checkpoint(M)) == M for every
    active allocation, freed allocations are not saved, allocations keep
    their registration order (Sec. 3.1-3.2);
  * closed forms: a first (full) image's payload is the concatenation of the
    allocations' bytes; the payload length equals the sum of the listed
    chunks' lengths; the chunk count is the sum of ceil(bytes/S);
  * brute force: the dirty set of an incremental image equals the set of
    chunks whose bytes differ (byte comparison), which equals the set the
    test mutated; an unmodified re-checkpoint yields an empty delta.
"""
import struct

import numpy as np
import pytest

import workloads as W
from oracle import oracle as O

pytestmark = pytest.mark.usefixtures("oracle_lib")


def _mk(sizes, seed=1, kind="u32_xorshift"):
    return [W.host_contents(kind, s, seed + i) for i, s in enumerate(sizes)]


def _ctx(sizes, S, base_ptr=1 << 40):
    ctx = O.OracleContext(S, lineage=7)
    p = base_ptr
    for s in sizes:
        ctx.register(p, s, O.KIND_DEVICE)
        p += (s + 4095) // 4096 * 4096 + 4096
    return ctx


SIZES = [1, 7, 8, 4095, 4096, 4097, 3 * 4096 + 5, 20000]


def test_full_image_payload_is_concatenation():
    bufs = _mk(SIZES)
    ctx = _ctx(SIZES, 4096)
    img = O.parse_image(ctx.checkpoint(bufs))
    assert img.full and img.parent_epoch == O.NO_PARENT and img.epoch == 1
    assert bytes(img.payload) == b"".join(b.tobytes() for b in bufs)
    assert img.n_chunks == sum(-(-s // 4096) for s in SIZES)
    assert img.idx.tolist() == list(range(img.n_chunks))
    assert [a[2] for a in img.allocs] == SIZES
    assert [a[0] for a in img.allocs] == list(range(len(SIZES)))


def test_header_layout_fields():
    bufs = _mk([100])
    ctx = _ctx([100], 64)
    raw = ctx.checkpoint(bufs)
    assert raw[:8] == b"CRACIMG1"
    version, flags, chunk, hid = struct.unpack_from("<IIII", raw, 8)
    assert (version, flags, chunk, hid) == (1, 1, 64, 1)
    lineage, epoch, parent, na, nc, k, pb = struct.unpack_from("<7Q", raw, 24)
    assert (lineage, epoch, parent, na, nc, k, pb) == (7, 1, 2**64 - 1, 1, 2, 2, 100)
    assert len(raw) == 80 + 40 + 8 * 2 + 8 * 2 + 100


def test_unmodified_recheckpoint_is_empty_delta():
    bufs = _mk(SIZES)
    ctx = _ctx(SIZES, 4096)
    ctx.checkpoint(bufs)
    img = O.parse_image(ctx.checkpoint(bufs))
    assert img.k == 0 and len(img.payload) == 0 and not img.full
    assert img.parent_epoch == 1 and img.epoch == 2


@pytest.mark.parametrize("S", [64, 4096])
def test_delta_equals_bytewise_dirty_set(S):
    sizes = [5000, 70000, 4096 * 3, 1]
    bufs = _mk(sizes, seed=3)
    ctx = _ctx(sizes, S)
    ctx.checkpoint(bufs)
    first = W.chunk_layout(sizes, S)
    n = int(first[-1])
    muts = W.choose_mutations(99, n, 0.1)
    before = [b.copy() for b in bufs]
    W.apply_mutations_host(bufs, first, S, muts)
    img = O.parse_image(ctx.checkpoint(bufs))
    # brute force: byte comparison chunk by chunk
    byte_dirty = []
    for a, s in enumerate(sizes):
        for local in range(-(-s // S)):
            lo, hi = local * S, min(local * S + S, s)
            if not np.array_equal(before[a][lo:hi], bufs[a][lo:hi]):
                byte_dirty.append(int(first[a]) + local)
    assert img.idx.tolist() == byte_dirty == sorted(m.chunk for m in muts)
    # payload = concatenation of exactly those chunks' new bytes
    exp = b""
    for c in byte_dirty:
        a = int(np.searchsorted(first, c, side="right") - 1)
        local = c - int(first[a])
        exp += bufs[a][local * S:min(local * S + S, sizes[a])].tobytes()
    assert bytes(img.payload) == exp


def test_roundtrip_full_and_chain():
    sizes = [9000, 4096 * 4, 77]
    bufs = _mk(sizes, seed=5)
    ctx = _ctx(sizes, 1024)
    chain = [ctx.checkpoint(bufs)]
    states = [[b.copy() for b in bufs]]
    first = W.chunk_layout(sizes, 1024)
    for r in range(3):
        W.apply_mutations_host(bufs, first, 1024, W.choose_mutations(10 + r, int(first[-1]), 0.2))
        chain.append(ctx.checkpoint(bufs))
        states.append([b.copy() for b in bufs])
    for t in range(4):
        r2 = _ctx(sizes, 1024)
        got = r2.restart(chain[:t + 1])
        for g, e in zip(got, states[t]):
            assert np.array_equal(g, e)
        # After restart the baseline is the image: an unmodified checkpoint is empty.
        img = O.parse_image(r2.checkpoint(states[t]))
        assert img.k == 0 and img.parent_epoch == t + 1


def test_freed_allocation_vanishes_and_new_one_is_all_dirty():
    sizes = [4096, 8192, 100]
    bufs = _mk(sizes, seed=8)
    ctx = _ctx(sizes, 4096)
    ctx.checkpoint(bufs)
    ptr1 = ctx.allocs[1].ptr
    ctx.free(ptr1)
    newbuf = W.host_contents("u32_xorshift", 5000, 77)
    ctx.register(1 << 50, 5000, O.KIND_MANAGED)
    img = O.parse_image(ctx.checkpoint([bufs[0], bufs[2], newbuf]))
    assert [a[0] for a in img.allocs] == [0, 2, 3]
    assert [a[3] for a in img.allocs] == [0, 0, 1]
    # alloc 0 and 2 unchanged (no chunks); the new allocation is all dirty
    assert img.idx.tolist() == [2, 3]
    assert bytes(img.payload) == newbuf.tobytes()


def test_chain_across_register_and_free():
    sizes = [4096 * 2, 4096 * 3]
    bufs = _mk(sizes, seed=12)
    ctx = _ctx(sizes, 4096)
    i0 = ctx.checkpoint(bufs)
    ctx.free(ctx.allocs[0].ptr)
    extra = W.host_contents("u32_xorshift", 4096 + 3, 13)
    ctx.register(1 << 51, 4096 + 3, O.KIND_DEVICE)
    bufs2 = [bufs[1], extra]
    bufs2[0][:4] ^= 0xFF
    i1 = ctx.checkpoint(bufs2)
    r = O.OracleContext(4096, lineage=7)
    r.register(1 << 30, 4096 * 3)
    r.register(1 << 31, 4096 + 3)
    got = r.restart([i0, i1])
    assert np.array_equal(got[0], bufs2[0]) and np.array_equal(got[1], bufs2[1])
    assert [a.id for a in r.allocs] == [1, 2] and r.next_id == 3


def test_restart_mismatch_and_corruption():
    bufs = _mk([4096, 100])
    ctx = _ctx([4096, 100], 4096)
    raw = ctx.checkpoint(bufs)
    r = _ctx([4096, 101], 4096)
    with pytest.raises(O.ImageMismatch):
        r.restart([raw])
    r = _ctx([4096], 4096)
    with pytest.raises(O.ImageMismatch):
        r.restart([raw])
    with pytest.raises(O.Corrupt):
        O.parse_image(raw[:-1])
    bad = bytearray(raw)
    bad[0] ^= 1
    with pytest.raises(O.Corrupt):
        O.parse_image(bytes(bad))
    delta = ctx.checkpoint(bufs)
    with pytest.raises(O.ImageMismatch):
        _ctx([4096, 100], 4096).restart([delta])


def test_registry_errors():
    ctx = O.OracleContext(4096)
    ctx.register(4096, 100)
    with pytest.raises(O.Overlap):
        ctx.register(4096 + 64, 10)
    with pytest.raises(O.InvalidArg):
        ctx.register(1 << 20, 0)
    with pytest.raises(O.InvalidArg):
        ctx.register((1 << 20) + 8, 16)
    with pytest.raises(O.UnknownPtr):
        ctx.free(12345 * 16)
    ctx.register(4096 + 112, 16)   # adjacent, not overlapping
    ctx.free(4096)
    ctx.register(4096, 100)


def test_allocation_kinds_are_recorded():
    """Device, managed and page-locked host allocations (Sec. 3.2 lists
    cudaMalloc, cudaMallocManaged and cudaMallocHost / cudaHostAlloc) are
    saved alike; the image's allocation table records each one's kind, and
    a restart into a registry whose kinds differ is refused."""
    sizes = [100, 5000, 64]
    kinds = [O.KIND_HOST, O.KIND_DEVICE, O.KIND_MANAGED]
    ctx = O.OracleContext(4096, lineage=9)
    for i, (n, k) in enumerate(zip(sizes, kinds)):
        ctx.register((1 << 40) + i * 8192, n, k)
    bufs = _mk(sizes)
    raw = ctx.checkpoint(bufs)
    img = O.parse_image(raw)
    assert [a[3] for a in img.allocs] == kinds
    assert bytes(img.payload) == b"".join(b.tobytes() for b in bufs)
    other = O.OracleContext(4096, lineage=9)
    for i, n in enumerate(sizes):
        other.register((1 << 41) + i * 8192, n, O.KIND_DEVICE)
    with pytest.raises(O.ImageMismatch):
        other.restart([raw])
    with pytest.raises(O.InvalidArg):
        other.register(1 << 42, 16, 3)


def test_offsets_and_counts_invariants():
    sizes = [123457, 4096, 65536 + 17]
    bufs = _mk(sizes, seed=21)
    ctx = _ctx(sizes, 4096)
    ctx.checkpoint(bufs)
    first = W.chunk_layout(sizes, 4096)
    W.apply_mutations_host(bufs, first, 4096, W.choose_mutations(4, int(first[-1]), 0.3))
    img = O.parse_image(ctx.checkpoint(bufs))
    lens = []
    for c in img.idx.tolist():
        a = int(np.searchsorted(first, c, side="right") - 1)
        lens.append(O.chunk_len(sizes[a], c - int(first[a]), 4096))
    assert sum(lens) == len(img.payload)
    assert img.n_chunks == int(first[-1])
    assert np.all(np.diff(img.idx.astype(np.int64)) > 0)


def test_by_alloc_reads_each_allocation_once_and_commits_last():
    """checkpoint_by_alloc reads every allocation once, in registration
    order, and hands out per-allocation parts that line up with the image's
    sections; a failure part way leaves the baseline as it was (the next
    image is still a delta against the last committed one)."""
    sizes = [5000, 1, 4096 * 3, 777]
    S = 1024
    bufs = _mk(sizes, seed=11)
    ref = _ctx(sizes, S)
    ctx = _ctx(sizes, S)
    img0 = O.parse_image(ref.checkpoint(bufs))
    reads, parts = [], []
    head = ctx.checkpoint_by_alloc(lambda i: (reads.append(i), bufs[i])[1],
                                   lambda i, fa, ids, pcs, zl: parts.append((i, fa, ids, pcs, zl)))
    assert reads == list(range(len(sizes)))
    assert head == ref_head(img0, sizes, S)
    first = W.chunk_layout(sizes, S)
    assert np.concatenate([p[1] for p in parts]).tolist() == img0.fp.tolist()
    for i, fa, ids, pcs, zl in parts:
        assert fa.size == first[i + 1] - first[i] and zl is None
        assert ids.tolist() == list(range(int(first[i]), int(first[i + 1])))   # first image: every chunk
        assert b"".join(pcs) == bufs[i].tobytes()
    # mutate one chunk; fail while reading allocation 2: nothing committed
    bufs[3] = bufs[3].copy()
    bufs[3][5] ^= 1

    def bad(i):
        if i == 2:
            raise RuntimeError("read failed")
        return bufs[i]
    with pytest.raises(RuntimeError):
        ctx.checkpoint_by_alloc(bad, lambda *a: None)
    img1 = O.parse_image(ctx.checkpoint(bufs))
    assert img1.epoch == 2 and img1.parent_epoch == 1
    assert img1.idx.tolist() == [int(first[3])]


def ref_head(img, sizes, S):
    """Header and allocation table of a parsed image, re-packed field by field."""
    out = [O.HEADER.pack(O.MAGIC, 1, img.flags, S, 1, img.lineage, img.epoch, img.parent_epoch,
                         len(img.allocs), img.n_chunks, img.k, len(img.payload))]
    for a in img.allocs:
        out.append(O.ALLOC.pack(a[0], a[1], a[2], a[3], 0, a[4]))
    return b"".join(out)


def test_chunk_size_switch_makes_the_next_image_full():
    """After set_chunk_bytes the previous fingerprints describe other chunks:
    the next image holds every chunk (closed form: the concatenation of the
    allocations) at the new size, and the epoch chain continues."""
    sizes = [70000, 3000]
    bufs = _mk(sizes, seed=21)
    ctx = _ctx(sizes, 4096)
    ctx.checkpoint(bufs)
    ctx.set_chunk_bytes(65536)
    img = O.parse_image(ctx.checkpoint(bufs))
    assert img.full and img.chunk_bytes == 65536 and img.epoch == 2 and img.parent_epoch == 1
    assert img.n_chunks == 2 + 1
    assert bytes(img.payload) == b"".join(b.tobytes() for b in bufs)
    again = O.parse_image(ctx.checkpoint(bufs))
    assert again.k == 0


def test_invalidate_makes_the_next_image_full():
    """Without a baseline every chunk is saved again: the payload is the
    concatenation of the allocations (closed form), and the epoch chain
    continues from the last image."""
    sizes = [9000, 4096]
    bufs = _mk(sizes, seed=31)
    ctx = _ctx(sizes, 4096)
    ctx.checkpoint(bufs)
    assert O.parse_image(ctx.checkpoint(bufs)).k == 0
    ctx.invalidate()
    img = O.parse_image(ctx.checkpoint(bufs))
    assert img.full and img.epoch == 3 and img.parent_epoch == 2
    assert bytes(img.payload) == b"".join(b.tobytes() for b in bufs)
