"""Pins for the oracle's CRZ1 chunk codec (oracle/crz.py) and its coded images.

The codec is this project's design (the paper's measurements run with
compression off, Sec. 4.4.1), so nothing in the paper fixes its bytes.  It
is pinned by hand-worked streams whose every byte follows from its
definition by inspection, by closed forms (zero and constant chunks, a
block that cannot shrink), by brute-force roundtrips over lengths and value
mixes, and by an image-level cross-check against the uncoded image of the
same memory.  A mistake in the byte rotation, the plane or unit order, the
bit-to-lane mapping, the header packing or padding, or the raw fallback
changes one of the fixed streams below.
"""
import struct

import numpy as np
import pytest

from oracle import crz
from oracle import oracle as O

F = 0xFFFFFFFF


def _u4(words):
    return struct.pack("<%dI" % len(words), *words)


def test_hand_worked_ramp_block():
    """One block with word i = i.  Byte 0 rotates to 2i (i < 128), the other
    bytes are 0: plane 0 has min 0 and width 8, planes 1-3 width 0.  Bit j of
    2(4l+q) is 0 for j = 0, bit 0 / bit 1 of q for j = 1 / 2, and bit j-3 of
    l for j >= 3."""
    w = np.arange(128, dtype="<u4")
    want = struct.pack("<Q", 8 << 32) + bytes(8)           # header + pad (nb odd)
    want += _u4([0, 0, 0, 0])                               # j = 0
    want += _u4([0, F, 0, F])                               # j = 1: q odd
    want += _u4([0, 0, F, F])                               # j = 2: q >= 2
    for pat in (0xAAAAAAAA, 0xCCCCCCCC, 0xF0F0F0F0, 0xFF00FF00, 0xFFFF0000):
        want += _u4([pat] * 4)                              # j = 3..7: bits of l
    got = crz.encode(w.view(np.uint8))
    assert got == want and len(got) == 144
    assert crz.decode(got, 512) == w.tobytes()


def test_sign_rotation_pin():
    """+1.0f = 3F 80 00 00 and -1.0f = BF 80 00 00: rotated, the top bytes are
    0x7E / 0x7F (width 1), the 0x80 bytes all 0x01 (width 0).  Without the
    rotation plane 3 would hold 0x3F and 0xBF and need all 8 bits."""
    neg = [(i % 3) == 0 for i in range(128)]
    f = np.array([-1.0 if n else 1.0 for n in neg], dtype="<f4")
    h = (0x01 << 16) | (0x7E << 24) | (1 << (32 + 12))
    words = [0, 0, 0, 0]
    for l in range(32):
        for q in range(4):
            if neg[4 * l + q]:
                words[q] |= 1 << l
    want = struct.pack("<Q", h) + bytes(8) + _u4(words)
    got = crz.encode(f.view(np.uint8))
    assert got == want
    assert crz.decode(got, 512) == f.tobytes()


def test_unit_order_is_plane_then_bit():
    """Word i = i | (i % 2) << 16: plane 0 as in the ramp block, plane 2 takes
    values {0, 2} (width 2).  Its two units follow plane 0's eight."""
    i = np.arange(128, dtype=np.uint32)
    w = (i | ((i % 2) << 16)).astype("<u4")
    got = crz.encode(w.view(np.uint8))
    assert got[:16] == struct.pack("<Q", (8 << 32) | (2 << 40)) + bytes(8)
    units = [got[16 + 16 * u:32 + 16 * u] for u in range(10)]
    assert units[1] == _u4([0, F, 0, F])                    # plane 0, j = 1
    assert units[8] == _u4([0, 0, 0, 0])                    # plane 2, j = 0
    assert units[9] == _u4([0, F, 0, F])                    # plane 2, j = 1: q odd
    assert len(got) == 16 + 160


@pytest.mark.parametrize("nb", [1, 2, 3, 128])
@pytest.mark.parametrize("tail", [0, 5])
def test_zero_and_constant_chunks(nb, tail):
    """Zero chunk: one zero header word per block, padded to 16 bytes, then the
    tail.  Constant byte c: every plane has min rot(c) and width 0."""
    L = 512 * nb + tail
    z = crz.encode(np.zeros(L, np.uint8))
    assert z == bytes(16 * (-(-nb // 2)) + tail)
    c = 0xA5                                                # rot(0xA5) = 0x4B
    zc = crz.encode(np.full(L, c, np.uint8))
    h = struct.pack("<Q", 0x4B4B4B4B)
    assert zc == h * nb + bytes(8 * (nb % 2)) + bytes([c]) * tail
    assert crz.decode(zc, L) == bytes([c]) * L


def test_block_that_cannot_shrink_is_raw():
    """Every plane spans 0..255 after rotation (width 8): the coded stream would
    be 16 + 512 bytes > 512, so the chunk is stored as itself."""
    r = np.zeros(128, dtype=np.uint32)
    r[1] = 0xFFFFFFFF                                       # rot of 0xFF is 0xFF
    a = r.astype("<u4").view(np.uint8)
    assert crz.encode(a) == a.tobytes()
    rng = np.random.default_rng(3)
    for L in (1, 100, 511, 4096, 65536 + 3):                # short chunks are always raw
        b = rng.integers(0, 256, L, dtype=np.uint8)
        assert crz.encode(b) == b.tobytes()


def _brute_widths(chunk):
    """Widths per block and plane, with Python integers only."""
    out = []
    for b in range(len(chunk) // 512):
        vals = [[] for _ in range(4)]
        for i in range(128):
            w = int.from_bytes(chunk[512 * b + 4 * i:512 * b + 4 * i + 4], "little")
            for p in range(4):
                byte = (w >> (8 * p)) & 0xFF
                vals[p].append(((byte << 1) | (byte >> 7)) & 0xFF)
        out.append([(max(v) - min(v)).bit_length() for v in vals])
    return out


@pytest.mark.parametrize("kind", ["f32", "bf16", "ints", "sparse"])
def test_length_follows_widths(kind):
    """Coded length = 16 ceil(nb/2) + 16 sum(widths) + tail, widths computed
    byte by byte with Python integers."""
    rng = np.random.default_rng(7)
    L = 512 * 5 + 37
    if kind == "f32":
        a = rng.standard_normal(L // 4 + 1).astype("<f4").view(np.uint8)[:L]
    elif kind == "bf16":
        a = (rng.standard_normal(L // 2 + 1).astype("<f4").view("<u4") >> 16).astype("<u2").view(np.uint8)[:L]
    elif kind == "ints":
        a = rng.integers(-40, 40, L // 8 + 1).astype("<i8").view(np.uint8)[:L]
    else:
        a = np.zeros(L, np.uint8)
        a[rng.integers(0, L, 30)] = rng.integers(1, 256, 30)
    a = bytes(a)
    W = _brute_widths(a)
    zc = 16 * 3 + 16 * sum(map(sum, W)) + 37
    got = crz.encode(np.frombuffer(a, np.uint8))
    assert len(got) == (zc if zc < L else L)
    assert crz.decode(got, L) == a


@pytest.mark.parametrize("L", [1, 15, 511, 512, 513, 1024, 4096 + 7, 65536, 65536 - 13])
def test_roundtrip(L):
    rng = np.random.default_rng(L)
    mixes = [np.zeros(L, np.uint8), rng.integers(0, 256, L, dtype=np.uint8),
             rng.standard_normal(L // 4 + 1).astype("<f4").view(np.uint8)[:L],
             (rng.standard_normal(L // 2 + 1).astype("<f4").view("<u4") >> 16).astype("<u2").view(np.uint8)[:L],
             rng.integers(0, 3, L // 8 + 1).astype("<i8").view(np.uint8)[:L]]
    for a in mixes:
        z = crz.encode(a)
        assert len(z) <= L
        assert crz.decode(z, L) == a.tobytes()


def test_decoder_rejects_bad_streams():
    w = np.arange(128, dtype="<u4").view(np.uint8)
    z = bytearray(crz.encode(w))
    bad_width = bytearray(z)
    bad_width[4] = 9                                        # plane 0 width 9
    with pytest.raises(crz.CodecError):
        crz.decode(bytes(bad_width), 512)
    reserved = bytearray(z)
    reserved[7] = 1
    with pytest.raises(crz.CodecError):
        crz.decode(bytes(reserved), 512)
    with pytest.raises(crz.CodecError):
        crz.decode(bytes(z[:-16]), 512)                     # one unit short
    overflow = bytearray(z)
    overflow[0] = 0xF0                                      # min 240 + values up to 254
    with pytest.raises(crz.CodecError):
        crz.decode(bytes(overflow), 512)


def _mem(rng, sizes):
    out = []
    for i, n in enumerate(sizes):
        if i % 3 == 0:
            a = rng.standard_normal(n // 4 + 1).astype("<f4").view(np.uint8)[:n]
        elif i % 3 == 1:
            a = np.zeros(n, np.uint8)
        else:
            a = rng.integers(0, 256, n, dtype=np.uint8)
        out.append(np.ascontiguousarray(a))
    return out


def test_coded_image_matches_uncoded_image():
    """Same memory, same chain: the coded image has the uncoded one's header
    fields (but CODED and payload_bytes), fingerprints and chunk list, and
    each stream decodes to the uncoded image's chunk."""
    S = 4096
    rng = np.random.default_rng(11)
    sizes = [3 * S + 700, 2 * S, 5000, 512]
    mem = _mem(rng, sizes)
    plain, coded = O.OracleContext(S, lineage=3), O.OracleContext(S, lineage=3, coded=True)
    for i, n in enumerate(sizes):
        plain.register(0x10000 * (i + 1), n)
        coded.register(0x10000 * (i + 1), n)
    for step in range(3):
        if step:
            mem[0][5:9] ^= 0xFF
            mem[1][S + 1] ^= 1
        a, b = O.parse_image(plain.checkpoint(mem)), O.parse_image(coded.checkpoint(mem))
        assert b.coded and not a.coded and b.flags == a.flags | O.FLAG_CODED
        assert (a.epoch, a.parent_epoch, a.allocs, a.n_chunks) == (b.epoch, b.parent_epoch, b.allocs, b.n_chunks)
        assert np.array_equal(a.fp, b.fp) and np.array_equal(a.idx, b.idx)
        pa = pb = 0
        firsts = [t[4] for t in a.allocs]
        for e, c in enumerate(a.idx.tolist()):
            al = int(np.searchsorted(firsts, c, side="right") - 1)
            ln = O.chunk_len(a.allocs[al][2], c - firsts[al], S)
            zl = int(b.zlen[e])
            assert zl <= ln
            stream = bytes(b.payload[pb:pb + crz.padded(zl)])
            assert stream[zl:] == bytes(crz.padded(zl) - zl)    # zero padding
            assert crz.decode(stream[:zl], ln) == bytes(a.payload[pa:pa + ln])
            pa += ln
            pb += crz.padded(zl)
        assert pb == len(b.payload) and pa == len(a.payload)
        if step == 0:   # the zero allocation shrinks, the random one does not
            assert len(b.payload) < len(a.payload)


def test_coded_chain_restarts():
    S = 1024
    rng = np.random.default_rng(5)
    sizes = [7 * S + 100, 3000, 4 * S]
    mem = _mem(rng, sizes)
    ctx = O.OracleContext(S, lineage=9, coded=True)
    for i, n in enumerate(sizes):
        ctx.register(0x100000 * (i + 1), n)
    chain = [ctx.checkpoint(mem)]
    mem[2][:S] = 0
    mem[0][3 * S:3 * S + 64] ^= 0x5A
    chain.append(ctx.checkpoint(mem))
    want = [m.copy() for m in mem]
    got = _restart(sizes, S, chain)
    assert all(np.array_equal(g, w) for g, w in zip(got, want))
    # a damaged stream is reported, not restored
    img = bytearray(chain[0])
    im = O.parse_image(bytes(img))
    zl = im.zlen.tolist()
    coded_e = next(e for e, z in enumerate(zl) if z < O.chunk_len(sizes[0], e, S))
    off = len(img) - len(im.payload) + sum(crz.padded(int(z)) for z in zl[:coded_e])
    img[off + 4] = 12                                       # width 12
    with pytest.raises(O.Corrupt):
        _restart(sizes, S, [bytes(img)])


def _restart(sizes, S, chain):
    r = O.OracleContext(S, lineage=9, coded=True)
    for i, n in enumerate(sizes):
        r.register(0x100000 * (i + 1), n)
    return r.restart(chain)
