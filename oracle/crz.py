"""CRZ1, the lossless chunk codec of coded images -- oracle side.

TEST INFRASTRUCTURE ONLY (see oracle.py): plain numpy, shares nothing with
the CUDA library.

The paper turns DMTCP's default gzip compression off for its checkpoint
measurements (Sec. 4.4.1, "Checkpoint overhead"), so the image it times is
uncompressed and the paper gives no codec.  CRZ1 is this project's own
design: a byte-plane frame-of-reference code that a GPU can write and read
at memory speed, aimed at what checkpointed device memory holds (floating-
point arrays, whose sign/exponent bytes take few values, and zero-filled
regions).  Definition, for one chunk of L bytes:

  1. nb = floor(L / 512) blocks of 512 bytes, then a tail of t = L - 512 nb
     bytes.
  2. Block b is read as 128 little-endian u32 words w_0 .. w_127.  Every
     byte of every word is rotated left by one bit:
        r(w) = ((w << 1) & 0xFEFEFEFE) | ((w >> 7) & 0x01010101)
     (the top bit of each byte -- a float's sign -- moves to the bottom, so
     small values of either sign land next to each other).
  3. Plane p (0..3) of the block holds the 128 bytes v_i = (r(w_i) >> 8p) &
     0xFF.  m_p = min_i v_i and W_p = the bit length of (max_i v_i - m_p),
     0..8.
  4. The block's header word is the u64
        h_b = sum_p m_p * 2^(8p)  +  sum_p W_p * 2^(32 + 4p).
  5. The block's plane data: for p = 0..3, for j = 0..W_p - 1, one 16-byte
     unit of four u32 words; word q (q = 0..3) has bit l (l = 0..31) equal
     to bit j of (v_(4l+q) - m_p).
  6. The coded stream is h_0 .. h_(nb-1), zero-padded to a multiple of 16
     bytes, then the plane data of blocks 0 .. nb-1 in order, then the t tail
     bytes unchanged.  Its length is
        z_c = 16 ceil(nb / 2) + 16 sum_b sum_p W_(b,p) + t.
  7. The chunk's stream is the coded stream if nb >= 1 and z_c < L, and
     otherwise the L bytes themselves ("raw").  Its length z therefore equals
     L exactly when the chunk is stored raw.

A coded image lists z for each chunk it holds (u64 zlen[k], after idx) and
its payload is the chunks' streams in idx order, each followed by zero bytes
up to a multiple of 16.
"""
from __future__ import annotations

import numpy as np

BLOCK = 512
_ROT_HI = np.uint32(0xFEFEFEFE)
_ROT_LO = np.uint32(0x01010101)


class CodecError(Exception):
    """A stream that no chunk of the given length encodes to."""


def _bit_length(d: np.ndarray) -> np.ndarray:
    """Bit length of each value in 0..255 (0 for 0)."""
    out = np.zeros(d.shape, dtype=np.int64)
    x = d.astype(np.int64)
    while np.any(x):
        out += x > 0
        x >>= 1
    return out


def rotate_bytes(w: np.ndarray) -> np.ndarray:
    """Step 2: every byte of each u32 rotated left by one bit."""
    w = w.astype(np.uint32)
    return ((w << np.uint32(1)) & _ROT_HI) | ((w >> np.uint32(7)) & _ROT_LO)


def unrotate_bytes(r: np.ndarray) -> np.ndarray:
    """Inverse of rotate_bytes: every byte rotated right by one bit."""
    r = r.astype(np.uint32)
    return ((r >> np.uint32(1)) & np.uint32(0x7F7F7F7F)) | ((r << np.uint32(7)) & np.uint32(0x80808080))


def coded_length(L: int, widths: np.ndarray) -> int:
    """Step 6: z_c for a chunk of L bytes whose blocks have these widths (nb x 4)."""
    nb = L // BLOCK
    return 16 * (-(-nb // 2)) + 16 * int(np.asarray(widths).sum()) + (L - BLOCK * nb)


def planes(chunk: np.ndarray):
    """Steps 1-3: per block the plane bytes v (nb x 4 x 128), minima and widths (nb x 4)."""
    a = np.ascontiguousarray(chunk, dtype=np.uint8).reshape(-1)
    nb = a.size // BLOCK
    w = a[:BLOCK * nb].view("<u4").reshape(nb, 128)
    r = rotate_bytes(w)
    v = np.stack([(r >> np.uint32(8 * p)) & np.uint32(0xFF) for p in range(4)], axis=1)
    m = v.min(axis=2)
    W = _bit_length(v.max(axis=2) - m)
    return v, m, W


def encode(chunk) -> bytes:
    """The chunk's stream (step 7): coded when that is shorter, else raw."""
    a = np.ascontiguousarray(np.frombuffer(bytes(chunk), dtype=np.uint8)
                             if not isinstance(chunk, np.ndarray) else chunk, dtype=np.uint8).reshape(-1)
    L = a.size
    nb = L // BLOCK
    if nb == 0:
        return a.tobytes()
    v, m, W = planes(a)
    if coded_length(L, W) >= L:
        return a.tobytes()
    # Step 4: header words.
    h = np.zeros(nb, dtype=np.uint64)
    for p in range(4):
        h |= m[:, p].astype(np.uint64) << np.uint64(8 * p)
        h |= W[:, p].astype(np.uint64) << np.uint64(32 + 4 * p)
    head = h.astype("<u8").tobytes()
    if nb % 2:
        head += bytes(8)
    # Step 5: unit (b, p, j) word q, bit l = bit j of (v[b, p, 4l + q] - m[b, p]),
    # for every j < 8; the units with j < W[b, p] are kept in (b, p, j) order.
    d = (v - m[:, :, None]).astype(np.uint32)                                  # nb, 4, 128
    bits = (d[:, :, None, :] >> np.arange(8, dtype=np.uint32)[None, None, :, None]) & np.uint32(1)
    bits = bits.reshape(nb, 4, 8, 32, 4)                                       # [.., l, q]
    words = (bits << np.arange(32, dtype=np.uint32)[None, None, None, :, None]).sum(axis=3, dtype=np.uint64)
    keep = np.arange(8)[None, None, :] < W[:, :, None]                         # nb, 4, 8
    units = words.astype(np.uint32)[keep]                                      # U, 4
    return head + units.astype("<u4").tobytes() + a[BLOCK * nb:].tobytes()


def decode(stream, L: int) -> bytes:
    """The L bytes of the chunk whose stream this is (inverse of encode)."""
    s = bytes(stream)
    z = len(s)
    if z == L:
        return s
    nb = L // BLOCK
    t = L - BLOCK * nb
    if z > L or nb == 0 or z < 16 * (-(-nb // 2)):
        raise CodecError("stream length impossible for this chunk length")
    h = np.frombuffer(s[:8 * nb], dtype="<u8").astype(np.uint64)
    if np.any(h >> np.uint64(48)):
        raise CodecError("reserved header bits set")
    m = np.stack([((h >> np.uint64(8 * p)) & np.uint64(0xFF)).astype(np.int64) for p in range(4)], axis=1)
    W = np.stack([((h >> np.uint64(32 + 4 * p)) & np.uint64(0xF)).astype(np.int64) for p in range(4)], axis=1)
    if np.any(W > 8):
        raise CodecError("plane width above 8")
    if coded_length(L, W) != z or z >= L:
        raise CodecError("stream length does not match its headers")
    head = 16 * (-(-nb // 2))
    units = np.frombuffer(s[head:head + 16 * int(W.sum())], dtype="<u4").reshape(-1, 4)
    # Unit u belongs to (block, plane) bp[u] and carries bit j[u] of its values.
    Wf = W.reshape(-1)
    bp = np.repeat(np.arange(nb * 4), Wf)
    j = np.arange(int(Wf.sum())) - np.repeat(np.cumsum(Wf) - Wf, Wf)
    # value index i = 4l + q takes bit l of word q
    bit = (units[:, None, :].astype(np.uint64) >> np.arange(32, dtype=np.uint64)[None, :, None]) & np.uint64(1)
    contrib = bit.reshape(-1, 128).astype(np.int64) << j[:, None]
    v = m.reshape(-1)[:, None].repeat(128, axis=1).astype(np.int64)      # nb*4, 128
    np.add.at(v, bp, contrib)
    v = v.reshape(nb, 4, 128)
    if np.any(v > 255):
        raise CodecError("plane value above 255")
    r = np.zeros((nb, 128), dtype=np.uint32)
    for p in range(4):
        r |= v[:, p, :].astype(np.uint32) << np.uint32(8 * p)
    w = unrotate_bytes(r)
    return w.astype("<u4").tobytes() + s[z - t:]


def padded(z: int) -> int:
    """Stream length rounded up to the 16-byte payload alignment."""
    return (z + 15) // 16 * 16
