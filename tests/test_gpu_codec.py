"""Coded images (GPU): with CRAC_FLAG_COMPRESS every image must serialize to
the oracle's coded image byte for byte (stream lengths, streams, zero
padding), every restart must bring the memory back exactly, the GPU decoder
must restore images the oracle encoded (independent of the GPU encoder), and
a damaged stream must come back as CRAC_ERR_CORRUPT, not as a fault."""
import numpy as np
import torch
import pytest

import paper_2008_10596_gb300 as C
import workloads as W
from oracle import crz
from oracle import oracle as O
from tests.gpu_harness import Harness, pattern_mutations

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("oracle_lib")]

KIB = 1024
CODED = C.CRAC_FLAG_COMPRESS
KINDS = ["f32_normal", "zeros", "bf16", "u8", "i64_small"]


def _contents(kind, n, seed):
    if kind == "zeros":
        return np.zeros(n, np.uint8)
    if kind == "i64_small":
        rng = np.random.default_rng(seed)
        return rng.integers(-300, 300, -(-n // 8)).astype("<i8").view(np.uint8)[:n].copy()
    return W.host_contents(kind, n, seed)


def _sizes(S):
    # ragged tails, a size that is not a multiple of 16 (later staging offsets
    # become unaligned), chunks below one 512-byte block
    return [S * 30 + 48, 7 * 4096 + 1, S * 5, 100000, 513, 16, 3 * S + 600]


def _fill(h, S, seed=0):
    for i, n in enumerate(_sizes(S)):
        h.add(n, data=_contents(KINDS[i % len(KINDS)], n, seed + 10 * i + 1))


def _zero_some(h, every=3):
    for b in h.bufs[::every]:
        b.zero()


CASES = [
    (C.CRAC_RESIDENCY_HOST, C.CRAC_PASS_AUTO, 0),
    (C.CRAC_RESIDENCY_HOST, C.CRAC_PASS_SPLIT, C.CRAC_FLAG_DIRECT_DRAIN),
    (C.CRAC_RESIDENCY_HOST, C.CRAC_PASS_LDG, 0),
    (C.CRAC_RESIDENCY_HOST, C.CRAC_PASS_TMA, C.CRAC_FLAG_DIRECT_DRAIN),
    (C.CRAC_RESIDENCY_DEVICE, C.CRAC_PASS_SPLIT, 0),
    (C.CRAC_RESIDENCY_DEVICE, C.CRAC_PASS_TMA, C.CRAC_FLAG_INCREMENTAL_RESTORE),
    (C.CRAC_RESIDENCY_DEVICE, C.CRAC_PASS_AUTO, 0),
]


@pytest.mark.parametrize("S", [512, 4 * KIB, 64 * KIB, 256 * KIB])
@pytest.mark.parametrize("residency,kern,flags", CASES)
def test_coded_images_match_oracle(S, residency, kern, flags):
    if kern == C.CRAC_PASS_TMA and not (KIB <= S <= 64 * KIB):
        pytest.skip("TMA pass: 1-64 KiB chunks")
    h = Harness(S, lineage=1200 + S // 256 + kern, image_residency=residency, pass_kernel=kern,
                flags=flags | CODED)
    try:
        _fill(h, S, seed=S // 512)
        chain_lib, images, states = [], [], []
        img, lib, ora = h.checkpoint()
        assert lib == ora
        assert O.parse_image(lib).coded
        info = C.crac_image_info(img)
        assert info["flags"] & C.CRAC_IMAGE_CODED and info["serialized_bytes"] == len(lib)
        assert info["raw_bytes"] == sum(b.nbytes for b in h.bufs)
        chain_lib.append(lib)
        images.append(img)
        states.append(h.host())
        for step, pattern in enumerate(["random10", "zero", "alternating", "none"]):
            if pattern == "zero":
                _zero_some(h)
            else:
                h.mutate(pattern_mutations(h.first(), [b.nbytes for b in h.bufs], S, pattern, seed=step + 5))
            img, lib, ora = h.checkpoint()
            assert lib == ora, (step, pattern)
            pi = C.crac_ctx_last_pass(h.ctx)
            assert pi["stored_bytes"] == C.crac_image_info(img)["payload_bytes"]
            chain_lib.append(lib)
            images.append(img)
            states.append(h.host())
        # restart the second image after wiping memory, then the newest
        for target in (1, len(images) - 1):
            for b in h.bufs:
                b.zero()
            h.restart(images[target])
            for b, w in zip(h.bufs, states[target]):
                assert np.array_equal(b.read(), w), target
        # the oracle restores the same chain to the same bytes
        got = h.oracle.restart(chain_lib)
        assert all(np.array_equal(g, w) for g, w in zip(got, states[-1]))
    finally:
        h.close()


def test_codec_shrinks_what_it_should():
    """Ratio of stored to raw bytes per content kind on a full checkpoint."""
    S = 64 * KIB
    for kind, lo, hi in [("zeros", 0.0, 0.02), ("f32_normal", 0.85, 0.93), ("bf16", 0.72, 0.80),
                         ("u8", 1.0, 1.0)]:
        h = Harness(S, lineage=1300, flags=CODED)
        try:
            h.add(64 * S, data=_contents(kind, 64 * S, 3))
            img, lib, ora = h.checkpoint()
            assert lib == ora
            info = C.crac_image_info(img)
            ratio = info["payload_bytes"] / info["raw_bytes"]
            assert lo <= ratio <= hi, (kind, ratio)
        finally:
            h.close()


@pytest.mark.parametrize("residency", [C.CRAC_RESIDENCY_HOST, C.CRAC_RESIDENCY_DEVICE])
def test_oracle_encoded_images_restore_on_gpu(residency):
    """The GPU decoder restores a chain the oracle encoded, deserialized from
    its bytes (the GPU encoder is not involved)."""
    S = 4 * KIB
    sizes = _sizes(S)
    h = Harness(S, lineage=1400, image_residency=residency, flags=CODED)
    try:
        _fill(h, S, seed=77)
        mem0 = h.host()
        ora = O.OracleContext(S, lineage=4242, coded=True)
        for b in h.bufs:
            ora.register(b.ptr, b.nbytes, b.kind)
        chain = [ora.checkpoint(mem0)]
        mem1 = [m.copy() for m in mem0]
        mem1[0][: 3 * S] = 0
        mem1[3][100:200] ^= 0x33
        chain.append(ora.checkpoint(mem1))
        imgs = [C.crac_image_deserialize(b) for b in chain]
        try:
            for b in h.bufs:
                b.zero()
            h2 = Harness(S, lineage=4242, flags=CODED)   # a context of the oracle's lineage
            try:
                for b in h.bufs:
                    C.crac_ctx_register_alloc(h2.ctx, b.ptr, b.nbytes, b.kind)
                C.crac_ctx_restart(h2.ctx, imgs[-1], h2.stream)
                for b, w in zip(h.bufs, mem1):
                    assert np.array_equal(b.read(), w)
                assert C.crac_ctx_last_restart(h2.ctx)["chunks_rewritten"] == int(h.first()[-1])
            finally:
                h2.close()
        finally:
            for i in imgs:
                C.crac_image_release(i)
        assert len(sizes) == len(h.bufs)
    finally:
        h.close()


def _damage(img_bytes, S, how):
    """Copy of a coded FULL image with its first coded stream damaged."""
    im = O.parse_image(img_bytes)
    firsts = [t[4] for t in im.allocs]
    off = len(img_bytes) - len(im.payload)
    for e, c in enumerate(im.idx.tolist()):
        a = int(np.searchsorted(firsts, c, side="right") - 1)
        ln = O.chunk_len(im.allocs[a][2], c - firsts[a], S)
        z = int(im.zlen[e])
        if z < ln:
            break
        off += crz.padded(z)
    else:
        raise AssertionError("no coded stream")
    b = bytearray(img_bytes)
    if how == "width":
        b[off + 4] = 0x0C          # plane 0 width 12
    elif how == "reserved":
        b[off + 7] = 0x80
    elif how == "overflow":        # plane 0 minimum 255 with a non-zero width
        b[off + 0] = 0xFF
        b[off + 4] = (b[off + 4] & 0xF0) | 0x08
    return bytes(b)


@pytest.mark.parametrize("how", ["width", "reserved"])
def test_damaged_stream_header_is_refused_at_deserialize(how):
    """A stream whose headers no chunk encodes to (a width above 8, a
    reserved bit) is refused when the image is deserialized, before any
    restore can touch memory."""
    S = 4 * KIB
    h = Harness(S, lineage=1500, flags=CODED)
    try:
        h.add(16 * S, data=_contents("f32_normal", 16 * S, 5))
        img, lib, ora = h.checkpoint()
        assert lib == ora
        with pytest.raises(C.CracError) as e:
            C.crac_image_deserialize(_damage(lib, S, how))
        assert e.value.code == C.CRAC_ERR_CORRUPT
    finally:
        h.close()


def test_plane_overflow_is_reported_at_restart():
    """A header that lets a plane value pass 255 is only found by decoding:
    the restart reports CRAC_ERR_CORRUPT (the allocations' contents are then
    unspecified), and the context still restores a good image."""
    S = 4 * KIB
    h = Harness(S, lineage=1500, flags=CODED)
    try:
        h.add(16 * S, data=_contents("f32_normal", 16 * S, 5))
        img, lib, ora = h.checkpoint()
        assert lib == ora
        want = h.host()
        bad = C.crac_image_deserialize(_damage(lib, S, "overflow"))
        try:
            h2 = Harness(S, lineage=1500, flags=CODED)
            try:
                C.crac_ctx_register_alloc(h2.ctx, h.bufs[0].ptr, h.bufs[0].nbytes)
                with pytest.raises(C.CracError) as e:
                    C.crac_ctx_restart(h2.ctx, bad, h2.stream)
                assert e.value.code == C.CRAC_ERR_CORRUPT
                C.crac_ctx_restart(h2.ctx, img, h2.stream)
                torch.cuda.synchronize()
                assert np.array_equal(h.bufs[0].read(), want[0])
            finally:
                h2.close()
        finally:
            C.crac_image_release(bad)
    finally:
        h.close()


def test_staged_flag_still_restores_coded_chain():
    """CRAC_FLAG_STAGED_RESTORE: coded host images are decoded in place anyway."""
    S = 4 * KIB
    h = Harness(S, lineage=1600, flags=CODED | C.CRAC_FLAG_STAGED_RESTORE)
    try:
        _fill(h, S, seed=9)
        img0, lib0, ora0 = h.checkpoint()
        assert lib0 == ora0
        h.mutate(pattern_mutations(h.first(), [b.nbytes for b in h.bufs], S, "random10", seed=2))
        img1, lib1, ora1 = h.checkpoint()
        assert lib1 == ora1
        want = h.host()
        for b in h.bufs:
            b.zero()
        h.restart(img1)
        for b, w in zip(h.bufs, want):
            assert np.array_equal(b.read(), w)
    finally:
        h.close()


@pytest.mark.parametrize("residency,flags", [(C.CRAC_RESIDENCY_HOST, 0),
                                             (C.CRAC_RESIDENCY_HOST, C.CRAC_FLAG_DIRECT_DRAIN),
                                             (C.CRAC_RESIDENCY_DEVICE, 0)])
def test_encoder_wait_runs_out_cleanly(residency, flags):
    """The encoder is launched so that its first tile is never processed: the
    later tiles' bounded look-back waits run out, the checkpoint reports
    CRAC_ERR_TIMEOUT, and the context's baseline is untouched (the next
    checkpoint equals the oracle's, which never saw the failed one)."""
    S = 4 * KIB
    h = Harness(S, lineage=1700, image_residency=residency, flags=flags | CODED, timeout_ns=20_000_000)
    try:
        for i, n in enumerate([64 * S + 100, 40 * S]):   # more than one 16-chunk tile
            h.add(n, data=_contents("f32_normal", n, 40 + i))
        _, lib1, ora1 = h.checkpoint()
        assert lib1 == ora1
        h.mutate(pattern_mutations(h.first(), [b.nbytes for b in h.bufs], S, "alternating", seed=3))
        C.crac_debug_inject_fault(C.CRAC_FAULT_ENCODE_WAIT, 1)
        with pytest.raises(C.CracError) as e:
            C.crac_ctx_checkpoint(h.ctx, h.stream)
        assert e.value.code == C.CRAC_ERR_TIMEOUT
        C.crac_debug_inject_fault(C.CRAC_FAULT_NONE, 0)
        _, lib2, ora2 = h.checkpoint()
        assert lib2 == ora2
        want = h.host()
        for b in h.bufs:
            b.zero()
        h.restart(h.images[-1])
        for b, w in zip(h.bufs, want):
            assert np.array_equal(b.read(), w)
    finally:
        C.crac_debug_inject_fault(C.CRAC_FAULT_NONE, 0)
        h.close()


@pytest.mark.parametrize("S", [16, 64, 256, 1 << 20])
@pytest.mark.parametrize("residency", [C.CRAC_RESIDENCY_HOST, C.CRAC_RESIDENCY_DEVICE])
def test_coded_extreme_chunk_sizes(S, residency):
    """Chunks below one block (every stream raw, up to 128 entries a tile) and
    1 MiB chunks (sixteen shared-memory windows each, a ragged last one)."""
    h = Harness(S, lineage=1800 + S.bit_length(), image_residency=residency, flags=CODED)
    try:
        sizes = [3 * S + 5, 2 * S, 4100] if S >= 1 << 20 else [5000, 777, 64 * S + 48]
        for i, n in enumerate(sizes):
            h.add(n, data=_contents(["f32_normal", "zeros", "bf16"][i % 3], n, 60 + i))
        img, lib, ora = h.checkpoint()
        assert lib == ora
        h.mutate(pattern_mutations(h.first(), sizes, S, "alternating", seed=4))
        img2, lib2, ora2 = h.checkpoint()
        assert lib2 == ora2
        want = h.host()
        for b in h.bufs:
            b.zero()
        h.restart(img2)
        for b, w in zip(h.bufs, want):
            assert np.array_equal(b.read(), w)
    finally:
        h.close()


def test_deserialize_rejects_bad_coded_tables():
    """Host-side checks of a coded image's tables: a stream longer than its
    chunk, an empty stream, a payload that does not match the padded stream
    lengths, an unknown flag bit."""
    S = 4 * KIB
    ora = O.OracleContext(S, lineage=1900, coded=True)
    mem = [_contents("f32_normal", 9 * S + 100, 1), np.zeros(3 * S, np.uint8)]
    for i, m in enumerate(mem):
        ora.register(0x100000 * (i + 1), m.size)
    good = ora.checkpoint(mem)
    im = O.parse_image(good)
    zoff = len(good) - len(im.payload) - 8 * im.k   # start of zlen[]

    def patched(e, value):
        b = bytearray(good)
        b[zoff + 8 * e:zoff + 8 * e + 8] = int(value).to_bytes(8, "little")
        return bytes(b)

    lens = [O.chunk_len(im.allocs[int(np.searchsorted([t[4] for t in im.allocs], c, side="right") - 1)][2],
                        c - im.allocs[int(np.searchsorted([t[4] for t in im.allocs], c, side="right") - 1)][4], S)
            for c in im.idx.tolist()]
    coded_e = next(e for e, z in enumerate(im.zlen.tolist()) if z < lens[e])
    bad = [patched(0, lens[0] + 1),                      # longer than the chunk
           patched(0, 0),                                # empty
           patched(coded_e, int(im.zlen[coded_e]) + 16)]  # padded lengths no longer add up to the payload
    flags = bytearray(good)
    flags[12] |= 4                                       # unknown flag bit
    bad.append(bytes(flags))
    for b in bad:
        with pytest.raises(C.CracError) as e:
            C.crac_image_deserialize(b)
        assert e.value.code == C.CRAC_ERR_CORRUPT
    img = C.crac_image_deserialize(good)                 # the untouched image is accepted
    assert C.crac_image_info(img)["raw_bytes"] == sum(lens)
    C.crac_image_release(img)


@pytest.mark.parametrize("base_coded", [True, False])
def test_mixed_coded_and_plain_chain(base_coded):
    """A chain whose base is coded and delta plain (or the reverse), written
    by the oracle and deserialized: the restore decodes the coded pieces and
    copies the plain ones in the same launch."""
    S = 4 * KIB
    h = Harness(S, lineage=2000 + base_coded)
    try:
        _fill(h, S, seed=90)
        mem0 = h.host()
        ora = O.OracleContext(S, lineage=7000 + base_coded, coded=base_coded)
        for b in h.bufs:
            ora.register(b.ptr, b.nbytes, b.kind)
        chain = [ora.checkpoint(mem0)]
        ora.coded = not base_coded
        mem1 = [m.copy() for m in mem0]
        mem1[0][: 2 * S] = 0
        mem1[2][S:S + 100] ^= 0x77
        chain.append(ora.checkpoint(mem1))
        assert O.parse_image(chain[0]).coded == base_coded and O.parse_image(chain[1]).coded != base_coded
        imgs = [C.crac_image_deserialize(b) for b in chain]
        try:
            for b in h.bufs:
                b.zero()
            h2 = Harness(S, lineage=7000 + base_coded)
            try:
                for b in h.bufs:
                    C.crac_ctx_register_alloc(h2.ctx, b.ptr, b.nbytes, b.kind)
                C.crac_ctx_restart(h2.ctx, imgs[-1], h2.stream)
                for b, w in zip(h.bufs, mem1):
                    assert np.array_equal(b.read(), w)
            finally:
                h2.close()
        finally:
            for i in imgs:
                C.crac_image_release(i)
    finally:
        h.close()


def test_pipelined_staged_encode_matches_oracle():
    """A FULL coded checkpoint into host images with enough 64 KiB tiles that
    the encoder runs as several launches, each launch's streams copied to the
    image while the next ones encode (given pinned regions with room for its
    worst case): the image must equal the oracle's byte
    for byte (fp32, zero and incompressible allocations, a ragged tail), have
    taken more encoder launches than the same pass into device images, and
    restart exactly; then the same with the first launch's first tile never
    processed: CRAC_ERR_TIMEOUT, and the baseline untouched."""
    S = 64 * KIB
    sizes = [150 * 1024 * KIB + 48, 56 * 1024 * KIB, 56 * 1024 * KIB, 5 * 1024 * KIB + 16]
    kinds = ["f32_normal", "zeros", "u8", "bf16"]
    infos = {}
    for residency in (C.CRAC_RESIDENCY_DEVICE, C.CRAC_RESIDENCY_HOST):
        # the pipelined encode carves its worst-case pinned block from existing regions only
        h = Harness(S, lineage=1900 + residency, image_residency=residency, flags=CODED, timeout_ns=50_000_000,
                    reserve_host_bytes=1 << 30)
        try:
            for i, (n, kd) in enumerate(zip(sizes, kinds)):
                h.add(n, data=_contents(kd, n, 90 + i))
            img, lib, ora = h.checkpoint(compare=residency == C.CRAC_RESIDENCY_HOST)
            infos[residency] = C.crac_ctx_last_pass(h.ctx)
            if residency == C.CRAC_RESIDENCY_DEVICE:
                continue
            assert lib == ora
            want = h.host()
            for b in h.bufs:
                b.zero()
            h.restart(img)
            for b, w in zip(h.bufs, want):
                assert np.array_equal(b.read(), w)
            # a failed pipelined encode: reported, and the baseline stays the first image's
            h.oracle.invalidate()
            C.crac_ctx_invalidate(h.ctx)
            C.crac_debug_inject_fault(C.CRAC_FAULT_ENCODE_WAIT, 1)
            with pytest.raises(C.CracError) as e:
                C.crac_ctx_checkpoint(h.ctx, h.stream)
            assert e.value.code == C.CRAC_ERR_TIMEOUT
            C.crac_debug_inject_fault(C.CRAC_FAULT_NONE, 0)
            h.mutate(pattern_mutations(h.first(), sizes, S, "random10", seed=5))
            _, lib2, ora2 = h.checkpoint()
            assert lib2 == ora2
        finally:
            C.crac_debug_inject_fault(C.CRAC_FAULT_NONE, 0)
            h.close()
    dev, host = infos[C.CRAC_RESIDENCY_DEVICE], infos[C.CRAC_RESIDENCY_HOST]
    assert host["kernel_launches"] >= dev["kernel_launches"] + 1, (host, dev)
