"""The allocation-free checkpoint pass against the regular checkpoint (GPU).

crac_pass_noalloc serves callers that cannot allocate memory when they must
checkpoint -- code inside an interposed cudaMalloc/cudaFree or an allocator
hook (where allocating again would recurse or deadlock), a preemption-time
save that must not change the device memory map, or a process whose
allocator is exhausted.  It runs the same pass with its scratch in a fixed
array of the library's device memory.  This file checks, through the C ABI,
that two calls in a row (a full pass, then an incremental one against the
first call's fingerprints) produce exactly the fingerprints, dirty list,
offsets and staged bytes of the CPU oracle's image of the same memory, and
of crac_ctx_checkpoint's, at 256-byte, 4 KiB and 64 KiB chunks and at the
scratch's tile limit.  The work is integer/byte work, so the comparison is
bit-exact.

The file name sorts last so that a run stopping at the first failure has
already run every other test.
"""
import os

import numpy as np
import pytest
import torch

import paper_2008_10596_gb300 as C
import workloads as W
from oracle import oracle as O
from paper_2008_10596_gb300 import testkit

pytestmark = pytest.mark.gpu

NO_BASE = np.uint64(0xFFFFFFFFFFFFFFFF)


def _u64_tensor(arr):
    return torch.from_numpy(np.ascontiguousarray(arr, dtype=np.uint64).view(np.int64)).to("cuda")


def _as_u64(t, n=None):
    a = t.cpu().numpy().view(np.uint64)
    return a if n is None else a[:n]


def _run_two_calls(S, sizes, mut_fraction, seed):
    """A full call (no baseline, fp_old NULL) and an incremental call against
    the first call's fingerprints, each compared with the oracle's image of
    the same memory and with crac_ctx_checkpoint's image."""
    bufs = []
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    for i, n in enumerate(sizes):
        if n <= (4 << 20):
            t = torch.from_numpy(W.host_contents("u32_xorshift", n, seed + i)).to("cuda")
        else:   # large regions: seeded bytes from torch's generator, made on the device
            t = torch.randint(0, 256, (n,), generator=g, device="cuda", dtype=torch.uint8)
        bufs.append(t)
    first = W.chunk_layout(sizes, S)
    n = int(first[-1])
    total = sum(sizes)
    stream = torch.cuda.current_stream()

    ctx = C.crac_ctx_create(C.crac_config_default(chunk_bytes=S, lineage=5))
    ora = O.OracleContext(S, lineage=5, workers=os.cpu_count() or 1)
    imgs = []
    try:
        for b, sz in zip(bufs, sizes):
            C.crac_ctx_register_alloc(ctx, b.data_ptr(), sz, C.CRAC_KIND_DEVICE)
            ora.register(b.data_ptr(), sz, O.KIND_DEVICE)

        regions = np.zeros((len(sizes), 4), dtype=np.uint64)
        for a, b in enumerate(bufs):
            regions[a] = (b.data_ptr(), sizes[a], first[a], NO_BASE)
        regions_dev = _u64_tensor(regions)
        fp_a = torch.empty(n, dtype=torch.int64, device="cuda")
        fp_b = torch.empty(n, dtype=torch.int64, device="cuda")
        idx = torch.empty(n, dtype=torch.int64, device="cuda")
        off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        staging = torch.empty(total, dtype=torch.uint8, device="cuda")
        totals = torch.empty(3, dtype=torch.int64, device="cuda")

        def run(fp_old, fp_new):
            C.crac_pass_noalloc(regions_dev, len(sizes), n, S, fp_old, fp_new, idx, off, n,
                                staging, total, totals, stream)
            torch.cuda.synchronize()
            t = totals.cpu().numpy().view(np.uint64)
            err = int(t[0] >> np.uint64(32))
            return err, int(t[1]), int(t[2])

        def check(raw, fp_new, k, d):
            im = O.parse_image(raw)
            assert k == im.k and d == len(im.payload)
            assert np.array_equal(_as_u64(fp_new), im.fp)
            assert np.array_equal(_as_u64(idx, k), im.idx)
            lens = [O.chunk_len(sizes[a], int(c) - int(first[a]), S)
                    for c, a in zip(im.idx.tolist(), (np.searchsorted(first, im.idx.astype(np.int64), side="right") - 1).tolist())]
            offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)
            assert np.array_equal(_as_u64(off, k + 1), offs)
            assert staging[:d].cpu().numpy().tobytes() == bytes(im.payload)

        # call 1: no baseline (fp_old NULL) -> every chunk
        img1 = C.crac_ctx_checkpoint(ctx, stream)
        imgs.append(img1)
        err, k, d = run(None, fp_a)
        assert err == 0 and k == n and d == total
        want = ora.checkpoint([b.cpu().numpy() for b in bufs])
        assert C.crac_image_serialize(img1) == want
        check(want, fp_a, k, d)

        # mutate a seeded set of chunks, then call 2 against call 1's fingerprints
        muts = W.choose_mutations(seed + 77, n, mut_fraction)
        ent = np.zeros((len(muts), 3), dtype=np.uint64)
        for i, m in enumerate(muts):
            a = int(np.searchsorted(first, m.chunk, side="right") - 1)
            lo = (m.chunk - int(first[a])) * S
            ent[i] = (bufs[a].data_ptr() + lo, min(S, sizes[a] - lo), m.mask)
        ent_dev = _u64_tensor(ent)
        testkit.mutate_xor(ent_dev.data_ptr(), len(muts), stream)
        img2 = C.crac_ctx_checkpoint(ctx, stream)
        imgs.append(img2)
        regions[:, 3] = first[:-1].astype(np.uint64)
        regions_dev.copy_(_u64_tensor(regions))
        err, k, d = run(fp_a, fp_b)
        assert err == 0 and k == len(muts)
        want = ora.checkpoint([b.cpu().numpy() for b in bufs])
        assert C.crac_image_serialize(img2) == want
        check(want, fp_b, k, d)
        return n
    finally:
        torch.cuda.synchronize()
        for i in imgs:
            C.crac_image_release(i)
        C.crac_ctx_destroy(ctx)


@pytest.mark.parametrize("S,sizes", [
    (256, [300000, 256 * 7, 5, 123457, 65536]),
    (4096, [300000, 4096 * 7, 5, 123457, 65536]),
    # 64 KiB chunks: eight warps per chunk (the second grid)
    (65536, [3 * 65536 + 48, 16, 1 << 20, 65536 * 5 + 4096]),
])
def test_noalloc_pass_matches_the_oracle_on_two_calls(S, sizes):
    _run_two_calls(S, sizes, 0.2, 900 + S % 1000)


def test_noalloc_pass_at_exactly_its_tile_limit():
    """128 KiB chunks take one chunk per tile: a pass over exactly
    CRAC_NOALLOC_MAX_TILES chunks (4 GiB, the last chunk ragged) fills the
    scratch to its last status word."""
    S = 128 * 1024
    n_max = C.CRAC_NOALLOC_MAX_TILES
    sizes = [(n_max // 2) * S, (n_max // 2 - 1) * S + 5]
    n = _run_two_calls(S, sizes, 0.01, 950)
    assert n == n_max


def test_noalloc_rejects_sizes_beyond_its_scratch():
    t = torch.empty(16, dtype=torch.int64, device="cuda")
    too_many = C.CRAC_NOALLOC_MAX_TILES * 2 + 1     # 64 KiB chunks: 2 chunks per tile
    with pytest.raises(C.CracError) as e:
        C.crac_pass_noalloc(t, 1, too_many, 65536, None, t, t, t, 1, t, 16, t, None)
    assert e.value.code == C.CRAC_ERR_INVALID_ARG
    with pytest.raises(C.CracError) as e:
        C.crac_pass_noalloc(t, 1, 4, 3000, None, t, t, t, 1, t, 16, t, None)
    assert e.value.code == C.CRAC_ERR_INVALID_ARG
