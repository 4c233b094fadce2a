"""The autotuner (GPU): observation rounds measure the real pass for every
candidate chunk size; the dirty bytes they report must be exactly the bytes
of the chunks that contain a rewritten 4 KiB page (integer work, compared
exactly), and the retuned context must keep producing oracle-exact images."""
import numpy as np
import pytest
import torch

import paper_2008_10596_gb300 as C
import workloads as W
from oracle import oracle as O
from paper_2008_10596_gb300 import testkit

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("oracle_lib")]

KIB = 1024
PAGE = 4 * KIB


def _mutate_pages(bufs, sizes, pages, seed):
    rng = W.XorShift64(seed)
    rows = []
    for a, p in pages:
        rows.append((bufs[a].data_ptr() + p * PAGE, min(PAGE, sizes[a] - p * PAGE), rng.mask32()))
    arr = np.array(rows, dtype=np.uint64)
    dev = torch.from_numpy(arr.view(np.int64)).to("cuda")
    testkit.mutate_xor(dev.data_ptr(), len(rows), torch.cuda.current_stream())
    torch.cuda.synchronize()


def _expected_dirty_bytes(sizes, pages, S):
    chunks = {(a, (p * PAGE) // S) for a, p in pages}
    return sum(min(S, sizes[a] - c * S) for a, c in chunks)


def test_tune_observe_exact_dirty_bytes_and_choice():
    sizes = [4 * 1024 * KIB, 3 * 1024 * KIB + 4 * KIB, 512 * KIB, 12 * 1024 * KIB]
    bufs = [torch.from_numpy(W.host_contents("u8", n, 500 + i)).to("cuda") for i, n in enumerate(sizes)]
    ctx = C.crac_ctx_create(C.crac_config_default(chunk_bytes=64 * KIB, lineage=44))
    stream = torch.cuda.current_stream()
    cands = [4 * KIB, 64 * KIB, 256 * KIB]
    imgs = []
    try:
        ora = O.OracleContext(4 * KIB, lineage=44)
        for b, n in zip(bufs, sizes):
            C.crac_ctx_register_alloc(ctx, b.data_ptr(), n)
            ora.register(b.data_ptr(), n)
        r0 = C.crac_ctx_tune_observe(ctx, cands, stream)
        assert r0["rounds"] == 0
        npages = [-(-n // PAGE) for n in sizes]
        all_pages = [(a, p) for a in range(len(sizes)) for p in range(npages[a])]
        rng = W.XorShift64(77)
        for rnd in range(2):
            picks = W.choose_distinct(rng, len(all_pages), len(all_pages) // 50)   # 2% of pages
            pages = [all_pages[i] for i in picks]
            _mutate_pages(bufs, sizes, pages, 100 + rnd)
            r = C.crac_ctx_tune_observe(ctx, cands, stream)
            assert r["rounds"] == rnd + 1
            for S, got in zip(r["chunk_bytes"], r["last_dirty_bytes"]):
                assert got == _expected_dirty_bytes(sizes, pages, S), S
        res = C.crac_ctx_tune_apply(ctx, 190.0, stream)
        assert res["chosen_chunk_bytes"] == 4 * KIB
        assert res["chosen_pass_kernel"] in (C.CRAC_PASS_SPLIT, C.CRAC_PASS_LDG, C.CRAC_PASS_TMA)
        assert all(v > 0 for v in res["variant_ms"][1:4])
        # LDG was timed at its default 4 KiB tile (32 chunks) and at half and twice it
        assert res["ldg_tiles"] == [32, 16, 64]
        assert all(m > 0 for m in res["ldg_tile_ms"])
        assert res["variant_ms"][C.CRAC_PASS_LDG] == min(res["ldg_tile_ms"])
        if res["chosen_pass_kernel"] == C.CRAC_PASS_LDG:
            assert res["chosen_chunks_per_tile"] in res["ldg_tiles"]
        else:
            assert res["chosen_chunks_per_tile"] == 0
        # the retuned context: a FULL image at 4 KiB, then an exact delta
        img = C.crac_ctx_checkpoint(ctx, stream)
        imgs.append(img)
        C.crac_image_wait(img)
        host = [b.cpu().numpy() for b in bufs]
        assert C.crac_image_serialize(img) == ora.checkpoint(host)
        _mutate_pages(bufs, sizes, [(0, 3), (3, 100), (1, 768)], 9)
        img2 = C.crac_ctx_checkpoint(ctx, stream)
        imgs.append(img2)
        C.crac_image_wait(img2)
        host = [b.cpu().numpy() for b in bufs]
        raw = C.crac_image_serialize(img2)
        assert raw == ora.checkpoint(host)
        assert O.parse_image(raw).k == 3
    finally:
        torch.cuda.synchronize()
        for i in imgs:
            C.crac_image_release(i)
        C.crac_ctx_destroy(ctx)


def test_tune_apply_needs_observations():
    ctx = C.crac_ctx_create(C.crac_config_default(chunk_bytes=64 * KIB))
    t = torch.zeros(1 << 20, dtype=torch.uint8, device="cuda")
    try:
        C.crac_ctx_register_alloc(ctx, t.data_ptr(), t.numel())
        with pytest.raises(C.CracError) as e:
            C.crac_ctx_tune_apply(ctx, 0.0)
        assert e.value.code == C.CRAC_ERR_UNSUPPORTED
        C.crac_ctx_tune_observe(ctx, [4 * KIB, 64 * KIB])
        with pytest.raises(C.CracError) as e:
            C.crac_ctx_tune_apply(ctx, 0.0)
        assert e.value.code == C.CRAC_ERR_UNSUPPORTED
        with pytest.raises(C.CracError) as e:
            C.crac_ctx_tune_observe(ctx, [3000])
        assert e.value.code == C.CRAC_ERR_INVALID_ARG
    finally:
        C.crac_ctx_destroy(ctx)


def test_tune_mostly_dirty_device_images_times_every_kernel():
    """With every page rewritten and device-resident images, apply times the
    split, LDG, TMA and sparse passes at the chosen size; whichever wins, the
    retuned context keeps producing the oracle's images."""
    sizes = [8 * 1024 * KIB, 2 * 1024 * KIB + 16 * 7, 1024 * KIB]
    bufs = [torch.from_numpy(W.host_contents("u8", n, 600 + i)).to("cuda") for i, n in enumerate(sizes)]
    ctx = C.crac_ctx_create(C.crac_config_default(chunk_bytes=64 * KIB, lineage=45,
                                                  image_residency=C.CRAC_RESIDENCY_DEVICE))
    stream = torch.cuda.current_stream()
    imgs = []
    try:
        for b, n in zip(bufs, sizes):
            C.crac_ctx_register_alloc(ctx, b.data_ptr(), n)
        cands = [4 * KIB, 64 * KIB]
        C.crac_ctx_tune_observe(ctx, cands, stream)
        all_pages = [(a, p) for a in range(len(sizes)) for p in range(-(-sizes[a] // PAGE))]
        for rnd in range(2):
            _mutate_pages(bufs, sizes, all_pages, 200 + rnd)
            C.crac_ctx_tune_observe(ctx, cands, stream)
        res = C.crac_ctx_tune_apply(ctx, 0.0, stream)
        vm = res["variant_ms"]
        assert all(vm[k] > 0 for k in (C.CRAC_PASS_SPLIT, C.CRAC_PASS_LDG, C.CRAC_PASS_TMA, C.CRAC_PASS_SPARSE))
        assert vm[res["chosen_pass_kernel"]] == min(v for v in vm if v > 0)
        # the context itself has no baseline yet: its next image is FULL at the chosen size
        ora = O.OracleContext(res["chosen_chunk_bytes"], lineage=45)
        for b, n in zip(bufs, sizes):
            ora.register(b.data_ptr(), n)
        for rnd in range(2):
            img = C.crac_ctx_checkpoint(ctx, stream)
            imgs.append(img)
            C.crac_image_wait(img)
            assert C.crac_image_serialize(img) == ora.checkpoint([b.cpu().numpy() for b in bufs])
            _mutate_pages(bufs, sizes, all_pages[::3], 300 + rnd)
    finally:
        torch.cuda.synchronize()
        for i in imgs:
            C.crac_image_release(i)
        C.crac_ctx_destroy(ctx)


def test_tune_coded_context_never_picks_sparse():
    """A coded context (CRAC_FLAG_COMPRESS, device images, mostly dirty pages,
    where the sparse pass would otherwise be a candidate): apply times the
    other kernels only, and the retuned context's coded images equal the
    oracle's."""
    sizes = [4 * 1024 * KIB, 2 * 1024 * KIB + 16 * 7]
    bufs = [torch.from_numpy(W.host_contents("f32_normal", n, 650 + i)).to("cuda") for i, n in enumerate(sizes)]
    ctx = C.crac_ctx_create(C.crac_config_default(chunk_bytes=64 * KIB, lineage=46,
                                                  image_residency=C.CRAC_RESIDENCY_DEVICE,
                                                  flags=C.CRAC_FLAG_COMPRESS))
    stream = torch.cuda.current_stream()
    imgs = []
    try:
        for b, n in zip(bufs, sizes):
            C.crac_ctx_register_alloc(ctx, b.data_ptr(), n)
        cands = [4 * KIB, 64 * KIB]
        C.crac_ctx_tune_observe(ctx, cands, stream)
        all_pages = [(a, p) for a in range(len(sizes)) for p in range(-(-sizes[a] // PAGE))]
        for rnd in range(2):
            _mutate_pages(bufs, sizes, all_pages, 210 + rnd)
            C.crac_ctx_tune_observe(ctx, cands, stream)
        res = C.crac_ctx_tune_apply(ctx, 0.0, stream)
        assert res["variant_ms"][C.CRAC_PASS_SPARSE] == 0
        assert res["chosen_pass_kernel"] != C.CRAC_PASS_SPARSE
        ora = O.OracleContext(res["chosen_chunk_bytes"], lineage=46, coded=True)
        for b, n in zip(bufs, sizes):
            ora.register(b.data_ptr(), n)
        for rnd in range(2):
            img = C.crac_ctx_checkpoint(ctx, stream)
            imgs.append(img)
            C.crac_image_wait(img)
            assert C.crac_image_serialize(img) == ora.checkpoint([b.cpu().numpy() for b in bufs])
            _mutate_pages(bufs, sizes, all_pages[::3], 310 + rnd)
    finally:
        torch.cuda.synchronize()
        for i in imgs:
            C.crac_image_release(i)
        C.crac_ctx_destroy(ctx)
