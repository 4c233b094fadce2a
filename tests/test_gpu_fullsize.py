"""Config 2 at full size in the benchmark's launch configuration (GPU).

256 allocations, log-uniform sizes rescaled to 4 GiB, fp32 N(0,1) contents,
64 KiB chunks, batched graph launch.  At this size the oracle checks sampled
chunks one by one (fingerprints, payload bytes) and the properties that hold
at any size: the dirty list equals the mutated set, the payload length is the
sum of those chunks' lengths, restore reproduces memory exactly.
"""
import numpy as np
import pytest
import torch

import paper_2008_10596_gb300 as C
import workloads as W
from oracle import oracle as O
from paper_2008_10596_gb300 import testkit

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("oracle_lib")]


def _alloc_c2(wl):
    g = torch.Generator(device="cuda")
    g.manual_seed(wl.seed)
    bufs = []
    for n in wl.sizes:
        t = torch.randn((n + 3) // 4, generator=g, device="cuda", dtype=torch.float32)
        bufs.append(t.view(torch.uint8)[:n])
    return bufs


def _mut_entries(bufs, first, S, muts):
    arr = np.zeros((len(muts), 3), dtype=np.uint64)
    for i, m in enumerate(muts):
        a = int(np.searchsorted(first, m.chunk, side="right") - 1)
        lo = (m.chunk - int(first[a])) * S
        arr[i] = (bufs[a].data_ptr() + lo, min(S, bufs[a].numel() - lo), m.mask)
    return torch.from_numpy(arr.view(np.int64)).to("cuda")


@pytest.mark.parametrize("residency", [C.CRAC_RESIDENCY_HOST, C.CRAC_RESIDENCY_DEVICE])
def test_config2_full_size(residency):
    wl = W.config2()
    S = wl.chunk_bytes
    bufs = _alloc_c2(wl)
    first = W.chunk_layout(wl.sizes, S)
    n = int(first[-1])
    stream = torch.cuda.current_stream()
    ctx = C.crac_ctx_create(C.crac_config_default(chunk_bytes=S, lineage=2, image_residency=residency))
    imgs = []
    try:
        for b in bufs:
            C.crac_ctx_register_alloc(ctx, b.data_ptr(), b.numel(), C.CRAC_KIND_DEVICE)
        img1 = C.crac_ctx_checkpoint(ctx, stream)
        imgs.append(img1)
        C.crac_image_wait(img1)
        info = C.crac_image_info(img1)
        assert info["k"] == n and info["payload_bytes"] == wl.total_bytes and info["flags"] == 1
        saved = [b.clone() for b in bufs]
        for b in bufs:
            b.zero_()
        C.crac_ctx_restart(ctx, img1, stream)
        torch.cuda.synchronize()
        assert all(torch.equal(a, b) for a, b in zip(bufs, saved))
        del saved

        muts = W.choose_mutations(wl.seed, n, wl.dirty_fraction)
        ent = _mut_entries(bufs, first, S, muts)
        testkit.mutate_xor(ent.data_ptr(), len(muts), stream)
        img2 = C.crac_ctx_checkpoint(ctx, stream)
        imgs.append(img2)
        raw = C.crac_image_serialize(img2)
        im = O.parse_image(raw)
        chosen = sorted(m.chunk for m in muts)
        assert im.idx.tolist() == chosen
        lens = {}
        for c in chosen:
            a = int(np.searchsorted(first, c, side="right") - 1)
            lens[c] = O.chunk_len(wl.sizes[a], c - int(first[a]), S)
        assert len(im.payload) == sum(lens.values())
        # sampled oracle checks: fingerprints of any chunk, payload of dirty chunks
        rng = np.random.default_rng(7)
        offs = np.concatenate([[0], np.cumsum([lens[c] for c in chosen])])
        for c in list(rng.choice(n, 48, replace=False)) + [0, n - 1]:
            a = int(np.searchsorted(first, c, side="right") - 1)
            lo = (int(c) - int(first[a])) * S
            dev_bytes = bufs[a][lo:lo + S].cpu().numpy()
            assert int(im.fp[c]) == O.fp64(dev_bytes)
        for j in rng.choice(len(chosen), 48, replace=False):
            c = chosen[j]
            a = int(np.searchsorted(first, c, side="right") - 1)
            lo = (c - int(first[a])) * S
            dev_bytes = bufs[a][lo:lo + S].cpu().numpy()
            assert bytes(im.payload[offs[j]:offs[j + 1]]) == dev_bytes.tobytes()
        # chain restore (full + delta) into zeroed memory
        saved = [b.clone() for b in bufs]
        for b in bufs:
            b.zero_()
        C.crac_ctx_restart(ctx, img2, stream)
        torch.cuda.synchronize()
        assert all(torch.equal(a, b) for a, b in zip(bufs, saved))
    finally:
        torch.cuda.synchronize()
        for i in imgs:
            C.crac_image_release(i)
        C.crac_ctx_destroy(ctx)
