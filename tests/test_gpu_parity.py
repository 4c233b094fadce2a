"""CUDA path vs the CPU oracle, byte for byte (GPU).

Every image the library produces is serialized and compared with the
oracle's image of the same device bytes; every restore is compared with the
bytes the oracle's restart produces.  The work is integer/byte work, so the
bar is bit-exactness.
"""
import numpy as np
import pytest
import torch

import paper_2008_10596_gb300 as C
import workloads as W
from oracle import oracle as O
from paper_2008_10596_gb300 import testkit
from tests.gpu_harness import Harness, pattern_mutations

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("oracle_lib")]

KIB = 1024


def test_config1_full_restore_incremental():
    """One 16 MiB xorshift64 buffer, 4 KiB chunks; full, restore, 1% mutated, incremental."""
    wl = W.config1()
    h = Harness(wl.chunk_bytes, lineage=101)
    try:
        data = W.host_contents("u32_xorshift", wl.sizes[0], wl.seed)
        b = h.add(wl.sizes[0], data=data)
        img1, lib1, ora1 = h.checkpoint()
        assert lib1 == ora1
        assert O.parse_image(lib1).full and bytes(O.parse_image(lib1).payload) == data.tobytes()
        b.zero()
        h.restart(img1)
        assert np.array_equal(b.read(), data)
        n = wl.sizes[0] // wl.chunk_bytes
        muts = W.choose_mutations(wl.seed, n, wl.dirty_fraction)
        assert len(muts) == 41
        h.mutate(muts)
        expect = data.copy()
        W.apply_mutations_host([expect], np.array([0, n]), wl.chunk_bytes, muts)
        assert np.array_equal(b.read(), expect)          # the mutator did what the spec says
        img2, lib2, ora2 = h.checkpoint()
        assert lib2 == ora2
        im2 = O.parse_image(lib2)
        assert im2.idx.tolist() == sorted(m.chunk for m in muts)
        assert im2.parent_epoch == 1 and im2.epoch == 2
        # an unmodified checkpoint is empty
        img3, lib3, ora3 = h.checkpoint()
        assert lib3 == ora3 and O.parse_image(lib3).k == 0
        # restore the chain into zeroed memory
        b.zero()
        h.restart(img3, [ora1, ora2, ora3])
        assert np.array_equal(b.read(), expect)
    finally:
        h.close()


SIZES = [1, 7, 8, 4095, 4096, 4097]


@pytest.mark.parametrize("S,kern", [(64, C.CRAC_PASS_AUTO), (4 * KIB, C.CRAC_PASS_TMA),
                                    (4 * KIB, C.CRAC_PASS_LDG), (64 * KIB, C.CRAC_PASS_TMA),
                                    (64 * KIB, C.CRAC_PASS_LDG), (256 * KIB, C.CRAC_PASS_AUTO)])
@pytest.mark.parametrize("pattern", ["none", "all", "first", "last", "tail", "alternating", "random10"])
def test_sweep_sizes_patterns(S, kern, pattern):
    sizes = SIZES + [3 * S + 5, 2 * S]
    h = Harness(S, lineage=200 + S % 97, pass_kernel=kern)
    try:
        for i, n in enumerate(sizes):
            h.add(n, seed=10 + i)
        _, lib1, ora1 = h.checkpoint()
        assert lib1 == ora1
        first = h.first()
        muts = pattern_mutations(first, sizes, S, pattern)
        h.mutate(muts)
        img2, lib2, ora2 = h.checkpoint()
        assert lib2 == ora2
        assert O.parse_image(lib2).idx.tolist() == sorted(m.chunk for m in muts)
        want = h.host()
        for b in h.bufs:
            b.zero()
        h.restart(img2)
        for b, w in zip(h.bufs, want):
            assert np.array_equal(b.read(), w)
    finally:
        h.close()


@pytest.mark.parametrize("cpt,wpc", [(1, 1), (3, 1), (8, 8), (17, 8), (256, 1)])
def test_work_split_variants_identical(cpt, wpc):
    """Tile size and warps-per-chunk change only the schedule, never the bytes."""
    S = 4 * KIB
    sizes = [123457, 4096 * 37 + 1, 64 * KIB, 5, 300000]
    h = Harness(S, lineage=7, chunks_per_tile=cpt, warps_per_chunk=wpc, pass_kernel=C.CRAC_PASS_LDG)
    try:
        for i, n in enumerate(sizes):
            h.add(n, seed=30 + i)
        _, lib1, ora1 = h.checkpoint()
        assert lib1 == ora1
        h.mutate(pattern_mutations(h.first(), sizes, S, "random10", seed=9))
        _, lib2, ora2 = h.checkpoint()
        assert lib2 == ora2
    finally:
        h.close()


@pytest.mark.parametrize("S,kern", [(s, C.CRAC_PASS_TMA) for s in (1 * KIB, 2 * KIB, 8 * KIB, 16 * KIB,
                                                                   32 * KIB, 64 * KIB)] +
                         [(s, C.CRAC_PASS_SPLIT) for s in (256, 512, 1 * KIB, 2 * KIB, 8 * KIB, 16 * KIB)])
def test_chunk_sizes_ragged(S, kern):
    """Every chunk-size regime of the TMA pass (1..64 chunks per 64 KiB tile,
    1..8 warps per chunk) and of the split pass (several chunks per warp
    iteration below 8 KiB, one whole chunk at 8 KiB, segments above), with
    ragged allocation ends that shift later chunks off 16-byte alignment in
    the staging buffer and segments that straddle allocation ends."""
    sizes = [S * 37 + 3, 5, S * 64, 4097, S * 3 + 16, 777777, S + 9]
    h = Harness(S, lineage=300 + S // 256, pass_kernel=kern)
    try:
        for i, n in enumerate(sizes):
            h.add(n, seed=90 + i)
        _, lib1, ora1 = h.checkpoint()
        assert lib1 == ora1
        for seed in (1, 2):
            h.mutate(pattern_mutations(h.first(), sizes, S, "random10", seed=seed))
            img, lib, ora = h.checkpoint()
            assert lib == ora
        want = h.host()
        for b in h.bufs:
            b.zero()
        h.restart(img)
        for b, w in zip(h.bufs, want):
            assert np.array_equal(b.read(), w)
    finally:
        h.close()


@pytest.mark.parametrize("S,staging", [(512, 0), (4 * KIB, 0), (8 * KIB, 0), (64 * KIB, 0), (256 * KIB, 0),
                                       (4 * KIB, 96 * KIB), (64 * KIB, 320 * KIB)])
@pytest.mark.parametrize("pattern", ["none", "all", "alternating", "random10"])
def test_sparse_pass(S, staging, pattern):
    """The sparse split pass (every chunk written at its uncompacted offset,
    the dirty list pointing into it): same serialized images as the oracle,
    device-side restore of the chain, in the hash kernel's direct (512 B -
    8 KiB) and segmented (64, 256 KiB) modes, in one or several staging
    segments.  All sizes are multiples of 16 bytes, so the pass is sparse."""
    sizes = [16, 4096, S * 5 + 48, 3 * S, 100000 // 16 * 16, S + 16]
    h = Harness(S, lineage=700 + S % 97, pass_kernel=C.CRAC_PASS_SPARSE, staging_bytes=staging,
                image_residency=C.CRAC_RESIDENCY_DEVICE)
    try:
        for i, n in enumerate(sizes):
            h.add(n, seed=120 + i)
        _, lib1, ora1 = h.checkpoint()
        assert lib1 == ora1
        assert C.crac_ctx_last_pass(h.ctx)["pass_kernel"] == C.CRAC_PASS_SPARSE
        imgs = []
        for seed in (1, 2):
            muts = pattern_mutations(h.first(), sizes, S, pattern, seed=seed)
            h.mutate(muts)
            img, lib, ora = h.checkpoint()
            assert lib == ora
            assert O.parse_image(lib).idx.tolist() == sorted(m.chunk for m in muts)
            info = C.crac_ctx_last_pass(h.ctx)
            assert info["pass_kernel"] == C.CRAC_PASS_SPARSE
            assert info["payload_bytes"] == C.crac_image_info(img)["payload_bytes"]
            imgs.append(img)
        want = h.host()
        for b in h.bufs:
            b.zero()
        h.restart(imgs[-1])
        for b, w in zip(h.bufs, want):
            assert np.array_equal(b.read(), w)
        _, lib4, ora4 = h.checkpoint()   # the restored image is the baseline
        assert lib4 == ora4 and O.parse_image(lib4).k == 0
    finally:
        h.close()


@pytest.mark.parametrize("S", [512, 1 * KIB, 4 * KIB])
def test_sparse_dirty_only_with_new_allocation(S):
    """On 512 B - 4 KiB chunks the sparse pass stores only the dirty chunks:
    at their uncompacted offsets, or, after a delta that found under a
    quarter of the chunks dirty, back to back in the order the warps reach
    them.  Deltas that mix baselined chunks with a newly registered
    allocation's (no baseline, all dirty) -- the first with uncompacted
    placement, the second with dense placement -- give the oracle's images
    with the dirty bytes as payload, the scattered chunks serialize back
    into chunk order, and the chain restores on the device and from
    deserialized copies."""
    sizes = [S * 37 + 16 * 3, 4096 * 5, 48000 // 16 * 16]
    h = Harness(S, lineage=740 + S // 256, pass_kernel=C.CRAC_PASS_SPARSE,
                image_residency=C.CRAC_RESIDENCY_DEVICE)
    try:
        for i, n in enumerate(sizes):
            h.add(n, seed=170 + i)
        libs, oras, imgs = [], [], []
        _, lib1, ora1 = h.checkpoint()
        assert lib1 == ora1
        libs.append(lib1)
        oras.append(ora1)
        for step, (extra, pattern) in enumerate(((S * 2 + 32, "random10"), (S * 3 + 16, "random10"),
                                                 (None, "alternating"))):
            if extra:
                h.add(extra, seed=180 + step)   # registered after the last image: no baseline
            h.mutate(pattern_mutations(h.first(), [b.nbytes for b in h.bufs], S, pattern, seed=4 + step))
            img, lib, ora = h.checkpoint()
            assert lib == ora, step
            assert C.crac_ctx_last_pass(h.ctx)["pass_kernel"] == C.CRAC_PASS_SPARSE
            assert C.crac_image_info(img)["payload_bytes"] == len(O.parse_image(ora).payload)
            libs.append(lib)
            oras.append(ora)
            imgs.append(img)
        want = h.host()
        for b in h.bufs:
            b.zero()
        h.restart(imgs[-1])
        for b, w in zip(h.bufs, want):
            assert np.array_equal(b.read(), w)
        # the same chain from deserialized copies, in a fresh context
        h2 = Harness(S, lineage=999)
        try:
            for b in h.bufs:
                h2.add(b.nbytes, data=np.zeros(b.nbytes, dtype=np.uint8))
            ds = [C.crac_image_deserialize(x) for x in libs]
            h2.images += ds
            h2.restart(ds[-1], oras)
            for b, w in zip(h2.bufs, want):
                assert np.array_equal(b.read(), w)
            _, lib5, ora5 = h2.checkpoint()   # the restored image is the baseline
            assert lib5 == ora5 and O.parse_image(lib5).k == 0
        finally:
            h2.close()
    finally:
        h.close()


@pytest.mark.parametrize("flags", [0, C.CRAC_FLAG_STAGED_RESTORE])
def test_sparse_pass_fallback_and_mixed_chain(flags):
    """A size that is not a multiple of 16 makes the sparse kernel choice run
    the compacting split pass.  And a chain whose FULL image comes back from
    serialization (host-resident) and whose delta is a sparse device image is
    restored through the host path, which reads the sparse offsets."""
    S = 4 * KIB
    dev = {"pass_kernel": C.CRAC_PASS_SPARSE, "image_residency": C.CRAC_RESIDENCY_DEVICE}
    h = Harness(S, lineage=711, **dev)
    try:
        h.add(40000, seed=1)
        h.add(12345, seed=2)
        for pattern in (None, "alternating"):
            if pattern:
                h.mutate(pattern_mutations(h.first(), [b.nbytes for b in h.bufs], S, pattern, seed=4))
            _, lib, ora = h.checkpoint()
            assert lib == ora
            assert C.crac_ctx_last_pass(h.ctx)["pass_kernel"] == C.CRAC_PASS_SPLIT
    finally:
        h.close()
    sizes = [40000, 12352, 4096 * 3]
    h1 = Harness(S, lineage=712, **dev)
    h2 = Harness(S, lineage=713, flags=flags, **dev)
    try:
        for i, n in enumerate(sizes):
            h1.add(n, seed=10 + i)
            h2.add(n, data=np.zeros(n, dtype=np.uint8))
        _, lib1, ora1 = h1.checkpoint()
        assert lib1 == ora1
        full = C.crac_image_deserialize(lib1)
        h2.images.append(full)
        h2.restart(full, [ora1])
        assert C.crac_image_info(full)["residency"] == C.CRAC_RESIDENCY_HOST
        h2.mutate(pattern_mutations(h2.first(), sizes, S, "alternating", seed=6))
        img2, lib2, ora2 = h2.checkpoint()
        assert lib2 == ora2 and O.parse_image(lib2).k > 0
        assert C.crac_ctx_last_pass(h2.ctx)["pass_kernel"] == C.CRAC_PASS_SPARSE
        want = h2.host()
        for b in h2.bufs:
            b.zero()
        h2.restart(img2)
        assert C.crac_ctx_last_restart(h2.ctx)["chain_length"] == 2
        for b, w in zip(h2.bufs, want):
            assert np.array_equal(b.read(), w)
    finally:
        h2.close()
        h1.close()


@pytest.mark.parametrize("residency,S,mostly_dirty_kernel", [
    (C.CRAC_RESIDENCY_DEVICE, 4 * KIB, C.CRAC_PASS_SPARSE),
    (C.CRAC_RESIDENCY_HOST, 4 * KIB, C.CRAC_PASS_TMA),
    (C.CRAC_RESIDENCY_HOST, 256 * KIB, C.CRAC_PASS_LDG)])
def test_auto_follows_dirty_fraction(residency, S, mostly_dirty_kernel):
    """CRAC_PASS_AUTO runs the split pass until a pass with a baseline finds
    more than half of the chunks dirty, then the kernel that reads each byte
    once (sparse for device images, else TMA, else LDG), and back to split
    after a sparse delta -- except on 4 KiB chunks of device images, where a
    delta with under a quarter of the chunks dirty is followed by the sparse
    pass with dense placement; every image stays the oracle's."""
    sizes = [S * 40, S * 3 + 16 * 5, 4096 * 7]
    h = Harness(S, lineage=720 + S // KIB, image_residency=residency)
    try:
        for i, n in enumerate(sizes):
            h.add(n, seed=140 + i)
        kernels = []
        for pattern in (None, "all", "random10", "random10"):
            if pattern:
                h.mutate(pattern_mutations(h.first(), sizes, S, pattern, seed=len(kernels) + 1))
            img, lib, ora = h.checkpoint()
            assert lib == ora, pattern
            kernels.append(C.crac_ctx_last_pass(h.ctx)["pass_kernel"])
        # FULL (no dirty fraction yet), the all-dirty delta (split), then the
        # kernel for mostly dirty memory, then split again
        low_dirty_kernel = (C.CRAC_PASS_SPARSE if residency == C.CRAC_RESIDENCY_DEVICE and S <= 4 * KIB
                            else C.CRAC_PASS_SPLIT)
        assert kernels == [C.CRAC_PASS_SPLIT, C.CRAC_PASS_SPLIT, mostly_dirty_kernel, low_dirty_kernel]
        want = h.host()
        for b in h.bufs:
            b.zero()
        h.restart(img)
        for b, w in zip(h.bufs, want):
            assert np.array_equal(b.read(), w)
    finally:
        h.close()


def test_sparse_kernel_with_per_allocation_launches():
    """CRAC_PASS_SPARSE under CRAC_LAUNCH_PER_ALLOC: the per-allocation path
    runs (it compacts) and the images are the oracle's."""
    S = 4 * KIB
    sizes = [50000 // 16 * 16, 4096 * 9, 16 * 1000]
    h = Harness(S, lineage=730, pass_kernel=C.CRAC_PASS_SPARSE, image_residency=C.CRAC_RESIDENCY_DEVICE,
                launch_mode=C.CRAC_LAUNCH_PER_ALLOC)
    try:
        for i, n in enumerate(sizes):
            h.add(n, seed=150 + i)
        _, lib1, ora1 = h.checkpoint()
        assert lib1 == ora1
        h.mutate(pattern_mutations(h.first(), sizes, S, "random10", seed=3))
        img, lib2, ora2 = h.checkpoint()
        assert lib2 == ora2
        want = h.host()
        for b in h.bufs:
            b.zero()
        h.restart(img)
        for b, w in zip(h.bufs, want):
            assert np.array_equal(b.read(), w)
    finally:
        h.close()


@pytest.mark.parametrize("kern,residency,flags", [
    (C.CRAC_PASS_AUTO, C.CRAC_RESIDENCY_HOST, 0),
    (C.CRAC_PASS_LDG, C.CRAC_RESIDENCY_DEVICE, C.CRAC_FLAG_INCREMENTAL_RESTORE),
    (C.CRAC_PASS_TMA, C.CRAC_RESIDENCY_HOST, C.CRAC_FLAG_STAGED_RESTORE),
    (C.CRAC_PASS_SPARSE, C.CRAC_RESIDENCY_DEVICE, 0),
    (C.CRAC_PASS_SPLIT, C.CRAC_RESIDENCY_HOST, C.CRAC_FLAG_DIRECT_DRAIN | C.CRAC_FLAG_INCREMENTAL_RESTORE)])
def test_host_kind_allocations(kern, residency, flags):
    """Page-locked host allocations (CRAC_KIND_HOST) next to device and
    managed ones: the pass hashes and gathers them through their device
    mapping and the restore writes them back the same way."""
    S = 4 * KIB
    h = Harness(S, lineage=740 + kern, pass_kernel=kern, image_residency=residency, flags=flags)
    try:
        kinds = [C.CRAC_KIND_HOST, C.CRAC_KIND_DEVICE, C.CRAC_KIND_HOST, C.CRAC_KIND_MANAGED]
        sizes = [S * 20, S * 7 + 32, 100000 // 16 * 16, S * 3]
        for i, (n, k) in enumerate(zip(sizes, kinds)):
            h.add(n, kind=k, seed=160 + i)
        _, lib1, ora1 = h.checkpoint()
        assert lib1 == ora1
        assert [a[3] for a in O.parse_image(lib1).allocs] == kinds
        for seed, pattern in ((1, "random10"), (2, "alternating")):
            h.mutate(pattern_mutations(h.first(), sizes, S, pattern, seed=seed))
            img, lib, ora = h.checkpoint()
            assert lib == ora
        want = h.host()
        for b in h.bufs:
            b.zero()
        h.restart(img)
        for b, w in zip(h.bufs, want):
            assert np.array_equal(b.read(), w)
    finally:
        h.close()


@pytest.mark.parametrize("n_allocs", [3072, 3073])
@pytest.mark.parametrize("residency", [C.CRAC_RESIDENCY_HOST, C.CRAC_RESIDENCY_DEVICE])
def test_tma_many_allocations(n_allocs, residency):
    """The TMA pass keeps the allocations' first_chunk column in shared memory
    up to 3072 allocations and searches the table in global memory beyond;
    both give the oracle's images.  The allocations are 256-byte-aligned
    pieces of one device buffer, with ragged sizes."""
    S = 4 * KIB
    rng = np.random.default_rng(n_allocs + residency)
    sizes = [int(x) for x in rng.integers(1, 3 * S, size=n_allocs)]
    offs = np.zeros(n_allocs + 1, dtype=np.int64)
    offs[1:] = np.cumsum([(n + 255) // 256 * 256 for n in sizes])
    buf = torch.from_numpy(W.host_contents("u32_xorshift", int(offs[-1]), 77)).to("cuda")
    base = buf.data_ptr()
    ctx = C.crac_ctx_create(C.crac_config_default(chunk_bytes=S, lineage=600 + n_allocs % 7,
                                                  pass_kernel=C.CRAC_PASS_TMA, image_residency=residency))
    ora = O.OracleContext(S, lineage=600 + n_allocs % 7)
    stream = torch.cuda.current_stream()
    imgs = []

    def host():
        h = buf.cpu().numpy()
        return [h[offs[i]:offs[i] + n] for i, n in enumerate(sizes)]

    def checkpoint():
        img = C.crac_ctx_checkpoint(ctx, stream)
        imgs.append(img)
        C.crac_image_wait(img)
        assert C.crac_ctx_last_pass(ctx)["pass_kernel"] == C.CRAC_PASS_TMA
        return img, C.crac_image_serialize(img), ora.checkpoint(host())

    try:
        for i, n in enumerate(sizes):
            C.crac_ctx_register_alloc(ctx, base + int(offs[i]), n)
            ora.register(base + int(offs[i]), n)
        _, lib1, ora1 = checkpoint()
        assert lib1 == ora1
        first = W.chunk_layout(sizes, S)
        muts = pattern_mutations(first, sizes, S, "random10", seed=n_allocs)
        rows = []
        for m in muts:
            a = int(np.searchsorted(first, m.chunk, side="right") - 1)
            lo = (m.chunk - int(first[a])) * S
            rows.append((base + int(offs[a]) + lo, min(S, sizes[a] - lo), m.mask))
        ent = torch.from_numpy(np.array(rows, dtype=np.uint64).view(np.int64)).to("cuda")
        testkit.mutate_xor(ent.data_ptr(), len(rows), stream)
        torch.cuda.synchronize()
        img2, lib2, ora2 = checkpoint()
        assert lib2 == ora2
        assert O.parse_image(lib2).idx.tolist() == sorted(m.chunk for m in muts)
        want = buf.clone()
        buf.zero_()
        C.crac_ctx_restart(ctx, img2, stream)
        torch.cuda.synchronize()
        for i, n in enumerate(sizes):   # the 256-byte padding between allocations stays zero
            assert torch.equal(buf[offs[i]:offs[i] + n], want[offs[i]:offs[i] + n])
    finally:
        torch.cuda.synchronize()
        for img in imgs:
            C.crac_image_release(img)
        C.crac_ctx_destroy(ctx)


@pytest.mark.parametrize("mode", ["per_alloc", "segments", "device", "device_segments", "staged",
                                  "staged_segments", "direct", "direct_segments", "direct_per_alloc"])
def test_launch_modes_and_residency(mode):
    """Launch modes, staging segments and residencies.  Host images are
    restored in place from pinned memory unless CRAC_FLAG_STAGED_RESTORE
    asks for the copy-engine path through staging windows."""
    S = 4 * KIB
    cfg = {}
    if mode.startswith("staged"):
        cfg["flags"] = C.CRAC_FLAG_STAGED_RESTORE
    if mode.startswith("direct"):      # host images written straight into pinned memory
        cfg["flags"] = C.CRAC_FLAG_DIRECT_DRAIN
    if mode == "per_alloc":
        cfg["launch_mode"] = C.CRAC_LAUNCH_PER_ALLOC
    if mode in ("segments", "device_segments", "staged_segments", "direct_segments"):
        cfg["staging_bytes"] = 40 * KIB      # forces many segments, allocations split
    if mode == "direct_per_alloc":
        cfg["launch_mode"] = C.CRAC_LAUNCH_PER_ALLOC
    if mode.startswith("device"):
        cfg["image_residency"] = C.CRAC_RESIDENCY_DEVICE
    sizes = [100000, 4096, 77, 250000, 8192 * 3 + 1]
    h = Harness(S, lineage=9, **cfg)
    try:
        for i, n in enumerate(sizes):
            h.add(n, seed=50 + i)
        img1, lib1, ora1 = h.checkpoint()
        assert lib1 == ora1
        h.mutate(pattern_mutations(h.first(), sizes, S, "random10", seed=4))
        img2, lib2, ora2 = h.checkpoint()
        assert lib2 == ora2
        h.mutate(pattern_mutations(h.first(), sizes, S, "alternating", seed=5))
        img3, lib3, ora3 = h.checkpoint()
        assert lib3 == ora3
        want = h.host()
        for b in h.bufs:
            b.zero()
        h.restart(img3)
        for b, w in zip(h.bufs, want):
            assert np.array_equal(b.read(), w)
        # the restored image is the baseline: an unmodified checkpoint is empty
        _, lib4, ora4 = h.checkpoint()
        assert lib4 == ora4 and O.parse_image(lib4).k == 0
        info = C.crac_ctx_last_restart(h.ctx)
        assert info["chain_length"] == 3 and info["restored_bytes"] == sum(sizes)
        if mode in ("per_alloc", "direct_per_alloc"):
            info = C.crac_ctx_last_pass(h.ctx)
            assert info["kernel_launches"] == 3 * len(sizes) + 1   # + the control-block report
    finally:
        h.close()


def test_register_free_between_checkpoints_and_chain_restore():
    S = 4 * KIB
    h = Harness(S, lineage=77)
    try:
        for i, n in enumerate([5000, 20000, 4096]):
            h.add(n, seed=70 + i)
        _, lib1, ora1 = h.checkpoint()
        assert lib1 == ora1
        h.free(1)
        h.add(9000, seed=80)
        h.mutate(pattern_mutations(h.first(), [b.nbytes for b in h.bufs], S, "first"))
        img2, lib2, ora2 = h.checkpoint()
        assert lib2 == ora2
        assert [a[0] for a in O.parse_image(lib2).allocs] == [0, 2, 3]
        want = h.host()
        # restore the chain in a fresh context from deserialized images
        h2 = Harness(S, lineage=999)
        try:
            for b in h.bufs:
                h2.add(b.nbytes, data=np.zeros(b.nbytes, dtype=np.uint8))
            d1 = C.crac_image_deserialize(lib1)
            d2 = C.crac_image_deserialize(lib2)
            h2.images += [d1, d2]
            h2.restart(d2, [ora1, ora2])
            for b, w in zip(h2.bufs, want):
                assert np.array_equal(b.read(), w)
            # the fresh context continues the lineage; an unmodified checkpoint is empty
            _, lib3, ora3 = h2.checkpoint()
            assert lib3 == ora3
            im3 = O.parse_image(lib3)
            assert im3.k == 0 and im3.lineage == 77 and im3.parent_epoch == 2
        finally:
            h2.close()
    finally:
        h.close()


def test_managed_allocations():
    S = 64 * KIB
    h = Harness(S, lineage=31)
    try:
        h.add(300000, seed=1)
        h.add(200000, kind=C.CRAC_KIND_MANAGED, seed=2)
        h.add(64 * KIB, kind=C.CRAC_KIND_MANAGED, seed=3)
        _, lib1, ora1 = h.checkpoint()
        assert lib1 == ora1
        assert [a[3] for a in O.parse_image(lib1).allocs] == [0, 1, 1]
        h.mutate(pattern_mutations(h.first(), [b.nbytes for b in h.bufs], S, "alternating"))
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


def test_restart_rejects_mismatch_and_leaves_memory():
    S = 4 * KIB
    h = Harness(S, lineage=3)
    try:
        h.add(10000, seed=1)
        img, _, _ = h.checkpoint()
        h2 = Harness(S, lineage=4)
        try:
            b = h2.add(10001, seed=2)
            before = b.read()
            with pytest.raises(C.CracError) as e:
                C.crac_ctx_restart(h2.ctx, img, h2.stream)
            assert e.value.code == C.CRAC_ERR_IMAGE_MISMATCH
            assert np.array_equal(b.read(), before)
        finally:
            h2.close()
        h3 = Harness(64, lineage=4)
        try:
            h3.add(10000, seed=2)
            with pytest.raises(C.CracError) as e:
                C.crac_ctx_restart(h3.ctx, img, h3.stream)
            assert e.value.code == C.CRAC_ERR_IMAGE_MISMATCH
        finally:
            h3.close()
    finally:
        h.close()


def test_default_context_forms():
    S = 64 * KIB
    t = torch.empty(100000, dtype=torch.uint8, device="cuda")
    data = W.host_contents("u8", 100000, 5)
    t.copy_(torch.from_numpy(data))
    C.crac_register_alloc(t.data_ptr(), 100000, C.CRAC_KIND_DEVICE)
    try:
        img = C.crac_checkpoint(torch.cuda.current_stream())
        C.crac_image_wait(img)
        info = C.crac_image_info(img)
        assert info["flags"] & C.CRAC_IMAGE_FULL and info["payload_bytes"] == 100000
        assert info["chunk_bytes"] == S and info["complete"] == 1
        t.zero_()
        C.crac_restart(img, None)
        torch.cuda.synchronize()
        assert np.array_equal(t.cpu().numpy(), data)
        C.crac_image_release(img)
    finally:
        C.crac_free(t.data_ptr())


def test_empty_registry():
    h = Harness(4 * KIB, lineage=12)
    try:
        img, lib, ora = h.checkpoint()
        assert lib == ora
        assert O.parse_image(lib).n_chunks == 0
        h.restart(img)
    finally:
        h.close()


@pytest.mark.parametrize("S", [1 * KIB, 4 * KIB, 8 * KIB, 64 * KIB])
@pytest.mark.parametrize("staging", [0, 300 * KIB])
def test_full_checkpoint_write_through(S, staging):
    """FULL checkpoints with every size a multiple of 16: the hash kernel writes
    chunks straight to their staging offsets (segments starting mid-allocation
    included) and the gather is skipped; the image must still be the oracle's."""
    sizes = [16 * 4097, S * 5, 48, 1024 * KIB + 16 * 3, S * 2 + 32]
    h = Harness(S, lineage=400 + S // KIB, staging_bytes=staging, pass_kernel=C.CRAC_PASS_SPLIT)
    try:
        for i, n in enumerate(sizes):
            h.add(n, seed=120 + i)
        img1, lib1, ora1 = h.checkpoint()
        assert lib1 == ora1
        h.mutate(pattern_mutations(h.first(), sizes, S, "random10", seed=6))
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
