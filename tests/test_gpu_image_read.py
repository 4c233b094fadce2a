"""Ranged reads of an image, and contexts that do not keep their images (GPU).

crac_image_read must return exactly the bytes crac_image_serialize writes,
for any range: host images, device images (compact split pass and the
uncompacted sparse pass, whose payload is compacted on the way out) and
coded images; ranges that cross section boundaries, empty ranges, and ranges
past the end (rejected).  crac_ctx_drop_history lets the context forget its
newest image while keeping the baseline: the next delta equals the oracle's,
restores only once its parent is loaded again, and then gives the memory the
oracle restores.
"""
import numpy as np
import pytest

import paper_2008_10596_gb300 as C
from tests.gpu_harness import Harness, pattern_mutations

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("oracle_lib")]

KIB = 1024
SIZES = [100 * KIB + 48, 16, 3 * 64 * KIB, 4096 * 5, 777 * 16]


def _fill(h, S):
    for i, n in enumerate(SIZES):
        h.add(n, seed=300 + i)


def _ranges(total, seed):
    rng = np.random.default_rng(seed)
    cuts = sorted(set([0, total] + rng.integers(0, total + 1, size=12).tolist()))
    return list(zip(cuts[:-1], cuts[1:]))


@pytest.mark.parametrize("mode", ["host", "device_split", "device_sparse", "coded_host", "coded_device"])
def test_ranges_equal_serialization(mode):
    S = 4 * KIB
    cfg = {}
    if mode.startswith("device"):
        cfg["image_residency"] = C.CRAC_RESIDENCY_DEVICE
    if mode == "device_sparse":
        cfg["pass_kernel"] = C.CRAC_PASS_SPARSE
    if mode.startswith("coded"):
        cfg["flags"] = C.CRAC_FLAG_COMPRESS
        if mode == "coded_device":
            cfg["image_residency"] = C.CRAC_RESIDENCY_DEVICE
    h = Harness(S, lineage=2100, **cfg)
    try:
        _fill(h, S)
        img0, lib0, ora0 = h.checkpoint()
        assert lib0 == ora0
        h.mutate(pattern_mutations(h.first(), SIZES, S, "alternating", seed=4))
        img1, lib1, ora1 = h.checkpoint()
        assert lib1 == ora1
        for img, raw in ((img0, lib0), (img1, lib1)):
            total = C.crac_image_info(img)["serialized_bytes"]
            assert total == len(raw)
            parts = [C.crac_image_read(img, a, b - a) for a, b in _ranges(total, 5)]
            assert b"".join(parts) == raw
            out = np.zeros(total, dtype=np.uint8)
            C.crac_image_read(img, 0, total, out=out)
            assert out.tobytes() == raw
            assert C.crac_image_read(img, total, 0) == b""
            for a, n in ((total, 1), (total - 3, 4), (1 << 62, 1)):
                with pytest.raises(C.CracError) as e:
                    C.crac_image_read(img, a, n)
                assert e.value.code == C.CRAC_ERR_INVALID_ARG
    finally:
        h.close()


@pytest.mark.parametrize("residency", [C.CRAC_RESIDENCY_HOST, C.CRAC_RESIDENCY_DEVICE])
def test_drop_history_keeps_the_baseline(residency):
    S = 4 * KIB
    h = Harness(S, lineage=2200, image_residency=residency)
    try:
        _fill(h, S)
        img0, lib0, ora0 = h.checkpoint()
        assert lib0 == ora0
        C.crac_ctx_drop_history(h.ctx)
        C.crac_image_release(h.images.pop(0))     # nothing holds the FULL image now
        h.mutate(pattern_mutations(h.first(), SIZES, S, "random10", seed=8))
        want = h.host()
        img1, lib1, ora1 = h.checkpoint()
        assert lib1 == ora1                       # still a delta against the dropped image
        assert not C.crac_image_info(img1)["flags"] & C.CRAC_IMAGE_FULL
        for b in h.bufs:
            b.zero()
        with pytest.raises(C.CracError) as e:     # its parent is gone
            C.crac_ctx_restart(h.ctx, img1, h.stream)
        assert e.value.code == C.CRAC_ERR_IMAGE_MISMATCH
        back = C.crac_image_deserialize(lib0)     # the parent, loaded again from its bytes
        try:
            h.restart(img1, [lib0, lib1])
            for b, w in zip(h.bufs, want):
                assert np.array_equal(b.read(), w)
        finally:
            C.crac_image_release(back)
    finally:
        h.close()
