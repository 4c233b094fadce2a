"""Incremental restore (GPU): with CRAC_FLAG_INCREMENTAL_RESTORE a restart
fingerprints the current memory against the target image's table and
rewrites only the chunks that differ.  The memory must come back exactly as
at the checkpoint, the count of rewritten chunks must be exactly the chunks
changed since (integer work: compared exactly), and the next checkpoint must
be the oracle's (empty)."""
import numpy as np
import pytest

import paper_2008_10596_gb300 as C
from oracle import oracle as O
from tests.gpu_harness import Harness, pattern_mutations

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("oracle_lib")]

KIB = 1024


@pytest.mark.parametrize("residency", [C.CRAC_RESIDENCY_DEVICE, C.CRAC_RESIDENCY_HOST])
@pytest.mark.parametrize("S", [4 * KIB, 64 * KIB])
@pytest.mark.parametrize("scenario", ["unchanged", "mutated", "zeroed", "chain"])
def test_incremental_restore(residency, S, scenario):
    sizes = [S * 30 + 48, 7 * 4096, S * 5, 100000]
    h = Harness(S, lineage=900 + S // KIB, image_residency=residency, flags=C.CRAC_FLAG_INCREMENTAL_RESTORE)
    try:
        for i, n in enumerate(sizes):
            h.add(n, seed=200 + i)
        img_a, lib_a, ora_a = h.checkpoint()
        assert lib_a == ora_a
        m1 = pattern_mutations(h.first(), sizes, S, "random10", seed=11)
        h.mutate(m1)
        img_b, lib_b, ora_b = h.checkpoint()
        assert lib_b == ora_b
        target, want = img_b, h.host()
        n_chunks = int(h.first()[-1])
        if scenario == "unchanged":
            expect = 0
        elif scenario == "mutated":
            m = pattern_mutations(h.first(), sizes, S, "random10", seed=12)
            h.mutate(m)
            expect = len({x.chunk for x in m})
        elif scenario == "zeroed":
            for b in h.bufs:
                b.zero()
            expect = n_chunks
        else:   # roll back one image along a chain, after further changes
            m2 = pattern_mutations(h.first(), sizes, S, "alternating", seed=13)
            h.mutate(m2)
            _, lib_c, ora_c = h.checkpoint()
            assert lib_c == ora_c
            m3 = pattern_mutations(h.first(), sizes, S, "tail", seed=14)
            h.mutate(m3)
            expect = len({x.chunk for x in m2} | {x.chunk for x in m3})
        h.restart(target)
        info = C.crac_ctx_last_restart(h.ctx)
        for b, w in zip(h.bufs, want):
            assert np.array_equal(b.read(), w)
        assert info["chunks_rewritten"] == expect
        # the restored image is the baseline: an unmodified checkpoint is empty,
        # and it is the oracle's once the oracle has restored the same chain
        h.oracle.restart([lib_a, lib_b])
        _, lib_d, ora_d = h.checkpoint()
        assert lib_d == ora_d and O.parse_image(lib_d).k == 0
    finally:
        h.close()


def test_incremental_flag_ignored_on_staged_path():
    """The staged host path restores every chunk even with the flag."""
    S = 4 * KIB
    h = Harness(S, lineage=950, flags=C.CRAC_FLAG_INCREMENTAL_RESTORE | C.CRAC_FLAG_STAGED_RESTORE)
    try:
        h.add(50000, seed=1)
        img, lib, ora = h.checkpoint()
        want = h.host()
        h.restart(img)
        info = C.crac_ctx_last_restart(h.ctx)
        assert info["chunks_rewritten"] == int(h.first()[-1])
        assert np.array_equal(h.bufs[0].read(), want[0])
    finally:
        h.close()
