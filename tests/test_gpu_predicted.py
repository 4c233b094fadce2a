"""Predicted write-through of the split pass (GPU).

A single-segment split pass records the staging offset of every dirty chunk;
the next pass's hash kernel writes the chunks that were dirty last time to
those offsets as it reads them, and its gather leaves an entry alone when
its offset is the predicted one.  Whatever the prediction -- exact, a
superset, a subset, disjoint -- every image must equal the oracle's.  When
the dirty set repeats, the entries are found in place (pass info
in_place); a chunk whose predicted offset is not 16-byte aligned (behind a
ragged chunk) is gathered as before.  After a prediction that found fewer
than half of the entries in place the context stops speculating for a few
passes.
"""
import numpy as np
import pytest

import paper_2008_10596_gb300 as C
import workloads as W
from tests.gpu_harness import Harness

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("oracle_lib")]


def _sets(n, seed):
    rng = np.random.default_rng(seed)
    perm = rng.permutation(n)
    a = sorted(perm[: n // 10].tolist())
    b = sorted(perm[n // 10: n // 10 + n // 20].tolist())
    d = sorted(perm[n // 2: n // 2 + n // 10].tolist())
    return a, b, d


def _muts(ids, seed):
    rng = W.XorShift64(seed)
    return [W.ChunkMutation(c, rng.mask32()) for c in ids]


@pytest.mark.parametrize("residency", [C.CRAC_RESIDENCY_HOST, C.CRAC_RESIDENCY_DEVICE])
@pytest.mark.parametrize("S,ragged", [(256, False), (4096, False), (4096, True), (65536, False), (65536, True)])
def test_prediction_exact_superset_subset_disjoint(S, ragged, residency):
    sizes = [S * 300, S * 41, S * 7 + (5 if ragged else 0), S * 120 + (1000 if ragged else 0), S * 2]
    h = Harness(S, lineage=90, image_residency=residency, pass_kernel=C.CRAC_PASS_SPLIT)
    try:
        for i, n in enumerate(sizes):
            h.add(n, seed=40 + i)
        _, lib, ora = h.checkpoint()
        assert lib == ora
        n = int(h.first()[-1])
        a, b, d = _sets(n, S)
        plan = [("first", a), ("exact", a), ("superset", sorted(set(a) | set(b))), ("subset", a[::2]),
                ("disjoint", d), ("after a poor prediction", d)]
        for step, (name, ids) in enumerate(plan):
            h.mutate(_muts(ids, 1000 + step))
            _, lib, ora = h.checkpoint()
            assert lib == ora, f"{name}: image differs from the oracle"
            info = C.crac_ctx_last_pass(h.ctx)
            assert info["k"] == len(ids) and info["pass_kernel"] == C.CRAC_PASS_SPLIT
            if name == "first":
                assert info["in_place"] == 0          # nothing predicted yet (after a FULL image)
            elif name == "exact" and not ragged:
                assert info["in_place"] == len(ids)   # every entry was written as it was read
            elif name == "exact":
                assert 0 < info["in_place"] <= len(ids)
            elif name == "disjoint":
                assert info["in_place"] == 0
            elif name == "after a poor prediction":
                assert info["in_place"] == 0          # speculation paused
        # the chain restores the last state
        want = h.host()
        for bb in h.bufs:
            bb.zero()
        h.restart(h.images[-1])
        for bb, w in zip(h.bufs, want):
            assert np.array_equal(bb.read(), w)
    finally:
        h.close()


def test_prediction_is_dropped_when_the_layout_changes():
    """A registration between passes changes the chunk layout: the next pass
    predicts nothing, and its image still equals the oracle's."""
    S = 4096
    h = Harness(S, lineage=91, pass_kernel=C.CRAC_PASS_SPLIT)
    try:
        for i, n in enumerate([S * 100, S * 50]):
            h.add(n, seed=60 + i)
        h.checkpoint()
        ids = list(range(0, 150, 7))
        for step in range(2):
            h.mutate(_muts(ids, 2000 + step))
            _, lib, ora = h.checkpoint()
            assert lib == ora
        assert C.crac_ctx_last_pass(h.ctx)["in_place"] == len(ids)
        h.add(S * 3, seed=70)                 # new allocation: new layout
        h.mutate(_muts(ids, 2100))
        _, lib, ora = h.checkpoint()
        assert lib == ora
        assert C.crac_ctx_last_pass(h.ctx)["in_place"] == 0
    finally:
        h.close()
