"""Randomized parity cases (GPU): for each seed a random registry (count,
sizes from 1 byte to ~1 MiB, some 16-byte multiples), a random chunk size,
pass kernel, residency, staging capacity and flags (coded images included), then a random sequence of
mutations, registrations and frees over several checkpoints.  Every image
must serialize to the oracle's bytes, and a restart of the last image must
bring back the memory exactly."""
import numpy as np
import pytest

import paper_2008_10596_gb300 as C
from tests.gpu_harness import Harness, pattern_mutations

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("oracle_lib")]

KIB = 1024
PATTERNS = ["none", "all", "first", "last", "tail", "alternating", "random10"]
KERNELS = [C.CRAC_PASS_AUTO, C.CRAC_PASS_SPLIT, C.CRAC_PASS_LDG, C.CRAC_PASS_TMA, C.CRAC_PASS_SPARSE]


def _case(seed):
    rng = np.random.default_rng(9000 + seed)
    kern = KERNELS[seed % len(KERNELS)]
    if kern == C.CRAC_PASS_TMA:
        S = int(rng.choice([1, 2, 4, 16, 64])) * KIB
    else:
        S = int(rng.choice([256, 512, 1 * KIB, 4 * KIB, 8 * KIB, 64 * KIB, 256 * KIB]))
    cfg = {"pass_kernel": kern}
    if kern == C.CRAC_PASS_SPARSE or rng.random() < 0.3:
        cfg["image_residency"] = C.CRAC_RESIDENCY_DEVICE
    if rng.random() < 0.3:
        cfg["staging_bytes"] = int(max(S, rng.integers(S, 64 * S)))
    flags = 0
    if cfg.get("image_residency", C.CRAC_RESIDENCY_HOST) == C.CRAC_RESIDENCY_HOST:
        if rng.random() < 0.4:
            flags |= C.CRAC_FLAG_DIRECT_DRAIN
        if rng.random() < 0.3:
            flags |= C.CRAC_FLAG_STAGED_RESTORE
    if rng.random() < 0.3:
        flags |= C.CRAC_FLAG_INCREMENTAL_RESTORE
    cfg["flags"] = flags
    if kern == C.CRAC_PASS_LDG and rng.random() < 0.5:
        cfg["chunks_per_tile"] = int(rng.integers(1, 40))
    # coded images, drawn from a generator of their own so that the other
    # draws of each seed stay as they were
    if kern != C.CRAC_PASS_SPARSE and np.random.default_rng(77000 + seed).random() < 0.35:
        cfg["flags"] |= C.CRAC_FLAG_COMPRESS
    return rng, S, cfg


def _size(rng, aligned):
    n = int(np.exp(rng.uniform(0, np.log(1 << 20))))
    return max(16, n // 16 * 16) if aligned else max(1, n)


@pytest.mark.parametrize("seed", range(48))
def test_random_registry_and_mutations(seed):
    rng, S, cfg = _case(seed)
    aligned = cfg["pass_kernel"] == C.CRAC_PASS_SPARSE and rng.random() < 0.8
    h = Harness(S, lineage=5000 + seed, **cfg)
    try:
        for i in range(int(rng.integers(1, 12))):
            h.add(_size(rng, aligned), seed=seed * 100 + i + 1)
        img, lib, ora = h.checkpoint()
        assert lib == ora
        for step in range(3):
            r = rng.random()
            if r < 0.2 and len(h.bufs) > 1:
                h.free(int(rng.integers(0, len(h.bufs))))
            elif r < 0.4:
                h.add(_size(rng, aligned), seed=seed * 100 + 51 + step)
            pattern = PATTERNS[int(rng.integers(0, len(PATTERNS)))]
            h.mutate(pattern_mutations(h.first(), [b.nbytes for b in h.bufs], S, pattern,
                                       seed=seed * 7 + step + 1))
            img, lib, ora = h.checkpoint()
            assert lib == ora, (step, pattern)
        want = h.host()
        for b in h.bufs:
            b.zero()
        h.restart(img)
        for b, w in zip(h.bufs, want):
            assert np.array_equal(b.read(), w)
    finally:
        h.close()
