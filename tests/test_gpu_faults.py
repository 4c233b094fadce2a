"""Failure handling without any GPU fault (GPU).

Failures are made on the host (fault injection at named steps) or by a
device wait that is made to run out: the batched kernel is launched so that
tile 0 is never processed, so tile 1's bounded look-back wait expires; the
kernel then finishes and reports CRAC_ERR_TIMEOUT (from the checkpoint call,
or, for a pass the call did not wait for, from its image).  Nothing traps,
faults or hangs.  After each failure the previous image and baseline must be intact:
the next successful checkpoint must equal the oracle's, which never saw the
failed attempt.
"""
import numpy as np
import pytest

import paper_2008_10596_gb300 as C
from tests.gpu_harness import Harness, pattern_mutations

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("oracle_lib")]


@pytest.mark.parametrize("kern", [C.CRAC_PASS_TMA, C.CRAC_PASS_LDG, C.CRAC_PASS_SPARSE, "direct"])
@pytest.mark.parametrize("step,code", [(C.CRAC_FAULT_PASS, C.CRAC_ERR_CUDA),
                                       (C.CRAC_FAULT_DRAIN, C.CRAC_ERR_CUDA),
                                       (C.CRAC_FAULT_ALLOC, C.CRAC_ERR_OOM),
                                       (C.CRAC_FAULT_DEVICE_WAIT, C.CRAC_ERR_TIMEOUT)])
def test_failed_checkpoint_leaves_state(step, code, kern):
    S = 4096
    extra = {"image_residency": C.CRAC_RESIDENCY_DEVICE} if kern == C.CRAC_PASS_SPARSE else {}
    if kern == "direct":   # the split pass writing host images through their device mapping
        kern, extra = C.CRAC_PASS_SPLIT, {"flags": C.CRAC_FLAG_DIRECT_DRAIN}
    h = Harness(S, lineage=61, timeout_ns=20_000_000, chunks_per_tile=2, pass_kernel=kern, **extra)
    try:
        # > 1024 chunks, so that the split finalize (the sparse pass's
        # look-back) has a second tile whose wait can run out
        for i, n in enumerate([200000, 70000, 4 * 1024 * 1024 + 65536]):
            h.add(n, seed=i + 1)
        _, lib1, ora1 = h.checkpoint()
        assert lib1 == ora1
        h.mutate(pattern_mutations(h.first(), [b.nbytes for b in h.bufs], S, "random10"))
        C.crac_debug_inject_fault(step, 1)
        try:
            img = C.crac_ctx_checkpoint(h.ctx, h.stream)
        except C.CracError as err:
            assert err.code == code
        else:
            # a pass the call did not wait for reports a device-side failure
            # on its image
            h.images.append(img)
            assert step == C.CRAC_FAULT_DEVICE_WAIT
            with pytest.raises(C.CracError) as e:
                C.crac_image_wait(img)
            assert e.value.code == code
        C.crac_debug_inject_fault(C.CRAC_FAULT_NONE, 0)
        # the context is still usable and its baseline untouched
        _, lib2, ora2 = h.checkpoint()
        assert lib2 == ora2
    finally:
        C.crac_debug_inject_fault(C.CRAC_FAULT_NONE, 0)
        h.close()


@pytest.mark.parametrize("residency,flags", [(C.CRAC_RESIDENCY_HOST, 0),
                                             (C.CRAC_RESIDENCY_HOST, C.CRAC_FLAG_STAGED_RESTORE),
                                             (C.CRAC_RESIDENCY_DEVICE, 0)])
def test_failed_restart_leaves_memory(residency, flags):
    S = 4096
    h = Harness(S, lineage=62, image_residency=residency, flags=flags)
    try:
        b = h.add(50000, seed=3)
        img, _, _ = h.checkpoint()
        b.zero()
        C.crac_debug_inject_fault(C.CRAC_FAULT_H2D, 1)
        with pytest.raises(C.CracError) as e:
            C.crac_ctx_restart(h.ctx, img, h.stream)
        assert e.value.code == C.CRAC_ERR_CUDA
        assert not b.read().any()
        h.restart(img)
        assert b.read().any()
    finally:
        C.crac_debug_inject_fault(C.CRAC_FAULT_NONE, 0)
        h.close()


def test_image_wait_timeout_argument():
    S = 4096
    h = Harness(S, lineage=63)
    try:
        h.add(4096, seed=1)
        img, _, _ = h.checkpoint()
        C.crac_image_wait(img, 1)     # already complete: returns at once
        assert C.crac_image_info(img)["complete"] == 1
    finally:
        h.close()


def test_deserialize_rejects_corruption():
    S = 4096
    h = Harness(S, lineage=64)
    try:
        h.add(10000, seed=1)
        _, lib, _ = h.checkpoint()
        for bad in (lib[:-1], lib + b"\0", b"X" + lib[1:]):
            with pytest.raises(C.CracError) as e:
                C.crac_image_deserialize(bad)
            assert e.value.code == C.CRAC_ERR_CORRUPT
        raw = bytearray(lib)
        k_off = 64
        raw[k_off] ^= 1              # k no longer matches the sizes
        with pytest.raises(C.CracError):
            C.crac_image_deserialize(bytes(raw))
        ok = C.crac_image_deserialize(lib)
        assert C.crac_image_serialize(ok) == lib
        C.crac_image_release(ok)
        assert np.frombuffer(lib[:8], dtype=np.uint8).tobytes() == b"CRACIMG1"
    finally:
        h.close()
