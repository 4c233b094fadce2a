"""Checkpoints that return once enqueued (GPU).

A single-segment pass into uncoded images is not waited for: the call returns
after enqueueing it on the caller's stream, behind whatever the application
enqueued before (here a delay kernel that keeps the stream busy), and the
image's sizes settle when its work completes.  Every image must still equal
the oracle's image of the memory as it was when its pass ran on the stream,
also with two checkpoints and their mutators in flight with no host
synchronization between them.  A pass whose device wait runs out reports
CRAC_ERR_TIMEOUT on its image (and on an image taken after it, which
compared against its fingerprints); the context's baseline then returns to
the last good image, so the next checkpoint equals the oracle's, which never
saw the failed ones.
"""
import time

import numpy as np
import pytest
import torch

import paper_2008_10596_gb300 as C
import workloads as W
from oracle import oracle as O
from paper_2008_10596_gb300 import testkit
from tests.gpu_harness import Harness, pattern_mutations
from workloads.device import rows_tensor

pytestmark = [pytest.mark.gpu, pytest.mark.usefixtures("oracle_lib")]

S = 4096
SIZES = [200000, 70000, 4 * 1024 * 1024 + 65536]   # > 1024 chunks: the finalize has several tiles


def _setup(**cfg):
    h = Harness(S, lineage=70, **cfg)
    # a stream of its own: the NULL stream means "synchronize the device
    # first" (the paper's queue drain before a checkpoint)
    h.stream = torch.cuda.Stream()
    for i, n in enumerate(SIZES):
        h.add(n, seed=i + 11)
    torch.cuda.synchronize()
    return h


def _rows(h, muts):
    first = h.first()
    rows = []
    for m in muts:
        a = int(np.searchsorted(first, m.chunk, side="right") - 1)
        lo = (m.chunk - int(first[a])) * S
        rows.append((h.bufs[a].ptr + lo, min(S, h.bufs[a].nbytes - lo), m.mask))
    return rows_tensor(rows, "cuda")


def _same(lib, want, what):
    """Byte equality, with the differing sections named on failure."""
    if lib == want:
        return
    a, b = O.parse_image(lib), O.parse_image(want)
    notes = []
    for f in ("flags", "epoch", "parent_epoch", "n_chunks", "k"):
        if getattr(a, f) != getattr(b, f):
            notes.append(f"{f} {getattr(a, f)} != {getattr(b, f)}")
    if a.fp.size == b.fp.size and not np.array_equal(a.fp, b.fp):
        notes.append(f"fp differs at {np.flatnonzero(a.fp != b.fp)[:8].tolist()} "
                     f"({int((a.fp != b.fp).sum())} chunks)")
    if a.idx.tolist() != b.idx.tolist():
        sa, sb = set(a.idx.tolist()), set(b.idx.tolist())
        notes.append(f"idx: {len(sa - sb)} extra {sorted(sa - sb)[:8]}, {len(sb - sa)} missing {sorted(sb - sa)[:8]}")
    elif bytes(a.payload) != bytes(b.payload):
        notes.append("payload differs")
    raise AssertionError(f"{what}: " + "; ".join(notes))


def _host_after(host, h, muts):
    out = [b.copy() for b in host]
    W.apply_mutations_host(out, h.first(), S, muts)
    return out


RESIDENCY = [C.CRAC_RESIDENCY_HOST, C.CRAC_RESIDENCY_DEVICE]


@pytest.mark.parametrize("residency", RESIDENCY)
def test_checkpoint_returns_before_its_pass(residency):
    h = _setup(image_residency=residency)
    try:
        _, lib0, ora0 = h.checkpoint()
        assert lib0 == ora0
        muts = pattern_mutations(h.first(), SIZES, S, "random10", seed=5)
        ent = _rows(h, muts)
        want = _host_after(h.host(), h, muts)
        torch.cuda.synchronize()
        testkit.delay(300_000_000, h.stream)          # the application is still busy for 0.3 s
        testkit.mutate_xor(ent.data_ptr(), len(muts), h.stream)
        t0 = time.perf_counter()
        img = C.crac_ctx_checkpoint(h.ctx, h.stream)
        dt = time.perf_counter() - t0
        h.images.append(img)
        assert dt < 0.1, f"the call waited {dt:.3f} s"
        with pytest.raises(C.CracError) as e:          # its pass has not run yet
            C.crac_image_wait(img, 1_000_000)
        assert e.value.code == C.CRAC_ERR_TIMEOUT
        C.crac_image_wait(img)
        assert C.crac_image_serialize(img) == h.oracle.checkpoint(want)
        assert C.crac_ctx_last_pass(h.ctx)["k"] == len(muts)
    finally:
        h.close()


@pytest.mark.parametrize("residency", RESIDENCY)
@pytest.mark.parametrize("kern", [C.CRAC_PASS_SPLIT, C.CRAC_PASS_LDG, C.CRAC_PASS_TMA])
def test_checkpoints_and_mutators_in_flight(residency, kern):
    """checkpoint -> mutator -> checkpoint -> mutator -> checkpoint on one
    stream, behind a busy stream, with no host synchronization in between."""
    h = _setup(image_residency=residency, pass_kernel=kern)
    try:
        _, lib0, ora0 = h.checkpoint()
        assert lib0 == ora0
        m1 = pattern_mutations(h.first(), SIZES, S, "random10", seed=6)
        m2 = pattern_mutations(h.first(), SIZES, S, "alternating", seed=7)
        e1, e2 = _rows(h, m1), _rows(h, m2)
        s0 = h.host()
        s1 = _host_after(s0, h, m1)
        s2 = _host_after(s1, h, m2)
        s3 = _host_after(s2, h, m1)
        torch.cuda.synchronize()
        testkit.delay(100_000_000, h.stream)
        imgs = []
        for ent, muts in ((e1, m1), (e2, m2), (e1, m1)):
            testkit.mutate_xor(ent.data_ptr(), len(muts), h.stream)
            imgs.append(C.crac_ctx_checkpoint(h.ctx, h.stream))
            h.images.append(imgs[-1])
        for j, (img, state) in enumerate(zip(imgs, (s1, s2, s3))):
            _same(C.crac_image_serialize(img), h.oracle.checkpoint(state), f"image {j}")
        # the chain restores the last state
        for b in h.bufs:
            b.zero()
        h.restart(imgs[-1])
        for b, w in zip(h.bufs, s3):
            assert np.array_equal(b.read(), w)
    finally:
        h.close()


@pytest.mark.parametrize("residency", RESIDENCY)
def test_failed_unsettled_passes_revert_the_baseline(residency):
    """The first of two in-flight checkpoints times out on the device: both
    report it on their images, and the next checkpoint is a delta against
    the last good image, equal to the oracle's."""
    h = _setup(image_residency=residency, timeout_ns=20_000_000, chunks_per_tile=2)
    try:
        img0, lib0, ora0 = h.checkpoint()
        assert lib0 == ora0
        m1 = pattern_mutations(h.first(), SIZES, S, "random10", seed=8)
        m2 = pattern_mutations(h.first(), SIZES, S, "random10", seed=9)
        e1, e2 = _rows(h, m1), _rows(h, m2)
        torch.cuda.synchronize()
        testkit.delay(100_000_000, h.stream)
        testkit.mutate_xor(e1.data_ptr(), len(m1), h.stream)
        C.crac_debug_inject_fault(C.CRAC_FAULT_DEVICE_WAIT, 1)
        a = C.crac_ctx_checkpoint(h.ctx, h.stream)
        h.images.append(a)
        C.crac_debug_inject_fault(C.CRAC_FAULT_NONE, 0)
        testkit.mutate_xor(e2.data_ptr(), len(m2), h.stream)
        b = C.crac_ctx_checkpoint(h.ctx, h.stream)
        h.images.append(b)
        for img in (a, b):
            with pytest.raises(C.CracError) as e:
                C.crac_image_wait(img)
            assert e.value.code == C.CRAC_ERR_TIMEOUT
        # the oracle never saw a or b: its next image is a delta against img0
        _, lib2, ora2 = h.checkpoint()
        assert lib2 == ora2
        im = O.parse_image(lib2)
        assert im.parent_epoch == O.parse_image(lib0).epoch and not im.full
    finally:
        C.crac_debug_inject_fault(C.CRAC_FAULT_NONE, 0)
        h.close()


def test_wait_pass_flag_makes_the_call_wait():
    """CRAC_FLAG_WAIT_PASS: the call returns only after its pass, with the
    image's sizes known; the image equals the oracle's."""
    h = _setup(flags=C.CRAC_FLAG_WAIT_PASS)
    try:
        _, lib0, ora0 = h.checkpoint()
        assert lib0 == ora0
        muts = pattern_mutations(h.first(), SIZES, S, "random10", seed=12)
        ent = _rows(h, muts)
        want = _host_after(h.host(), h, muts)
        torch.cuda.synchronize()
        testkit.delay(200_000_000, h.stream)
        testkit.mutate_xor(ent.data_ptr(), len(muts), h.stream)
        t0 = time.perf_counter()
        img = C.crac_ctx_checkpoint(h.ctx, h.stream)
        dt = time.perf_counter() - t0
        h.images.append(img)
        assert dt >= 0.15, f"the call returned after {dt:.3f} s"
        assert C.crac_ctx_last_pass(h.ctx)["k"] == len(muts)
        _same(C.crac_image_serialize(img), h.oracle.checkpoint(want), "image")
    finally:
        h.close()


@pytest.mark.parametrize("residency", RESIDENCY)
def test_restart_then_mutator_then_checkpoint_on_one_stream(residency):
    """A restart returns once its restore has run (it checks the restore's
    error word before adopting the image); the application's next work and
    the next checkpoint are then enqueued behind a busy stream with no host
    synchronization, and that checkpoint equals the oracle's delta against
    the restored image."""
    h = _setup(image_residency=residency)
    try:
        _, lib0, ora0 = h.checkpoint()
        assert lib0 == ora0
        m1 = pattern_mutations(h.first(), SIZES, S, "random10", seed=13)
        m2 = pattern_mutations(h.first(), SIZES, S, "alternating", seed=14)
        e1, e2 = _rows(h, m1), _rows(h, m2)
        testkit.mutate_xor(e1.data_ptr(), len(m1), h.stream)
        torch.cuda.synchronize()
        img1, lib1, ora1 = h.checkpoint()
        assert lib1 == ora1
        s1 = h.host()
        testkit.mutate_xor(e2.data_ptr(), len(m2), h.stream)   # lost by the restart below
        C.crac_ctx_restart(h.ctx, img1, h.stream)
        testkit.delay(100_000_000, h.stream)
        testkit.mutate_xor(e2.data_ptr(), len(m2), h.stream)
        img = C.crac_ctx_checkpoint(h.ctx, h.stream)
        h.images.append(img)
        want = _host_after(s1, h, m2)
        _same(C.crac_image_serialize(img), h.oracle.checkpoint(want), "image after the restart")
        im = O.parse_image(C.crac_image_serialize(img))
        assert not im.full and im.parent_epoch == O.parse_image(lib1).epoch
    finally:
        h.close()
