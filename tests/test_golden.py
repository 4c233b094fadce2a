"""The oracle against its frozen fixtures in tests/golden (CPU only)."""
import os

import numpy as np
import pytest

from oracle import fp_bigint
from oracle import oracle as O
from tests.golden import make_golden as G

pytestmark = pytest.mark.usefixtures("oracle_lib")
HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_fp_vectors():
    rows = open(os.path.join(HERE, "fp_vectors.txt")).read().split()
    rows = [rows[i:i + 3] for i in range(0, len(rows), 3)]
    assert len(rows) == len(G.FP_CASES)
    for seed, n, v in rows:
        b = G.chunk_bytes_for(int(seed), int(n))
        assert O.fp64(b) == int(v, 16)
        assert fp_bigint.fp64(b) == int(v, 16)


def test_tiny_chain():
    want = [bytes.fromhex(x) for x in open(os.path.join(HERE, "tiny_chain.txt")).read().split()]
    got = G.tiny_chain()
    assert got == want
    imgs = [O.parse_image(b) for b in want]
    assert imgs[0].full and imgs[1].idx.tolist() == [0, 2] and imgs[2].k == 0
    r = O.OracleContext(64)
    r.register(1 << 20, 37)
    r.register(1 << 21, 130, O.KIND_MANAGED)
    mem = r.restart(want[:2])
    assert np.array_equal(np.concatenate(mem), np.frombuffer(
        bytes(imgs[0].payload), dtype=np.uint8) ^ _flip_mask())


def _flip_mask():
    m = np.zeros(167, dtype=np.uint8)
    m[36] = 0x80
    m[37 + 70] = 0x01
    return m
