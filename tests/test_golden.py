"""The oracle against its frozen fixtures in tests/golden (CPU only)."""
import os

import numpy as np
import pytest

from oracle import crz
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


def test_crz_vectors():
    rows = [line.split() for line in open(os.path.join(HERE, "crz_vectors.txt")).read().splitlines()]
    assert [(c, int(s), int(n)) for c, s, n, _ in rows] == G.CRZ_CASES
    for content, seed, n, hexz in rows:
        raw = G.crz_input(content, int(seed), int(n))
        z = bytes.fromhex(hexz)
        assert crz.encode(raw) == z
        assert crz.decode(z, int(n)) == raw
        if content in ("u32_xorshift",):
            assert z == raw            # incompressible: stored as itself
        if content == "zeros":             # zero header words, padded, then the zero tail
            nb = int(n) // 512
            assert z == bytes(16 * (-(-nb // 2)) + int(n) % 512)
