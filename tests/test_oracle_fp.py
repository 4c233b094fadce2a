"""Pins for the oracle's CRAC-FP64 chunk fingerprint (CPU only).

The paper has no fingerprint (it copies every active allocation, Sec. 3.2);
the hash is this project's definition.  It is pinned by (a) its constants'
defining formulas checked against independent decimal expansions, (b) two
independent restatements (plain C, Python big integers) agreeing, and (c)
structural properties any correct implementation must have: a single-word
change always changes the fingerprint (the per-word map is a bijection and
the sum is mod 2^64), the sum is order-independent, words are keyed by
position, and the length is folded into the finalizer.
"""
import random
from decimal import Decimal, getcontext

import numpy as np
import pytest

from oracle import fp_bigint
from oracle import oracle as O

pytestmark = pytest.mark.usefixtures("oracle_lib")


def _dec_frac_sqrt(p: int) -> Decimal:
    getcontext().prec = 60
    r = Decimal(p).sqrt()
    return r - int(r)


def test_constants_match_decimal_definitions():
    two64 = Decimal(2) ** 64
    getcontext().prec = 60
    phi = (1 + Decimal(5).sqrt()) / 2
    assert fp_bigint.K1 == int(two64 / phi)
    assert fp_bigint.K1 == 0x9E3779B97F4A7C15
    for p, m in ((2, fp_bigint.M1), (3, fp_bigint.M2), (5, fp_bigint.M3)):
        assert m == int(two64 * _dec_frac_sqrt(p)) | 1
        assert m & 1
    # SHA-512's first three IV words are the same fractional square roots
    # (FIPS 180-4, Sec. 5.3.5); odd-forcing sets only the low bit.
    assert fp_bigint.M1 == 0x6A09E667F3BCC908 | 1
    assert fp_bigint.M2 == 0xBB67AE8584CAA73B | 1
    assert fp_bigint.M3 == 0x3C6EF372FE94F82B | 1


@pytest.mark.parametrize("n", list(range(1, 41)) + [63, 64, 65, 255, 256, 257, 4095, 4096, 4097])
def test_c_matches_bigint(n):
    rnd = random.Random(1000 + n)
    for _ in range(3):
        b = bytes(rnd.getrandbits(8) for _ in range(n))
        assert O.fp64(b) == fp_bigint.fp64(b)


def test_c_matches_bigint_special_patterns():
    for n in (1, 7, 8, 9, 16, 17, 4096):
        for fill in (0x00, 0xFF, 0x80):
            b = bytes([fill]) * n
            assert O.fp64(b) == fp_bigint.fp64(b)


def test_fp_chunks_tail():
    rnd = np.random.default_rng(5)
    buf = rnd.integers(0, 256, size=3 * 64 + 5, dtype=np.uint8)
    got = O.fp_chunks(buf, 64)
    exp = [fp_bigint.fp64(buf[i:i + 64].tobytes()) for i in range(0, buf.size, 64)]
    assert got.tolist() == exp
    assert len(exp) == 4


@pytest.mark.parametrize("n", [8, 24, 64, 4096])
def test_single_word_change_always_changes_fp(n):
    rnd = random.Random(n)
    base = bytearray(rnd.getrandbits(8) for _ in range(n))
    f0 = O.fp64(bytes(base))
    for j in range(n // 8):
        for _ in range(4):
            delta = rnd.getrandbits(64) | 1
            b = bytearray(base)
            w = int.from_bytes(b[8 * j:8 * j + 8], "little") ^ delta
            b[8 * j:8 * j + 8] = w.to_bytes(8, "little")
            assert O.fp64(bytes(b)) != f0


def test_single_byte_change_in_partial_tail_word():
    rnd = random.Random(3)
    for n in (9, 13, 15, 4097):
        base = bytearray(rnd.getrandbits(8) for _ in range(n))
        f0 = O.fp64(bytes(base))
        b = bytearray(base)
        b[-1] ^= 0x5A
        assert O.fp64(bytes(b)) != f0


def test_words_are_position_keyed():
    # Without the (j+1)*K1 key the sum would be invariant under word swaps.
    rnd = random.Random(11)
    for _ in range(20):
        a = rnd.getrandbits(64)
        c = rnd.getrandbits(64)
        if a == c:
            continue
        b1 = a.to_bytes(8, "little") + c.to_bytes(8, "little")
        b2 = c.to_bytes(8, "little") + a.to_bytes(8, "little")
        assert O.fp64(b1) != O.fp64(b2)


def test_length_is_folded_in():
    # 5 and 8 zero bytes pad to the same single word; only len differs.
    assert O.fp64(b"\0" * 5) != O.fp64(b"\0" * 8)
    assert O.fp64(b"\0" * 1) != O.fp64(b"\0" * 7)


def test_reduction_order_independent():
    rnd = random.Random(7)
    b = bytes(rnd.getrandbits(8) for _ in range(4096 + 3))
    terms = fp_bigint.word_terms(b)
    for _ in range(5):
        rnd.shuffle(terms)
        acc = 0
        # Pairwise tree sum in a random order, as a GPU reduction would do it.
        vals = list(terms)
        while len(vals) > 1:
            nxt = [(vals[i] + vals[i + 1]) % (1 << 64) for i in range(0, len(vals) - 1, 2)]
            if len(vals) % 2:
                nxt.append(vals[-1])
            vals = nxt
        acc = vals[0]
        assert fp_bigint.finalize(acc, len(b)) == O.fp64(b)


def test_zero_word_term_is_not_zero():
    # An all-zero chunk still hashes every word (keys make x_j non-zero), so
    # a zero-padded extra word would change the value: the tail must only
    # count ceil(len/8) words.
    t = fp_bigint.word_terms(b"\0" * 16)
    assert all(v != 0 for v in t)
    assert fp_bigint.fp64(b"\0" * 8) != fp_bigint.finalize(sum(t) % (1 << 64), 8)


@pytest.mark.parametrize("workers", [2, 3, 7, 64])
def test_fp_chunks_split_over_threads_is_the_same_table(workers):
    """The per-chunk loop cut into runs over threads: every fingerprint is
    still the one-chunk definition (brute force, chunk by chunk, through the
    big-integer restatement), ragged tail included, also with more threads
    than chunks."""
    for n, S in [(10 * 64 + 13, 64), (5 * 256, 256), (40, 16), (3, 4096)]:
        buf = np.random.default_rng(4000 + n).integers(0, 256, size=n, dtype=np.uint8)
        got = O.fp_chunks(buf, S, workers=workers)
        want = [fp_bigint.fp64(buf[c * S:(c + 1) * S].tobytes()) for c in range(-(-n // S))]
        assert got.tolist() == want
