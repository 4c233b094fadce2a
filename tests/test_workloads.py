"""The seeded input generators (CPU only)."""
import numpy as np

import workloads as W


def test_xorshift_parallel_matches_sequential():
    seed = W.SEED_BASE + 1
    got = W.xorshift64_u32(seed, 5000, lane_steps=37)
    s = seed
    exp = []
    for _ in range(5000):
        s = W.xorshift64_next(s)
        exp.append(s >> 32)
    assert got.tolist() == exp


def test_xorshift_known_first_values():
    # Marsaglia (2003) example: x ^= x<<13; x ^= x>>7; x ^= x<<17 from x = 1.
    x = W.xorshift64_next(1)
    assert x == (1 ^ (1 << 13)) ^ ((1 ^ (1 << 13)) >> 7) ^ ((((1 ^ (1 << 13)) ^ ((1 ^ (1 << 13)) >> 7)) << 17) & ((1 << 64) - 1))


def test_choose_distinct():
    r = W.XorShift64(123)
    picks = W.choose_distinct(r, 4096, 41)
    assert len(set(picks)) == 41 and all(0 <= p < 4096 for p in picks)
    r = W.XorShift64(5)
    assert sorted(W.choose_distinct(r, 10, 10)) == list(range(10))


def test_water_fill_and_config_sizes():
    s = W.config2_sizes()
    assert len(s) == 256
    assert abs(sum(s) - 4 * W.GIB) <= 256 * 256
    assert min(s) >= 4 * W.KIB and max(s) <= 64 * W.MIB
    assert all(x % 256 == 0 for x in s)
    c3 = W.config3()
    assert sum(c3.sizes) == 12 * W.GIB and sum(c3.managed_sizes) == 4 * W.GIB
    c4 = W.config4()
    assert len(c4.sizes) == 2048 and abs(sum(c4.sizes) - 120 * W.GIB) <= 2048 * 4096
    assert min(c4.sizes) >= 4096 and all(x % 4096 == 0 for x in c4.sizes)


def test_mutations_change_every_chosen_chunk():
    sizes = [4096 * 3 + 3, 10]
    bufs = [W.host_contents("u8", s, i) for i, s in enumerate(sizes)]
    before = [b.copy() for b in bufs]
    first = W.chunk_layout(sizes, 4096)
    muts = W.choose_mutations(1, int(first[-1]), 1.0)
    W.apply_mutations_host(bufs, first, 4096, muts)
    for a, s in enumerate(sizes):
        for local in range(-(-s // 4096)):
            lo, hi = local * 4096, min(s, local * 4096 + 4096)
            assert not np.array_equal(before[a][lo:hi], bufs[a][lo:hi])


def test_bf16_rne():
    f = np.array([1.0, 1.00390625, 1.01171875, -2.5], dtype=np.float32)
    assert W.f32_to_bf16_rne(f).tolist() == [0x3F80, 0x3F80, 0x3F82, 0xC020]
