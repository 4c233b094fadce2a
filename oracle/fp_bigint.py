"""CRAC-FP64 restated with Python arbitrary-precision integers.

TEST INFRASTRUCTURE ONLY (part of the oracle; never imported by the product
library).  A second, independent statement of the project's chunk
fingerprint: the chunk is read as one big little-endian integer and split
into 64-bit limbs; every product and sum is reduced modulo 2^64 explicitly.
The paper has no fingerprint (it copies all active allocations, Sec. 3.2);
the hash exists so an incremental checkpoint can carry only changed chunks.

Constants are computed here from their definitions with integer square
roots rather than written out, so a mistyped hex literal elsewhere shows up
as a mismatch against this module.
"""
from math import isqrt

_MOD = 1 << 64


def _frac_sqrt_bits(p: int) -> int:
    """floor(2^64 * frac(sqrt(p))) for a non-square p."""
    return isqrt(p << 128) - (isqrt(p) << 64)


def golden_k1() -> int:
    """floor(2^64 / phi) = floor(2^64 * (sqrt(5) - 1) / 2)."""
    return (isqrt(5 << 128) - (1 << 64)) // 2


K1 = golden_k1()
M1 = _frac_sqrt_bits(2) | 1
M2 = _frac_sqrt_bits(3) | 1
M3 = _frac_sqrt_bits(5) | 1


def fp64(chunk: bytes) -> int:
    """Fingerprint of one chunk (1 <= len(chunk))."""
    n = len(chunk)
    if n == 0:
        raise ValueError("empty chunk")
    m = (n + 7) // 8
    big = int.from_bytes(bytes(chunk) + b"\0" * (8 * m - n), "little")
    acc = 0
    for j in range(m):
        w = (big >> (64 * j)) % _MOD
        x = w ^ (((j + 1) * K1) % _MOD)
        y = (x * M1) % _MOD
        f = y ^ (y >> 32)
        acc = (acc + f) % _MOD
    z = acc ^ ((n * M3) % _MOD)
    z ^= z >> 31
    z = (z * M2) % _MOD
    z ^= z >> 29
    z = (z * M1) % _MOD
    z ^= z >> 32
    return z


def word_terms(chunk: bytes) -> list[int]:
    """The per-word summands f_j (exposed for the reduction-order tests)."""
    n = len(chunk)
    m = (n + 7) // 8
    big = int.from_bytes(bytes(chunk) + b"\0" * (8 * m - n), "little")
    out = []
    for j in range(m):
        w = (big >> (64 * j)) % _MOD
        y = ((w ^ (((j + 1) * K1) % _MOD)) * M1) % _MOD
        out.append(y ^ (y >> 32))
    return out


def finalize(acc: int, n: int) -> int:
    z = acc ^ ((n * M3) % _MOD)
    z ^= z >> 31
    z = (z * M2) % _MOD
    z ^= z >> 29
    z = (z * M1) % _MOD
    z ^= z >> 32
    return z
