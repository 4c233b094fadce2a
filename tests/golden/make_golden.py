"""Write the golden fixtures in this folder from the oracle alone.

    python tests/golden/make_golden.py

fp_vectors.txt   CRAC-FP64 known-answer vectors: one line per case,
                 "<xorshift seed> <length> <fp hex>"; the chunk bytes are the
                 first <length> bytes of workloads.xorshift64_u32(seed, ...).
                 Values come from the Python big-integer restatement
                 (oracle/fp_bigint.py) and are cross-checked against the C one.
tiny_chain.txt   A three-image chain (full, delta, empty delta) of a tiny
                 two-allocation scenario, one image per line in hex.
crz_vectors.txt  CRZ1 streams (oracle/crz.py): one line per case,
                 "<content> <seed> <length> <stream hex>"; the chunk is
                 crz_input(content, seed, length).

The paper prints no worked example for this pass; these fixtures freeze the
oracle's own output so that later edits to either restatement are caught.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import workloads as W  # noqa: E402
from oracle import crz  # noqa: E402
from oracle import fp_bigint  # noqa: E402
from oracle import oracle as O  # noqa: E402

FP_CASES = [(s, n) for s in (1, 2, 2008105961) for n in (1, 3, 8, 9, 15, 16, 17, 31, 64, 100, 4096, 4099)]
CRZ_CASES = [(k, 7, n) for k in ("f32_normal", "bf16", "u32_xorshift", "zeros") for n in (512, 1100)]


def crz_input(content: str, seed: int, n: int) -> bytes:
    if content == "zeros":
        return bytes(n)
    return W.host_contents(content, n, seed).tobytes()


def chunk_bytes_for(seed: int, n: int) -> bytes:
    return W.xorshift64_u32(seed, (n + 3) // 4).view("u1")[:n].tobytes()


def tiny_chain():
    sizes = [37, 130]
    ctx = O.OracleContext(64, lineage=3)
    ctx.register(0x7000_0000_0000, sizes[0], O.KIND_DEVICE)
    ctx.register(0x7000_0000_1000, sizes[1], O.KIND_MANAGED)
    bufs = [W.host_contents("u32_xorshift", s, 40 + i) for i, s in enumerate(sizes)]
    imgs = [ctx.checkpoint(bufs)]
    bufs[1][70] ^= 0x01
    bufs[0][36] ^= 0x80
    imgs.append(ctx.checkpoint(bufs))
    imgs.append(ctx.checkpoint(bufs))
    return imgs


def main():
    lines = []
    for seed, n in FP_CASES:
        b = chunk_bytes_for(seed, n)
        v = fp_bigint.fp64(b)
        assert v == O.fp64(b), "restatements disagree"
        lines.append(f"{seed} {n} {v:016x}")
    with open(os.path.join(HERE, "fp_vectors.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")
    with open(os.path.join(HERE, "tiny_chain.txt"), "w") as f:
        f.write("\n".join(i.hex() for i in tiny_chain()) + "\n")
    rows = []
    for content, seed, n in CRZ_CASES:
        z = crz.encode(crz_input(content, seed, n))
        assert crz.decode(z, n) == crz_input(content, seed, n)
        rows.append(f"{content} {seed} {n} {z.hex()}")
    with open(os.path.join(HERE, "crz_vectors.txt"), "w") as f:
        f.write("\n".join(rows) + "\n")


if __name__ == "__main__":
    main()
