// CRZ1, the chunk codec of coded images: device helpers shared by the
// encoder (crac_codec.cu) and the restore kernels (crac_restore.cu).
//
// The paper times its checkpoints with DMTCP's gzip turned off (Sec. 4.4.1,
// "Checkpoint overhead"), so it has no codec; CRZ1 is this project's.  One
// chunk of L bytes is cut into nb = L / 512 blocks and a tail of L % 512
// bytes.  A block is 128 little-endian u32 words; every byte of every word
// is rotated left by one bit (a float's sign moves to the byte's bottom), and
// byte p of the 128 rotated words forms plane p.  Each plane is stored as
// its minimum m_p and the offsets from it in W_p = bitlength(max - m_p) bits:
// header word h = sum m_p << 8p + sum W_p << (32 + 4p), then, for p = 0..3
// and j < W_p, a 16-byte unit of four words q = 0..3 whose bit l is bit j
// of plane value 4l + q.  A stream is the nb header words (zero-padded to 16
// bytes), the blocks' units in order, then the tail; a chunk whose stream
// would not be shorter than L is stored as itself.
//
// Warp layout: lane l holds words 4l .. 4l+3 of a block (one 16-byte load),
// so unit (p, j) word q is __ballot_sync of bit j of the lane's value q.
#pragma once

#include "crac_device.cuh"

namespace crac {
namespace {

constexpr uint32_t kCrzBlock = 512;

__device__ __forceinline__ uint32_t crz_rot(uint32_t w) {
    return ((w << 1) & 0xFEFEFEFEu) | ((w >> 7) & 0x01010101u);
}

__device__ __forceinline__ uint32_t crz_unrot(uint32_t r) {
    return ((r >> 1) & 0x7F7F7F7Fu) | ((r << 7) & 0x80808080u);
}

__device__ __forceinline__ uint32_t crz_width(uint64_t h, int p) {
    return (uint32_t)(h >> (32 + 4 * p)) & 15u;
}

__device__ __forceinline__ uint32_t crz_width_sum(uint64_t h) {
    return crz_width(h, 0) + crz_width(h, 1) + crz_width(h, 2) + crz_width(h, 3);
}

// Header words of nb blocks, zero-padded to 16 bytes.
__device__ __forceinline__ uint64_t crz_head_bytes(uint64_t nb) { return 16ull * ((nb + 1) >> 1); }

// 16 bytes from any address (the raw payload is byte-aligned after a chunk
// whose length is not a multiple of 16).
__device__ __forceinline__ uint4 load16_any(const uint8_t *p) {
    const uintptr_t a = (uintptr_t)p;
    if ((a & 15u) == 0) return *reinterpret_cast<const uint4 *>(p);
    if ((a & 3u) == 0) {
        const uint32_t *q = reinterpret_cast<const uint32_t *>(p);
        return make_uint4(q[0], q[1], q[2], q[3]);
    }
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
        w[i] = (uint32_t)p[4 * i] | ((uint32_t)p[4 * i + 1] << 8) | ((uint32_t)p[4 * i + 2] << 16) |
               ((uint32_t)p[4 * i + 3] << 24);
    return make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ void store16_any(uint8_t *p, uint4 v) {
    const uintptr_t a = (uintptr_t)p;
    if ((a & 15u) == 0) {
        *reinterpret_cast<uint4 *>(p) = v;
        return;
    }
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int b = 0; b < 4; ++b) p[4 * i + b] = (uint8_t)(w[i] >> (8 * b));
}

// Header word of the block whose words 4*lane .. 4*lane+3 the calling lane
// holds (rotated).  Whole warp.
__device__ __forceinline__ uint64_t crz_block_header(const uint32_t r[4]) {
    uint64_t h = 0;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const uint32_t v0 = (r[0] >> (8 * p)) & 255u, v1 = (r[1] >> (8 * p)) & 255u;
        const uint32_t v2 = (r[2] >> (8 * p)) & 255u, v3 = (r[3] >> (8 * p)) & 255u;
        const uint32_t lo = min(min(v0, v1), min(v2, v3)), hi = max(max(v0, v1), max(v2, v3));
        const uint32_t m = __reduce_min_sync(kFull, lo), M = __reduce_max_sync(kFull, hi);
        const uint32_t W = M == m ? 0u : 32u - (uint32_t)__clz(M - m);
        h |= ((uint64_t)m << (8 * p)) | ((uint64_t)W << (32 + 4 * p));
    }
    return h;
}

// Units of one block: lanes 0 .. sum(W)-1 each store one 16-byte unit at
// out + 16 * lane (out 16-byte aligned).  Whole warp.
__device__ __forceinline__ void crz_block_units(uint64_t h, const uint32_t r[4], uint8_t *out, int lane) {
    uint4 mine = make_uint4(0u, 0u, 0u, 0u);
    uint32_t u = 0;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const uint32_t m = (uint32_t)(h >> (8 * p)) & 255u, W = crz_width(h, p);
        const uint32_t d0 = ((r[0] >> (8 * p)) & 255u) - m, d1 = ((r[1] >> (8 * p)) & 255u) - m;
        const uint32_t d2 = ((r[2] >> (8 * p)) & 255u) - m, d3 = ((r[3] >> (8 * p)) & 255u) - m;
        for (uint32_t j = 0; j < W; ++j) {
            const uint32_t b0 = __ballot_sync(kFull, (d0 >> j) & 1u);
            const uint32_t b1 = __ballot_sync(kFull, (d1 >> j) & 1u);
            const uint32_t b2 = __ballot_sync(kFull, (d2 >> j) & 1u);
            const uint32_t b3 = __ballot_sync(kFull, (d3 >> j) & 1u);
            if ((uint32_t)lane == u + j) mine = make_uint4(b0, b1, b2, b3);
        }
        u += W;
    }
    if ((uint32_t)lane < u) *reinterpret_cast<uint4 *>(out + 16u * lane) = mine;
}

// Decode the z-byte stream at src (16-byte aligned) into the len bytes at
// dst (16-byte aligned).  Whole warp.  Every read stays inside [src, src+z)
// and every write inside [dst, dst+len).  Returns false for a stream that
// no chunk of len bytes encodes to: nothing is written when its lengths or
// headers are inconsistent, and the chunk may be partly written when a
// plane value overflows a byte.
__device__ __forceinline__ bool crz_decode_warp(uint8_t *dst, const uint8_t *src, uint64_t len, uint64_t z,
                                                int lane) {
    const uint64_t nb = len >> 9, tl = len & 511u, head = crz_head_bytes(nb);
    if (nb == 0 || z >= len || z < head || ((uintptr_t)src & 15u)) return false;
    const uint64_t *H = reinterpret_cast<const uint64_t *>(src);
    uint32_t tot = 0;
    bool bad = false;
    for (uint64_t b = lane; b < nb; b += 32) {
        const uint64_t h = H[b];
        bad |= (h >> 48) != 0;
#pragma unroll
        for (int p = 0; p < 4; ++p) bad |= crz_width(h, p) > 8u;
        tot += crz_width_sum(h);
    }
    bad = __any_sync(kFull, bad);
    tot = __reduce_add_sync(kFull, tot);   // <= 32 per block, nb <= 2^15
    if (bad || head + 16ull * tot + tl != z) return false;
    const uint8_t *units = src + head;
    uint32_t carry = 0;
    bool over = false;
    for (uint64_t b0 = 0; b0 < nb; b0 += 32) {
        const uint64_t b = b0 + lane;
        const uint64_t h = b < nb ? H[b] : 0ull;
        const uint32_t ws = crz_width_sum(h);
        uint32_t incl = ws;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        const uint32_t excl = carry + incl - ws;
        carry += __shfl_sync(kFull, incl, 31);
        const int nblk = (int)umin64(32, nb - b0);
        for (int i = 0; i < nblk; ++i) {
            const uint64_t hb = __shfl_sync(kFull, h, i);
            const uint32_t ub = __shfl_sync(kFull, excl, i);
            const uint32_t wsb = crz_width_sum(hb);
            uint4 u = make_uint4(0u, 0u, 0u, 0u);
            if ((uint32_t)lane < wsb) u = *reinterpret_cast<const uint4 *>(units + 16ull * (ub + lane));
            uint32_t o[4] = {0u, 0u, 0u, 0u};
            uint32_t uu = 0;
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                const uint32_t m = (uint32_t)(hb >> (8 * p)) & 255u, W = crz_width(hb, p);
                uint32_t v0 = 0, v1 = 0, v2 = 0, v3 = 0;
                for (uint32_t j = 0; j < W; ++j) {
                    const int sl = (int)(uu + j);
                    v0 |= ((__shfl_sync(kFull, u.x, sl) >> lane) & 1u) << j;
                    v1 |= ((__shfl_sync(kFull, u.y, sl) >> lane) & 1u) << j;
                    v2 |= ((__shfl_sync(kFull, u.z, sl) >> lane) & 1u) << j;
                    v3 |= ((__shfl_sync(kFull, u.w, sl) >> lane) & 1u) << j;
                }
                uu += W;
                v0 += m;
                v1 += m;
                v2 += m;
                v3 += m;
                over |= ((v0 | v1 | v2 | v3) > 255u);
                o[0] |= (v0 & 255u) << (8 * p);
                o[1] |= (v1 & 255u) << (8 * p);
                o[2] |= (v2 & 255u) << (8 * p);
                o[3] |= (v3 & 255u) << (8 * p);
            }
            store16_any(dst + 512ull * (b0 + i) + 16u * lane,
                        make_uint4(crz_unrot(o[0]), crz_unrot(o[1]), crz_unrot(o[2]), crz_unrot(o[3])));
        }
    }
    for (uint64_t i = lane; i < tl; i += 32) dst[512ull * nb + i] = units[16ull * tot + i];
    return !__any_sync(kFull, over);
}

}  // namespace
}  // namespace crac
