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
// Warp layout: lane l holds words 4l .. 4l+3 of a block (one 16-byte load).
// Gathering byte p of its four words gives the lane's plane-p word (byte q =
// value 4l + q); the 32 plane words form a 32x32 bit matrix whose transpose
// across the warp is exactly the plane's units (lane 8q + j: unit j, word q).
#pragma once

#include "crac_device.cuh"

namespace crac {
namespace {

constexpr uint32_t kCrzBlock = 512;
constexpr int kCrzDecodeGroup = 2;                           // blocks decoded per step
constexpr int kCrzDecodeScratch = 512 * kCrzDecodeGroup;     // shared bytes per decoding warp

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

// 4x4 byte transpose: byte q of out[p] = byte p of in[q].  Turns a lane's
// four rotated words into its four plane words (byte q = value 4*lane+q of
// the plane), and back.
__device__ __forceinline__ void crz_bytes_transpose(const uint32_t in[4], uint32_t out[4]) {
    const uint32_t t01 = __byte_perm(in[0], in[1], 0x5140), t23 = __byte_perm(in[2], in[3], 0x5140);
    const uint32_t u01 = __byte_perm(in[0], in[1], 0x7362), u23 = __byte_perm(in[2], in[3], 0x7362);
    out[0] = __byte_perm(t01, t23, 0x5410);
    out[1] = __byte_perm(t01, t23, 0x7632);
    out[2] = __byte_perm(u01, u23, 0x5410);
    out[3] = __byte_perm(u01, u23, 0x7632);
}

// Per-lane constants of the warp bit transpose: for each butterfly stage
// (distance s = 16, 8, 4, 2, 1) the rotation that brings the partner's bit
// groups into place and the mask of the groups this lane keeps.
struct CrzLane {
    uint32_t amt[5], keep[5];
};

__device__ __forceinline__ CrzLane crz_lane(int lane) {
    constexpr uint32_t kMask[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
    CrzLane L;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const uint32_t s = 16u >> i;
        const bool hi = (lane & s) != 0;
        L.amt[i] = hi ? 32u - s : s;   // rotate left by s, or right by s
        L.keep[i] = hi ? ~kMask[i] : kMask[i];
    }
    return L;
}

// 32x32 bit transpose across the warp: on entry lane r holds row r (bit c =
// column c), on return lane c holds column c (bit r = row r's bit c).  Five
// butterfly stages, each swapping the off-diagonal halves of every 2s x 2s
// block: the partner's word rotated by s towards this lane's half, merged
// under the keep mask (a shuffle, a funnel shift and one three-input logic
// operation per stage).
__device__ __forceinline__ uint32_t crz_warp_transpose(uint32_t v, const CrzLane &L) {
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const uint32_t x = __shfl_xor_sync(kFull, v, 16 >> i);
        const uint32_t r = __funnelshift_l(x, x, L.amt[i]);
        v = (v & L.keep[i]) | (r & ~L.keep[i]);
    }
    return v;
}

__device__ __forceinline__ uint32_t min_u16x2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

__device__ __forceinline__ uint32_t max_u16x2(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("max.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// Header word of the block whose rotated words 4*lane .. 4*lane+3 the calling
// lane holds.  Planes 0 and 2 (the even bytes) and 1 and 3 (the odd bytes)
// are reduced in pairs as 16-bit lanes, then across the warp.  Whole warp.
__device__ __forceinline__ uint64_t crz_block_header(const uint32_t r[4]) {
    uint32_t e[4], o[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        e[q] = r[q] & 0x00FF00FFu;                   // bytes 0, 2 -> 16-bit lanes
        o[q] = __byte_perm(r[q], 0u, 0x4341);        // bytes 1, 3 -> 16-bit lanes
    }
    const uint32_t emin = min_u16x2(min_u16x2(e[0], e[1]), min_u16x2(e[2], e[3]));
    const uint32_t emax = max_u16x2(max_u16x2(e[0], e[1]), max_u16x2(e[2], e[3]));
    const uint32_t omin = min_u16x2(min_u16x2(o[0], o[1]), min_u16x2(o[2], o[3]));
    const uint32_t omax = max_u16x2(max_u16x2(o[0], o[1]), max_u16x2(o[2], o[3]));
    const uint32_t lo[4] = {emin & 0xFFFFu, omin & 0xFFFFu, emin >> 16, omin >> 16};
    const uint32_t hi[4] = {emax & 0xFFFFu, omax & 0xFFFFu, emax >> 16, omax >> 16};
    uint32_t mins = 0, widths = 0;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const uint32_t m = __reduce_min_sync(kFull, lo[p]), M = __reduce_max_sync(kFull, hi[p]);
        const uint32_t W = 32u - (uint32_t)__clz(M - m);   // bit length; 0 when M == m
        mins |= m << (8 * p);
        widths |= W << (4 * p);
    }
    return ((uint64_t)widths << 32) | mins;
}

// Units of one block: unit (p, j) word q is column 8q + j of the 32x32 bit
// matrix whose row l is lane l's plane word minus the plane minimum (every
// byte is at least the minimum, so the subtraction borrows across no byte).
// After the transpose lane 8q + j holds it and parks it in the warp's
// 512-byte shared scratch at 16 * (u_p + j) + 4q when j < W_p; lanes
// 0 .. sum(W)-1 then store one 16-byte unit each at out + 16 * lane (out
// 16-byte aligned): one coalesced store per block, which matters most when
// out is mapped host memory.  Whole warp.
__device__ __forceinline__ void crz_block_units(uint64_t h, const uint32_t P[4], uint8_t *out, int lane,
                                                const CrzLane &L, uint8_t *scratch) {
    if ((uint32_t)(h >> 32) == 0) return;   // every plane constant: no units
    const uint32_t j = (uint32_t)lane & 7u, q = (uint32_t)lane >> 3;
    // All four transposes run unconditionally (a plane of width 0 stores
    // nothing), so their dependency chains interleave.
    uint32_t col[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) col[p] = crz_warp_transpose(P[p] - ((uint32_t)(h >> (8 * p)) & 255u) * 0x01010101u, L);
    uint32_t u = 0;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const uint32_t W = crz_width(h, p);
        if (j < W) *reinterpret_cast<uint32_t *>(scratch + 16u * (u + j) + 4u * q) = col[p];
        u += W;
    }
    __syncwarp();
    if ((uint32_t)lane < u)
        *reinterpret_cast<uint4 *>(out + 16u * lane) = *reinterpret_cast<const uint4 *>(scratch + 16u * lane);
    __syncwarp();   // the scratch is rewritten by the next block
}

// Decode the z-byte stream at src (16-byte aligned) into the len bytes at
// dst.  Whole warp; scratch is the warp's kCrzDecodeScratch bytes of shared
// memory (16-byte aligned).  Every read stays inside [src, src+z) and every write
// inside [dst, dst+len).  Returns false for a stream that no chunk of len
// bytes encodes to: nothing is written when its lengths or headers are
// inconsistent, and the chunk may be partly written when a plane value
// overflows a byte.
__device__ __forceinline__ bool crz_decode_warp(uint8_t *dst, const uint8_t *src, uint64_t len, uint64_t z,
                                                int lane, uint8_t *scratch) {
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
    const uint32_t j = (uint32_t)lane & 7u, q = (uint32_t)lane >> 3;
    const CrzLane LT = crz_lane(lane);
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
        // Groups of kCrzDecodeGroup blocks: each block's units arrive with one
        // coalesced 16-byte load per lane (lane k: unit k), all of the group's
        // before any is used, and are parked in the warp's shared scratch,
        // from which lane 8q + j takes word q of each plane's unit j.
        constexpr int kG = kCrzDecodeGroup;
        for (int i = 0; i < nblk; i += kG) {
            uint64_t hb[kG];
            uint4 raw[kG];
#pragma unroll
            for (int g = 0; g < kG; ++g) {
                hb[g] = i + g < nblk ? __shfl_sync(kFull, h, (i + g) & 31) : 0ull;
                const uint32_t u = __shfl_sync(kFull, excl, (i + g) & 31);
                if ((uint32_t)lane < crz_width_sum(hb[g]))
                    raw[g] = *reinterpret_cast<const uint4 *>(units + 16ull * (u + lane));
            }
#pragma unroll
            for (int g = 0; g < kG; ++g)
                if ((uint32_t)lane < crz_width_sum(hb[g]))
                    *reinterpret_cast<uint4 *>(scratch + 512 * g + 16 * lane) = raw[g];
            __syncwarp();
#pragma unroll
            for (int g = 0; g < kG; ++g) {
                if (i + g >= nblk) break;
                uint32_t P[4];
                if ((uint32_t)(hb[g] >> 32) == 0) {
                    // every plane constant: each byte is its plane's minimum
#pragma unroll
                    for (int p = 0; p < 4; ++p) P[p] = ((uint32_t)(hb[g] >> (8 * p)) & 255u) * 0x01010101u;
                } else {
                    uint32_t col[4];   // lane 8q + j: word q of the plane's unit j
                    uint32_t u = 0;
#pragma unroll
                    for (int p = 0; p < 4; ++p) {
                        const uint32_t W = crz_width(hb[g], p);
                        col[p] = j < W ? *reinterpret_cast<const uint32_t *>(scratch + 512 * g + 16 * (u + j) + 4 * q)
                                       : 0u;
                        u += W;
                    }
#pragma unroll
                    for (int p = 0; p < 4; ++p) {
                        const uint32_t m = (uint32_t)(hb[g] >> (8 * p)) & 255u, W = crz_width(hb[g], p);
                        // the transpose hands lane l its four values' offsets from the
                        // minimum (unconditionally: a width-0 plane transposes zeros, and
                        // the four planes' chains interleave)
                        const uint32_t d = crz_warp_transpose(col[p], LT);
                        const uint32_t m4 = m * 0x01010101u;
                        if (m + (1u << W) - 1u <= 255u) {
                            P[p] = d + m4;   // no byte can pass 255: a plain add carries nowhere
                        } else {
                            // bytewise d + m: the sum without carries between bytes,
                            // and the bytes whose sum passes 255
                            const uint32_t s7 = (d & 0x7F7F7F7Fu) + (m4 & 0x7F7F7F7Fu);
                            const uint32_t sum = s7 ^ ((d ^ m4) & 0x80808080u);
                            over |= (((d & m4) | ((d | m4) & ~sum)) & 0x80808080u) != 0;
                            P[p] = sum;
                        }
                    }
                }
                uint32_t r[4];
                crz_bytes_transpose(P, r);
                store16_any(dst + 512ull * (b0 + i + g) + 16u * lane,
                            make_uint4(crz_unrot(r[0]), crz_unrot(r[1]), crz_unrot(r[2]), crz_unrot(r[3])));
            }
            __syncwarp();   // the scratch is rewritten by the next group
        }
    }
    for (uint64_t i = lane; i < tl; i += 32) dst[512ull * nb + i] = units[16ull * tot + i];
    return !__any_sync(kFull, over);
}

}  // namespace
}  // namespace crac
