// The split pass (hash -> finalize + compaction -> gather, one graph) and its
// sparse variant.
#include "crac_codec.cuh"

namespace crac {

namespace {

// ---------------------------------------------------------------------------
// Split pass: H (hash) -> F (finalize + dirty test + compaction) -> G (gather).
//
// H streams the tracked bytes with no inter-CTA dependency: every warp takes
// a contiguous range of segments (8 KiB, or the chunk if smaller), issues all
// of a segment's 128-bit loads at once (16 per lane), sums the per-word
// terms, and adds the warp's sum into the chunk's accumulator with one 64-bit
// atomicAdd.  The CRAC-FP64 sum is taken mod 2^64, so the order of these
// additions does not change a bit.  F turns each accumulator into the
// fingerprint, tests it against the baseline, and compacts the dirty chunks
// (ballot + block scan per 1024-chunk tile, decoupled look-back across
// tiles).  G copies the listed chunks into staging.  HBM traffic: B + 2D plus
// small tables, against B + D for the fused kernels, in exchange for three
// dependency-free streaming phases.
// ---------------------------------------------------------------------------
constexpr int kHashNT = 256;
constexpr int kFinNT = 1024;
constexpr int kGatherNT = 256;

// In the pass graph, finalize and gather hang off their producer by a
// programmatic edge, so they are launched while it drains: each waits here
// until the producing grid has completed and its writes are visible before
// touching what it wrote.  In an ordinary stream launch this returns at once.
__device__ __forceinline__ void wait_for_producer() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

// A chunk of len bytes predicted at staging offset po is written there by the
// hash kernels (and then found in place by the gather) when the offset is
// 16-byte aligned (vector stores) and the chunk fits the staging buffer.
__device__ __forceinline__ bool spec_ok(const CkptParams &P, uint64_t po, uint64_t len) {
    return po != ~0ull && (po & 15u) == 0 && po <= P.staging_cap && len <= P.staging_cap - po;
}

// Partial CRAC-FP64 sum of a segment (<= 8 KiB) whose first word is word j0
// of its chunk, over the lanes of one warp; with copy_to, the segment's bytes
// are also stored there, and then (kHdr) the CRZ1 header word of each whole
// 512-byte block of the segment goes to hdr[block] (lane l holds bytes
// 16l .. 16l+15 of block u in q[u], the encoder's layout of a block).  Only
// chunks written to staging get headers, so their cost follows the dirty bytes.
template <bool kHdr = false>
__device__ __forceinline__ uint64_t hash_seg(const uint8_t *__restrict__ src, uint32_t len, uint64_t j0,
                                             int lane, uint4 *__restrict__ copy_to = nullptr,
                                             uint64_t *__restrict__ hdr = nullptr) {
    const uint4 *p = reinterpret_cast<const uint4 *>(src);
    const uint32_t nv = len >> 4;
    constexpr int U = 16;
    uint4 q[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const uint32_t v = lane + 32u * u;
        if (v < nv) q[u] = __ldg(p + v);
    }
    if (copy_to) {   // FULL checkpoint: the vectors also go straight to staging
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t v = lane + 32u * u;
            if (v < nv) __stcs(copy_to + v, q[u]);
        }
    }
    uint64_t acc = 0;
    uint64_t key = (j0 + 2ull * (uint64_t)lane + 1ull) * kK1;
    constexpr uint64_t kStep = 64ull * kK1;
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const uint32_t v = lane + 32u * u;
        if (v < nv) {
            acc += mixw(((uint64_t)q[u].y << 32) | q[u].x, key);
            acc += mixw(((uint64_t)q[u].w << 32) | q[u].z, key + kK1);
        }
        key += kStep;
    }
    if (kHdr && copy_to) {
        const uint32_t nb = len >> 9;   // whole blocks (warp-uniform)
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if ((uint32_t)u < nb) {
                const uint32_t r[4] = {crz_rot(q[u].x), crz_rot(q[u].y), crz_rot(q[u].z), crz_rot(q[u].w)};
                const uint64_t h = crz_block_header(r);
                if (lane == 0) hdr[u] = h;
            }
        }
    }
    const uint32_t rem = len & 15u;
    if (rem && lane == (int)(nv & 31u)) {
        const uint8_t *t = src + 16ull * nv;
        uint64_t w0 = 0, w1 = 0;
        for (uint32_t b = 0; b < rem; ++b) {
            const uint64_t byte = t[b];
            if (b < 8) w0 |= byte << (8 * b);
            else w1 |= byte << (8 * (b - 8));
            if (copy_to) reinterpret_cast<uint8_t *>(copy_to + nv)[b] = (uint8_t)byte;
        }
        const uint64_t kt = (j0 + 2ull * nv + 1ull) * kK1;
        acc += mixw(w0, kt);
        if (rem > 8) acc += mixw(w1, kt + kK1);
    }
    return acc;
}

// One warp copies a chunk of len bytes from src (16-byte aligned) to dst and
// stores the CRZ1 header word of each whole 512-byte block b at hdr[b], in the
// encoder's layout (lane l holds bytes 16l .. 16l+15 of the block).  A dst off
// the 16-byte grid is copied by copy_group, which re-reads the (cached) source.
__device__ __forceinline__ void copy_with_headers(uint8_t *__restrict__ dst, const uint8_t *__restrict__ src,
                                                  uint64_t len, int lane, uint64_t *__restrict__ hdr) {
    const uint64_t nb = len >> 9;
    const uint4 *s = reinterpret_cast<const uint4 *>(src);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    const bool vec = ((uintptr_t)dst & 15u) == 0;
    constexpr int U = 8;
    for (uint64_t b = 0; b < nb; b += U) {   // warp-uniform
        uint4 q[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (b + u < nb) q[u] = __ldg(s + 32 * (b + u) + lane);
        if (vec) {
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (b + u < nb) __stcs(d + 32 * (b + u) + lane, q[u]);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (b + u < nb) {
                const uint32_t r[4] = {crz_rot(q[u].x), crz_rot(q[u].y), crz_rot(q[u].z), crz_rot(q[u].w)};
                const uint64_t h = crz_block_header(r);
                if (lane == 0) hdr[b + u] = h;
            }
        }
    }
    if (vec) copy_group<32>(dst + (nb << 9), src + (nb << 9), len - (nb << 9), lane);
    else copy_group<32>(dst, src, len, lane);
}

template <bool kHdr>
__global__ void __launch_bounds__(kHashNT, 2)
split_hash_kernel(const CkptParams P, unsigned long long *__restrict__ acc, uint32_t log2Seg) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp_g = ((uint64_t)blockIdx.x * kHashNT + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * kHashNT) >> 5;
    const uint32_t log2S = P.log2_chunk;
    const uint32_t spc = log2S - log2Seg;   // log2 of segments per chunk
    const uint64_t n_slots = (P.c_end - P.c_begin) << spc;
    const uint64_t per = (n_slots + n_warps - 1) / n_warps;
    uint64_t q = warp_g * per;
    const uint64_t q_end = umin64(q + per, n_slots);
    CkptDesc d{};
    uint64_t a_next = 0;
    uint32_t a = 0;
    bool have = false;
    uint32_t writes = 0;   // chunks this warp wrote speculatively (lane 0)
    for (; q < q_end; ++q) {
        const uint64_t c = P.c_begin + (q >> spc);
        if (!have || c >= a_next) {
            a = find_alloc(P.desc, P.n_allocs, c);
            d = P.desc[a];
            a_next = a + 1 < P.n_allocs ? P.desc[a + 1].first_chunk : ~0ull;
            have = true;
        }
        const uint64_t local = c - d.first_chunk;
        const uint64_t rest = d.bytes - (local << log2S);
        const uint64_t clen = rest < (1ull << log2S) ? rest : (1ull << log2S);
        const uint64_t off = (q & ((1ull << spc) - 1)) << log2Seg;
        if (off >= clen) continue;   // beyond the end of a short last chunk (warp-uniform)
        const uint32_t len = (uint32_t)umin64(1ull << log2Seg, clen - off);
        // Direct mode (S <= 8 KiB, the warp sees the whole chunk): the baseline
        // fingerprint is loaded before the chunk so that both latencies overlap.
        uint64_t fo = 0;
        const bool has = d.base_first != kNoBase;
        if (spc == 0 && lane == 0 && has) fo = __ldg(P.fp_old + d.base_first + local);
        const uint8_t *src = reinterpret_cast<const uint8_t *>(d.ptr) + (local << log2S) + off;
        uint4 *copy_to = nullptr;
        if (P.full_copy) {   // FULL checkpoint: the segment's final staging offset is known
            const uint64_t o = P.alloc_prefix[a] + (local << log2S) + off - P.seg_base;
            if (o + len <= P.staging_cap) copy_to = reinterpret_cast<uint4 *>(P.staging + o);
            else if (lane == 0) atomicOr(&P.ctrl->err, kErrBounds);
        } else if (P.ppos) {   // predicted dirty: written to the offset it had last time
            const uint64_t po = __ldg(P.ppos + (c - P.c_begin));
            if (spec_ok(P, po, clen)) {
                copy_to = reinterpret_cast<uint4 *>(P.staging + po + off);
                writes += off == 0 ? 1u : 0u;
            }
        }
        uint64_t sum = kHdr ? hash_seg<true>(src, len, off >> 3, lane, copy_to,
                                             P.crz_hdr + (c << (log2S - 9)) + (off >> 9))
                            : hash_seg(src, len, off >> 3, lane, copy_to);
        sum = warp_sum(sum);
        if (lane == 0) {
            if (spc == 0) {
                // The warp has seen the whole chunk: finalize here and leave only
                // the length and the dirty bit for the compaction kernel.
                const uint64_t fp = fp_finalize(sum, len);
                P.fp_new[c] = fp;
                acc[c - P.c_begin] = len | ((!has || fo != fp) ? kAccDirty : 0ull);
            } else {
                atomicAdd(acc + (c - P.c_begin), (unsigned long long)sum);
            }
        }
    }
    if (lane == 0 && writes) atomicAdd(&P.ctrl->spec_writes, (unsigned long long)writes);
}

// When log2Seg == log2_chunk the hash kernel has already finalized every
// chunk and left its length and dirty bit in acc; only the compaction remains.
// Hash kernel for chunks of 512 B..4 KiB: one warp iteration covers 8 KiB,
// i.e. 8192/S whole chunks, one group of LPC = 32*S/8192 lanes per chunk (16
// vectors per lane), so a warp keeps 8 KiB in flight whatever the chunk size.
// Every chunk is finalized in place (direct mode: acc receives the dirty
// length).
template <int LPC>
__device__ __forceinline__ void hash_small_iter(const CkptParams &P, unsigned long long *__restrict__ acc,
                                                uint64_t c, const CkptDesc &d_warp, uint32_t a_warp,
                                                uint64_t a_next, int li, uint32_t &writes) {
    const uint32_t log2S = P.log2_chunk;
    uint64_t sum = 0, fo = 0;
    uint32_t len = 0, nv = 0;
    bool has = false;
    CkptDesc d = d_warp;
    uint32_t a = a_warp;
    uint64_t local = 0;
    uint4 q[16];
    // Sparse delta pass: the group holds its whole chunk in q until the
    // fingerprint is known and stores it only if it is dirty (B + D of HBM
    // traffic instead of B + B); clean chunks' bytes are never referenced.
    bool hold = false;
    if (c < P.c_end) {
        if (c >= a_next) {   // the segment crosses an allocation end
            a = find_alloc(P.desc, P.n_allocs, c);
            d = P.desc[a];
        }
        local = c - d.first_chunk;
        const uint64_t rest = d.bytes - (local << log2S);
        len = (uint32_t)umin64(rest, 1ull << log2S);
        has = d.base_first != kNoBase;
        hold = P.sparse && has;
        if (li == 0 && has) fo = __ldg(P.fp_old + d.base_first + local);
        const uint4 *p = reinterpret_cast<const uint4 *>(reinterpret_cast<const uint8_t *>(d.ptr) + (local << log2S));
        nv = len >> 4;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const uint32_t v = li + LPC * u;
            if (v < nv) q[u] = __ldg(p + v);
        }
        uint64_t key = (2ull * (uint64_t)li + 1ull) * kK1;
        constexpr uint64_t kStep = 2ull * LPC * kK1;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const uint32_t v = li + LPC * u;
            if (v < nv) {
                sum += mixw(((uint64_t)q[u].y << 32) | q[u].x, key);
                sum += mixw(((uint64_t)q[u].w << 32) | q[u].z, key + kK1);
            }
            key += kStep;
        }
        if (P.full_copy && !hold) {   // FULL checkpoint: the chunk goes straight to its staging offset
            const uint64_t o = P.alloc_prefix[a] + (local << log2S) - P.seg_base;
            if (o + len <= P.staging_cap) {
                uint4 *dst = reinterpret_cast<uint4 *>(P.staging + o);
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const uint32_t v = li + LPC * u;
                    if (v < nv) __stcs(dst + v, q[u]);
                }
            } else if (li == 0) {
                atomicOr(&P.ctrl->err, kErrBounds);
            }
        } else if (P.ppos) {   // predicted dirty: written to the offset it had last time
            const uint64_t po = __ldg(P.ppos + (c - P.c_begin));
            if (spec_ok(P, po, len)) {
                writes += li == 0 ? 1u : 0u;
                uint8_t *dst = P.staging + po;
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const uint32_t v = li + LPC * u;
                    if (v < nv) __stcs(reinterpret_cast<uint4 *>(dst) + v, q[u]);
                }
                const uint32_t rem = len & 15u;
                if (rem && (uint32_t)li == (nv % LPC)) {
                    const uint8_t *t = reinterpret_cast<const uint8_t *>(p + nv);
                    for (uint32_t b = 0; b < rem; ++b) dst[16 * nv + b] = t[b];
                }
            }
        }
        const uint32_t rem = len & 15u;
        if (rem && (uint32_t)li == (nv % LPC)) {
            const uint8_t *t = reinterpret_cast<const uint8_t *>(p + nv);
            uint64_t w0 = 0, w1 = 0;
            for (uint32_t b = 0; b < rem; ++b) {
                const uint64_t byte = t[b];
                if (b < 8) w0 |= byte << (8 * b);
                else w1 |= byte << (8 * (b - 8));
            }
            const uint64_t kt = (2ull * nv + 1ull) * kK1;
            sum += mixw(w0, kt);
            if (rem > 8) sum += mixw(w1, kt + kK1);
        }
    }
    // butterfly: every lane of the group ends with the group's sum
#pragma unroll
    for (int o = LPC / 2; o; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
    const uint64_t fp = fp_finalize(sum, len);
    // the group leader's baseline fingerprint, for every lane of the group
    fo = __shfl_sync(kFull, fo, (int)(threadIdx.x & 31u) - li);
    const bool dirty = !has || fo != fp;
    if (li == 0 && c < P.c_end) {
        P.fp_new[c] = fp;
        acc[c - P.c_begin] = len | (dirty ? kAccDirty : 0ull);
    }
    if (hold && dirty) {   // sparse delta pass: sizes are multiples of 16 (no tail bytes)
        const uint64_t o = P.alloc_prefix[a] + (local << log2S) - P.seg_base;
        if (o + len <= P.staging_cap) {
            uint4 *dst = reinterpret_cast<uint4 *>(P.staging + o);
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const uint32_t v = li + LPC * u;
                if (v < nv) __stcs(dst + v, q[u]);
            }
        } else if (li == 0) {
            atomicOr(&P.ctrl->err, kErrBounds);
        }
    }
}

template <int LPC>
__global__ void __launch_bounds__(kHashNT, 2)
split_hash_small_kernel(const CkptParams P, unsigned long long *__restrict__ acc, uint32_t) {
    constexpr int CPS = 32 / LPC;   // chunks per 8 KiB segment
    const int lane = threadIdx.x & 31;
    const uint64_t warp_g = ((uint64_t)blockIdx.x * kHashNT + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * kHashNT) >> 5;
    const uint64_t n_slots = (P.c_end - P.c_begin + CPS - 1) / CPS;
    const uint64_t per = (n_slots + n_warps - 1) / n_warps;
    uint64_t q = warp_g * per;
    const uint64_t q_end = umin64(q + per, n_slots);
    CkptDesc d{};
    uint64_t a_next = 0;
    uint32_t a = 0;
    bool have = false;
    uint32_t writes = 0;   // chunks this lane's groups wrote speculatively (group leaders)
    for (; q < q_end; ++q) {
        const uint64_t c0 = P.c_begin + q * CPS;
        if (!have || c0 >= a_next) {
            a = find_alloc(P.desc, P.n_allocs, c0);
            d = P.desc[a];
            a_next = a + 1 < P.n_allocs ? P.desc[a + 1].first_chunk : ~0ull;
            have = true;
        }
        hash_small_iter<LPC>(P, acc, c0 + lane / LPC, d, a, a_next, lane % LPC, writes);
    }
    writes = __reduce_add_sync(kFull, writes);
    if (lane == 0 && writes) atomicAdd(&P.ctrl->spec_writes, (unsigned long long)writes);
}

// ---------------------------------------------------------------------------
// Sparse pass on 512 B - 4 KiB chunks with dense placement (P.sparse == 2).
// Each warp iteration hashes 8 KiB of whole chunks as split_hash_small_kernel
// does, then stages its dirty chunks back to back in the warp's 8 KiB of
// shared memory and takes their room in the image from a running byte
// counter (P.ctrl->pad[0], one atomicAdd per iteration with dirty bytes).
// The counter's answer is used one iteration later: after the next
// iteration's loads are issued, one lane stores the staged bytes with a bulk
// copy (shared -> global) and the group leaders record each chunk's offset
// in its accumulator word, so neither the atomic's round trip nor the store
// holds the loads up.  The image's span is then exactly its dirty bytes.
// Sizes are multiples of 16 (a sparse pass requires it), so every staged
// chunk and every offset is 16-byte aligned.
// ---------------------------------------------------------------------------
constexpr uint32_t kDenseWarpBytes = 8192;   // shared memory per warp
constexpr uint64_t kAccLenMask = (1ull << 24) - 1;   // accumulator word: length in bits 0-23,
constexpr int kAccPosShift = 24;                     // the chunk's offset in bits 24-62 (dense
constexpr uint64_t kAccPosMask = (1ull << 39) - 1;   // sparse placement), kAccDirty in bit 63

__device__ __forceinline__ void dense_bulk_store(void *dst, const void *src_smem, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                 "r"((uint32_t)__cvta_generic_to_shared(src_smem)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void dense_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void dense_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void dense_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

template <int LPC>
__global__ void __launch_bounds__(kHashNT, 2)
split_hash_small_dense_kernel(const CkptParams P, unsigned long long *__restrict__ acc, uint32_t) {
    extern __shared__ __align__(128) uint8_t dense_smem[];
    constexpr int CPS = 32 / LPC;   // chunks per 8 KiB iteration
    const int lane = threadIdx.x & 31;
    const int li = lane % LPC;
    uint8_t *buf = dense_smem + (threadIdx.x >> 5) * kDenseWarpBytes;
    const uint64_t warp_g = ((uint64_t)blockIdx.x * kHashNT + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * kHashNT) >> 5;
    const uint64_t n_slots = (P.c_end - P.c_begin + CPS - 1) / CPS;
    const uint64_t per = (n_slots + n_warps - 1) / n_warps;
    uint64_t q = warp_g * per;
    const uint64_t q_end = umin64(q + per, n_slots);
    const uint32_t log2S = P.log2_chunk;
    CkptDesc dw{};
    uint64_t a_next = 0;
    uint32_t aw = 0;
    bool have = false;
    // the previous iteration's staged chunks: warp-uniform byte count, the
    // counter's answer (lane 0), and each group's chunk, length and offset
    uint32_t pend_total = 0;
    unsigned long long pend_base = 0;
    uint64_t pend_c = 0;
    uint32_t pend_len = 0, pend_loc = 0;
    bool pend_dirty = false;
    auto flush = [&]() {
        if (!pend_total) return;   // warp-uniform
        const uint64_t base = __shfl_sync(kFull, (uint64_t)pend_base, 0);
        const bool fits = base + pend_total <= P.staging_cap;
        if (lane == 0) {
            if (fits) dense_bulk_store(P.staging + base, buf, pend_total);
            else atomicOr(&P.ctrl->err, kErrBounds);
        }
        if (li == 0 && pend_dirty)
            acc[pend_c - P.c_begin] = pend_len | kAccDirty | ((fits ? base + pend_loc : 0ull) << kAccPosShift);
        pend_total = 0;
    };
    for (; q < q_end; ++q) {
        const uint64_t c0 = P.c_begin + q * CPS;
        if (!have || c0 >= a_next) {
            aw = find_alloc(P.desc, P.n_allocs, c0);
            dw = P.desc[aw];
            a_next = aw + 1 < P.n_allocs ? P.desc[aw + 1].first_chunk : ~0ull;
            have = true;
        }
        const uint64_t c = c0 + lane / LPC;
        uint64_t sum = 0, fo = 0;
        uint32_t len = 0, nv = 0;
        bool has = false;
        uint4 v16[16];
        if (c < P.c_end) {
            CkptDesc d = dw;
            if (c >= a_next) d = P.desc[find_alloc(P.desc, P.n_allocs, c)];   // the iteration crosses an allocation end
            const uint64_t local = c - d.first_chunk;
            len = (uint32_t)umin64(d.bytes - (local << log2S), 1ull << log2S);
            has = d.base_first != kNoBase;
            if (li == 0 && has) fo = __ldg(P.fp_old + d.base_first + local);
            const uint4 *p = reinterpret_cast<const uint4 *>(reinterpret_cast<const uint8_t *>(d.ptr) + (local << log2S));
            nv = len >> 4;
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const uint32_t v = li + LPC * u;
                if (v < nv) v16[u] = __ldg(p + v);
            }
        }
        flush();   // the previous iteration's chunks leave shared memory while these loads are in flight
        if (c < P.c_end) {
            uint64_t key = (2ull * (uint64_t)li + 1ull) * kK1;
            constexpr uint64_t kStep = 2ull * LPC * kK1;
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const uint32_t v = li + LPC * u;
                if (v < nv) {
                    sum += mixw(((uint64_t)v16[u].y << 32) | v16[u].x, key);
                    sum += mixw(((uint64_t)v16[u].w << 32) | v16[u].z, key + kK1);
                }
                key += kStep;
            }
        }
#pragma unroll
        for (int o = LPC / 2; o; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
        const uint64_t fp = fp_finalize(sum, len);
        fo = __shfl_sync(kFull, fo, lane - li);
        const bool dirty = c < P.c_end && (!has || fo != fp);
        if (li == 0 && c < P.c_end) {
            P.fp_new[c] = fp;
            if (!dirty) acc[c - P.c_begin] = len;
        }
        // stage the dirty chunks back to back in the warp's buffer
        const uint64_t mine = (li == 0 && dirty) ? len : 0u;
        const uint64_t incl = warp_incl_scan(mine, lane);
        const uint32_t total = (uint32_t)__shfl_sync(kFull, incl, 31);
        const uint32_t loc = (uint32_t)__shfl_sync(kFull, incl - mine, lane - li);
        if (total) {   // warp-uniform
            if (lane == 0) dense_wait_read();   // the previous bulk store has read the buffer
            __syncwarp();
            if (dirty) {
                uint4 *dst = reinterpret_cast<uint4 *>(buf + loc);
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    const uint32_t v = li + LPC * u;
                    if (v < nv) dst[v] = v16[u];
                }
            }
            dense_fence();   // the staged bytes are visible to the bulk copy
            __syncwarp();
            if (lane == 0) pend_base = atomicAdd(&P.ctrl->pad[0], (unsigned long long)total);
        }
        pend_total = total;
        pend_c = c;
        pend_len = len;
        pend_loc = loc;
        pend_dirty = dirty;
    }
    flush();
    if (lane == 0) dense_wait_all();   // shared memory stays until the bulk stores have finished
}

constexpr uint32_t kFinCachedAllocs = 4096;   // first_chunk columns the finalize keeps on chip

__global__ void __launch_bounds__(kFinNT)
split_finalize_kernel(const CkptParams P, unsigned long long *__restrict__ acc, uint32_t log2Seg) {
    const bool direct = log2Seg == P.log2_chunk;
    // Segmented chunks need their allocation: searched in an on-chip copy of
    // the first_chunk column when it fits (a search in global memory is a
    // chain of dependent loads per chunk).
    __shared__ uint64_t s_first[kFinCachedAllocs];
    const bool cached = !direct && P.n_allocs <= kFinCachedAllocs;
    if (cached)   // the descriptors were copied before the pass
        for (uint32_t a = threadIdx.x; a < P.n_allocs; a += kFinNT) s_first[a] = P.desc[a].first_chunk;
    wait_for_producer();   // the hash kernel's accumulators
    __shared__ uint32_t s_wcnt[32];
    __shared__ uint64_t s_wbytes[32];
    __shared__ uint64_t s_wdirty[32];
    __shared__ uint64_t s_k0, s_d0;
    __shared__ uint32_t s_tile;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t log2S = P.log2_chunk;
    const uint64_t S = 1ull << log2S;
    for (;;) {
        if (threadIdx.x == 0) {
            uint32_t t = atomicAdd(&P.ctrl->ticket, 1u);
            if (P.skip_first_ticket && t == 0) t = atomicAdd(&P.ctrl->ticket, 1u);
            s_tile = t;
        }
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= P.n_tiles) break;
        const uint64_t c = P.c_begin + (uint64_t)tile * kFinNT + threadIdx.x;
        uint32_t dl = 0, len = 0;
        uint64_t dpos = 0;   // dense sparse placement: the chunk's offset in the span
        if (c < P.c_end && direct) {
            const uint64_t v = acc[c - P.c_begin];
            len = (uint32_t)(v & kAccLenMask);
            dl = (v & kAccDirty) ? len : 0u;
            dpos = (v >> kAccPosShift) & kAccPosMask;
        } else if (c < P.c_end) {
            uint32_t a;
            if (cached) {
                uint32_t lo = 0, hi = P.n_allocs;
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (s_first[mid] <= c) lo = mid;
                    else hi = mid;
                }
                a = lo;
            } else {
                a = find_alloc(P.desc, P.n_allocs, c);
            }
            const CkptDesc d = P.desc[a];
            const uint64_t local = c - d.first_chunk;
            len = (uint32_t)min(S, d.bytes - (local << log2S));
            const uint64_t fp = fp_finalize(acc[c - P.c_begin], len);
            P.fp_new[c] = fp;
            const bool dirty = d.base_first == kNoBase || P.fp_old[d.base_first + local] != fp;
            dl = dirty ? len : 0u;
        }
        if (P.ppos_next && c < P.c_end) P.ppos_next[c - P.c_begin] = ~0ull;   // the gather sets the dirty ones
        // Bytes that advance the staging offset: the dirty ones, or in the
        // sparse pass every chunk's (each sits at its uncompacted offset);
        // under dense placement the dirty ones, whose offsets the hash kernel
        // recorded.
        const uint32_t sv = P.sparse == 1u ? len : dl;
        const unsigned m = __ballot_sync(kFull, dl != 0);
        const uint64_t incl = warp_incl_scan(sv, lane);
        if (P.sparse) {
            const uint64_t wd = warp_sum((uint64_t)dl);
            if (lane == 0) s_wdirty[warp] = wd;
        }
        if (lane == 31) {
            s_wcnt[warp] = __popc(m);
            s_wbytes[warp] = incl;
        }
        __syncthreads();
        if (P.sparse && warp == 1) {   // the tile's dirty bytes, one atomic per tile
            const uint64_t td = warp_sum(s_wdirty[lane]);
            if (lane == 0 && td) atomicAdd(&P.ctrl->payload, (unsigned long long)td);
        }
        if (warp == 0) {
            const uint32_t wc = s_wcnt[lane];
            const uint64_t wb = s_wbytes[lane];
            uint32_t ic = wc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(kFull, ic, o);
                if (lane >= o) ic += t;
            }
            const uint64_t ib = warp_incl_scan(wb, lane);
            const uint32_t cnt = __shfl_sync(kFull, ic, 31);
            const uint64_t bytes = __shfl_sync(kFull, ib, 31);
            s_wcnt[lane] = ic - wc;
            s_wbytes[lane] = ib - wb;
            uint64_t k0 = 0, d0 = 0;
            if (tile == 0) {
                if (lane == 0) {
                    st_status(P.tile_cnt, kFlagInc | cnt);
                    st_status(P.tile_bytes, kFlagInc | bytes);
                }
            } else {
                if (lane == 0) {
                    st_status(P.tile_cnt + tile, kFlagAgg | cnt);
                    st_status(P.tile_bytes + tile, kFlagAgg | bytes);
                }
                lookback(P, tile, lane, &k0, &d0);
                if (lane == 0) {
                    st_status(P.tile_cnt + tile, kFlagInc | ((k0 + cnt) & kValMask));
                    st_status(P.tile_bytes + tile, kFlagInc | ((d0 + bytes) & kValMask));
                }
            }
            if (lane == 0) {
                s_k0 = k0;
                s_d0 = d0;
                if (tile == P.n_tiles - 1) {
                    P.ctrl->k = k0 + cnt;
                    P.ctrl->D = d0 + bytes;
                    if (k0 + cnt <= P.idx_cap) P.off_out[k0 + cnt] = d0 + bytes;
                    else atomicOr(&P.ctrl->err, kErrBounds);
                }
            }
        }
        __syncthreads();
        if (dl) {
            const uint64_t j = s_k0 + s_wcnt[warp] + __popc(m & ((1u << lane) - 1u));
            if (j < P.idx_cap) {
                P.idx_out[j] = c;
                P.off_out[j] = P.sparse == 2u ? dpos : s_d0 + s_wbytes[warp] + incl - sv;
            } else {
                atomicOr(&P.ctrl->err, kErrBounds);
            }
        }
        __syncthreads();
    }
}

// kHdr: P.crz_hdr is set, and each copied chunk's block headers are written
// too (a separate instance, so that the plain gather keeps its registers low).
template <bool kHdr>
__global__ void __launch_bounds__(kGatherNT)
split_gather_kernel(const CkptParams P, unsigned long long *, uint32_t) {
    if (P.full_copy) return;   // the hash kernel has already written every chunk
    wait_for_producer();       // the finalize kernel's list and counts
    const int lane = threadIdx.x & 31;
    const uint64_t kd = (uint64_t)P.ctrl->k;
    const uint64_t k = kd < P.idx_cap ? kd : P.idx_cap;
    const uint32_t log2S = P.log2_chunk;
    const uint64_t S = 1ull << log2S;
    const uint64_t nw = ((uint64_t)gridDim.x * kGatherNT) >> 5;
    // The next pass predicts this pass's offsets, if few enough chunks are dirty.
    uint64_t *next = (P.ppos_next && 2 * kd <= P.c_end - P.c_begin) ? P.ppos_next : nullptr;
    // Every entry ends by the segment's dirty bytes, which must fit staging.
    if (blockIdx.x == 0 && threadIdx.x == 0 && P.ctrl->D > P.staging_cap) atomicOr(&P.ctrl->err, kErrBounds);
    __shared__ unsigned int s_hits;
    if (threadIdx.x == 0) s_hits = 0;
    __syncthreads();
    uint32_t hits = 0;
    for (uint64_t j = ((uint64_t)blockIdx.x * kGatherNT + threadIdx.x) >> 5; j < k; j += nw) {
        const uint64_t c = P.idx_out[j];
        const uint64_t o = P.off_out[j];
        if (next && lane == 0) next[c - P.c_begin] = o;
        // Written there by the hash kernel already: a predicted offset equal
        // to the entry's is aligned, and the chunk fits (it ends by D).
        if (P.ppos) {
            const uint64_t po = P.ppos[c - P.c_begin];
            if (po == o && (po & 15u) == 0) {
                ++hits;
                continue;
            }
        }
        const CkptDesc d = P.desc[find_alloc(P.desc, P.n_allocs, c)];
        const uint64_t local = c - d.first_chunk;
        const uint64_t len = min(S, d.bytes - (local << log2S));
        if (o + len > P.staging_cap) {
            if (lane == 0) atomicOr(&P.ctrl->err, kErrBounds);
            continue;
        }
        const uint8_t *src = reinterpret_cast<const uint8_t *>(d.ptr) + (local << log2S);
        if (kHdr) copy_with_headers(P.staging + o, src, len, lane, P.crz_hdr + (c << (log2S - 9)));
        else copy_group<32>(P.staging + o, src, len, lane);
    }
    if (lane == 0 && hits) atomicAdd(&s_hits, hits);
    __syncthreads();
    if (threadIdx.x == 0 && s_hits) atomicAdd(&P.ctrl->spec_hits, (unsigned long long)s_hits);
}

}  // namespace

const void *split_hash_fn(bool crz_headers) {
    return crz_headers ? reinterpret_cast<const void *>(&split_hash_kernel<true>)
                       : reinterpret_cast<const void *>(&split_hash_kernel<false>);
}
const void *split_hash_small_fn(int lanes_per_chunk) {
    switch (lanes_per_chunk) {
    case 2: return reinterpret_cast<const void *>(&split_hash_small_kernel<2>);
    case 4: return reinterpret_cast<const void *>(&split_hash_small_kernel<4>);
    case 8: return reinterpret_cast<const void *>(&split_hash_small_kernel<8>);
    case 16: return reinterpret_cast<const void *>(&split_hash_small_kernel<16>);
    default: return nullptr;
    }
}
const void *split_finalize_fn() { return reinterpret_cast<const void *>(&split_finalize_kernel); }
const void *split_gather_fn(bool crz_headers) {
    return crz_headers ? reinterpret_cast<const void *>(&split_gather_kernel<true>)
                       : reinterpret_cast<const void *>(&split_gather_kernel<false>);
}
int split_hash_threads() { return kHashNT; }
int split_finalize_threads() { return kFinNT; }
int split_gather_threads() { return kGatherNT; }
const void *split_hash_small_dense_fn(int lanes_per_chunk) {
    switch (lanes_per_chunk) {
    case 2: return reinterpret_cast<const void *>(&split_hash_small_dense_kernel<2>);
    case 4: return reinterpret_cast<const void *>(&split_hash_small_dense_kernel<4>);
    case 8: return reinterpret_cast<const void *>(&split_hash_small_dense_kernel<8>);
    case 16: return reinterpret_cast<const void *>(&split_hash_small_dense_kernel<16>);
    default: return nullptr;
    }
}
size_t split_dense_smem() { return (size_t)(kHashNT / 32) * kDenseWarpBytes; }
cudaError_t split_dense_prepare(const void *fn) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)split_dense_smem());
}
int split_max_ctas_per_sm_smem(const void *fn, int threads, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}
int split_max_ctas_per_sm(const void *fn, int threads) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, 0) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

}  // namespace crac
