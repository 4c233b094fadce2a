// Device-side building blocks of the checkpoint/restart data pass (sm_103a),
// shared by the kernel units:
//   crac_pass_split.cu      the split pass (default) and the sparse pass
//   crac_pass_fused.cu      the fused LDG pass
//   crac_pass_tma.cu        the fused TMA pass
//   crac_pass_per_alloc.cu  the per-allocation comparison path
//   crac_restore.cu         chain resolution and scatter (restart)
//   crac_noalloc.cu         the allocation-free entry point
//
// The paper drains the device and copies the memory of every active
// allocation to the host at checkpoint, and copies it back at restart
// (Sec. 3.2, "Saving the library-allocated arena" and "restoring the CUDA
// library-allocated regions").  The kernel units implement that copy as an
// incremental, HBM-bound pass:
//
//   K1 fingerprint  each chunk of each allocation -> 64-bit CRAC-FP64 value
//   K2 dirty test   fp_new != fp_old (or no baseline) -> compacted dirty list
//                   in ascending global chunk order, with byte offsets
//   K3 gather       dirty chunks -> contiguous staging buffer
//   K4 scatter      staging (or a device-resident image) -> allocations
//
// The batched path fuses K1-K3 into one persistent kernel: CTAs take tiles
// of consecutive global chunks from an atomic ticket counter, hash them,
// publish the tile's dirty count and bytes, and find their exclusive prefix
// with a decoupled look-back over earlier tiles (Merrill & Garland,
// "Single-pass Parallel Prefix Scan with Decoupled Look-back", 2016).  The
// gather then re-reads the tile's dirty chunks, which the hash has just
// pulled into L2.  The per-allocation path runs K1, K2 and K3 as separate
// launches per allocation and is kept as the comparison baseline.
//
// CRAC-FP64 (this project's hash; the paper has none), per chunk of len
// bytes read as little-endian u64 words w_j (last word zero-padded):
//   acc = sum_j f(w_j ^ (j+1)*K1)  mod 2^64,   f(x) = y ^ (y >> 32), y = x*M1
//   fp  = fmix(acc ^ len*M3) with fmix: z^=z>>31; z*=M2; z^=z>>29; z*=M1; z^=z>>32
// K1 = floor(2^64/phi); M1, M2, M3 = odd-forced 2^64*frac(sqrt 2, 3, 5).
// The sum is associative and commutative, so any reduction order gives the
// same bits.
//
// Every device-side wait is bounded by a %globaltimer limit; a wait that
// runs out sets an error bit in the control block and the kernel finishes
// with its output discarded by the host.  No kernel traps.
#pragma once

#include <cstdint>
#include <mutex>
#include <cuda_runtime.h>

#include "crac.h"
#include "crac_kernels.cuh"

namespace crac {

// Internal linkage: every kernel unit gets its own copy of these inlined helpers.
namespace {

constexpr uint64_t kK1 = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kM1 = 0x6A09E667F3BCC909ull;
constexpr uint64_t kM2 = 0xBB67AE8584CAA73Bull;
constexpr uint64_t kM3 = 0x3C6EF372FE94F82Bull;

constexpr unsigned kFull = 0xffffffffu;
constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagInc = 2ull << 62;
constexpr uint64_t kValMask = (1ull << 62) - 1;
constexpr int kMaxCpt = 256;
// Direct-mode hash output per chunk: its length, and this bit when dirty.
constexpr uint64_t kAccDirty = 1ull << 63;

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

__device__ __forceinline__ uint64_t mixw(uint64_t w, uint64_t key) {
    const uint64_t y = (w ^ key) * kM1;
    return y ^ (y >> 32);
}

__device__ __forceinline__ uint64_t fp_finalize(uint64_t acc, uint64_t len) {
    uint64_t z = acc ^ (len * kM3);
    z ^= z >> 31;
    z *= kM2;
    z ^= z >> 29;
    z *= kM1;
    z ^= z >> 32;
    return z;
}

__device__ __forceinline__ uint64_t warp_sum(uint64_t v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Look-back status words.  A word holds the flag and the value together and
// its reader needs nothing else the writing CTA produced (it only adds the
// values up), so plain gpu-scope (relaxed) accesses suffice: a release would
// make every publish wait for the writer's earlier stores, such as its
// fingerprints, to be acknowledged.
__device__ __forceinline__ void st_status(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t ld_status(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Partial CRAC-FP64 sum of one chunk over the vectors owned by thread gl of
// a GT-thread group.  Vector v (16 bytes) holds words 2v and 2v+1.
template <int GT>
__device__ __forceinline__ uint64_t hash_partial(const uint8_t *__restrict__ src, uint32_t len,
                                                 int gl) {
    const uint4 *p = reinterpret_cast<const uint4 *>(src);
    const uint32_t nv = len >> 4;
    uint64_t acc = 0;
    uint64_t key = (2ull * (uint64_t)gl + 1ull) * kK1;   // key of word 2v at v = gl
    constexpr uint64_t kStep = 2ull * GT * kK1;          // key advance for v += GT
    uint32_t v = gl;
    constexpr int U = 8;
    for (; v + (U - 1) * GT < nv; v += U * GT) {
        uint4 q[U];
#pragma unroll
        for (int u = 0; u < U; ++u) q[u] = __ldg(p + v + u * GT);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t w0 = ((uint64_t)q[u].y << 32) | q[u].x;
            const uint64_t w1 = ((uint64_t)q[u].w << 32) | q[u].z;
            acc += mixw(w0, key);
            acc += mixw(w1, key + kK1);
            key += kStep;
        }
    }
    for (; v < nv; v += GT) {
        const uint4 q = __ldg(p + v);
        acc += mixw(((uint64_t)q.y << 32) | q.x, key);
        acc += mixw(((uint64_t)q.w << 32) | q.z, key + kK1);
        key += kStep;
    }
    const uint32_t rem = len & 15u;
    if (rem && v == nv) {   // this thread owns the partial tail vector
        const uint8_t *t = src + 16ull * nv;
        uint64_t w0 = 0, w1 = 0;
        for (uint32_t b = 0; b < rem; ++b) {
            const uint64_t byte = t[b];
            if (b < 8) w0 |= byte << (8 * b);
            else w1 |= byte << (8 * (b - 8));
        }
        acc += mixw(w0, key);
        if (rem > 8) acc += mixw(w1, key + kK1);
    }
    return acc;
}

// Copy len bytes with the GT threads of a group (thread gl).
template <int GT>
__device__ __forceinline__ void copy_group(uint8_t *__restrict__ dst,
                                           const uint8_t *__restrict__ src, uint64_t len, int gl) {
    if ((((uintptr_t)dst | (uintptr_t)src) & 15u) == 0) {
        const uint64_t nv = len >> 4;
        const uint4 *s = reinterpret_cast<const uint4 *>(src);
        uint4 *d = reinterpret_cast<uint4 *>(dst);
        uint64_t v = gl;
        constexpr int U = 8;
        for (; v + (U - 1) * GT < nv; v += U * GT) {
            uint4 q[U];
#pragma unroll
            for (int u = 0; u < U; ++u) q[u] = s[v + u * GT];
#pragma unroll
            for (int u = 0; u < U; ++u) __stcs(d + v + u * GT, q[u]);
        }
        for (; v < nv; v += GT) __stcs(d + v, s[v]);
        for (uint64_t b = nv * 16 + gl; b < len; b += GT) dst[b] = src[b];
    } else if ((((uintptr_t)dst | (uintptr_t)src) & 3u) == 0) {
        const uint64_t nw = len >> 2;
        const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
        uint32_t *d = reinterpret_cast<uint32_t *>(dst);
        for (uint64_t w = gl; w < nw; w += GT) d[w] = s[w];
        for (uint64_t b = nw * 4 + gl; b < len; b += GT) dst[b] = src[b];
    } else {
        for (uint64_t b = gl; b < len; b += GT) dst[b] = src[b];
    }
}

// Last allocation whose first chunk is <= c (allocations are non-empty, so
// first_chunk is strictly increasing).
__device__ __forceinline__ uint32_t find_alloc(const CkptDesc *__restrict__ d, uint32_t n,
                                               uint64_t c) {
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (d[mid].first_chunk <= c) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ uint32_t find_scatter(const ScatterDesc *__restrict__ d, uint32_t n,
                                                 uint64_t c) {
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (d[mid].img_first <= c) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Decoupled look-back for tile `tile` (> 0), run by one full warp.  Returns
// the exclusive prefix of dirty chunks (*k0) and dirty bytes (*d0).  Each of
// the two quantities has its own status array and is resolved separately.
__device__ void lookback(const CkptParams &P, uint32_t tile, int lane, uint64_t *k0,
                         uint64_t *d0) {
    uint64_t kacc = 0, dacc = 0;
    bool kdone = false, ddone = false;
    int64_t j = (int64_t)tile - 1;
    const uint64_t t0 = globaltimer();
    bool gave_up = false;
    while (!(kdone && ddone)) {
        const int64_t t = j - lane;
        uint64_t wk = kFlagInc, wd = kFlagInc;   // tiles before 0: inclusive 0
        if (t >= 0) {
            uint32_t spins = 0;
            for (;;) {
                wk = ld_status(P.tile_cnt + t);
                wd = ld_status(P.tile_bytes + t);
                if ((wk >> 62) && (wd >> 62)) break;
                if (gave_up || ((++spins & 31u) == 0 &&
                                (globaltimer() - t0 > P.timeout_ns || spins > (1u << 28)))) {
                    gave_up = true;
                    atomicOr(&P.ctrl->err, kErrTimeout);
                    wk = kFlagInc;
                    wd = kFlagInc;
                    break;
                }
                __nanosleep(64);
            }
        }
        if (!kdone) {
            const unsigned inc = __ballot_sync(kFull, (wk >> 62) == 2);
            const int lim = inc ? __ffs(inc) - 1 : 31;
            kacc += warp_sum(lane <= lim ? (wk & kValMask) : 0);
            kdone = inc != 0;
        }
        if (!ddone) {
            const unsigned inc = __ballot_sync(kFull, (wd >> 62) == 2);
            const int lim = inc ? __ffs(inc) - 1 : 31;
            dacc += warp_sum(lane <= lim ? (wd & kValMask) : 0);
            ddone = inc != 0;
        }
        j -= 32;
    }
    *k0 = kacc;
    *d0 = dacc;
}

// Last allocation whose first chunk is <= c, over a first_chunk column
// cached in shared memory.
__device__ __forceinline__ uint32_t find_first_cached(const uint64_t *first, uint32_t n, uint64_t c) {
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (first[mid] <= c) lo = mid;
        else hi = mid;
    }
    return lo;
}

}  // namespace
}  // namespace crac
