// Device kernels of the checkpoint/restart data pass (sm_103a).
//
// The paper drains the device and copies the memory of every active
// allocation to the host at checkpoint, and copies it back at restart
// (Sec. 3.2, "Saving the library-allocated arena" and "restoring the CUDA
// library-allocated regions").  This file implements that copy as an
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
#include <cstdint>
#include <mutex>
#include <cuda_runtime.h>

#include "crac.h"
#include "crac_kernels.cuh"

namespace crac {

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

// ---------------------------------------------------------------------------
// Fused batched checkpoint pass: K1 + K2 + K3 in one persistent kernel.
// ---------------------------------------------------------------------------
template <int NT, int WPC>
__global__ void __launch_bounds__(NT) ckpt_fused_kernel(const CkptParams P) {
    constexpr int W = NT / 32;
    constexpr int G = W / WPC;        // chunk groups per CTA
    constexpr int GT = WPC * 32;      // threads per group
    __shared__ uint32_t s_alloc[kMaxCpt];
    __shared__ uint32_t s_len[kMaxCpt];    // dirty: chunk length; clean: 0
    __shared__ uint32_t s_pos[kMaxCpt];    // position among the tile's dirty chunks
    __shared__ uint64_t s_boff[kMaxCpt];   // byte offset among the tile's dirty bytes
    __shared__ uint64_t s_part[2][W];
    __shared__ uint64_t s_k0, s_d0;
    __shared__ uint32_t s_tile;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int g = warp / WPC;
    const int gl = threadIdx.x - g * GT;
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
        const uint64_t c0 = P.c_begin + (uint64_t)tile * P.cpt;
        const uint32_t nc = (uint32_t)min((uint64_t)P.cpt, P.c_end - c0);
        for (uint32_t t = threadIdx.x; t < nc; t += NT) s_alloc[t] = find_alloc(P.desc, P.n_allocs, c0 + t);
        __syncthreads();

        // K1 + K2 per chunk: fingerprint, then compare with the baseline.
        for (uint32_t r = 0; r * G < nc; ++r) {
            const uint32_t ci = r * G + g;
            uint64_t acc = 0;
            uint32_t len = 0;
            CkptDesc d{};
            uint64_t local = 0;
            if (ci < nc) {
                d = P.desc[s_alloc[ci]];
                local = c0 + ci - d.first_chunk;
                len = (uint32_t)min(S, d.bytes - (local << log2S));
                acc = hash_partial<GT>(reinterpret_cast<const uint8_t *>(d.ptr) + (local << log2S),
                                       len, gl);
            }
            acc = warp_sum(acc);
            if (WPC > 1) {
                if (lane == 0) s_part[r & 1][warp] = acc;
                __syncthreads();
                if (ci < nc && gl == 0) {
                    acc = 0;
#pragma unroll
                    for (int w = 0; w < WPC; ++w) acc += s_part[r & 1][g * WPC + w];
                }
            }
            if (ci < nc && gl == 0) {
                const uint64_t fp = fp_finalize(acc, len);
                P.fp_new[c0 + ci] = fp;
                const bool dirty = d.base_first == kNoBase || P.fp_old[d.base_first + local] != fp;
                s_len[ci] = dirty ? len : 0u;
            }
        }
        __syncthreads();

        // K2 compaction: positions within the tile (ballot + warp scan), then
        // the tile's global prefix by decoupled look-back.
        if (warp == 0) {
            uint32_t cnt = 0;
            uint64_t bytes = 0;
            for (uint32_t base = 0; base < nc; base += 32) {
                const uint32_t i = base + lane;
                const uint32_t l = i < nc ? s_len[i] : 0u;
                const unsigned m = __ballot_sync(kFull, l != 0);
                const uint64_t incl = warp_incl_scan(l, lane);
                if (i < nc) {
                    s_pos[i] = cnt + __popc(m & ((1u << lane) - 1u));
                    s_boff[i] = bytes + incl - l;
                }
                cnt += __popc(m);
                bytes += __shfl_sync(kFull, incl, 31);
            }
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
        const uint64_t k0 = s_k0, d0 = s_d0;
        for (uint32_t t = threadIdx.x; t < nc; t += NT) {
            if (s_len[t]) {
                const uint64_t j = k0 + s_pos[t];
                if (j < P.idx_cap) {
                    P.idx_out[j] = c0 + t;
                    P.off_out[j] = d0 + s_boff[t];
                } else {
                    atomicOr(&P.ctrl->err, kErrBounds);
                }
            }
        }
        // K3 gather of this tile's dirty chunks into the staging buffer.
        for (uint32_t ci = g; ci < nc; ci += G) {
            const uint32_t len = s_len[ci];
            if (!len) continue;
            const CkptDesc d = P.desc[s_alloc[ci]];
            const uint64_t local = c0 + ci - d.first_chunk;
            const uint64_t dst = d0 + s_boff[ci];
            if (dst + len > P.staging_cap) {
                if (gl == 0) atomicOr(&P.ctrl->err, kErrBounds);
                continue;
            }
            copy_group<GT>(P.staging + dst,
                           reinterpret_cast<const uint8_t *>(d.ptr) + (local << log2S), len, gl);
        }
        __syncthreads();
    }
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

// ---------------------------------------------------------------------------
// Per-allocation path (comparison baseline): K1, K2, K3 as separate launches.
// ---------------------------------------------------------------------------
constexpr int kRangeNT = 256;
constexpr int kRangeWPC = 8;

// K1 over chunks [c0, c1) of one allocation: fingerprints and dirty lengths.
__global__ void __launch_bounds__(kRangeNT)
fp_range_kernel(const CkptDesc *__restrict__ dp, uint64_t c0, uint64_t c1, uint32_t log2S,
                const uint64_t *__restrict__ fp_old, uint64_t *__restrict__ fp_new,
                uint32_t *__restrict__ lens, uint64_t lens_base) {
    constexpr int GT = kRangeWPC * 32;
    __shared__ uint64_t s_part[kRangeNT / 32];
    const CkptDesc d = *dp;
    const uint64_t S = 1ull << log2S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (uint64_t c = c0 + blockIdx.x; c < c1; c += gridDim.x) {
        const uint64_t local = c - d.first_chunk;
        const uint32_t len = (uint32_t)min(S, d.bytes - (local << log2S));
        uint64_t acc = hash_partial<GT>(reinterpret_cast<const uint8_t *>(d.ptr) + (local << log2S),
                                        len, threadIdx.x);
        acc = warp_sum(acc);
        if (lane == 0) s_part[warp] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            acc = 0;
            for (int w = 0; w < kRangeNT / 32; ++w) acc += s_part[w];
            const uint64_t fp = fp_finalize(acc, len);
            fp_new[c] = fp;
            const bool dirty = d.base_first == kNoBase || fp_old[d.base_first + local] != fp;
            lens[c - lens_base] = dirty ? len : 0u;
        }
        __syncthreads();
    }
}

// K2 over chunks [c0, c1): one CTA scans the dirty lengths and appends the
// dirty chunks to the running list held in `carry`.
__global__ void __launch_bounds__(1024)
compact_range_kernel(const uint32_t *__restrict__ lens, uint64_t lens_base, uint64_t c0,
                     uint64_t c1, uint64_t *__restrict__ idx_out, uint64_t *__restrict__ off_out,
                     uint64_t idx_cap, PerAllocCarry *carry, CkptCtrl *ctrl) {
    __shared__ uint32_t s_wcnt[32];
    __shared__ uint64_t s_wbytes[32];
    __shared__ uint64_t s_k, s_d;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        s_k = carry->k;
        s_d = carry->D;
        carry->unit_k0 = carry->k;
    }
    __syncthreads();
    const uint64_t k_start = s_k;
    for (uint64_t base = c0; base < c1; base += 1024) {
        const uint64_t c = base + threadIdx.x;
        const uint32_t l = c < c1 ? lens[c - lens_base] : 0u;
        const unsigned m = __ballot_sync(kFull, l != 0);
        const uint64_t incl = warp_incl_scan(l, lane);
        if (lane == 31) {
            s_wcnt[warp] = __popc(m);
            s_wbytes[warp] = incl;
        }
        __syncthreads();
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
            s_wcnt[lane] = ic - wc;      // exclusive
            s_wbytes[lane] = ib - wb;
        }
        __syncthreads();
        const uint64_t k = s_k + s_wcnt[warp] + __popc(m & ((1u << lane) - 1u));
        const uint64_t o = s_d + s_wbytes[warp] + incl - l;
        if (l) {
            if (k < idx_cap) {
                idx_out[k] = c;
                off_out[k] = o;
            } else {
                atomicOr(&ctrl->err, kErrBounds);
            }
        }
        __syncthreads();
        if (threadIdx.x == 1023) {
            s_k = k + (l ? 1 : 0);
            s_d = o + l;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        carry->unit_k = s_k - k_start;
        carry->k = s_k;
        carry->D = s_d;
        ctrl->k = s_k;
        ctrl->D = s_d;
        if (s_k <= idx_cap) off_out[s_k] = s_d;
        else atomicOr(&ctrl->err, kErrBounds);
    }
}

// K3: copy the dirty chunks listed by the last K2 of this allocation.
__global__ void __launch_bounds__(kRangeNT)
gather_range_kernel(const CkptDesc *__restrict__ dp, uint32_t log2S,
                    const uint64_t *__restrict__ idx, const uint64_t *__restrict__ off,
                    const PerAllocCarry *__restrict__ carry, uint64_t idx_cap,
                    uint8_t *__restrict__ staging, uint64_t staging_cap, CkptCtrl *ctrl) {
    constexpr int GT = kRangeWPC * 32;
    const CkptDesc d = *dp;
    const uint64_t k0 = carry->unit_k0;
    const uint64_t room = idx_cap > k0 ? idx_cap - k0 : 0ull;
    const uint64_t kn = (uint64_t)carry->unit_k < room ? (uint64_t)carry->unit_k : room;
    const uint64_t S = 1ull << log2S;
    for (uint64_t j = k0 + blockIdx.x; j < k0 + kn; j += gridDim.x) {
        const uint64_t local = idx[j] - d.first_chunk;
        const uint64_t len = min(S, d.bytes - (local << log2S));
        const uint64_t o = off[j];
        if (o + len > staging_cap) {
            if (threadIdx.x == 0) atomicOr(&ctrl->err, kErrBounds);
            continue;
        }
        copy_group<GT>(staging + o, reinterpret_cast<const uint8_t *>(d.ptr) + (local << log2S),
                       len, threadIdx.x);
    }
}

// ---------------------------------------------------------------------------
// K4 restore scatter: payload chunks -> allocations, filtered by the owner map
// so that each target chunk is written once, by the newest image holding it.
// ---------------------------------------------------------------------------
constexpr int kScatterNT = 256;

__global__ void __launch_bounds__(kScatterNT) scatter_kernel(const ScatterParams P) {
    constexpr int GT = 32;
    // A resolution or bounds error found earlier on this stream (chain not
    // covering the target, index out of range) leaves memory untouched.
    if (*(volatile unsigned int *)P.err) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t S = 1ull << P.log2_chunk;
    const uint64_t n = P.j1 - P.j0;
    for (uint64_t e = (uint64_t)blockIdx.x * (kScatterNT / 32) + warp; e < n;
         e += (uint64_t)gridDim.x * (kScatterNT / 32)) {
        const uint64_t c = P.full ? P.j0 + e : P.idx[e];
        const ScatterDesc d = P.desc[find_scatter(P.desc, P.n_desc, c)];
        const uint64_t local = c - d.img_first;
        if (d.dst == 0) continue;
        const uint64_t tc = d.tgt_first + local;
        if (tc >= P.n_owner) {
            if (lane == 0) atomicOr(P.err, kErrBounds);
            continue;
        }
        if (P.owner[tc] != P.image_index) continue;
        const uint64_t len = min(S, d.bytes - (local << P.log2_chunk));
        const uint64_t o = P.full ? d.payload_base + (local << P.log2_chunk) : P.off[e];
        if (o < P.origin || o - P.origin + len > P.window) {
            if (lane == 0) atomicOr(P.err, kErrBounds);
            continue;
        }
        copy_group<GT>(reinterpret_cast<uint8_t *>(d.dst) + (local << P.log2_chunk),
                       P.payload + (o - P.origin), len, lane);
    }
}

// ---------------------------------------------------------------------------
// TMA-staged fused pass (chunk sizes 1-64 KiB).
//
// One CTA per SM, warp-specialized, with a ring of three 64 KiB shared-memory
// slots.  A tile is one slot: 64 KiB / S consecutive global chunks.
//   producer warp  takes tile tickets, maps chunks to allocations, loads the
//                  baseline fingerprints, and fills a free slot with one
//                  cp.async.bulk per chunk (the last <16 bytes of a ragged
//                  chunk by plain loads), completing on the slot's `full`
//                  mbarrier;
//   8 hasher warps CRAC-FP64 from shared memory, dirty test -> `hashed`;
//   scan warp      tile compaction (ballot + warp scan) and decoupled
//                  look-back -> the tile's global offsets -> `scanned`;
//   store warp     idx/off and the gather: dirty chunks leave shared memory
//                  by cp.async.bulk stores (plain stores when misaligned),
//                  then the slot is released -> `empty`.
// Every byte is read from HBM once and every dirty byte written once.  Each
// mbarrier wait is bounded; a wait that runs out sets kErrTimeout and the
// role stops; the kernel still waits (bounded) for the bulk copies it issued.
// ---------------------------------------------------------------------------
namespace tma {
constexpr uint32_t kSlot = 65536;
constexpr int kNSlot = 3;
constexpr int kHW = 8;                       // hasher warps
constexpr int kThreads = (kHW + 3) * 32;     // + producer, scan, store
constexpr int kMaxT = 64;                    // chunks per tile (S >= 1 KiB)
constexpr uint32_t kDone = 0xffffffffu;

struct __align__(16) Meta {
    uint64_t c0;
    uint64_t has_base;        // bit i: chunk i has a baseline fingerprint
    uint32_t tile, nc;
    uint64_t k0, d0;          // the tile's exclusive prefix (scan warp)
    uint32_t len[kMaxT];
    uint64_t fpo[kMaxT];      // index of the baseline fingerprint in fp_old (if has_base)
    uint32_t dlen[kMaxT];     // dirty ? len : 0 (hashers)
    uint32_t cnt;             // the tile's dirty chunks / bytes (hasher warp 0)
    uint64_t bytes;
    uint32_t pos[kMaxT];      // position among the tile's dirty chunks
    uint64_t boff[kMaxT];     // byte offset among the tile's dirty bytes
    uint64_t part[2][kHW];    // cross-warp partial sums
};
constexpr size_t kBarOff = (size_t)kNSlot * kSlot + (size_t)kNSlot * sizeof(Meta);
constexpr size_t kSmemBytes = kBarOff + 4 * kNSlot * sizeof(uint64_t) + kNSlot * sizeof(uint32_t);
// The allocations' first_chunk column, when it fits in what the slots leave
// of the 227 KiB a CTA may have, so that the producer's chunk -> allocation
// search stays on chip.
constexpr size_t kFirstOff = (kSmemBytes + 15) & ~(size_t)15;
constexpr uint32_t kCachedAllocs = 3072;
constexpr size_t kSmemMax = kFirstOff + (size_t)kCachedAllocs * sizeof(uint64_t);
static_assert(kSmemMax <= 227 * 1024, "TMA pass shared memory");
}  // namespace tma

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t tx) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(tx)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase of `parity` to complete; false (and kErrTimeout)
// if it does not within timeout_ns.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, const CkptParams &P) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63u) == 0 && (globaltimer() - t0 > P.timeout_ns || i > (1u << 28))) {
            atomicOr(&P.ctrl->err, kErrTimeout);
            return false;
        }
    }
}
__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src_smem, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                 "r"(smem_u32(src_smem)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void hashers_sync() {
    asm volatile("bar.sync 1, %0;" ::"n"(tma::kHW * 32) : "memory");
}

// Partial CRAC-FP64 sum of one chunk held in shared memory; the vector after
// the last whole one is zero-padded there, so it can be read whole.
template <int GT>
__device__ __forceinline__ uint64_t hash_smem(const uint8_t *chunk, uint32_t len, int gl) {
    const uint4 *p = reinterpret_cast<const uint4 *>(chunk);
    const uint32_t nv = len >> 4;
    uint64_t acc = 0;
    uint64_t key = (2ull * (uint64_t)gl + 1ull) * kK1;
    constexpr uint64_t kStep = 2ull * GT * kK1;
    uint32_t v = gl;
#pragma unroll 4
    for (; v < nv; v += GT) {
        const uint4 q = p[v];
        acc += mixw(((uint64_t)q.y << 32) | q.x, key);
        acc += mixw(((uint64_t)q.w << 32) | q.z, key + kK1);
        key += kStep;
    }
    const uint32_t rem = len & 15u;
    if (rem && v == nv) {
        const uint4 q = p[nv];
        acc += mixw(((uint64_t)q.y << 32) | q.x, key);
        if (rem > 8) acc += mixw(((uint64_t)q.w << 32) | q.z, key + kK1);
    }
    return acc;
}

__device__ __forceinline__ void tma_producer(const CkptParams &P, uint8_t *slots, tma::Meta *meta, uint64_t *full,
                                             uint64_t *scanned, uint64_t *empty, uint32_t *armed,
                                             const uint64_t *s_first, int lane) {
    using namespace tma;
    const uint32_t log2S = P.log2_chunk;
    const uint64_t S = 1ull << log2S;
    // The next tile's ticket is taken once the slot's previous tile has its
    // staging offset (its store is being issued), so a tile is held without
    // loading only for the length of one store, and the ticket round trip
    // and the chunk lookups overlap that store.  The slot and its Meta are
    // written only after the store has read them (`empty`).
    for (uint32_t it = 0;; ++it) {
        const uint32_t s = it % kNSlot, par = (it / kNSlot) & 1u;
        if (!mbar_wait(&scanned[s], par ^ 1u, P)) return;
        uint32_t t = 0;
        if (lane == 0) {
            t = atomicAdd(&P.ctrl->ticket, 1u);
            if (P.skip_first_ticket && t == 0) t = atomicAdd(&P.ctrl->ticket, 1u);
        }
        const uint32_t tile = __shfl_sync(kFull, t, 0);
        Meta &m = meta[s];
        if (tile >= P.n_tiles) {
            if (!mbar_wait(&empty[s], par ^ 1u, P)) return;
            if (lane == 0) {
                m.tile = kDone;
                armed[s] = 2u | par;   // the last phase of this slot is the done marker
                mbar_arrive(&full[s]);
            }
            return;
        }
        uint8_t *base = slots + (size_t)s * kSlot;
        const uint64_t c0 = P.c_begin + (uint64_t)tile * P.cpt;
        const uint32_t nc = (uint32_t)min((uint64_t)P.cpt, P.c_end - c0);
        const uint8_t *src[2] = {nullptr, nullptr};
        uint32_t len[2] = {0, 0};
        uint64_t fpo[2] = {0, 0};
        uint32_t tx = 0;
        uint64_t hb = 0;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const uint32_t i = lane + 32 * k;
            bool has = false;
            if (i < nc) {
                const uint64_t c = c0 + i;
                const uint32_t a = P.first_cached ? find_first_cached(s_first, P.n_allocs, c)
                                                  : find_alloc(P.desc, P.n_allocs, c);
                const CkptDesc d = P.desc[a];
                const uint64_t local = c - d.first_chunk;
                len[k] = (uint32_t)min(S, d.bytes - (local << log2S));
                src[k] = reinterpret_cast<const uint8_t *>(d.ptr) + (local << log2S);
                has = d.base_first != kNoBase;
                fpo[k] = has ? d.base_first + local : 0ull;
                tx += len[k] & ~15u;
            }
            hb |= (uint64_t)__ballot_sync(kFull, has) << (32 * k);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) tx += __shfl_xor_sync(kFull, tx, o);
        if (!mbar_wait(&empty[s], par ^ 1u, P)) return;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const uint32_t i = lane + 32 * k;
            if (i < nc) {
                m.fpo[i] = fpo[k];
                m.len[i] = len[k];
            }
        }
        if (lane == 0) {
            m.tile = tile;
            m.nc = nc;
            m.c0 = c0;
            m.has_base = hb;
            armed[s] = 2u | par;
            mbar_expect_tx(&full[s], tx);
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const uint32_t i = lane + 32 * k;
            if (i >= nc) continue;
            const uint32_t l16 = len[k] & ~15u;
            uint8_t *dst = base + ((size_t)i << log2S);
            if (l16) bulk_g2s(dst, src[k], l16, &full[s]);
            if (len[k] & 15u) {   // ragged end of an allocation: plain loads, zero-padded vector
                uint64_t lo = 0, hi = 0;
                for (uint32_t b = 0; b < (len[k] & 15u); ++b) {
                    const uint64_t byte = src[k][l16 + b];
                    if (b < 8) lo |= byte << (8 * b);
                    else hi |= byte << (8 * (b - 8));
                }
                *reinterpret_cast<uint4 *>(dst + l16) =
                    make_uint4((uint32_t)lo, (uint32_t)(lo >> 32), (uint32_t)hi, (uint32_t)(hi >> 32));
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&full[s]);
    }
}

// Hasher warp 0 does the bounded wait on `full` and broadcasts the outcome
// (0 timed out, 1 tile, 2 done) so that all hasher warps leave together and
// none is left waiting at the hashers' named barrier.
template <int WPC>
__device__ __forceinline__ void tma_hasher(const CkptParams &P, const uint8_t *slots, tma::Meta *meta,
                                           uint64_t *full, uint64_t *hashed, volatile uint32_t *go,
                                           int warp, int lane) {
    using namespace tma;
    constexpr int G = kHW / WPC;
    constexpr int GT = WPC * 32;
    const int g = warp / WPC;
    const int gl = (warp % WPC) * 32 + lane;
    const uint32_t log2S = P.log2_chunk;
    for (uint32_t it = 0;; ++it) {
        const uint32_t s = it % kNSlot, par = (it / kNSlot) & 1u;
        Meta &m = meta[s];
        if (warp == 0) {
            const bool ok = mbar_wait(&full[s], par, P);
            if (lane == 0) go[it & 1] = !ok ? 0u : (m.tile == kDone ? 2u : 1u);
        }
        hashers_sync();
        const uint32_t state = go[it & 1];
        if (state == 0) return;
        mbar_try_wait(&full[s], par);   // completed: acquire for this warp too
        if (state == 2) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&hashed[s]);
            return;
        }
        const uint32_t nc = m.nc;
        const uint8_t *base = slots + (size_t)s * kSlot;
        for (uint32_t r = 0; r * G < nc; ++r) {
            const uint32_t ci = r * G + g;
            uint64_t acc = 0, fo = 0;
            uint32_t len = 0;
            bool has = false;
            if (ci < nc) {
                len = m.len[ci];
                has = (m.has_base >> ci) & 1ull;
                if (gl == 0 && has) fo = P.fp_old[m.fpo[ci]];   // overlaps the hash below
                acc = hash_smem<GT>(base + ((size_t)ci << log2S), len, gl);
            }
            acc = warp_sum(acc);
            if (WPC > 1) {
                if (lane == 0) m.part[r & 1][warp] = acc;
                hashers_sync();
                if (ci < nc && gl == 0) {
                    acc = 0;
#pragma unroll
                    for (int w = 0; w < WPC; ++w) acc += m.part[r & 1][g * WPC + w];
                }
            }
            if (ci < nc && gl == 0) {
                const uint64_t fp = fp_finalize(acc, len);
                P.fp_new[m.c0 + ci] = fp;
                m.dlen[ci] = (!has || fo != fp) ? len : 0u;
            }
        }
        // The tile's aggregate is published as soon as it is known.
        hashers_sync();
        if (warp == 0) {
            uint32_t cnt = 0;
            uint64_t bytes = 0;
            for (uint32_t b0 = 0; b0 < nc; b0 += 32) {
                const uint32_t i = b0 + lane;
                const uint32_t l = i < nc ? m.dlen[i] : 0u;
                const unsigned msk = __ballot_sync(kFull, l != 0);
                const uint64_t incl = warp_incl_scan(l, lane);
                if (i < nc) {
                    m.pos[i] = cnt + __popc(msk & ((1u << lane) - 1u));
                    m.boff[i] = bytes + incl - l;
                }
                cnt += __popc(msk);
                bytes += __shfl_sync(kFull, incl, 31);
            }
            if (lane == 0) {
                m.cnt = cnt;
                m.bytes = bytes;
                const uint64_t f = m.tile == 0 ? kFlagInc : kFlagAgg;
                st_status(P.tile_cnt + m.tile, f | cnt);
                st_status(P.tile_bytes + m.tile, f | bytes);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&hashed[s]);
    }
}

__device__ __forceinline__ void tma_scan(const CkptParams &P, tma::Meta *meta, uint64_t *hashed, uint64_t *scanned,
                                         int lane) {
    using namespace tma;
    for (uint32_t it = 0;; ++it) {
        const uint32_t s = it % kNSlot, par = (it / kNSlot) & 1u;
        if (!mbar_wait(&hashed[s], par, P)) return;
        Meta &m = meta[s];
        const uint32_t tile = m.tile;
        if (tile == kDone) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&scanned[s]);
            return;
        }
        const uint32_t cnt = m.cnt;
        const uint64_t bytes = m.bytes;
        uint64_t k0 = 0, d0 = 0;
        if (tile != 0) {   // tile 0 was published inclusive by the hashers
            lookback(P, tile, lane, &k0, &d0);
            if (lane == 0) {
                st_status(P.tile_cnt + tile, kFlagInc | ((k0 + cnt) & kValMask));
                st_status(P.tile_bytes + tile, kFlagInc | ((d0 + bytes) & kValMask));
            }
        }
        if (lane == 0) {
            m.k0 = k0;
            m.d0 = d0;
            if (tile == P.n_tiles - 1) {
                P.ctrl->k = k0 + cnt;
                P.ctrl->D = d0 + bytes;
                if (k0 + cnt <= P.idx_cap) P.off_out[k0 + cnt] = d0 + bytes;
                else atomicOr(&P.ctrl->err, kErrBounds);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&scanned[s]);
    }
}

__device__ __forceinline__ void tma_store(const CkptParams &P, const uint8_t *slots, tma::Meta *meta,
                                          uint64_t *scanned, uint64_t *empty, int lane) {
    using namespace tma;
    const uint32_t log2S = P.log2_chunk;
    for (uint32_t it = 0;; ++it) {
        const uint32_t s = it % kNSlot, par = (it / kNSlot) & 1u;
        if (!mbar_wait(&scanned[s], par, P)) break;
        Meta &m = meta[s];
        if (m.tile == kDone) break;
        const uint32_t nc = m.nc;
        const uint64_t k0 = m.k0, d0 = m.d0, c0 = m.c0;
        const uint8_t *base = slots + (size_t)s * kSlot;
        fence_proxy_async_smem();
        for (uint32_t i = lane; i < nc; i += 32) {
            const uint32_t len = m.dlen[i];
            if (!len) continue;
            const uint64_t j = k0 + m.pos[i];
            if (j < P.idx_cap) {
                P.idx_out[j] = c0 + i;
                P.off_out[j] = d0 + m.boff[i];
            } else {
                atomicOr(&P.ctrl->err, kErrBounds);
            }
            const uint64_t o = d0 + m.boff[i];
            if (o + len > P.staging_cap) {
                atomicOr(&P.ctrl->err, kErrBounds);
                continue;
            }
            uint8_t *dst = P.staging + o;
            if ((((uintptr_t)dst) & 15u) == 0 && (len & 15u) == 0)
                bulk_s2g(dst, base + ((size_t)i << log2S), len);
        }
        bulk_commit();
        // Chunks a bulk store cannot take (ragged length or unaligned offset).
        for (uint32_t i = 0; i < nc; ++i) {
            const uint32_t len = m.dlen[i];
            if (!len) continue;
            const uint64_t o = d0 + m.boff[i];
            uint8_t *dst = P.staging + o;
            if (o + len > P.staging_cap) continue;
            if ((((uintptr_t)dst) & 15u) == 0 && (len & 15u) == 0) continue;
            const uint8_t *src = base + ((size_t)i << log2S);
            for (uint32_t b = lane; b < len; b += 32) dst[b] = src[b];
        }
        bulk_wait_read0();
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
    }
    bulk_wait0();
}

template <int WPC>
__global__ void __launch_bounds__(tma::kThreads, 1) ckpt_tma_kernel(const CkptParams P) {
    using namespace tma;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *slots = smem;
    Meta *meta = reinterpret_cast<Meta *>(smem + (size_t)kNSlot * kSlot);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kBarOff);
    uint64_t *full = bars, *hashed = bars + kNSlot, *scanned = bars + 2 * kNSlot, *empty = bars + 3 * kNSlot;
    uint32_t *armed = reinterpret_cast<uint32_t *>(bars + 4 * kNSlot);
    uint64_t *s_first = reinterpret_cast<uint64_t *>(smem + kFirstOff);
    __shared__ uint32_t go[2];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (P.first_cached)
        for (uint32_t a = threadIdx.x; a < P.n_allocs; a += kThreads) s_first[a] = P.desc[a].first_chunk;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kNSlot; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&hashed[s], kHW);
            mbar_init(&scanned[s], 1);
            mbar_init(&empty[s], 1);
            armed[s] = 0;
        }
        fence_mbar_init();
    }
    __syncthreads();
    if (warp < kHW) tma_hasher<WPC>(P, slots, meta, full, hashed, go, warp, lane);
    else if (warp == kHW) tma_producer(P, slots, meta, full, scanned, empty, armed, s_first, lane);
    else if (warp == kHW + 1) tma_scan(P, meta, hashed, scanned, lane);
    else tma_store(P, slots, meta, scanned, empty, lane);
    __syncthreads();
    // Bulk loads still in flight (only after a role stopped on a timeout):
    // wait for the last phase armed on each slot before the CTA exits.
    if (threadIdx.x == 0) {
        for (int s = 0; s < kNSlot; ++s)
            if (armed[s] & 2u) mbar_wait(&full[s], armed[s] & 1u, P);
    }
}

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

// Partial CRAC-FP64 sum of a segment (<= 8 KiB) whose first word is word j0
// of its chunk, over the lanes of one warp.
__device__ __forceinline__ uint64_t hash_seg(const uint8_t *__restrict__ src, uint32_t len, uint64_t j0,
                                             int lane, uint4 *__restrict__ copy_to = nullptr) {
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
    const uint32_t rem = len & 15u;
    if (rem && lane == (int)(nv & 31u)) {
        const uint8_t *t = src + 16ull * nv;
        uint64_t w0 = 0, w1 = 0;
        for (uint32_t b = 0; b < rem; ++b) {
            const uint64_t byte = t[b];
            if (b < 8) w0 |= byte << (8 * b);
            else w1 |= byte << (8 * (b - 8));
        }
        const uint64_t kt = (j0 + 2ull * nv + 1ull) * kK1;
        acc += mixw(w0, kt);
        if (rem > 8) acc += mixw(w1, kt + kK1);
    }
    return acc;
}

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
        }
        uint64_t sum = hash_seg(src, len, off >> 3, lane, copy_to);
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
                                                uint64_t a_next, int li) {
    const uint32_t log2S = P.log2_chunk;
    uint64_t sum = 0, fo = 0;
    uint32_t len = 0;
    bool has = false;
    CkptDesc d = d_warp;
    uint32_t a = a_warp;
    if (c < P.c_end) {
        if (c >= a_next) {   // the segment crosses an allocation end
            a = find_alloc(P.desc, P.n_allocs, c);
            d = P.desc[a];
        }
        const uint64_t local = c - d.first_chunk;
        const uint64_t rest = d.bytes - (local << log2S);
        len = (uint32_t)umin64(rest, 1ull << log2S);
        has = d.base_first != kNoBase;
        if (li == 0 && has) fo = __ldg(P.fp_old + d.base_first + local);
        const uint4 *p = reinterpret_cast<const uint4 *>(reinterpret_cast<const uint8_t *>(d.ptr) + (local << log2S));
        const uint32_t nv = len >> 4;
        uint4 q[16];
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
        if (P.full_copy) {   // FULL checkpoint: the chunk goes straight to its staging offset
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
#pragma unroll
    for (int o = LPC / 2; o; o >>= 1) sum += __shfl_xor_sync(kFull, sum, o);
    if (li == 0 && c < P.c_end) {
        const uint64_t fp = fp_finalize(sum, len);
        P.fp_new[c] = fp;
        acc[c - P.c_begin] = len | ((!has || fo != fp) ? kAccDirty : 0ull);
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
    for (; q < q_end; ++q) {
        const uint64_t c0 = P.c_begin + q * CPS;
        if (!have || c0 >= a_next) {
            a = find_alloc(P.desc, P.n_allocs, c0);
            d = P.desc[a];
            a_next = a + 1 < P.n_allocs ? P.desc[a + 1].first_chunk : ~0ull;
            have = true;
        }
        hash_small_iter<LPC>(P, acc, c0 + lane / LPC, d, a, a_next, lane % LPC);
    }
}

__global__ void __launch_bounds__(kFinNT)
split_finalize_kernel(const CkptParams P, unsigned long long *__restrict__ acc, uint32_t log2Seg) {
    const bool direct = log2Seg == P.log2_chunk;
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
        if (c < P.c_end && direct) {
            const uint64_t v = acc[c - P.c_begin];
            len = (uint32_t)v;
            dl = (v & kAccDirty) ? len : 0u;
        } else if (c < P.c_end) {
            const CkptDesc d = P.desc[find_alloc(P.desc, P.n_allocs, c)];
            const uint64_t local = c - d.first_chunk;
            len = (uint32_t)min(S, d.bytes - (local << log2S));
            const uint64_t fp = fp_finalize(acc[c - P.c_begin], len);
            P.fp_new[c] = fp;
            const bool dirty = d.base_first == kNoBase || P.fp_old[d.base_first + local] != fp;
            dl = dirty ? len : 0u;
        }
        // Bytes that advance the staging offset: the dirty ones, or in the
        // sparse pass every chunk's (each sits at its uncompacted offset).
        const uint32_t sv = P.sparse ? len : dl;
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
                P.off_out[j] = s_d0 + s_wbytes[warp] + incl - sv;
            } else {
                atomicOr(&P.ctrl->err, kErrBounds);
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kGatherNT)
split_gather_kernel(const CkptParams P, unsigned long long *, uint32_t) {
    if (P.full_copy) return;   // the hash kernel has already written every chunk
    const int lane = threadIdx.x & 31;
    const uint64_t kd = (uint64_t)P.ctrl->k;
    const uint64_t k = kd < P.idx_cap ? kd : P.idx_cap;
    const uint32_t log2S = P.log2_chunk;
    const uint64_t S = 1ull << log2S;
    const uint64_t nw = ((uint64_t)gridDim.x * kGatherNT) >> 5;
    for (uint64_t j = ((uint64_t)blockIdx.x * kGatherNT + threadIdx.x) >> 5; j < k; j += nw) {
        const uint64_t c = P.idx_out[j];
        const uint64_t o = P.off_out[j];
        const CkptDesc d = P.desc[find_alloc(P.desc, P.n_allocs, c)];
        const uint64_t local = c - d.first_chunk;
        const uint64_t len = min(S, d.bytes - (local << log2S));
        if (o + len > P.staging_cap) {
            if (lane == 0) atomicOr(&P.ctrl->err, kErrBounds);
            continue;
        }
        copy_group<32>(P.staging + o, reinterpret_cast<const uint8_t *>(d.ptr) + (local << log2S), len, lane);
    }
}

// ---------------------------------------------------------------------------
// Chain resolution and restore on the device (R3 + R2 for device-resident
// chains), over every piece of every image of the chain in one launch each.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t find_piece(const RestorePiece *__restrict__ p, uint32_t n, uint64_t e) {
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (p[mid].entry_base <= e) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Target chunk of entry e, or ~0 when its allocation is not restored.
__device__ __forceinline__ uint64_t restore_target(const RestoreParams &P, const RestorePiece &pc, uint64_t e,
                                                   uint64_t *c_out, ScatterDesc *d_out) {
    const uint64_t c = reinterpret_cast<const uint64_t *>(pc.idx)[e - pc.entry_base];
    const ScatterDesc *dd = P.desc + pc.desc_off;
    const ScatterDesc d = dd[find_scatter(dd, pc.n_desc, c)];
    *c_out = c;
    *d_out = d;
    if (d.dst == 0) return ~0ull;
    return d.tgt_first + (c - d.img_first);
}

__global__ void __launch_bounds__(256) restore_mark_kernel(const RestoreParams P) {
    for (uint64_t e = (uint64_t)blockIdx.x * 256 + threadIdx.x; e < P.n_entries; e += (uint64_t)gridDim.x * 256) {
        const RestorePiece pc = P.pieces[find_piece(P.pieces, P.n_pieces, e)];
        uint64_t c;
        ScatterDesc d;
        const uint64_t tc = restore_target(P, pc, e, &c, &d);
        if (tc == ~0ull) continue;
        if (tc < P.n_owner) atomicMax(P.owner + tc, pc.image_index + 1u);
        else atomicOr(P.err, kErrBounds);
    }
}

__global__ void __launch_bounds__(256) restore_check_kernel(const RestoreParams P) {
    for (uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x; i < P.n_owner; i += (uint64_t)gridDim.x * 256)
        if (P.owner[i] == 0) atomicOr(P.err, kErrUncovered);
}

__global__ void __launch_bounds__(kScatterNT) restore_scatter_kernel(const RestoreParams P) {
    if (*(volatile unsigned int *)P.err) return;   // uncovered or out of range: memory untouched
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint64_t S = 1ull << P.log2_chunk;
    for (uint64_t e = (uint64_t)blockIdx.x * (kScatterNT / 32) + warp; e < P.n_entries;
         e += (uint64_t)gridDim.x * (kScatterNT / 32)) {
        const RestorePiece pc = P.pieces[find_piece(P.pieces, P.n_pieces, e)];
        uint64_t c;
        ScatterDesc d;
        const uint64_t tc = restore_target(P, pc, e, &c, &d);
        if (tc >= P.n_owner || P.owner[tc] != pc.image_index + 1u) continue;
        const uint64_t local = c - d.img_first;
        const uint64_t len = min(S, d.bytes - (local << P.log2_chunk));
        const uint64_t o = reinterpret_cast<const uint64_t *>(pc.off)[e - pc.entry_base];
        if (o + len > pc.bytes) {
            if (lane == 0) atomicOr(P.err, kErrBounds);
            continue;
        }
        copy_group<32>(reinterpret_cast<uint8_t *>(d.dst) + (local << P.log2_chunk),
                       reinterpret_cast<const uint8_t *>(pc.payload) + o, len, lane);
    }
}

template <int NT, int WPC>
cudaError_t launch_fused_t(const CkptParams &p, int grid, cudaStream_t s) {
    ckpt_fused_kernel<NT, WPC><<<grid, NT, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------

static uint64_t g_launches = 0;   // guarded by the callers' context lock is not enough
                                  // across contexts; use an atomic builtin
void count_launches(uint64_t n) { __atomic_fetch_add(&g_launches, n, __ATOMIC_RELAXED); }
uint64_t launches_so_far() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

const void *ckpt_tma_fn(int wpc) {
    switch (wpc) {
    case 1: return reinterpret_cast<const void *>(&ckpt_tma_kernel<1>);
    case 2: return reinterpret_cast<const void *>(&ckpt_tma_kernel<2>);
    case 4: return reinterpret_cast<const void *>(&ckpt_tma_kernel<4>);
    case 8: return reinterpret_cast<const void *>(&ckpt_tma_kernel<8>);
    default: return nullptr;
    }
}

int ckpt_tma_threads() { return tma::kThreads; }
size_t ckpt_tma_smem(uint32_t n_allocs) {
    return n_allocs <= tma::kCachedAllocs ? tma::kFirstOff + (size_t)n_allocs * sizeof(uint64_t) : tma::kSmemBytes;
}
uint32_t ckpt_tma_cached_allocs() { return tma::kCachedAllocs; }
uint32_t ckpt_tma_slot_bytes() { return tma::kSlot; }

cudaError_t ckpt_tma_prepare() {
    for (int w : {1, 2, 4, 8}) {
        const cudaError_t e = cudaFuncSetAttribute(ckpt_tma_fn(w), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)tma::kSmemMax);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

const void *split_hash_fn() { return reinterpret_cast<const void *>(&split_hash_kernel); }
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
const void *split_gather_fn() { return reinterpret_cast<const void *>(&split_gather_kernel); }
int split_hash_threads() { return kHashNT; }
int split_finalize_threads() { return kFinNT; }
int split_gather_threads() { return kGatherNT; }
int split_max_ctas_per_sm(const void *fn, int threads) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, 0) != cudaSuccess) return 1;
    return n > 0 ? n : 1;
}

const void *ckpt_fused_fn(int threads, int wpc) {
    if (threads != 256) return nullptr;
    if (wpc == 1) return reinterpret_cast<const void *>(&ckpt_fused_kernel<256, 1>);
    if (wpc == 8) return reinterpret_cast<const void *>(&ckpt_fused_kernel<256, 8>);
    return nullptr;
}

int ckpt_fused_max_ctas_per_sm(int threads, int wpc) {
    const void *fn = ckpt_fused_fn(threads, wpc);
    if (!fn) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, 0) != cudaSuccess) return 0;
    return n;
}

cudaError_t launch_ckpt_fused(const CkptParams &p, int threads, int wpc, int grid,
                              cudaStream_t s) {
    if (p.cpt == 0 || p.cpt > (uint32_t)kMaxCpt || grid <= 0) return cudaErrorInvalidValue;
    cudaError_t e = cudaErrorInvalidValue;
    if (threads == 256 && wpc == 1) e = launch_fused_t<256, 1>(p, grid, s);
    else if (threads == 256 && wpc == 8) e = launch_fused_t<256, 8>(p, grid, s);
    if (e == cudaSuccess) count_launches(1);
    return e;
}

cudaError_t launch_fp_range(const CkptDesc *d, uint64_t c0, uint64_t c1, uint32_t log2S,
                            const uint64_t *fp_old, uint64_t *fp_new, uint32_t *lens,
                            uint64_t lens_base, int grid, cudaStream_t s) {
    if (c1 <= c0) return cudaSuccess;
    fp_range_kernel<<<grid, kRangeNT, 0, s>>>(d, c0, c1, log2S, fp_old, fp_new, lens, lens_base);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) count_launches(1);
    return e;
}

cudaError_t launch_compact_range(const uint32_t *lens, uint64_t lens_base, uint64_t c0, uint64_t c1,
                                 uint64_t *idx_out, uint64_t *off_out, uint64_t idx_cap,
                                 PerAllocCarry *carry, CkptCtrl *ctrl, cudaStream_t s) {
    compact_range_kernel<<<1, 1024, 0, s>>>(lens, lens_base, c0, c1, idx_out, off_out, idx_cap,
                                            carry, ctrl);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) count_launches(1);
    return e;
}

cudaError_t launch_gather_range(const CkptDesc *d, uint32_t log2S, const uint64_t *idx,
                                const uint64_t *off, PerAllocCarry *carry, uint64_t max_entries,
                                uint64_t idx_cap, uint8_t *staging, uint64_t staging_cap,
                                CkptCtrl *ctrl, int grid, cudaStream_t s) {
    if (max_entries == 0) return cudaSuccess;
    gather_range_kernel<<<grid, kRangeNT, 0, s>>>(d, log2S, idx, off, carry, idx_cap, staging,
                                                  staging_cap, ctrl);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) count_launches(1);
    return e;
}

cudaError_t launch_restore_mark(const RestoreParams &p, int grid, cudaStream_t s) {
    if (p.n_entries == 0) return cudaSuccess;
    restore_mark_kernel<<<grid, 256, 0, s>>>(p);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) count_launches(1);
    return e;
}

cudaError_t launch_restore_check(const RestoreParams &p, int grid, cudaStream_t s) {
    if (p.n_owner == 0) return cudaSuccess;
    restore_check_kernel<<<grid, 256, 0, s>>>(p);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) count_launches(1);
    return e;
}

cudaError_t launch_restore_scatter(const RestoreParams &p, int grid, cudaStream_t s) {
    if (p.n_entries == 0) return cudaSuccess;
    restore_scatter_kernel<<<grid, kScatterNT, 0, s>>>(p);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) count_launches(1);
    return e;
}

cudaError_t launch_scatter(const ScatterParams &p, int grid, cudaStream_t s) {
    if (p.j1 <= p.j0) return cudaSuccess;
    scatter_kernel<<<grid, kScatterNT, 0, s>>>(p);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) count_launches(1);
    return e;
}

}  // namespace crac

// ---------------------------------------------------------------------------
// Allocation-free checkpoint pass (crac_pass_noalloc).
//
// For callers that must not allocate (an interposed cudaMalloc/cudaFree
// wrapper, an allocator hook, a preemption-time checkpoint, a process out of
// memory): the same fused kernel, with its scratch -- the control block and
// the look-back status words -- in a fixed array of this library's device
// memory instead of a buffer obtained from cudaMalloc.
// ---------------------------------------------------------------------------

namespace {

constexpr size_t kNoAllocScratchBytes =
    sizeof(crac::CkptCtrl) + 2 * sizeof(uint64_t) * (size_t)CRAC_NOALLOC_MAX_TILES;   // 512 KiB + 64 B

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_addr[kNoAllocMaxDevices];     // device address of the scratch, per device
int g_noalloc_grid[kNoAllocMaxDevices][2];   // SMs x occupancy for warps-per-chunk 1 and 8

uint32_t noalloc_split(uint32_t chunk_bytes, int *wpc) {
    *wpc = chunk_bytes >= 16384u ? 8 : 1;
    uint32_t cpt = (128u << 10) / chunk_bytes;
    if (cpt < 1) cpt = 1;
    const uint32_t groups = 8u / (uint32_t)*wpc;
    if (cpt < groups) cpt = groups;
    if (cpt > 256) cpt = 256;
    return cpt;
}

}  // namespace

// Every call of crac_pass_noalloc shares this array (it keeps the last call's
// contents; each call zeroes the part it uses before its pass).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

extern "C" crac_status_t crac_pass_noalloc(const crac_region_t *regions_dev, uint32_t n_regions,
                                           uint64_t n_chunks, uint32_t chunk_bytes,
                                           const uint64_t *fp_old_dev, uint64_t *fp_new_dev,
                                           uint64_t *idx_dev, uint64_t *off_dev, uint64_t idx_cap,
                                           uint8_t *staging_dev, uint64_t staging_cap,
                                           crac_pass_totals_t *totals_dev, crac_stream_t stream) {
    using namespace crac;
    static_assert(sizeof(crac_region_t) == sizeof(CkptDesc), "region layout");
    static_assert(sizeof(crac_pass_totals_t) == 24, "totals layout");
    if (chunk_bytes < 16 || chunk_bytes > (1u << 24) || (chunk_bytes & (chunk_bytes - 1)))
        return CRAC_ERR_INVALID_ARG;
    if (!totals_dev || (n_chunks && (!regions_dev || !n_regions || !fp_new_dev || !idx_dev || !off_dev)))
        return CRAC_ERR_INVALID_ARG;
    int wpc;
    const uint32_t cpt = noalloc_split(chunk_bytes, &wpc);
    const uint64_t n_tiles = (n_chunks + cpt - 1) / cpt;
    if (n_tiles > CRAC_NOALLOC_MAX_TILES) return CRAC_ERR_INVALID_ARG;   // beyond the fixed scratch
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev >= kNoAllocMaxDevices) {
        note_cuda_error(e == cudaSuccess ? (int)cudaErrorInvalidDevice : (int)e);
        return CRAC_ERR_CUDA;
    }
    void *scratch = nullptr;
    int grid_per[2] = {0, 0};
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            // One-time set-up on this device (it is current): the host-side name
            // g_noalloc_scratch is only a stand-in, the kernel needs the device address.
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) {
                note_cuda_error((int)e);
                return CRAC_ERR_CUDA;
            }
            int sms = 0;
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) {
                note_cuda_error((int)e);
                return CRAC_ERR_CUDA;
            }
            g_noalloc_grid[dev][0] = sms * (ckpt_fused_max_ctas_per_sm(256, 1) > 0 ? ckpt_fused_max_ctas_per_sm(256, 1) : 1);
            g_noalloc_grid[dev][1] = sms * (ckpt_fused_max_ctas_per_sm(256, 8) > 0 ? ckpt_fused_max_ctas_per_sm(256, 8) : 1);
            g_noalloc_addr[dev] = p;
        }
        scratch = g_noalloc_addr[dev];
        grid_per[0] = g_noalloc_grid[dev][0];
        grid_per[1] = g_noalloc_grid[dev][1];
    }
    const size_t used = sizeof(CkptCtrl) + 16 * n_tiles;
    e = cudaMemsetAsync(scratch, 0, used, s);   // control block + status words start at zero
    if (e == cudaSuccess && n_tiles) {
        CkptParams P{};
        P.desc = reinterpret_cast<const CkptDesc *>(regions_dev);
        P.n_allocs = n_regions;
        uint32_t l = 0;
        while ((1u << l) < chunk_bytes) ++l;
        P.log2_chunk = l;
        P.c_begin = 0;
        P.c_end = n_chunks;
        P.cpt = cpt;
        P.n_tiles = (uint32_t)n_tiles;
        P.fp_old = fp_old_dev;
        P.fp_new = fp_new_dev;
        P.idx_out = idx_dev;
        P.off_out = off_dev;
        P.idx_cap = idx_cap;
        P.staging = staging_dev;
        P.staging_cap = staging_dev ? staging_cap : 0;
        P.ctrl = reinterpret_cast<CkptCtrl *>(scratch);
        P.tile_cnt = reinterpret_cast<uint64_t *>(static_cast<unsigned char *>(scratch) + sizeof(CkptCtrl));
        P.tile_bytes = P.tile_cnt + n_tiles;
        P.timeout_ns = 2000000000ull;
        P.skip_first_ticket = 0;
        const uint64_t g = grid_per[wpc == 8 ? 1 : 0];
        e = launch_ckpt_fused(P, 256, wpc, (int)(n_tiles < g ? n_tiles : g), s);
    }
    // totals = {reserved, err, k, payload_bytes}: the control block's layout from byte 0
    if (e == cudaSuccess) e = cudaMemcpyAsync(totals_dev, scratch, sizeof(crac_pass_totals_t), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
        note_cuda_error((int)e);
        return CRAC_ERR_CUDA;
    }
    return CRAC_OK;
}
