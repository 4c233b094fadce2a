// The fused TMA pass: warp-specialized, bulk copies into a shared-memory ring.
#include "crac_device.cuh"

namespace crac {

namespace {

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
    // wait, in bounded rounds, for the last phase armed on each slot before
    // the CTA exits, so that no later CTA is given shared memory that a copy
    // is still writing; a copy that never lands sets kErrLostCopy.
    if (threadIdx.x == 0) {
        for (int s = 0; s < kNSlot; ++s) {
            if (!(armed[s] & 2u)) continue;
            bool landed = false;
            for (int r = 0; r < kCopyDrainRounds && !landed; ++r) landed = mbar_wait(&full[s], armed[s] & 1u, P);
            if (!landed) atomicOr(&P.ctrl->err, kErrLostCopy);
        }
    }
}

}  // namespace

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

}  // namespace crac
