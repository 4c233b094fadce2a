// The CRZ1 encoder: a segment's raw payload (device staging) -> one stream
// per entry, written to device memory or straight into mapped pinned memory.
#include "crac_codec.cuh"

namespace crac {

namespace {

constexpr int kCodecNT = 256;
constexpr int kCodecWarps = kCodecNT / 32;
constexpr uint32_t kCodecTileMax = 128;   // entries per tile (a 64 KiB tile of 512-byte chunks)

// Exclusive prefix over the CTA of one value per thread, and the total.
// Every thread calls it; s_warp holds kCodecWarps values.
template <typename T>
__device__ __forceinline__ T cta_excl_scan(T v, T *s_warp, T *total) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T t = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    T before = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < kCodecWarps; ++w) {
        const T x = s_warp[w];
        if (w < warp) before += x;
        tot += x;
    }
    __syncthreads();   // s_warp may be reused
    *total = tot;
    return before + inc - v;
}

// Decoupled look-back over one status array (one full warp, tile > 0):
// the exclusive prefix of the tiles before `tile`.  A wait that runs out
// sets kErrTimeout and counts the tile as empty.
__device__ uint64_t lookback1(uint64_t *status, uint32_t tile, int lane, uint64_t timeout_ns, unsigned int *err) {
    uint64_t acc = 0;
    int64_t j = (int64_t)tile - 1;
    const uint64_t t0 = globaltimer();
    // once a wait has run out anywhere, later tiles give up at once
    bool gave_up = (*(volatile unsigned int *)err & kErrTimeout) != 0;
    for (;;) {
        const int64_t t = j - lane;
        uint64_t w = kFlagInc;   // tiles before 0: inclusive 0
        if (t >= 0) {
            uint32_t spins = 0;
            for (;;) {
                w = ld_status(status + t);
                if (w >> 62) break;
                if (gave_up || ((++spins & 31u) == 0 && (globaltimer() - t0 > timeout_ns || spins > (1u << 28)))) {
                    gave_up = true;
                    atomicOr(err, kErrTimeout);
                    w = kFlagInc;
                    break;
                }
                __nanosleep(64);
            }
        }
        const unsigned inc = __ballot_sync(kFull, (w >> 62) == 2);
        const int lim = inc ? __ffs(inc) - 1 : 31;
        acc += warp_sum(lane <= lim ? (w & kValMask) : 0);
        if (inc) return acc;
        j -= 32;
    }
}

// ---- shared-memory staging of the raw payload --------------------------
// A tile's raw bytes (at most one 64 KiB window; a chunk above 64 KiB is
// taken window by window) are brought into shared memory by one bulk async
// copy completing on an mbarrier, so both passes over them (headers, then
// units) read shared memory and the staging buffer is read from HBM once.
constexpr uint32_t kWin = 65536;
constexpr uint32_t kWinBlocks = kWin / 512;
constexpr size_t kEncSmem = kWin + 32 + 16;   // window (+ alignment slack), mbarrier

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the mbarrier phase `par`; false if it does not complete
// within the time limit.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t par, uint64_t timeout_ns) {
    if (mbar_try(bar, par)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try(bar, par)) return true;
        if ((i & 63u) == 0 && (globaltimer() - t0 > timeout_ns || i > (1u << 28))) return false;
    }
}

// Staging bytes [wa, wb) -> shared memory (whole CTA, after every thread is
// done with the previous window).  *sb receives where byte wa landed.
// Returns false on every thread if the copy did not complete in time: then
// kErrTimeout is set and the CTA must stop.  Before that the CTA stays
// resident while the copy may still land in its shared memory (in bounded
// rounds), so that no later CTA is given that memory while it is written;
// a copy that never lands also sets kErrLostCopy.
__device__ bool load_window(const CodecParams &P, uint8_t *sdata, uint64_t *bar, uint32_t *phase, uint64_t wa,
                            uint64_t wb, const uint8_t **sb) {
    const uint64_t a0 = wa & ~15ull, a1 = (wb + 15) & ~15ull;   // 16-byte aligned, inside the staging slack
    if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.relaxed.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                     "r"((uint32_t)(a1 - a0))
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_addr(sdata)),
            "l"(P.src + a0), "r"((uint32_t)(a1 - a0)), "r"(smem_addr(bar))
            : "memory");
    }
    const uint32_t par = *phase;
    *phase ^= 1u;
    const bool ok = mbar_wait_bounded(bar, par, P.timeout_ns);
    if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) {
            atomicOr(P.err, kErrTimeout);
            bool landed = false;
            for (int r = 0; r < kCopyDrainRounds && !landed; ++r) landed = mbar_wait_bounded(bar, par, P.timeout_ns);
            if (!landed) atomicOr(P.err, kErrLostCopy);
        }
        __syncthreads();
        return false;
    }
    *sb = sdata + (wa - a0);
    return true;
}

// 16 bytes at p (generic, any alignment) to a 16-byte aligned q.
__device__ __forceinline__ void copy_bytes_cta(uint8_t *q, const uint8_t *p, uint64_t len, int tid) {
    const uint64_t nv = len >> 4;
    for (uint64_t v = tid; v < nv; v += kCodecNT) *reinterpret_cast<uint4 *>(q + 16 * v) = load16_any(p + 16 * v);
    for (uint64_t i = 16 * nv + tid; i < len; i += kCodecNT) q[i] = p[i];
}

__global__ void __launch_bounds__(kCodecNT, 3) crz_encode_kernel(const CodecParams P) {
    extern __shared__ __align__(16) uint8_t dsm[];
    uint8_t *sdata = dsm;
    uint64_t *bar = reinterpret_cast<uint64_t *>(dsm + kWin + 32);
    __shared__ uint32_t s_tile, s_skip;
    __shared__ uint32_t s_nbp[kCodecTileMax + 1];    // tile-local prefix of block counts
    __shared__ uint32_t s_wsum[kCodecTileMax];       // per entry: sum of its blocks' widths
    __shared__ uint32_t s_z[kCodecTileMax];          // per entry: stream length
    __shared__ uint64_t s_zpre[kCodecTileMax + 1];   // tile-local prefix of padded stream lengths
    __shared__ uint64_t s_base;                      // the tile's output offset
    __shared__ uint32_t s_boff[kWinBlocks];          // prefix of unit counts over a window's blocks
    __shared__ uint8_t s_bent[kWinBlocks];           // one-window tile: the entry of each block
    __shared__ __align__(16) uint8_t s_units[kCodecWarps][512];   // per warp: a block's units
    __shared__ uint64_t s_off[kCodecTileMax + 1];    // the tile's entry offsets in staging
    __shared__ uint64_t s_hdr[kWinBlocks];           // header words of the window's blocks
    __shared__ uint32_t s_w32[kCodecWarps];
    __shared__ uint64_t s_w64[kCodecWarps];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const CrzLane LT = crz_lane(lane);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    uint32_t phase = 0;
    for (;;) {
        __syncthreads();   // the previous tile's shared state (and window) is consumed
        if (tid == 0) {
            uint32_t t = atomicAdd(P.ticket, 1u);
            // fault injection: tile 0 is never processed, so the wait of the
            // tiles after it runs out (bounded) and the launch reports kErrTimeout
            if (P.skip_first_ticket && t == 0) t = atomicAdd(P.ticket, 1u);
            s_tile = P.tile_begin + t;
        }
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= P.n_tiles) return;
        const uint64_t e0 = (uint64_t)tile * P.tile_entries;
        const uint32_t ne = (uint32_t)umin64(P.tile_entries, P.k - e0);   // 1 .. kCodecTileMax
        const uint64_t r0 = P.off[e0], r1 = P.off[e0 + ne];
        // One window, or (a single chunk above 64 KiB) several.
        const uint32_t n_win = r1 - r0 <= kWin ? 1u : (uint32_t)((r1 - r0 + kWin - 1) / kWin);

        // Entry lengths and block counts.
        uint64_t L_t = 0;
        uint32_t nb_t = 0;
        if ((uint32_t)tid < ne) {
            const uint64_t a = P.off[e0 + tid], b = P.off[e0 + tid + 1];
            s_off[tid] = a;
            if ((uint32_t)tid == ne - 1) s_off[ne] = b;
            L_t = b - a;
            nb_t = (uint32_t)(L_t >> 9);
            s_wsum[tid] = 0;
        }
        uint32_t nb_all;
        const uint32_t nb_ex = cta_excl_scan<uint32_t>(nb_t, s_w32, &nb_all);
        if ((uint32_t)tid < ne) s_nbp[tid] = nb_ex;
        if (tid == 0) s_nbp[ne] = nb_all;
        __syncthreads();
        // Entry of each block, searched once (a several-window tile is one
        // entry): the passes below look it up instead of searching per block.
        if (n_win == 1 && (uint32_t)tid < nb_all) {
            uint32_t lo = 0, hi = ne;   // last entry whose first block is <= tid
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (s_nbp[mid] <= (uint32_t)tid) lo = mid;
                else hi = mid;
            }
            s_bent[tid] = (uint8_t)lo;
        }
        __syncthreads();

        // Phase 1: every block's header word -- made by the pass (then only a
        // one-window tile's window is brought in here, for phase 2), else
        // computed from the window in shared memory.
        bool dead = false;
        if (P.chdr) {
            if (n_win == 1) {
                const uint8_t *sb = nullptr;
                dead = !load_window(P, sdata, bar, &phase, r0, r1, &sb);   // uniform across the CTA
            }
            for (uint32_t fb = tid; fb < nb_all && !dead; fb += kCodecNT) {
                const uint32_t lo = n_win == 1 ? s_bent[fb] : 0u;
                const uint32_t b = fb - s_nbp[lo];
                const uint64_t h = P.chdr[(P.idx[e0 + lo] << P.log2_bpc) + b];
                if (n_win == 1) s_hdr[fb] = h;
                else P.hdr[(s_off[lo] >> 9) + b] = h;   // read back window by window in phase 2
                atomicAdd(&s_wsum[lo], crz_width_sum(h));
            }
            __syncthreads();
        }
        for (uint32_t w = 0; w < (P.chdr ? 0u : n_win); ++w) {
            const uint64_t wa = r0 + (uint64_t)w * kWin, wb = umin64(r1, wa + kWin);
            const uint8_t *sb = nullptr;
            if (!load_window(P, sdata, bar, &phase, wa, wb, &sb)) {
                dead = true;   // uniform across the CTA
                break;
            }
            // blocks of this window, as tile-flattened ids [f0, f1)
            const uint32_t f0 = n_win == 1 ? 0u : w * kWinBlocks;
            const uint32_t f1 = n_win == 1 ? nb_all : (uint32_t)umin64(nb_all, (uint64_t)(w + 1) * kWinBlocks);
            for (uint32_t fb = f0 + warp; fb < f1; fb += kCodecWarps) {
                const uint32_t lo = n_win == 1 ? s_bent[fb] : 0u;
                const uint32_t b = fb - s_nbp[lo];
                const uint64_t o = s_off[lo];
                const uint4 v = load16_any(sb + (o - wa) + 512ull * b + 16u * lane);
                const uint32_t r[4] = {crz_rot(v.x), crz_rot(v.y), crz_rot(v.z), crz_rot(v.w)};
                const uint64_t h = crz_block_header(r);
                if (lane == 0) {
                    s_hdr[fb - f0] = h;
                    if (n_win > 1) P.hdr[(o >> 9) + b] = h;   // for the second pass over the windows
                    atomicAdd(&s_wsum[lo], crz_width_sum(h));
                }
            }
            __syncthreads();
        }

        // Stream lengths: coded when that is shorter, else the chunk itself.
        uint64_t pz = 0;
        if ((uint32_t)tid < ne) {
            const uint64_t zc = crz_head_bytes(nb_t) + 16ull * s_wsum[tid] + (L_t & 511u);
            const uint64_t z = (nb_t && zc < L_t) ? zc : L_t;
            s_z[tid] = (uint32_t)z;   // <= chunk bytes <= 2^24
            P.zlen[e0 + tid] = z;
            pz = (z + 15) & ~15ull;
        }
        uint64_t tile_bytes;
        const uint64_t z_ex = cta_excl_scan<uint64_t>(pz, s_w64, &tile_bytes);
        if ((uint32_t)tid < ne) s_zpre[tid] = z_ex;
        if (tid == 0) s_zpre[ne] = tile_bytes;

        // The tile's output offset: publish, look back, publish.
        if (warp == 0) {
            uint64_t base = 0;
            if (tile == 0) {
                if (lane == 0) st_status(P.status, kFlagInc | tile_bytes);
            } else {
                if (lane == 0) st_status(P.status + tile, kFlagAgg | tile_bytes);
                base = lookback1(P.status, tile, lane, P.timeout_ns, P.err);
                if (lane == 0) st_status(P.status + tile, kFlagInc | ((base + tile_bytes) & kValMask));
            }
            if (lane == 0) {
                s_base = base;
                const bool over = base + tile_bytes > P.dst_cap;
                if (over) atomicOr(P.err, kErrBounds);
                s_skip = over || (*(volatile unsigned int *)P.err & kErrTimeout) ? 1u : 0u;
            }
        }
        __syncthreads();
        const uint64_t base = s_base;
        if ((uint32_t)tid < ne) P.zoff[e0 + tid] = base + s_zpre[tid];
        // The end offset of the last tile (of the launch): zoff[k], or the
        // first offset of the next launch's first tile, which writes the same.
        if (tid == 0 && (e0 + ne == P.k || tile + 1 == P.n_tiles)) P.zoff[e0 + ne] = base + tile_bytes;
        if (dead) return;   // a copy that never completed: this CTA stops (error reported)
        if (s_skip) continue;

        // Phase 2: headers and padding of every coded entry, then the units
        // and raw bytes window by window.
        for (uint32_t fb = tid; fb < nb_all; fb += kCodecNT) {
            const uint32_t lo = n_win == 1 ? s_bent[fb] : 0u;
            const uint64_t o = s_off[lo], L = s_off[lo + 1] - o;
            if (s_z[lo] == L) continue;   // raw entry
            const uint32_t b = fb - s_nbp[lo];
            reinterpret_cast<uint64_t *>(P.dst + base + s_zpre[lo])[b] = n_win == 1 ? s_hdr[fb] : P.hdr[(o >> 9) + b];
        }
        for (uint32_t t = tid; t < ne; t += kCodecNT) {
            const uint64_t L = s_off[t + 1] - s_off[t], z = s_z[t];
            uint8_t *d = P.dst + base + s_zpre[t];
            const uint32_t nb = s_nbp[t + 1] - s_nbp[t];
            if (z != L && (nb & 1)) reinterpret_cast<uint64_t *>(d)[nb] = 0;   // header pad
            for (uint64_t i = z; i < ((z + 15) & ~15ull); ++i) d[i] = 0;            // stream pad
        }
        uint32_t carry = 0;   // multi-window chunk: units of the earlier windows' blocks
        for (uint32_t w = 0; w < n_win; ++w) {
            const uint64_t wa = r0 + (uint64_t)w * kWin, wb = umin64(r1, wa + kWin);
            const uint8_t *sb = sdata + (wa & 15u);
            const uint32_t f0 = n_win == 1 ? 0u : w * kWinBlocks;
            const uint32_t f1 = n_win == 1 ? nb_all : (uint32_t)umin64(nb_all, (uint64_t)(w + 1) * kWinBlocks);
            if (n_win > 1) {
                __syncthreads();   // every thread is done with the previous window
                if (!load_window(P, sdata, bar, &phase, wa, wb, &sb)) return;   // uniform; error reported
                // one entry: its header words of this window, back from global scratch
                if (f0 + tid < f1) s_hdr[tid] = P.hdr[(s_off[0] >> 9) + f0 + tid];
                __syncthreads();
            }
            // unit offsets: prefix of the blocks' unit counts over the window
            uint32_t wcount = 0;
            {
                uint32_t v = 0;
                if (f0 + tid < f1) v = crz_width_sum(s_hdr[tid]);
                const uint32_t ex = cta_excl_scan<uint32_t>(v, s_w32, &wcount);
                if ((uint32_t)tid < kWinBlocks) s_boff[tid] = ex;
            }
            __syncthreads();
            for (uint32_t fb = f0 + warp; fb < f1; fb += kCodecWarps) {
                const uint32_t lo = n_win == 1 ? s_bent[fb] : 0u;
                const uint64_t o = s_off[lo], L = s_off[lo + 1] - o;
                if (s_z[lo] == L) continue;   // raw entry: copied below
                const uint32_t b = fb - s_nbp[lo];
                // units before this block within its entry
                const uint32_t before = n_win == 1 ? s_boff[fb] - s_boff[s_nbp[lo]] : carry + s_boff[fb - f0];
                const uint4 v = load16_any(sb + (o - wa) + 512ull * b + 16u * lane);
                const uint32_t r[4] = {crz_rot(v.x), crz_rot(v.y), crz_rot(v.z), crz_rot(v.w)};
                uint32_t pw[4];
                crz_bytes_transpose(r, pw);
                uint8_t *d = P.dst + base + s_zpre[lo] + crz_head_bytes(L >> 9) + 16ull * before;
                crz_block_units(s_hdr[fb - f0], pw, d, lane, LT, s_units[warp]);
            }
            carry += wcount;
            // raw entries, and the tails of coded ones, where they overlap the window
            for (uint32_t t = 0; t < ne; ++t) {
                const uint64_t o = s_off[t], L = s_off[t + 1] - o;
                uint8_t *d = P.dst + base + s_zpre[t];
                uint64_t lo_b, hi_b, to;   // entry bytes [lo_b, hi_b) go to d + to + (x - lo_b)
                if (s_z[t] == L) {
                    lo_b = 0;
                    hi_b = L;
                    to = 0;
                } else {
                    lo_b = L & ~511ull;
                    hi_b = L;
                    to = s_z[t] - (L & 511u);
                }
                const uint64_t x0 = o + lo_b > wa ? o + lo_b : wa, x1 = umin64(o + hi_b, wb);
                if (x1 > x0) copy_bytes_cta(d + to + (x0 - o - lo_b), sb + (x0 - wa), x1 - x0, tid);
            }
        }
    }
}

// ---- the encoder when the pass made the block headers --------------------
// With every block's header word already in P.chdr, a stream's length needs
// only its headers' widths: crz_size_kernel sizes and places every stream
// first, and crz_encode_sized_kernel then codes without any wait between
// CTAs, one warp per 64 KiB segment of an entry, straight from staging.
constexpr uint32_t kSizeTile = kCodecNT;   // entries per tile of the sizing kernel
constexpr uint32_t kSegBlocks = 128;       // blocks per work item of the sized encoder

// zlen and zoff of every entry (and zoff[k]) from the header widths: one warp
// per entry sums them; a tile's padded lengths are scanned and placed by a
// decoupled look-back over the earlier tiles (tiles are taken in ticket
// order, so every predecessor has started).  piece_off[i] receives zoff of
// entry k * i / pieces, for i = 0 .. pieces.
__global__ void __launch_bounds__(kCodecNT) crz_size_kernel(const CodecParams P) {
    __shared__ uint32_t s_tile;
    __shared__ uint64_t s_z[kSizeTile];
    __shared__ uint64_t s_w64[kCodecWarps];
    __shared__ uint64_t s_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (;;) {
        __syncthreads();   // the previous tile's shared state is consumed
        if (tid == 0) {
            uint32_t t = atomicAdd(P.ticket, 1u);
            // fault injection: tile 0 is never sized, so the later tiles'
            // bounded look-back waits run out and the launch reports kErrTimeout
            if (P.skip_first_ticket && t == 0) t = atomicAdd(P.ticket, 1u);
            s_tile = t;
        }
        __syncthreads();
        const uint64_t e0 = (uint64_t)s_tile * kSizeTile;
        if (e0 >= P.k) return;
        const uint32_t ne = (uint32_t)umin64(kSizeTile, P.k - e0);
        for (uint32_t t = warp; t < ne; t += kCodecWarps) {
            const uint64_t e = e0 + t;
            const uint64_t L = P.off[e + 1] - P.off[e], nb = L >> 9;
            const uint64_t *h = P.chdr + (P.idx[e] << P.log2_bpc);
            uint32_t w = 0;
            for (uint64_t b = lane; b < nb; b += 32) w += crz_width_sum(h[b]);
            w = __reduce_add_sync(kFull, w);   // <= 32 per block, nb <= 2^15
            if (lane == 0) {
                const uint64_t zc = crz_head_bytes(nb) + 16ull * w + (L & 511u);
                const uint64_t z = (nb && zc < L) ? zc : L;
                P.zlen[e] = z;
                s_z[t] = (z + 15) & ~15ull;
            }
        }
        __syncthreads();
        uint64_t tile_bytes;
        const uint64_t ex = cta_excl_scan<uint64_t>((uint32_t)tid < ne ? s_z[tid] : 0ull, s_w64, &tile_bytes);
        const uint32_t tile = (uint32_t)(e0 / kSizeTile);
        if (warp == 0) {
            uint64_t base = 0;
            if (tile == 0) {
                if (lane == 0) st_status(P.status, kFlagInc | tile_bytes);
            } else {
                if (lane == 0) st_status(P.status + tile, kFlagAgg | tile_bytes);
                base = lookback1(P.status, tile, lane, P.timeout_ns, P.err);
                if (lane == 0) st_status(P.status + tile, kFlagInc | ((base + tile_bytes) & kValMask));
            }
            if (lane == 0) s_base = base;
        }
        __syncthreads();
        const uint64_t base = s_base;
        if ((uint32_t)tid < ne) {
            const uint64_t e = e0 + tid, zo = base + ex;
            P.zoff[e] = zo;
            // entries that start a piece: k * i / pieces == e for some i
            const uint64_t i = (e * P.pieces + P.k - 1) / P.k;   // smallest i with k * i / pieces >= e
            if (i < P.pieces && P.k * i / P.pieces == e) P.piece_off[i] = zo;
        }
        if (tid == 0 && e0 + ne == P.k) {
            P.zoff[P.k] = base + tile_bytes;
            P.piece_off[P.pieces] = base + tile_bytes;
        }
    }
}

// Bytes [x0, x1) of a raw entry (src, any alignment) to d (16-byte aligned),
// one warp.
__device__ __forceinline__ void copy_raw_warp(uint8_t *d, const uint8_t *src, uint64_t x0, uint64_t x1, int lane) {
    const uint64_t nv = (x1 - x0) >> 4;
    for (uint64_t v = lane; v < nv; v += 32)
        *reinterpret_cast<uint4 *>(d + x0 + 16 * v) = load16_any(src + x0 + 16 * v);
    for (uint64_t i = x0 + 16 * nv + lane; i < x1; i += 32) d[i] = src[i];
}

// Entries [e_begin, e_end) -> their streams at zoff (made by crz_size_kernel):
// work item = (entry, 64 KiB segment), one warp each, in entry order.  A
// coded segment writes its blocks' header words and units (unit offsets: the
// widths of the entry's earlier blocks, then a warp scan over the segment's),
// and the segment holding the entry's last block also the header pad, the
// raw tail and the stream pad; a raw entry is copied segment by segment.
__global__ void __launch_bounds__(kCodecNT, 4) crz_encode_sized_kernel(const CodecParams P) {
    __shared__ __align__(16) uint8_t s_units[kCodecWarps][512];
    __shared__ uint32_t s_boff[kCodecWarps][kSegBlocks];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const CrzLane LT = crz_lane(lane);
    const uint32_t spe = P.segs_per_entry;
    const uint64_t items = (P.e_end - P.e_begin) * spe;
    const uint64_t nw = ((uint64_t)gridDim.x * kCodecNT) >> 5;
    for (uint64_t it = ((uint64_t)blockIdx.x * kCodecNT + tid) >> 5; it < items; it += nw) {
        const uint64_t e = P.e_begin + it / spe;
        const uint32_t sg = (uint32_t)(it % spe);
        const uint64_t o = P.off[e], L = P.off[e + 1] - o;
        const uint64_t z = P.zlen[e];
        uint8_t *d = P.dst + P.zoff[e];
        const uint8_t *src = P.src + o;
        if (z == L) {   // stored raw
            const uint64_t x0 = (uint64_t)sg * (512ull * kSegBlocks);
            if (x0 >= L) continue;
            const uint64_t x1 = umin64(L, x0 + 512ull * kSegBlocks);
            copy_raw_warp(d, src, x0, x1, lane);
            if (x1 == L)
                for (uint64_t i = L + lane; i < ((L + 15) & ~15ull); i += 32) d[i] = 0;
            continue;
        }
        const uint64_t nb = L >> 9;   // >= 1: a coded stream is shorter than its entry
        const uint32_t last = (uint32_t)((nb - 1) / kSegBlocks);
        if (sg > last) continue;
        const uint64_t b0 = (uint64_t)sg * kSegBlocks;
        const uint32_t nseg = (uint32_t)umin64(kSegBlocks, nb - b0);
        const uint64_t *h = P.chdr + (P.idx[e] << P.log2_bpc);
        uint64_t *dh = reinterpret_cast<uint64_t *>(d);
        // units of the entry's blocks before this segment
        uint32_t before = 0;
        for (uint64_t b = lane; b < b0; b += 32) before += crz_width_sum(h[b]);
        before = __reduce_add_sync(kFull, before);
        // lane l: blocks b0 + 4l .. 4l + 3 of the segment -> header words, unit offsets
        uint32_t wq[4], sum = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t j = 4u * lane + q;
            wq[q] = 0;
            if (j < nseg) {
                const uint64_t hw = h[b0 + j];
                dh[b0 + j] = hw;
                wq[q] = crz_width_sum(hw);
            }
            sum += wq[q];
        }
        uint32_t inc = sum;
#pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, inc, s);
            if (lane >= s) inc += t;
        }
        uint32_t run = before + inc - sum;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t j = 4u * lane + q;
            if (j < nseg) s_boff[warp][j] = run;
            run += wq[q];
        }
        const uint64_t head = crz_head_bytes(nb);
        if (sg == last && lane == 0 && (nb & 1)) dh[nb] = 0;   // header pad
        __syncwarp();
        // blocks, the next one's 16 bytes loaded while this one is coded
        uint4 v = load16_any(src + 512ull * b0 + 16u * lane);
        for (uint32_t j = 0; j < nseg; ++j) {
            const uint64_t b = b0 + j;
            uint4 nx = v;
            if (j + 1 < nseg) nx = load16_any(src + 512ull * (b + 1) + 16u * lane);
            const uint32_t r[4] = {crz_rot(v.x), crz_rot(v.y), crz_rot(v.z), crz_rot(v.w)};
            uint32_t pw[4];
            crz_bytes_transpose(r, pw);
            crz_block_units(__ldg(h + b), pw, d + head + 16ull * s_boff[warp][j], lane, LT, s_units[warp]);
            v = nx;
        }
        if (sg == last) {   // the raw tail, then the stream pad
            const uint64_t tl = L & 511u;
            copy_raw_warp(d + z - tl - 512ull * nb, src, 512ull * nb, L, lane);
            for (uint64_t i = z + lane; i < ((z + 15) & ~15ull); i += 32) d[i] = 0;
        }
        __syncwarp();   // s_boff is rewritten by the warp's next item
    }
}

}  // namespace

uint32_t crz_tile_max() { return kCodecTileMax; }

uint32_t crz_sized_segs(uint32_t log2S) { return log2S > 16 ? 1u << (log2S - 16) : 1u; }

cudaError_t launch_crz_size(const CodecParams &p, int grid, cudaStream_t s) {
    if (p.k == 0) return cudaSuccess;
    crz_size_kernel<<<grid, kCodecNT, 0, s>>>(p);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) count_launches(1);
    return e;
}

cudaError_t launch_crz_encode_sized(const CodecParams &p, int grid, cudaStream_t s) {
    if (p.e_end <= p.e_begin) return cudaSuccess;
    crz_encode_sized_kernel<<<grid, kCodecNT, 0, s>>>(p);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) count_launches(1);
    return e;
}

int crz_sized_max_ctas_per_sm() {
    static int v = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, crz_encode_sized_kernel, kCodecNT, 0) != cudaSuccess)
            n = 1;
        cudaGetLastError();
        v = n > 0 ? n : 1;
    });
    return v;
}

int crz_encode_max_ctas_per_sm() {
    static int v = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        int n = 0;
        if (cudaFuncSetAttribute(crz_encode_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEncSmem) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, crz_encode_kernel, kCodecNT, kEncSmem) != cudaSuccess)
            n = 1;
        cudaGetLastError();
        v = n > 0 ? n : 1;
    });
    return v;
}

cudaError_t launch_crz_encode(const CodecParams &p, int grid, cudaStream_t s) {
    if (p.k == 0) return cudaSuccess;
    crz_encode_max_ctas_per_sm();   // sets the dynamic shared memory limit once
    crz_encode_kernel<<<grid, kCodecNT, kEncSmem, s>>>(p);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) count_launches(1);
    return e;
}

}  // namespace crac
