// The CRZ1 encoder: a segment's raw payload (device staging) -> one stream
// per entry, written to device memory or straight into mapped pinned memory.
#include "crac_codec.cuh"

namespace crac {

namespace {

constexpr int kCodecNT = 256;
constexpr int kCodecWarps = kCodecNT / 32;
constexpr uint32_t kCodecTileMax = kCodecNT;   // one entry per thread in the tile bookkeeping

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
    bool gave_up = false;
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

__global__ void __launch_bounds__(kCodecNT) crz_encode_kernel(const CodecParams P) {
    __shared__ uint32_t s_tile, s_skip;
    __shared__ uint32_t s_nbp[kCodecTileMax + 1];    // tile-local prefix of block counts
    __shared__ uint32_t s_wsum[kCodecTileMax];       // per entry: sum of its blocks' widths
    __shared__ uint32_t s_z[kCodecTileMax];          // per entry: stream length
    __shared__ uint64_t s_zpre[kCodecTileMax + 1];   // tile-local prefix of padded stream lengths
    __shared__ uint64_t s_base;                      // the tile's output offset
    __shared__ uint32_t s_boff[kCodecNT];            // units before each block of a batch
    __shared__ uint32_t s_w32[kCodecWarps];
    __shared__ uint64_t s_w64[kCodecWarps];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (;;) {
        __syncthreads();   // the previous tile's shared state is consumed
        if (tid == 0) s_tile = atomicAdd(P.ticket, 1u);
        __syncthreads();
        const uint32_t tile = s_tile;
        if (tile >= P.n_tiles) return;
        const uint64_t e0 = (uint64_t)tile * P.tile_entries;
        const uint32_t ne = (uint32_t)umin64(P.tile_entries, P.k - e0);   // 1 .. kCodecTileMax

        // Entry lengths and block counts.
        uint64_t L_t = 0;
        uint32_t nb_t = 0;
        if ((uint32_t)tid < ne) {
            L_t = P.off[e0 + tid + 1] - P.off[e0 + tid];
            nb_t = (uint32_t)(L_t >> 9);
            s_wsum[tid] = 0;
        }
        uint32_t nb_all;
        const uint32_t nb_ex = cta_excl_scan<uint32_t>(nb_t, s_w32, &nb_all);
        if ((uint32_t)tid < ne) s_nbp[tid] = nb_ex;
        if (tid == 0) s_nbp[ne] = nb_all;
        __syncthreads();

        // Phase 1: the header word of every block of the tile (a warp per block).
        for (uint32_t fb = warp; fb < nb_all; fb += kCodecWarps) {
            uint32_t lo = 0, hi = ne;   // last entry whose first block is <= fb
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (s_nbp[mid] <= fb) lo = mid;
                else hi = mid;
            }
            const uint32_t b = fb - s_nbp[lo];
            const uint64_t o = P.off[e0 + lo];
            const uint4 w = load16_any(P.src + o + 512ull * b + 16u * lane);
            const uint32_t r[4] = {crz_rot(w.x), crz_rot(w.y), crz_rot(w.z), crz_rot(w.w)};
            const uint64_t h = crz_block_header(r);
            if (lane == 0) {
                P.hdr[(o >> 9) + b] = h;
                atomicAdd(&s_wsum[lo], crz_width_sum(h));
            }
        }
        __syncthreads();

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
        if (tid == 0 && e0 + ne == P.k) P.zoff[P.k] = base + tile_bytes;
        if (s_skip) continue;

        // Phase 2: each entry's stream, entry by entry with the whole CTA.
        for (uint32_t t = 0; t < ne; ++t) {
            const uint64_t o = P.off[e0 + t];
            const uint64_t L = P.off[e0 + t + 1] - o;
            const uint64_t z = s_z[t];
            const uint64_t zpad = (z + 15) & ~15ull;
            uint8_t *d = P.dst + base + s_zpre[t];
            const uint8_t *sp = P.src + o;
            if (z == L) {
                copy_group<kCodecNT>(d, sp, L, tid);
                for (uint64_t i = L + tid; i < zpad; i += kCodecNT) d[i] = 0;
                continue;
            }
            const uint64_t nb = L >> 9, head = crz_head_bytes(nb);
            const uint64_t *hb = P.hdr + (o >> 9);
            uint64_t *dh = reinterpret_cast<uint64_t *>(d);
            for (uint64_t b = tid; b < nb; b += kCodecNT) dh[b] = hb[b];
            if ((nb & 1) && tid == 0) dh[nb] = 0;
            uint32_t carry = 0;   // units of the blocks before this batch
            for (uint64_t B = 0; B < nb; B += kCodecNT) {
                const uint32_t ws = B + tid < nb ? crz_width_sum(hb[B + tid]) : 0u;
                uint32_t batch_units;
                s_boff[tid] = carry + cta_excl_scan<uint32_t>(ws, s_w32, &batch_units);
                __syncthreads();
                const uint32_t nbatch = (uint32_t)umin64(kCodecNT, nb - B);
                for (uint32_t bb = warp; bb < nbatch; bb += kCodecWarps) {
                    const uint64_t blk = B + bb;
                    const uint4 w = load16_any(sp + 512ull * blk + 16u * lane);
                    const uint32_t r[4] = {crz_rot(w.x), crz_rot(w.y), crz_rot(w.z), crz_rot(w.w)};
                    crz_block_units(hb[blk], r, d + head + 16ull * s_boff[bb], lane);
                }
                carry += batch_units;
                __syncthreads();   // s_boff is rewritten by the next batch
            }
            const uint64_t tl = L & 511u, tail_at = head + 16ull * carry;
            for (uint64_t i = tid; i < tl; i += kCodecNT) d[tail_at + i] = sp[512ull * nb + i];
            for (uint64_t i = z + tid; i < zpad; i += kCodecNT) d[i] = 0;
        }
    }
}

}  // namespace

uint32_t crz_tile_max() { return kCodecTileMax; }

int crz_encode_max_ctas_per_sm() {
    static int v = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, crz_encode_kernel, kCodecNT, 0) != cudaSuccess)
            n = 1;
        cudaGetLastError();
        v = n > 0 ? n : 1;
    });
    return v;
}

cudaError_t launch_crz_encode(const CodecParams &p, int grid, cudaStream_t s) {
    if (p.k == 0) return cudaSuccess;
    crz_encode_kernel<<<grid, kCodecNT, 0, s>>>(p);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) count_launches(1);
    return e;
}

}  // namespace crac
