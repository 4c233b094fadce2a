// Restart kernels: owner marks, coverage check and scatter over every piece of
// a chain (device path), and the windowed scatter of the staged path.
#include "crac_codec.cuh"

namespace crac {

namespace {

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

// Incremental restore: a target chunk that already holds the image's bytes
// (same fingerprint) keeps them; clearing its owner makes the scatter skip it.
__global__ void __launch_bounds__(256) restore_unmark_kernel(const RestoreParams P) {
    for (uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x; i < P.n_owner; i += (uint64_t)gridDim.x * 256)
        if (P.fp_now[i] == P.fp_img[i]) P.owner[i] = 0;
}

// kCoded: some piece of the chain is coded (its decoder needs registers the
// plain copy does not, so chains without coded images keep the lean build,
// restore_scatter_kernel; coded chains run restore_scatter_coded_kernel).
template <bool kCoded>
__device__ __forceinline__ void restore_scatter_body(const RestoreParams &P, uint8_t *scratch) {
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
        // Coded image: the entry's stream length (equal to len when stored raw).
        const uint64_t z = (kCoded && pc.zlen) ? reinterpret_cast<const uint64_t *>(pc.zlen)[e - pc.entry_base] : len;
        if (o > pc.bytes || z > pc.bytes - o) {
            if (lane == 0) atomicOr(P.err, kErrBounds);
            continue;
        }
        uint8_t *dst = reinterpret_cast<uint8_t *>(d.dst) + (local << P.log2_chunk);
        const uint8_t *src = reinterpret_cast<const uint8_t *>(pc.payload) + o;
        if (!kCoded || z == len) copy_group<32>(dst, src, len, lane);
        else if (!crz_decode_warp(dst, src, len, z, lane, scratch + kCrzDecodeScratch * warp) && lane == 0)
            atomicOr(P.err, kErrCodec);
    }
}

__global__ void __launch_bounds__(kScatterNT) restore_scatter_kernel(const RestoreParams P) {
    restore_scatter_body<false>(P, nullptr);
}

__global__ void __launch_bounds__(kScatterNT, 4) restore_scatter_coded_kernel(const RestoreParams P) {
    __shared__ __align__(16) uint8_t scratch[kCrzDecodeScratch * (kScatterNT / 32)];
    restore_scatter_body<true>(P, scratch);
}

}  // namespace

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

cudaError_t launch_restore_unmark(const RestoreParams &p, int grid, cudaStream_t s) {
    if (p.n_owner == 0) return cudaSuccess;
    restore_unmark_kernel<<<grid, 256, 0, s>>>(p);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) count_launches(1);
    return e;
}

cudaError_t launch_restore_scatter(const RestoreParams &p, int grid, cudaStream_t s) {
    if (p.n_entries == 0) return cudaSuccess;
    if (p.coded) restore_scatter_coded_kernel<<<grid, kScatterNT, 0, s>>>(p);
    else restore_scatter_kernel<<<grid, kScatterNT, 0, s>>>(p);
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
