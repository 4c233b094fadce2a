// The per-allocation comparison path: K1, K2, K3 as separate launches.
#include "crac_device.cuh"

namespace crac {

namespace {

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

}  // namespace

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

}  // namespace crac
