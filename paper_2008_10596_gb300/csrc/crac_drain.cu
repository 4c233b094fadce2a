// Drain of a delta pass into host images whose sizes only the device knows.
#include "crac_device.cuh"

namespace crac {

namespace {

constexpr int kDrainNT = 256;

// A checkpoint into host-resident images that returns before its pass has
// finished cannot size a copy-engine transfer of the payload: the dirty byte
// count D (and chunk count k) is only in the pass's control block in device
// memory.  This kernel, enqueued on the side stream after the pass, reads k
// and D there and copies the compacted chunk list, and the payload unless the
// pass already wrote it into host memory (src == nullptr), into the image's
// pinned blocks through their device mapping (A5, at the host link's rate).
// It copies nothing if the pass failed or a count exceeds its block.
__global__ void __launch_bounds__(kDrainNT) drain_kernel(const CkptCtrl *ctrl, const uint8_t *src, uint8_t *dst,
                                                          uint64_t cap, const uint64_t *idx_src, uint64_t *idx_dst,
                                                          uint64_t idx_cap) {
    const unsigned err = ctrl->err;
    const uint64_t k = ctrl->k, D = ctrl->D;
    if (err || D > cap || k > idx_cap) return;
    const uint64_t tid = (uint64_t)blockIdx.x * kDrainNT + threadIdx.x;
    const uint64_t nt = (uint64_t)gridDim.x * kDrainNT;
    if (src) {
        const uint64_t nv = D >> 4;   // staging and the pinned block start 256-byte aligned
        const uint4 *s16 = reinterpret_cast<const uint4 *>(src);
        uint4 *d16 = reinterpret_cast<uint4 *>(dst);
        for (uint64_t v = tid; v < nv; v += nt) __stcs(d16 + v, __ldcs(s16 + v));
        for (uint64_t i = 16 * nv + tid; i < D; i += nt) dst[i] = src[i];
    }
    for (uint64_t j = tid; j < k; j += nt) idx_dst[j] = idx_src[j];
}

// A copy of `bytes` between device memory and pinned host memory (either
// direction) by SM loads and stores through the pinned memory's device
// mapping.  On GB300 the copy engines' device-to-host rate into pinned memory
// was seen to fall to 12-30 GB/s for seconds at a time while SM stores over
// the same link held 185-193 GB/s, and every other copy-engine transfer
// (descriptor uploads, fingerprint tables) then queued behind the slow one;
// the library's per-operation transfers therefore go through this kernel.
// Both pointers 16-byte aligned take the vector path; otherwise bytes.
__global__ void __launch_bounds__(kDrainNT) link_copy_kernel(uint8_t *dst, const uint8_t *src, uint64_t bytes) {
    const uint64_t tid = (uint64_t)blockIdx.x * kDrainNT + threadIdx.x;
    const uint64_t nt = (uint64_t)gridDim.x * kDrainNT;
    uint64_t done = 0;
    if ((((uintptr_t)dst | (uintptr_t)src) & 15u) == 0) {
        const uint64_t nv = bytes >> 4;
        const uint4 *s16 = reinterpret_cast<const uint4 *>(src);
        uint4 *d16 = reinterpret_cast<uint4 *>(dst);
        for (uint64_t v = tid; v < nv; v += nt) __stcs(d16 + v, __ldcs(s16 + v));
        done = nv << 4;
    }
    for (uint64_t i = done + tid; i < bytes; i += nt) dst[i] = src[i];
}

// A small report (a pass's control block, an encoder launch's end offset and
// error bits, a restart's error word) for the host: n 8-byte words from
// device memory, then one 4-byte word zero-extended, stored by one warp into
// pinned host memory through its device mapping.  A copy-engine copy of these
// few bytes would queue behind the bulk drains on the copy engines (other
// images', other contexts') and hold up whoever waits for the report.
__global__ void report_kernel(const uint64_t *words, uint32_t n, const uint32_t *word32, uint64_t *dst) {
    for (uint32_t i = threadIdx.x; i < n; i += 32) dst[i] = words[i];
    if (word32 && threadIdx.x == 0) dst[n] = *word32;
}


// Entries [0, n) of a sparse device piece packed back to back: entry j's
// cum[j+1] - cum[j] bytes from span + off[j] to dst + cum[j] - cum[0], one
// warp per entry (serialization and ranged reads of sparse images, whose
// dirty chunks are scattered over the span one or two at a time).
__global__ void __launch_bounds__(kDrainNT) sparse_pack_kernel(uint8_t *dst, const uint8_t *span,
                                                               const uint64_t *off, const uint64_t *cum, uint64_t n) {
    const int lane = threadIdx.x & 31;
    const uint64_t nw = ((uint64_t)gridDim.x * kDrainNT) >> 5;
    const uint64_t base = cum[0];
    for (uint64_t j = ((uint64_t)blockIdx.x * kDrainNT + threadIdx.x) >> 5; j < n; j += nw) {
        const uint64_t o = off[j], d = cum[j] - base, len = cum[j + 1] - cum[j];
        const uint8_t *s = span + o;
        uint8_t *t = dst + d;
        if (((o | d | len) & 15u) == 0) {
            for (uint64_t v = lane; v < (len >> 4); v += 32)
                reinterpret_cast<uint4 *>(t)[v] = reinterpret_cast<const uint4 *>(s)[v];
        } else {
            for (uint64_t i = lane; i < len; i += 32) t[i] = s[i];
        }
    }
}

}  // namespace

const void *report_fn() { return reinterpret_cast<const void *>(&report_kernel); }

cudaError_t launch_report(const void *words, uint32_t n, const uint32_t *word32, void *dst, cudaStream_t s) {
    report_kernel<<<1, 32, 0, s>>>(reinterpret_cast<const uint64_t *>(words), n, word32,
                                   reinterpret_cast<uint64_t *>(dst));
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) count_launches(1);
    return e;
}

// Load the kernel now (modules load lazily on first launch, which can block
// the host): a checkpoint that returns once enqueued must not be the first.
cudaError_t prepare_drain() {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, drain_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, link_copy_kernel);
    return e != cudaSuccess ? e : cudaFuncGetAttributes(&a, report_kernel);
}

cudaError_t launch_link_copy(void *dst, const void *src, uint64_t bytes, int max_grid, cudaStream_t s) {
    if (bytes == 0) return cudaSuccess;
    // one CTA per 64 KiB, up to max_grid: a descriptor table takes one CTA,
    // a bulk drain two per SM (one per SM already paces the link)
    const uint64_t want = (bytes + (64u << 10) - 1) >> 16;
    const int grid = (int)(want < (uint64_t)max_grid ? want : (uint64_t)max_grid);
    link_copy_kernel<<<grid > 0 ? grid : 1, kDrainNT, 0, s>>>(reinterpret_cast<uint8_t *>(dst),
                                                             reinterpret_cast<const uint8_t *>(src), bytes);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) count_launches(1);
    return e;
}

cudaError_t launch_drain(const CkptCtrl *ctrl, const uint8_t *src, uint8_t *dst, uint64_t cap,
                         const uint64_t *idx_src, uint64_t *idx_dst, uint64_t idx_cap, int grid, cudaStream_t s) {
    drain_kernel<<<grid, kDrainNT, 0, s>>>(ctrl, src, dst, cap, idx_src, idx_dst, idx_cap);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) count_launches(1);
    return e;
}

cudaError_t launch_sparse_pack(void *dst, const void *span, const uint64_t *off, const uint64_t *cum, uint64_t n,
                               int grid, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    sparse_pack_kernel<<<grid, kDrainNT, 0, s>>>(reinterpret_cast<uint8_t *>(dst),
                                                 reinterpret_cast<const uint8_t *>(span), off, cum, n);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) count_launches(1);
    return e;
}

}  // namespace crac
