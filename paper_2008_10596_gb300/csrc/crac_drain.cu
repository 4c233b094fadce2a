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
    const cudaError_t e = cudaFuncGetAttributes(&a, drain_kernel);
    return e != cudaSuccess ? e : cudaFuncGetAttributes(&a, report_kernel);
}

cudaError_t launch_drain(const CkptCtrl *ctrl, const uint8_t *src, uint8_t *dst, uint64_t cap,
                         const uint64_t *idx_src, uint64_t *idx_dst, uint64_t idx_cap, int grid, cudaStream_t s) {
    drain_kernel<<<grid, kDrainNT, 0, s>>>(ctrl, src, dst, cap, idx_src, idx_dst, idx_cap);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) count_launches(1);
    return e;
}

}  // namespace crac
