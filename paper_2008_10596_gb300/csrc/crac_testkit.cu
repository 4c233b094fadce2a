// Workload mutators for tests and benchmarks (built as libcrac_testkit.so,
// separate from libcrac.so).  They play the role of the application that
// rewrites part of its memory between two checkpoints; nothing here is part
// of the checkpoint/restart data pass.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

struct MutEntry {
    uint64_t ptr;    // device address of the chunk
    uint64_t len;    // bytes
    uint32_t mask;   // XOR mask for every uint32 word; tail bytes use its low bytes in order
    uint32_t pad;
};

// One warp per entry: XOR every whole uint32 with the mask and each byte of
// a trailing partial word with mask byte (offset % 4).
__global__ void mutate_xor_kernel(const MutEntry *__restrict__ e, uint32_t n) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (uint64_t i = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp; i < n;
         i += (uint64_t)gridDim.x * (blockDim.x >> 5)) {
        const MutEntry m = e[i];
        uint8_t *p = reinterpret_cast<uint8_t *>(m.ptr);
        const uint64_t nw = m.len >> 2;
        if ((m.ptr & 15u) == 0) {
            const uint64_t nv = nw >> 2;
            uint4 *v = reinterpret_cast<uint4 *>(p);
            for (uint64_t j = lane; j < nv; j += 32) {
                uint4 q = v[j];
                q.x ^= m.mask;
                q.y ^= m.mask;
                q.z ^= m.mask;
                q.w ^= m.mask;
                v[j] = q;
            }
            uint32_t *w = reinterpret_cast<uint32_t *>(p);
            for (uint64_t j = nv * 4 + lane; j < nw; j += 32) w[j] ^= m.mask;
        } else {
            for (uint64_t j = lane; j < nw; j += 32) {
                uint32_t *w = reinterpret_cast<uint32_t *>(p + 4 * j);
                *w ^= m.mask;
            }
        }
        for (uint64_t b = nw * 4 + lane; b < m.len; b += 32) p[b] ^= (uint8_t)(m.mask >> (8 * (b & 3)));
    }
}

// Page rewrite: copy `len` bytes from a source pool (e.g. random bf16 values)
// over each page; one warp per entry.
struct CopyEntry {
    uint64_t dst, src, len;
};

__global__ void rewrite_kernel(const CopyEntry *__restrict__ e, uint32_t n) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (uint64_t i = (uint64_t)blockIdx.x * (blockDim.x >> 5) + warp; i < n;
         i += (uint64_t)gridDim.x * (blockDim.x >> 5)) {
        const CopyEntry c = e[i];
        if (((c.dst | c.src | c.len) & 15u) == 0) {
            uint4 *d = reinterpret_cast<uint4 *>(c.dst);
            const uint4 *s = reinterpret_cast<const uint4 *>(c.src);
            for (uint64_t j = lane; j < (c.len >> 4); j += 32) d[j] = s[j];
        } else {
            uint8_t *d = reinterpret_cast<uint8_t *>(c.dst);
            const uint8_t *s = reinterpret_cast<const uint8_t *>(c.src);
            for (uint64_t j = lane; j < c.len; j += 32) d[j] = s[j];
        }
    }
}

// Application work that keeps a stream busy for `ns` nanoseconds of the
// device clock (one thread; the loop also stops after 2^31 iterations).
__global__ void delay_kernel(uint64_t ns) {
    uint64_t t0, t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (uint32_t i = 0; i < (1u << 31); ++i) {
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 >= ns) break;
    }
}

}  // namespace

extern "C" __attribute__((visibility("default"))) int crac_testkit_delay(uint64_t ns, void *stream) {
    if (ns > 10000000000ull) return (int)cudaErrorInvalidValue;   // at most 10 s
    delay_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(ns);
    return (int)cudaGetLastError();
}

extern "C" __attribute__((visibility("default"))) int crac_testkit_mutate_xor(const void *entries_dev,
                                                                               uint32_t n, void *stream) {
    if (n == 0) return 0;
    const uint32_t grid = (n + 7) / 8 < 4096 ? (n + 7) / 8 : 4096;
    mutate_xor_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>((const MutEntry *)entries_dev, n);
    return (int)cudaGetLastError();
}

extern "C" __attribute__((visibility("default"))) int crac_testkit_rewrite(const void *entries_dev, uint32_t n,
                                                                            void *stream) {
    if (n == 0) return 0;
    const uint32_t grid = (n + 7) / 8 < 4096 ? (n + 7) / 8 : 4096;
    rewrite_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>((const CopyEntry *)entries_dev, n);
    return (int)cudaGetLastError();
}
