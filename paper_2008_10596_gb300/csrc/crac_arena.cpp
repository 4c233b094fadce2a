// Device and pinned-host arenas for image payloads, and grow-only buffers.
#include "crac_runtime.h"

#include <atomic>

using namespace crac;

namespace {

std::mutex g_arena_mu;
std::map<int, std::unique_ptr<Arena>> g_dev_arenas;
std::unique_ptr<Arena> g_pinned_arena;

}  // namespace

namespace crac {

Arena &device_arena(int dev) {
    std::lock_guard<std::mutex> lk(g_arena_mu);
    auto &a = g_dev_arenas[dev];
    if (!a) a.reset(new Arena(true, dev, 1ull << 30));
    return *a;
}

Arena &pinned_arena() {
    std::lock_guard<std::mutex> lk(g_arena_mu);
    if (!g_pinned_arena) g_pinned_arena.reset(new Arena(false, 0, 256ull << 20));
    return *g_pinned_arena;
}

std::atomic<uint32_t> g_scratch_grows{0};

crac_status_t ensure_dev(DevBuf &b, size_t bytes) {
    bytes = std::max<size_t>(bytes, 256);
    if (b.cap >= bytes) return CRAC_OK;
    if (b.borrowed) return CRAC_ERR_OOM;   // a lease cannot grow (and is not ours to free)
    if (fault_hit(CRAC_FAULT_ALLOC)) return CRAC_ERR_OOM;
    g_scratch_grows++;
    if (b.p) {
        CK(cudaDeviceSynchronize());
        CK(cudaFree(b.p));
        b = DevBuf{};
    }
    const size_t sz = round_up(bytes + bytes / 4, 1 << 20);
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, sz);
    if (e != cudaSuccess) {
        cudaGetLastError();
        e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cuda_status(e);
        }
        b.cap = bytes;
    } else {
        b.cap = sz;
    }
    b.p = p;
    return CRAC_OK;
}

crac_status_t ensure_host(HostBuf &b, size_t bytes) {
    bytes = std::max<size_t>(bytes, 256);
    if (b.cap >= bytes) return CRAC_OK;
    g_scratch_grows++;
    if (b.p) {
        CK(cudaFreeHost(b.p));
        b = HostBuf{};
    }
    const size_t sz = round_up(bytes + bytes / 4, 1 << 16);
    CK(cudaHostAlloc(&b.p, sz, cudaHostAllocPortable));
    b.cap = sz;
    return CRAC_OK;
}

}  // namespace crac

extern "C" {

crac_status_t crac_memory_stats(crac_memory_stats_t *out) {
    if (!out) return CRAC_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    pinned_arena().stats(&out->host_region_bytes, &out->host_used_bytes, &out->host_regions, &out->host_grow_events);
    std::lock_guard<std::mutex> lk(g_arena_mu);
    for (auto &kv : g_dev_arenas) {
        uint64_t t, u;
        uint32_t r, gcount;
        kv.second->stats(&t, &u, &r, &gcount);
        out->device_region_bytes += t;
        out->device_used_bytes += u;
        out->device_regions += r;
        out->device_grow_events += gcount;
    }
    out->scratch_grow_events = g_scratch_grows.load();
    return CRAC_OK;
}

}  // extern "C"
