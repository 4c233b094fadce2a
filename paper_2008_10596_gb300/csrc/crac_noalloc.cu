#include "crac_device.cuh"

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
