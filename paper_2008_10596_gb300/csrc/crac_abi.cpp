// The C ABI's context calls, the default context, status strings, managed
// allocation helpers and host-side fault injection.
#include "crac_runtime.h"

using namespace crac;

namespace crac {

thread_local int t_last_cuda = 0;
std::atomic<int> g_fault_step{CRAC_FAULT_NONE};
std::atomic<int> g_fault_count{0};
std::atomic<uint64_t> g_lineage_counter{0};

crac_status_t cuda_status(cudaError_t e) {
    t_last_cuda = (int)e;
    return e == cudaErrorMemoryAllocation ? CRAC_ERR_OOM : CRAC_ERR_CUDA;
}

bool fault_hit(int step) {
    if (g_fault_step.load() != step) return false;
    int c = g_fault_count.load();
    while (c > 0) {
        if (g_fault_count.compare_exchange_weak(c, c - 1)) {
            if (c - 1 == 0) g_fault_step.store(CRAC_FAULT_NONE);
            return true;
        }
    }
    return false;
}

void note_cuda_error(int e) { t_last_cuda = e; }

namespace {

crac_ctx *g_default = nullptr;
std::mutex g_default_mu;

}  // namespace

crac_status_t default_ctx(crac_ctx **out) {
    std::lock_guard<std::mutex> lk(g_default_mu);
    if (!g_default) {
        crac_ctx *c = new crac_ctx();
        const crac_status_t st = ctx_init(c, nullptr);
        if (st != CRAC_OK) {
            ctx_free_all(c);
            delete c;
            return st;
        }
        g_default = c;
    }
    *out = g_default;
    return CRAC_OK;
}

}  // namespace crac

extern "C" {


void crac_config_default(crac_config_t *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->struct_size = sizeof(crac_config_t);
    cfg->chunk_bytes = 65536;
    cfg->image_residency = CRAC_RESIDENCY_HOST;
    cfg->launch_mode = CRAC_LAUNCH_BATCHED;
    cfg->timeout_ns = kDefaultTimeoutNs;
    cfg->device = -1;
}

crac_status_t crac_ctx_create(const crac_config_t *cfg, crac_ctx_t **out) {
    if (!out) return CRAC_ERR_INVALID_ARG;
    *out = nullptr;
    crac_ctx *c = new crac_ctx();
    crac_status_t st = ctx_init(c, cfg);
    // A reservation is made now, so that no checkpoint pays for it.
    if (st == CRAC_OK && (c->cfg.reserve_host_bytes || c->cfg.reserve_device_bytes)) st = ctx_cuda_ready(c);
    if (st != CRAC_OK) {
        ctx_free_all(c);
        delete c;
        return st;
    }
    *out = c;
    return CRAC_OK;
}

crac_status_t crac_ctx_destroy(crac_ctx_t *ctx) {
    if (!ctx) return CRAC_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(g_default_mu);
        if (ctx == g_default) g_default = nullptr;
    }
    ctx_free_all(ctx);
    delete ctx;
    return CRAC_OK;
}

crac_status_t crac_ctx_register_alloc(crac_ctx_t *ctx, void *ptr, size_t bytes, crac_kind_t kind) {
    if (!ctx || !ptr || bytes == 0 || ((uintptr_t)ptr & 15u) ||
        (kind != CRAC_KIND_DEVICE && kind != CRAC_KIND_MANAGED && kind != CRAC_KIND_HOST))
        return CRAC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    const uint64_t p = (uint64_t)(uintptr_t)ptr;
    if (p + bytes < p) return CRAC_ERR_INVALID_ARG;
    for (const AllocRec &r : ctx->allocs)
        if (p < r.ptr + r.bytes && r.ptr < p + bytes) return CRAC_ERR_OVERLAP;
    ctx->allocs.push_back(AllocRec{ctx->next_id++, p, (uint64_t)bytes, (uint32_t)kind});
    ctx->layout_version++;
    return CRAC_OK;
}

crac_status_t crac_ctx_free(crac_ctx_t *ctx, void *ptr) {
    if (!ctx) return CRAC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    const uint64_t p = (uint64_t)(uintptr_t)ptr;
    for (size_t i = 0; i < ctx->allocs.size(); ++i) {
        if (ctx->allocs[i].ptr == p) {
            ctx->base_first.erase(ctx->allocs[i].id);
            ctx->allocs.erase(ctx->allocs.begin() + i);
            ctx->layout_version++;
            return CRAC_OK;
        }
    }
    return CRAC_ERR_UNKNOWN_PTR;
}

crac_status_t crac_ctx_checkpoint(crac_ctx_t *ctx, crac_stream_t stream, crac_image_t **image_out) {
    if (!ctx) return CRAC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    TRY(ctx_cuda_ready(ctx));
    return ctx_checkpoint(ctx, (cudaStream_t)stream, image_out);
}

crac_status_t crac_ctx_restart(crac_ctx_t *ctx, const crac_image_t *image, crac_stream_t stream) {
    if (!ctx || !image) return CRAC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    TRY(ctx_cuda_ready(ctx));
    return ctx_restart(ctx, const_cast<crac_image *>(image), (cudaStream_t)stream);
}

// Settle the context's unsettled checkpoints (their failure would revert the
// baseline these calls change or report on).
static void settle_all(crac_ctx *c) {
    if (!c->cuda_ready || c->pending.empty()) return;
    DeviceGuard g(c->device);
    ctx_settle(c, true);
}

crac_status_t crac_ctx_invalidate(crac_ctx_t *ctx) {
    if (!ctx) return CRAC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    settle_all(ctx);
    ctx->base_valid = false;
    ctx->base_first.clear();
    return CRAC_OK;
}

crac_status_t crac_ctx_drop_history(crac_ctx_t *ctx) {
    if (!ctx) return CRAC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    settle_all(ctx);
    img_unref(ctx->parent);
    ctx->parent = nullptr;
    return CRAC_OK;
}

crac_status_t crac_ctx_last_pass(crac_ctx_t *ctx, crac_pass_info_t *out) {
    if (!ctx || !out) return CRAC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    settle_all(ctx);
    *out = ctx->last;
    return CRAC_OK;
}

crac_status_t crac_ctx_last_restart(crac_ctx_t *ctx, crac_restart_info_t *out) {
    if (!ctx || !out) return CRAC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    *out = ctx->last_restart;
    return CRAC_OK;
}

crac_status_t crac_register_alloc(void *ptr, size_t bytes, crac_kind_t kind) {
    crac_ctx *c;
    TRY(default_ctx(&c));
    return crac_ctx_register_alloc(c, ptr, bytes, kind);
}

crac_status_t crac_free(void *ptr) {
    crac_ctx *c;
    TRY(default_ctx(&c));
    return crac_ctx_free(c, ptr);
}

crac_status_t crac_checkpoint(crac_stream_t stream, crac_image_t **image_out) {
    crac_ctx *c;
    TRY(default_ctx(&c));
    return crac_ctx_checkpoint(c, stream, image_out);
}

crac_status_t crac_restart(const crac_image_t *image, crac_stream_t stream) {
    crac_ctx *c;
    TRY(default_ctx(&c));
    return crac_ctx_restart(c, image, stream);
}

const char *crac_status_str(crac_status_t s) {
    switch (s) {
    case CRAC_OK: return "CRAC_OK";
    case CRAC_ERR_INVALID_ARG: return "CRAC_ERR_INVALID_ARG";
    case CRAC_ERR_UNKNOWN_PTR: return "CRAC_ERR_UNKNOWN_PTR";
    case CRAC_ERR_OVERLAP: return "CRAC_ERR_OVERLAP";
    case CRAC_ERR_CUDA: return "CRAC_ERR_CUDA";
    case CRAC_ERR_OOM: return "CRAC_ERR_OOM";
    case CRAC_ERR_IMAGE_MISMATCH: return "CRAC_ERR_IMAGE_MISMATCH";
    case CRAC_ERR_TIMEOUT: return "CRAC_ERR_TIMEOUT";
    case CRAC_ERR_BUSY: return "CRAC_ERR_BUSY";
    case CRAC_ERR_UNSUPPORTED: return "CRAC_ERR_UNSUPPORTED";
    case CRAC_ERR_CORRUPT: return "CRAC_ERR_CORRUPT";
    default: return "CRAC_ERR_UNKNOWN";
    }
}

int crac_last_cuda_error(void) { return t_last_cuda; }

uint64_t crac_kernel_launches(void) { return launches_so_far(); }

crac_status_t crac_alloc_managed(size_t bytes, void **out) {
    if (!out || !bytes) return CRAC_ERR_INVALID_ARG;
    *out = nullptr;
    CK(cudaMallocManaged(out, bytes, cudaMemAttachGlobal));
    return CRAC_OK;
}

crac_status_t crac_free_managed(void *ptr) {
    if (!ptr) return CRAC_ERR_INVALID_ARG;
    CK(cudaFree(ptr));
    return CRAC_OK;
}

void crac_debug_inject_fault(int step, int count) {
    g_fault_count.store(count > 0 ? count : 0);
    g_fault_step.store(count > 0 ? step : CRAC_FAULT_NONE);
}

}  // extern "C"
