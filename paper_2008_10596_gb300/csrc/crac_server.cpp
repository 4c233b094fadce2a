// The request server: worker threads, per-context ordering, staging
// budget leases, and its part of the C ABI.
#include "crac_runtime.h"

using namespace crac;

namespace crac {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Run an operation of `c` with a leased staging buffer in place of its own.
template <class F>
crac_status_t with_staging(crac_ctx *c, void *p, uint64_t bytes, F &&op) {
    const DevBuf saved = c->staging;
    const uint64_t saved_cfg = c->cfg.staging_bytes;
    if (p) {
        c->staging = DevBuf{p, (size_t)bytes, true};
        c->cfg.staging_bytes = bytes;
    }
    const crac_status_t st = op();
    if (p) {
        c->staging = saved;
        c->cfg.staging_bytes = saved_cfg;
    }
    return st;
}

}  // namespace crac

namespace {

struct ServerReq {
    crac_request_result_t r{};
    crac_ctx *ctx = nullptr;
    crac_image *img = nullptr;
    cudaStream_t stream = nullptr;
    crac_prepare_fn prep = nullptr;
    void *prep_arg = nullptr;
    uint64_t lease_off = 0;
};

}  // namespace

struct crac_server {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ServerReq *> queue;
    std::map<uint64_t, ServerReq *> done;
    std::map<crac_ctx *, int> busy;
    std::vector<std::thread> workers;
    bool stopping = false;
    int device = 0;
    uint64_t budget = 0, max_lease = 0, used = 0, high_water = 0;
    uint64_t next_ticket = 1, submitted = 0, completed = 0;
    uint32_t in_flight = 0, max_in_flight = 0;
    void *staging = nullptr;
    std::unique_ptr<RangeAlloc> ra;
};

namespace {

uint64_t ctx_tracked(const crac_ctx *c) {
    uint64_t t = 0;
    for (const AllocRec &a : c->allocs) t += a.bytes;
    return t;
}

void server_worker(crac_server *sv) {
    cudaSetDevice(sv->device);
    for (;;) {
        ServerReq *q = nullptr;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            for (;;) {
                if (sv->stopping && sv->queue.empty()) return;
                // first request (arrival order) whose context is idle; it must
                // fit the staging budget, otherwise everything waits behind it
                auto it = sv->queue.begin();
                while (it != sv->queue.end() && sv->busy.count((*it)->ctx)) ++it;
                if (it != sv->queue.end()) {
                    ServerReq *c = *it;
                    uint64_t off = 0;
                    const uint64_t want = c->r.lease_bytes;
                    if (want == 0 || sv->ra->alloc(want, &off)) {
                        c->lease_off = off;
                        sv->used += want;
                        sv->high_water = std::max(sv->high_water, sv->used);
                        sv->busy[c->ctx] = 1;
                        sv->queue.erase(it);
                        sv->in_flight++;
                        sv->max_in_flight = std::max(sv->max_in_flight, sv->in_flight);
                        q = c;
                        break;
                    }
                }
                sv->cv_work.wait(lk);
            }
        }
        q->r.t_admit = now_s();
        void *lease = q->r.lease_bytes ? (uint8_t *)sv->staging + q->lease_off : nullptr;
        if (q->prep) q->prep((crac_stream_t)q->stream, q->prep_arg);
        q->r.t_op = now_s();
        crac_status_t st;
        {
            std::lock_guard<std::mutex> lk(q->ctx->mu);
            st = ctx_cuda_ready(q->ctx);
            if (st == CRAC_OK) {
                if (q->r.type == CRAC_REQ_CHECKPOINT) {
                    crac_image *img = nullptr;
                    st = with_staging(q->ctx, lease, q->r.lease_bytes,
                                      [&] { return ctx_checkpoint(q->ctx, q->stream, &img); });
                    if (st == CRAC_OK) q->r.image = img;
                } else {
                    st = with_staging(q->ctx, lease, q->r.lease_bytes,
                                      [&] { return ctx_restart(q->ctx, q->img, q->stream); });
                    if (st == CRAC_OK) q->r.payload_bytes = q->img->payload_bytes;
                }
            }
        }
        q->r.t_op_end = now_s();
        // The lease is free once the drain has finished reading it; the
        // image's sizes are known then.
        if (st == CRAC_OK && q->r.image) st = img_wait(q->r.image, 0);
        if (st == CRAC_OK && q->r.image) q->r.payload_bytes = q->r.image->payload_bytes;
        q->r.status = st;
        q->r.t_done = now_s();
        if (q->img) {
            img_unref(q->img);
            q->img = nullptr;
        }
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            if (q->r.lease_bytes) {
                sv->ra->release(q->lease_off, q->r.lease_bytes);
                sv->used -= q->r.lease_bytes;
            }
            sv->busy.erase(q->ctx);
            sv->in_flight--;
            sv->completed++;
            sv->done[q->r.ticket] = q;
        }
        sv->cv_work.notify_all();
        sv->cv_done.notify_all();
    }
}

}  // namespace

extern "C" {

double crac_time_now(void) { return now_s(); }

crac_status_t crac_server_create(const crac_server_config_t *cfg, crac_server_t **out) {
    if (!out) return CRAC_ERR_INVALID_ARG;
    *out = nullptr;
    crac_server_config_t c{};
    if (cfg) c = *cfg;
    std::unique_ptr<crac_server> sv(new crac_server());
    const uint32_t workers = c.workers ? c.workers : 4;
    sv->budget = round_up(c.staging_budget ? c.staging_budget : (24ull << 30), 256);
    sv->max_lease = round_up(c.max_lease ? c.max_lease : (4ull << 30), 256);
    if (sv->max_lease > sv->budget) sv->max_lease = sv->budget;
    int dev = c.device;
    if (dev < 0) CK(cudaGetDevice(&dev));
    sv->device = dev;
    {
        DeviceGuard g(dev);
        if (fault_hit(CRAC_FAULT_ALLOC)) return CRAC_ERR_OOM;
        const cudaError_t e = cudaMalloc(&sv->staging, sv->budget);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cuda_status(e);
        }
    }
    sv->ra.reset(new RangeAlloc(sv->budget));
    for (uint32_t i = 0; i < workers; ++i) sv->workers.emplace_back(server_worker, sv.get());
    *out = sv.release();
    return CRAC_OK;
}

crac_status_t crac_server_destroy(crac_server_t *sv) {
    if (!sv) return CRAC_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stopping = true;
    }
    sv->cv_work.notify_all();
    for (std::thread &t : sv->workers) t.join();
    for (auto &kv : sv->done) {
        if (kv.second->r.image) img_unref(kv.second->r.image);
        delete kv.second;
    }
    {
        DeviceGuard g(sv->device);
        cudaFree(sv->staging);
        cudaGetLastError();
    }
    delete sv;
    return CRAC_OK;
}

crac_status_t crac_server_submit(crac_server_t *sv, crac_ctx_t *ctx, uint32_t type, const crac_image_t *image,
                                 crac_stream_t stream, crac_prepare_fn prepare, void *prepare_arg, double t_arrival,
                                 uint64_t *ticket) {
    if (!sv || !ctx || !ticket || type > CRAC_REQ_RESTART || (type == CRAC_REQ_RESTART && !image))
        return CRAC_ERR_INVALID_ARG;
    ServerReq *q = new ServerReq();
    q->ctx = ctx;
    q->img = const_cast<crac_image *>(image);
    q->stream = (cudaStream_t)stream;
    q->prep = prepare;
    q->prep_arg = prepare_arg;
    q->r.type = type;
    q->r.t_arrival = t_arrival > 0 ? t_arrival : now_s();
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        q->r.tracked_bytes = ctx_tracked(ctx);
        const uint64_t S = 1ull << ctx->log2S;
        uint64_t lease = 0;
        if (type == CRAC_REQ_CHECKPOINT && ctx->cfg.image_residency == CRAC_RESIDENCY_HOST)
            lease = q->r.tracked_bytes;
        if (type == CRAC_REQ_RESTART && image->residency == CRAC_RESIDENCY_HOST) lease = q->r.tracked_bytes;
        if (lease) lease = std::max(round_up(std::min(lease, sv->max_lease), 256), round_up(S, 256));
        // coded images: a segment leaves 256 bytes of the lease for the
        // encoder's aligned reads, so the lease holds at least a chunk more
        if (lease && (ctx->cfg.flags & CRAC_FLAG_COMPRESS)) lease = std::max(lease, round_up(S, 256) + 256);
        if (lease > sv->budget) {
            delete q;
            return CRAC_ERR_INVALID_ARG;
        }
        q->r.lease_bytes = lease;
    }
    if (q->img) img_ref(q->img);   // kept alive until the request completes
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->stopping) {
            img_unref(q->img);
            delete q;
            return CRAC_ERR_BUSY;
        }
        q->r.ticket = sv->next_ticket++;
        sv->submitted++;
        sv->queue.push_back(q);
        *ticket = q->r.ticket;
    }
    sv->cv_work.notify_all();
    return CRAC_OK;
}

crac_status_t crac_server_wait(crac_server_t *sv, uint64_t ticket, uint64_t timeout_ns, crac_request_result_t *out) {
    if (!sv || !out) return CRAC_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(sv->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::nanoseconds(timeout_ns);
    for (;;) {
        auto it = sv->done.find(ticket);
        if (it != sv->done.end()) {
            *out = it->second->r;
            delete it->second;
            sv->done.erase(it);
            return CRAC_OK;
        }
        if (ticket == 0 || ticket >= sv->next_ticket) return CRAC_ERR_INVALID_ARG;
        if (timeout_ns) {
            if (sv->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) return CRAC_ERR_TIMEOUT;
        } else {
            sv->cv_done.wait(lk);
        }
    }
}

crac_status_t crac_server_stats(crac_server_t *sv, crac_server_stats_t *out) {
    if (!sv || !out) return CRAC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(sv->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = sv->submitted;
    out->completed = sv->completed;
    out->queued = (uint32_t)sv->queue.size();
    out->in_flight = sv->in_flight;
    out->max_in_flight = sv->max_in_flight;
    out->staging_used = sv->used;
    out->staging_high_water = sv->high_water;
    out->staging_budget = sv->budget;
    return CRAC_OK;
}

}  // extern "C"
