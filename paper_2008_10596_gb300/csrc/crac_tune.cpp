// The autotuner: shadow contexts per candidate chunk size, observation
// rounds, and the choice of chunk size, pass kernel and LDG tile.
#include "crac_runtime.h"

using namespace crac;

namespace crac {

void tune_clear(crac_ctx *c) {
    for (crac_ctx *t : c->tune_ctx) {
        ctx_free_all(t);
        delete t;
    }
    c->tune_ctx.clear();
    c->tune_sum_ms.clear();
    c->tune_sum_bytes.clear();
    c->tune_last_ms.clear();
    c->tune_last_bytes.clear();
    c->tune_rounds = 0;
}

void tune_fill(const crac_ctx *c, crac_tune_result_t *out) {
    if (!out) return;
    std::memset(out, 0, sizeof(*out));
    out->n = (uint32_t)c->tune_ctx.size();
    out->rounds = c->tune_rounds;
    for (size_t i = 0; i < c->tune_ctx.size(); ++i) {
        out->chunk_bytes[i] = 1u << c->tune_ctx[i]->log2S;
        out->last_pass_ms[i] = c->tune_last_ms[i];
        out->last_dirty_bytes[i] = c->tune_last_bytes[i];
        if (c->tune_rounds) {
            out->mean_pass_ms[i] = (float)(c->tune_sum_ms[i] / c->tune_rounds);
            out->mean_dirty_bytes[i] = c->tune_sum_bytes[i] / c->tune_rounds;
        }
    }
}

crac_status_t ctx_tune_observe(crac_ctx *c, cudaStream_t s, const uint32_t *sizes, uint32_t n,
                               crac_tune_result_t *out) {
    if (!sizes || n == 0 || n > CRAC_TUNE_MAX) return CRAC_ERR_INVALID_ARG;
    TRY(ctx_settle(c, true));
    bool same = c->tune_ctx.size() == n;
    for (uint32_t i = 0; same && i < n; ++i) same = (1u << c->tune_ctx[i]->log2S) == sizes[i];
    if (!same) {
        tune_clear(c);
        for (uint32_t i = 0; i < n; ++i) {
            crac_config_t cfg = c->cfg;
            cfg.chunk_bytes = sizes[i];
            cfg.device = c->device;
            cfg.reserve_host_bytes = cfg.reserve_device_bytes = 0;
            if (c->cpt_tuned) cfg.chunks_per_tile = 0;
            if (cfg.pass_kernel == CRAC_PASS_TMA && (sizes[i] < 1024 || sizes[i] > 65536)) cfg.pass_kernel = CRAC_PASS_AUTO;
            crac_ctx *t = new crac_ctx();
            const crac_status_t st = ctx_init(t, &cfg);
            if (st != CRAC_OK) {
                ctx_free_all(t);
                delete t;
                tune_clear(c);
                return st;
            }
            c->tune_ctx.push_back(t);
        }
        c->tune_sum_ms.assign(n, 0.0);
        c->tune_sum_bytes.assign(n, 0.0);
        c->tune_last_ms.assign(n, 0.f);
        c->tune_last_bytes.assign(n, 0);
        c->tune_rounds = 0;
    }
    bool counted = true;
    for (uint32_t i = 0; i < n; ++i) {
        crac_ctx *t = c->tune_ctx[i];
        const bool had_base = t->base_valid;
        counted = counted && had_base;
        t->allocs = c->allocs;
        float ms = 0;
        uint64_t k = 0, d = 0;
        TRY(ctx_trial_pass(t, s, true, &ms, &k, &d));
        c->tune_last_ms[i] = ms;
        c->tune_last_bytes[i] = d;
        if (had_base) {
            c->tune_sum_ms[i] += ms;
            c->tune_sum_bytes[i] += (double)d;
        }
    }
    if (counted) c->tune_rounds++;
    tune_fill(c, out);
    return CRAC_OK;
}

// Pass kernels (and LDG tiles) timed on one candidate chunk size.
struct VariantTiming {
    float vms[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // best time per CRAC_PASS_*; 0 = not applicable
    uint32_t best_v = CRAC_PASS_SPLIT;
    uint32_t tiles[3] = {0, 0, 0};
    float tile_ms[3] = {0, 0, 0};
    uint32_t best_tile = 0;        // LDG tile of the best LDG time (0 = configured)
};

// Time every pass kernel on the shadow context `t`, each against the
// baseline before its last observation (still in the other fingerprint
// buffer), so that they see the last round's dirty set rather than an
// unchanged memory.  With chunks_per_tile unset, LDG is timed at half, equal
// to and twice its default tile.
crac_status_t time_variants(crac_ctx *t, cudaStream_t s, VariantTiming *vt) {
    const uint32_t S = 1u << t->log2S;
    if (t->prev_base_valid) {
        t->fp_cur = t->prev_fp;
        t->base_first = t->prev_base_first;
        t->base_valid = true;
        t->prev_base_valid = false;
    }
    const uint32_t saved = t->cfg.pass_kernel, saved_cpt = t->cfg.chunks_per_tile;
    vt->tiles[0] = saved_cpt;
    if (saved_cpt == 0) {
        int w;
        uint32_t t0;
        pick_split(t, &w, &t0);
        const uint32_t lo = std::max<uint32_t>(1, t0 / 2), hi = std::min<uint32_t>(256, 2 * t0);
        vt->tiles[0] = t0;
        vt->tiles[1] = lo != t0 ? lo : 0;
        vt->tiles[2] = hi != t0 ? hi : 0;
    }
    uint64_t k_seen = 0;   // dirty chunks of the timed passes (all see the same dirty set)
    auto time_pass = [&](float *best_ms) {
        for (int r = 0; r < 2; ++r) {
            float ms = 0;
            uint64_t k = 0, d = 0;
            TRY(ctx_trial_pass(t, s, false, &ms, &k, &d));
            k_seen = k;
            if (r == 0 || ms < *best_ms) *best_ms = ms;
        }
        return CRAC_OK;
    };
    uint64_t n_chunks = 0;
    for (const AllocRec &r : t->allocs) n_chunks += (r.bytes + S - 1) / S;
    for (uint32_t v : {(uint32_t)CRAC_PASS_SPLIT, (uint32_t)CRAC_PASS_LDG, (uint32_t)CRAC_PASS_TMA,
                       (uint32_t)CRAC_PASS_SPARSE}) {
        if (v == CRAC_PASS_TMA && (S < 1024 || S > 65536)) continue;
        if (v == CRAC_PASS_SPARSE && t->cfg.image_residency != CRAC_RESIDENCY_DEVICE) continue;
        if (v == CRAC_PASS_SPARSE && (t->cfg.flags & CRAC_FLAG_COMPRESS)) continue;   // needs a compact payload
        // A sparse image holds every tracked byte's room whatever the dirty
        // bytes, so it is timed only where at least 40% of the chunks are
        // dirty (at most 2.5 times the room of a compact image; the split
        // pass, timed first, gives the count), or, on chunks of 512 B -
        // 4 KiB, where under a quarter are: its passes then place the dirty
        // chunks densely, as the context's passes will after such a delta.
        const bool dense = S < 8192 && 4 * k_seen < n_chunks;
        if (v == CRAC_PASS_SPARSE && !dense && 5 * k_seen < 2 * n_chunks) continue;
        t->dense_hint = v == CRAC_PASS_SPARSE && dense;
        // Coded images on chunks of 8 KiB and more: only the split pass makes
        // the block headers that the two-launch encoder needs; a read-once
        // pass saves less in the pass than the one-launch encoder costs.
        if (v != CRAC_PASS_SPLIT && (t->cfg.flags & CRAC_FLAG_COMPRESS) && S >= 8192) continue;
        t->cfg.pass_kernel = v;
        float bestm = 0;
        const bool ldg_tiles = v == CRAC_PASS_LDG && saved_cpt == 0;
        for (int j = 0; j < (ldg_tiles ? 3 : 1); ++j) {
            if (ldg_tiles) {
                if (!vt->tiles[j]) continue;
                t->cfg.chunks_per_tile = vt->tiles[j];
            }
            float ms = 0;
            const crac_status_t st = time_pass(&ms);
            t->cfg.chunks_per_tile = saved_cpt;
            if (st != CRAC_OK) {
                t->cfg.pass_kernel = saved;
                t->dense_hint = false;
                return st;
            }
            if (v == CRAC_PASS_LDG) vt->tile_ms[j] = ms;
            if (bestm == 0 || ms < bestm) {
                bestm = ms;
                if (ldg_tiles) vt->best_tile = vt->tiles[j];
            }
        }
        t->dense_hint = false;
        vt->vms[v] = bestm;
        if (vt->vms[vt->best_v] == 0 || bestm < vt->vms[vt->best_v]) vt->best_v = v;
    }
    t->cfg.pass_kernel = saved;
    if (vt->best_v != CRAC_PASS_LDG) vt->best_tile = 0;
    return CRAC_OK;
}

crac_status_t ctx_tune_apply(crac_ctx *c, cudaStream_t s, double link_gbs, crac_tune_result_t *out) {
    if (c->tune_ctx.empty() || c->tune_rounds == 0) return CRAC_ERR_UNSUPPORTED;
    TRY(ctx_settle(c, true));
    const uint32_t n = (uint32_t)c->tune_ctx.size();
    std::vector<float> cost(n), drain(n);
    uint32_t best = 0;
    for (uint32_t i = 0; i < n; ++i) {
        const double ms = c->tune_sum_ms[i] / c->tune_rounds;
        const double bytes = c->tune_sum_bytes[i] / c->tune_rounds;
        drain[i] = (float)(link_gbs > 0 ? bytes / (link_gbs * 1e9) * 1e3 : 0.0);
        cost[i] = (float)ms + drain[i];
        if (cost[i] < cost[best]) best = i;
    }
    // The observations ran one pass kernel; sizes that come close under it
    // may differ once every kernel is tried (a fused kernel is fastest where
    // most chunks are dirty, at the sizes it supports), so every size within
    // 5% of the lowest cost has its kernels timed, and the lowest pass +
    // drain time wins.
    uint32_t win = best;
    VariantTiming win_vt;
    float win_total = 0;
    bool have = false;
    for (uint32_t i = 0; i < n; ++i) {
        if (cost[i] > cost[best] * 1.05f) continue;
        VariantTiming vt;
        TRY(time_variants(c->tune_ctx[i], s, &vt));
        const float total = vt.vms[vt.best_v] + drain[i];
        if (!have || total < win_total) {
            win = i;
            win_vt = vt;
            win_total = total;
            have = true;
        }
    }
    crac_ctx *t = c->tune_ctx[win];
    const uint32_t S = 1u << t->log2S;
    const uint32_t saved_cpt = t->cfg.chunks_per_tile;
    tune_fill(c, out);
    if (out) {
        for (uint32_t i = 0; i < n; ++i) out->cost_ms[i] = cost[i];
        for (int v = 0; v < 8; ++v) out->variant_ms[v] = win_vt.vms[v];
        out->chosen_chunk_bytes = S;
        out->chosen_pass_kernel = win_vt.best_v;
        out->chosen_chunks_per_tile = win_vt.best_tile;
        for (int j = 0; j < 3; ++j) {
            out->ldg_tiles[j] = win_vt.vms[CRAC_PASS_LDG] > 0 ? win_vt.tiles[j] : 0;
            out->ldg_tile_ms[j] = out->ldg_tiles[j] ? win_vt.tile_ms[j] : 0.f;
        }
    }
    if (saved_cpt == 0) {
        c->cfg.chunks_per_tile = win_vt.best_tile;
        c->cpt_tuned = win_vt.best_tile != 0;
    }
    if (S != (1u << c->log2S)) {
        c->cfg.chunk_bytes = S;
        c->log2S = t->log2S;
        c->layout_version++;
        c->base_valid = false;
        c->base_first.clear();
    }
    c->cfg.pass_kernel = win_vt.best_v;
    tune_clear(c);
    return CRAC_OK;
}

}  // namespace crac

extern "C" {

crac_status_t crac_ctx_tune_observe(crac_ctx_t *ctx, crac_stream_t stream, const uint32_t *chunk_sizes,
                                    uint32_t n, crac_tune_result_t *out) {
    if (!ctx) return CRAC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    TRY(ctx_cuda_ready(ctx));
    return ctx_tune_observe(ctx, (cudaStream_t)stream, chunk_sizes, n, out);
}

crac_status_t crac_ctx_tune_apply(crac_ctx_t *ctx, crac_stream_t stream, double link_gbs, crac_tune_result_t *out) {
    if (!ctx) return CRAC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    TRY(ctx_cuda_ready(ctx));
    return ctx_tune_apply(ctx, (cudaStream_t)stream, link_gbs, out);
}

}  // extern "C"
