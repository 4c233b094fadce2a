// Restart: chain resolution (R3), payload to the device (R1), scatter (R2).
#include "crac_runtime.h"

using namespace crac;

namespace crac {

// After a successful restore: the registry takes the image's identities and
// its fingerprints (already in fp[fp_cur]) become the baseline.
void restart_commit(crac_ctx *c, crac_image *img) {
    c->base_first.clear();
    for (size_t a = 0; a < img->allocs.size(); ++a) {
        c->allocs[a].id = img->allocs[a].id;
        c->next_id = std::max(c->next_id, img->allocs[a].id + 1);
        c->base_first[img->allocs[a].id] = img->allocs[a].first_chunk;
    }
    c->base_valid = true;
    c->lineage = img->lineage;
    c->epoch_max = std::max(c->epoch_max, img->epoch);
    c->parent_epoch = img->epoch;
    img_ref(img);
    img_unref(c->parent);
    c->parent = img;
}

// Image allocation -> target allocation (-1: not restored), by allocation id.
std::vector<int64_t> map_allocs(const crac_image *im, const crac_image *tgt,
                                const std::unordered_map<uint64_t, size_t> &tpos) {
    std::vector<int64_t> m(im->allocs.size());
    for (size_t a = 0; a < im->allocs.size(); ++a) {
        auto it = tpos.find(im->allocs[a].id);
        m[a] = (it == tpos.end() || tgt->allocs[it->second].bytes != im->allocs[a].bytes) ? -1 : (int64_t)it->second;
    }
    return m;
}

// Offset of every entry's bytes inside its piece's payload, for a host image
// (its payload is compact: the prefix of the entries' chunk lengths, or of a
// coded image's 16-byte padded stream lengths).  Made once per image, in
// pinned memory that the restore kernels read in place.
crac_status_t img_offsets(crac_image *im) {
    std::lock_guard<std::mutex> lk(im->mu);
    if (im->off_h.p || im->k == 0) return CRAC_OK;
    Arena &pa = pinned_arena();
    TRY(pa.alloc(im->k * 8, &im->off_h));
    uint64_t *off = (uint64_t *)im->off_h.p;
    const uint64_t *idx = (const uint64_t *)im->idx_h.p;
    const uint32_t log2S = log2u(im->chunk_bytes);
    const uint64_t *zlen = (im->flags & CRAC_IMAGE_CODED) ? (const uint64_t *)im->zlen_h.p : nullptr;
    size_t a = 0;
    for (const Piece &pc : im->pieces) {
        uint64_t acc = 0;
        for (uint64_t j = pc.k0; j < pc.k0 + pc.k; ++j) {
            while (a + 1 < im->allocs.size() && im->allocs[a + 1].first_chunk <= idx[j]) ++a;
            off[j] = acc;
            acc += zlen ? round_up(zlen[j], 16) : chunk_len(im->allocs[a].bytes, idx[j] - im->allocs[a].first_chunk, log2S);
        }
        if (acc != pc.bytes) {
            pa.free(im->off_h);
            return CRAC_ERR_CORRUPT;
        }
    }
    return CRAC_OK;
}

// Scratch of a device-side restore of nt target chunks from a chain with
// `descs` allocation entries and `pieces` pieces in all (owner map, scatter
// descriptors and their pinned copy, error word).  Checkpoints size it for
// a chain of a few images ahead of time, so that a restart allocates
// nothing (allocating may synchronize the device, which a request server
// would feel as a latency spike).
crac_status_t reserve_restart(crac_ctx *c, uint64_t nt, size_t descs, size_t pieces) {
    const size_t bytes = round_up(descs * sizeof(ScatterDesc), 256) +
                         round_up(std::max<size_t>(pieces, 1) * sizeof(RestorePiece), 256);
    TRY(ensure_dev(c->owner, std::max<uint64_t>(nt, 1) * 4));
    TRY(ensure_dev(c->sdesc, bytes));
    TRY(ensure_host(c->sdesc_h, bytes));
    TRY(ensure_dev(c->serr, 256));
    return CRAC_OK;
}

// Restore a chain on the device, resolved in three launches over every
// piece of every image of the chain: owner marks (the newest image wins), a
// coverage check, owner-filtered scatter -- no host round trip before them.
// A device image's tables and payload are in device memory; a host image's
// are read in place from pinned memory, which the device addresses directly
// (unified addressing), so of a host image only the chunks it still owns
// cross the host link.  An uncovered chunk stops the scatter (memory
// untouched) and reports IMAGE_MISMATCH.
crac_status_t restart_device(crac_ctx *c, crac_image *img, const std::vector<crac_image *> &chain, cudaStream_t s) {
    DeviceGuard g(c->device);
    for (crac_image *im : chain) {
        if (im->residency == CRAC_RESIDENCY_DEVICE) continue;
        TRY(img_wait(im, 0));   // the offsets are computed from its chunk list
        TRY(img_offsets(im));
    }
    const uint64_t nt = img->n_chunks;
    std::unordered_map<uint64_t, size_t> tpos;
    for (size_t a = 0; a < img->allocs.size(); ++a) tpos[img->allocs[a].id] = a;
    if (fault_hit(CRAC_FAULT_H2D)) {
        t_last_cuda = (int)cudaErrorLaunchFailure;
        return CRAC_ERR_CUDA;
    }
    if (!s) CK(cudaDeviceSynchronize());
    size_t total_desc = 0, n_pieces = 0;
    for (crac_image *im : chain) {
        total_desc += im->allocs.size();
        for (const Piece &pc : im->pieces) n_pieces += pc.k ? 1 : 0;
    }
    const size_t desc_bytes = round_up(total_desc * sizeof(ScatterDesc), 256);
    TRY(reserve_restart(c, nt, total_desc, n_pieces));
    const int spare = spare_fp(c);
    TRY(ensure_dev(c->fp[spare], std::max<uint64_t>(nt, 1) * 8));
    if (c->ev_last) CK(cudaEventSynchronize(c->ev_last));   // pinned descriptor scratch reuse
    ScatterDesc *sdh = (ScatterDesc *)c->sdesc_h.p;
    RestorePiece *rph = (RestorePiece *)((uint8_t *)c->sdesc_h.p + desc_bytes);
    size_t dpos = 0, ppos = 0;
    uint64_t entries = 0;
    for (size_t i = 0; i < chain.size(); ++i) {
        const crac_image *im = chain[i];
        const std::vector<int64_t> m = map_allocs(im, img, tpos);
        const size_t d0 = dpos;
        for (size_t a = 0; a < im->allocs.size(); ++a, ++dpos)
            sdh[dpos] = ScatterDesc{im->allocs[a].first_chunk, im->allocs[a].bytes,
                                    m[a] < 0 ? 0 : img->allocs[m[a]].first_chunk, m[a] < 0 ? 0 : c->allocs[m[a]].ptr,
                                    0, {0, 0, 0}};
        const bool host = im->residency != CRAC_RESIDENCY_DEVICE;
        const bool coded = (im->flags & CRAC_IMAGE_CODED) != 0;
        for (const Piece &pc : im->pieces) {
            if (!pc.k) continue;
            if (host)
                rph[ppos++] = RestorePiece{(uint64_t)(im->idx_h.p + pc.k0 * 8), (uint64_t)(im->off_h.p + pc.k0 * 8),
                                           (uint64_t)pc.host.p, pc.k, entries, pc.bytes, (uint32_t)i, (uint32_t)d0,
                                           (uint32_t)im->allocs.size(), 0,
                                           coded ? (uint64_t)(im->zlen_h.p + pc.k0 * 8) : 0ull};
            else
                rph[ppos++] = RestorePiece{(uint64_t)pc.idx_dev.p, (uint64_t)pc.off_dev.p, (uint64_t)pc.dev.p, pc.k,
                                           entries, pc.span ? pc.span : pc.bytes, (uint32_t)i, (uint32_t)d0,
                                           (uint32_t)im->allocs.size(), 0, coded ? (uint64_t)pc.zlen_dev.p : 0ull};
            entries += pc.k;
        }
    }
    for (crac_image *im : chain)   // deserialized images have no event: complete from the start
        if (im->done) CK(cudaStreamWaitEvent(s, im->done, 0));
    CK(cudaStreamWaitEvent(s, c->ev_last, 0));
    CK(cudaMemsetAsync(c->serr.p, 0, 256, s));
    if (nt) CK(cudaMemsetAsync(c->owner.p, 0, nt * 4, s));
    CK(link_copy(c, c->sdesc.p, c->sdesc_h.p, desc_bytes + ppos * sizeof(RestorePiece), cudaMemcpyHostToDevice, s));
    crac_restart_info_t ri{};
    ri.chain_length = ri.images_used = (uint32_t)chain.size();
    for (const ImgAlloc &a : img->allocs) ri.restored_bytes += a.bytes;
    ri.entries_scanned = entries;
    ri.scatter_launches = entries ? 1 : 0;
    RestoreParams P{};
    P.pieces = (const RestorePiece *)((uint8_t *)c->sdesc.p + desc_bytes);
    P.n_pieces = (uint32_t)ppos;
    P.log2_chunk = c->log2S;
    P.n_entries = entries;
    P.desc = (const ScatterDesc *)c->sdesc.p;
    P.owner = (uint32_t *)c->owner.p;
    P.n_owner = nt;
    P.err = (unsigned int *)c->serr.p;
    for (const crac_image *im : chain) P.coded |= (im->flags & CRAC_IMAGE_CODED) ? 1u : 0u;
    // Reads of host images are paced by the host link, which one CTA per SM
    // already saturates (4 KiB in flight per warp); a bigger grid would only
    // keep SMs from other streams' work for the length of the transfer.
    // Decoding coded images is compute-heavy: four CTAs per SM (the coded
    // scatter's occupancy) keep the link busy while they decode.
    bool any_host = false;
    for (const crac_image *im : chain) any_host = any_host || im->residency != CRAC_RESIDENCY_DEVICE;
    const uint64_t grid = (uint64_t)c->sm_count * (any_host ? (P.coded ? 4 : 1) : 8);
    // Incremental: fingerprint the current contents against the target's
    // table first; chunks that match are then left alone.
    const bool incremental = (c->cfg.flags & CRAC_FLAG_INCREMENTAL_RESTORE) && nt > 0;
    const uint64_t *fp_img = img->residency == CRAC_RESIDENCY_DEVICE ? (const uint64_t *)img->fp_dev.p
                                                                      : (const uint64_t *)img->fp_h.p;
    const CkptCtrl *vctrl = nullptr;
    CK(cudaEventRecord(c->ev_r0, s));
    if (incremental) TRY(fingerprint_against(c, fp_img, s, &P.fp_now, &vctrl));
    P.fp_img = fp_img;
    CK(launch_restore_mark(P, (int)std::max<uint64_t>(1, std::min<uint64_t>((entries + 255) / 256, grid)), s));
    CK(launch_restore_check(P, (int)std::max<uint64_t>(1, std::min<uint64_t>((nt + 255) / 256, grid)), s));
    if (incremental)
        CK(launch_restore_unmark(P, (int)std::max<uint64_t>(1, std::min<uint64_t>((nt + 255) / 256, grid)), s));
    CK(launch_restore_scatter(P, (int)std::max<uint64_t>(1, std::min<uint64_t>((entries + 7) / 8, grid)), s));
    CK(cudaEventRecord(c->ev_r1, s));
    if (incremental) CK(launch_report(vctrl, sizeof(CkptCtrl) / 8, nullptr, c->ctrl_h.p, s));
    if (nt) {
        const void *fp = img->residency == CRAC_RESIDENCY_DEVICE ? (const void *)img->fp_dev.p : (const void *)img->fp_h.p;
        CK(link_copy(c, c->fp[spare].p, fp, nt * 8, cudaMemcpyDefault, s));
    }
    CK(launch_report(nullptr, 0, (const uint32_t *)c->serr.p, c->serr_h.p, s));
    CK(cudaEventRecord(c->ev_last, s));
    CK(cudaEventSynchronize(c->ev_last));
    const unsigned err = *(const unsigned *)c->serr_h.p;
    if (err & kErrUncovered) return CRAC_ERR_IMAGE_MISMATCH;
    if (err) return CRAC_ERR_CORRUPT;
    cudaEventElapsedTime(&ri.device_ms, c->ev_r0, c->ev_r1);
    ri.chunks_rewritten = nt;
    if (incremental) {
        // The fingerprints the unmark used are written before the pass's
        // look-back, so the restore is right even if the counts are not.
        const CkptCtrl *vc = (const CkptCtrl *)c->ctrl_h.p;
        if (vc->err == 0) {
            ri.chunks_rewritten = vc->k;
            ri.restored_bytes = vc->D;
        }
    }
    c->last_restart = ri;
    c->fp_cur = spare;
    restart_commit(c, img);
    return CRAC_OK;
}

crac_status_t ctx_restart(crac_ctx *c, crac_image *img, cudaStream_t s) {
    if (!img) return CRAC_ERR_INVALID_ARG;
    {
        DeviceGuard g(c->device);
        TRY(ctx_settle(c, true));   // the context's unsettled checkpoints first
    }
    TRY(img_wait(img, 0));          // its sizes and FULL flag are known once its pass has finished
    if (img->chunk_bytes != (1u << c->log2S)) return CRAC_ERR_IMAGE_MISMATCH;
    if (img->allocs.size() != c->allocs.size()) return CRAC_ERR_IMAGE_MISMATCH;
    for (size_t a = 0; a < c->allocs.size(); ++a)
        if (img->allocs[a].bytes != c->allocs[a].bytes || img->allocs[a].kind != c->allocs[a].kind)
            return CRAC_ERR_IMAGE_MISMATCH;
    // Chain back to the nearest FULL image.
    std::vector<crac_image *> chain;
    for (crac_image *cur = img;;) {
        chain.push_back(cur);
        if (cur->flags & CRAC_IMAGE_FULL) break;
        if (chain.size() >= 65535) return CRAC_ERR_UNSUPPORTED;
        crac_image *p = img_parent(cur);
        if (!p || p->lineage != cur->lineage || p->chunk_bytes != cur->chunk_bytes) return CRAC_ERR_IMAGE_MISMATCH;
        TRY(img_wait(p, 0));
        cur = p;
    }
    std::reverse(chain.begin(), chain.end());
    // On the device unless an image is on another device, or a host image
    // must be staged (no unified addressing, or CRAC_FLAG_STAGED_RESTORE).
    // Coded images are decoded by the in-place restore kernels only, so a
    // chain holding one reads its host images in place whenever the device
    // can address them.
    bool any_coded = false;
    for (crac_image *im : chain) any_coded = any_coded || (im->flags & CRAC_IMAGE_CODED);
    const bool mapped = c->uva && (!(c->cfg.flags & CRAC_FLAG_STAGED_RESTORE) || any_coded);
    bool on_device = true;
    for (crac_image *im : chain) {
        const bool dev_ok = im->residency == CRAC_RESIDENCY_DEVICE && im->device == c->device &&
                            (im->n_chunks == 0 || im->fp_dev.region >= 0);
        const bool host_ok = im->residency != CRAC_RESIDENCY_DEVICE && mapped;
        on_device = on_device && (dev_ok || host_ok);
    }
    if (on_device) return restart_device(c, img, chain, s);
    if (any_coded) return CRAC_ERR_UNSUPPORTED;
    for (crac_image *im : chain) {
        TRY(img_wait(im, 0));
        TRY(img_host_tables(im));
    }

    DeviceGuard g(c->device);
    const uint32_t log2S = c->log2S;
    const size_t na = img->allocs.size();
    const uint64_t nt = img->n_chunks;
    std::unordered_map<uint64_t, size_t> tpos;
    for (size_t a = 0; a < na; ++a) tpos[img->allocs[a].id] = a;

    // Owner map: for every target chunk, the newest chain image holding it.
    TRY(ensure_host(c->owner_h, std::max<uint64_t>(nt, 1) * 2));
    if (c->ev_last) CK(cudaEventSynchronize(c->ev_last));   // pinned scratch reuse
    uint16_t *owner = (uint16_t *)c->owner_h.p;
    std::fill(owner, owner + nt, (uint16_t)0xFFFF);
    std::vector<uint64_t> survivors(chain.size(), 0);
    std::vector<std::vector<int64_t>> img_map(chain.size());   // image alloc -> target alloc or -1
    for (size_t i = 0; i < chain.size(); ++i) {
        crac_image *im = chain[i];
        std::vector<int64_t> &m = img_map[i];
        m.resize(im->allocs.size());
        for (size_t a = 0; a < im->allocs.size(); ++a) {
            auto it = tpos.find(im->allocs[a].id);
            m[a] = (it == tpos.end() || img->allocs[it->second].bytes != im->allocs[a].bytes) ? -1 : (int64_t)it->second;
        }
        if (im->flags & CRAC_IMAGE_FULL) {
            for (size_t a = 0; a < im->allocs.size(); ++a) {
                if (m[a] < 0) continue;
                const uint64_t nch = ((im->allocs[a].bytes - 1) >> log2S) + 1;
                std::fill(owner + img->allocs[m[a]].first_chunk, owner + img->allocs[m[a]].first_chunk + nch, (uint16_t)i);
            }
        } else {
            const uint64_t *idx = (const uint64_t *)im->idx_h.p;
            size_t a = 0;
            for (uint64_t j = 0; j < im->k; ++j) {
                const uint64_t cc = idx[j];
                while (a + 1 < im->allocs.size() && im->allocs[a + 1].first_chunk <= cc) ++a;
                if (m[a] < 0) continue;
                owner[img->allocs[m[a]].first_chunk + (cc - im->allocs[a].first_chunk)] = (uint16_t)i;
            }
        }
    }
    for (uint64_t t = 0; t < nt; ++t) {
        if (owner[t] == 0xFFFF) return CRAC_ERR_IMAGE_MISMATCH;
        survivors[owner[t]]++;
    }
    if (fault_hit(CRAC_FAULT_H2D)) {
        t_last_cuda = (int)cudaErrorLaunchFailure;
        return CRAC_ERR_CUDA;
    }

    if (!s) CK(cudaDeviceSynchronize());
    // Scratch: owner map, per-image scatter descriptors, list offsets.
    size_t total_desc = 0;
    uint64_t host_k_total = 0;
    for (crac_image *im : chain) {
        total_desc += im->allocs.size();
        if (im->residency == CRAC_RESIDENCY_HOST && !(im->flags & CRAC_IMAGE_FULL)) host_k_total += im->k;
    }
    uint64_t cap = c->cfg.staging_bytes ? c->cfg.staging_bytes : kDefaultStagingMax;
    uint64_t max_host_payload = 0;
    for (crac_image *im : chain)
        if (im->residency == CRAC_RESIDENCY_HOST) max_host_payload = std::max(max_host_payload, im->payload_bytes);
    cap = std::max<uint64_t>(std::min(cap, round_up(std::max<uint64_t>(max_host_payload, 1), 256)), 1ull << log2S);
    TRY(ensure_dev(c->owner, std::max<uint64_t>(nt, 1) * 2));
    TRY(ensure_dev(c->sdesc, total_desc * sizeof(ScatterDesc)));
    TRY(ensure_host(c->sdesc_h, total_desc * sizeof(ScatterDesc)));
    TRY(ensure_dev(c->serr, 256));
    if (max_host_payload) {
        TRY(ensure_dev(c->staging, cap));
        TRY(ensure_dev(c->sidx, host_k_total * 8));
        TRY(ensure_dev(c->soff, host_k_total * 8));
        TRY(ensure_host(c->soff_h, host_k_total * 8));
    }
    CK(cudaStreamWaitEvent(s, c->ev_last, 0));
    CK(cudaMemsetAsync(c->serr.p, 0, 256, s));
    CK(cudaMemcpyAsync(c->owner.p, owner, nt * 2, cudaMemcpyHostToDevice, s));
    crac_restart_info_t ri{};
    ri.chain_length = (uint32_t)chain.size();
    for (size_t i = 0; i < chain.size(); ++i) ri.images_used += survivors[i] ? 1u : 0u;
    for (const ImgAlloc &a : img->allocs) ri.restored_bytes += a.bytes;
    CK(cudaEventRecord(c->ev_r0, s));
    ScatterDesc *sdh = (ScatterDesc *)c->sdesc_h.p;
    ScatterDesc *sdd = (ScatterDesc *)c->sdesc.p;
    const int grid = c->sm_count * 8;
    size_t dpos = 0;
    uint64_t lpos = 0;   // start of this image's region in sidx / soff / soff_h
    for (size_t i = 0; i < chain.size(); ++i) {
        crac_image *im = chain[i];
        const size_t nd = im->allocs.size();
        ScatterDesc *dh = sdh + dpos;
        ScatterDesc *dd = sdd + dpos;
        dpos += nd;
        if (!survivors[i]) continue;
        uint64_t pbase = 0;
        for (size_t a = 0; a < nd; ++a) {
            const int64_t t = img_map[i][a];
            dh[a] = ScatterDesc{im->allocs[a].first_chunk, im->allocs[a].bytes,
                                t < 0 ? 0 : img->allocs[t].first_chunk, t < 0 ? 0 : c->allocs[t].ptr, pbase, {0, 0, 0}};
            pbase += im->allocs[a].bytes;
        }
        CK(cudaMemcpyAsync(dd, dh, nd * sizeof(ScatterDesc), cudaMemcpyHostToDevice, s));
        ScatterParams P{};
        P.desc = dd;
        P.n_desc = (uint32_t)nd;
        P.log2_chunk = log2S;
        P.image_index = (uint32_t)i;
        P.owner = (const uint16_t *)c->owner.p;
        P.n_owner = nt;
        P.err = (unsigned int *)c->serr.p;
        if (im->residency == CRAC_RESIDENCY_DEVICE) {
            for (const Piece &pc : im->pieces) {
                if (!pc.k) continue;
                P.full = 0;
                P.j0 = 0;
                P.j1 = pc.k;
                P.idx = (const uint64_t *)pc.idx_dev.p;
                P.off = (const uint64_t *)pc.off_dev.p;
                P.payload = pc.dev.p;
                P.origin = 0;
                P.window = pc.span ? pc.span : pc.bytes;
                CK(launch_scatter(P, (int)std::min<uint64_t>((pc.k + 7) / 8, (uint64_t)grid), s));
                ri.entries_scanned += pc.k;
                ri.scatter_launches++;
            }
            continue;
        }
        // Host image: H2D windows of at most `cap` payload bytes into staging.
        const bool full = (im->flags & CRAC_IMAGE_FULL) != 0;
        const uint64_t nent = full ? im->n_chunks : im->k;
        const uint64_t *idx_h = (const uint64_t *)im->idx_h.p;
        uint64_t *soff_h = (uint64_t *)c->soff_h.p + lpos;
        uint64_t *sidx_d = (uint64_t *)c->sidx.p + lpos;
        uint64_t *soff_d = (uint64_t *)c->soff.p + lpos;
        if (!full) lpos += nent;
        std::vector<uint64_t> fpre;   // FULL: payload offset of each allocation
        if (full) {
            fpre.resize(nd);
            uint64_t acc = 0;
            for (size_t a = 0; a < nd; ++a) {
                fpre[a] = acc;
                acc += im->allocs[a].bytes;
            }
        } else {
            size_t a = 0;
            uint64_t acc = 0;
            for (uint64_t j = 0; j < nent; ++j) {
                while (a + 1 < nd && im->allocs[a + 1].first_chunk <= idx_h[j]) ++a;
                soff_h[j] = acc;
                acc += chunk_len(im->allocs[a].bytes, idx_h[j] - im->allocs[a].first_chunk, log2S);
            }
            if (acc != im->payload_bytes) return CRAC_ERR_CORRUPT;
        }
        // offset and length of entry j
        size_t fa = 0;
        auto entry = [&](uint64_t j, uint64_t *o, uint64_t *len) {
            if (full) {
                while (fa + 1 < nd && im->allocs[fa + 1].first_chunk <= j) ++fa;
                while (fa > 0 && im->allocs[fa].first_chunk > j) --fa;
                const uint64_t local = j - im->allocs[fa].first_chunk;
                *o = fpre[fa] + (local << log2S);
                *len = chunk_len(im->allocs[fa].bytes, local, log2S);
            } else {
                *o = soff_h[j];
                *len = (j + 1 < nent ? soff_h[j + 1] : im->payload_bytes) - soff_h[j];
            }
        };
        if (!full && nent) {
            CK(cudaMemcpyAsync(sidx_d, idx_h, nent * 8, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(soff_d, soff_h, nent * 8, cudaMemcpyHostToDevice, s));
        }
        uint64_t j0 = 0;
        while (j0 < nent) {
            uint64_t o0, l0;
            entry(j0, &o0, &l0);
            uint64_t j1 = j0 + 1, end = o0 + l0;
            while (j1 < nent) {
                uint64_t o, l;
                entry(j1, &o, &l);
                if (o + l - o0 > cap) break;
                end = o + l;
                ++j1;
            }
            // H2D payload bytes [o0, end) from the pieces that hold them.
            for (const Piece &pc : im->pieces) {
                const uint64_t lo = std::max(o0, pc.off0), hi = std::min(end, pc.off0 + pc.bytes);
                if (hi <= lo) continue;
                CK(cudaMemcpyAsync((uint8_t *)c->staging.p + (lo - o0), pc.host.p + (lo - pc.off0), hi - lo,
                                   cudaMemcpyHostToDevice, s));
                ri.h2d_bytes += hi - lo;
            }
            P.full = full ? 1u : 0u;
            P.j0 = j0;
            P.j1 = j1;
            P.idx = full ? nullptr : sidx_d + j0;
            P.off = full ? nullptr : soff_d + j0;
            P.payload = (const uint8_t *)c->staging.p;
            P.origin = o0;
            P.window = end - o0;
            CK(launch_scatter(P, (int)std::min<uint64_t>((j1 - j0 + 7) / 8, (uint64_t)grid), s));
            ri.entries_scanned += j1 - j0;
            ri.scatter_launches++;
            j0 = j1;
        }
    }
    // The image's fingerprints go to the spare table, which becomes the
    // baseline only once the restore has succeeded.
    const int spare = spare_fp(c);
    TRY(ensure_dev(c->fp[spare], std::max<uint64_t>(nt, 1) * 8));
    CK(cudaEventRecord(c->ev_r1, s));
    if (nt) CK(cudaMemcpyAsync(c->fp[spare].p, img->fp_h.p, nt * 8, cudaMemcpyHostToDevice, s));
    CK(launch_report(nullptr, 0, (const uint32_t *)c->serr.p, c->serr_h.p, s));
    CK(cudaEventRecord(c->ev_last, s));
    CK(cudaEventSynchronize(c->ev_last));
    if (*(const unsigned *)c->serr_h.p) return CRAC_ERR_CORRUPT;
    cudaEventElapsedTime(&ri.device_ms, c->ev_r0, c->ev_r1);
    ri.chunks_rewritten = nt;   // the staged path restores every chunk
    c->last_restart = ri;
    c->fp_cur = spare;
    restart_commit(c, img);
    (void)na;
    return CRAC_OK;
}

}  // namespace crac
