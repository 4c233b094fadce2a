// Contexts and the checkpoint pass: registry snapshot (A0), managed prefetch
// (A1), the batched pass launched as one CUDA graph (A2-A4), the drain to
// pinned host memory (A5) and the commit (A6); also the trial pass the
// autotuner runs.
#include "crac_runtime.h"

using namespace crac;

namespace crac {

crac_status_t ctx_init(crac_ctx *c, const crac_config_t *cfg_in) {
    crac_config_default(&c->cfg);
    if (cfg_in) {
        if (cfg_in->struct_size && cfg_in->struct_size != sizeof(crac_config_t)) return CRAC_ERR_INVALID_ARG;
        c->cfg = *cfg_in;
        c->cfg.struct_size = sizeof(crac_config_t);
    }
    crac_config_t &cfg = c->cfg;
    if (cfg.chunk_bytes == 0) cfg.chunk_bytes = 65536;
    if (cfg.chunk_bytes < 16 || cfg.chunk_bytes > (1u << 24) || (cfg.chunk_bytes & (cfg.chunk_bytes - 1)))
        return CRAC_ERR_INVALID_ARG;
    if (cfg.image_residency > CRAC_RESIDENCY_DEVICE || cfg.launch_mode > CRAC_LAUNCH_PER_ALLOC)
        return CRAC_ERR_INVALID_ARG;
    if (cfg.threads && cfg.threads != 256) return CRAC_ERR_INVALID_ARG;
    if (cfg.warps_per_chunk && cfg.warps_per_chunk != 1 && cfg.warps_per_chunk != 8)
        return CRAC_ERR_INVALID_ARG;
    if (cfg.chunks_per_tile > 256) return CRAC_ERR_INVALID_ARG;
    if (cfg.pass_kernel > CRAC_PASS_SPARSE) return CRAC_ERR_INVALID_ARG;
    if (cfg.flags & ~(CRAC_FLAG_STAGED_RESTORE | CRAC_FLAG_INCREMENTAL_RESTORE | CRAC_FLAG_DIRECT_DRAIN |
                      CRAC_FLAG_COMPRESS | CRAC_FLAG_WAIT_PASS))
        return CRAC_ERR_INVALID_ARG;
    if (cfg.pass_kernel == CRAC_PASS_SPARSE && (cfg.flags & CRAC_FLAG_COMPRESS)) return CRAC_ERR_INVALID_ARG;
    if (cfg.pass_kernel == CRAC_PASS_SPARSE && cfg.image_residency != CRAC_RESIDENCY_DEVICE)
        return CRAC_ERR_INVALID_ARG;
    if (cfg.pass_kernel == CRAC_PASS_TMA && (cfg.chunk_bytes < 1024 || cfg.chunk_bytes > 65536))
        return CRAC_ERR_INVALID_ARG;
    if (cfg.timeout_ns == 0) cfg.timeout_ns = kDefaultTimeoutNs;
    c->log2S = log2u(cfg.chunk_bytes);
    c->lineage = cfg.lineage ? cfg.lineage : (g_lineage_counter.fetch_add(1) + 1);
    return CRAC_OK;
}

// CUDA resources are created on the first checkpoint or restart, so that the
// registry works (and can be tested) without touching the device.
crac_status_t ctx_cuda_ready(crac_ctx *c) {
    if (c->lost) return CRAC_ERR_CUDA;
    if (c->cuda_ready) return CRAC_OK;
    int dev = c->cfg.device;
    if (dev < 0) CK(cudaGetDevice(&dev));
    c->device = dev;
    DeviceGuard g(dev);
    CK(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev));
    int uva = 0;
    CK(cudaDeviceGetAttribute(&uva, cudaDevAttrUnifiedAddressing, dev));
    c->uva = uva != 0;
    CK(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->ev_last, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&c->ev_pass, cudaEventDisableTiming));
    CK(cudaEventCreate(&c->ev_t0));
    CK(cudaEventCreate(&c->ev_t1));
    CK(cudaEventCreate(&c->ev_p0));
    CK(cudaEventCreate(&c->ev_p1));
    for (cudaEvent_t &e : c->sev) CK(cudaEventCreate(&e));
    CK(cudaEventCreate(&c->ev_r0));
    CK(cudaEventCreate(&c->ev_r1));
    CK(prepare_drain());
    TRY(ensure_host(c->ctrl_h, sizeof(CkptCtrl) + 16 * (1 + kEncPieces)));   // + the encoder's offsets, errors
    for (cudaEvent_t &e : c->ev_piece) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    CK(cudaEventCreate(&c->ev_z0));
    CK(cudaEventCreate(&c->ev_z1));
    TRY(ensure_host(c->serr_h, 256));
    if (c->cfg.reserve_host_bytes) {
        TRY(pinned_arena().reserve(c->cfg.reserve_host_bytes));
        pinned_arena().mark_reserved();
    }
    if (c->cfg.reserve_device_bytes) {
        TRY(device_arena(dev).reserve(c->cfg.reserve_device_bytes));
        device_arena(dev).mark_reserved();
    }
    c->cuda_ready = true;
    return CRAC_OK;
}

void ctx_free_all(crac_ctx *c) {
    tune_clear(c);
    if (!c->cuda_ready) {
        img_unref(c->parent);
        c->parent = nullptr;
        return;
    }
    DeviceGuard g(c->device);
    ctx_settle(c, true);
    img_unref(c->settled.parent);
    c->settled.parent = nullptr;
    cudaDeviceSynchronize();
    for (DevBuf *b : {&c->fp[0], &c->fp[1], &c->fp[2], &c->ppos[0], &c->ppos[1], &c->chdr, &c->desc, &c->work, &c->idx, &c->off, &c->staging,
                      &c->lens, &c->carry, &c->owner, &c->sdesc, &c->sidx, &c->soff, &c->serr,
                      &c->vdesc, &c->vwork, &c->vfp, &c->vidx, &c->voff, &c->cstage, &c->zwork, &c->zoff,
                      &c->zlen})
        if (b->p) cudaFree(b->p);
    for (HostBuf *b : {&c->desc_h, &c->desc_h2, &c->ctrl_h, &c->owner_h, &c->sdesc_h, &c->soff_h, &c->serr_h, &c->vdesc_h})
        if (b->p) cudaFreeHost(b->p);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->sgexec) cudaGraphExecDestroy(c->sgexec);
    if (c->sgraph) cudaGraphDestroy(c->sgraph);
    for (cudaEvent_t e : {c->ev_last, c->ev_pass, c->ev_t0, c->ev_t1, c->ev_p0, c->ev_p1, c->sev[0], c->sev[1],
                          c->sev[2], c->sev[3], c->ev_r0, c->ev_r1})
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : c->ev_piece)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : {c->ev_z0, c->ev_z1})
        if (e) cudaEventDestroy(e);
    if (c->side) cudaStreamDestroy(c->side);
    cudaGetLastError();
    img_unref(c->parent);
    c->parent = nullptr;
}

// Work split of the fused kernel for the context's chunk size.
void pick_split(const crac_ctx *c, int *wpc, uint32_t *cpt) {
    const uint64_t S = 1ull << c->log2S;
    int w = (int)c->cfg.warps_per_chunk;
    if (!w) w = S >= 16384 ? 8 : 1;
    uint32_t t = c->cfg.chunks_per_tile;
    if (!t) {
        // One chunk per warp: 128 KiB tiles; a CTA per chunk: 256 KiB tiles,
        // which hide the look-back better (measured at 64 KiB chunks).
        const uint64_t tile_bytes = w == 8 ? 256ull << 10 : 128ull << 10;
        t = (uint32_t)std::max<uint64_t>(1, tile_bytes / S);
        const uint32_t groups = 8 / w;
        t = std::max(t, groups);
        t = std::min<uint32_t>(t, 256);
    }
    *wpc = w;
    *cpt = t;
}

struct Segment {
    uint64_t c0, c1, bytes;
};

// Split the global chunk range into segments of at most `cap` bytes.
std::vector<Segment> make_segments(const std::vector<AllocRec> &allocs, const std::vector<uint64_t> &first,
                                   uint32_t log2S, uint64_t cap) {
    std::vector<Segment> out;
    const uint64_t S = 1ull << log2S;
    Segment cur{0, 0, 0};
    for (size_t a = 0; a < allocs.size(); ++a) {
        const uint64_t nch = first[a + 1] - first[a];
        uint64_t local = 0;
        while (local < nch) {
            const uint64_t rest_bytes = allocs[a].bytes - (local << log2S);
            const uint64_t room = cap - cur.bytes;
            uint64_t take, tb;
            if (rest_bytes <= room) {
                take = nch - local;
                tb = rest_bytes;
            } else {
                take = room / S;
                tb = take * S;
            }
            if (take == 0) {
                out.push_back(cur);
                cur = Segment{cur.c1, cur.c1, 0};
                continue;
            }
            cur.c1 += take;
            cur.bytes += tb;
            local += take;
        }
    }
    if (cur.c1 > cur.c0) out.push_back(cur);
    return out;
}

// Kernel-node parameters of the control block's report to the host (args
// must outlive the node's add or update call).
struct ReportNode {
    const void *words;
    uint32_t n = sizeof(CkptCtrl) / 8;
    const uint32_t *word32 = nullptr;
    void *dst;
    void *args[4];
    cudaKernelNodeParams kp{};
    ReportNode(const void *src, void *to) : words(src), dst(to) {
        args[0] = &words;
        args[1] = &n;
        args[2] = &word32;
        args[3] = &dst;
        kp.func = const_cast<void *>(report_fn());
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(32);
        kp.kernelParams = args;
    }
};

// Build (or update) the graph memset -> fused kernel -> ctrl report and launch it.
crac_status_t launch_fused_graph(crac_ctx *c, const CkptParams &P, size_t work_bytes, const void *fn,
                                 int threads, size_t smem, int grid, void *ctrl_dst, cudaStream_t s) {
    if (!fn) return CRAC_ERR_INVALID_ARG;
    CkptParams Pc = P;
    void *args[] = {&Pc};
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void *>(fn);
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(threads);
    kp.sharedMemBytes = (unsigned)smem;
    kp.kernelParams = args;
    cudaMemsetParams mp{};
    mp.dst = c->work.p;
    mp.value = 0;
    mp.elementSize = 4;
    mp.width = work_bytes / 4;
    mp.height = 1;
    mp.pitch = 0;
    bool rebuilt = false;
    ReportNode rep(P.ctrl, ctrl_dst);
    if (c->gexec && c->g_fn == fn) {
        // Width changes of a memset node may be rejected; rebuild then.
        if (cudaGraphExecMemsetNodeSetParams(c->gexec, c->g_memset, &mp) != cudaSuccess ||
            cudaGraphExecKernelNodeSetParams(c->gexec, c->g_kernel, &kp) != cudaSuccess ||
            cudaGraphExecKernelNodeSetParams(c->gexec, c->g_copy, &rep.kp) != cudaSuccess) {
            cudaGetLastError();
            c->g_fn = nullptr;
        }
    }
    if (!c->gexec || c->g_fn != fn) {
        if (c->gexec) cudaGraphExecDestroy(c->gexec);
        if (c->graph) cudaGraphDestroy(c->graph);
        c->gexec = nullptr;
        c->graph = nullptr;
        CK(cudaGraphCreate(&c->graph, 0));
        CK(cudaGraphAddMemsetNode(&c->g_memset, c->graph, nullptr, 0, &mp));
        CK(cudaGraphAddKernelNode(&c->g_kernel, c->graph, &c->g_memset, 1, &kp));
        CK(cudaGraphAddKernelNode(&c->g_copy, c->graph, &c->g_kernel, 1, &rep.kp));
        CK(cudaGraphInstantiate(&c->gexec, c->graph, 0));
        c->g_fn = fn;
        c->g_threads = threads;
        rebuilt = true;
    }
    (void)rebuilt;
    CK(cudaEventRecord(c->ev_t0, s));   // after the host-side updates: times the device work only
    CK(cudaGraphLaunch(c->gexec, s));
    count_launches(2);
    return CRAC_OK;
}

// Build (or update) the split-pass graph and launch it.
crac_status_t launch_split_graph(crac_ctx *c, const CkptParams &P, size_t work_bytes, unsigned long long *acc,
                                 uint32_t log2Seg, const void *hash_fn, size_t hash_smem, const int grids[3],
                                 void *ctrl_dst, cudaStream_t s) {
    // The gather instance follows P.crz_hdr, which only the hash instance
    // split_hash_kernel<true> runs with: hash_fn alone keys the cached graph.
    const void *fns[3] = {hash_fn, split_finalize_fn(), split_gather_fn(P.crz_hdr != nullptr)};
    const int thr[3] = {split_hash_threads(), split_finalize_threads(), split_gather_threads()};
    CkptParams Pc = P;
    unsigned long long *accv = acc;
    uint32_t segv = log2Seg;
    void *args[] = {&Pc, &accv, &segv};
    cudaKernelNodeParams kp[3];
    for (int i = 0; i < 3; ++i) {
        kp[i] = cudaKernelNodeParams{};
        kp[i].func = const_cast<void *>(fns[i]);
        kp[i].gridDim = dim3(grids[i]);
        kp[i].blockDim = dim3(thr[i]);
        kp[i].sharedMemBytes = i == 0 ? (unsigned)hash_smem : 0u;
        kp[i].kernelParams = args;
    }
    cudaMemsetParams mp{};
    mp.dst = c->work.p;
    mp.value = 0;
    mp.elementSize = 4;
    mp.width = work_bytes / 4;
    mp.height = 1;
    ReportNode rep(P.ctrl, ctrl_dst);
    bool ok = c->sgexec != nullptr && c->s_hash_fn == hash_fn;
    if (ok) {
        ok = cudaGraphExecMemsetNodeSetParams(c->sgexec, c->s_memset, &mp) == cudaSuccess;
        for (int i = 0; ok && i < 3; ++i)
            ok = cudaGraphExecKernelNodeSetParams(c->sgexec, c->s_k[i], &kp[i]) == cudaSuccess;
        if (ok) ok = cudaGraphExecKernelNodeSetParams(c->sgexec, c->s_copy, &rep.kp) == cudaSuccess;
        if (!ok) cudaGetLastError();
    }
    if (!ok) {
        if (c->sgexec) cudaGraphExecDestroy(c->sgexec);
        if (c->sgraph) cudaGraphDestroy(c->sgraph);
        c->sgexec = nullptr;
        c->sgraph = nullptr;
        // memset -> event 0 -> hash => finalize => gather -> control block report,
        // where => is a programmatic edge (the consumer is launched as its
        // producer drains and waits in-kernel for its completion); events 1-3
        // record each kernel's end on side branches, off the critical path.
        CK(cudaGraphCreate(&c->sgraph, 0));
        CK(cudaGraphAddMemsetNode(&c->s_memset, c->sgraph, nullptr, 0, &mp));
        cudaGraphNode_t ev;
        CK(cudaGraphAddEventRecordNode(&ev, c->sgraph, &c->s_memset, 1, c->sev[0]));
        CK(cudaGraphAddKernelNode(&c->s_k[0], c->sgraph, &ev, 1, &kp[0]));
        cudaGraphEdgeData pe{};
        pe.from_port = cudaGraphKernelNodePortProgrammatic;
        pe.type = cudaGraphDependencyTypeProgrammatic;
        for (int i = 1; i < 3; ++i) {
            CK(cudaGraphAddKernelNode(&c->s_k[i], c->sgraph, nullptr, 0, &kp[i]));
            CK(cudaGraphAddDependencies(c->sgraph, &c->s_k[i - 1], &c->s_k[i], &pe, 1));
        }
        for (int i = 0; i < 3; ++i) CK(cudaGraphAddEventRecordNode(&ev, c->sgraph, &c->s_k[i], 1, c->sev[i + 1]));
        CK(cudaGraphAddKernelNode(&c->s_copy, c->sgraph, &c->s_k[2], 1, &rep.kp));
        CK(cudaGraphInstantiate(&c->sgexec, c->sgraph, 0));
        c->s_hash_fn = hash_fn;
    }
    CK(cudaEventRecord(c->ev_t0, s));
    CK(cudaGraphLaunch(c->sgexec, s));
    count_launches(4);
    return CRAC_OK;
}

// Enqueue one segment of the checkpoint pass on s, reading the baseline
// fp[fp_cur] and writing fingerprints to fp[out_fp]; the control block is
// copied to the host at ctrl_dst after the pass, and ev_pass is recorded.
crac_status_t launch_segment(crac_ctx *c, const Segment &sg, const CkptDesc *desc_dev,
                             const std::vector<uint64_t> &first, uint64_t *idx_d, uint64_t *off_d,
                             uint64_t idx_cap, uint8_t *staging, uint64_t staging_cap, int out_fp,
                             void *ctrl_dst, cudaStream_t s) {
    const uint64_t nseg = sg.c1 - sg.c0;
    const uint64_t *fp_old = (const uint64_t *)c->fp[c->fp_cur].p;
    uint64_t *fp_new = (uint64_t *)c->fp[out_fp].p;
    const bool inject_wait = c->cfg.launch_mode == CRAC_LAUNCH_BATCHED;
    if (fault_hit(CRAC_FAULT_PASS)) {
        t_last_cuda = (int)cudaErrorLaunchFailure;
        return CRAC_ERR_CUDA;
    }
    const bool split = c->cfg.launch_mode == CRAC_LAUNCH_BATCHED &&
                       (c->pass_now == CRAC_PASS_SPLIT || c->pass_now == CRAC_PASS_SPARSE);
    if (split) {
        const uint32_t cptF = (uint32_t)split_finalize_threads();
        const uint64_t n_tiles = (nseg + cptF - 1) / cptF;
        if (n_tiles > 0x7fffffffull) return CRAC_ERR_UNSUPPORTED;
        const size_t status_bytes = sizeof(CkptCtrl) + 16 * n_tiles;
        const size_t work_bytes = status_bytes + 8 * nseg;
        TRY(ensure_dev(c->work, work_bytes));
        // 512 B..4 KiB chunks: several whole chunks per warp iteration.
        const bool small = c->log2S >= 9 && c->log2S < 13;
        const uint32_t log2Seg = std::min<uint32_t>(c->log2S, 13);
        // Coded contexts with chunks of 8 KiB and more: the kernel that writes a
        // chunk to staging (hash or gather) also writes its CRZ1 block headers
        // for the encoder.
        uint64_t *crz_hdr = c->crz_hdr_now ? (uint64_t *)c->chdr.p : nullptr;
        // The sparse pass on 512 B - 4 KiB chunks may place the dirty chunks
        // densely (a bulk store per warp iteration from shared memory).
        const bool dense = small && c->sparse_ok && staging && c->dense_now;
        const void *hash_fn = dense ? split_hash_small_dense_fn(1 << (c->log2S - 8))
                              : small ? split_hash_small_fn(1 << (c->log2S - 8)) : split_hash_fn(crz_hdr != nullptr);
        const size_t hash_smem = dense ? split_dense_smem() : 0;
        if (dense) CK(split_dense_prepare(hash_fn));
        CkptParams P{};
        P.crz_hdr = crz_hdr;
        P.desc = desc_dev;
        P.n_allocs = (uint32_t)c->allocs.size();
        P.log2_chunk = c->log2S;
        P.c_begin = sg.c0;
        P.c_end = sg.c1;
        P.cpt = cptF;
        P.n_tiles = (uint32_t)n_tiles;
        P.fp_old = fp_old;
        P.fp_new = fp_new;
        P.idx_out = idx_d;
        P.off_out = off_d;
        P.idx_cap = idx_cap;
        P.staging = staging;
        P.staging_cap = staging_cap;
        P.ctrl = (CkptCtrl *)c->work.p;
        P.tile_cnt = (uint64_t *)((uint8_t *)c->work.p + sizeof(CkptCtrl));
        P.tile_bytes = P.tile_cnt + n_tiles;
        P.timeout_ns = c->cfg.timeout_ns;
        P.skip_first_ticket = (n_tiles >= 2 && fault_hit(CRAC_FAULT_DEVICE_WAIT)) ? 1u : 0u;
        // FULL pass, or the sparse pass: chunks are written to staging by the
        // hash kernel, at their uncompacted offsets.
        P.sparse = c->sparse_ok && staging ? (dense ? 2u : 1u) : 0u;
        P.full_copy = (c->full_copy_ok || P.sparse) && staging ? 1u : 0u;
        P.alloc_prefix = (const uint64_t *)(desc_dev + c->allocs.size());
        if (c->spec_now) {
            P.ppos = c->spec_use ? (const uint64_t *)c->ppos[c->ppos_cur].p : nullptr;
            P.ppos_next = (uint64_t *)c->ppos[1 - c->ppos_cur].p;
        }
        {
            const size_t a0 = std::upper_bound(first.begin(), first.end(), sg.c0) - first.begin() - 1;
            uint64_t pre = 0;
            for (size_t a = 0; a < a0; ++a) pre += c->allocs[a].bytes;
            P.seg_base = pre + ((sg.c0 - first[a0]) << c->log2S);
        }
        unsigned long long *acc = (unsigned long long *)((uint8_t *)c->work.p + status_bytes);
        const uint64_t n_slots = small ? (nseg + (8192u >> c->log2S) - 1) / (8192u >> c->log2S)
                                       : nseg << (c->log2S - log2Seg);
        const int gh = (int)std::max<uint64_t>(1, std::min<uint64_t>(
                           (n_slots + 7) / 8,
                           (uint64_t)c->sm_count * split_max_ctas_per_sm_smem(hash_fn, split_hash_threads(), hash_smem)));
        const int gf = (int)std::min<uint64_t>(n_tiles, (uint64_t)c->sm_count * 2);
        const int gg = c->sm_count * 8;
        const int grids[3] = {gh, gf, gg};
        TRY(launch_split_graph(c, P, work_bytes, acc, log2Seg, hash_fn, hash_smem, grids, ctrl_dst, s));
        if (c->spec_now) {   // this pass's offsets predict the next one's
            c->ppos_cur ^= 1;
            c->ppos_ok = true;
            c->ppos_layout = c->layout_version;
        }
        c->last.grid = (uint32_t)gh;
        c->last.chunks_per_tile = cptF;
        c->last.warps_per_chunk = 0;
        c->last.kernel_launches += 4;   // hash, finalize, gather, control-block report
        c->last.pass_kernel = P.sparse ? CRAC_PASS_SPARSE : CRAC_PASS_SPLIT;
    } else if (c->cfg.launch_mode == CRAC_LAUNCH_BATCHED) {
        const uint64_t S = 1ull << c->log2S;
        const bool tma = c->pass_now == CRAC_PASS_TMA;
        int wpc;
        uint32_t cpt;
        const void *fn;
        int threads;
        size_t smem = 0;
        int per_sm;
        if (tma) {
            if (!c->tma_ready) {
                CK(ckpt_tma_prepare());
                c->tma_ready = true;
            }
            cpt = (uint32_t)(ckpt_tma_slot_bytes() / S);
            wpc = (int)std::max<uint64_t>(1, 8 * S / ckpt_tma_slot_bytes());
            fn = ckpt_tma_fn(wpc);
            threads = ckpt_tma_threads();
            smem = ckpt_tma_smem((uint32_t)std::min<size_t>(c->allocs.size(), UINT32_MAX));
            per_sm = 1;
        } else {
            pick_split(c, &wpc, &cpt);
            fn = ckpt_fused_fn(256, wpc);
            threads = 256;
            per_sm = (int)c->cfg.ctas_per_sm;
            if (!per_sm) per_sm = std::max(1, ckpt_fused_max_ctas_per_sm(256, wpc));
        }
        const uint64_t n_tiles = (nseg + cpt - 1) / cpt;
        if (n_tiles > 0x7fffffffull) return CRAC_ERR_UNSUPPORTED;
        const size_t work_bytes = sizeof(CkptCtrl) + 16 * n_tiles;
        TRY(ensure_dev(c->work, work_bytes));
        const int grid = (int)std::min<uint64_t>(n_tiles, (uint64_t)c->sm_count * per_sm);
        CkptParams P{};
        P.desc = desc_dev;
        P.n_allocs = (uint32_t)c->allocs.size();
        P.log2_chunk = c->log2S;
        P.c_begin = sg.c0;
        P.c_end = sg.c1;
        P.cpt = cpt;
        P.n_tiles = (uint32_t)n_tiles;
        P.fp_old = fp_old;
        P.fp_new = fp_new;
        P.idx_out = idx_d;
        P.off_out = off_d;
        P.idx_cap = idx_cap;
        P.staging = staging;
        P.staging_cap = staging_cap;
        P.ctrl = (CkptCtrl *)c->work.p;
        P.tile_cnt = (uint64_t *)((uint8_t *)c->work.p + sizeof(CkptCtrl));
        P.tile_bytes = P.tile_cnt + n_tiles;
        P.timeout_ns = c->cfg.timeout_ns;
        P.skip_first_ticket = (inject_wait && n_tiles >= 2 && fault_hit(CRAC_FAULT_DEVICE_WAIT)) ? 1u : 0u;
        P.first_cached = tma && c->allocs.size() <= ckpt_tma_cached_allocs() ? 1u : 0u;
        TRY(launch_fused_graph(c, P, work_bytes, fn, threads, smem, grid, ctrl_dst, s));
        c->last.pass_kernel = tma ? CRAC_PASS_TMA : CRAC_PASS_LDG;
        c->last.grid = (uint32_t)grid;
        c->last.chunks_per_tile = cpt;
        c->last.warps_per_chunk = (uint32_t)wpc;
        c->last.kernel_launches += 2;   // the pass, control-block report
    } else {
        TRY(ensure_dev(c->work, sizeof(CkptCtrl)));
        TRY(ensure_dev(c->lens, nseg * sizeof(uint32_t)));
        TRY(ensure_dev(c->carry, sizeof(PerAllocCarry)));
        CkptCtrl *ctrl = (CkptCtrl *)c->work.p;
        CK(cudaEventRecord(c->ev_t0, s));
        CK(cudaMemsetAsync(ctrl, 0, sizeof(CkptCtrl), s));
        CK(cudaMemsetAsync(c->carry.p, 0, sizeof(PerAllocCarry), s));
        const size_t a0 = std::upper_bound(first.begin(), first.end(), sg.c0) - first.begin() - 1;
        for (size_t a = a0; a < c->allocs.size() && first[a] < sg.c1; ++a) {
            const uint64_t u0 = std::max(first[a], sg.c0), u1 = std::min(first[a + 1], sg.c1);
            if (u1 <= u0) continue;
            const int g = (int)std::min<uint64_t>(u1 - u0, (uint64_t)c->sm_count * 8);
            CK(launch_fp_range(desc_dev + a, u0, u1, c->log2S, fp_old, fp_new, (uint32_t *)c->lens.p,
                               sg.c0, g, s));
            CK(launch_compact_range((const uint32_t *)c->lens.p, sg.c0, u0, u1, idx_d, off_d, idx_cap,
                                    (PerAllocCarry *)c->carry.p, ctrl, s));
            CK(launch_gather_range(desc_dev + a, c->log2S, idx_d, off_d, (PerAllocCarry *)c->carry.p,
                                   u1 - u0, idx_cap, staging, staging_cap, ctrl, g, s));
            c->last.kernel_launches += 3;
        }
        CK(launch_report(ctrl, sizeof(CkptCtrl) / 8, nullptr, ctrl_dst, s));
        c->last.kernel_launches += 1;
    }
    c->split_now = split;
    CK(cudaEventRecord(c->ev_t1, s));
    CK(cudaEventRecord(c->ev_pass, s));
    return CRAC_OK;
}

// The timings of the pass just enqueued (its events must have completed):
// device time added to *ms, the split pass's per-kernel times to c->last.
void pass_timings(crac_ctx *c, float *ms) {
    float t = 0;
    if (cudaEventElapsedTime(&t, c->ev_t0, c->ev_t1) == cudaSuccess) *ms += t;
    cudaGetLastError();
    if (c->split_now) {
        float a = 0, b = 0, d = 0;
        if (cudaEventElapsedTime(&a, c->sev[0], c->sev[1]) == cudaSuccess &&
            cudaEventElapsedTime(&b, c->sev[1], c->sev[2]) == cudaSuccess &&
            cudaEventElapsedTime(&d, c->sev[2], c->sev[3]) == cudaSuccess) {
            c->last.hash_ms += a;
            c->last.finalize_ms += b;
            c->last.gather_ms += d;
        }
        cudaGetLastError();
    }
}

// One segment of the checkpoint pass, waited for; on return the control
// block is on the host.
crac_status_t run_segment(crac_ctx *c, const Segment &sg, const CkptDesc *desc_dev,
                          const std::vector<uint64_t> &first, uint64_t *idx_d, uint64_t *off_d,
                          uint64_t idx_cap, uint8_t *staging, uint64_t staging_cap, int out_fp,
                          cudaStream_t s, CkptCtrl *ctrl_out, float *ms) {
    TRY(launch_segment(c, sg, desc_dev, first, idx_d, off_d, idx_cap, staging, staging_cap, out_fp, c->ctrl_h.p, s));
    CK(cudaEventSynchronize(c->ev_pass));
    pass_timings(c, ms);
    *ctrl_out = *(const CkptCtrl *)c->ctrl_h.p;
    if (ctrl_out->err & kErrLostCopy) {
        c->lost = true;
        return CRAC_ERR_CUDA;
    }
    if (ctrl_out->err & kErrTimeout) return CRAC_ERR_TIMEOUT;
    if (ctrl_out->err) return CRAC_ERR_CORRUPT;
    return CRAC_OK;
}


// Entries per tile of the encoder: about 64 KiB of raw payload.
uint32_t crz_tile_entries(uint32_t log2S) {
    return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(crz_tile_max(), 65536ull >> std::min<uint32_t>(log2S, 16)));
}

// Encoder scratch of a segment with k entries and D raw bytes: the error
// word, one tile counter per launch, then one look-back word per tile and the
// block header words of multi-window chunks.
constexpr size_t kZworkTickets = 4;                             // after the error word
constexpr size_t kZworkPieceOff = 48;                           // the sized encoder's piece offsets
constexpr size_t kZworkHead = kZworkPieceOff + 8 * (kEncPieces + 1) + 8;   // rounded up to 16
static_assert(kZworkTickets + 4 * kEncPieces <= kZworkPieceOff && kZworkHead % 16 == 0, "encoder scratch head");

size_t crz_work_bytes(uint64_t k, uint64_t D, uint32_t log2S) {
    const uint64_t tiles = (k + crz_tile_entries(log2S) - 1) / crz_tile_entries(log2S);
    return kZworkHead + 8 * tiles + 8 * (D / 512 + 1);
}

// CRAC_FLAG_COMPRESS: the segment's raw payload (device staging, offsets in
// c->off) -> its streams.  Host images: into the piece's pinned block when
// direct drain finds room, else into c->cstage, from where the side stream
// copies them to the piece's pinned block; tables in c->zoff / c->zlen.
// Staged encodes of many tiles run as several launches over consecutive tile
// ranges, and each range's streams are copied as soon as the host sees that
// launch end (its end offset comes back with it), so the copy of the first
// ranges overlaps the encoding of the rest; the pinned block is carved at the
// worst case from the regions as they are (else the copy follows the whole
// encode, as for a single launch).  Device images: into pc.dev, with the
// stream offsets in pc.off_dev and lengths in pc.zlen_dev.  On return the
// total stream bytes are known (*Z), and *zplaced says that the streams are
// in pc.host, or on their way there on the side stream.
// encode_segment when the pass made the block headers (c->crz_hdr_now):
// crz_size_kernel sizes and places every stream from the headers, the host
// reads the total (and the piece boundaries), takes an exact destination,
// and crz_encode_sized_kernel codes in up to kEncPieces launches; for staged
// host images each launch's streams are copied to the pinned block as soon
// as it ends (its bytes are known already), overlapping the later launches.
crac_status_t encode_segment_sized(crac_ctx *c, Piece &pc, const CkptCtrl &ctrl, bool host_res, bool direct_flag,
                                   cudaStream_t s, uint64_t *Z, bool *zplaced, cudaEvent_t *drain0) {
    const uint64_t k = ctrl.k, D = ctrl.D, zmax = D + 16 * k;
    *zplaced = false;
    TRY(ensure_dev(c->zwork, crz_work_bytes(k, D, c->log2S)));
    uint8_t *w = (uint8_t *)c->zwork.p;
    const uint64_t size_tiles = (k + 255) / 256;
    const uint32_t spe = crz_sized_segs(c->log2S);
    const uint64_t warps = (uint64_t)c->sm_count * crz_sized_max_ctas_per_sm() * 8;
    // staged host images: launches of at least 32 MiB of raw payload each (the
    // copy of a piece's streams takes far longer than its encoding)
    uint32_t pieces = 1;
    if (host_res && !direct_flag)
        pieces = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>({(uint64_t)kEncPieces, k, D >> 25}));
    CodecParams P{};
    P.src = (const uint8_t *)c->staging.p;
    P.off = (const uint64_t *)c->off.p;
    P.k = k;
    P.chdr = (const uint64_t *)c->chdr.p;
    P.idx = host_res ? (const uint64_t *)c->idx.p : (const uint64_t *)pc.idx_dev.p;
    P.log2_bpc = c->log2S - 9;
    P.zoff = host_res ? (uint64_t *)c->zoff.p : (uint64_t *)pc.off_dev.p;
    P.zlen = host_res ? (uint64_t *)c->zlen.p : (uint64_t *)pc.zlen_dev.p;
    P.err = (unsigned int *)w;
    P.ticket = (uint32_t *)(w + kZworkTickets);
    P.status = (uint64_t *)(w + kZworkHead);
    P.piece_off = (uint64_t *)(w + kZworkPieceOff);
    P.pieces = pieces;
    P.segs_per_entry = spe;
    P.timeout_ns = c->cfg.timeout_ns;
    P.skip_first_ticket = (size_tiles >= 2 && fault_hit(CRAC_FAULT_ENCODE_WAIT)) ? 1u : 0u;
    uint64_t *out_h = (uint64_t *)((uint8_t *)c->ctrl_h.p + sizeof(CkptCtrl));
    std::memset(out_h, 0, 16 * (1 + kEncPieces));
    CK(cudaMemsetAsync(w, 0, kZworkHead + 8 * size_tiles, s));
    CK(cudaEventRecord(c->ev_t0, s));
    CK(launch_crz_size(P, (int)std::max<uint64_t>(1, std::min<uint64_t>(size_tiles, (uint64_t)c->sm_count * 4)), s));
    CK(cudaEventRecord(c->ev_z0, s));
    CK(launch_report(P.piece_off, pieces + 1, P.err, out_h, s));   // piece offsets, then the error bits
    CK(cudaEventRecord(c->ev_pass, s));
    CK(cudaEventSynchronize(c->ev_pass));
    const unsigned err = (uint32_t)out_h[pieces + 1];
    if (err & kErrTimeout) return CRAC_ERR_TIMEOUT;
    if (err) return CRAC_ERR_CORRUPT;
    for (uint32_t i = 0; i < pieces; ++i)
        if (out_h[i] > out_h[i + 1]) return CRAC_ERR_CORRUPT;
    const uint64_t z_all = out_h[pieces];
    if (out_h[0] != 0 || z_all > zmax) return CRAC_ERR_CORRUPT;
    uint64_t poff[kEncPieces + 1];
    for (uint32_t i = 0; i <= pieces; ++i) poff[i] = out_h[i];
    bool piped = false;
    if (host_res) {
        P.zoff = (uint64_t *)c->zoff.p;
        if (direct_flag && pinned_arena().try_alloc(z_all, &pc.host)) {
            P.dst = pc.host.p;
            *zplaced = true;
        } else {
            TRY(ensure_dev(c->cstage, std::max<uint64_t>(z_all, 16)));
            P.dst = (uint8_t *)c->cstage.p;
            if (pieces > 1 && pinned_arena().alloc(z_all, &pc.host) == CRAC_OK) piped = *zplaced = true;
        }
    } else {
        TRY(device_arena(c->device).alloc(std::max<uint64_t>(z_all, 16), &pc.dev));
        P.dst = pc.dev.p;
    }
    const int grid = (int)std::max<uint64_t>(1, warps / 8);
    CK(cudaEventRecord(c->ev_z1, s));
    for (uint32_t i = 0; i < pieces; ++i) {
        CodecParams Q = P;
        Q.e_begin = k * i / pieces;
        Q.e_end = k * (i + 1) / pieces;
        CK(launch_crz_encode_sized(Q, grid, s));
        if (piped) {
            CK(cudaEventRecord(c->ev_piece[i], s));
            if (poff[i + 1] > poff[i]) {
                CK(cudaStreamWaitEvent(c->side, c->ev_piece[i], 0));
                if (drain0 && *drain0) CK(cudaEventRecord(*drain0, c->side));   // the image's drain starts here
                if (drain0) *drain0 = nullptr;
                CK(cudaMemcpyAsync(pc.host.p + poff[i], c->cstage.p + poff[i], poff[i + 1] - poff[i],
                                   cudaMemcpyDeviceToHost, c->side));
            }
        }
    }
    CK(cudaEventRecord(c->ev_t1, s));
    CK(cudaEventRecord(c->ev_pass, s));
    CK(cudaEventSynchronize(c->ev_pass));
    c->last.kernel_launches += 2 + pieces;
    // device time of the sizing and of the coding (not the host's read of the
    // sizes in between)
    float ms = 0, ms2 = 0;
    if (cudaEventElapsedTime(&ms, c->ev_t0, c->ev_z0) == cudaSuccess &&
        cudaEventElapsedTime(&ms2, c->ev_z1, c->ev_t1) == cudaSuccess)
        c->last.codec_ms += ms + ms2;
    cudaGetLastError();
    *Z = z_all;
    return CRAC_OK;
}

crac_status_t encode_segment(crac_ctx *c, Piece &pc, const CkptCtrl &ctrl, bool host_res, bool direct_flag,
                             cudaStream_t s, uint64_t *Z, bool *zplaced, cudaEvent_t *drain0) {
    if (c->crz_hdr_now) return encode_segment_sized(c, pc, ctrl, host_res, direct_flag, s, Z, zplaced, drain0);
    const uint64_t k = ctrl.k, D = ctrl.D, zmax = D + 16 * k;
    const uint32_t T = crz_tile_entries(c->log2S);
    const uint64_t n_tiles = (k + T - 1) / T;
    if (n_tiles > 0x7fffffffull) return CRAC_ERR_UNSUPPORTED;
    *zplaced = false;
    TRY(ensure_dev(c->zwork, crz_work_bytes(k, D, c->log2S)));
    const int grid_max = (int)std::max<uint64_t>(1, (uint64_t)c->sm_count * crz_encode_max_ctas_per_sm());
    uint32_t pieces = 1;
    CodecParams P{};
    if (host_res) {
        P.zoff = (uint64_t *)c->zoff.p;
        P.zlen = (uint64_t *)c->zlen.p;
        if (direct_flag && pinned_arena().try_alloc(zmax, &pc.host)) {
            P.dst = pc.host.p;
            *zplaced = true;
        } else {
            TRY(ensure_dev(c->cstage, zmax));
            P.dst = (uint8_t *)c->cstage.p;
            // a launch of at least four waves of tiles per piece
            pieces = (uint32_t)std::min<uint64_t>(kEncPieces, n_tiles / (4ull * grid_max));
            if (pieces > 1 && !pinned_arena().try_alloc(zmax, &pc.host)) pieces = 1;
        }
    } else {
        TRY(device_arena(c->device).alloc(zmax, &pc.dev));
        P.dst = pc.dev.p;
        P.zoff = (uint64_t *)pc.off_dev.p;
        P.zlen = (uint64_t *)pc.zlen_dev.p;
    }
    if (pieces < 1) pieces = 1;
    uint8_t *w = (uint8_t *)c->zwork.p;
    P.src = (const uint8_t *)c->staging.p;
    P.off = (const uint64_t *)c->off.p;
    if (c->crz_hdr_now) {   // the pass made the block headers
        P.chdr = (const uint64_t *)c->chdr.p;
        P.idx = host_res ? (const uint64_t *)c->idx.p : (const uint64_t *)pc.idx_dev.p;
        P.log2_bpc = c->log2S - 9;
    }
    P.k = k;
    P.dst_cap = zmax;
    P.err = (unsigned int *)w;
    P.status = (uint64_t *)(w + kZworkHead);
    P.hdr = P.status + n_tiles;
    P.piece_off = (uint64_t *)(w + kZworkPieceOff);
    P.tile_entries = T;
    P.timeout_ns = c->cfg.timeout_ns;
    const bool inject = n_tiles >= 2 && fault_hit(CRAC_FAULT_ENCODE_WAIT);
    // out_h: the total and the error bits; then per piece its end offset and
    // its error bits (16 bytes each)
    uint64_t *out_h = (uint64_t *)((uint8_t *)c->ctrl_h.p + sizeof(CkptCtrl));
    std::memset(out_h, 0, 16 * (1 + kEncPieces));
    CK(cudaMemsetAsync(w, 0, kZworkHead + 8 * n_tiles, s));
    CK(cudaEventRecord(c->ev_t0, s));
    for (uint32_t i = 0; i < pieces; ++i) {
        const uint64_t t0 = n_tiles * i / pieces, t1 = n_tiles * (i + 1) / pieces;
        CodecParams Q = P;
        Q.ticket = (uint32_t *)(w + kZworkTickets) + i;
        Q.tile_begin = (uint32_t)t0;
        Q.n_tiles = (uint32_t)t1;
        Q.skip_first_ticket = (i == 0 && inject) ? 1u : 0u;
        CK(launch_crz_encode(Q, (int)std::min<uint64_t>(t1 - t0, (uint64_t)grid_max), s));
        if (pieces > 1) {   // the piece's end offset and error bits so far
            CK(launch_report(P.zoff + std::min<uint64_t>(k, t1 * T), 1, P.err, out_h + 2 + 2 * i, s));
            CK(cudaEventRecord(c->ev_piece[i], s));
        }
    }
    CK(cudaEventRecord(c->ev_t1, s));
    CK(launch_report(P.zoff + k, 1, P.err, out_h, s));   // the total and the error bits
    CK(cudaEventRecord(c->ev_pass, s));
    c->last.kernel_launches += pieces + (pieces > 1 ? pieces : 0) + 1;
    if (pieces > 1) {
        // Copy each piece's streams once it has ended; a piece with an error,
        // or an end offset out of order, stops the copies (the total's check
        // below reports it).
        uint64_t z0 = 0;
        bool stop = false;
        for (uint32_t i = 0; i < pieces; ++i) {
            CK(cudaEventSynchronize(c->ev_piece[i]));
            const uint64_t z1 = out_h[2 + 2 * i];
            if (stop || (uint32_t)out_h[3 + 2 * i] != 0 || z1 < z0 || z1 > zmax) {
                stop = true;
                continue;
            }
            if (z1 > z0) {
                CK(cudaStreamWaitEvent(c->side, c->ev_piece[i], 0));
                CK(cudaMemcpyAsync(pc.host.p + z0, c->cstage.p + z0, z1 - z0, cudaMemcpyDeviceToHost, c->side));
            }
            z0 = z1;
        }
        *zplaced = true;
    }
    CK(cudaEventSynchronize(c->ev_pass));
    float ms = 0;
    if (cudaEventElapsedTime(&ms, c->ev_t0, c->ev_t1) == cudaSuccess) c->last.codec_ms += ms;
    cudaGetLastError();
    const unsigned err = (uint32_t)out_h[1];
    crac_status_t st = CRAC_OK;
    if (err & kErrLostCopy) {
        c->lost = true;
        st = CRAC_ERR_CUDA;
    } else if (err & kErrTimeout) {
        st = CRAC_ERR_TIMEOUT;
    } else if (err || out_h[0] > zmax) {
        st = CRAC_ERR_CORRUPT;
    }
    if (st != CRAC_OK) {
        // the pinned block goes back with the failed image: no copy may
        // still be writing it
        if (pieces > 1) cudaStreamSynchronize(c->side);
        return st;
    }
    *Z = out_h[0];
    if (*zplaced) pinned_arena().shrink(pc.host, *Z);
    return CRAC_OK;
}

// CRAC_PASS_AUTO: the split pass, unless the last pass with a baseline found
// more than half of the chunks dirty (or, on 512 B - 4 KiB chunks of device
// images, under a quarter); then a pass that reads every byte once
// (at 100% dirty 4 KiB pages and 64 KiB chunks: sparse 0.94, TMA 0.72, LDG
// 0.69, split 0.66 of the HBM peak), the best one the images and sizes allow,
// except for coded images on chunks of 8 KiB and more.
uint32_t resolve_pass_kernel(const crac_ctx *c, bool dev_res, bool all16) {
    const bool coded = (c->cfg.flags & CRAC_FLAG_COMPRESS) != 0;
    // the encoder reads a compact payload, which the sparse pass does not leave
    if (c->cfg.pass_kernel == CRAC_PASS_SPARSE && coded) return CRAC_PASS_SPLIT;
    if (c->cfg.pass_kernel != CRAC_PASS_AUTO) return c->cfg.pass_kernel;
    // 512 B - 4 KiB chunks of device images, after a delta with under a
    // quarter of the chunks dirty: the sparse pass places the dirty chunks
    // densely and reads every byte once (32 GiB at 4 KiB chunks, 10% dirty
    // pages: 0.93 of the HBM peak against the split pass's 0.84).
    if (c->delta_frac_valid && c->delta_frac < 0.25f && dev_res && all16 && !coded && c->log2S >= 9 &&
        c->log2S <= 12 && c->cfg.launch_mode == CRAC_LAUNCH_BATCHED)
        return CRAC_PASS_SPARSE;
    if (!c->delta_frac_valid || c->delta_frac <= 0.5f) return CRAC_PASS_SPLIT;
    // coded images on chunks of 8 KiB and more: the split pass makes the block
    // headers of the two-launch encoder (4 GiB fp32, every chunk dirty: split
    // 2.0 + 2.1 ms, TMA 1.7 + 3.8 ms for the one-launch encoder)
    if (coded && c->log2S >= 13 && c->cfg.launch_mode == CRAC_LAUNCH_BATCHED) return CRAC_PASS_SPLIT;
    if (dev_res && all16 && !coded) return CRAC_PASS_SPARSE;
    if (c->log2S >= 10 && c->log2S <= 16) return CRAC_PASS_TMA;
    return CRAC_PASS_LDG;
}

constexpr size_t kReservedChain = 8;   // images per chain that restart scratch is sized for ahead

// The fingerprint table the next pass writes: neither the current baseline
// nor, while passes are unsettled, the settled state's table.
int spare_fp(const crac_ctx *c) {
    for (int i = 0; i < 3; ++i)
        if (i != c->fp_cur && (c->pending.empty() || i != c->settled.fp)) return i;
    return -1;   // unreachable: at most two tables are in use
}

namespace {

// After a pass that wrote predicted chunks: if fewer than half of those
// writes were found in place, the dirty set does not repeat well enough to
// pay for them; skip the speculative writes for the next passes.
void spec_feedback(crac_ctx *c, uint64_t hits, uint64_t writes) {
    if (writes && 2 * hits < writes) c->spec_rest = 8;
}

// Pass statistics of a settled deferred image, if no later pass has started.
void fill_last(crac_ctx *c, const crac_image *im) {
    if (im->seq != c->pass_seq) return;
    c->last.k = im->k;
    c->last.payload_bytes = im->raw_bytes;
    c->last.stored_bytes = im->payload_bytes;
    c->last.in_place = im->spec_hits;
    float ms = 0;
    c->last.hash_ms = c->last.finalize_ms = c->last.gather_ms = 0;
    pass_timings(c, &ms);
    c->last.device_ms = ms;
    if (c->prefetch_now) {
        float pm = 0;
        if (cudaEventElapsedTime(&pm, c->ev_p0, c->ev_p1) == cudaSuccess) c->last.prefetch_ms = pm;
        cudaGetLastError();
    }
}

// Settle the oldest unsettled image: wait for its pass (and drain) and
// resolve its sizes.  On success the settled state becomes the one after it;
// on failure the context returns to the settled state, so that its baseline
// is as if the failed checkpoint had never been taken, and the later
// unsettled images, which depend on it, fail too.
void settle_front(crac_ctx *c) {
    crac_image *im = c->pending.front();
    c->pending.pop_front();
    const crac_status_t st = img_wait(im, 0);
    crac_ctx::Settled &sd = c->settled;
    if (st == CRAC_OK) {
        sd.fp = im->out_fp;
        sd.valid = true;
        sd.first.clear();
        for (const ImgAlloc &a : im->allocs) sd.first[a.id] = a.first_chunk;
        img_ref(im);
        img_unref(sd.parent);
        sd.parent = im;
        sd.parent_epoch = im->epoch;
        sd.epoch_max = std::max(sd.epoch_max, im->epoch);
        if (im->had_base) {
            c->delta_frac = (float)((double)im->k / (double)std::max<uint64_t>(im->n_chunks, 1));
            c->delta_frac_valid = true;
        }
        spec_feedback(c, im->spec_hits, im->spec_writes);
        fill_last(c, im);
    } else {
        if (im->lost) c->lost = true;
        c->ppos_ok = false;
        c->fp_cur = sd.fp;
        c->base_valid = sd.valid;
        c->base_first = sd.first;
        img_ref(sd.parent);
        img_unref(c->parent);
        c->parent = sd.parent;
        c->parent_epoch = sd.parent_epoch;
        c->epoch_max = sd.epoch_max;
        for (crac_image *r : c->pending) img_unref(r);   // they fail through their dep link
        c->pending.clear();
    }
    img_unref(im);
    if (c->pending.empty()) {   // the snapshot is only needed while passes are unsettled
        img_unref(sd.parent);
        sd.parent = nullptr;
    }
}

}  // namespace

// Settle unsettled checkpoints: all of them (block), or those whose work has
// already completed.  A failed image reports its own error; settling it only
// reverts the context, so this returns CRAC_OK.
crac_status_t ctx_settle(crac_ctx *c, bool block) {
    while (!c->pending.empty()) {
        if (!block) {
            const cudaError_t e = cudaEventQuery(c->pending.front()->done);
            if (e == cudaErrorNotReady) break;
            cudaGetLastError();
        }
        settle_front(c);
    }
    return CRAC_OK;
}

// The passes of a checkpoint that waits for each segment's dirty counts:
// several staging segments, coded images or per-allocation launches.  Each
// segment is enqueued, waited for, sized and drained (A2-A5) before the
// next; on return the image's sizes are known.
crac_status_t checkpoint_wait(crac_ctx *c, crac_image *im, const std::vector<Segment> &segs,
                              const std::vector<uint64_t> &first, int out_fp, bool direct, bool direct_flag,
                              bool coded, cudaStream_t s) {
    Arena &pa = pinned_arena();
    Arena &da = device_arena(c->device);
    const bool host_res = c->cfg.image_residency == CRAC_RESIDENCY_HOST;
    const uint64_t n = im->n_chunks;
    crac_status_t st = CRAC_OK;
    uint64_t k_base = 0, d_base = 0, raw_base = 0;
    float ms = 0;
    bool drain_started = false;   // drain0 recorded (host images)
    for (const Segment &sg : segs) {
        const uint64_t nseg = sg.c1 - sg.c0;
        Piece pc;
        uint64_t *idx_d = (uint64_t *)c->idx.p, *off_d = (uint64_t *)c->off.p;
        uint8_t *stg = (uint8_t *)c->staging.p;
        if (!host_res) {
            // coded: pc.dev is sized by the encoder, after the pass
            if (!coded) st = da.alloc(sg.bytes, &pc.dev);
            if (st == CRAC_OK) st = da.alloc(nseg * 8, &pc.idx_dev);
            if (st == CRAC_OK) st = da.alloc((nseg + 1) * 8, &pc.off_dev);
            if (st == CRAC_OK && coded) st = da.alloc(nseg * 8, &pc.zlen_dev);
            if (st != CRAC_OK) {
                im->pieces.push_back(pc);
                return st;
            }
            idx_d = (uint64_t *)pc.idx_dev.p;
            if (!coded) {
                off_d = (uint64_t *)pc.off_dev.p;
                stg = pc.dev.p;
            }
        }
        // The worst-case block comes from the pinned regions as they are
        // (growing them, or starting their background growth, mid-loop
        // would stall the device); without room this segment drains
        // through staging.  The unused tail is returned after the pass.
        const bool direct_seg = direct && pa.try_alloc(sg.bytes, &pc.host);
        if (direct_seg) stg = pc.host.p;
        if (cudaStreamWaitEvent(s, c->ev_last, 0) != cudaSuccess) {
            im->pieces.push_back(pc);
            return cuda_status(cudaGetLastError());
        }
        CkptCtrl ctrl{};
        st = run_segment(c, sg, (const CkptDesc *)c->desc.p, first, idx_d, off_d, nseg, stg, sg.bytes, out_fp, s,
                         &ctrl, &ms);
        if (st != CRAC_OK) {
            im->pieces.push_back(pc);
            return st;
        }
        spec_feedback(c, ctrl.spec_hits, ctrl.spec_writes);
        c->last.in_place += ctrl.spec_hits;
        pc.k0 = k_base;
        pc.k = ctrl.k;
        pc.off0 = d_base;
        const bool sparse = c->sparse_ok && !host_res;
        pc.bytes = sparse ? ctrl.payload : ctrl.D;
        pc.span = sparse ? ctrl.D : 0;
        bool zplaced = false;
        if (coded && ctrl.k) {
            uint64_t Z = 0;
            cudaEvent_t d0 = drain_started || !host_res ? nullptr : im->drain0;
            st = encode_segment(c, pc, ctrl, host_res, direct_flag, s, &Z, &zplaced, &d0);
            if (host_res && !d0) drain_started = true;   // recorded as the first copy was issued
            if (st != CRAC_OK) {
                im->pieces.push_back(pc);
                return st;
            }
            pc.bytes = Z;
        }
        raw_base += sparse ? ctrl.payload : ctrl.D;
        if (fault_hit(CRAC_FAULT_DRAIN)) {
            im->pieces.push_back(pc);
            t_last_cuda = (int)cudaErrorLaunchFailure;
            return CRAC_ERR_CUDA;
        }
        cudaError_t e = cudaStreamWaitEvent(c->side, c->ev_pass, 0);
        if (e == cudaSuccess && host_res && !drain_started) e = cudaEventRecord(im->drain0, c->side);
        drain_started = true;
        if (direct_seg) {
            if (ctrl.D) pa.shrink(pc.host, ctrl.D);
            else pa.free(pc.host);
        } else if (host_res) {
            if (pc.bytes && !zplaced) {
                st = pa.alloc(pc.bytes, &pc.host);
                if (st != CRAC_OK) {
                    im->pieces.push_back(pc);
                    return st;
                }
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(pc.host.p, coded ? c->cstage.p : c->staging.p, pc.bytes,
                                        cudaMemcpyDeviceToHost, c->side);
            }
        } else {
            da.shrink(pc.dev, coded ? pc.bytes : ctrl.D);   // sparse: the span
            da.shrink(pc.idx_dev, ctrl.k * 8);
            da.shrink(pc.off_dev, (ctrl.k + 1) * 8);
            if (coded) da.shrink(pc.zlen_dev, ctrl.k * 8);
        }
        if (e == cudaSuccess && ctrl.k && host_res)
            e = link_copy(c, im->idx_h.p + k_base * 8, idx_d, ctrl.k * 8, cudaMemcpyDeviceToHost, c->side);
        if (e == cudaSuccess && ctrl.k && host_res && coded)
            e = link_copy(c, im->zlen_h.p + k_base * 8, c->zlen.p, ctrl.k * 8, cudaMemcpyDeviceToHost, c->side);
        if (e == cudaSuccess) e = cudaEventRecord(c->ev_last, c->side);
        im->pieces.push_back(pc);
        if (e != cudaSuccess) return cuda_status(e);
        k_base += ctrl.k;
        d_base += pc.bytes;
    }
    cudaError_t e;
    if (host_res) {
        e = link_copy(c, im->fp_h.p, c->fp[out_fp].p, n * 8, cudaMemcpyDeviceToHost, c->side);
        if (e == cudaSuccess) e = cudaEventRecord(im->done, c->side);
        if (e == cudaSuccess) e = cudaEventRecord(c->ev_last, c->side);
    } else {
        // Device image: its tables stay in device memory; done once the
        // fingerprint table has its own copy.
        e = cudaMemcpyAsync(im->fp_dev.p, c->fp[out_fp].p, n * 8, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaEventRecord(im->done, s);
        if (e == cudaSuccess) e = cudaEventRecord(c->ev_last, s);
    }
    if (e != cudaSuccess) return cuda_status(e);
    im->k = k_base;
    im->payload_bytes = d_base;
    im->raw_bytes = raw_base;
    if (host_res) pa.shrink(im->idx_h, k_base * 8);
    if (host_res && coded) pa.shrink(im->zlen_h, k_base * 8);
    c->last.k = k_base;
    c->last.payload_bytes = raw_base;
    c->last.stored_bytes = d_base;
    c->last.segments = (uint32_t)segs.size();
    c->last.device_ms = ms;
    if (c->prefetch_now) {
        float pm = 0;
        cudaEventElapsedTime(&pm, c->ev_p0, c->ev_p1);
        c->last.prefetch_ms = pm;
    }
    return CRAC_OK;
}

// A single-segment pass into uncoded images, enqueued and not waited for
// (A2-A5).  Its control block lands in the image's pinned ctrl_b; a device
// image's payload, chunk list and offsets go to worst-case blocks of the
// device arena, a host image's payload to the pinned block in pieces[0] (the
// pass writes it there directly, or drain_kernel on the side stream copies
// it from staging, reading the sizes from the control block; SM stores, not
// a copy engine, whose device-to-host rate was seen to collapse).  The blocks
// are shrunk to the counts, and the counts become the image's, when the
// image settles.
crac_status_t checkpoint_enqueue(crac_ctx *c, crac_image *im, const Segment &sg, const std::vector<uint64_t> &first,
                                 int out_fp, bool direct, bool any_base, cudaStream_t s) {
    Arena &pa = pinned_arena();
    Arena &da = device_arena(c->device);
    const bool host_res = c->cfg.image_residency == CRAC_RESIDENCY_HOST;
    const uint64_t n = im->n_chunks;
    if (im->pieces.empty()) im->pieces.push_back(Piece{});
    Piece &pc = im->pieces[0];
    uint64_t *idx_d = (uint64_t *)c->idx.p, *off_d = (uint64_t *)c->off.p;
    uint8_t *stg = (uint8_t *)c->staging.p;
    if (!host_res) {
        TRY(da.alloc(sg.bytes, &pc.dev));
        TRY(da.alloc(n * 8, &pc.idx_dev));
        TRY(da.alloc((n + 1) * 8, &pc.off_dev));
        idx_d = (uint64_t *)pc.idx_dev.p;
        off_d = (uint64_t *)pc.off_dev.p;
        stg = pc.dev.p;
    } else if (direct) {
        stg = pc.host.p;
    }
    TRY(pa.alloc(sizeof(CkptCtrl), &im->ctrl_b));
    CK(cudaStreamWaitEvent(s, c->ev_last, 0));
    TRY(launch_segment(c, sg, (const CkptDesc *)c->desc.p, first, idx_d, off_d, n, stg, sg.bytes, out_fp,
                       im->ctrl_b.p, s));
    if (fault_hit(CRAC_FAULT_DRAIN)) {
        t_last_cuda = (int)cudaErrorLaunchFailure;
        return CRAC_ERR_CUDA;
    }
    if (host_res) {
        CK(cudaStreamWaitEvent(c->side, c->ev_pass, 0));
        CK(cudaEventRecord(im->drain0, c->side));
        // FULL or delta alike: the sizes come from the control block, the
        // bytes cross by SM stores into the pinned blocks (this path requires
        // the device mapping of pinned memory)
        CK(launch_drain((const CkptCtrl *)c->work.p, direct ? nullptr : (const uint8_t *)c->staging.p, pc.host.p,
                        sg.bytes, idx_d, (uint64_t *)im->idx_h.p, n, c->sm_count * 2, c->side));
        CK(link_copy(c, im->fp_h.p, c->fp[out_fp].p, n * 8, cudaMemcpyDeviceToHost, c->side));
        CK(cudaEventRecord(im->done, c->side));
        CK(cudaEventRecord(c->ev_last, c->side));
    } else {
        CK(cudaMemcpyAsync(im->fp_dev.p, c->fp[out_fp].p, n * 8, cudaMemcpyDeviceToDevice, s));
        CK(cudaEventRecord(im->done, s));
        CK(cudaEventRecord(c->ev_last, s));
    }
    pc.k0 = 0;
    pc.off0 = 0;
    im->deferred = true;
    im->sparse_pass = c->sparse_ok && !host_res;
    im->predicted_full = !any_base;
    c->last.segments = 1;
    return CRAC_OK;
}

crac_status_t ctx_checkpoint(crac_ctx *c, cudaStream_t s, crac_image_t **out) {
    if (!out) return CRAC_ERR_INVALID_ARG;
    *out = nullptr;
    DeviceGuard g(c->device);
    if (!s) CK(cudaDeviceSynchronize());   // the paper's queue drain before a checkpoint
    const size_t na = c->allocs.size();
    const uint32_t log2S = c->log2S;
    const uint64_t S = 1ull << log2S;
    std::vector<uint64_t> first(na + 1, 0);
    uint64_t tracked = 0;
    for (size_t a = 0; a < na; ++a) {
        first[a + 1] = first[a] + ((c->allocs[a].bytes + S - 1) >> log2S);
        tracked += c->allocs[a].bytes;
    }
    const uint64_t n = first[na];
    for (const AllocRec &r : c->allocs)   // host memory is read through its device mapping
        if (r.kind == CRAC_KIND_HOST && !c->uva) return CRAC_ERR_UNSUPPORTED;
    const bool dev_res = c->cfg.image_residency == CRAC_RESIDENCY_DEVICE;
    const bool host_res = !dev_res;
    // Coded images: the pass gathers into device staging as usual and the
    // encoder writes the streams (encode_segment).
    const bool coded = (c->cfg.flags & CRAC_FLAG_COMPRESS) != 0;
    // Segments bounded by the staging capacity.
    uint64_t cap = c->cfg.staging_bytes ? c->cfg.staging_bytes : std::min(tracked, kDefaultStagingMax);
    cap = std::max(round_up(cap, 256), S);
    // Coded images: the encoder's aligned bulk reads may pass the end of the
    // payload by up to 15 bytes, so with a given staging capacity (a
    // configured one, or a server lease that cannot grow) the segments leave
    // 256 bytes of it free.
    if (coded && c->cfg.staging_bytes && cap >= S + 256) cap -= 256;
    const std::vector<Segment> segs = make_segments(c->allocs, first, log2S, cap);
    uint64_t max_seg_chunks = 0, max_seg_bytes = 0;
    for (const Segment &sg : segs) {
        max_seg_chunks = std::max(max_seg_chunks, sg.c1 - sg.c0);
        max_seg_bytes = std::max(max_seg_bytes, sg.bytes);
    }
    Arena &pa = pinned_arena();
    Arena &da = device_arena(c->device);

    // A single-segment batched pass into uncoded images is not waited for:
    // the call returns once it is enqueued, and the image's sizes are settled
    // when its work has completed (img_resolve).  Every other pass waits for
    // the dirty counts of each segment before the next one.  At most two
    // checkpoints stay unsettled; earlier ones whose work has completed are
    // settled here, and all of them before a pass that waits.
    bool defer = n > 0 && segs.size() == 1 && !coded && c->cfg.launch_mode == CRAC_LAUNCH_BATCHED &&
                 (dev_res || c->uva) && !(c->cfg.flags & CRAC_FLAG_WAIT_PASS);
    TRY(ctx_settle(c, false));
    while (c->pending.size() >= 2) settle_front(c);
    // Which chunks have a baseline (no settling after this point may move it).
    auto base_of = [&](size_t a) {
        if (!c->base_valid) return kNoBase;
        auto it = c->base_first.find(c->allocs[a].id);
        return it == c->base_first.end() ? kNoBase : it->second;
    };
    bool any_base = false;
    for (size_t a = 0; a < na; ++a) any_base |= base_of(a) != kNoBase;
    // A host image's payload block is taken before the pass: the whole
    // segment for a FULL pass (its size is known), else the worst case from
    // the pinned regions as they are (growing them mid-loop would stall the
    // device); without room the pass waits instead.
    Piece dpc;
    if (defer && host_res) {
        if (!any_base) {
            if (pa.alloc(segs[0].bytes, &dpc.host) != CRAC_OK) defer = false;
        } else if (!pa.try_alloc(segs[0].bytes, &dpc.host)) {
            defer = false;
        }
    }
    if (!defer) {
        pa.free(dpc.host);
        TRY(ctx_settle(c, true));
        any_base = false;
        for (size_t a = 0; a < na; ++a) any_base |= base_of(a) != kNoBase;
    }
    c->last = crac_pass_info_t{};
    c->last.tracked_bytes = tracked;
    c->last.n_chunks = n;

    std::unique_ptr<crac_image> im(new crac_image());
    im->device = c->device;
    im->chunk_bytes = (uint32_t)S;
    im->residency = c->cfg.image_residency;
    im->lineage = c->lineage;
    im->epoch = c->epoch_max + 1;
    im->parent_epoch = c->parent_epoch;
    im->n_chunks = n;
    im->allocs.resize(na);
    for (size_t a = 0; a < na; ++a)
        im->allocs[a] = ImgAlloc{c->allocs[a].id, c->allocs[a].ptr, c->allocs[a].bytes, c->allocs[a].kind, first[a]};
    // done and drain0 time the drain of a host image (crac_image_info_t.drain_ms)
    if (cudaEventCreate(&im->done) != cudaSuccess ||
        (host_res && cudaEventCreate(&im->drain0) != cudaSuccess)) {
        pa.free(dpc.host);
        return cuda_status(cudaGetLastError());
    }
    crac_status_t st = CRAC_OK;
    auto fail = [&](crac_status_t code) {
        cudaStreamSynchronize(s);
        cudaStreamSynchronize(c->side);
        cudaGetLastError();
        free_image_blocks(im.release());
        c->ppos_ok = false;   // a failed pass's offsets predict nothing
        return code;
    };
    if (dpc.host.region >= 0) im->pieces.push_back(dpc);   // freed with the image on failure

    im->host_tables = !dev_res;
    int out_fp = c->fp_cur;
    if (n > 0) {
        if (dev_res) {
            st = da.alloc(n * 8, &im->fp_dev);
        } else {
            st = pa.alloc(n * 8, &im->fp_h);
            if (st == CRAC_OK) st = pa.alloc(n * 8, &im->idx_h);
        }
        if (st != CRAC_OK) return fail(st);
        // fingerprint tables and descriptors
        // Only the output table may grow: the baseline table keeps the previous
        // layout, which it still fully holds.
        out_fp = spare_fp(c);
        // Two pinned descriptor buffers in turn: an unsettled pass's copy may
        // not have run yet when the next pass writes its own.
        HostBuf &dbuf = c->desc_flip ? c->desc_h2 : c->desc_h;
        c->desc_flip ^= 1;
        // Tables grow together, so that a steady checkpoint loop allocates
        // nothing (allocating may synchronize the device): every fingerprint
        // table that holds nothing still needed (not the baseline, not the
        // settled state's) and both descriptor buffers (growing one in use
        // waits for its copy).
        for (int t = 0; t < 3 && st == CRAC_OK; ++t)
            if (t == out_fp || !c->fp[t].p || (t != c->fp_cur && (c->pending.empty() || t != c->settled.fp)))
                st = ensure_dev(c->fp[t], n * 8);   // (a table never allocated holds nothing either)
        if (st == CRAC_OK) st = ensure_dev(c->desc, na * (sizeof(CkptDesc) + 8));
        if (st == CRAC_OK) st = ensure_host(c->desc_h, na * (sizeof(CkptDesc) + 8));
        if (st == CRAC_OK) st = ensure_host(c->desc_h2, na * (sizeof(CkptDesc) + 8));
        if (st != CRAC_OK) return fail(st);
        CkptDesc *dh = (CkptDesc *)dbuf.p;
        uint64_t *prefix_h = (uint64_t *)(dh + na);   // payload bytes before each allocation
        bool all16 = true;
        uint64_t pre = 0;
        for (size_t a = 0; a < na; ++a) {
            all16 &= (c->allocs[a].bytes & 15) == 0;
            dh[a] = CkptDesc{c->allocs[a].ptr, c->allocs[a].bytes, first[a], base_of(a)};
            prefix_h[a] = pre;
            pre += c->allocs[a].bytes;
        }
        c->full_copy_ok = !any_base && all16;
        c->pass_now = resolve_pass_kernel(c, dev_res, all16);
        c->sparse_ok = c->pass_now == CRAC_PASS_SPARSE && dev_res && all16 &&
                       c->cfg.launch_mode == CRAC_LAUNCH_BATCHED;
        // Dense placement takes one atomic on a single counter per warp
        // iteration with dirty chunks, whose rate bounds it once many chunks
        // are dirty: only after a delta that found under a quarter dirty.
        c->dense_now = c->sparse_ok && any_base && c->delta_frac_valid && c->delta_frac < 0.25f;
        // Order after the previous operation of this context (drain / restore).
        if (cudaStreamWaitEvent(s, c->ev_last, 0) != cudaSuccess) return fail(cuda_status(cudaGetLastError()));
        if (link_copy(c, c->desc.p, dh, na * (sizeof(CkptDesc) + 8), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return fail(cuda_status(cudaGetLastError()));
        // Managed regions migrate to the device before they are read.
        bool any_managed = false;
        for (const AllocRec &r : c->allocs) any_managed |= r.kind == CRAC_KIND_MANAGED;
        c->prefetch_now = any_managed;
        if (any_managed) {
            cudaEventRecord(c->ev_p0, s);
            cudaMemLocation loc{};
            loc.type = cudaMemLocationTypeDevice;
            loc.id = c->device;
            for (const AllocRec &r : c->allocs) {
                if (r.kind != CRAC_KIND_MANAGED) continue;
                cudaError_t e = cudaMemPrefetchAsync((const void *)r.ptr, r.bytes, loc, 0, s);
                if (e != cudaSuccess) return fail(cuda_status(e));
            }
            cudaEventRecord(c->ev_p1, s);
        }
        // Direct drain: the pass (uncoded) or the encoder (coded) writes the
        // payload straight into the image's pinned block through its device
        // mapping (not the TMA pass, whose bulk stores stay within device
        // memory).
        const bool direct_flag = host_res && c->uva && (c->cfg.flags & CRAC_FLAG_DIRECT_DRAIN);
        const bool direct = direct_flag && !coded && c->pass_now != CRAC_PASS_TMA;
        if (host_res || coded) {
            // coded: + the 16-byte slack of the encoder's aligned bulk reads
            st = ensure_dev(c->staging, max_seg_bytes + (coded ? 16 : 0));   // also the direct drain's fallback
            if (st == CRAC_OK) st = ensure_dev(c->idx, max_seg_chunks * 8);
            if (st == CRAC_OK) st = ensure_dev(c->off, (max_seg_chunks + 1) * 8);
            if (st != CRAC_OK) return fail(st);
        }
        // The split pass writes the CRZ1 block headers of chunks of 8 KiB and
        // more (one word per 512 bytes) for the encoder.
        c->crz_hdr_now = coded && log2S >= 13 && c->cfg.launch_mode == CRAC_LAUNCH_BATCHED &&
                         c->pass_now == CRAC_PASS_SPLIT;
        if (c->crz_hdr_now) {
            st = ensure_dev(c->chdr, (n << (log2S - 9)) * 8);
            if (st != CRAC_OK) return fail(st);
        }
        if (coded) {
            st = ensure_dev(c->zwork, crz_work_bytes(max_seg_chunks, max_seg_bytes, log2S));
            if (st == CRAC_OK && host_res) st = ensure_dev(c->zoff, (max_seg_chunks + 1) * 8);
            if (st == CRAC_OK && host_res) st = ensure_dev(c->zlen, max_seg_chunks * 8);
            if (st == CRAC_OK && host_res && !direct_flag)
                st = ensure_dev(c->cstage, max_seg_bytes + 16 * max_seg_chunks);
            if (st == CRAC_OK && host_res) st = pa.alloc(n * 8, &im->zlen_h);
            if (st != CRAC_OK) return fail(st);
        }
        // Predicted write-through: a single-segment split pass records its
        // offsets, and uses the previous one's if the layout is unchanged and
        // its staging is device memory (speculative writes over the host link
        // would cost link time).
        c->spec_now = segs.size() == 1 && c->cfg.launch_mode == CRAC_LAUNCH_BATCHED &&
                      c->pass_now == CRAC_PASS_SPLIT && !c->sparse_ok;
        c->spec_use = c->spec_now && c->ppos_ok && c->ppos_layout == c->layout_version && !c->full_copy_ok &&
                      !direct && c->spec_rest == 0;
        if (c->spec_now && c->ppos_ok && !c->full_copy_ok && c->spec_rest) --c->spec_rest;
        if (c->spec_now) {
            st = ensure_dev(c->ppos[0], n * 8);
            if (st == CRAC_OK) st = ensure_dev(c->ppos[1], n * 8);
            if (st != CRAC_OK) return fail(st);
        } else {
            c->ppos_ok = false;
        }
        // A restart of a chain of up to kReservedChain images of this layout
        // finds its scratch ready.
        if (c->uva && (dev_res || !(c->cfg.flags & CRAC_FLAG_STAGED_RESTORE)))
            st = reserve_restart(c, n, na * kReservedChain, segs.size() * kReservedChain);
        if (st != CRAC_OK) return fail(st);
        if (defer) {
            st = checkpoint_enqueue(c, im.get(), segs[0], first, out_fp, direct, any_base, s);
            if (st != CRAC_OK) return fail(st);
        } else {
            st = checkpoint_wait(c, im.get(), segs, first, out_fp, direct, direct_flag, coded, s);
            if (st != CRAC_OK) return fail(st);
            if (any_base) {
                c->delta_frac = (float)((double)im->k / (double)n);
                c->delta_frac_valid = true;
            }
        }
    } else {
        CK(cudaEventRecord(im->done, s));
    }

    // Commit: the new fingerprints become the baseline (for an unsettled
    // pass, provisionally: a failure found when it settles reverts this).
    im->flags = (im->deferred ? (any_base ? 0u : CRAC_IMAGE_FULL) : (im->k == n ? CRAC_IMAGE_FULL : 0u)) |
                (coded ? CRAC_IMAGE_CODED : 0u);
    if (!(im->flags & CRAC_IMAGE_FULL) && c->parent) {   // an unsettled delta drops it if it turns out FULL
        img_ref(c->parent);
        im->parent = c->parent;
    }
    im->seq = ++c->pass_seq;
    if (im->deferred) {
        crac_ctx::Settled &sd = c->settled;
        if (c->pending.empty()) {   // the state a failure of this pass reverts to
            sd.fp = c->fp_cur;
            sd.valid = c->base_valid;
            sd.first = c->base_first;
            img_ref(c->parent);
            img_unref(sd.parent);
            sd.parent = c->parent;
            sd.parent_epoch = c->parent_epoch;
            sd.epoch_max = c->epoch_max;
        } else {
            im->dep = c->pending.back();
            img_ref(im->dep);
        }
        im->out_fp = out_fp;
        im->had_base = any_base;
    }
    c->fp_cur = out_fp;
    c->base_first.clear();
    for (size_t a = 0; a < na; ++a) c->base_first[c->allocs[a].id] = first[a];
    c->base_valid = true;
    c->epoch_max = im->epoch;
    c->parent_epoch = im->epoch;
    crac_image *img = im.release();
    img->refs.store(img->deferred ? 3 : 2);   // the caller's, the context's (and the unsettled list's)
    img_unref(c->parent);
    c->parent = img;
    table_add(img);
    if (img->deferred) c->pending.push_back(img);
    *out = img;
    return CRAC_OK;
}

// ---------------------------------------------------------------------------
// Trial passes (the autotuner's observations)
// ---------------------------------------------------------------------------

// The checkpoint pass without an image: fingerprints, dirty test, compaction
// and gather into the context's staging, segment by segment.  With commit the
// new fingerprints become the context's baseline.
crac_status_t ctx_trial_pass(crac_ctx *c, cudaStream_t s, bool commit, float *ms, uint64_t *k_out,
                             uint64_t *d_out) {
    TRY(ctx_cuda_ready(c));
    DeviceGuard g(c->device);
    const size_t na = c->allocs.size();
    const uint32_t log2S = c->log2S;
    const uint64_t S = 1ull << log2S;
    std::vector<uint64_t> first(na + 1, 0);
    uint64_t tracked = 0;
    for (size_t a = 0; a < na; ++a) {
        first[a + 1] = first[a] + ((c->allocs[a].bytes + S - 1) >> log2S);
        tracked += c->allocs[a].bytes;
    }
    const uint64_t n = first[na];
    *ms = 0;
    *k_out = 0;
    *d_out = 0;
    for (const AllocRec &r : c->allocs)
        if (r.kind == CRAC_KIND_HOST && !c->uva) return CRAC_ERR_UNSUPPORTED;
    TRY(ctx_settle(c, true));
    c->last = crac_pass_info_t{};
    ++c->pass_seq;
    c->spec_now = c->spec_use = false;
    c->ppos_ok = false;
    c->crz_hdr_now = false;
    if (n == 0) return CRAC_OK;
    const int out_fp = spare_fp(c);
    TRY(ensure_dev(c->fp[out_fp], n * 8));
    TRY(ensure_dev(c->desc, na * (sizeof(CkptDesc) + 8)));
    TRY(ensure_host(c->desc_h, na * (sizeof(CkptDesc) + 8)));
    CkptDesc *dh = (CkptDesc *)c->desc_h.p;
    uint64_t *prefix_h = (uint64_t *)(dh + na);
    bool any_base = false, all16 = true;
    uint64_t pre = 0;
    for (size_t a = 0; a < na; ++a) {
        uint64_t bf = kNoBase;
        if (c->base_valid) {
            auto it = c->base_first.find(c->allocs[a].id);
            if (it != c->base_first.end()) bf = it->second;
        }
        any_base |= bf != kNoBase;
        all16 &= (c->allocs[a].bytes & 15) == 0;
        dh[a] = CkptDesc{c->allocs[a].ptr, c->allocs[a].bytes, first[a], bf};
        prefix_h[a] = pre;
        pre += c->allocs[a].bytes;
    }
    c->full_copy_ok = !any_base && all16;
    // Trial passes run the configured kernel; AUTO is the split pass here, so
    // that the tuner's observations of different sizes are comparable.
    c->pass_now = c->cfg.pass_kernel == CRAC_PASS_AUTO ? (uint32_t)CRAC_PASS_SPLIT : c->cfg.pass_kernel;
    c->sparse_ok = c->pass_now == CRAC_PASS_SPARSE && c->cfg.image_residency == CRAC_RESIDENCY_DEVICE &&
                   all16 && c->cfg.launch_mode == CRAC_LAUNCH_BATCHED;
    c->dense_now = c->sparse_ok && any_base && c->dense_hint;
    CK(cudaStreamWaitEvent(s, c->ev_last, 0));
    CK(link_copy(c, c->desc.p, dh, na * (sizeof(CkptDesc) + 8), cudaMemcpyHostToDevice, s));
    uint64_t cap = c->cfg.staging_bytes ? c->cfg.staging_bytes : std::min(tracked, kDefaultStagingMax);
    cap = std::max(round_up(cap, 256), S);
    const std::vector<Segment> segs = make_segments(c->allocs, first, log2S, cap);
    uint64_t max_c = 0, max_b = 0;
    for (const Segment &sg : segs) {
        max_c = std::max(max_c, sg.c1 - sg.c0);
        max_b = std::max(max_b, sg.bytes);
    }
    TRY(ensure_dev(c->staging, max_b));
    TRY(ensure_dev(c->idx, max_c * 8));
    TRY(ensure_dev(c->off, (max_c + 1) * 8));
    for (const Segment &sg : segs) {
        CkptCtrl ctrl{};
        TRY(run_segment(c, sg, (const CkptDesc *)c->desc.p, first, (uint64_t *)c->idx.p, (uint64_t *)c->off.p,
                        sg.c1 - sg.c0, (uint8_t *)c->staging.p, sg.bytes, out_fp, s, &ctrl, ms));
        *k_out += ctrl.k;
        *d_out += c->sparse_ok ? ctrl.payload : ctrl.D;
    }
    CK(cudaEventRecord(c->ev_last, s));
    if (commit) {
        c->prev_base_first = c->base_first;
        c->prev_base_valid = c->base_valid;
        c->prev_fp = c->fp_cur;
        c->fp_cur = out_fp;
        c->base_first.clear();
        for (size_t a = 0; a < na; ++a) c->base_first[c->allocs[a].id] = first[a];
        c->base_valid = true;
    }
    return CRAC_OK;
}

// Fingerprints of the registered allocations' current contents, each tested
// against fp_ref[global chunk id] (the split pass's hash and finalize kernels
// over every chunk, without a gather): *fp_out receives the fingerprints,
// and *ctrl_out is the device control block whose k and D count the chunks
// that differ and their bytes.  Enqueued on s; the caller reads the results
// after the stream reaches them.  Incremental restore runs this first.
crac_status_t fingerprint_against(crac_ctx *c, const uint64_t *fp_ref, cudaStream_t s, const uint64_t **fp_out,
                                  const CkptCtrl **ctrl_out) {
    const size_t na = c->allocs.size();
    const uint32_t log2S = c->log2S;
    const uint64_t S = 1ull << log2S;
    std::vector<uint64_t> first(na + 1, 0);
    for (size_t a = 0; a < na; ++a) first[a + 1] = first[a] + ((c->allocs[a].bytes + S - 1) >> log2S);
    const uint64_t n = first[na];
    const uint32_t cptF = (uint32_t)split_finalize_threads();
    const uint64_t n_tiles = (n + cptF - 1) / cptF;
    if (n_tiles > 0x7fffffffull) return CRAC_ERR_UNSUPPORTED;
    const size_t status_bytes = sizeof(CkptCtrl) + 16 * n_tiles;
    const size_t work_bytes = status_bytes + 8 * n;
    TRY(ensure_dev(c->vdesc, std::max<size_t>(na, 1) * sizeof(CkptDesc)));
    TRY(ensure_host(c->vdesc_h, std::max<size_t>(na, 1) * sizeof(CkptDesc)));
    TRY(ensure_dev(c->vwork, work_bytes));
    TRY(ensure_dev(c->vfp, std::max<uint64_t>(n, 1) * 8));
    TRY(ensure_dev(c->vidx, std::max<uint64_t>(n, 1) * 8));
    TRY(ensure_dev(c->voff, (n + 1) * 8));
    CkptDesc *dh = (CkptDesc *)c->vdesc_h.p;
    for (size_t a = 0; a < na; ++a)   // the reference table has the same chunk layout
        dh[a] = CkptDesc{c->allocs[a].ptr, c->allocs[a].bytes, first[a], first[a]};
    CK(link_copy(c, c->vdesc.p, dh, na * sizeof(CkptDesc), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(c->vwork.p, 0, work_bytes, s));
    const bool small = log2S >= 9 && log2S < 13;
    uint32_t log2Seg = std::min<uint32_t>(log2S, 13);
    const void *hash_fn = small ? split_hash_small_fn(1 << (log2S - 8)) : split_hash_fn();
    CkptParams P{};
    P.desc = (const CkptDesc *)c->vdesc.p;
    P.n_allocs = (uint32_t)na;
    P.log2_chunk = log2S;
    P.c_begin = 0;
    P.c_end = n;
    P.cpt = cptF;
    P.n_tiles = (uint32_t)n_tiles;
    P.fp_old = fp_ref;
    P.fp_new = (uint64_t *)c->vfp.p;
    P.idx_out = (uint64_t *)c->vidx.p;
    P.off_out = (uint64_t *)c->voff.p;
    P.idx_cap = n;
    P.ctrl = (CkptCtrl *)c->vwork.p;
    P.tile_cnt = (uint64_t *)((uint8_t *)c->vwork.p + sizeof(CkptCtrl));
    P.tile_bytes = P.tile_cnt + n_tiles;
    P.timeout_ns = c->cfg.timeout_ns;
    unsigned long long *acc = (unsigned long long *)((uint8_t *)c->vwork.p + status_bytes);
    const uint64_t n_slots = small ? (n + (8192u >> log2S) - 1) / (8192u >> log2S) : n << (log2S - log2Seg);
    const int gh = (int)std::max<uint64_t>(1, std::min<uint64_t>(
                       (n_slots + 7) / 8, (uint64_t)c->sm_count * split_max_ctas_per_sm(hash_fn, split_hash_threads())));
    const int gf = (int)std::max<uint64_t>(1, std::min<uint64_t>(n_tiles, (uint64_t)c->sm_count * 2));
    void *args[] = {&P, &acc, &log2Seg};
    CK(cudaLaunchKernel(hash_fn, dim3(gh), dim3(split_hash_threads()), args, 0, s));
    CK(cudaLaunchKernel(split_finalize_fn(), dim3(gf), dim3(split_finalize_threads()), args, 0, s));
    count_launches(2);
    *fp_out = (const uint64_t *)c->vfp.p;
    *ctrl_out = P.ctrl;
    return CRAC_OK;
}

}  // namespace crac
