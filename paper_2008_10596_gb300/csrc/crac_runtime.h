// Internal declarations shared by the host runtime's translation units (not
// part of the C ABI): the arenas, the image and context records, and the
// functions one unit calls in another.
//
// The paper keeps its own table of active cudaMalloc-family allocations
// (only the pointers the app got back, not the library's arenas) and saves
// exactly those buffers (Sec. 3.2, "Issue of library-allocated memory" and
// "Saving the library-allocated arena").  Restart copies the saved bytes
// back, in allocation order (Sec. 3.1-3.2).  The runtime is that table plus
// the device-side machinery: per-context device scratch, a ping-pong pair of
// fingerprint tables, arenas for image payloads in device and pinned host
// memory, a side stream for the device-to-host drain, and CUDA graphs that
// launch the checkpoint pass.
//
//   crac_arena.cpp    arenas and grow-only buffers
//   crac_image.cpp    the image store, image access and (de)serialization
//   crac_pass.cpp     context setup, the checkpoint pass (A0-A6), trial passes
//   crac_restart.cpp  restart (R1-R3)
//   crac_tune.cpp     the autotuner
//   crac_server.cpp   the request server
//   crac_abi.cpp      the rest of the C ABI, status and fault injection
#pragma once

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <climits>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "crac.h"
#include "crac_kernels.cuh"

namespace crac {

constexpr uint64_t kNoParent = ~0ull;
constexpr uint64_t kHeaderBytes = 80;
constexpr uint64_t kAllocEntryBytes = 40;
constexpr uint64_t kDefaultStagingMax = 8ull << 30;
constexpr uint64_t kDefaultTimeoutNs = 2000000000ull;
constexpr uint32_t kEncPieces = 8;   // launches of a pipelined encode of host images (at most)

extern thread_local int t_last_cuda;
extern std::atomic<int> g_fault_step;
extern std::atomic<int> g_fault_count;
extern std::atomic<uint64_t> g_lineage_counter;

crac_status_t cuda_status(cudaError_t e);   // records e for crac_last_cuda_error

#define CK(expr)                                   \
    do {                                           \
        cudaError_t e_ = (expr);                   \
        if (e_ != cudaSuccess) return cuda_status(e_); \
    } while (0)

#define TRY(expr)                                  \
    do {                                           \
        crac_status_t s_ = (expr);                 \
        if (s_ != CRAC_OK) return s_;              \
    } while (0)

bool fault_hit(int step);   // consumes one injected fault at `step`

inline uint64_t round_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// ---------------------------------------------------------------------------
// First-fit range allocator over [0, size) with coalescing frees.
// ---------------------------------------------------------------------------
class RangeAlloc {
  public:
    explicit RangeAlloc(uint64_t size) { free_[0] = size; }
    // Best fit (the smallest free range that holds len, the lowest such on a
    // tie): small tables fill small holes and leave the large ones for
    // payloads, which matters in a loop that mixes 64-byte control blocks,
    // per-image tables and multi-GiB images.
    bool alloc(uint64_t len, uint64_t *off) {
        auto best = free_.end();
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= len && (best == free_.end() || it->second < best->second)) best = it;
        if (best == free_.end()) return false;
        const uint64_t o = best->first, rest = best->second - len;
        free_.erase(best);
        if (rest) free_[o + len] = rest;
        *off = o;
        return true;
    }
    void release(uint64_t off, uint64_t len) {
        if (!len) return;
        auto it = free_.emplace(off, len).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }

  private:
    std::map<uint64_t, uint64_t> free_;
};

struct Block {
    uint8_t *p = nullptr;
    uint64_t len = 0;
    int region = -1;
    uint64_t off = 0;
};

// Device or pinned-host memory arena: regions from cudaMalloc/cudaHostAlloc,
// carved best-fit.  Image payloads and tables live here so that a steady
// checkpoint loop allocates nothing from CUDA after warm-up.
class Arena {
  public:
    Arena(bool device, int dev, uint64_t quantum) : device_(device), dev_(dev), quantum_(quantum) {}
    ~Arena() {
        if (grower_.joinable()) grower_.join();
    }
    // Make sure at least `bytes` are free in one region (grows the arena once,
    // so that later image allocations need no cudaMalloc / cudaHostAlloc).
    crac_status_t reserve(uint64_t bytes) {
        Block b;
        crac_status_t st = alloc(bytes, &b);
        if (st == CRAC_OK) free(b);
        return st;
    }
    crac_status_t alloc(uint64_t len, Block *b) {
        if (fault_hit(CRAC_FAULT_ALLOC)) return CRAC_ERR_OOM;
        len = round_up(std::max<uint64_t>(len, 1), 256);
        std::lock_guard<std::mutex> lk(mu_);
        for (size_t r = 0; r < regions_.size(); ++r) {
            uint64_t off;
            if (regions_[r].ra.alloc(len, &off)) {
                *b = Block{regions_[r].base + off, len, (int)r, off};
                used_ += len;
                maybe_pregrow_locked();
                return CRAC_OK;
            }
        }
        grows_++;
        // Whole quanta: a region made for one block is reusable for any block
        // up to its size (blocks sized by staging segments vary by a few KiB).
        uint64_t sz = round_up(std::max(len, quantum_), quantum_);
        void *p = nullptr;
        cudaError_t e;
        {
            DeviceGuard g(dev_);
            e = device_ ? cudaMalloc(&p, sz) : cudaHostAlloc(&p, sz, cudaHostAllocPortable);
            if (e != cudaSuccess && sz > len) {
                cudaGetLastError();
                sz = len;
                e = device_ ? cudaMalloc(&p, sz) : cudaHostAlloc(&p, sz, cudaHostAllocPortable);
            }
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            t_last_cuda = (int)e;
            return CRAC_ERR_OOM;
        }
        regions_.push_back(Region{(uint8_t *)p, sz, RangeAlloc(sz)});
        total_ += sz;
        const int r = (int)regions_.size() - 1;
        uint64_t off = 0;
        regions_[r].ra.alloc(len, &off);
        *b = Block{regions_[r].base + off, len, r, off};
        used_ += len;
        return CRAC_OK;
    }
    // Carve from the existing regions only: no growth and no background
    // pre-grow, for temporary worst-case blocks that are shrunk right after.
    bool try_alloc(uint64_t len, Block *b) {
        len = round_up(std::max<uint64_t>(len, 1), 256);
        std::lock_guard<std::mutex> lk(mu_);
        for (size_t r = 0; r < regions_.size(); ++r) {
            uint64_t off;
            if (regions_[r].ra.alloc(len, &off)) {
                *b = Block{regions_[r].base + off, len, (int)r, off};
                used_ += len;
                return true;
            }
        }
        return false;
    }
    void free(Block &b) {
        if (b.region < 0) return;
        std::lock_guard<std::mutex> lk(mu_);
        regions_[b.region].ra.release(b.off, b.len);
        used_ -= b.len;
        b = Block{};
    }
    void shrink(Block &b, uint64_t new_len) {
        if (b.region < 0) return;
        new_len = round_up(std::max<uint64_t>(new_len, 1), 256);
        if (new_len >= b.len) return;
        std::lock_guard<std::mutex> lk(mu_);
        regions_[b.region].ra.release(b.off + new_len, b.len - new_len);
        used_ -= b.len - new_len;
        b.len = new_len;
    }
    // Pinned memory takes a long time to obtain (page pinning), so once the
    // pinned arena is 80% used a background thread adds a region of a quarter
    // of its size (at least 1 GiB): a steady workload then rarely pins memory
    // on the request path.
    void maybe_pregrow_locked() {
        if (device_ || growing_ || total_ == 0 || used_ * 5 < total_ * 4) return;
        if (grower_.joinable()) grower_.join();
        growing_ = true;
        const uint64_t sz = std::max<uint64_t>(total_ / 4, 1ull << 30);
        grower_ = std::thread([this, sz] {
            void *p = nullptr;
            const cudaError_t e = cudaHostAlloc(&p, sz, cudaHostAllocPortable);
            std::lock_guard<std::mutex> lk(mu_);
            if (e == cudaSuccess) {
                regions_.push_back(Region{(uint8_t *)p, sz, RangeAlloc(sz)});
                total_ += sz;
                pregrows_++;
            } else {
                cudaGetLastError();
            }
            growing_ = false;
        });
    }
    // Growth after a reservation counts from here on.
    void mark_reserved() {
        std::lock_guard<std::mutex> lk(mu_);
        grows_ = 0;
    }
    void stats(uint64_t *total, uint64_t *used, uint32_t *regions, uint32_t *grows) {
        std::lock_guard<std::mutex> lk(mu_);
        *total = total_;
        *used = used_;
        *regions = (uint32_t)regions_.size();
        *grows = grows_;
    }

  private:
    struct Region {
        uint8_t *base;
        uint64_t size;
        RangeAlloc ra;
    };
    bool device_;
    int dev_;
    uint64_t quantum_;
    std::mutex mu_;
    std::vector<Region> regions_;
    uint64_t total_ = 0, used_ = 0;
    uint32_t grows_ = 0, pregrows_ = 0;
    bool growing_ = false;
    std::thread grower_;
};

Arena &device_arena(int dev);
Arena &pinned_arena();

// Grow-only device buffer owned by a context.
struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    bool borrowed = false;   // a server lease: never freed or replaced by ensure_dev
};
crac_status_t ensure_dev(DevBuf &b, size_t bytes);

struct HostBuf {
    void *p = nullptr;
    size_t cap = 0;
};
crac_status_t ensure_host(HostBuf &b, size_t bytes);

struct ImgAlloc {
    uint64_t id, orig_ptr, bytes;
    uint32_t kind;
    uint64_t first_chunk;
};

// One segment of an image's payload.
struct Piece {
    uint64_t k0 = 0, k = 0;         // entries [k0, k0+k) of the image's dirty list
    uint64_t off0 = 0, bytes = 0;   // payload bytes [off0, off0+bytes)
    uint64_t span = 0;              // sparse piece: bytes of `dev` that the entries'
                                    // offsets index (0: compact, offsets are prefixes)
    Block host;                     // host residency: pinned copy
    Block dev;                      // device residency: payload
    Block idx_dev, off_dev;         // device residency: idx[k], off[k+1] (piece-relative)
    Block zlen_dev;                 // device residency, coded image: zlen[k]
    // Sparse piece, made on the first ranged read: host copies of the
    // entries' span offsets and of the running sum of their chunk lengths
    // (the compact offsets, k + 1 values).
    std::vector<uint64_t> sp_off, sp_cum;
};

struct AllocRec {
    uint64_t id, ptr, bytes;
    uint32_t kind;
};

}  // namespace crac

using crac::AllocRec;
using crac::Block;
using crac::DevBuf;
using crac::HostBuf;
using crac::ImgAlloc;
using crac::Piece;
using crac::kNoParent;

struct crac_image {
    std::atomic<int> refs{1};
    int device = 0;
    uint32_t flags = 0, chunk_bytes = 0, residency = CRAC_RESIDENCY_HOST;
    uint64_t lineage = 0, epoch = 0, parent_epoch = kNoParent;
    std::vector<ImgAlloc> allocs;
    uint64_t n_chunks = 0, k = 0, payload_bytes = 0;
    Block fp_h, idx_h;              // pinned: fp[n_chunks], idx[k] (device images: on demand)
    Block fp_dev;                   // device images: fp[n_chunks] in device memory
    Block off_h;                    // host images: offset of each entry's bytes inside its
                                    // piece's payload (made by the first mapped restore)
    Block zlen_h;                   // coded images: stream length of each entry (pinned;
                                    // device images: on demand, like idx_h)
    uint64_t raw_bytes = 0;         // bytes of the chunks present, before coding
    bool host_tables = true;        // fp_h / idx_h hold the tables
    std::vector<Piece> pieces;
    crac_image *parent = nullptr;   // strong reference, set for delta images
    cudaEvent_t done = nullptr;     // drain complete
    cudaEvent_t drain0 = nullptr;   // host images: recorded on the side stream as the drain starts
    std::atomic<int> state{0};      // 0 pending, 1 complete, < 0 failed (status)
    std::mutex mu;
    // A checkpoint that returned before its pass finished (single segment):
    // the pass's counts land in ctrl_b, and k, the payload size, the FULL flag
    // and the pieces' block sizes are settled once `done` has completed
    // (img_resolve).  dep is the context's previous unsettled image, whose
    // failure fails this one too.
    bool deferred = false;
    bool sparse_pass = false;       // the pass left an uncompacted payload
    bool predicted_full = false;    // no baseline anywhere: k and D known before the pass
    Block ctrl_b;                   // pinned landing of the pass's control block
    crac_image *dep = nullptr;
    int out_fp = -1;                // fingerprint table of the context the pass wrote
    bool had_base = false;          // some chunk had a baseline (the pass measured a dirty fraction)
    bool lost = false;              // its kernel reported kErrLostCopy
    uint64_t seq = 0;               // the context's pass counter at this pass
    uint64_t spec_hits = 0;         // ... this many of its entries were found in place
    uint64_t spec_writes = 0;       // ... of this many chunks written speculatively
};

namespace crac {

void table_add(crac_image *im);
void table_remove(crac_image *im);
void img_ref(crac_image *im);
void img_unref(crac_image *im);
crac_status_t img_wait(const crac_image *cim, uint64_t timeout_ns);
crac_status_t img_host_tables(crac_image *im);
crac_status_t img_resolve(crac_image *im);
crac_image *img_parent(crac_image *im);
void free_image_blocks(crac_image *im);

inline uint64_t chunk_len(uint64_t bytes, uint64_t local, uint32_t log2S) {
    return std::min<uint64_t>(1ull << log2S, bytes - (local << log2S));
}

inline uint32_t log2u(uint64_t x) {
    uint32_t l = 0;
    while ((1ull << l) < x) ++l;
    return l;
}

}  // namespace crac

struct crac_ctx {
    std::mutex mu;
    crac_config_t cfg{};
    int device = 0;
    int sm_count = 0;
    bool uva = false;            // the device addresses pinned host memory directly
    uint32_t log2S = 16;
    std::vector<AllocRec> allocs;
    uint64_t next_id = 0;
    uint64_t lineage = 0;
    uint64_t epoch_max = 0;
    crac_image *parent = nullptr;
    uint64_t parent_epoch = kNoParent;
    // fingerprint baseline: fp[fp_cur] holds the fingerprints the next pass
    // compares against; a pass writes spare_fp(); three tables, so that the
    // baseline of the last settled image survives while up to two images
    // are unsettled (their passes may still fail)
    DevBuf fp[3];
    int fp_cur = 0;
    int prev_fp = 1;             // autotuner shadows: the table before the last committed trial pass
    bool base_valid = false;
    std::unordered_map<uint64_t, uint64_t> base_first;   // alloc id -> first chunk in fp[fp_cur]
    std::unordered_map<uint64_t, uint64_t> prev_base_first;   // autotuner shadows: the baseline before the last
    bool prev_base_valid = false;                             // committed trial pass (still in fp[1 - fp_cur])
    // pass scratch
    DevBuf desc, work, idx, off, staging, lens, carry;
    HostBuf desc_h, desc_h2, ctrl_h;
    int desc_flip = 0;           // which of desc_h / desc_h2 the next pass fills
    DevBuf cstage, zwork, zoff, zlen;   // CRAC_FLAG_COMPRESS: streams, encoder scratch, tables
    // restart scratch
    DevBuf owner, sdesc, sidx, soff, serr;
    DevBuf vdesc, vwork, vfp, vidx, voff;   // incremental restore: fingerprint pass scratch
    HostBuf vdesc_h;
    HostBuf owner_h, sdesc_h, soff_h, serr_h;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_last = nullptr, ev_pass = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
    cudaEvent_t ev_p0 = nullptr, ev_p1 = nullptr;
    cudaEvent_t ev_piece[crac::kEncPieces] = {};   // ends of the launches of a pipelined encode
    cudaEvent_t ev_z0 = nullptr, ev_z1 = nullptr;   // the sized encoder: end of sizing, start of coding
    // graph for the fused pass: memset(ctrl+status) -> kernel -> D2H(ctrl)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaGraphNode_t g_memset = nullptr, g_kernel = nullptr, g_copy = nullptr;
    int g_threads = 0, g_wpc = 0;
    const void *g_fn = nullptr;
    bool tma_ready = false;
    // graph for the split pass: memset -> hash -> finalize -> gather -> ctrl D2H
    cudaGraph_t sgraph = nullptr;
    cudaGraphExec_t sgexec = nullptr;
    cudaGraphNode_t s_memset = nullptr, s_k[3] = {nullptr, nullptr, nullptr}, s_copy = nullptr;
    cudaEvent_t sev[4] = {nullptr, nullptr, nullptr, nullptr};   // around each split-pass kernel
    const void *s_hash_fn = nullptr;
    crac_pass_info_t last{};
    crac_restart_info_t last_restart{};
    bool full_copy_ok = false;   // current pass: no baseline anywhere and 16-byte sizes
    bool sparse_ok = false;      // current pass: CRAC_PASS_SPARSE, device images, 16-byte sizes
    bool dense_now = false;      // ... and, on 512 B - 4 KiB chunks, dense placement of the dirty chunks
    bool dense_hint = false;     // trial passes: dense placement (set by the tuner for a sparse timing)
    uint32_t pass_now = CRAC_PASS_SPLIT;   // kernel of the current pass (CRAC_PASS_AUTO resolved)
    bool split_now = false;      // the current pass is the split graph (per-kernel timing events)
    bool prefetch_now = false;   // the current pass prefetched managed memory (ev_p0 / ev_p1)
    // Predicted write-through of the split pass (CkptParams::ppos): ppos[ppos_cur]
    // holds the last such pass's staging offsets (its successor's prediction),
    // valid while ppos_ok and the chunk layout is the one it was made for.
    DevBuf ppos[2];
    int ppos_cur = 0;
    bool ppos_ok = false;
    uint64_t ppos_layout = 0;
    uint64_t layout_version = 0;   // bumped when the registry's chunk layout changes
    DevBuf chdr;                   // coded contexts: CRZ1 block headers made by the split pass
    bool crz_hdr_now = false;      // the current pass makes them (split pass, chunks >= 8 KiB)
    bool spec_now = false;         // the current pass records offsets (single-segment split pass)
    bool spec_use = false;         // ... and writes its predicted chunks as it reads them
    uint32_t spec_rest = 0;        // passes left without speculation after a poor prediction
    float delta_frac = 0.f;      // dirty chunks / chunks of the last pass that had a baseline
    bool delta_frac_valid = false;
    cudaEvent_t ev_r0 = nullptr, ev_r1 = nullptr;
    bool cuda_ready = false;
    bool lost = false;   // a kernel reported kErrLostCopy: no further device work on this context
    // Checkpoints whose passes were still running when the call returned, in
    // order, and the state after the last settled one (the state a failure of
    // an unsettled pass reverts to).
    std::deque<crac_image *> pending;
    struct Settled {
        int fp = 0;
        bool valid = false;
        std::unordered_map<uint64_t, uint64_t> first;
        crac_image *parent = nullptr;   // strong reference
        uint64_t parent_epoch = kNoParent, epoch_max = 0;
    } settled;
    uint64_t pass_seq = 0;       // passes started; pass info describes pass `pass_seq`
    // autotuner session: one shadow context per candidate chunk size
    std::vector<crac_ctx *> tune_ctx;
    std::vector<double> tune_sum_ms, tune_sum_bytes;
    std::vector<float> tune_last_ms;
    std::vector<uint64_t> tune_last_bytes;
    uint32_t tune_rounds = 0;
    bool cpt_tuned = false;      // cfg.chunks_per_tile was written by the tuner
};

namespace crac {

// Contexts and the checkpoint pass (crac_pass.cpp).
crac_status_t ctx_init(crac_ctx *c, const crac_config_t *cfg_in);
crac_status_t ctx_cuda_ready(crac_ctx *c);
void ctx_free_all(crac_ctx *c);
void pick_split(const crac_ctx *c, int *wpc, uint32_t *cpt);
crac_status_t ctx_checkpoint(crac_ctx *c, cudaStream_t s, crac_image_t **out);
crac_status_t ctx_settle(crac_ctx *c, bool block);
int spare_fp(const crac_ctx *c);
crac_status_t ctx_trial_pass(crac_ctx *c, cudaStream_t s, bool commit, float *ms, uint64_t *k_out,
                             uint64_t *d_out);
crac_status_t fingerprint_against(crac_ctx *c, const uint64_t *fp_ref, cudaStream_t s, const uint64_t **fp_out,
                                  const CkptCtrl **ctrl_out);

// Restart (crac_restart.cpp).
crac_status_t ctx_restart(crac_ctx *c, crac_image *img, cudaStream_t s);
crac_status_t reserve_restart(crac_ctx *c, uint64_t nt, size_t descs, size_t pieces);

// The autotuner (crac_tune.cpp).
void tune_clear(crac_ctx *c);

// The default context of the four context-free calls (crac_abi.cpp).
crac_status_t default_ctx(crac_ctx **out);

// Steady clock in seconds (crac_time_now).
double now_s();

// bytes from src to dst, one of them pinned host memory addressed through its
// device mapping (or both device memory), by SM loads and stores on s with at
// most max_grid CTAs, instead of a copy engine (crac_drain.cu).
cudaError_t launch_link_copy(void *dst, const void *src, uint64_t bytes, int max_grid, cudaStream_t s);

// The sparse pass's dense-placement hash kernel for 512 B - 4 KiB chunks
// (lanes_per_chunk = chunk bytes / 256), the dynamic shared memory it runs
// with, the attribute that allows it (before its first launch or graph
// node), and occupancy with dynamic shared memory (crac_pass_split.cu).
const void *split_hash_small_dense_fn(int lanes_per_chunk);
size_t split_dense_smem();
cudaError_t split_dense_prepare(const void *fn);
int split_max_ctas_per_sm_smem(const void *fn, int threads, size_t smem);

// Entries [0, n) of a sparse device piece packed back to back into device
// memory dst: entry j's cum[j+1] - cum[j] bytes from span + off[j] to
// dst + cum[j] - cum[0]; off and cum are device arrays (crac_drain.cu).
cudaError_t launch_sparse_pack(void *dst, const void *span, const uint64_t *off, const uint64_t *cum, uint64_t n,
                               int grid, cudaStream_t s);

// A per-operation transfer between device memory and pinned host memory on
// s: by an SM copy kernel where the device addresses pinned memory directly
// (the copy engines' device-to-host rate was seen to collapse for seconds on
// GB300, and transfers queued behind it), else by the copy engine.
inline cudaError_t link_copy(const crac_ctx *c, void *dst, const void *src, size_t bytes, cudaMemcpyKind kind,
                             cudaStream_t s) {
    if (c->uva) return launch_link_copy(dst, src, bytes, c->sm_count * 2, s);
    return cudaMemcpyAsync(dst, src, bytes, kind, s);
}

}  // namespace crac
