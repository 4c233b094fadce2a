// Host runtime of libcrac: allocation registry, fingerprint baseline,
// checkpoint and restart orchestration, image store, and the C ABI.
//
// The paper keeps its own table of active cudaMalloc-family allocations
// (only the pointers the app got back, not the library's arenas) and saves
// exactly those buffers (Sec. 3.2, "Issue of library-allocated memory" and
// "Saving the library-allocated arena").  Restart copies the saved bytes
// back, in allocation order (Sec. 3.1-3.2).  This runtime is that table
// plus the device-side machinery: per-context device scratch, a ping-pong
// pair of fingerprint tables, arenas for image payloads in device and pinned
// host memory, a side stream for the device-to-host drain, and a CUDA graph
// that launches the fused checkpoint pass.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <climits>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "crac.h"
#include "crac_kernels.cuh"

using namespace crac;

namespace {

constexpr uint64_t kNoParent = ~0ull;
constexpr uint64_t kHeaderBytes = 80;
constexpr uint64_t kAllocEntryBytes = 40;
constexpr uint64_t kDefaultStagingMax = 8ull << 30;
constexpr uint64_t kDefaultTimeoutNs = 2000000000ull;

thread_local int t_last_cuda = 0;
std::atomic<int> g_fault_step{CRAC_FAULT_NONE};
std::atomic<int> g_fault_count{0};
std::atomic<uint64_t> g_lineage_counter{0};

crac_status_t cuda_status(cudaError_t e) {
    t_last_cuda = (int)e;
    return e == cudaErrorMemoryAllocation ? CRAC_ERR_OOM : CRAC_ERR_CUDA;
}

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

uint64_t round_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

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
    bool alloc(uint64_t len, uint64_t *off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= len) {
                const uint64_t o = it->first, rest = it->second - len;
                free_.erase(it);
                if (rest) free_[o + len] = rest;
                *off = o;
                return true;
            }
        }
        return false;
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
// carved first-fit.  Image payloads and tables live here so that a steady
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
        uint64_t sz = std::max(len, quantum_);
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

std::mutex g_arena_mu;
std::map<int, std::unique_ptr<Arena>> g_dev_arenas;
std::unique_ptr<Arena> g_pinned_arena;

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

// Grow-only device buffer owned by a context.
struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

crac_status_t ensure_dev(DevBuf &b, size_t bytes) {
    bytes = std::max<size_t>(bytes, 256);
    if (b.cap >= bytes) return CRAC_OK;
    if (fault_hit(CRAC_FAULT_ALLOC)) return CRAC_ERR_OOM;
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

struct HostBuf {
    void *p = nullptr;
    size_t cap = 0;
};

crac_status_t ensure_host(HostBuf &b, size_t bytes) {
    bytes = std::max<size_t>(bytes, 256);
    if (b.cap >= bytes) return CRAC_OK;
    if (b.p) {
        CK(cudaFreeHost(b.p));
        b = HostBuf{};
    }
    const size_t sz = round_up(bytes + bytes / 4, 1 << 16);
    CK(cudaHostAlloc(&b.p, sz, cudaHostAllocPortable));
    b.cap = sz;
    return CRAC_OK;
}

}  // namespace

void crac::note_cuda_error(int e) { t_last_cuda = e; }

// ---------------------------------------------------------------------------
// Images
// ---------------------------------------------------------------------------

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
};

struct crac_image {
    std::atomic<int> refs{1};
    int device = 0;
    uint32_t flags = 0, chunk_bytes = 0, residency = CRAC_RESIDENCY_HOST;
    uint64_t lineage = 0, epoch = 0, parent_epoch = kNoParent;
    std::vector<ImgAlloc> allocs;
    uint64_t n_chunks = 0, k = 0, payload_bytes = 0;
    Block fp_h, idx_h;              // pinned: fp[n_chunks], idx[k] (device images: on demand)
    Block fp_dev;                   // device images: fp[n_chunks] in device memory
    bool host_tables = true;        // fp_h / idx_h hold the tables
    std::vector<Piece> pieces;
    crac_image *parent = nullptr;   // strong reference, set for delta images
    cudaEvent_t done = nullptr;     // drain complete
    std::atomic<int> state{0};      // 0 pending, 1 complete, < 0 failed (status)
    std::mutex mu;
};

namespace {

std::mutex g_img_mu;
std::multimap<std::pair<uint64_t, uint64_t>, crac_image *> g_images;   // (lineage, epoch)

void table_add(crac_image *im) {
    std::lock_guard<std::mutex> lk(g_img_mu);
    g_images.emplace(std::make_pair(im->lineage, im->epoch), im);
}

void table_remove(crac_image *im) {
    std::lock_guard<std::mutex> lk(g_img_mu);
    auto r = g_images.equal_range(std::make_pair(im->lineage, im->epoch));
    for (auto it = r.first; it != r.second; ++it) {
        if (it->second == im) {
            g_images.erase(it);
            return;
        }
    }
}

void img_ref(crac_image *im) {
    if (im) im->refs.fetch_add(1);
}

crac_status_t img_wait(const crac_image *cim, uint64_t timeout_ns) {
    crac_image *im = const_cast<crac_image *>(cim);
    if (im->state.load() == 1) return CRAC_OK;
    if (im->state.load() < 0) return im->state.load();
    DeviceGuard g(im->device);
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaEventQuery(im->done);
        if (e == cudaSuccess) {
            im->state.store(1);
            return CRAC_OK;
        }
        if (e != cudaErrorNotReady) {
            cudaGetLastError();
            im->state.store(cuda_status(e));
            return im->state.load();
        }
        if (timeout_ns) {
            const uint64_t el = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
                                    std::chrono::steady_clock::now() - t0).count();
            if (el >= timeout_ns) return CRAC_ERR_TIMEOUT;
        }
        std::this_thread::yield();
    }
}

void img_unref(crac_image *im) {
    while (im) {
        if (im->refs.fetch_sub(1) != 1) return;
        if (im->done) {
            DeviceGuard g(im->device);
            cudaEventSynchronize(im->done);
            cudaEventDestroy(im->done);
            cudaGetLastError();
        }
        table_remove(im);
        Arena &pa = pinned_arena();
        pa.free(im->fp_h);
        pa.free(im->idx_h);
        if (im->fp_dev.region >= 0) device_arena(im->device).free(im->fp_dev);
        for (Piece &p : im->pieces) {
            pa.free(p.host);
            if (p.dev.region >= 0 || p.idx_dev.region >= 0 || p.off_dev.region >= 0) {
                Arena &da = device_arena(im->device);
                da.free(p.dev);
                da.free(p.idx_dev);
                da.free(p.off_dev);
            }
        }
        crac_image *parent = im->parent;
        delete im;
        im = parent;
    }
}

// Host copies of a device image's fingerprint table and chunk list (made on
// the first request: serialization, or a restart chain resolved on the host).
crac_status_t img_host_tables(crac_image *im) {
    std::lock_guard<std::mutex> lk(im->mu);
    if (im->host_tables) return CRAC_OK;
    TRY(img_wait(im, 0));
    Arena &pa = pinned_arena();
    if (im->n_chunks) TRY(pa.alloc(im->n_chunks * 8, &im->fp_h));
    if (im->k) TRY(pa.alloc(im->k * 8, &im->idx_h));
    DeviceGuard g(im->device);
    if (im->n_chunks) CK(cudaMemcpy(im->fp_h.p, im->fp_dev.p, im->n_chunks * 8, cudaMemcpyDeviceToHost));
    for (const Piece &pc : im->pieces)
        if (pc.k) CK(cudaMemcpy(im->idx_h.p + pc.k0 * 8, pc.idx_dev.p, pc.k * 8, cudaMemcpyDeviceToHost));
    im->host_tables = true;
    return CRAC_OK;
}

// Parent of a delta: the direct link if set, else a live image with the same
// lineage and the parent's epoch (deserialized images).
crac_image *img_parent(crac_image *im) {
    std::lock_guard<std::mutex> lk(im->mu);
    if (im->parent) return im->parent;
    if (im->parent_epoch == kNoParent) return nullptr;
    std::lock_guard<std::mutex> lk2(g_img_mu);
    auto r = g_images.equal_range(std::make_pair(im->lineage, im->parent_epoch));
    for (auto it = r.first; it != r.second; ++it) {
        if (it->second != im && it->second->state.load() >= 0) {
            img_ref(it->second);
            im->parent = it->second;
            return im->parent;
        }
    }
    return nullptr;
}

uint64_t chunk_len(uint64_t bytes, uint64_t local, uint32_t log2S) {
    return std::min<uint64_t>(1ull << log2S, bytes - (local << log2S));
}

uint32_t log2u(uint64_t x) {
    uint32_t l = 0;
    while ((1ull << l) < x) ++l;
    return l;
}

}  // namespace

// ---------------------------------------------------------------------------
// Contexts
// ---------------------------------------------------------------------------

struct AllocRec {
    uint64_t id, ptr, bytes;
    uint32_t kind;
};

struct crac_ctx {
    std::mutex mu;
    crac_config_t cfg{};
    int device = 0;
    int sm_count = 0;
    uint32_t log2S = 16;
    std::vector<AllocRec> allocs;
    uint64_t next_id = 0;
    uint64_t lineage = 0;
    uint64_t epoch_max = 0;
    crac_image *parent = nullptr;
    uint64_t parent_epoch = kNoParent;
    // fingerprint baseline
    DevBuf fp[2];
    int fp_cur = 0;
    bool base_valid = false;
    std::unordered_map<uint64_t, uint64_t> base_first;   // alloc id -> first chunk in fp[fp_cur]
    std::unordered_map<uint64_t, uint64_t> prev_base_first;   // autotuner shadows: the baseline before the last
    bool prev_base_valid = false;                             // committed trial pass (still in fp[1 - fp_cur])
    // pass scratch
    DevBuf desc, work, idx, off, staging, lens, carry;
    HostBuf desc_h, ctrl_h;
    // restart scratch
    DevBuf owner, sdesc, sidx, soff, serr;
    HostBuf owner_h, sdesc_h, soff_h, serr_h;
    cudaStream_t side = nullptr;
    cudaEvent_t ev_last = nullptr, ev_pass = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
    cudaEvent_t ev_p0 = nullptr, ev_p1 = nullptr;
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
    cudaEvent_t ev_r0 = nullptr, ev_r1 = nullptr;
    bool cuda_ready = false;
    // autotuner session: one shadow context per candidate chunk size
    std::vector<crac_ctx *> tune_ctx;
    std::vector<double> tune_sum_ms, tune_sum_bytes;
    std::vector<float> tune_last_ms;
    std::vector<uint64_t> tune_last_bytes;
    uint32_t tune_rounds = 0;
    bool cpt_tuned = false;      // cfg.chunks_per_tile was written by the tuner
};

namespace {

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
    if (c->cuda_ready) return CRAC_OK;
    int dev = c->cfg.device;
    if (dev < 0) CK(cudaGetDevice(&dev));
    c->device = dev;
    DeviceGuard g(dev);
    CK(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev));
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
    TRY(ensure_host(c->ctrl_h, sizeof(CkptCtrl)));
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

void ctx_free_all(crac_ctx *c);

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

void ctx_free_all(crac_ctx *c) {
    tune_clear(c);
    if (!c->cuda_ready) {
        img_unref(c->parent);
        c->parent = nullptr;
        return;
    }
    DeviceGuard g(c->device);
    cudaDeviceSynchronize();
    for (DevBuf *b : {&c->fp[0], &c->fp[1], &c->desc, &c->work, &c->idx, &c->off, &c->staging,
                      &c->lens, &c->carry, &c->owner, &c->sdesc, &c->sidx, &c->soff, &c->serr})
        if (b->p) cudaFree(b->p);
    for (HostBuf *b : {&c->desc_h, &c->ctrl_h, &c->owner_h, &c->sdesc_h, &c->soff_h, &c->serr_h})
        if (b->p) cudaFreeHost(b->p);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->sgexec) cudaGraphExecDestroy(c->sgexec);
    if (c->sgraph) cudaGraphDestroy(c->sgraph);
    for (cudaEvent_t e : {c->ev_last, c->ev_pass, c->ev_t0, c->ev_t1, c->ev_p0, c->ev_p1, c->sev[0], c->sev[1],
                          c->sev[2], c->sev[3], c->ev_r0, c->ev_r1})
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

// Build (or update) the graph memset -> fused kernel -> ctrl D2H and launch it.
crac_status_t launch_fused_graph(crac_ctx *c, const CkptParams &P, size_t work_bytes, const void *fn,
                                 int threads, size_t smem, int grid, cudaStream_t s) {
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
    if (c->gexec && c->g_fn == fn) {
        // Width changes of a memset node may be rejected; rebuild then.
        if (cudaGraphExecMemsetNodeSetParams(c->gexec, c->g_memset, &mp) != cudaSuccess ||
            cudaGraphExecKernelNodeSetParams(c->gexec, c->g_kernel, &kp) != cudaSuccess ||
            cudaGraphExecMemcpyNodeSetParams1D(c->gexec, c->g_copy, c->ctrl_h.p, P.ctrl, sizeof(CkptCtrl),
                                               cudaMemcpyDeviceToHost) != cudaSuccess) {
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
        CK(cudaGraphAddMemcpyNode1D(&c->g_copy, c->graph, &c->g_kernel, 1, c->ctrl_h.p, P.ctrl,
                                    sizeof(CkptCtrl), cudaMemcpyDeviceToHost));
        CK(cudaGraphInstantiate(&c->gexec, c->graph, 0));
        c->g_fn = fn;
        c->g_threads = threads;
        rebuilt = true;
    }
    (void)rebuilt;
    CK(cudaEventRecord(c->ev_t0, s));   // after the host-side updates: times the device work only
    CK(cudaGraphLaunch(c->gexec, s));
    count_launches(1);
    return CRAC_OK;
}

// Build (or update) the split-pass graph and launch it.
crac_status_t launch_split_graph(crac_ctx *c, const CkptParams &P, size_t work_bytes, unsigned long long *acc,
                                 uint32_t log2Seg, const void *hash_fn, const int grids[3], cudaStream_t s) {
    const void *fns[3] = {hash_fn, split_finalize_fn(), split_gather_fn()};
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
        kp[i].sharedMemBytes = 0;
        kp[i].kernelParams = args;
    }
    cudaMemsetParams mp{};
    mp.dst = c->work.p;
    mp.value = 0;
    mp.elementSize = 4;
    mp.width = work_bytes / 4;
    mp.height = 1;
    bool ok = c->sgexec != nullptr && c->s_hash_fn == hash_fn;
    if (ok) {
        ok = cudaGraphExecMemsetNodeSetParams(c->sgexec, c->s_memset, &mp) == cudaSuccess;
        for (int i = 0; ok && i < 3; ++i)
            ok = cudaGraphExecKernelNodeSetParams(c->sgexec, c->s_k[i], &kp[i]) == cudaSuccess;
        if (ok)
            ok = cudaGraphExecMemcpyNodeSetParams1D(c->sgexec, c->s_copy, c->ctrl_h.p, P.ctrl, sizeof(CkptCtrl),
                                                    cudaMemcpyDeviceToHost) == cudaSuccess;
        if (!ok) cudaGetLastError();
    }
    if (!ok) {
        if (c->sgexec) cudaGraphExecDestroy(c->sgexec);
        if (c->sgraph) cudaGraphDestroy(c->sgraph);
        c->sgexec = nullptr;
        c->sgraph = nullptr;
        CK(cudaGraphCreate(&c->sgraph, 0));
        CK(cudaGraphAddMemsetNode(&c->s_memset, c->sgraph, nullptr, 0, &mp));
        cudaGraphNode_t prev = c->s_memset;
        cudaGraphNode_t ev;
        CK(cudaGraphAddEventRecordNode(&ev, c->sgraph, &prev, 1, c->sev[0]));
        prev = ev;
        for (int i = 0; i < 3; ++i) {
            CK(cudaGraphAddKernelNode(&c->s_k[i], c->sgraph, &prev, 1, &kp[i]));
            CK(cudaGraphAddEventRecordNode(&ev, c->sgraph, &c->s_k[i], 1, c->sev[i + 1]));
            prev = ev;
        }
        CK(cudaGraphAddMemcpyNode1D(&c->s_copy, c->sgraph, &prev, 1, c->ctrl_h.p, P.ctrl, sizeof(CkptCtrl),
                                    cudaMemcpyDeviceToHost));
        CK(cudaGraphInstantiate(&c->sgexec, c->sgraph, 0));
        c->s_hash_fn = hash_fn;
    }
    CK(cudaEventRecord(c->ev_t0, s));
    CK(cudaGraphLaunch(c->sgexec, s));
    count_launches(3);
    return CRAC_OK;
}

// One segment of the checkpoint pass; on return the ctrl block is on the host.
crac_status_t run_segment(crac_ctx *c, const Segment &sg, const CkptDesc *desc_dev,
                          const std::vector<uint64_t> &first, uint64_t *idx_d, uint64_t *off_d,
                          uint64_t idx_cap, uint8_t *staging, uint64_t staging_cap,
                          cudaStream_t s, CkptCtrl *ctrl_out, float *ms) {
    const uint64_t nseg = sg.c1 - sg.c0;
    const uint64_t *fp_old = (const uint64_t *)c->fp[c->fp_cur].p;
    uint64_t *fp_new = (uint64_t *)c->fp[1 - c->fp_cur].p;
    const bool inject_wait = c->cfg.launch_mode == CRAC_LAUNCH_BATCHED;
    if (fault_hit(CRAC_FAULT_PASS)) {
        t_last_cuda = (int)cudaErrorLaunchFailure;
        return CRAC_ERR_CUDA;
    }
    const bool split = c->cfg.launch_mode == CRAC_LAUNCH_BATCHED &&
                       (c->cfg.pass_kernel == CRAC_PASS_SPLIT || c->cfg.pass_kernel == CRAC_PASS_AUTO ||
                        c->cfg.pass_kernel == CRAC_PASS_SPARSE);
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
        const void *hash_fn = small ? split_hash_small_fn(1 << (c->log2S - 8)) : split_hash_fn();
        CkptParams P{};
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
        P.sparse = c->sparse_ok && staging ? 1u : 0u;
        P.full_copy = (c->full_copy_ok || P.sparse) && staging ? 1u : 0u;
        P.alloc_prefix = (const uint64_t *)(desc_dev + c->allocs.size());
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
                           (n_slots + 7) / 8, (uint64_t)c->sm_count * split_max_ctas_per_sm(hash_fn, split_hash_threads())));
        const int gf = (int)std::min<uint64_t>(n_tiles, (uint64_t)c->sm_count * 2);
        const int gg = c->sm_count * 8;
        const int grids[3] = {gh, gf, gg};
        TRY(launch_split_graph(c, P, work_bytes, acc, log2Seg, hash_fn, grids, s));
        c->last.grid = (uint32_t)gh;
        c->last.chunks_per_tile = cptF;
        c->last.warps_per_chunk = 0;
        c->last.kernel_launches += 3;
        c->last.pass_kernel = P.sparse ? CRAC_PASS_SPARSE : CRAC_PASS_SPLIT;
    } else if (c->cfg.launch_mode == CRAC_LAUNCH_BATCHED) {
        const uint64_t S = 1ull << c->log2S;
        const bool tma = c->cfg.pass_kernel == CRAC_PASS_TMA;
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
        TRY(launch_fused_graph(c, P, work_bytes, fn, threads, smem, grid, s));
        c->last.pass_kernel = tma ? CRAC_PASS_TMA : CRAC_PASS_LDG;
        c->last.grid = (uint32_t)grid;
        c->last.chunks_per_tile = cpt;
        c->last.warps_per_chunk = (uint32_t)wpc;
        c->last.kernel_launches += 1;
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
        CK(cudaMemcpyAsync(c->ctrl_h.p, ctrl, sizeof(CkptCtrl), cudaMemcpyDeviceToHost, s));
    }
    CK(cudaEventRecord(c->ev_t1, s));
    CK(cudaEventRecord(c->ev_pass, s));
    CK(cudaEventSynchronize(c->ev_pass));
    float t = 0;
    CK(cudaEventElapsedTime(&t, c->ev_t0, c->ev_t1));
    *ms += t;
    if (split) {
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
    *ctrl_out = *(const CkptCtrl *)c->ctrl_h.p;
    if (ctrl_out->err & kErrTimeout) return CRAC_ERR_TIMEOUT;
    if (ctrl_out->err) return CRAC_ERR_CORRUPT;
    return CRAC_OK;
}

void free_image_blocks(crac_image *im) {
    im->refs.store(1);
    im->parent = nullptr;
    img_unref(im);
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
    CK(cudaEventCreateWithFlags(&im->done, cudaEventDisableTiming));

    Arena &pa = pinned_arena();
    Arena &da = device_arena(c->device);
    crac_status_t st = CRAC_OK;
    auto fail = [&](crac_status_t code) {
        cudaStreamSynchronize(s);
        cudaStreamSynchronize(c->side);
        cudaGetLastError();
        free_image_blocks(im.release());
        return code;
    };

    const bool dev_res = c->cfg.image_residency == CRAC_RESIDENCY_DEVICE;
    im->host_tables = !dev_res;
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
        st = ensure_dev(c->fp[1 - c->fp_cur], n * 8);
        if (st == CRAC_OK) st = ensure_dev(c->desc, na * (sizeof(CkptDesc) + 8));
        if (st == CRAC_OK) st = ensure_host(c->desc_h, na * (sizeof(CkptDesc) + 8));
        if (st != CRAC_OK) return fail(st);
        CkptDesc *dh = (CkptDesc *)c->desc_h.p;
        uint64_t *prefix_h = (uint64_t *)(dh + na);   // payload bytes before each allocation
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
        c->sparse_ok = c->cfg.pass_kernel == CRAC_PASS_SPARSE && dev_res && all16;
        // Order after the previous operation of this context (drain / restore).
        if (cudaStreamWaitEvent(s, c->ev_last, 0) != cudaSuccess) return fail(cuda_status(cudaGetLastError()));
        if (cudaMemcpyAsync(c->desc.p, dh, na * (sizeof(CkptDesc) + 8), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return fail(cuda_status(cudaGetLastError()));
        // Managed regions migrate to the device before they are read.
        bool any_managed = false;
        for (const AllocRec &r : c->allocs) any_managed |= r.kind == CRAC_KIND_MANAGED;
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
        // Segments bounded by the staging capacity.
        uint64_t cap = c->cfg.staging_bytes ? c->cfg.staging_bytes : std::min(tracked, kDefaultStagingMax);
        cap = std::max(round_up(cap, 256), S);
        const std::vector<Segment> segs = make_segments(c->allocs, first, log2S, cap);
        uint64_t max_seg_chunks = 0, max_seg_bytes = 0;
        for (const Segment &sg : segs) {
            max_seg_chunks = std::max(max_seg_chunks, sg.c1 - sg.c0);
            max_seg_bytes = std::max(max_seg_bytes, sg.bytes);
        }
        const bool host_res = c->cfg.image_residency == CRAC_RESIDENCY_HOST;
        if (host_res) {
            st = ensure_dev(c->staging, max_seg_bytes);
            if (st == CRAC_OK) st = ensure_dev(c->idx, max_seg_chunks * 8);
            if (st == CRAC_OK) st = ensure_dev(c->off, (max_seg_chunks + 1) * 8);
            if (st != CRAC_OK) return fail(st);
        }
        uint64_t k_base = 0, d_base = 0;
        float ms = 0;
        for (const Segment &sg : segs) {
            const uint64_t nseg = sg.c1 - sg.c0;
            Piece pc;
            uint64_t *idx_d = (uint64_t *)c->idx.p, *off_d = (uint64_t *)c->off.p;
            uint8_t *stg = (uint8_t *)c->staging.p;
            if (!host_res) {
                st = da.alloc(sg.bytes, &pc.dev);
                if (st == CRAC_OK) st = da.alloc(nseg * 8, &pc.idx_dev);
                if (st == CRAC_OK) st = da.alloc((nseg + 1) * 8, &pc.off_dev);
                if (st != CRAC_OK) {
                    da.free(pc.dev);
                    da.free(pc.idx_dev);
                    da.free(pc.off_dev);
                    return fail(st);
                }
                idx_d = (uint64_t *)pc.idx_dev.p;
                off_d = (uint64_t *)pc.off_dev.p;
                stg = pc.dev.p;
            }
            if (cudaStreamWaitEvent(s, c->ev_last, 0) != cudaSuccess) {
                im->pieces.push_back(pc);
                return fail(cuda_status(cudaGetLastError()));
            }
            CkptCtrl ctrl{};
            st = run_segment(c, sg, (const CkptDesc *)c->desc.p, first, idx_d, off_d, nseg, stg, sg.bytes, s,
                             &ctrl, &ms);
            if (st != CRAC_OK) {
                im->pieces.push_back(pc);
                return fail(st);
            }
            pc.k0 = k_base;
            pc.k = ctrl.k;
            pc.off0 = d_base;
            const bool sparse = c->sparse_ok && !host_res;
            pc.bytes = sparse ? ctrl.payload : ctrl.D;
            pc.span = sparse ? ctrl.D : 0;
            if (fault_hit(CRAC_FAULT_DRAIN)) {
                im->pieces.push_back(pc);
                t_last_cuda = (int)cudaErrorLaunchFailure;
                return fail(CRAC_ERR_CUDA);
            }
            cudaError_t e = cudaStreamWaitEvent(c->side, c->ev_pass, 0);
            if (host_res) {
                if (ctrl.D) {
                    st = pa.alloc(ctrl.D, &pc.host);
                    if (st != CRAC_OK) {
                        im->pieces.push_back(pc);
                        return fail(st);
                    }
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(pc.host.p, c->staging.p, ctrl.D, cudaMemcpyDeviceToHost, c->side);
                }
            } else {
                da.shrink(pc.dev, ctrl.D);
                da.shrink(pc.idx_dev, ctrl.k * 8);
                da.shrink(pc.off_dev, (ctrl.k + 1) * 8);
            }
            if (e == cudaSuccess && ctrl.k && host_res)
                e = cudaMemcpyAsync(im->idx_h.p + k_base * 8, idx_d, ctrl.k * 8, cudaMemcpyDeviceToHost, c->side);
            if (e == cudaSuccess) e = cudaEventRecord(c->ev_last, c->side);
            im->pieces.push_back(pc);
            if (e != cudaSuccess) return fail(cuda_status(e));
            k_base += ctrl.k;
            d_base += pc.bytes;
        }
        cudaError_t e;
        if (host_res) {
            e = cudaMemcpyAsync(im->fp_h.p, c->fp[1 - c->fp_cur].p, n * 8, cudaMemcpyDeviceToHost, c->side);
            if (e == cudaSuccess) e = cudaEventRecord(im->done, c->side);
            if (e == cudaSuccess) e = cudaEventRecord(c->ev_last, c->side);
        } else {
            // Device image: its tables stay in device memory; done once the
            // fingerprint table has its own copy.
            e = cudaMemcpyAsync(im->fp_dev.p, c->fp[1 - c->fp_cur].p, n * 8, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = cudaEventRecord(im->done, s);
            if (e == cudaSuccess) e = cudaEventRecord(c->ev_last, s);
        }
        if (e != cudaSuccess) return fail(cuda_status(e));
        im->k = k_base;
        im->payload_bytes = d_base;
        if (host_res) pa.shrink(im->idx_h, k_base * 8);
        c->last.k = k_base;
        c->last.payload_bytes = d_base;
        c->last.segments = (uint32_t)segs.size();
        c->last.device_ms = ms;
        if (any_managed) {
            float pm = 0;
            cudaEventElapsedTime(&pm, c->ev_p0, c->ev_p1);
            c->last.prefetch_ms = pm;
        }
    } else {
        CK(cudaEventRecord(im->done, s));
    }

    // Commit: the new fingerprints become the baseline.
    im->flags = im->k == n ? CRAC_IMAGE_FULL : 0u;
    if (!(im->flags & CRAC_IMAGE_FULL) && c->parent) {
        img_ref(c->parent);
        im->parent = c->parent;
    }
    c->fp_cur = 1 - c->fp_cur;
    c->base_first.clear();
    for (size_t a = 0; a < na; ++a) c->base_first[c->allocs[a].id] = first[a];
    c->base_valid = true;
    c->epoch_max = im->epoch;
    c->parent_epoch = im->epoch;
    crac_image *img = im.release();
    img->refs.store(2);   // the caller's reference and the context's
    img_unref(c->parent);
    c->parent = img;
    table_add(img);
    *out = img;
    return CRAC_OK;
}

// ---------------------------------------------------------------------------
// Restart
// ---------------------------------------------------------------------------

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

// Restore from a chain held entirely in device memory, resolved on the device
// in three launches over every piece of every image of the chain: owner
// marks (the newest image wins), a coverage check, owner-filtered scatter --
// no host round trip before them.  An uncovered chunk stops the scatter
// (memory untouched) and reports IMAGE_MISMATCH.
crac_status_t restart_device(crac_ctx *c, crac_image *img, const std::vector<crac_image *> &chain, cudaStream_t s) {
    DeviceGuard g(c->device);
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
    const size_t piece_bytes = round_up(std::max<size_t>(n_pieces, 1) * sizeof(RestorePiece), 256);
    TRY(ensure_dev(c->owner, std::max<uint64_t>(nt, 1) * 4));
    TRY(ensure_dev(c->sdesc, desc_bytes + piece_bytes));
    TRY(ensure_host(c->sdesc_h, desc_bytes + piece_bytes));
    TRY(ensure_dev(c->serr, 256));
    TRY(ensure_dev(c->fp[1 - c->fp_cur], std::max<uint64_t>(nt, 1) * 8));
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
        for (const Piece &pc : im->pieces) {
            if (!pc.k) continue;
            rph[ppos++] = RestorePiece{(uint64_t)pc.idx_dev.p, (uint64_t)pc.off_dev.p, (uint64_t)pc.dev.p, pc.k,
                                       entries, pc.span ? pc.span : pc.bytes, (uint32_t)i, (uint32_t)d0,
                                       (uint32_t)im->allocs.size(), 0};
            entries += pc.k;
        }
    }
    for (crac_image *im : chain) CK(cudaStreamWaitEvent(s, im->done, 0));
    CK(cudaStreamWaitEvent(s, c->ev_last, 0));
    CK(cudaMemsetAsync(c->serr.p, 0, 256, s));
    if (nt) CK(cudaMemsetAsync(c->owner.p, 0, nt * 4, s));
    CK(cudaMemcpyAsync(c->sdesc.p, c->sdesc_h.p, desc_bytes + ppos * sizeof(RestorePiece), cudaMemcpyHostToDevice, s));
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
    const uint64_t grid = (uint64_t)c->sm_count * 8;
    CK(cudaEventRecord(c->ev_r0, s));
    CK(launch_restore_mark(P, (int)std::max<uint64_t>(1, std::min<uint64_t>((entries + 255) / 256, grid)), s));
    CK(launch_restore_check(P, (int)std::max<uint64_t>(1, std::min<uint64_t>((nt + 255) / 256, grid)), s));
    CK(launch_restore_scatter(P, (int)std::max<uint64_t>(1, std::min<uint64_t>((entries + 7) / 8, grid)), s));
    CK(cudaEventRecord(c->ev_r1, s));
    if (nt) CK(cudaMemcpyAsync(c->fp[1 - c->fp_cur].p, img->fp_dev.p, nt * 8, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(c->serr_h.p, c->serr.p, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(c->ev_last, s));
    CK(cudaEventSynchronize(c->ev_last));
    const unsigned err = *(const unsigned *)c->serr_h.p;
    if (err & kErrUncovered) return CRAC_ERR_IMAGE_MISMATCH;
    if (err) return CRAC_ERR_CORRUPT;
    cudaEventElapsedTime(&ri.device_ms, c->ev_r0, c->ev_r1);
    c->last_restart = ri;
    c->fp_cur = 1 - c->fp_cur;
    restart_commit(c, img);
    return CRAC_OK;
}

crac_status_t ctx_restart(crac_ctx *c, crac_image *img, cudaStream_t s) {
    if (!img) return CRAC_ERR_INVALID_ARG;
    if (img->state.load() < 0) return img->state.load();
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
        cur = p;
    }
    std::reverse(chain.begin(), chain.end());
    bool all_dev = true;
    for (crac_image *im : chain)
        all_dev = all_dev && im->residency == CRAC_RESIDENCY_DEVICE && im->device == c->device &&
                  (im->n_chunks == 0 || im->fp_dev.region >= 0);
    if (all_dev) return restart_device(c, img, chain, s);
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
    TRY(ensure_dev(c->fp[1 - c->fp_cur], std::max<uint64_t>(nt, 1) * 8));
    CK(cudaEventRecord(c->ev_r1, s));
    if (nt) CK(cudaMemcpyAsync(c->fp[1 - c->fp_cur].p, img->fp_h.p, nt * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(c->serr_h.p, c->serr.p, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaEventRecord(c->ev_last, s));
    CK(cudaEventSynchronize(c->ev_last));
    if (*(const unsigned *)c->serr_h.p) return CRAC_ERR_CORRUPT;
    cudaEventElapsedTime(&ri.device_ms, c->ev_r0, c->ev_r1);
    c->last_restart = ri;
    c->fp_cur = 1 - c->fp_cur;
    restart_commit(c, img);
    (void)na;
    return CRAC_OK;
}

// ---------------------------------------------------------------------------
// Trial passes and the autotuner
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
    c->last = crac_pass_info_t{};
    if (n == 0) return CRAC_OK;
    TRY(ensure_dev(c->fp[1 - c->fp_cur], n * 8));
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
    c->sparse_ok = c->cfg.pass_kernel == CRAC_PASS_SPARSE &&
                   c->cfg.image_residency == CRAC_RESIDENCY_DEVICE && all16;
    CK(cudaStreamWaitEvent(s, c->ev_last, 0));
    CK(cudaMemcpyAsync(c->desc.p, dh, na * (sizeof(CkptDesc) + 8), cudaMemcpyHostToDevice, s));
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
                        sg.c1 - sg.c0, (uint8_t *)c->staging.p, sg.bytes, s, &ctrl, ms));
        *k_out += ctrl.k;
        *d_out += c->sparse_ok ? ctrl.payload : ctrl.D;
    }
    CK(cudaEventRecord(c->ev_last, s));
    if (commit) {
        c->prev_base_first = c->base_first;
        c->prev_base_valid = c->base_valid;
        c->fp_cur = 1 - c->fp_cur;
        c->base_first.clear();
        for (size_t a = 0; a < na; ++a) c->base_first[c->allocs[a].id] = first[a];
        c->base_valid = true;
    }
    return CRAC_OK;
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
        t->fp_cur = 1 - t->fp_cur;
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
    auto time_pass = [&](float *best_ms) {
        for (int r = 0; r < 2; ++r) {
            float ms = 0;
            uint64_t k = 0, d = 0;
            TRY(ctx_trial_pass(t, s, false, &ms, &k, &d));
            if (r == 0 || ms < *best_ms) *best_ms = ms;
        }
        return CRAC_OK;
    };
    for (uint32_t v : {(uint32_t)CRAC_PASS_SPLIT, (uint32_t)CRAC_PASS_LDG, (uint32_t)CRAC_PASS_TMA,
                       (uint32_t)CRAC_PASS_SPARSE}) {
        if (v == CRAC_PASS_TMA && (S < 1024 || S > 65536)) continue;
        if (v == CRAC_PASS_SPARSE && t->cfg.image_residency != CRAC_RESIDENCY_DEVICE) continue;
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
                return st;
            }
            if (v == CRAC_PASS_LDG) vt->tile_ms[j] = ms;
            if (bestm == 0 || ms < bestm) {
                bestm = ms;
                if (ldg_tiles) vt->best_tile = vt->tiles[j];
            }
        }
        vt->vms[v] = bestm;
        if (vt->vms[vt->best_v] == 0 || bestm < vt->vms[vt->best_v]) vt->best_v = v;
    }
    t->cfg.pass_kernel = saved;
    if (vt->best_v != CRAC_PASS_LDG) vt->best_tile = 0;
    return CRAC_OK;
}

crac_status_t ctx_tune_apply(crac_ctx *c, cudaStream_t s, double link_gbs, crac_tune_result_t *out) {
    if (c->tune_ctx.empty() || c->tune_rounds == 0) return CRAC_ERR_UNSUPPORTED;
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
        c->base_valid = false;
        c->base_first.clear();
    }
    c->cfg.pass_kernel = win_vt.best_v;
    tune_clear(c);
    return CRAC_OK;
}

// ---------------------------------------------------------------------------
// Request server
// ---------------------------------------------------------------------------

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Run an operation of `c` with a leased staging buffer in place of its own.
template <class F>
crac_status_t with_staging(crac_ctx *c, void *p, uint64_t bytes, F &&op) {
    const DevBuf saved = c->staging;
    const uint64_t saved_cfg = c->cfg.staging_bytes;
    if (p) {
        c->staging = DevBuf{p, (size_t)bytes};
        c->cfg.staging_bytes = bytes;
    }
    const crac_status_t st = op();
    if (p) {
        c->staging = saved;
        c->cfg.staging_bytes = saved_cfg;
    }
    return st;
}

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
        crac_status_t st;
        {
            std::lock_guard<std::mutex> lk(q->ctx->mu);
            st = ctx_cuda_ready(q->ctx);
            if (st == CRAC_OK) {
                if (q->r.type == CRAC_REQ_CHECKPOINT) {
                    crac_image *img = nullptr;
                    st = with_staging(q->ctx, lease, q->r.lease_bytes,
                                      [&] { return ctx_checkpoint(q->ctx, q->stream, &img); });
                    if (st == CRAC_OK) {
                        q->r.image = img;
                        q->r.payload_bytes = img->payload_bytes;
                    }
                } else {
                    st = with_staging(q->ctx, lease, q->r.lease_bytes,
                                      [&] { return ctx_restart(q->ctx, q->img, q->stream); });
                    if (st == CRAC_OK) q->r.payload_bytes = q->img->payload_bytes;
                }
            }
        }
        // The lease is free once the drain has finished reading it.
        if (st == CRAC_OK && q->r.image) st = img_wait(q->r.image, 0);
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

crac_ctx *g_default = nullptr;
std::mutex g_default_mu;

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

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

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
    const crac_status_t st = ctx_init(c, cfg);
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
        (kind != CRAC_KIND_DEVICE && kind != CRAC_KIND_MANAGED))
        return CRAC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    const uint64_t p = (uint64_t)(uintptr_t)ptr;
    if (p + bytes < p) return CRAC_ERR_INVALID_ARG;
    for (const AllocRec &r : ctx->allocs)
        if (p < r.ptr + r.bytes && r.ptr < p + bytes) return CRAC_ERR_OVERLAP;
    ctx->allocs.push_back(AllocRec{ctx->next_id++, p, (uint64_t)bytes, (uint32_t)kind});
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

crac_status_t crac_ctx_invalidate(crac_ctx_t *ctx) {
    if (!ctx) return CRAC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->base_valid = false;
    ctx->base_first.clear();
    return CRAC_OK;
}

crac_status_t crac_ctx_last_pass(crac_ctx_t *ctx, crac_pass_info_t *out) {
    if (!ctx || !out) return CRAC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
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

crac_status_t crac_image_wait(const crac_image_t *image, uint64_t timeout_ns) {
    if (!image) return CRAC_ERR_INVALID_ARG;
    return img_wait(image, timeout_ns);
}

crac_status_t crac_image_info(const crac_image_t *image, crac_image_info_t *out) {
    if (!image || !out) return CRAC_ERR_INVALID_ARG;
    crac_image *im = const_cast<crac_image *>(image);
    if (im->state.load() == 0 && im->done && cudaEventQuery(im->done) == cudaSuccess) im->state.store(1);
    cudaGetLastError();
    std::memset(out, 0, sizeof(*out));
    out->lineage = im->lineage;
    out->epoch = im->epoch;
    out->parent_epoch = im->parent_epoch;
    out->flags = im->flags;
    out->chunk_bytes = im->chunk_bytes;
    out->n_allocs = im->allocs.size();
    out->n_chunks = im->n_chunks;
    out->k = im->k;
    out->payload_bytes = im->payload_bytes;
    out->serialized_bytes = kHeaderBytes + kAllocEntryBytes * im->allocs.size() + 8 * im->n_chunks + 8 * im->k +
                            im->payload_bytes;
    out->residency = im->residency;
    out->complete = im->state.load() == 1 ? 1u : 0u;
    return CRAC_OK;
}

static void put32(uint8_t *&p, uint32_t v) {
    for (int i = 0; i < 4; ++i) *p++ = (uint8_t)(v >> (8 * i));
}
static void put64(uint8_t *&p, uint64_t v) {
    for (int i = 0; i < 8; ++i) *p++ = (uint8_t)(v >> (8 * i));
}
static uint32_t get32(const uint8_t *p) {
    uint32_t v = 0;
    for (int i = 0; i < 4; ++i) v |= (uint32_t)p[i] << (8 * i);
    return v;
}
static uint64_t get64(const uint8_t *p) {
    uint64_t v = 0;
    for (int i = 0; i < 8; ++i) v |= (uint64_t)p[i] << (8 * i);
    return v;
}

namespace {
// Compact payload of a sparse device piece: its dirty chunks, in list order,
// taken from their uncompacted offsets.
crac_status_t sparse_compact(const crac_image *im, const Piece &pc, uint8_t *out) {
    std::vector<uint8_t> span(pc.span);
    std::vector<uint64_t> off(pc.k);
    CK(cudaMemcpy(span.data(), pc.dev.p, pc.span, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(off.data(), pc.off_dev.p, pc.k * 8, cudaMemcpyDeviceToHost));
    const uint64_t *idx = (const uint64_t *)im->idx_h.p + pc.k0;
    const uint32_t log2S = log2u(im->chunk_bytes);
    uint64_t o = 0;
    size_t a = 0;
    for (uint64_t j = 0; j < pc.k; ++j) {
        const uint64_t c = idx[j];   // ascending
        while (a + 1 < im->allocs.size() && im->allocs[a + 1].first_chunk <= c) ++a;
        const uint64_t len = chunk_len(im->allocs[a].bytes, c - im->allocs[a].first_chunk, log2S);
        if (off[j] + len > pc.span || o + len > pc.bytes) return CRAC_ERR_CORRUPT;
        std::memcpy(out + o, span.data() + off[j], len);
        o += len;
    }
    return o == pc.bytes ? CRAC_OK : CRAC_ERR_CORRUPT;
}
}  // namespace

crac_status_t crac_image_serialize(const crac_image_t *image, void *dst, size_t cap, size_t *need) {
    if (!image || !need) return CRAC_ERR_INVALID_ARG;
    crac_image *im = const_cast<crac_image *>(image);
    const uint64_t total = kHeaderBytes + kAllocEntryBytes * im->allocs.size() + 8 * im->n_chunks + 8 * im->k +
                           im->payload_bytes;
    *need = (size_t)total;
    if (!dst) return CRAC_OK;
    if (cap < total) return CRAC_ERR_INVALID_ARG;
    TRY(img_wait(im, 0));
    TRY(img_host_tables(im));
    uint8_t *p = (uint8_t *)dst;
    std::memcpy(p, "CRACIMG1", 8);
    p += 8;
    put32(p, 1);
    put32(p, im->flags);
    put32(p, im->chunk_bytes);
    put32(p, 1);
    put64(p, im->lineage);
    put64(p, im->epoch);
    put64(p, im->parent_epoch);
    put64(p, im->allocs.size());
    put64(p, im->n_chunks);
    put64(p, im->k);
    put64(p, im->payload_bytes);
    for (const ImgAlloc &a : im->allocs) {
        put64(p, a.id);
        put64(p, a.orig_ptr);
        put64(p, a.bytes);
        put32(p, a.kind);
        put32(p, 0);
        put64(p, a.first_chunk);
    }
    if (im->n_chunks) std::memcpy(p, im->fp_h.p, 8 * im->n_chunks);
    p += 8 * im->n_chunks;
    if (im->k) std::memcpy(p, im->idx_h.p, 8 * im->k);
    p += 8 * im->k;
    for (const Piece &pc : im->pieces) {
        if (!pc.bytes) continue;
        if (im->residency == CRAC_RESIDENCY_DEVICE) {
            DeviceGuard g(im->device);
            if (pc.span) TRY(sparse_compact(im, pc, p + pc.off0));
            else CK(cudaMemcpy(p + pc.off0, pc.dev.p, pc.bytes, cudaMemcpyDeviceToHost));
        } else {
            std::memcpy(p + pc.off0, pc.host.p, pc.bytes);
        }
    }
    return CRAC_OK;
}

crac_status_t crac_image_deserialize(const void *src, size_t n, crac_image_t **out) {
    if (!src || !out) return CRAC_ERR_INVALID_ARG;
    *out = nullptr;
    const uint8_t *b = (const uint8_t *)src;
    if (n < kHeaderBytes || std::memcmp(b, "CRACIMG1", 8) != 0) return CRAC_ERR_CORRUPT;
    if (get32(b + 8) != 1 || get32(b + 20) != 1) return CRAC_ERR_CORRUPT;
    const uint32_t flags = get32(b + 12), chunk = get32(b + 16);
    if (chunk < 16 || chunk > (1u << 24) || (chunk & (chunk - 1)) || (flags & ~CRAC_IMAGE_FULL)) return CRAC_ERR_CORRUPT;
    const uint64_t na = get64(b + 48), nc = get64(b + 56), k = get64(b + 64), pb = get64(b + 72);
    if (na > (n / kAllocEntryBytes) || nc > n / 8 || k > nc || pb > n) return CRAC_ERR_CORRUPT;
    const uint64_t need = kHeaderBytes + kAllocEntryBytes * na + 8 * nc + 8 * k + pb;
    if (need != n) return CRAC_ERR_CORRUPT;
    std::unique_ptr<crac_image> im(new crac_image());
    cudaGetDevice(&im->device);
    im->flags = flags;
    im->chunk_bytes = chunk;
    im->residency = CRAC_RESIDENCY_HOST;
    im->lineage = get64(b + 24);
    im->epoch = get64(b + 32);
    im->parent_epoch = get64(b + 40);
    im->n_chunks = nc;
    im->k = k;
    im->payload_bytes = pb;
    const uint32_t log2S = log2u(chunk);
    const uint8_t *p = b + kHeaderBytes;
    uint64_t expect_first = 0;
    im->allocs.resize(na);
    for (uint64_t a = 0; a < na; ++a, p += kAllocEntryBytes) {
        ImgAlloc &r = im->allocs[a];
        r = ImgAlloc{get64(p), get64(p + 8), get64(p + 16), get32(p + 24), get64(p + 32)};
        if (r.bytes == 0 || r.kind > 1 || r.first_chunk != expect_first) return CRAC_ERR_CORRUPT;
        expect_first += ((r.bytes - 1) >> log2S) + 1;
    }
    if (expect_first != nc || ((flags & CRAC_IMAGE_FULL) != 0) != (k == nc)) return CRAC_ERR_CORRUPT;
    const uint8_t *fp = p, *idx = p + 8 * nc, *payload = idx + 8 * k;
    // idx strictly ascending and payload length equal to the listed chunks' lengths
    uint64_t acc = 0, prev = 0;
    size_t a = 0;
    for (uint64_t j = 0; j < k; ++j) {
        const uint64_t c = get64(idx + 8 * j);
        if (c >= nc || (j && c <= prev)) return CRAC_ERR_CORRUPT;
        prev = c;
        while (a + 1 < na && im->allocs[a + 1].first_chunk <= c) ++a;
        acc += chunk_len(im->allocs[a].bytes, c - im->allocs[a].first_chunk, log2S);
    }
    if (acc != pb) return CRAC_ERR_CORRUPT;
    Arena &pa = pinned_arena();
    crac_status_t st = CRAC_OK;
    Piece pc;
    pc.k = k;
    pc.bytes = pb;
    if (nc) st = pa.alloc(8 * nc, &im->fp_h);
    if (st == CRAC_OK && k) st = pa.alloc(8 * k, &im->idx_h);
    if (st == CRAC_OK && pb) st = pa.alloc(pb, &pc.host);
    if (st != CRAC_OK) {
        im->pieces.push_back(pc);
        free_image_blocks(im.release());
        return st;
    }
    if (nc) std::memcpy(im->fp_h.p, fp, 8 * nc);
    if (k) std::memcpy(im->idx_h.p, idx, 8 * k);
    if (pb) std::memcpy(pc.host.p, payload, pb);
    im->pieces.push_back(pc);
    im->state.store(1);
    crac_image *img = im.release();
    table_add(img);
    *out = img;
    return CRAC_OK;
}

crac_status_t crac_image_release(crac_image_t *image) {
    if (!image) return CRAC_ERR_INVALID_ARG;
    img_unref(image);
    return CRAC_OK;
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
    return CRAC_OK;
}

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
