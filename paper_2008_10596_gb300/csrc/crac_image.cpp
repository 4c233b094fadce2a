// The image store: reference counts, completion, host copies of device
// tables, delta chains, and the image part of the C ABI.
#include "crac_runtime.h"

using namespace crac;

namespace {

std::mutex g_img_mu;
std::multimap<std::pair<uint64_t, uint64_t>, crac_image *> g_images;   // (lineage, epoch)

}  // namespace

namespace crac {

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
            const crac_status_t st = img_resolve(im);   // an unsettled pass: its counts, its errors
            int zero = 0;
            if (st == CRAC_OK) im->state.compare_exchange_strong(zero, 1);
            return im->state.load() < 0 ? im->state.load() : CRAC_OK;
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
            if (im->drain0) cudaEventDestroy(im->drain0);
            cudaGetLastError();
        }
        table_remove(im);
        if (im->dep) img_unref(im->dep);
        Arena &pa = pinned_arena();
        pa.free(im->ctrl_b);
        pa.free(im->fp_h);
        pa.free(im->idx_h);
        pa.free(im->off_h);
        pa.free(im->zlen_h);
        if (im->fp_dev.region >= 0) device_arena(im->device).free(im->fp_dev);
        for (Piece &p : im->pieces) {
            pa.free(p.host);
            if (p.dev.region >= 0 || p.idx_dev.region >= 0 || p.off_dev.region >= 0 || p.zlen_dev.region >= 0) {
                Arena &da = device_arena(im->device);
                da.free(p.dev);
                da.free(p.idx_dev);
                da.free(p.off_dev);
                da.free(p.zlen_dev);
            }
        }
        crac_image *parent = im->parent;
        delete im;
        im = parent;
    }
}

// Host copies of a device image's fingerprint table and chunk list (made on
// the first request: serialization, or a restart chain resolved on the host).
// A checkpoint that returned before its pass finished, once `done` has
// completed: the pass's control block gives the dirty count and bytes, which
// become the image's k, payload size, FULL flag and block sizes; an error bit
// (or the failure of the context's previous unsettled image, whose
// fingerprints this pass compared against) fails the image.  Idempotent;
// the failure is stored in `state`.
crac_status_t img_resolve(crac_image *im) {
    crac_image *dep = nullptr;
    {
        std::lock_guard<std::mutex> lk(im->mu);
        if (!im->deferred) return im->state.load() < 0 ? im->state.load() : CRAC_OK;
        dep = im->dep;
        im->dep = nullptr;
    }
    crac_status_t st = CRAC_OK;
    if (dep) {
        st = img_wait(dep, 0);
        img_unref(dep);
    }
    crac_image *drop = nullptr;
    {
        std::lock_guard<std::mutex> lk(im->mu);
        if (!im->deferred) return im->state.load() < 0 ? im->state.load() : CRAC_OK;
        const CkptCtrl ctrl = *(const CkptCtrl *)im->ctrl_b.p;
        if (st == CRAC_OK) {
            if (ctrl.err & kErrLostCopy) {
                im->lost = true;
                st = CRAC_ERR_CUDA;
            } else if (ctrl.err & kErrTimeout) {
                st = CRAC_ERR_TIMEOUT;
            } else if (ctrl.err) {
                st = CRAC_ERR_CORRUPT;
            }
        }
        Piece &pc = im->pieces[0];
        const bool host = im->residency != CRAC_RESIDENCY_DEVICE;
        const uint64_t bytes = im->sparse_pass ? ctrl.payload : ctrl.D;
        uint64_t total = 0;
        for (const ImgAlloc &a : im->allocs) total += a.bytes;
        if (st == CRAC_OK && (ctrl.k > im->n_chunks || ctrl.D > total ||
                              (im->predicted_full && (ctrl.k != im->n_chunks || ctrl.D != total))))
            st = CRAC_ERR_CORRUPT;
        if (st == CRAC_OK) {
            im->spec_hits = ctrl.spec_hits;
            im->spec_writes = ctrl.spec_writes;
            pc.k = ctrl.k;
            pc.bytes = bytes;
            pc.span = im->sparse_pass ? ctrl.D : 0;
            im->k = ctrl.k;
            im->payload_bytes = bytes;
            im->raw_bytes = bytes;
            if (host) {
                Arena &pa = pinned_arena();
                if (bytes) pa.shrink(pc.host, bytes);
                else pa.free(pc.host);
                pa.shrink(im->idx_h, ctrl.k * 8);
            } else {
                Arena &da = device_arena(im->device);
                da.shrink(pc.dev, ctrl.D);   // sparse: the span
                da.shrink(pc.idx_dev, ctrl.k * 8);
                da.shrink(pc.off_dev, (ctrl.k + 1) * 8);
            }
            im->flags = (im->flags & ~CRAC_IMAGE_FULL) | (ctrl.k == im->n_chunks ? CRAC_IMAGE_FULL : 0u);
            if ((im->flags & CRAC_IMAGE_FULL) && im->parent) {   // a FULL image needs no parent
                drop = im->parent;
                im->parent = nullptr;
            }
        } else {
            im->state.store(st);
        }
        pinned_arena().free(im->ctrl_b);
        im->deferred = false;
    }
    img_unref(drop);
    return st;
}

crac_status_t img_host_tables(crac_image *im) {
    std::lock_guard<std::mutex> lk(im->mu);
    if (im->host_tables) return CRAC_OK;
    TRY(img_wait(im, 0));
    Arena &pa = pinned_arena();
    if (im->n_chunks) TRY(pa.alloc(im->n_chunks * 8, &im->fp_h));
    if (im->k) TRY(pa.alloc(im->k * 8, &im->idx_h));
    const bool coded = (im->flags & CRAC_IMAGE_CODED) != 0;
    if (im->k && coded) TRY(pa.alloc(im->k * 8, &im->zlen_h));
    DeviceGuard g(im->device);
    if (im->n_chunks) CK(cudaMemcpy(im->fp_h.p, im->fp_dev.p, im->n_chunks * 8, cudaMemcpyDeviceToHost));
    for (const Piece &pc : im->pieces) {
        if (pc.k) CK(cudaMemcpy(im->idx_h.p + pc.k0 * 8, pc.idx_dev.p, pc.k * 8, cudaMemcpyDeviceToHost));
        if (pc.k && coded)
            CK(cudaMemcpy(im->zlen_h.p + pc.k0 * 8, pc.zlen_dev.p, pc.k * 8, cudaMemcpyDeviceToHost));
    }
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

void free_image_blocks(crac_image *im) {
    im->refs.store(1);
    im->parent = nullptr;
    img_unref(im);
}

}  // namespace crac

static uint64_t serialized_size(const crac_image *im) {
    const uint64_t tables = 8 * im->k * ((im->flags & CRAC_IMAGE_CODED) ? 2 : 1);
    return kHeaderBytes + kAllocEntryBytes * im->allocs.size() + 8 * im->n_chunks + tables + im->payload_bytes;
}

extern "C" {

crac_status_t crac_image_wait(const crac_image_t *image, uint64_t timeout_ns) {
    if (!image) return CRAC_ERR_INVALID_ARG;
    return img_wait(image, timeout_ns);
}

crac_status_t crac_image_info(const crac_image_t *image, crac_image_info_t *out) {
    if (!image || !out) return CRAC_ERR_INVALID_ARG;
    crac_image *im = const_cast<crac_image *>(image);
    bool unsettled;
    {
        std::lock_guard<std::mutex> lk(im->mu);
        unsettled = im->deferred;
    }
    if (unsettled) {
        img_wait(im, 0);   // its counts are known once its pass has finished
    } else if (im->state.load() == 0 && im->done && cudaEventQuery(im->done) == cudaSuccess) {
        im->state.store(1);
    }
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
    out->serialized_bytes = serialized_size(im);
    out->residency = im->residency;
    out->complete = im->state.load() == 1 ? 1u : 0u;
    out->raw_bytes = im->raw_bytes;
    if (out->complete && im->drain0 && im->done) {
        DeviceGuard g(im->device);
        float ms = 0;
        if (cudaEventElapsedTime(&ms, im->drain0, im->done) == cudaSuccess) out->drain_ms = ms;
        cudaGetLastError();
    }
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

// Header and allocation table of the serialized form.
std::vector<uint8_t> image_prefix(const crac_image *im) {
    std::vector<uint8_t> v(kHeaderBytes + kAllocEntryBytes * im->allocs.size());
    uint8_t *p = v.data();
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
    return v;
}

// A sparse device piece's host tables (span offset and compact offset of
// every entry), made once per piece.
crac_status_t sparse_tables(crac_image *im, Piece &pc) {
    std::lock_guard<std::mutex> lk(im->mu);
    if (!pc.sp_cum.empty()) return CRAC_OK;
    std::vector<uint64_t> off(pc.k), cum(pc.k + 1);
    if (pc.k) CK(cudaMemcpy(off.data(), pc.off_dev.p, pc.k * 8, cudaMemcpyDeviceToHost));
    const uint64_t *idx = (const uint64_t *)im->idx_h.p + pc.k0;
    const uint32_t log2S = log2u(im->chunk_bytes);
    size_t a = 0;
    cum[0] = 0;
    for (uint64_t j = 0; j < pc.k; ++j) {
        const uint64_t c = idx[j];   // ascending
        while (a + 1 < im->allocs.size() && im->allocs[a + 1].first_chunk <= c) ++a;
        const uint64_t len = chunk_len(im->allocs[a].bytes, c - im->allocs[a].first_chunk, log2S);
        if (off[j] > pc.span || len > pc.span - off[j]) return CRAC_ERR_CORRUPT;
        cum[j + 1] = cum[j] + len;
    }
    if (cum[pc.k] != pc.bytes) return CRAC_ERR_CORRUPT;
    pc.sp_off.swap(off);
    pc.sp_cum.swap(cum);
    return CRAC_OK;
}

// Bytes [a, b) of a sparse piece's compact payload (its entries' chunks in
// list order, taken from their offsets in the span): one copy per run of
// entries that lie back to back in the span when there are few runs, else
// the entries are packed on the device (sparse_pack_kernel) in windows of
// up to 256 MiB and each window is copied out once.
crac_status_t sparse_range(crac_image *im, Piece &pc, uint64_t a, uint64_t b, uint8_t *out) {
    TRY(sparse_tables(im, pc));
    const std::vector<uint64_t> &off = pc.sp_off, &cum = pc.sp_cum;
    const uint64_t j0 = (uint64_t)(std::upper_bound(cum.begin(), cum.end(), a) - cum.begin()) - 1;
    const uint64_t j1 = std::min<uint64_t>(pc.k, (uint64_t)(std::lower_bound(cum.begin(), cum.end(), b) - cum.begin()));
    uint64_t runs = 1;
    for (uint64_t j = j0 + 1; j < j1 && runs <= 64; ++j) runs += off[j] != off[j - 1] + (cum[j] - cum[j - 1]);
    if (runs > 64) {
        constexpr uint64_t kWindow = 256ull << 20;
        Arena &da = device_arena(im->device);
        Block win, dcum;
        TRY(da.alloc(std::min<uint64_t>(kWindow, cum[j1] - cum[j0]), &win));
        crac_status_t st = da.alloc((j1 - j0 + 1) * 8, &dcum);
        if (st == CRAC_OK) {
            const cudaError_t e = cudaMemcpy(dcum.p, cum.data() + j0, (j1 - j0 + 1) * 8, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) st = cuda_status(e);
        }
        for (uint64_t w0 = j0; st == CRAC_OK && w0 < j1;) {
            uint64_t w1 = w0 + 1;   // one entry always fits: entries are at most a chunk
            while (w1 < j1 && cum[w1 + 1] - cum[w0] <= kWindow) ++w1;
            cudaError_t e = launch_sparse_pack(win.p, pc.dev.p, (const uint64_t *)pc.off_dev.p + w0,
                                               (const uint64_t *)dcum.p + (w0 - j0), w1 - w0, 1024, 0);
            const uint64_t lo = std::max(a, cum[w0]), hi = std::min(b, cum[w1]);
            if (e == cudaSuccess && lo < hi)
                e = cudaMemcpy(out + (lo - a), win.p + (lo - cum[w0]), hi - lo, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) st = cuda_status(e);
            w0 = w1;
        }
        da.free(dcum);
        da.free(win);
        return st;
    }
    uint64_t j = j0;
    uint64_t pos = a;
    while (pos < b && j < pc.k) {
        const uint64_t src = off[j] + (pos - cum[j]);
        uint64_t jj = j;
        while (cum[jj + 1] < b && jj + 1 < pc.k && off[jj + 1] == off[jj] + (cum[jj + 1] - cum[jj])) ++jj;
        const uint64_t take = std::min(cum[jj + 1], b) - pos;
        CK(cudaMemcpy(out + (pos - a), pc.dev.p + src, take, cudaMemcpyDeviceToHost));
        pos += take;
        j = jj + 1;
    }
    return pos == b ? CRAC_OK : CRAC_ERR_CORRUPT;
}

// Bytes [offset, offset + n) of the serialized form into host memory dst.
// Serialization is the whole range; ranged reads let a caller stream an
// image out (to a file, or to a checker) without holding it whole.
crac_status_t read_range(crac_image *im, uint64_t offset, uint8_t *dst, uint64_t n) {
    TRY(img_wait(im, 0));   // an unsettled pass's sizes are known once it has finished
    const uint64_t total = serialized_size(im);
    if (offset > total || n > total - offset) return CRAC_ERR_INVALID_ARG;
    if (n == 0) return CRAC_OK;
    TRY(img_host_tables(im));
    const uint64_t end = offset + n;
    // Copy the part of section [s0, s0 + len) that the range covers.
    auto part = [&](uint64_t s0, uint64_t len, const std::function<crac_status_t(uint64_t, uint64_t, uint8_t *)> &copy) {
        const uint64_t a = std::max(offset, s0), b = std::min(end, s0 + len);
        return a < b ? copy(a - s0, b - a, dst + (a - offset)) : CRAC_OK;
    };
    auto from_host = [](const uint8_t *src) {
        return [src](uint64_t o, uint64_t l, uint8_t *out) {
            std::memcpy(out, src + o, l);
            return CRAC_OK;
        };
    };
    const std::vector<uint8_t> pre = image_prefix(im);
    uint64_t pos = 0;
    TRY(part(pos, pre.size(), from_host(pre.data())));
    pos += pre.size();
    TRY(part(pos, 8 * im->n_chunks, from_host(im->fp_h.p)));
    pos += 8 * im->n_chunks;
    TRY(part(pos, 8 * im->k, from_host(im->idx_h.p)));
    pos += 8 * im->k;
    if (im->flags & CRAC_IMAGE_CODED) {
        TRY(part(pos, 8 * im->k, from_host(im->zlen_h.p)));
        pos += 8 * im->k;
    }
    DeviceGuard g(im->device);
    for (Piece &pc : im->pieces) {
        if (!pc.bytes) continue;
        TRY(part(pos + pc.off0, pc.bytes, [&](uint64_t o, uint64_t l, uint8_t *out) -> crac_status_t {
            if (im->residency != CRAC_RESIDENCY_DEVICE) {
                std::memcpy(out, pc.host.p + o, l);
                return CRAC_OK;
            }
            if (pc.span) return sparse_range(im, pc, o, o + l, out);
            CK(cudaMemcpy(out, pc.dev.p + o, l, cudaMemcpyDeviceToHost));
            return CRAC_OK;
        }));
    }
    return CRAC_OK;
}

}  // namespace

crac_status_t crac_image_serialize(const crac_image_t *image, void *dst, size_t cap, size_t *need) {
    if (!image || !need) return CRAC_ERR_INVALID_ARG;
    crac_image *im = const_cast<crac_image *>(image);
    TRY(img_wait(im, 0));
    const uint64_t total = serialized_size(im);
    *need = (size_t)total;
    if (!dst) return CRAC_OK;
    if (cap < total) return CRAC_ERR_INVALID_ARG;
    return read_range(im, 0, (uint8_t *)dst, total);
}

crac_status_t crac_image_read(const crac_image_t *image, uint64_t offset, void *dst, size_t n) {
    if (!image || (!dst && n)) return CRAC_ERR_INVALID_ARG;
    return read_range(const_cast<crac_image *>(image), offset, (uint8_t *)dst, n);
}

// A coded CRZ1 stream of z bytes for a chunk of L bytes (z < L): every block
// header has its reserved bits (48..63) clear and plane widths of at most 8,
// and the header-padded length plus 16 bytes per unit plus the tail is z.
// What only decoding can find (a plane value above 255) is left to the
// restore.
static bool crz_stream_header_ok(const uint8_t *s, uint64_t z, uint64_t L) {
    const uint64_t nb = L / 512, tail = L % 512, head = 16 * ((nb + 1) / 2);
    if (nb == 0 || z < head) return false;
    uint64_t units = 0;
    for (uint64_t b = 0; b < nb; ++b) {
        const uint64_t h = get64(s + 8 * b);
        if (h >> 48) return false;
        for (int p = 0; p < 4; ++p) {
            const uint64_t w = (h >> (32 + 4 * p)) & 0xF;
            if (w > 8) return false;
            units += w;
        }
    }
    return head + 16 * units + tail == z;
}

crac_status_t crac_image_deserialize(const void *src, size_t n, crac_image_t **out) {
    if (!src || !out) return CRAC_ERR_INVALID_ARG;
    *out = nullptr;
    const uint8_t *b = (const uint8_t *)src;
    if (n < kHeaderBytes || std::memcmp(b, "CRACIMG1", 8) != 0) return CRAC_ERR_CORRUPT;
    if (get32(b + 8) != 1 || get32(b + 20) != 1) return CRAC_ERR_CORRUPT;
    const uint32_t flags = get32(b + 12), chunk = get32(b + 16);
    if (chunk < 16 || chunk > (1u << 24) || (chunk & (chunk - 1)) || (flags & ~(CRAC_IMAGE_FULL | CRAC_IMAGE_CODED)))
        return CRAC_ERR_CORRUPT;
    const bool coded = (flags & CRAC_IMAGE_CODED) != 0;
    const uint64_t na = get64(b + 48), nc = get64(b + 56), k = get64(b + 64), pb = get64(b + 72);
    if (na > (n / kAllocEntryBytes) || nc > n / 8 || k > nc || pb > n) return CRAC_ERR_CORRUPT;
    const uint64_t need = kHeaderBytes + kAllocEntryBytes * na + 8 * nc + 8 * k * (coded ? 2 : 1) + pb;
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
        if (r.bytes == 0 || r.kind > CRAC_KIND_HOST || r.first_chunk != expect_first) return CRAC_ERR_CORRUPT;
        expect_first += ((r.bytes - 1) >> log2S) + 1;
    }
    if (expect_first != nc || ((flags & CRAC_IMAGE_FULL) != 0) != (k == nc)) return CRAC_ERR_CORRUPT;
    const uint8_t *fp = p, *idx = p + 8 * nc, *zlen = idx + 8 * k, *payload = zlen + (coded ? 8 * k : 0);
    // idx strictly ascending; payload length equal to the listed chunks'
    // lengths, or (coded) to their streams' padded lengths, no stream longer
    // than its chunk
    uint64_t acc = 0, zacc = 0, prev = 0;
    size_t a = 0;
    for (uint64_t j = 0; j < k; ++j) {
        const uint64_t c = get64(idx + 8 * j);
        if (c >= nc || (j && c <= prev)) return CRAC_ERR_CORRUPT;
        prev = c;
        while (a + 1 < na && im->allocs[a + 1].first_chunk <= c) ++a;
        const uint64_t len = chunk_len(im->allocs[a].bytes, c - im->allocs[a].first_chunk, log2S);
        acc += len;
        if (coded) {
            const uint64_t z = get64(zlen + 8 * j);
            if (z == 0 || z > len || zacc > pb || z > pb - zacc) return CRAC_ERR_CORRUPT;
            if (z < len && !crz_stream_header_ok(payload + zacc, z, len)) return CRAC_ERR_CORRUPT;
            zacc += round_up(z, 16);
        }
    }
    if ((coded ? zacc : acc) != pb) return CRAC_ERR_CORRUPT;
    im->raw_bytes = acc;
    Arena &pa = pinned_arena();
    crac_status_t st = CRAC_OK;
    Piece pc;
    pc.k = k;
    pc.bytes = pb;
    if (nc) st = pa.alloc(8 * nc, &im->fp_h);
    if (st == CRAC_OK && k) st = pa.alloc(8 * k, &im->idx_h);
    if (st == CRAC_OK && k && coded) st = pa.alloc(8 * k, &im->zlen_h);
    if (st == CRAC_OK && pb) st = pa.alloc(pb, &pc.host);
    if (st != CRAC_OK) {
        im->pieces.push_back(pc);
        free_image_blocks(im.release());
        return st;
    }
    if (nc) std::memcpy(im->fp_h.p, fp, 8 * nc);
    if (k) std::memcpy(im->idx_h.p, idx, 8 * k);
    if (k && coded) std::memcpy(im->zlen_h.p, zlen, 8 * k);
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

}  // extern "C"
