// Internal interface between the host runtime (crac_runtime.h and its units)
// and the device kernel units (crac_pass_*.cu, crac_restore.cu,
// crac_noalloc.cu).  Not part of the public ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace crac {

// One registered allocation as the checkpoint pass sees it.
struct CkptDesc {
    uint64_t ptr;          // device / managed address (16-byte aligned)
    uint64_t bytes;        // allocation size
    uint64_t first_chunk;  // global id of its first chunk in this layout
    uint64_t base_first;   // its first chunk in the baseline table, or kNoBase
};
constexpr uint64_t kNoBase = ~0ull;

// Control block of one pass launch; zeroed before every launch.
struct CkptCtrl {
    unsigned int ticket;       // next tile to hand out
    unsigned int err;          // kErr* bits
    unsigned long long k;      // dirty chunks in this segment
    unsigned long long D;      // dirty bytes in this segment (sparse pass: all its bytes)
    unsigned long long payload;  // sparse pass: dirty bytes in this segment
    unsigned long long spec_hits;  // split pass: dirty entries found in place (predicted write-through)
    unsigned long long spec_writes;  // ... and chunks written speculatively
    unsigned long long pad[2];
};
static_assert(sizeof(CkptCtrl) == 64, "CkptCtrl layout");
constexpr unsigned kErrTimeout = 1u;   // a look-back wait ran out
constexpr unsigned kErrBounds = 2u;    // an output index/offset exceeded its buffer
constexpr unsigned kErrUncovered = 4u; // restore: a target chunk no image of the chain holds
constexpr unsigned kErrCodec = 8u;     // restore: a coded stream no chunk encodes to
constexpr unsigned kErrLostCopy = 16u; // a bulk copy into shared memory never completed, even
                                       // after the CTA waited for it in bounded rounds: the
                                       // device's state is unspecified
constexpr int kCopyDrainRounds = 8;    // bounded waits for an in-flight bulk copy before a CTA exits

// Parameters of the fused batched pass over global chunks [c_begin, c_end).
struct CkptParams {
    const CkptDesc *desc;
    uint32_t n_allocs;
    uint32_t log2_chunk;
    uint64_t c_begin, c_end;
    uint32_t cpt;              // chunks per tile
    uint32_t n_tiles;
    const uint64_t *fp_old;    // baseline fingerprints (indexed by base_first + local)
    uint64_t *fp_new;          // indexed by global chunk id
    uint64_t *idx_out;         // segment-relative dirty list (global chunk ids)
    uint64_t *off_out;         // segment-relative byte offsets, k+1 entries
    uint64_t idx_cap;          // entries available in idx_out (off_out has idx_cap+1)
    uint8_t *staging;
    uint64_t staging_cap;
    uint64_t *tile_cnt;        // look-back status words, n_tiles each
    uint64_t *tile_bytes;
    CkptCtrl *ctrl;
    uint64_t timeout_ns;
    uint32_t skip_first_ticket;  // fault injection: tile 0 is never processed
    // Split pass, FULL checkpoints only (no chunk has a baseline, every size a
    // multiple of 16): the hash kernels write each chunk straight to its final
    // staging offset alloc_prefix[a] + local*S - seg_base, and the gather is
    // skipped.
    uint32_t full_copy;
    const uint64_t *alloc_prefix;   // payload bytes of all allocations before each one
    uint64_t seg_base;              // payload offset of the segment's first chunk
    // Sparse split pass (with full_copy, on delta checkpoints too): chunks
    // are written at their uncompacted offsets (on a delta with chunks of
    // 512 B - 4 KiB only the dirty ones, which the hash kernel holds in
    // registers until their fingerprint is known; larger chunks all), each
    // dirty entry's offset points there, ctrl->D counts the segment's bytes
    // and ctrl->payload the dirty ones; nothing is gathered.
    uint32_t sparse;
    // TMA pass: the allocations' first_chunk column fits in the CTA's shared
    // memory (n_allocs <= ckpt_tma_cached_allocs()) and is searched there.
    uint32_t first_cached;
    // Split pass, predicted write-through: ppos[c - c_begin] is the staging
    // offset chunk c had in the previous pass's compacted payload (~0 if it
    // was not dirty then).  The hash kernels write such a chunk there as they
    // read it, and the gather leaves an entry alone when its offset is the
    // predicted one (the bytes are already in place); any other entry is
    // copied as usual, after the speculative writes, so the result never
    // depends on the prediction.  The gather records this pass's offsets in
    // ppos_next (pre-set to ~0) when at most half of the chunks are dirty.
    const uint64_t *ppos;
    uint64_t *ppos_next;
    // Coded contexts, split pass on chunks of 8 KiB and more: the CRZ1 header
    // word of every 512-byte block of every chunk written to staging, at
    // (c << (log2_chunk - 9)) + block, written by whichever kernel writes the
    // chunk (hash: FULL or predicted; gather: the rest) from the vectors it
    // holds (laid out across the warp as the encoder lays out a block), so
    // that the encoder does not compute them again.
    uint64_t *crz_hdr;
};

// Restore: one image allocation mapped onto the target layout.
struct ScatterDesc {
    uint64_t img_first;     // first chunk of this allocation in the image layout
    uint64_t bytes;
    uint64_t tgt_first;     // its first chunk in the target layout (owner map index)
    uint64_t dst;           // current device address of the target allocation; 0 = dropped
    uint64_t payload_base;  // FULL images: byte offset of its first chunk in the payload
    uint64_t pad[3];
};

struct ScatterParams {
    const ScatterDesc *desc;
    uint32_t n_desc;
    uint32_t log2_chunk;
    uint32_t full;            // 1: entries are image chunk ids j0..j1 with implicit offsets
    uint32_t image_index;     // position in the chain; only chunks owned by it are written
    uint64_t j0, j1;          // entry range
    const uint64_t *idx;      // list mode: image chunk id of entry j (indexed j - j0)
    const uint64_t *off;      // list mode: payload offset of entry j (indexed j - j0)
    const uint8_t *payload;   // device address of payload byte `origin`
    uint64_t origin;
    uint64_t window;          // bytes valid from `payload`
    const uint16_t *owner;    // chain position owning each target chunk
    uint64_t n_owner;
    unsigned int *err;
};

// Per-allocation (baseline) path: running totals carried between launches.
struct PerAllocCarry {
    unsigned long long k, D;
    unsigned long long unit_k0, unit_k;   // dirty-list range of the current unit
    unsigned long long pad[4];
};

// ---- launchers (return cudaGetLastError() of the launch) ----------------
cudaError_t launch_ckpt_fused(const CkptParams &p, int threads, int warps_per_chunk, int grid,
                              cudaStream_t s);
// Kernel entry of the fused pass for a (threads, warps_per_chunk) variant, for
// building a graph kernel node; nullptr if the variant does not exist.
const void *ckpt_fused_fn(int threads, int warps_per_chunk);
int ckpt_fused_max_ctas_per_sm(int threads, int warps_per_chunk);


// TMA-staged variant of the fused pass (chunk sizes 1-64 KiB): one CTA per
// SM, ckpt_tma_threads() threads, ckpt_tma_smem() bytes of dynamic shared
// memory, a tile of ckpt_tma_slot_bytes() / chunk_bytes chunks, and
// warps_per_chunk = max(1, 8 * chunk_bytes / slot_bytes).
const void *ckpt_tma_fn(int warps_per_chunk);
int ckpt_tma_threads();
size_t ckpt_tma_smem(uint32_t n_allocs);   // dynamic shared memory of a launch over n_allocs
uint32_t ckpt_tma_cached_allocs();
uint32_t ckpt_tma_slot_bytes();
cudaError_t ckpt_tma_prepare();   // raise the dynamic shared memory limit (once per device)

// Split pass: three kernels with the signature (CkptParams, u64 *acc, u32 log2Seg),
// run in order H -> F -> G.  acc holds one u64 per chunk of the segment and
// must be zero before H; F uses cpt = split_finalize_threads() chunks per
// tile and the look-back status words; G reads k from ctrl.
const void *split_hash_fn(bool crz_headers = false);
// Hash kernel for 512 B <= chunk < 8 KiB: lanes_per_chunk = 32 * chunk / 8192;
// it finalizes every chunk itself, so finalize runs with log2Seg = log2_chunk.
const void *split_hash_small_fn(int lanes_per_chunk);
const void *split_finalize_fn();
const void *split_gather_fn(bool crz_headers);
int split_hash_threads();
int split_finalize_threads();
int split_gather_threads();
int split_max_ctas_per_sm(const void *fn, int threads);

cudaError_t launch_fp_range(const CkptDesc *d, uint64_t c0, uint64_t c1, uint32_t log2_chunk,
                            const uint64_t *fp_old, uint64_t *fp_new, uint32_t *lens,
                            uint64_t lens_base, int grid, cudaStream_t s);
cudaError_t launch_compact_range(const uint32_t *lens, uint64_t lens_base, uint64_t c0,
                                 uint64_t c1, uint64_t *idx_out, uint64_t *off_out,
                                 uint64_t idx_cap, PerAllocCarry *carry, CkptCtrl *ctrl,
                                 cudaStream_t s);
cudaError_t launch_gather_range(const CkptDesc *d, uint32_t log2_chunk, const uint64_t *idx,
                                const uint64_t *off, PerAllocCarry *carry, uint64_t max_entries,
                                uint64_t idx_cap, uint8_t *staging, uint64_t staging_cap,
                                CkptCtrl *ctrl, int grid, cudaStream_t s);

cudaError_t launch_scatter(const ScatterParams &p, int grid, cudaStream_t s);

// Side-stream drain of a delta pass into host images, sized on the device
// from the pass's control block (crac_drain.cu); prepare_drain loads it.
cudaError_t prepare_drain();
// n 8-byte words at `words` (device), then the 4-byte word32 (device, or
// null) zero-extended, to dst (pinned host memory, through its device
// mapping), by a one-warp kernel on s rather than by a copy engine.
cudaError_t launch_report(const void *words, uint32_t n, const uint32_t *word32, void *dst, cudaStream_t s);
const void *report_fn();   // the kernel, for graph nodes: args (words, n, word32, dst)
cudaError_t launch_drain(const CkptCtrl *ctrl, const uint8_t *src, uint8_t *dst, uint64_t cap,
                         const uint64_t *idx_src, uint64_t *idx_dst, uint64_t idx_cap, int grid, cudaStream_t s);
// One piece of a device-resident image in a multi-image restore: its chunk
// list, offsets and payload, where its entries start in the combined entry
// space, its image's position in the chain and its descriptor range.
struct RestorePiece {
    uint64_t idx, off, payload;   // device addresses
    uint64_t k;                   // entries
    uint64_t entry_base;          // first entry in the combined space
    uint64_t bytes;               // payload bytes (window)
    uint32_t image_index;         // chain position (oldest = 0)
    uint32_t desc_off, n_desc, pad;
    uint64_t zlen;                // coded image: device address of each entry's
                                  // stream length (0: entries are raw chunks)
};
struct RestoreParams {
    const RestorePiece *pieces;
    uint32_t n_pieces;
    uint32_t log2_chunk;
    uint64_t n_entries;
    const ScatterDesc *desc;      // all images' descriptors, RestorePiece::desc_off into it
    uint32_t *owner;              // per target chunk: newest chain position + 1 (0 = none)
    uint64_t n_owner;
    unsigned int *err;
    // Incremental restore: current and target fingerprints per target chunk.
    const uint64_t *fp_now, *fp_img;
    uint32_t coded;               // some piece has a zlen table (coded image)
};
// Multi-image restore: mark owners for every entry of every piece (atomicMax,
// so the newest image wins in any order), check coverage, scatter owned chunks.
cudaError_t launch_restore_mark(const RestoreParams &p, int grid, cudaStream_t s);
cudaError_t launch_restore_check(const RestoreParams &p, int grid, cudaStream_t s);
cudaError_t launch_restore_scatter(const RestoreParams &p, int grid, cudaStream_t s);
// Incremental restore, between check and scatter: clears the owner of every
// chunk whose current fingerprint equals the target's, so it is not written.
cudaError_t launch_restore_unmark(const RestoreParams &p, int grid, cudaStream_t s);

// CRZ1 encoder (crac_codec.cu): the raw payload of one segment, as the pass
// left it in device staging, -> one stream per entry (coded, or the chunk
// itself when coding does not shrink it), each at a 16-byte multiple.
// Persistent CTAs take tiles of tile_entries consecutive entries from a
// ticket, compute every block's header word, find the tile's output offset
// by a decoupled look-back over earlier tiles, then write the streams.
struct CodecParams {
    const uint8_t *src;       // raw payload: entry e at off[e], off[e+1] - off[e] bytes
    const uint64_t *off;      // k + 1 offsets
    uint64_t k;
    uint8_t *dst;             // streams (device memory or mapped pinned memory), 16-byte aligned
    uint64_t dst_cap;
    uint64_t *zoff;           // out: k + 1 stream offsets (prefix of 16-byte padded lengths)
    uint64_t *zlen;           // out: k stream lengths
    uint64_t *hdr;            // scratch: block header words, entry e's from off[e] / 512
    uint64_t *status;         // scratch: one look-back word per tile, zeroed
    uint32_t *ticket;         // scratch: tile counter of this launch, zeroed
    unsigned int *err;        // kErr* bits, zeroed
    uint32_t tile_entries;    // entries per tile, 1..crz_tile_max()
    // This launch encodes tiles [tile_begin, n_tiles); an earlier launch on the
    // same stream has encoded the tiles before (their look-back words are
    // final).  The last tile writes zoff[its last entry + 1].
    uint32_t tile_begin;
    uint32_t n_tiles;
    uint64_t timeout_ns;
    uint32_t skip_first_ticket;   // fault injection: tile 0 is never processed
    // Block header words made by the pass (CkptParams::crz_hdr), or null:
    // entry e's block b has chdr[(idx[e] << log2_bpc) + b].
    const uint64_t *chdr;
    const uint64_t *idx;          // the entries' global chunk ids
    uint32_t log2_bpc;            // log2 of 512-byte blocks per chunk
    // With chdr, the streams are sized and placed first (crz_size_kernel:
    // zlen, zoff; piece_off[i] = zoff[k * i / pieces], i = 0 .. pieces), then
    // coded by crz_encode_sized_kernel over entries [e_begin, e_end), each
    // entry as segs_per_entry work items of 64 KiB.
    uint64_t *piece_off;
    uint32_t pieces;
    uint32_t segs_per_entry;
    uint64_t e_begin, e_end;
};
cudaError_t launch_crz_encode(const CodecParams &p, int grid, cudaStream_t s);
cudaError_t launch_crz_size(const CodecParams &p, int grid, cudaStream_t s);
cudaError_t launch_crz_encode_sized(const CodecParams &p, int grid, cudaStream_t s);
int crz_sized_max_ctas_per_sm();
uint32_t crz_sized_segs(uint32_t log2S);   // work items per entry of the sized encoder
uint32_t crz_tile_max();
int crz_encode_max_ctas_per_sm();

void count_launches(uint64_t n);
uint64_t launches_so_far();
// Record a CUDA error for crac_last_cuda_error() (calling thread).
void note_cuda_error(int e);

}  // namespace crac
