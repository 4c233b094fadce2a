/*
 * crac.h -- C ABI of libcrac: the device data pass of CRAC-style transparent
 * CUDA checkpoint-restart on one GPU (sm_103a).
 *
 * The paper ("CRAC: Checkpoint-Restart Architecture for CUDA with Streams and
 * UVM") interposes on the cudaMalloc family, logs the pointers of the
 * buffers it creates, and at checkpoint time saves only the memory of the
 * *active* allocations -- allocated and not yet freed -- copying it back at
 * restart (Sec. 3.2, "Issue of library-allocated memory", "Saving the
 * library-allocated arena", "restoring the CUDA library-allocated regions").
 * Device (cudaMalloc) and unified-memory (cudaMallocManaged) regions are both
 * saved (same subsection; UVM support, Sec. 1 and 2).  Before copying, the
 * device's queue of pending work is drained (Sec. 2.2, step (a) of the
 * CheCUDA scheme that CRAC keeps).
 *
 * This library is that data pass, re-designed for one GB300:
 *   - crac_register_alloc / crac_free are the interposition points: the
 *     caller reports each cudaMalloc-family allocation and each free.
 *   - crac_checkpoint turns every registered allocation into an image.  Each
 *     allocation is cut into fixed-size chunks; every chunk gets a 64-bit
 *     content fingerprint; chunks whose fingerprint differs from the previous
 *     checkpoint's are compacted into a contiguous device staging buffer and
 *     drained to pinned host memory on a side stream.  The incremental
 *     (fingerprint/delta) design is this library's, not the paper's: the
 *     paper copies every active allocation at every checkpoint.
 *   - crac_restart writes an image (and, for a delta, its chain of parents)
 *     back into the registered allocations.
 *
 * All functions return crac_status_t: 0 on success, a negative CRAC_ERR_*
 * code on failure.  No function aborts the process or traps on the device;
 * on a CUDA failure the call returns CRAC_ERR_CUDA and crac_last_cuda_error()
 * gives the cudaError_t value.  A failed checkpoint leaves the previous image
 * and the fingerprint baseline untouched.
 *
 * Threads: each context has one mutex; calls on different contexts may run
 * concurrently.  Streams are CUDA runtime streams (cudaStream_t); pass them
 * as crac_stream_t.  A NULL stream means "drain the whole device first"
 * (cudaDeviceSynchronize), as the paper does before it copies.
 */
#ifndef CRAC_H
#define CRAC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define CRAC_API __attribute__((visibility("default")))
#else
#define CRAC_API
#endif

/* Same object as cudaStream_t; declared here so callers need no CUDA header. */
typedef struct CUstream_st *crac_stream_t;

typedef int crac_status_t;
#define CRAC_OK                   0
#define CRAC_ERR_INVALID_ARG     -1  /* bad size, pointer, alignment or config */
#define CRAC_ERR_UNKNOWN_PTR     -2  /* crac_free of a pointer never registered */
#define CRAC_ERR_OVERLAP         -3  /* range overlaps a registered allocation */
#define CRAC_ERR_CUDA            -4  /* a CUDA call failed; see crac_last_cuda_error */
#define CRAC_ERR_OOM             -5  /* device or pinned host memory exhausted */
#define CRAC_ERR_IMAGE_MISMATCH  -6  /* image does not fit the registry / chain */
#define CRAC_ERR_TIMEOUT         -7  /* a bounded device or host wait ran out */
#define CRAC_ERR_BUSY            -8  /* resource in use (e.g. image still draining) */
#define CRAC_ERR_UNSUPPORTED     -9  /* not supported in this build/config */
#define CRAC_ERR_CORRUPT        -10  /* serialized image malformed or truncated */

typedef enum {
    CRAC_KIND_DEVICE = 0,   /* cudaMalloc */
    CRAC_KIND_MANAGED = 1,  /* cudaMallocManaged; prefetched to the device before the pass */
    CRAC_KIND_HOST = 2      /* page-locked host memory (cudaMallocHost / cudaHostAlloc), which
                               the paper also tracks (Sec. 3.2); the pass and the restore
                               read and write it in place through its device mapping, at
                               the host link's rate (needs unified addressing, else a
                               checkpoint returns CRAC_ERR_UNSUPPORTED) */
} crac_kind_t;

/* Where a checkpoint image keeps its payload. */
#define CRAC_RESIDENCY_HOST    0  /* drained to pinned host memory (default) */
#define CRAC_RESIDENCY_DEVICE  1  /* kept in device memory (fast in-HBM rollback) */

/* How the checkpoint device pass is launched. */
#define CRAC_LAUNCH_BATCHED    0  /* one persistent graph-launched kernel over all allocations */
#define CRAC_LAUNCH_PER_ALLOC  1  /* fingerprint + compact + gather launched per allocation */

typedef struct crac_ctx crac_ctx_t;      /* one simulated process context */
typedef struct crac_image crac_image_t;  /* library-owned, reference counted */

/*
 * Context configuration.  Call crac_config_default() first, then override.
 * chunk_bytes:     power of two in [16, 2^24]; 0 means 65536.
 * staging_bytes:   device staging capacity for one segment of the pass; the
 *                  tracked bytes are processed in segments of at most this
 *                  many bytes.  0 means min(tracked bytes, 8 GiB), at least
 *                  one chunk.
 * lineage:         identifier written into every image of this context (and
 *                  used to find a deserialized delta's parent); 0 = assign a
 *                  process-unique value.
 * image_residency: CRAC_RESIDENCY_HOST or CRAC_RESIDENCY_DEVICE.
 * launch_mode:     CRAC_LAUNCH_BATCHED or CRAC_LAUNCH_PER_ALLOC.
 * threads, chunks_per_tile, ctas_per_sm, warps_per_chunk: work split of the
 *                  batched kernel; 0 = automatic.  threads is 256;
 *                  warps_per_chunk is 1 or 8.
 * timeout_ns:      limit on every device-side spin-wait; 0 = 2 s.
 * reserve_host_bytes, reserve_device_bytes: image memory (pinned host,
 *                  device) reserved by crac_ctx_create (which then needs the
 *                  GPU; a context without a reservation touches it only at
 *                  its first checkpoint or restart), so that no checkpoint
 *                  allocates from CUDA.  The arenas are process-wide and
 *                  only grow.
 */
typedef struct crac_config {
    uint32_t struct_size;
    uint32_t chunk_bytes;
    uint64_t staging_bytes;
    uint64_t lineage;
    uint32_t image_residency;
    uint32_t launch_mode;
    uint32_t threads;
    uint32_t chunks_per_tile;
    uint32_t ctas_per_sm;
    uint32_t warps_per_chunk;
    uint64_t timeout_ns;
    int32_t device;          /* CUDA device ordinal; -1 = current device */
    uint32_t pad0;
    uint64_t reserve_host_bytes;    /* pinned image memory to reserve up front */
    uint64_t reserve_device_bytes;  /* device image memory to reserve up front */
    uint32_t pass_kernel;           /* CRAC_PASS_* */
    uint32_t flags;                 /* CRAC_FLAG_* */
} crac_config_t;

/* crac_config_t.flags.
 * CRAC_FLAG_STAGED_RESTORE: restore host-resident images by copying each
 *   image's whole payload into device staging (copy engine) and scattering
 *   from there, window by window.  By default the restore kernels read a host
 *   image's chunks in place from its pinned memory (mapped into the device's
 *   address space), so only the chunks that survive into the restored state
 *   cross the host link and no staging is needed; the staged path is used
 *   anyway when the device has no unified addressing. */
#define CRAC_FLAG_STAGED_RESTORE 1u
/* CRAC_FLAG_INCREMENTAL_RESTORE: before a restart writes anything, the
 *   current contents of the registered allocations are fingerprinted and
 *   compared with the target image's fingerprint table; only the chunks that
 *   differ are restored (the others already hold the image's bytes, up to a
 *   CRAC-FP64 collision, the same trust as an incremental checkpoint).  A
 *   rollback to a recent image then costs one read of the tracked bytes plus
 *   the changed chunks.  Not on the staged path, which restores everything. */
#define CRAC_FLAG_INCREMENTAL_RESTORE 2u
/* CRAC_FLAG_DIRECT_DRAIN: a checkpoint into host-resident images writes the
 *   dirty chunks straight into the image's pinned memory through its device
 *   mapping, instead of into device staging followed by a device-to-host
 *   copy on the side stream: no staging round trip (2 x dirty bytes of HBM
 *   traffic, and no staging buffer), but the pass itself then runs at the
 *   host link's rate, on the caller's stream.  Not for the TMA pass (which
 *   keeps the staged drain). */
#define CRAC_FLAG_DIRECT_DRAIN 4u
/* CRAC_FLAG_COMPRESS: images store each chunk as its CRZ1 stream, a
 *   lossless byte-plane code of this library (the paper measures with
 *   DMTCP's gzip compression turned off, Sec. 4.4.1, and has none).  A chunk
 *   is cut into 512-byte blocks of 128 u32 words; every byte is rotated left
 *   by one bit (a float's sign moves to the bottom), byte p of the words forms
 *   plane p, and each plane is stored as its minimum and the offsets from it
 *   in as many bits as their range needs; a chunk that this would not shrink
 *   is stored as it is.  Floating-point data with few distinct exponents and
 *   zero-filled memory shrink (fp32 N(0,1): 0.89, bf16: 0.76, zeros:
 *   0.016); uniformly random bytes are stored as they are.  The pass gathers
 *   into device staging as usual and an encoder kernel writes the streams --
 *   into the device image, the staging drain, or, with
 *   CRAC_FLAG_DIRECT_DRAIN, straight into the image's pinned memory -- so
 *   only the coded bytes cross the host link.  Restores decode in the scatter
 *   kernel, reading host images in place; a context that has to stage its
 *   host restores (no unified addressing) cannot restore coded images
 *   (CRAC_ERR_UNSUPPORTED).  Images carry CRAC_IMAGE_CODED.  Not with
 *   CRAC_PASS_SPARSE, whose payload is not compacted (rejected at creation;
 *   the autotuner never picks it for a coded context).  Under the request
 *   server a coded context's lease is at least one chunk plus 256 bytes. */
#define CRAC_FLAG_COMPRESS 8u
/* CRAC_FLAG_WAIT_PASS: every checkpoint call waits for its pass, so the
 *   image's dirty count and payload size are known when it returns and its
 *   blocks are sized to them (no worst-case blocks while it runs); the
 *   single-segment passes that otherwise return once enqueued behave like
 *   the others.  A pass failure is then reported by the call. */
#define CRAC_FLAG_WAIT_PASS 16u

/* Kernel of the batched pass (crac_config_t.pass_kernel). */
#define CRAC_PASS_AUTO  0  /* the split pass, or, when the last pass with a baseline
                              found more than half of the chunks dirty, the first of
                              SPARSE (device images, 16-byte sizes), TMA (1-64 KiB
                              chunks), LDG that applies, or SPARSE (dense placement)
                              when it found under a quarter dirty on 512 B - 4 KiB
                              chunks of device images with 16-byte sizes; trial
                              passes of the tuner use the split pass */
#define CRAC_PASS_LDG   1  /* one fused persistent kernel, 128-bit loads to registers;
                              the gather re-reads dirty chunks from L2 */
#define CRAC_PASS_TMA   2  /* one fused kernel, bulk copies into a shared-memory ring,
                              warp-specialized; chunk sizes 1 KiB..64 KiB only */
#define CRAC_PASS_SPLIT 3  /* three kernels in one graph: streaming hash, finalize +
                              compaction, gather */
#define CRAC_PASS_SPARSE 4 /* the split pass without compaction: the hash kernel writes
                              every chunk (on 512 B - 4 KiB chunks only the dirty
                              ones) to its uncompacted offset in the image's payload
                              buffer and the dirty list points into it, so no byte is
                              read twice (B read + B, or D, written, against B + 2D).
                              Pays off when most chunks are dirty.  Device-resident
                              images only; an image then holds the tracked bytes of
                              its segments instead of the dirty ones (serialization
                              still writes the compact payload), except on 512 B -
                              4 KiB chunks after a delta that found under a quarter
                              of the chunks dirty: the dirty chunks are then placed
                              back to back and the image holds only them.  Falls back to the
                              split pass when an allocation size is not a multiple of
                              16 bytes. */

/* Summary of an image (crac_image_info). */
typedef struct crac_image_info {
    uint64_t lineage;
    uint64_t epoch;          /* 1 for a context's first checkpoint, then increasing */
    uint64_t parent_epoch;   /* UINT64_MAX if none */
    uint32_t flags;          /* bit 0 CRAC_IMAGE_FULL: every chunk is present */
    uint32_t chunk_bytes;
    uint64_t n_allocs;
    uint64_t n_chunks;
    uint64_t k;              /* chunks present in this image */
    uint64_t payload_bytes;
    uint64_t serialized_bytes;
    uint32_t residency;
    uint32_t complete;       /* 1 once the drain has finished */
    uint64_t raw_bytes;      /* bytes of the chunks present before coding (payload_bytes,
                                the stored bytes, for an uncoded image) */
    float drain_ms;          /* host image, once complete: device time on the context's side
                                stream from the start of its drain (the pass's end, or the
                                first copy of a coded image's streams) to its completion;
                                else 0 */
    uint32_t reserved;
} crac_image_info_t;
#define CRAC_IMAGE_FULL 1u
#define CRAC_IMAGE_CODED 2u  /* chunks are stored as CRZ1 streams (CRAC_FLAG_COMPRESS) */

/* Measurements of a context's most recent checkpoint (crac_ctx_last_pass). */
typedef struct crac_pass_info {
    uint64_t tracked_bytes;  /* sum of registered allocation sizes */
    uint64_t n_chunks;
    uint64_t k;              /* dirty chunks */
    uint64_t payload_bytes;  /* dirty bytes */
    uint32_t segments;
    uint32_t kernel_launches;
    float device_ms;         /* device time of the pass launches (CUDA events) */
    float prefetch_ms;       /* device time of managed-memory prefetch */
    uint32_t grid;           /* CTAs of the batched kernel */
    uint32_t chunks_per_tile;
    uint32_t warps_per_chunk;
    float hash_ms;           /* split pass: device time of each of its kernels */
    float finalize_ms;
    float gather_ms;
    uint32_t pass_kernel;    /* CRAC_PASS_* that ran */
    float codec_ms;          /* CRAC_FLAG_COMPRESS: device time of the encoder launches */
    uint64_t stored_bytes;   /* payload bytes of the image (coded: its streams) */
    uint64_t in_place;       /* split pass: dirty chunks the hash kernel had already written to
                                staging as it read them (the previous pass's dirty chunks, at
                                the offsets that pass gave them), which the gather left alone */
} crac_pass_info_t;

/* ---- configuration and contexts --------------------------------------- */

CRAC_API void crac_config_default(crac_config_t *cfg);

/* Create a context.  cfg may be NULL (defaults).  *out receives the handle. */
CRAC_API crac_status_t crac_ctx_create(const crac_config_t *cfg, crac_ctx_t **out);

/* Destroy a context after waiting for its device work.  Images it produced
 * stay valid until released. */
CRAC_API crac_status_t crac_ctx_destroy(crac_ctx_t *ctx);

/*
 * Report an active allocation (the paper logs the pointers returned by the
 * cudaMalloc family, Sec. 3.2).  ptr is a device or managed pointer, 16-byte
 * aligned (every cudaMalloc-family pointer is 256-byte aligned); bytes >= 1.
 * The library never frees or owns it.  Errors: CRAC_ERR_INVALID_ARG (NULL or
 * misaligned ptr, bytes == 0, bad kind), CRAC_ERR_OVERLAP (intersects a
 * registered range -- the overlap hazard of Sec. 3.2, "Issue of memory
 * overlapping").  Allocations are kept in registration order, which is the
 * order of their chunks in every image.
 */
CRAC_API crac_status_t crac_ctx_register_alloc(crac_ctx_t *ctx, void *ptr, size_t bytes,
                                               crac_kind_t kind);

/* Drop an allocation (the paper's cudaFree interposition).  The next image no
 * longer contains it.  CRAC_ERR_UNKNOWN_PTR if ptr was not registered. */
CRAC_API crac_status_t crac_ctx_free(crac_ctx_t *ctx, void *ptr);

/*
 * Checkpoint every registered allocation.
 * Ordering: the image reflects all work enqueued on `stream` before the call
 * (other streams must be joined by the caller); stream == NULL first
 * synchronizes the whole device.  Managed allocations are prefetched to the
 * device on `stream` before the pass.
 * The call returns after enqueueing (Sec. 2.2's drain of pending work
 * becomes stream order) when the pass is one batched launch into uncoded
 * images whose tracked bytes fit the staging capacity: the image's dirty
 * count and payload size are then known, and settle, once its pass has run
 * (crac_image_wait, crac_image_info, crac_image_serialize and a restart wait
 * for that).  Until then the image holds worst-case blocks (the tracked
 * bytes, from the device arena or the pinned regions as they are).  Up to
 * two such checkpoints of a context may be unsettled; a third call, and
 * every other kind of pass, first waits for the earlier ones.  The other
 * passes (several staging segments, coded images, per-allocation launches)
 * wait for each segment's dirty counts, and return once the pass has
 * finished; the drain to host memory may still be running.  A call that has
 * to grow the context's tables (more chunks than before) may synchronize
 * the device while it allocates.
 * The first checkpoint of an allocation carries all of its chunks; later
 * ones carry only chunks whose fingerprint changed.  *image_out receives a
 * new reference that the caller releases with crac_image_release.
 * A device wait that runs out gives CRAC_ERR_TIMEOUT with the baseline
 * untouched: from this call, or, for a pass it did not wait for, from the
 * image (crac_image_wait); the context's baseline then returns to its last
 * good image before its next operation, and an image taken meanwhile, whose
 * pass compared against the failed one, fails with the same error.  If a kernel reports that a bulk copy into its shared memory
 * never completed, even after it waited for it in bounded rounds, the
 * device's state is unspecified: the call returns CRAC_ERR_CUDA and the
 * context refuses every later checkpoint and restart with CRAC_ERR_CUDA.
 */
CRAC_API crac_status_t crac_ctx_checkpoint(crac_ctx_t *ctx, crac_stream_t stream,
                                           crac_image_t **image_out);

/*
 * Write `image` back into the registered allocations (Sec. 3.2: the saved
 * memory is "copied back at restart time").  For a delta image the chain of
 * parents back to the nearest image with CRAC_IMAGE_FULL is applied, each
 * chunk taken from the newest image that holds it.  The registry must match
 * the image's allocation table in count, sizes, kinds and order, and the
 * context's chunk size must equal the image's; otherwise
 * CRAC_ERR_IMAGE_MISMATCH and device memory is untouched.  Work is enqueued
 * on `stream` (NULL: device-wide sync first), after all work enqueued there
 * before the call.  The call then waits on the host until that work has
 * finished: the registry adopts the image (its fingerprints become the
 * baseline, its allocation identities the registry's) only once the
 * restore's error word says it succeeded, so a failed restore never leaves
 * a baseline that does not describe memory.  Afterwards an unmodified
 * checkpoint is empty.
 * Errors found on the device: a chunk of the target no chain image holds
 * (CRAC_ERR_IMAGE_MISMATCH; memory untouched, the scatter does not start);
 * a coded stream whose plane values pass 255, which only decoding finds
 * (CRAC_ERR_CORRUPT; the allocations' contents are then unspecified, the
 * context's baseline is unchanged).  Coded streams of deserialized images
 * are checked for impossible headers when they are deserialized.
 */
CRAC_API crac_status_t crac_ctx_restart(crac_ctx_t *ctx, const crac_image_t *image,
                                        crac_stream_t stream);

/* ---- serving: many contexts, one GPU ---------------------------------- */

/*
 * A request server for many process contexts sharing one GPU.  Requests
 * (checkpoint or restart of a context) are queued in arrival order; a
 * request is admitted when a worker slot is free, no earlier request of the
 * same context is still running, and its staging lease fits in the staging
 * budget (best-fit in one device region; an earlier request that does not
 * fit blocks later ones, so none starves).  Admitted requests run at once on
 * their own streams, so the passes of different contexts overlap on the
 * device, and requests arriving meanwhile join as slots and staging free up.
 * Fingerprint baselines stay in each context's device memory between
 * requests.  Each result is the same as if the request had run alone.
 */
typedef struct crac_server crac_server_t;

typedef struct crac_server_config {
    uint32_t struct_size;
    uint32_t workers;          /* requests in flight at once; 0 = 4 */
    uint64_t staging_budget;   /* device bytes shared by in-flight requests; 0 = 24 GiB */
    uint64_t max_lease;        /* staging leased by one request (its segment size); 0 = 4 GiB */
    int32_t device;            /* -1 = current device */
    uint32_t reserved[5];
} crac_server_config_t;

#define CRAC_REQ_CHECKPOINT 0
#define CRAC_REQ_RESTART    1

/* Called on the worker thread right before a request's operation, with the
 * request's stream: the application's own work to order before it. */
typedef void (*crac_prepare_fn)(crac_stream_t stream, void *arg);

typedef struct crac_request_result {
    uint64_t ticket;
    int32_t status;              /* CRAC_OK or the operation's error */
    uint32_t type;
    crac_image_t *image;         /* checkpoint: the new image (caller releases) */
    double t_arrival, t_admit, t_done;   /* crac_time_now() clock, seconds */
    uint64_t tracked_bytes;      /* the context's registered bytes */
    uint64_t payload_bytes;      /* checkpoint: dirty bytes; restart: image payload */
    uint64_t lease_bytes;        /* staging leased while it ran */
    /* Where the service time (t_admit .. t_done) went: t_op is when the
     * operation was called (after the prepare callback), t_op_end when the
     * call returned; from there to t_done a checkpoint waits for its image to
     * settle (pass and drain finished). */
    double t_op, t_op_end;
} crac_request_result_t;

typedef struct crac_server_stats {
    uint64_t submitted, completed;
    uint32_t queued, in_flight, max_in_flight, pad;
    uint64_t staging_used, staging_high_water, staging_budget;
} crac_server_stats_t;

CRAC_API double crac_time_now(void);
CRAC_API crac_status_t crac_server_create(const crac_server_config_t *cfg, crac_server_t **out);
/* Waits for queued and running requests, then frees the server.  Results not
 * yet collected are dropped (their images released). */
CRAC_API crac_status_t crac_server_destroy(crac_server_t *server);
/* Queue a request.  image: the image to restore (restart only; the server
 * holds a reference until the request completes).  t_arrival: the request's scheduled
 * arrival on the crac_time_now() clock (latency is measured from it); <= 0
 * means now.  *ticket identifies the result. */
CRAC_API crac_status_t crac_server_submit(crac_server_t *server, crac_ctx_t *ctx, uint32_t type,
                                          const crac_image_t *image, crac_stream_t stream,
                                          crac_prepare_fn prepare, void *prepare_arg, double t_arrival,
                                          uint64_t *ticket);
/* Wait (at most timeout_ns; 0 = no limit) for a request and take its result. */
CRAC_API crac_status_t crac_server_wait(crac_server_t *server, uint64_t ticket, uint64_t timeout_ns,
                                        crac_request_result_t *out);
CRAC_API crac_status_t crac_server_stats(crac_server_t *server, crac_server_stats_t *out);

/* ---- autotuning (chunk size and pass kernel) ------------------------- */

#define CRAC_TUNE_MAX 8
typedef struct crac_tune_result {
    uint32_t n;                            /* candidate chunk sizes */
    uint32_t rounds;                       /* delta observations per candidate */
    uint32_t chosen_chunk_bytes;           /* set by crac_ctx_tune_apply */
    uint32_t chosen_pass_kernel;
    uint32_t chunk_bytes[CRAC_TUNE_MAX];
    float last_pass_ms[CRAC_TUNE_MAX];     /* most recent observation (device time) */
    uint64_t last_dirty_bytes[CRAC_TUNE_MAX];
    float mean_pass_ms[CRAC_TUNE_MAX];     /* over the delta observations */
    double mean_dirty_bytes[CRAC_TUNE_MAX];
    float cost_ms[CRAC_TUNE_MAX];          /* pass + drain estimate (apply) */
    float variant_ms[8];                   /* pass time per CRAC_PASS_* at the chosen
                                              size (apply); 0 = not applicable or
                                              not timed */
    uint32_t chosen_chunks_per_tile;       /* LDG tile kept by apply (0 = not tuned:
                                              fixed in the config, or LDG not chosen) */
    uint32_t ldg_tiles[3];                 /* LDG tiles (chunks) timed by apply; 0 = unused */
    float ldg_tile_ms[3];                  /* pass time of each of those tiles */
    uint32_t pad0;
} crac_tune_result_t;

/*
 * One observation round of the autotuner, taken between two steps of the
 * application (typically right before a checkpoint).  For every candidate
 * chunk size (chunk_sizes[0..n), n <= CRAC_TUNE_MAX, each a valid chunk size)
 * the library keeps a private fingerprint baseline of the registered memory;
 * each round runs the real checkpoint pass for that size against its own
 * baseline, on `stream`, without producing an image and without touching the
 * context's own baseline, and records the device time and dirty bytes.  The
 * first round only establishes the baselines.  A different list of sizes
 * restarts the session.  *out (may be NULL) receives the statistics.
 */
CRAC_API crac_status_t crac_ctx_tune_observe(crac_ctx_t *ctx, crac_stream_t stream, const uint32_t *chunk_sizes,
                                             uint32_t n, crac_tune_result_t *out);

/*
 * End the session.  Each candidate chunk size has a mean cost from the
 * observations (pass time + dirty bytes / link_gbs; link_gbs <= 0 counts the
 * device pass only).  At every size whose cost is within 5% of the lowest,
 * each pass kernel is timed on the last observation's dirty set, and the
 * size and kernel with the lowest pass + drain time are kept.  When the
 * configuration leaves chunks_per_tile at 0, the LDG kernel is timed at three
 * tile sizes (half, equal to and twice its default) and, if LDG wins, the
 * fastest tile is written to the context's chunks_per_tile.  If the chunk size changes, the context's baseline is
 * dropped, so its next checkpoint is FULL (which also ends the delta chain,
 * since a chain holds one chunk size).  Needs at least two observe rounds
 * (CRAC_ERR_UNSUPPORTED otherwise).
 */
CRAC_API crac_status_t crac_ctx_tune_apply(crac_ctx_t *ctx, crac_stream_t stream, double link_gbs,
                                           crac_tune_result_t *out);

/* Forget the fingerprint baseline: the next checkpoint carries every chunk
 * (a FULL image, which cuts the delta chain). */
CRAC_API crac_status_t crac_ctx_invalidate(crac_ctx_t *ctx);

/* Let go of the context's own reference to its newest image (a checkpoint's
 * image, or the image a restart restored), keeping the fingerprint baseline:
 * the next checkpoint is still a delta against the state that image holds,
 * but it no longer keeps that image alive.  Such a delta finds its parent by
 * (lineage, parent_epoch) among loaded images when it is restored, as a
 * deserialized delta does, so its chain restores only while the parent (or a
 * deserialized copy of it) is loaded.  For callers that write each image out
 * (crac_image_read, crac_image_serialize) and release it, so that memory
 * holds only the newest image -- the paper's images are files on disk
 * (Sec. 3.2), not kept in memory. */
CRAC_API crac_status_t crac_ctx_drop_history(crac_ctx_t *ctx);

/* Measurements of the context's most recent checkpoint pass. */
CRAC_API crac_status_t crac_ctx_last_pass(crac_ctx_t *ctx, crac_pass_info_t *out);

/* Measurements of a context's most recent restart (crac_ctx_last_restart). */
typedef struct crac_restart_info {
    uint32_t chain_length;       /* images from the nearest FULL one to the target */
    uint32_t images_used;        /* images that still owned at least one chunk */
    uint64_t restored_bytes;     /* bytes written into allocations (= tracked bytes,
                                    or the differing chunks' bytes when incremental) */
    uint64_t entries_scanned;    /* chunk entries the scatter kernels visited */
    uint64_t h2d_bytes;          /* host image payload copied to the device (staged
                                    restore; a mapped restore reads in place) */
    uint32_t scatter_launches;
    float device_ms;             /* device time from the first copy/launch to the last */
    uint64_t chunks_rewritten;   /* chunks written into allocations (incremental restore:
                                    those that differed from the image; else all) */
    uint32_t reserved[2];
} crac_restart_info_t;

CRAC_API crac_status_t crac_ctx_last_restart(crac_ctx_t *ctx, crac_restart_info_t *out);

/* ---- default-context forms (one implicit context per process) -------- */

CRAC_API crac_status_t crac_register_alloc(void *ptr, size_t bytes, crac_kind_t kind);
CRAC_API crac_status_t crac_free(void *ptr);
CRAC_API crac_status_t crac_checkpoint(crac_stream_t stream, crac_image_t **image_out);
CRAC_API crac_status_t crac_restart(const crac_image_t *image, crac_stream_t stream);

/* ---- images ----------------------------------------------------------- */

/* Block until the image's pass and drain have completed, at most timeout_ns
 * (0 = no limit).  CRAC_ERR_TIMEOUT if the limit passes first.  For a
 * checkpoint whose call returned before its pass finished, this is where a
 * device-side failure of the pass is reported (CRAC_ERR_TIMEOUT for a device
 * wait that ran out, CRAC_ERR_CORRUPT, CRAC_ERR_CUDA), and again on every
 * later call that needs the image. */
CRAC_API crac_status_t crac_image_wait(const crac_image_t *image, uint64_t timeout_ns);

/* The image's header fields.  For an image whose pass may still be running
 * (crac_ctx_checkpoint returned before it finished) this first waits for it,
 * since k and the payload size come from the pass. */
CRAC_API crac_status_t crac_image_info(const crac_image_t *image, crac_image_info_t *out);

/*
 * Serialize into dst (cap bytes), little-endian:
 *   header (80 B): "CRACIMG1", u32 version=1, u32 flags, u32 chunk_bytes,
 *     u32 hash_id=1, u64 lineage, u64 epoch, u64 parent_epoch, u64 n_allocs,
 *     u64 n_chunks, u64 k, u64 payload_bytes;
 *   n_allocs x {u64 id, u64 orig_ptr, u64 bytes, u32 kind, u32 0, u64 first_chunk};
 *   u64 fp[n_chunks]; u64 idx[k] (ascending); payload (chunks in idx order,
 *   the last chunk of an allocation unpadded).
 * A coded image (flags bit 1, CRAC_IMAGE_CODED) has u64 zlen[k] after idx
 * (each chunk's stream length; equal to the chunk's length when it is stored
 * as it is) and its payload is the streams in idx order, each zero-padded to
 * a multiple of 16 bytes.
 * *need receives the size.  dst == NULL: only *need is set.  cap < need:
 * CRAC_ERR_INVALID_ARG.  Waits for the image's pass and drain first (also
 * when only the size is asked for), and returns the image's error if they
 * failed.
 */
CRAC_API crac_status_t crac_image_serialize(const crac_image_t *image, void *dst, size_t cap,
                                            size_t *need);

/*
 * Copy bytes [offset, offset + n) of the serialized form (the layout above)
 * into host memory dst, without building the whole of it: a caller can write
 * an image out piece by piece (the paper's checkpoint is a file that the
 * saved regions are written into, Sec. 3.2 "Saving the library-allocated
 * arena"), or check a multi-GiB image section by section.  Reading every
 * range once gives exactly the bytes crac_image_serialize writes.  Waits for
 * the drain first.  CRAC_ERR_INVALID_ARG if the range passes the end
 * (crac_image_info's serialized_bytes) or dst is NULL with n > 0.
 */
CRAC_API crac_status_t crac_image_read(const crac_image_t *image, uint64_t offset, void *dst, size_t n);

/* Parse a serialized image into a new host-resident image (CRAC_ERR_CORRUPT if
 * malformed: sizes, chunk list, stream lengths, or a coded stream whose block
 * headers have reserved bits set, a plane width above 8, or a length that
 * does not match them).  A delta's parent is found among live images by (lineage,
 * parent_epoch) when it is restored. */
CRAC_API crac_status_t crac_image_deserialize(const void *src, size_t n, crac_image_t **out);

/* Drop a reference.  The memory is freed when the last reference goes (a
 * child delta holds a reference to its parent). */
CRAC_API crac_status_t crac_image_release(crac_image_t *image);

/* ---- diagnostics ------------------------------------------------------ */

CRAC_API const char *crac_status_str(crac_status_t s);
/* cudaError_t of the last CUDA failure seen by this thread (0 if none). */
CRAC_API int crac_last_cuda_error(void);
/* Number of kernels this library has launched in the process (graph kernel
 * nodes included). */
CRAC_API uint64_t crac_kernel_launches(void);

/* Image memory held by the library's arenas (process-wide). */
typedef struct crac_memory_stats {
    uint64_t host_region_bytes;     /* pinned host memory obtained from CUDA */
    uint64_t host_used_bytes;       /* of which carved out for live images */
    uint64_t device_region_bytes;   /* device memory obtained for device images */
    uint64_t device_used_bytes;
    uint32_t host_regions, device_regions;
    uint32_t host_grow_events;      /* cudaHostAlloc calls made on the request path after
                                       start-up reservations (background growth, which
                                       starts once the pinned arena is 80% used, is not
                                       counted) */
    uint32_t device_grow_events;
    uint32_t scratch_grow_events;   /* context scratch buffers (re)allocated from CUDA: fingerprint
                                       tables, staging, chunk lists, restart tables; a growth
                                       that replaces a buffer synchronizes the device first */
    uint32_t reserved;
} crac_memory_stats_t;

CRAC_API crac_status_t crac_memory_stats(crac_memory_stats_t *out);

/* Managed-memory helpers for callers without their own (e.g. PyTorch, which
 * does not allocate managed memory): cudaMallocManaged / cudaFree. */
CRAC_API crac_status_t crac_alloc_managed(size_t bytes, void **out);
CRAC_API crac_status_t crac_free_managed(void *ptr);

/* ---- allocation-free pass ------------------------------------------- */

/* One region for crac_pass_noalloc, stored in device memory (32 bytes). */
typedef struct crac_region {
    uint64_t ptr;          /* device or managed address, 16-byte aligned */
    uint64_t bytes;        /* >= 1 */
    uint64_t first_chunk;  /* global id of its first chunk: regions are laid out
                              back to back, first_chunk[i+1] = first_chunk[i] +
                              ceil(bytes[i] / chunk_bytes) */
    uint64_t base_first;   /* where its previous fingerprints start in fp_old,
                              or UINT64_MAX: no previous ones, every chunk dirty */
} crac_region_t;

/* Results of crac_pass_noalloc, written to device memory (24 bytes). */
typedef struct crac_pass_totals {
    uint32_t reserved;
    uint32_t err;            /* 0; bit 0: a device wait ran out; bit 1: idx_cap
                                or staging_cap was too small */
    uint64_t k;              /* dirty chunks */
    uint64_t payload_bytes;  /* dirty bytes written to staging */
} crac_pass_totals_t;

/* Tiles the scratch of crac_pass_noalloc holds.  A tile is 128 KiB of chunks
 * (at least 1 chunk, 8..256 chunks below 16 KiB chunks), so the pass takes up
 * to 4 GiB of regions for chunk sizes 512 B..128 KiB, and 32768 chunks for
 * larger chunks. */
#define CRAC_NOALLOC_MAX_TILES 32768u

/*
 * The checkpoint pass (fingerprint, dirty test, compaction, gather) over
 * caller-owned device buffers, for callers that cannot allocate memory:
 * code running where cudaMalloc is forbidden or unsafe -- inside an
 * allocator hook or interposed cudaMalloc/cudaFree wrapper (the interposition
 * point itself, where re-entering the allocator would recurse or deadlock),
 * in a signal-driven or preemption-time checkpoint that must not change the
 * device memory map, or in a process whose allocator is out of memory at the
 * moment it must save its state.  The paper has no counterpart; it is an
 * addition of this library.
 *
 * It allocates nothing: no cudaMalloc, cudaFree, pinned memory or library
 * allocation.  Its only scratch (the pass control block and the look-back
 * status words, 64 + 16 * CRAC_NOALLOC_MAX_TILES bytes) is a fixed array in
 * the library's device memory, present on every device that loads the
 * library until the process exits.  The first call on a device looks up that
 * array's address (once per device); make that first call before any stream
 * capture.  Every call shares the array: calls whose work overlaps on the GPU
 * (different streams, or different host threads, without ordering) race and
 * give wrong results.  Each call clears the part it uses before the pass.
 *
 * Works on the current device.  Inputs: regions_dev (n_regions entries,
 * device memory), n_chunks (their total chunk count), chunk_bytes (power of
 * two in [16, 2^24]), fp_old_dev (read where base_first != UINT64_MAX; may
 * be NULL, and then no region has a baseline and every chunk is dirty).
 * Outputs (device memory): fp_new_dev[n_chunks]; idx_dev[idx_cap] ascending
 * dirty chunk ids; off_dev[idx_cap + 1] their byte offsets in staging (off[k]
 * = payload bytes); staging_dev[staging_cap]; *totals_dev.  Enqueued on
 * `stream`; returns without waiting.  The result equals what
 * crac_ctx_checkpoint computes for the same regions and baseline.
 * Errors: CRAC_ERR_INVALID_ARG for NULL pointers, a bad chunk size, or a pass
 * whose tiles exceed CRAC_NOALLOC_MAX_TILES (n_chunks beyond the limit for
 * this chunk size); CRAC_ERR_CUDA if a launch fails.
 */
CRAC_API crac_status_t crac_pass_noalloc(const crac_region_t *regions_dev, uint32_t n_regions,
                                         uint64_t n_chunks, uint32_t chunk_bytes,
                                         const uint64_t *fp_old_dev, uint64_t *fp_new_dev,
                                         uint64_t *idx_dev, uint64_t *off_dev, uint64_t idx_cap,
                                         uint8_t *staging_dev, uint64_t staging_cap,
                                         crac_pass_totals_t *totals_dev, crac_stream_t stream);

/* Host-side fault injection for tests: the next `count` times the named step
 * is reached it fails as if the CUDA call there had failed (or, for
 * CRAC_FAULT_DEVICE_WAIT, the batched kernel is launched so that one tile's
 * predecessor never publishes, and its bounded wait runs out).  count 0
 * clears.  No GPU fault is raised. */
#define CRAC_FAULT_NONE         0
#define CRAC_FAULT_PASS         1  /* launch of the checkpoint pass */
#define CRAC_FAULT_DRAIN        2  /* D2H drain enqueue */
#define CRAC_FAULT_H2D          3  /* restart H2D enqueue */
#define CRAC_FAULT_ALLOC        4  /* staging / image memory allocation */
#define CRAC_FAULT_DEVICE_WAIT  5  /* look-back wait times out on the device */
#define CRAC_FAULT_ENCODE_WAIT  6  /* the CRZ1 encoder's look-back wait times out (CRAC_FLAG_COMPRESS) */
CRAC_API void crac_debug_inject_fault(int step, int count);

#ifdef __cplusplus
}
#endif
#endif /* CRAC_H */
