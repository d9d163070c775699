/*
 * me.h -- C ABI of libme, edge detection of binary images by the method of
 * masks (Sadeq, Wahdan, Mahdi, "Edge detection of binary images using the
 * method of masks", Sci. Bull. Fac. Eng. Ain Shams Univ. 35(3), 2000).
 *
 * What every call computes (Sections 3-5 of the paper, fused):
 *
 *     mask      M  = NOT I                               (Section 3)
 *     left      FL = M AND I(x-1, y)   right FR = M AND I(x+1, y)
 *     up        FU = M AND I(x, y-1)   down  FD = M AND I(x, y+1)  (Section 4)
 *     edge      E  = FL OR FR OR FU OR FD                (Section 5)
 *
 * which is the Boolean function Edge(p) = (p)' and (2 or 4 or 6 or 8) of
 * Section 1 (neighbour numbers of Fig. 1) applied to every pixel at once.
 * All results are exact: integer bitwise work, no rounding anywhere.
 *
 * Image layout (every call): packed rows of 32-bit words.  Pixel (x, y) is
 * bit x % 32 of word y * stride_words + x / 32; the least significant bit is
 * the leftmost pixel, row 0 is the top row, 0 = black and 1 = white (Section
 * 2: one bit per pixel, 0 for black, 1 for white).  nw = ceil(w / 32) words
 * of a row hold pixels; bits x >= w of word nw-1 and words nw .. stride-1
 * are padding.  Input padding is ignored (read as outside the image).  In
 * every output, the padding bits of word nw-1 and the padding words
 * nw .. stride-1 are written 0, so whole rows are written (no output sector
 * is ever partly written and read back).
 *
 * Edge polarity: an output bit of 1 marks an edge point (Edge(p) true,
 * Section 1).  Section 5 inverts the OR only to draw edges black on white;
 * me_edges_display gives that drawn form.
 *
 * Outside the image: pixels beyond the border take the boundary colour,
 * ME_BOUNDARY_WHITE (the default reading: black pixels on the border are
 * edge points) or ME_BOUNDARY_BLACK.
 *
 * Memory: "device pointer" means memory the current CUDA device can read
 * and write (cudaMalloc, torch CUDA tensors).  Buffers are owned by the
 * caller unless stated otherwise.  Calls that take a stream are
 * asynchronous on it: inputs must stay valid and outputs must not be read
 * until the stream has passed the call.  Unless stated otherwise, a call
 * allocates nothing.
 *
 * Errors: every call returns ME_OK (0), a positive progress code, or a
 * negative error code; me_status_string() names it.  A call that returns an
 * error has enqueued no work.  ME_ERR_CUDA also records the CUDA error,
 * readable once through me_last_cuda_error().
 */
#ifndef ME_H
#define ME_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* cudaStream_t without the CUDA headers; NULL is the legacy default stream. */
typedef struct CUstream_st *me_stream_t;

/* ---- status codes ------------------------------------------------------ */
#define ME_OK            0
#define ME_PENDING       1   /* serve: result not ready (poll with timeout 0) */
#define ME_TIMEOUT       2   /* serve: result not ready when the wait ran out */
#define ME_ERR_ARG      -1   /* NULL pointer, w or h <= 0, stride < ceil(w/32),
                                bad boundary, host pointer where device needed */
#define ME_ERR_ALIAS    -2   /* input and output ranges overlap */
#define ME_ERR_ALIGN    -3   /* a forced 128-bit path was given unaligned data */
#define ME_ERR_BUDGET   -4   /* serve: one request alone exceeds the budget */
#define ME_ERR_CUDA     -5   /* a CUDA call failed; see me_last_cuda_error() */
#define ME_ERR_CLOSED   -6   /* serve: the server is closed or closing */
#define ME_ERR_TICKET   -7   /* serve: unknown or already collected ticket */
#define ME_ERR_NOMEM    -8   /* host allocation failed */
#define ME_ERR_UNSUPPORTED -9 /* no sm_103a device / feature not built */
#define ME_ERR_TOO_BIG  -10  /* image larger than me_edges_staged_static holds */

#define ME_BOUNDARY_WHITE 0
#define ME_BOUNDARY_BLACK 1

/* Name of a status code ("ME_OK", "ME_ERR_ARG", ...).  Never NULL. */
const char *me_status_string(int status);

/* The CUDA error code behind the last ME_ERR_CUDA on this thread, then 0. */
int me_last_cuda_error(void);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int me_version(void);

/* ---- single image ------------------------------------------------------- */

/*
 * Fused method of masks, Sections 3-5 in one pass:
 *     edge = NOT img AND (I(x-1) OR I(x+1) OR I(y-1) OR I(y+1)).
 * Each input word is read once from HBM and each output word written once.
 *
 * img, edge     device pointers to h rows of stride_words words each; they
 *               must not overlap (ME_ERR_ALIAS).  128-bit accesses are
 *               used when both are 16-byte aligned and stride_words % 4 == 0,
 *               64-bit ones when both are 8-byte aligned and stride_words is
 *               even, 32-bit ones otherwise; all give the same bits.
 * w, h          image size in pixels, each >= 1.
 * stride_words  words per row, >= ceil(w / 32).
 * boundary      ME_BOUNDARY_WHITE or ME_BOUNDARY_BLACK.
 * stream        CUDA stream the kernel is enqueued on.
 */
int me_edges(const uint32_t *img, int32_t w, int32_t h, int32_t stride_words,
             uint32_t *edge, int32_t boundary, me_stream_t stream);

/*
 * The same result as me_edges, computed the way the paper's Section 2
 * describes its bit-block transfers: five separate whole-image passes,
 *     1. M  = NOT I                       (Section 3)
 *     2. E  = M AND I(x-1)                (Section 4, left edge)
 *     3. E |= M AND I(x+1)    4. E |= M AND I(y-1)    5. E |= M AND I(y+1)
 *                                          (Section 4 edges ORed, Section 5)
 * It moves about 17 bits of HBM traffic per pixel instead of 2 and is kept
 * as the baseline form.  Arguments as me_edges.  The mask image M is
 * scratch (h * stride_words * 4 bytes) the library takes on `stream` from a
 * stream-ordered memory pool it owns on each device and returns after pass
 * 5; the pool keeps up to 512 MiB reserved between calls, until
 * me_shutdown().  Failure to get it returns ME_ERR_CUDA with nothing
 * enqueued.
 */
int me_edges_staged(const uint32_t *img, int32_t w, int32_t h,
                    int32_t stride_words, uint32_t *edge, int32_t boundary,
                    me_stream_t stream);

/*
 * me_edges_staged without any allocation, for callers that cannot allocate
 * device memory while they run: code under a framework's caching allocator
 * that owns the whole device, real-time loops where an allocation may block
 * or fail, and processes whose device memory is capped after start-up.
 * (The paper has no counterpart; it is a deployment variant of the staged
 * form.)  The mask image lives in one fixed device array built into the
 * library, ME_STATIC_MASK_WORDS words (4 MiB), which every GPU that loads
 * the library keeps until the process exits.  Images with
 * h * stride_words > ME_STATIC_MASK_WORDS return ME_ERR_TOO_BIG with nothing
 * enqueued.  The first call on a device looks up the array's device address
 * (no allocation by the library); make that first call before any stream
 * capture.  Under CUDA's lazy module loading (the default) that first call
 * is also when the driver places the array in device memory, so a caller
 * whose device memory is capped, or handed to a caching allocator, after
 * start-up must make one call at start-up, before that happens.  The
 * address is kept for the life of the process; after a cudaDeviceReset,
 * call me_shutdown() before the next call so that it is looked up again.
 * All calls on a device share the array, so calls whose GPU work may
 * overlap (unordered streams) race and must be serialised by the caller.
 * Nothing is read from the array before the call has written it.  Other
 * arguments and results as me_edges_staged.
 */
#define ME_STATIC_MASK_WORDS 1048576
int me_edges_staged_static(const uint32_t *img, int32_t w, int32_t h,
                           int32_t stride_words, uint32_t *edge, int32_t boundary,
                           me_stream_t stream);

/*
 * The four fundamental edges of Section 4 from one read of the image:
 *     left  = M AND I(x-1, y)  (Fig. 2 b)    right = M AND I(x+1, y) (Fig. 2 a)
 *     up    = M AND I(x, y-1)  (Fig. 2 c)    down  = M AND I(x, y+1) (Fig. 2 d)
 * Four device outputs in the layout of img; none may overlap img or each
 * other.  Other arguments as me_edges.
 */
int me_fundamental_edges(const uint32_t *img, int32_t w, int32_t h,
                         int32_t stride_words, uint32_t *left, uint32_t *right,
                         uint32_t *up, uint32_t *down, int32_t boundary,
                         me_stream_t stream);

/*
 * Section 5 as drawn: the OR of the four edges inverted, so edge points are
 * 0 (black) and everything else 1 (white) -- the negation of me_edges on
 * the w pixels of each row (padding bits still written 0).  Arguments as
 * me_edges.
 */
int me_edges_display(const uint32_t *img, int32_t w, int32_t h,
                     int32_t stride_words, uint32_t *out, int32_t boundary,
                     me_stream_t stream);

/*
 * Second clause of the Section 1 definition on its own: out = 1 at a black
 * pixel with at most one black 8-neighbour (Fig. 1 neighbours 1-8), i.e.
 * isolated points and the ends of one-pixel lines.  Every such point is
 * also an edge point of me_edges (Section 1: the two-clause definition
 * reduces to the four edge-point types).  Arguments as me_edges.
 */
int me_end_points(const uint32_t *img, int32_t w, int32_t h,
                  int32_t stride_words, uint32_t *out, int32_t boundary,
                  me_stream_t stream);

/*
 * me_edges computed in place: the edge map replaces the image in img (the
 * result the paper draws over its input, with no second buffer of the
 * caller's).  Images up to 32 MiB (h * stride_words * 4 bytes; the environment
 * variable ME_INPLACE_COPY_MAX, read on every call, sets another limit in
 * bytes) are copied whole to scratch and computed from the copy.  Larger ones are cut into
 * bands of rows, one CTA per band walking it top to bottom so that each row
 * is overwritten only after every read of its original bits, and the two
 * rows on either side of every band seam are first copied to scratch
 * (2 * (bands - 1) * stride_words * 4 bytes, bands = about 4 per SM, at
 * least 32 rows each).  Scratch comes from the library's stream-ordered
 * pool on `stream` (as for me_edges_staged) and is returned when the call's
 * work is done.
 *
 * img           device pointer, 4-byte aligned; 128-bit accesses when it
 *               is 16-byte aligned and stride_words % 4 == 0.
 * w, h, stride_words, boundary, stream   as me_edges.
 * Above the copy limit, rows wider than 2048 groups of 4 words (262,144
 * pixels) return ME_ERR_TOO_BIG with nothing enqueued; failure to get the
 * scratch returns ME_ERR_CUDA with nothing enqueued.
 */
int me_edges_inplace(uint32_t *img, int32_t w, int32_t h, int32_t stride_words,
                     int32_t boundary, me_stream_t stream);

/*
 * Thresholding fused ahead of the method.  Section 7 makes a grey
 * photograph binary and then finds its edges, but names no rule; one global
 * threshold is taken: pixel (x, y) is white where
 * grey[y * pitch_bytes + x] >= threshold and black below it, and edge is
 * me_edges of that binary image.  One pass: 8 bits of grey read per pixel,
 * 1 bit written (2 with binary).
 *
 * grey          device u8[h][pitch_bytes], pitch_bytes >= w; 128-bit loads
 *               when grey and pitch_bytes are 16-byte aligned, byte loads
 *               otherwise.
 * threshold     <= 0 makes every pixel white, > 255 every pixel black.
 * edge          device output, h rows of stride_words words
 *               (>= ceil(w / 32)), 4-byte aligned, layout and zeroed padding
 *               as me_edges.
 * binary        NULL, or a device output of the same layout that receives
 *               the thresholded image packed.
 * boundary, stream   as me_edges.
 * grey, edge and binary must not overlap (ME_ERR_ALIAS).
 */
int me_threshold_edges(const uint8_t *grey, int32_t w, int32_t h, int32_t pitch_bytes,
                       int32_t threshold, uint32_t *edge, int32_t stride_words,
                       uint32_t *binary, int32_t boundary, me_stream_t stream);

/*
 * As me_threshold_edges with the threshold chosen from the image by Otsu's
 * rule (N. Otsu, IEEE Trans. SMC 9(1), 1979; Section 7 names no rule): the
 * t in 1..255 whose classes grey < t and grey >= t have the largest
 * between-class variance, scored as D(t) = x^2 / (n0 (N - n0)) with
 * x = S n0 - s0 N (N pixels, S their grey sum, n0 and s0 the same below t),
 * each operation a correctly rounded double operation in that order; the
 * first largest t wins, and an image of one grey value v takes t = v (all
 * white).  Three kernels on the stream: the grey histogram (8 bits read per
 * pixel), the choice of t (one CTA), then the one-pass threshold and edge
 * kernel reading t from device memory.  Asynchronous: t is not returned to
 * the host.
 *
 * grey, w, h, pitch_bytes, edge, stride_words, binary, boundary, stream
 *               as me_threshold_edges.
 * threshold_out NULL, or a 4-byte aligned device int32 that receives t.
 * Scratch of about 2 KB comes from the library's stream-ordered pool (as
 * for me_edges_staged); failure to
 * get it returns ME_ERR_CUDA with nothing enqueued.  threshold_out must not
 * overlap grey, edge or binary (ME_ERR_ALIAS).
 */
int me_threshold_edges_otsu(const uint8_t *grey, int32_t w, int32_t h, int32_t pitch_bytes,
                            uint32_t *edge, int32_t stride_words, uint32_t *binary,
                            int32_t boundary, int32_t *threshold_out, me_stream_t stream);

/* ---- many images in one launch ----------------------------------------- */

typedef struct me_desc {
    const uint32_t *img;     /* device input, layout as me_edges */
    uint32_t *edge;          /* device output, must not overlap img */
    int32_t w, h;            /* pixels, >= 1 */
    int32_t stride_words;    /* >= ceil(w / 32) */
    int32_t boundary;        /* ME_BOUNDARY_WHITE or ME_BOUNDARY_BLACK */
} me_desc;

/*
 * me_edges on n images of any sizes in ONE persistent kernel launch.
 * descs is a HOST array, copied
 * before the call returns (the caller may reuse it at once).  Image and
 * edge buffers are caller-owned device memory, checked for NULL, size and
 * overlap within each descriptor but not against one another: two
 * descriptors writing the same edge words race.  Images are split into
 * warp tiles (rows x word columns) that the launch walks in one pass;
 * 128-bit (else 64-bit) accesses are used per image where its buffers
 * allow them, as for me_edges.
 *
 * The tile configuration is that of the batch's kind: ME_KIND_BATCH if
 * every image allows 128-bit accesses, else ME_KIND_BATCH_ANY.  The
 * library owns a pinned staging ring, a device descriptor arena and (for
 * the bulk-copy engine) a graph cache keyed by tile configuration; all of
 * them live until me_shutdown().  A batch submitted again with the same
 * descriptors (byte for byte) under the same configuration launches on the
 * plan already on the device, without planning or uploading it; its images
 * are read and its edge maps written as on any call.  The kernel may be
 * placed while the kernel before it on the stream finishes (programmatic
 * dependent launch) and waits for it before touching memory.  n == 0
 * returns ME_OK with nothing enqueued.
 */
int me_edges_batch(const me_desc *descs, int32_t n, me_stream_t stream);

/*
 * A batch planned once and replayed many times: the descriptors are
 * uploaded to a device arena owned by the plan, and every me_batch_run is
 * one launch of the kernel alone (by programmatic dependent launch; the
 * bulk-copy engine's from a graph).  The plan keeps the tile configuration
 * of its batch kind current at creation.  Runs of one plan on different
 * streams must be ordered by the caller.
 */
typedef struct me_batch_plan me_batch_plan;
int me_batch_plan_create(const me_desc *descs, int32_t n, me_stream_t stream,
                         me_batch_plan **out);
int me_batch_run(me_batch_plan *plan, me_stream_t stream);
/* Algorithmic bytes a run moves: sum of 2 * h * stride_words * 4. */
int64_t me_batch_plan_bytes(const me_batch_plan *plan);
/* Waits for the plan's uploads, then frees it.  NULL is ignored. */
int me_batch_plan_destroy(me_batch_plan *plan);

/*
 * A batch that lives in HOST memory, end to end: every image is a range of
 * one host input buffer and its edge map goes to the same range of one host
 * output buffer (a ragged batch, as a serving front end or a file reader
 * lays it out).
 *
 * host_in, host_out  host buffers; pinned memory (cudaHostAlloc,
 *                    cudaHostRegister, torch pin_memory) moves at full link
 *                    speed, pageable memory works through the driver's
 *                    staging.  They must not overlap.
 * imgs[i]            offset_words: where image i starts in both buffers (16-
 *                    byte aligned offsets keep the 128-bit path); the image
 *                    takes h * stride_words words from there; w, h,
 *                    stride_words, boundary as me_desc.
 * chunk_bytes        input bytes per pipeline chunk (0: 16 MiB); images are
 *                    grouped into chunks in order, at least one per chunk.
 * stream             the work starts after what `stream` already holds.
 *
 * The library copies chunk k+1 up, computes chunk k (one persistent batch
 * launch) and copies chunk k-1 down at the same time, on its own streams,
 * into device staging it owns (three chunk slots of input and output,
 * kept until me_shutdown).
 * Synchronous: returns when every edge map is in host_out.
 */
typedef struct me_host_image {
    int64_t offset_words;
    int32_t w, h, stride_words, boundary;
} me_host_image;

int me_edges_batch_host(const uint32_t *host_in, uint32_t *host_out,
                        const me_host_image *imgs, int32_t n, int64_t chunk_bytes,
                        me_stream_t stream);

/* ---- tile configuration and autotuning --------------------------------- */

#define ME_KIND_SINGLE    0  /* me_edges and its single-image relatives */
#define ME_KIND_BATCH     1  /* me_edges_batch, plans, the host-buffer batch
                                and the server: batches whose every image
                                allows 128-bit accesses (both buffers 16-byte
                                aligned, stride_words % 4 == 0) */
#define ME_KIND_BATCH_ANY 2  /* the same calls on batches holding at least
                                one image that does not (the batch kernel
                                form with 64- and 32-bit accesses, whose best
                                tile shape differs) */

#define ME_ENGINE_REGS 0     /* rows slide through registers, 128/32-bit loads */
#define ME_ENGINE_BULK 1     /* row bands staged in shared memory by bulk
                                asynchronous copies (TMA), mbarrier pipeline */

typedef struct me_tile_cfg {
    int32_t engine;          /* ME_ENGINE_REGS or ME_ENGINE_BULK */
    int32_t rows_per_lane;   /* REGS: rows one lane walks: 4, 8, 16 or 32 */
    int32_t vec_words;       /* REGS: 4 = four words per lane, moved as one
                                128-bit access where both buffers are 16-byte
                                aligned and stride_words % 4 == 0, as two
                                64-bit accesses where they are 8-byte aligned
                                and stride_words is even, else as four 32-bit
                                accesses; 1 = 32-bit accesses only
                                (single images: one word per lane; batches:
                                four words per lane) */
    int32_t cta_threads;     /* 128, 256 or 512 */
    int32_t ctas_per_sm;     /* persistent grid of SMs x this, capped by what
                                fits on an SM; 0 = REGS: one warp per tile
                                (one chunk per warp in a batch), BULK: as
                                many as fit */
    int32_t stage_kb;        /* BULK: KiB per shared-memory stage (4..64) */
    int32_t stages;          /* BULK: stages in the ring (2..8); stages x
                                stage_kb <= 216 */
    int32_t chunk_tiles;     /* REGS batch: consecutive tiles a warp takes
                                at a time (1..64); warp w takes chunks w,
                                w + W, w + 2W, ... of the batch's tiles, so
                                the warps running at any moment work on
                                neighbouring memory.  0 = 4 */
} me_tile_cfg;

/* Read or replace the configuration used by the calls of `kind`. */
int me_get_tile_cfg(int32_t kind, me_tile_cfg *out);
int me_set_tile_cfg(int32_t kind, const me_tile_cfg *cfg);

/*
 * Time every candidate configuration on the caller's images (device
 * buffers; results are written to their edge buffers) with CUDA events on
 * `stream`, set the fastest for `kind`, and return it in *best.  A batch
 * sample must be of the batch kind named (ME_ERR_ARG otherwise: its
 * launches would not use the configurations being timed).  Each
 * candidate runs `reps` calls back to back (steady-state throughput), best
 * of three such runs.  Runs synchronously.  If the environment variable
 * ME_TUNE_CACHE names a file, the choice is also written there and read
 * back by the next process (keyed by device name and kind).
 */
int me_autotune(int32_t kind, const me_desc *sample, int32_t n, int32_t reps,
                me_stream_t stream, me_tile_cfg *best);

/* ---- serving ------------------------------------------------------------ */

typedef struct me_serve_cfg {
    int64_t hbm_budget_bytes;   /* device bytes for resident request images
                                   and edge maps (in + out) */
    int64_t staging_bytes;      /* pinned host bytes for request staging;
                                   0 = same as hbm_budget_bytes */
    int32_t max_inflight;       /* launched, unfinished batches (>= 1) */
    int32_t max_batch;          /* requests per launch (>= 1) */
    int32_t tick_us;            /* while batches are in flight, the period
                                   in microseconds at which the completion
                                   thread checks the oldest one; 0 checks
                                   continuously (lowest latency, one host
                                   core busy while the GPU works) */
    int32_t device;             /* CUDA device ordinal */
} me_serve_cfg;

typedef struct me_timing {
    double queue_us;            /* submit -> admitted (device memory given) */
    double device_us;           /* admitted -> result copied back to host */
    double total_us;            /* submit -> result ready */
} me_timing;

typedef struct me_server me_server;

/*
 * Start a server: a library thread that admits submitted requests against
 * the HBM budget, keeps their packed images and edge maps resident on the
 * device, and runs whatever is admitted as batches (continuous batching:
 * requests that arrive while batches run join the next launch once memory
 * and an in-flight slot are free), and a second thread that retires
 * finished batches in order.  Copies and kernels overlap on separate
 * streams.  The server owns a device pool of hbm_budget_bytes and a pinned
 * pool of staging_bytes, each split into halves for images and edge maps; a
 * request takes its packed size (rounded up to 256 bytes) in each half.
 * Requests of a batch that lie next to one another in both pools move
 * together, one copy each way.
 */
int me_serve_open(const me_serve_cfg *cfg, me_server **out);

/*
 * Queue one image.  host_img (h rows of stride_words words, layout as
 * me_edges) is copied before the call returns.  Returns ME_ERR_BUDGET when
 * this image's input plus output alone exceed the budget (or the staging
 * pool); otherwise the request waits until memory frees up.  *ticket
 * identifies the request to me_serve_poll.
 */
int me_serve_submit(me_server *srv, const uint32_t *host_img, int32_t w,
                    int32_t h, int32_t stride_words, int32_t boundary,
                    uint64_t *ticket);

/*
 * Collect a result.  Waits up to timeout_us microseconds (0: do not wait,
 * negative: wait without limit) and returns ME_OK with the edge map copied
 * to host_edge (h rows of the request's stride_words, padding written 0;
 * NULL for a direct ticket, whose edge map is in its own buffer already)
 * and the timing in *t (may be NULL); ME_PENDING (timeout 0) or
 * ME_TIMEOUT when not ready; ME_ERR_TICKET for an unknown or already
 * collected ticket; ME_ERR_ARG if another thread is already waiting for the
 * same ticket.  A collected ticket is forgotten.  Only the thread waiting
 * for a request is woken when it completes, so many threads can each wait
 * for their own requests.
 */
int me_serve_poll(me_server *srv, uint64_t ticket, uint32_t *host_edge,
                  int64_t timeout_us, me_timing *t);

/*
 * Direct submit, for images that already sit in host memory the GPU can
 * reach (cudaHostAlloc, cudaHostRegister, torch pin_memory): the batch
 * kernel reads host_img and writes the edge map into host_edge over the
 * CPU-GPU link, with no staging copy, no device memory and no copies on the
 * host or by the copy engines.  Both buffers (h rows of stride_words words,
 * 4-byte aligned, not overlapping) belong to the caller and must stay valid,
 * host_img unchanged and host_edge unread, until the ticket is collected
 * (or, after me_serve_cancel, until me_serve_close).  me_serve_poll of a
 * direct ticket takes host_edge = NULL (the edge map is already in the
 * buffer given here); me_serve_poll_view points at that buffer.
 * ME_ERR_ARG for a buffer the GPU cannot reach.  The HBM budget is not
 * charged.
 */
int me_serve_submit_direct(me_server *srv, const uint32_t *host_img, uint32_t *host_edge,
                           int32_t w, int32_t h, int32_t stride_words, int32_t boundary,
                           uint64_t *ticket);

/*
 * Zero-copy submit.  Reserves room for one image (h rows of stride_words
 * words) in the server's pinned staging and points *host_img at it; the
 * caller writes the image there and then calls me_serve_commit.  The
 * request joins the queue at once, in arrival order, but neither it nor
 * the requests behind it are admitted before it is committed, so commit
 * promptly.  ME_PENDING (nothing reserved) when staging has no room now:
 * retry, or use me_serve_submit, which waits in heap memory.  Otherwise
 * errors as me_serve_submit.  A reserved request may be cancelled.
 */
int me_serve_reserve(me_server *srv, int32_t w, int32_t h, int32_t stride_words,
                     int32_t boundary, uint64_t *ticket, uint32_t **host_img);

/* The image of a reserved ticket is written: the request may be admitted.
 * ME_ERR_ARG for a ticket that is not reserved or is committed already. */
int me_serve_commit(me_server *srv, uint64_t ticket);

/*
 * Zero-copy collect: waits as me_serve_poll, then points *host_edge at the
 * edge map in the server's staging instead of copying it out.  The edge
 * map stays there, and the ticket known, until me_serve_release(ticket).
 */
int me_serve_poll_view(me_server *srv, uint64_t ticket, int64_t timeout_us,
                       const uint32_t **host_edge, me_timing *t);

/* Give back the staging of a finished ticket and forget it (after
 * me_serve_poll_view).  ME_ERR_ARG while the request is unfinished. */
int me_serve_release(me_server *srv, uint64_t ticket);

/*
 * Forget a ticket.  A request still queued is dropped at once; one already
 * on the GPU finishes there and its memory is reclaimed when its batch
 * retires; a finished one is freed.  ME_ERR_TICKET for an unknown ticket;
 * ME_ERR_ARG while another thread's me_serve_poll is waiting for it.
 */
int me_serve_cancel(me_server *srv, uint64_t ticket);

/*
 * Counters since open: requests submitted, completed, batches launched,
 * and the most device bytes ever in use.  Any pointer may be NULL.
 */
int me_serve_stats(me_server *srv, int64_t *submitted, int64_t *completed,
                   int64_t *batches, int64_t *peak_bytes);

/*
 * Host-device copies the server has issued since open, both directions
 * (at most two per request; fewer when neighbouring requests move
 * together).
 */
int me_serve_copies(me_server *srv, int64_t *copies);

/*
 * Stop accepting requests, finish the ones admitted or queued (waiting at
 * most drain_timeout_us; negative = no limit), then free the server.
 * Uncollected results are dropped.  Returns ME_TIMEOUT if the drain ran
 * out (the server is freed all the same once its GPU work has ended).
 * No other call on the same server may run at the same time or after it.
 */
int me_serve_close(me_server *srv, int64_t drain_timeout_us);

/*
 * Faults that library kernels recorded since the last clear, as a bit set
 * (0 in a healthy run).  Bit 0: a bounded wait ran out (a bulk-copy stage
 * never arrived); the kernel stopped early and its outputs are incomplete.
 * Bit 1: the batch kernel without 32-bit tiles met an image that needs them
 * and skipped its tiles (the library picks the kernel from the same test,
 * so this marks a library fault).  clear != 0 resets both.  Synchronises
 * with the current device.
 */
int me_device_faults(int32_t clear, uint32_t *flags);

/* Free the batch rings, graphs and plans' shared state and the scratch
 * pools on every device (synchronising each), and forget the device
 * addresses me_edges_staged_static has looked up. */
int me_shutdown(void);

#ifdef __cplusplus
}
#endif

#endif /* ME_H */
