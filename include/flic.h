/*
 * flic.h — C ABI of libflic: the data-parallel hot path of FLIC (Fast Lidar Image
 * Clustering, Hasecke, Hahn & Kummert, arXiv 2003.00575) on one GB300 (sm_103a).
 *
 * The path, in the paper's terms:
 *   1. (optional) spherical projection of an xyz cloud into the range image (§I, Fig. 1);
 *   2. the neighbour test: the law-of-cosines distance between two range readings
 *      d1, d2 separated by beam angle alpha (Eq. 2), evaluated through a pre-computed
 *      per-offset constant (Eq. 3), against the single distance threshold delta
 *      (§III-B), for row and column offsets 1..S — the paper's Map Connections /
 *      skip connections (§III-B-2) — with azimuth wrap-around;
 *   3. connected-component labelling of the resulting pixel graph (§III-B-1);
 *   4. (optional) the scatter of pixel labels back onto the points (§I, Fig. 1).
 *
 * Conventions shared by every entry point
 *   - Images are row-major, row = laser channel, column = azimuth position (§III).
 *     Pixel p = r * cols + c.
 *   - Every pointer named "device" is a CUDA device pointer (or managed memory)
 *     allocated by the caller; the caller owns it.  Pointers named "host" are
 *     ordinary host memory, read during the call only, except for the host buffers of
 *     flic_label_batch_host and flic_server_submit, which are copied asynchronously.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).
 *     Every compute call only enqueues work on that stream and returns; results are
 *     ready once the stream reaches that point.  Only the *_create / *_destroy calls
 *     and flic_device_status synchronise.
 *   - Nothing throws across the ABI.  Each call returns a flic_status; on a non-OK
 *     status flic_last_error() returns a thread-local message describing it.
 *   - A handle is not thread-safe: use one handle per sensor and per host thread.  Calls
 *     on one handle (or one batch object) must not overlap on the GPU: their launches
 *     share the object's working memory (task counters, projection keys), so issue them
 *     on one stream or order them with events.
 *
 * Edge predicate (identical on every path; fixed here so that results are exact):
 *   valid(x)  :=  x > 0 and x finite            (0, negative, NaN, inf are "no return")
 *   K         :=  (float)(4 sin^2(alpha / 2))    computed in double on the host
 *                 (= 2 - 2 cos alpha, the constant of Eq. 3 in cancellation-free form)
 *   edge(a,b) :=  valid(a) && valid(b) && d2 <= delta2, with, in fp32, round-to-nearest,
 *                 no fused multiply-add:
 *                     t = a - b;  d2 = t*t + K*(a*b);  delta2 = delta*delta
 *   Vertical pair (r,c)-(r+k,c), k = 1..S, r+k < rows:
 *                 alpha = |elev[r+k] - elev[r]|       (K table Kv[r][k-1])
 *   Horizontal pair (r,c)-(r,(c+k) mod cols), k = 1..S (no wrap: c+k < cols):
 *                 alpha = k * az_step                 (K table Kh[r][k-1])
 *   With FLIC_FLAG_SUBLATTICE a pair of offset k >= 2 exists only for k = S and (r,c) with
 *   r and c multiples of S.
 * Labels: label[p] = the minimum linear index over p's connected component when p is
 * valid, -1 otherwise.
 */
#ifndef FLIC_H
#define FLIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FLIC_ABI_VERSION 1

typedef struct flic_ctx* flic_handle;
typedef struct flic_batch_ctx* flic_batch;

typedef enum {
    FLIC_OK = 0,
    FLIC_ERR_INVALID = 1,     /* bad argument: sizes, NULL pointers, non-finite delta ... */
    FLIC_ERR_OOM = 2,         /* a device or pinned-host allocation failed */
    FLIC_ERR_CUDA = 3,        /* a CUDA runtime call failed (message has the CUDA error) */
    FLIC_ERR_TIMEOUT = 4,     /* a bounded device loop gave up (see flic_device_status) */
    FLIC_ERR_BUSY = 5,        /* a batch object was given more frames than it holds */
    FLIC_ERR_UNSUPPORTED = 6  /* valid request this build does not handle (e.g. frame too large) */
} flic_status;

/* flic_create_ex flags */
#define FLIC_FLAG_NO_WRAP 0x1u  /* columns do not wrap (sensor covers < 360 deg azimuth) */
/* horizontal Eq. 3 constants from the true angle between a row's rays k columns apart,
 * cos(alpha) = cos^2(e) cos(k az_step) + sin^2(e), i.e. K = 4 cos^2(e) sin^2(k az_step / 2),
 * instead of the paper's k * az_step (§III-B) */
#define FLIC_FLAG_EXACT_RAY 0x2u
/* the paper's sparse Map Connection (§III-B-2, "connecting only every n-th point", n = skip):
 * offset 1 from every pixel, offset skip only from pixels whose row and column are both
 * multiples of skip (the pair's left or upper end; its column before any wrap), offsets
 * 2..skip-1 not at all.  Without it every pixel uses every offset 1..skip. */
#define FLIC_FLAG_SUBLATTICE 0x4u
/* Map Connections along the diagonals (§III-B-2, "MCs along the main diagonal"): besides
 * the row and column offsets, pixel (r,c) is joined to (r+k,(c+k) mod cols) and
 * (r+k,(c-k) mod cols) for k = 1..skip (no wrap: inside the frame only), with the Eq. 3
 * constant of the true angle between the two beams' rays, K = |u1 - u2|^2 for the unit rays
 * at (elev[r], 0) and (elev[r+k], k az_step), computed in double and rounded once.  Not
 * combined with FLIC_FLAG_SUBLATTICE.  flic_edges reports the row and column pairs only. */
#define FLIC_FLAG_DIAGONAL 0x8u

/* Largest frame the labeller accepts: rows * cols <= FLIC_MAX_PIXELS, rows <= FLIC_MAX_ROWS.
 * A frame is split into at most 64 full-height column strips of at most 32768 (padded)
 * pixels each; a shape that does not fit gives FLIC_ERR_UNSUPPORTED from flic_create. */
#define FLIC_MAX_PIXELS (1 << 21)
#define FLIC_MAX_ROWS 512
#define FLIC_MAX_SKIP 8

/* ABI version compiled into the library (FLIC_ABI_VERSION of its build). */
int32_t flic_abi_version(void);

/* Thread-local description of the last non-OK status returned on this thread. */
const char* flic_last_error(void);

/*
 * flic_create — build a sensor handle: the per-offset cosine constants of Eq. 3
 * (§III-B; "pre-calculating the cosine of the given angles") and the projection
 * boundary tables, resident on the current CUDA device.
 *   rows, cols        range-image shape, 1 <= rows <= FLIC_MAX_ROWS,
 *                     rows*cols <= FLIC_MAX_PIXELS
 *   elevation         host, rows doubles: elevation angle of each row's beam in radians,
 *                     any order (the channel-angle lookup table of §III-A)
 *   az_step           radians between adjacent columns (> 0, finite)
 *   delta             distance threshold in metres (> 0, finite); §III-B uses 0.8
 *   skip              S, 1..FLIC_MAX_SKIP: offsets 1..S are tested along rows and
 *                     columns (§III-B-2; S = 1 is the plain 4-neighbourhood)
 *   out               receives the handle; the handle owns all device memory it uses
 * Synchronises the device.  Errors: FLIC_ERR_INVALID, FLIC_ERR_OOM, FLIC_ERR_CUDA.
 */
flic_status flic_create(int32_t rows, int32_t cols, const double* elevation, double az_step,
                        float delta, int32_t skip, flic_handle* out);

/* flic_create with FLIC_FLAG_* flags (flags = 0 gives flic_create). */
flic_status flic_create_ex(int32_t rows, int32_t cols, const double* elevation, double az_step,
                           float delta, int32_t skip, uint32_t flags, flic_handle* out);

/* Frees everything the handle owns.  Synchronises the device.  NULL is accepted. */
flic_status flic_destroy(flic_handle h);

/*
 * flic_get_tables — copy the handle's fp32 constants to host memory (for checking):
 *   kv, kh   host, rows*skip floats each, [r][k-1] layout; Kv entries with r+k >= rows
 *            are 0.  Either pointer may be NULL.
 */
flic_status flic_get_tables(flic_handle h, float* kv, float* kh);

/*
 * flic_get_diag_table — copy the handle's diagonal constants (FLIC_FLAG_DIAGONAL, §III-B-2)
 * to host memory: kd, host, rows*skip floats, [r][k-1] = the constant of the pairs
 * (r,c)-(r+k,c+-k), 0 where r+k >= rows.  FLIC_ERR_INVALID when the handle was created
 * without the flag.
 */
flic_status flic_get_diag_table(flic_handle h, float* kd);

/*
 * flic_edges — the neighbour test alone (Eq. 2/3 with Map Connections, §III-B-2):
 *   range    device, rows*cols fp32 (see valid())
 *   mask     device, rows*cols uint16: bit (k-1) = horizontal edge (r,c)-(r,(c+k) mod cols),
 *            bit (8+k-1) = vertical edge (r,c)-(r+k,c), for k = 1..S.
 * Errors: FLIC_ERR_INVALID (NULL pointer), FLIC_ERR_CUDA.
 */
flic_status flic_edges(flic_handle h, const float* range, uint16_t* mask, void* stream);

/*
 * flic_label — the neighbour test followed by connected-component labelling of the
 * pixel graph (§III-B, §III-B-1, §III-B-2), one frame:
 *   range    device, rows*cols fp32, not modified
 *   labels   device, rows*cols int32, written: min linear index of the component, or -1
 * The labels buffer is also the kernel's only global working memory; it must not alias
 * range.  Errors: FLIC_ERR_INVALID, FLIC_ERR_CUDA.  A bounded device loop that gives up
 * is reported by flic_device_status as FLIC_ERR_TIMEOUT.
 */
flic_status flic_label(flic_handle h, const float* range, int32_t* labels, void* stream);

/*
 * flic_project — spherical projection of a point cloud into the range image (§I: used
 * when raw ranges are unavailable; §IV-B on one-to-one point/pixel matching):
 *   xyz          device, n*3 fp32, point i = (x, y, z) at xyz[3i..3i+2], sensor at origin
 *   n            number of points, 0 <= n < 2^31
 *   range_out    device, rows*cols fp32, written (0 where no point lands); may be NULL,
 *                then the handle's own buffer is used (see flic_range_buffer)
 *   point_pixel  device, n int32, written: pixel index of point i, or -1 when the point
 *                is invalid (range <= 0 or non-finite) or outside the elevation span
 * Column c holds azimuth [c*az_step, (c+1)*az_step) measured counter-clockwise from +x;
 * row boundaries are the midpoints between adjacent beam elevations, the outer rows
 * extending half a spacing beyond their beam.  Bin membership is decided by exact fp32
 * sign tests against host-built boundary vectors.  Several points in one pixel: the
 * pixel takes the smallest of their ranges; every point still records its pixel.
 * Requires rows >= 2 and cols*az_step = 2*pi (full revolution; |error| < 1e-6).
 * Uses a handle-owned scratch of rows*cols 32-bit keys.
 * Errors: FLIC_ERR_INVALID, FLIC_ERR_UNSUPPORTED (partial revolution), FLIC_ERR_OOM,
 * FLIC_ERR_CUDA.
 */
flic_status flic_project(flic_handle h, const float* xyz, int64_t n, float* range_out,
                         int32_t* point_pixel, void* stream);

/* Device pointer of the handle's own range image (allocated on first use), or NULL. */
float* flic_range_buffer(flic_handle h);

/*
 * flic_scatter — back-projection of pixel labels onto the points (§I, Fig. 1):
 *   labels        device, rows*cols int32 (a flic_label result)
 *   point_pixel   device, n int32 (a flic_project result)
 *   point_labels  device, n int32, written: labels[point_pixel[i]], or -1 when
 *                 point_pixel[i] < 0
 * Errors: FLIC_ERR_INVALID, FLIC_ERR_CUDA.
 */
flic_status flic_scatter(flic_handle h, const int32_t* labels, const int32_t* point_pixel,
                         int64_t n, int32_t* point_labels, void* stream);

/*
 * flic_project_batch — flic_project on nclouds clouds at once (no counterpart in the paper):
 * three launches in all (keys cleared, points projected, range images decoded, at most 96
 * clouds per launch), each cloud on its own handle's tables and key scratch, so the
 * handles must be distinct.  Results equal flic_project cloud by cloud.
 *   hs           host array of nclouds distinct handles (each able to project)
 *   xyz          host array of nclouds device pointers (cloud i: n[i]*3 fp32)
 *   n            host array of nclouds point counts (0 <= n[i] < 2^31)
 *   range_out    host array of nclouds device pointers (rows_i*cols_i fp32), or NULL: the
 *                handles' own buffers (flic_range_buffer)
 *   point_pixel  host array of nclouds device pointers (n[i] int32)
 * flic_scatter_batch — flic_scatter on nclouds clouds in one launch per 96 clouds:
 *   labels[i] (rows_i*cols_i int32), point_pixel[i] and point_labels[i] (n[i] int32).
 * The host arrays are read during the call only.  Errors: FLIC_ERR_INVALID (NULL, bad
 * count, a handle repeated), FLIC_ERR_UNSUPPORTED (a handle cannot project), FLIC_ERR_CUDA.
 */
flic_status flic_project_batch(const flic_handle* hs, int32_t nclouds, const float* const* xyz,
                               const int64_t* n, float* const* range_out,
                               int32_t* const* point_pixel, void* stream);
flic_status flic_scatter_batch(const flic_handle* hs, int32_t nclouds, const int32_t* const* labels,
                               const int32_t* const* point_pixel, const int64_t* n,
                               int32_t* const* point_labels, void* stream);

/*
 * Batched labelling (no counterpart in the paper, which labels one frame at a time on one
 * CPU core): many frames of different sensors labelled by one persistent kernel launch,
 * replayed from a CUDA graph.  Results are identical to flic_label on each frame.
 *
 * flic_batch_create — a batch object holding device descriptors for up to max_frames
 *   frames and the captured graph.  Synchronises.  Errors: INVALID, OOM, CUDA.
 * flic_label_batch — label nframes frames:
 *   hs        host array of nframes handles (may repeat; each frame uses its handle's
 *             shape, tables, delta and skip)
 *   ranges    host array of nframes device pointers (frame i: rows_i*cols_i fp32)
 *   labels    host array of nframes device pointers (frame i: rows_i*cols_i int32)
 *   The host arrays are read during the call only.  A call with the same handles and
 *   buffers as the previous call on this object only replays the captured launch; any
 *   other call re-plans, waits on the host until the previous descriptor upload has left
 *   the staging buffer, and orders its upload after the previous launch on the device.
 *   Errors: INVALID, BUSY (nframes > max_frames), CUDA.
 * flic_batch_destroy — frees the object.  Synchronises.  NULL is accepted.
 */
flic_status flic_batch_create(int32_t max_frames, flic_batch* out);
flic_status flic_label_batch(flic_batch b, const flic_handle* hs, const float* const* ranges,
                             int32_t* const* labels, int32_t nframes, void* stream);
flic_status flic_batch_destroy(flic_batch b);

/*
 * flic_label_batch_host — flic_label_batch on frames held in host memory (no counterpart
 * in the paper; the labels equal flic_label_batch's):
 *   hs           host array of nframes handles, as for flic_label_batch
 *   host_ranges  host, the frames' range images back to back: frame i (rows_i*cols_i
 *                fp32, row-major) starts right after frame i-1
 *   host_labels  host, int32, the same packed layout; written when the work queued by
 *                this call has finished on `stream`
 *   groups       0: built-in (4); otherwise 1..16 groups of consecutive frames of about
 *                equal pixel counts (at most nframes): each group's upload, labelling and
 *                download are queued on separate streams, so that one group's copies run
 *                under another group's labelling and both copy directions run at once
 *   flags        0, or FLIC_HOST_INPUT_READY: host_ranges already hold this call's
 *                readings, so the uploads and the labelling need not wait for work queued
 *                earlier on `stream`; a call's uploads then run under the previous call's
 *                downloads.  Without it the whole call is ordered after that work.
 *   stream       the end of the call (labels in host_labels) is ordered before later work
 *                on it
 *   Host memory should be page-locked (cudaHostAlloc or cudaHostRegister) for the copies
 *   to overlap; pageable memory gives the same labels with serialised copies.  The object
 *   keeps two sets of device copies, used by alternate calls (each as large as the
 *   largest batch seen; growing them waits for all earlier calls of this kind), and one
 *   internal batch object per group and set, with this object's tuning and schedule.
 *   The host buffers must not be modified or freed until the work on `stream` has
 *   finished.  flic_batch_last_plan does not report these calls.
 *   Errors: INVALID (NULL argument, bad groups or flags, the buffers overlap), BUSY
 *   (nframes > max_frames), OOM, CUDA; on an error, work queued before it may still run.
 */
#define FLIC_HOST_INPUT_READY 0x1u
flic_status flic_label_batch_host(flic_batch b, const flic_handle* hs, int32_t nframes,
                                  const float* host_ranges, int32_t* host_labels,
                                  int32_t groups, uint32_t flags, void* stream);

/*
 * Launch-shape tuning (no counterpart in the paper).  px_per_cta: target pixels per
 * strip, the tile of the shared-memory union pass (0 = built-in default: 2048 for a
 * handle's single-frame calls, where more blocks per frame lower the latency, and 16384
 * for a batch object, where many frames fill the GPU);
 * threads: threads per block (128..512, multiple of 32; 0 = 512); max_strips: upper
 * bound on the strips one frame is split into (1..64; 0 = 64); ctas_per_sm (batch only):
 * cap on resident blocks per SM (0 = as many as fit).  flic_set_tuning applies to the
 * handle's single-frame calls, flic_batch_set_tuning to a batch object.  Results never
 * depend on these values.  Errors: FLIC_ERR_INVALID, FLIC_ERR_UNSUPPORTED (the frame
 * does not fit the requested shape; the previous tuning stays).
 */
flic_status flic_set_tuning(flic_handle h, int32_t px_per_cta, int32_t threads, int32_t max_strips);
flic_status flic_batch_set_tuning(flic_batch b, int32_t px_per_cta, int32_t threads,
                                  int32_t max_strips, int32_t ctas_per_sm);
/* Merge schedule of a batch object: a frame's flatten tasks are queued this many waves of
 * resident blocks after its last strip task (0..64; default 8).  Results never depend
 * on it.  Errors: FLIC_ERR_INVALID. */
flic_status flic_batch_set_schedule(flic_batch b, int32_t p3_delay_waves);

/*
 * flic_plan_info — the handle's single-frame launch shape (no counterpart in the paper):
 *   info  host, 5 ints: strips, strip width, shared-memory row pitch, shared-memory bytes
 *         per block, threads per block.
 * flic_batch_last_plan — shape of the last flic_label_batch launch:
 *   info  host, 8 ints: queued tasks, blocks launched (persistent grid), max strips per
 *         frame, threads per block, shared-memory bytes per block, strips over all frames,
 *         frames, blocks that fit at once.
 */
flic_status flic_plan_info(flic_handle h, int32_t* info);

/*
 * flic_plan_frame — the strip split flic_create would choose, computed on the host only
 * (no CUDA call): info, host, 4 ints: strips, strip width, shared-memory row pitch,
 * shared-memory bytes per block.  Errors: INVALID, UNSUPPORTED (does not fit).
 */
flic_status flic_plan_frame(int32_t rows, int32_t cols, int32_t skip, int32_t px_per_cta,
                            int32_t max_strips, int32_t* info);
flic_status flic_batch_last_plan(flic_batch b, int32_t* info);

/*
 * flic_set_ground — ground extraction (§III-A) before labelling, for this handle's
 * flic_label, flic_label_batch and flic_edges calls and its served frames: a reading that
 * spans a horizontal surface with the reading above it (row r-1, the previous channel) —
 * the angle beta of Eq. 1 within +-theta of the upper beam's depression angle, tested in
 * Eq. 1's tangent form with per-row constants, den > 0 and
 * tan(gamma - theta)*den <= d2*sin(alpha) <= tan(gamma + theta)*den — counts as no
 * measurement (label -1, no edges).  The first row decides as the second.  With
 * mount_height > 0 (metres from the sensor down to the wheels' contact plane), horizontal
 * readings above the line z = rho*tan(theta) - mount_height are kept (raised surfaces such
 * as car roofs, §III-A's height image).  theta in radians (the paper uses 10 degrees);
 * theta <= 0 turns it off.  Synchronises (the table is uploaded).  Errors:
 * FLIC_ERR_INVALID (theta >= 90 degrees or not finite), FLIC_ERR_OOM, FLIC_ERR_CUDA.
 */
flic_status flic_set_ground(flic_handle h, double theta, double mount_height);

/*
 * flic_filter_relabel — cluster candidates (§III-B: labelled clusters with fewer than a
 * minimum number of measurements are discarded as sensor noise; the paper's minimum is
 * 100 points).  In place, on labels produced by flic_label / flic_label_batch for this
 * handle's frame shape (component minima, -1 where no measurement): every component with
 * fewer than min_size pixels becomes -1, and the others are numbered 0..N-1 in ascending
 * order of their minimum index, i.e. in the raster order of their first pixels (the
 * numbering of scipy.ndimage.label, minus one).
 *   labels    device int32 rows*cols, read and rewritten
 *   min_size  pixels a component needs to be kept (<= 1 keeps every component)
 *   num_out   device int32 receiving N, or NULL
 * Uses handle-owned scratch (8 bytes per pixel, allocated on the first call; the call
 * then synchronises once).  Other labels (values outside 0..rows*cols-1) are left in
 * place and reported by flic_device_status; values inside that range that are not
 * component minima give an unspecified numbering.  Errors: FLIC_ERR_INVALID (NULL),
 * FLIC_ERR_OOM, FLIC_ERR_CUDA.
 */
flic_status flic_filter_relabel(flic_handle h, int32_t* labels, int32_t min_size,
                                int32_t* num_out, void* stream);

/*
 * flic_filter_relabel_batch — the same for nframes frames in one set of launches: frame i
 * has hs[i]'s shape and labels[i] (device int32, rewritten in place); num_out is a device
 * int32 array of nframes (N of each frame) or NULL.  Scratch (8 bytes per pixel of the
 * batch) belongs to the batch object and grows on demand; growing waits for the batch's
 * previous relabel.  Errors: FLIC_ERR_INVALID, FLIC_ERR_OOM, FLIC_ERR_CUDA.
 */
flic_status flic_filter_relabel_batch(flic_batch b, const flic_handle* hs,
                                      int32_t* const* labels, int32_t nframes, int32_t min_size,
                                      int32_t* num_out, void* stream);

/*
 * flic_label_filter_batch — flic_label_batch followed by flic_filter_relabel_batch on the
 * same frames, with the component sizes counted by the labelling kernel itself: each
 * strip counts the pixels of its strip-local components from its runs (a run's length is
 * one bit scan of its edge words) and, after the border merges, adds the count of every
 * root that a merge hooked into its component's root.  The relabel step then reads only
 * the roots' counts and skips the size histogram over the labels.  Arguments as the two
 * calls: frame i has hs[i]'s shape, ranges[i] (device float32, read) and labels[i]
 * (device int32, written: after the call -1 or the component's id 0..N-1); num_out a
 * device int32 array of nframes or NULL.  Uses the batch's relabel scratch (8 bytes per
 * pixel, grown on demand).  The result equals flic_label_batch + flic_filter_relabel_batch.
 * Errors: those of the two calls.
 */
flic_status flic_label_filter_batch(flic_batch b, const flic_handle* hs,
                                    const float* const* ranges, int32_t* const* labels,
                                    int32_t nframes, int32_t min_size, int32_t* num_out,
                                    void* stream);

/*
 * flic_device_status — synchronise the device, read and (if clear != 0) reset the
 * handle's device error word.  Returns FLIC_OK; FLIC_ERR_TIMEOUT when a bounded loop in a
 * kernel gave up since the last reset (labels of that call are then not valid); or
 * FLIC_ERR_INVALID when flic_filter_relabel(_batch) met a label outside 0..rows*cols-1
 * (such labels are left as they are and never used as an index).
 */
flic_status flic_device_status(flic_handle h, int32_t clear);

/*
 * flic_debug_set_iter_limit — set the iteration bound of the handle's device loops
 * (0 = built-in default).  Used to test the timeout path without a real fault.
 */
flic_status flic_debug_set_iter_limit(flic_handle h, int32_t limit);

/*
 * Serving (no counterpart in the paper, which processes one recorded frame at a time):
 * a request loop for several sensors that admits frames as device memory frees up,
 * batches whatever has arrived into one labelling launch, and overlaps batches on
 * several streams (continuous batching).  Results equal the single-frame calls.
 *
 * flic_server_create — a server for nsensors sensors:
 *   sensors         host array of handles; each slot gets its own copy of the sensor's
 *                   tables and scratch, so the caller may destroy these afterwards
 *   max_points      host array: largest cloud per sensor (0: range images only)
 *   nstreams        CUDA streams batches rotate over (1..8; 2 overlaps one batch's
 *                   copies and kernels with the next)
 *   max_batch       frames per launch (1..4096)
 *   mem_budget      device bytes for frame slots (each slot holds one in-flight frame:
 *                   range image, labels, xyz, pixel map, point labels); at least one slot
 *                   per sensor is created
 *   max_queue       requests that may wait for a slot before submit refuses (>= 1)
 *   Starts one dispatcher thread.  Each stream has two batch objects: a batch too small
 *   to give every SM one 16384-pixel strip, launched while no other stream has a batch in
 *   flight, is labelled with 2048-pixel strips (lower latency); under load, and for
 *   larger batches, the batch default is used.  Each batch object reserves the shared
 *   memory of its largest sensor, so every mix of sensors has one launch shape, and is
 *   launched once at creation (on zeroed slots), so that no CUDA graph is captured while
 *   frames are served; creation synchronises.  A batch's clouds are projected by one
 *   launch per step (keys cleared, points projected, range images decoded) and their
 *   labels scattered by one more.  Errors: INVALID, OOM, CUDA.
 * flic_server_submit — queue one frame; returns at once:
 *   sensor, kind    sensor index; kind 0 = range image (host_in: rows*cols fp32),
 *                   kind 1 = point cloud (host_in: n*3 fp32 xyz, n <= max_points)
 *   host_out        labels, written when the frame completes: rows*cols int32 (kind 0)
 *                   or n int32 point labels (kind 1)
 *   Both host buffers must stay valid until the frame's completion is polled; pinned
 *   (page-locked) buffers keep the copies asynchronous.  FLIC_ERR_BUSY when max_queue
 *   requests are already waiting (counted as rejected).
 * flic_server_hold — hold != 0 pauses admission (requests keep queueing, nothing new
 *   is launched; batches already in flight finish); 0 resumes.  Lets a caller that knows
 *   frames arrive together have them labelled in one launch.
 * flic_server_poll — move up to max completion records to out (non-blocking); returns
 *   the number moved.
 * flic_server_drain — wait until every submitted frame has completed (or timeout_s).
 * flic_server_stats — out, host, 8 int64: submitted, rejected, completed, batches,
 *   largest batch, slots, device bytes of the slots, batches in flight now.
 * flic_server_destroy — drains, stops the dispatcher, frees everything.
 */
typedef struct flic_server_ctx* flic_server;
typedef struct {
    uint64_t tag;        /* caller's tag from flic_server_submit */
    int32_t sensor;
    int32_t kind;
    int64_t n;           /* points (kind 1) or pixels (kind 0) */
    int32_t status;      /* FLIC_OK, or the error of the launch that carried the frame */
    int32_t batch_size;  /* frames in the launch that carried it */
    double t_submit;     /* seconds on the server's monotonic clock */
    double t_launch;     /* its batch was enqueued */
    double t_done;       /* its results were in host memory */
} flic_completion;

flic_status flic_server_create(const flic_handle* sensors, int32_t nsensors,
                               const int64_t* max_points, int32_t nstreams, int32_t max_batch,
                               int64_t mem_budget, int32_t max_queue, flic_server* out);
flic_status flic_server_submit(flic_server s, int32_t sensor, int32_t kind, const void* host_in,
                               int64_t n, int32_t* host_out, uint64_t tag);
flic_status flic_server_hold(flic_server s, int32_t hold);
int32_t flic_server_poll(flic_server s, flic_completion* out, int32_t max);
flic_status flic_server_drain(flic_server s, double timeout_s);
flic_status flic_server_stats(flic_server s, int64_t* out);
flic_status flic_server_destroy(flic_server s);
/* The server's monotonic clock in seconds (the clock of the completion records). */
double flic_server_clock(void);

/*
 * flic_project_noalloc — flic_project for callers that cannot allocate device memory
 * (the paper has no counterpart; this is an integration entry point).  Some callers may
 * only use the buffers they are handed: code running inside a host framework whose
 * device memory belongs to its own pool, or plugins that must not call cudaMalloc.  This
 * call needs no handle and allocates nothing: its working memory (the 32-bit per-pixel
 * keys, the boundary and seed tables and a status word) lives in static device arrays of
 * fixed size inside libflic, held by every GPU that loads the library until the process
 * exits (about 1.1 MiB).
 *   rows, cols   2 <= rows <= FLIC_MAX_ROWS, cols <= FLIC_NOALLOC_MAX_COLS,
 *                rows*cols <= FLIC_NOALLOC_MAX_PIXELS; larger shapes give FLIC_ERR_INVALID
 *   elevation    host, rows doubles (radians, any order, distinct); az_step as in
 *                flic_create (cols*az_step must be 2*pi: FLIC_ERR_UNSUPPORTED otherwise)
 *   xyz, n, range_out, point_pixel, stream: as in flic_project (range_out is required)
 * Results are identical to flic_project on a handle of the same geometry.  The first call
 * on each device looks up the static arrays' device addresses (cudaGetSymbolAddress) with
 * that device current.  Each call copies the tables on `stream` from fixed host arrays
 * that the next call overwrites (pageable copies, which wait for the work queued earlier
 * on `stream`), clears the keys it uses and the status word, and — unlike the other
 * compute calls — returns only when its own work on `stream` has finished, so that a
 * bounded pixel search that gave up is reported as FLIC_ERR_TIMEOUT.  It can therefore
 * not be captured into a CUDA graph: a capturing stream gives FLIC_ERR_UNSUPPORTED.  All
 * calls share the arrays, so calls that overlap on the GPU (other streams or threads) race
 * and must be serialised by the caller.  Errors: FLIC_ERR_INVALID, FLIC_ERR_UNSUPPORTED,
 * FLIC_ERR_TIMEOUT, FLIC_ERR_CUDA.
 */
#define FLIC_NOALLOC_MAX_PIXELS (1 << 18)
#define FLIC_NOALLOC_MAX_COLS 8192
flic_status flic_project_noalloc(int32_t rows, int32_t cols, const double* elevation,
                                 double az_step, const float* xyz, int64_t n, float* range_out,
                                 int32_t* point_pixel, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FLIC_H */
