/*
 * fsr.h - C-ABI of the GB300 (sm_103a) Frequency Selective Reconstruction
 * library (libfsr_gb300.so).
 *
 * Method: Regensky, Grosche, Seiler, Kaup, "Real-Time Frequency Selective
 * Reconstruction through Register-Based Argmax Calculation", MMSP 2020.
 * Every B x B target block of the image is reconstructed on its own
 * S x S support, S = B + 2L (Sec. II; Sec. III-A, Eq. 13):
 *   w = rho^dist on known pixels, 0 elsewhere            (Eq. 5)
 *   R_w = F2{f~ w},  W = F2{w}                             (Eq. 7)
 *   K times: (u,v) = argmax w_f |R_w|^2                    (Eqs. 8, 9)
 *            p = R_w[u,v] / W[0,0]                          (Eq. 10)
 *            G[u,v] += gamma p S^2                          (Eq. 11)
 *            R_w[k,l] -= gamma p W[(k-u) mod S, (l-v) mod S] (Eqs. 12, 14, 15)
 *   g = IDFT2(G); out = f on known pixels, Re g elsewhere (end of Sec. II)
 *
 * Conventions fixed by this library where the paper is silent:
 *   - forward DFT e^{-j2pi(km+ln)/S} unnormalised, inverse 1/S^2 e^{+j...};
 *     k pairs with the row index m;
 *   - argmax ties go to the lowest linear index k*S + l;
 *   - the output at unknown pixels is Re g (the model is complex because
 *     single components are updated);
 *   - pixels outside the image are unknown; a block with no known pixel in
 *     its support outputs 0 at its unknown pixels;
 *   - the weight centre of the even support is (S-1)/2.
 *
 * All entry points return an int status (FSR_OK or an FSR_ERR_* code); the
 * text of the last error of a handle is available from fsr_last_error().
 * Device pointers are owned by the caller; the library owns only its handle
 * and the workspace it allocates inside it.  Entry points that take a stream
 * are asynchronous on that stream unless stated otherwise; work of one
 * handle may be queued on several streams at once.  A handle is not
 * thread-safe: calls on one handle must not overlap in time on the host (use
 * one handle per host thread; a server's entry points are thread-safe).
 */
#ifndef FSR_GB300_H
#define FSR_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define FSR_OK              0
#define FSR_ERR_INVALID_ARG 1   /* a pointer, size or parameter is out of range */
#define FSR_ERR_OOM         2   /* a device or pinned allocation failed / cap exceeded */
#define FSR_ERR_CUDA        3   /* a CUDA runtime call or a kernel launch failed */
#define FSR_ERR_TIMEOUT     4   /* a bounded device-side wait gave up */
#define FSR_ERR_UNSUPPORTED 5   /* valid request this library does not implement */

/* Arithmetic of the iteration (fsr_params.precision). */
#define FSR_FP32       0  /* FP32 everywhere (the production path) */
#define FSR_FP64_DEBUG 1  /* FP64 everywhere; selection sequences comparable with an FP64 reference */
/* Precision study (single-image entry points, B = 4): the forward 2-D DFT of
 * the support and the inverse 2-D DFT of the model coefficients on tensor
 * cores with FP32 accumulation; the iteration in FP32; W[0][0] of Eq. (10)
 * summed in FP64 from the weights. */
#define FSR_TC_BF16X3  2  /* operands split into BF16 hi + lo, products hi.hi + hi.lo + lo.hi */
#define FSR_TC_TF32    3  /* operands rounded to TF32 */

/* Model update per iteration (fsr_params.update). */
#define FSR_UPDATE_SINGLE    0  /* the paper's: one complex component (Eqs. 11-12) */
/* Ablation (the original FSR's real model; S = 32, B = 4, FSR_FP32 or
 * FSR_FP64_DEBUG): with a = gamma p (Eq. 10) the selected component and its
 * conjugate are updated together, G[u,v] += a S^2, G[-u,-v] += a* S^2,
 * R_w[k,l] -= a W[k-u,l-v] + a* W[k+u,l+v] (once for a self-conjugate
 * (u,v)), so R_w stays Hermitian and g real. */
#define FSR_UPDATE_CONJ_PAIR 1

/* Library configuration (fsr_create). */
typedef struct fsr_config {
    int device;                  /* CUDA device ordinal the handle is bound to */
    size_t workspace_bytes;      /* cap on device memory the handle may allocate; 0 = no cap */
    const char *schedule_cache;  /* optional path of the batch-schedule cache written by
                                    fsr_autotune_batch; read at creation; NULL = none */
} fsr_config;

/* Method parameters (Sec. II; defaults of Sec. IV: B=4, rho=0.7, gamma=0.5). */
typedef struct fsr_params {
    int block;        /* B: target block size; one of 2, 4, 8, 16 */
    int border;       /* L: border; the support S = B + 2L is 32 (any B), 24 (B in
                         {4, 8}), 16 (B in {2, 4, 8}), 8 or 4 (B in {2, 4}); S < 32
                         runs FSR_FP32 and FSR_FP64_DEBUG only */
    int iters;        /* K: number of iterations, 0 <= K <= 65535 */
    float rho;        /* rho-hat of Eq. (5), in (0, 1] */
    float gamma;      /* gamma of Eqs. (11)-(12), in (0, 1] */
    int freq_weight;  /* 1: objective w_f |R_w|^2 (Eq. 8, paper default); 0: |R_w|^2 */
    int precision;    /* FSR_FP32, FSR_FP64_DEBUG, or (single image, B = 4, K <= 256) FSR_TC_BF16X3 /
                         FSR_TC_TF32: both 2-D DFTs as tcgen05 tensor-core GEMMs */
    int16_t *seq_out; /* optional DEVICE buffer of N*K entries (N = number of blocks,
                         block b = by*ceil(width/B) + bx): the selected u*S+v of each
                         iteration, -1 for a block without known pixels; NULL = off */
    int update;       /* FSR_UPDATE_SINGLE (0, zero-initialised default) or FSR_UPDATE_CONJ_PAIR */
    float reuse;      /* re-use weight delta in [0, 1].  0 (zero-initialised default): the
                         paper's independent blocks (Sec. II refrains from re-using
                         reconstructed pixels).  > 0: the sequential form of the original
                         FSR: blocks in raster order, and an unknown pixel of an earlier
                         block's target takes part in later supports with its
                         reconstruction and the weight delta * rho^dist of Eq. (5).
                         Runs as one launch per wavefront of blocks (t = a*by + bx,
                         a = ceil(L/B) + 1); fsr_reconstruct, fsr_reconstruct_host and
                         fsr_reconstruct_batch (each image its own raster order, the
                         images sharing the wavefront launches), S = 32,
                         FSR_UPDATE_SINGLE, FSR_FP32 / FSR_FP64_DEBUG only. */
} fsr_params;

typedef struct fsr_handle fsr_handle;

/* Create a handle on cfg->device.  Checks that the device runs this library
 * (sm_103a) and sets the kernels' shared-memory limits.
 * Errors: INVALID_ARG (NULL pointers, bad ordinal), UNSUPPORTED (other GPU),
 * CUDA.  On error *out is set to NULL. */
int fsr_create(const fsr_config *cfg, fsr_handle **out);

/* Release the handle and every device/pinned buffer it owns.  Waits for
 * nothing: the caller must not destroy a handle with work in flight.
 * NULL is accepted and ignored. */
int fsr_destroy(fsr_handle *h);

/* Text of the last error recorded on h (never NULL; "" after success).
 * With h == NULL: the last error of fsr_create in this thread. */
const char *fsr_last_error(const fsr_handle *h);

/* Reconstruct one single-channel image on the device (Sec. II, Sec. III-A).
 *   img    DEVICE float32, height x width, row pitch `pitch` elements;
 *          values at unknown pixels are never used (may be NaN)
 *   mask   DEVICE uint8, same geometry and pitch; nonzero = known pixel
 *   out    DEVICE float32, same geometry and pitch; every in-image pixel is
 *          written: known pixels bit-exact copies of img, unknown ones Re g.
 *          out must not overlap img or mask (supports read neighbour halos).
 *   stream cudaStream_t (NULL = legacy default stream); the call only
 *          enqueues work and returns.
 * Errors: INVALID_ARG (NULL pointers, sizes <= 0, pitch < width, overlap,
 * parameters out of range), UNSUPPORTED (a support or block size not listed at
 * fsr_params.border, a tensor-core mode with S < 32, FSR_UPDATE_CONJ_PAIR
 * outside S = 32, B = 4, FSR_FP32 / FSR_FP64_DEBUG, reuse > 0 outside S = 32,
 * FSR_UPDATE_SINGLE, FSR_FP32 / FSR_FP64_DEBUG),
 * CUDA (launch failure). */
int fsr_reconstruct(fsr_handle *h, const float *img, const uint8_t *mask,
                    int height, int width, int pitch, const fsr_params *p,
                    float *out, void *stream);

/* Same as fsr_reconstruct with HOST buffers (tightly packed when pitch ==
 * width): copies img and mask to handle-owned device buffers, reconstructs,
 * copies the result back into host `out` and synchronises `stream` before
 * returning.  Pinned host memory gives full copy bandwidth; pageable memory
 * works but is slower.  p->seq_out, if set, must still be a device buffer.
 * Errors: as fsr_reconstruct, plus OOM when the device buffers cannot be
 * allocated within the handle's workspace cap. */
int fsr_reconstruct_host(fsr_handle *h, const float *img, const uint8_t *mask,
                         int height, int width, int pitch, const fsr_params *p,
                         float *out, void *stream);

/* Support tiles (step a1 of every block, Sec. III-A, Eq. 13): when img and
 * mask are 16-byte aligned and pitch is a multiple of 16, the single-image
 * kernels bring each block's 32 x 32 support in by two TMA tile copies (the
 * image and the mask), with pixels outside the image filled as unknown;
 * otherwise by plain loads.  Both give identical results.  A warp waits for
 * its copies with a bounded wait (about one second); when the wait gives up,
 * the warp sets a bit in the handle's device status word and takes no more
 * blocks (their output pixels are left unwritten).
 *
 * fsr_check_status synchronises `stream`, then reads and clears the status
 * word: FSR_OK, or FSR_ERR_TIMEOUT with a message when a wait gave up in any
 * single-image launch on h since the last check.  fsr_reconstruct_host does
 * this check itself.  Errors: INVALID_ARG (h NULL), CUDA. */
int fsr_check_status(fsr_handle *h, void *stream);

/* Test hook (no counterpart in the paper): the next single-image launch on h
 * that uses tile copies expects 16 bytes more per block than its copies
 * deliver, so every wait runs out and the launch ends with FSR_ERR_TIMEOUT
 * from fsr_check_status.  No GPU fault is involved: the copies complete, only
 * the barrier's phase does not.  Launches after it are unaffected.
 * Errors: INVALID_ARG (h NULL). */
int fsr_inject_tile_wait_fault(fsr_handle *h);

/* Blocks without any known pixel in their support (W[0][0] = 0: no
 * iterations, g = 0, unknown target pixels written as 0; Sec. II, Eq. 10).
 * The single-image and batch entry points of h count them on the device;
 * this call synchronises `stream`, stores the count since the previous call
 * in *count and resets it.  (fsr_server and fsr_reconstruct_batch_static do
 * not count.)  Errors: INVALID_ARG (NULL h or count), CUDA. */
int fsr_empty_blocks(fsr_handle *h, void *stream, long long *count);

/* Number of target blocks N = ceil(height/B) * ceil(width/B) (Eq. 13);
 * 0 for invalid sizes. */
long long fsr_num_blocks(int height, int width, int block);

/* ---- Batch form: many images in one persistent launch ------------------
 * The blocks of all images form one work list, images ordered by decreasing
 * K (the long blocks start first); every warp of a persistent grid takes
 * `chunk` entries at a time from a device counter.  Each block is computed by
 * one warp with the same arithmetic as fsr_reconstruct, so results do not
 * depend on the schedule and equal the single-image results bit for bit. */

/* One image of a batch.  Pointer and geometry rules as in fsr_reconstruct. */
typedef struct fsr_image_desc {
    const float *img;    /* DEVICE float32, height x width, row pitch `pitch` elements */
    const uint8_t *mask; /* DEVICE uint8, same geometry; nonzero = known */
    float *out;          /* DEVICE float32, same geometry; may not overlap img or mask */
    int height, width, pitch;
    int iters;           /* K of this image, 0 <= K <= 65535 */
    int16_t *seq_out;    /* optional DEVICE buffer of N_i*K_i selected indices, or NULL */
} fsr_image_desc;

/* Schedule of the persistent batch launch. */
typedef struct fsr_schedule {
    int warps;   /* warps per CTA = support blocks in flight per CTA (FP32: 8, or 12/16 for B = 4; FP64: 4) */
    int chunk;   /* blocks a warp takes per counter increment, 1..64 */
} fsr_schedule;

typedef struct fsr_batch fsr_batch;

/* Reconstruct n >= 1 images in one launch, asynchronously on `stream`.
 * p supplies B, L, rho, gamma, freq_weight and precision; p->iters and
 * p->seq_out are ignored (per image in d).  The work table lives in
 * handle-owned device memory: a call waits on the host until the previous
 * fsr_reconstruct_batch of this handle has finished before reusing it.
 * With p->reuse > 0 the images run in the re-use form instead: one launch per
 * wavefront index t holds wavefront t of every image that has one (up to 48
 * images per launch), no work table; each image's output equals its
 * single-image fsr_reconstruct bit for bit.
 * Errors: as fsr_reconstruct, for every image; OOM for the table. */
int fsr_reconstruct_batch(fsr_handle *h, int n, const fsr_image_desc *d, const fsr_params *p, void *stream);

/* Prepare a reusable batch: validates the images, uploads the work table to
 * device memory owned by the batch and captures the launch (counter reset +
 * kernel) in a CUDA graph, with the handle's current schedule.  The image
 * buffers must stay valid while the batch is used.  Synchronous.
 * UNSUPPORTED for p->reuse > 0 (plans run independent blocks). */
int fsr_batch_create(fsr_handle *h, int n, const fsr_image_desc *d, const fsr_params *p, fsr_batch **out);

/* Replay the captured launch on `stream` (asynchronous).  Launches of one
 * batch share its work counter: do not let two of them overlap on the device
 * (launch them on one stream, or wait in between). */
int fsr_batch_launch(fsr_batch *b, void *stream);

/* Release a batch (waits for nothing; no launch of it may be in flight). */
int fsr_batch_destroy(fsr_batch *b);

/* Time every instantiated schedule (warps x chunk in {1, 2, 4, 8}) on this
 * batch (its outputs are written), keep the fastest for (p->block,
 * p->precision) in the handle and, if the handle has a schedule cache path,
 * store it there.  best / best_ms may be NULL.  Synchronous.  The outputs of
 * every schedule are identical, so the choice only affects time.
 * UNSUPPORTED for p->reuse > 0. */
int fsr_autotune_batch(fsr_handle *h, int n, const fsr_image_desc *d, const fsr_params *p,
                       fsr_schedule *best, float *best_ms);

/* Read or set the batch schedule used for (block, precision).
 * Errors: INVALID_ARG, UNSUPPORTED (schedule not instantiated). */
int fsr_get_schedule(const fsr_handle *h, int block, int precision, fsr_schedule *out);
int fsr_set_schedule(fsr_handle *h, int block, int precision, const fsr_schedule *s);

/* ---- Serving form: continuous batching of a request stream --------------
 * A server owns a device-memory pool of a fixed budget and a worker thread.
 * fsr_server_submit queues a request (HOST buffers) and returns at once.  The
 * worker admits queued requests in arrival order while the pool has room for
 * their image, mask and output and a slot is free, starts their host-to-device
 * copies, and launches the admitted, not yet launched requests as batches
 * (fsr_reconstruct_batch's kernel): requests of at most 1920 x 1088 pixels
 * together on the first compute stream, which has the highest stream
 * priority, larger ones together on the other streams (with one stream,
 * everything on it).  Requests that arrive while others run join the next launch, and
 * launches, copies in and copies out of different requests overlap on the
 * device.  With S = 32 the server's launches run short-lived CTAs (each warp
 * takes one chunk of blocks), so the blocks of a launch of small
 * requests start as soon as CTAs of a running launch of large ones finish.  A finished request's output is copied back to its host buffer, its
 * pool memory is released, and its latency (submit to output on the host) is
 * recorded.  Results do not depend on what else is in flight: every block is
 * computed by one warp with the arithmetic of fsr_reconstruct. */

typedef struct fsr_server fsr_server;

typedef struct fsr_server_config {
    size_t pool_bytes;   /* device-memory budget of in-flight requests (image, mask,
                            output and launch tables), allocated once at creation */
    int max_inflight;    /* admitted requests at most (slots), >= 1 */
    int streams;         /* compute streams launches rotate over, 1..8 */
} fsr_server_config;

/* Create a server on the handle's device; p gives B, L, rho, gamma,
 * freq_weight and precision for every request (p->iters, p->seq_out ignored).
 * Errors: INVALID_ARG, OOM (the pool cannot be allocated), CUDA. */
int fsr_server_create(fsr_handle *h, const fsr_server_config *cfg, const fsr_params *p, fsr_server **out);

/* Queue one request.  img/mask/out are HOST buffers, tightly packed
 * (pitch = width), owned by the caller and left untouched by the caller until
 * the request completes (pinned memory lets the copies overlap compute).
 * *ticket receives the request's id (0, 1, 2, ... in submission order).
 * Errors: INVALID_ARG (bad sizes, or a request larger than the whole pool). */
int fsr_server_submit(fsr_server *s, const float *img, const uint8_t *mask, int height, int width, int iters,
                      float *out, long long *ticket);

/* Completed requests since the last call, in completion order: up to `max`
 * tickets and their latencies in milliseconds; *n receives the count.
 * With wait_ms > 0 the call blocks up to that long for at least one.
 * A request whose device work failed is reported with latency -1. */
int fsr_server_poll(fsr_server *s, long long *tickets, double *latency_ms, int max, int *n, int wait_ms);

/* Counters: submitted, completed, requests currently queued and admitted,
 * launches issued, peak pool bytes in use.  Any pointer may be NULL. */
int fsr_server_stats(const fsr_server *s, long long *submitted, long long *completed, int *queued,
                     int *inflight, long long *launches, size_t *peak_pool_bytes);

/* Stop accepting work, finish everything admitted or queued, release the
 * pool and streams.  NULL is accepted. */
int fsr_server_destroy(fsr_server *s);

/* ---- Batch form without device allocation -------------------------------
 * The paper has no counterpart of this entry point: it exists for callers
 * that may not allocate device memory, e.g. code running under a framework
 * whose allocator owns the whole device-memory budget, real-time loops that
 * cannot afford an allocation (cudaMalloc may synchronise the device and stall
 * other streams), or plug-ins that may not keep device memory between calls.
 *
 * Same work as fsr_reconstruct_batch on the calling thread's current device,
 * with the default schedule, but with no handle and no allocation: the work
 * table (counter, block prefix sums, per-image arguments) lives in a fixed
 * FSR_STATIC_SCRATCH_BYTES array of the library's static device memory, which
 * every device that loads the library holds until the process exits.
 *   - At most FSR_STATIC_MAX_IMAGES images per call; larger batches are
 *     rejected with FSR_ERR_INVALID_ARG and a message.
 *   - The first call on a device does a one-time set-up there (finds the
 *     array's device address, sets the kernels' shared-memory limits); make
 *     that first call before any stream capture.  The set-up is kept for the
 *     life of the process: do not use this entry point on a device after
 *     cudaDeviceReset.
 *   - Every call shares the one array per device and overwrites it (the work
 *     counter is reset by each call's table copy): calls whose work overlaps
 *     on the device race and give wrong results.  Keep them on one stream, or
 *     wait for one to finish before the next starts.
 *   - The table goes to the device in the launch parameters of a small copy
 *     kernel on `stream`, so no host memory is read after the call returns;
 *     the call is asynchronous on `stream`.
 *   - err/err_len: optional buffer for the text of an error (may be NULL).
 * Errors: INVALID_ARG, UNSUPPORTED (also for a device ordinal >= 64), CUDA,
 * as for fsr_reconstruct_batch. */
#define FSR_STATIC_MAX_IMAGES 64
#define FSR_STATIC_SCRATCH_BYTES 8192
int fsr_reconstruct_batch_static(int n, const fsr_image_desc *d, const fsr_params *p, void *stream,
                                 char *err, size_t err_len);

#ifdef __cplusplus
}
#endif
#endif /* FSR_GB300_H */
