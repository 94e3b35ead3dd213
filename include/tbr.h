/*
 * tbr.h -- C ABI of the B300-native transport-based renderer (TBR, capsule
 * deposition strokes).
 *
 * The library renders an ordered program of capsule strokes by pulling each
 * pixel back through the closed-form inverse exterior transport of every later
 * stroke (Sec. 3, Eq. chain and Eq. render; Sec. 4, Eq. back), and
 * differentiates the soft render with the replay adjoint of Sec. 5.2 (Eq. rpos,
 * Eq. rT, Eq. adjstep, Eq. adjparam): exterior states are regenerated with the
 * forward map (Eq. fwd) and only the samples the epsilon-floor touched are read
 * from a side table.
 *
 * Conventions shared by every entry point
 *   - Program order: stroke 0 is executed first (the paper's g_1); rendering
 *     visits strokes n-1 down to 0.
 *   - A stroke is (cx, cy, theta, length, half_width): the segment
 *     [m - L e/2, m + L e/2] with m = (cx, cy), e = (cos theta, sin theta),
 *     L = length >= 0 (0 is a drop) and r = half_width > 0 (Sec. 3).
 *   - Colour c_i = softmax(logits_i / color_temp) . palette (Sec. 5.1); the hard
 *     render can snap to the palette entry of the largest logit.
 *   - The canvas is [0,1]^2; pixel (row, col) is sampled once at
 *     ((col + 0.5)/W, (row + 0.5)/H).  Images are row-major [H][W][3] float32
 *     (RGB interleaved); index maps are [H][W] int32.
 *   - Unless stated otherwise every pointer is a DEVICE pointer owned by the
 *     caller; the library never frees it.  Opaque handles (tbr_ctx, tbr_fit,
 *     tbr_server) are owned by the library and released by their *_destroy.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls enqueue
 *     work and return without synchronising unless their comment says so.
 *   - Errors: every call returns a tbr_status; tbr_last_error() gives a
 *     thread-local message for the last failure.  Argument checks that need
 *     only host data (sizes, NULL pointers) fail synchronously.  Value checks
 *     that need device data (r <= 0, L < 0, non-finite parameters) run in the
 *     packing kernel; a program that fails them renders NaN and the failure is
 *     reported by the next synchronising call (tbr_ctx_status, tbr_fit_step,
 *     a call given a stats pointer) as TBR_ERR_INVALID_ARG.
 */
#ifndef TBR_H_
#define TBR_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TBR_API __attribute__((visibility("default")))
#else
#define TBR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TBR_OK = 0,
  TBR_ERR_INVALID_ARG = 1,  /* bad size, NULL pointer, or bad parameter value */
  TBR_ERR_OOM = 2,          /* device allocation failed */
  TBR_ERR_CUDA = 3,         /* a CUDA runtime call failed (message has the detail) */
  TBR_ERR_TIMEOUT = 4,      /* a bounded device wait gave up (status word set) */
  TBR_ERR_ADMISSION = 5,    /* serving: request refused by the memory cap */
  TBR_ERR_OVERFLOW = 6,     /* side table overflowed its per-pixel capacity */
  TBR_ERR_NOT_FOUND = 7     /* serving: unknown program or request id */
} tbr_status;

/* A stroke program (Sec. 3 problem statement, re-expressed as centre,
 * direction, length, half-width and palette logits).  Device pointers, fp32,
 * arrays of length n in program order unless noted. */
typedef struct {
  int32_t n;                /* number of strokes N >= 0 */
  int32_t k;                /* palette size K >= 1 */
  const float* cx;          /* segment centre x, canvas units */
  const float* cy;          /* segment centre y */
  const float* theta;       /* direction angle (radians) */
  const float* length;      /* full segment length L >= 0 */
  const float* half_width;  /* r > 0 */
  const float* logits;      /* [n][k] palette-assignment logits */
  const float* palette;     /* [k][3] sRGB colours */
  float background[3];      /* c_0, host value */
  float color_temp;         /* softmax temperature tau_c > 0, host value */
  const float* coupling;    /* [n][3] c_1..c_3 of the coupling variant's profile
                               g(v) = 1 + sum_k c_k cos(4 pi k v) (Sec. "A variant
                               closer to line-source potential flow", Eq. coupling,
                               Eq. profile), or NULL for the capsule map (g = 1).
                               Each stroke's g must be positive on the whole leaf
                               (checked exactly; else the stroke fails the value
                               checks).  Supported by the hard render, the soft
                               render (capsule transport, not inert) with or
                               without a replay context, its replay adjoint
                               (tbr_render_backward; local Jacobians by dual
                               numbers, no FP64 repair), the loss-fused call and
                               the fit (which keeps the profile fixed); the
                               serving and compensation entry points reject a
                               non-NULL coupling. */
} tbr_program;

/* Transport of a render: the paper's capsule insertion map psi (Eq. back), or
 * the sixteen-drop operator psi_D of the transfer renderer R_D (Sec. "Transfer
 * across transport constructions"): stroke i's displacement is the
 * composition of 16 classical drop maps of radius s = sqrt(A_L(r) / (16 pi))
 * centred at the midpoints of 16 equal sub-segments, inserted in one sweep from
 * the segment's start; coverage and membership stay the capsule's.  Inside a
 * drop's disc the pull-back is floored on the same ray at 1e-3 s (the
 * epsilon-floor of Sec. 5.2 applied per drop). */
enum { TBR_TRANSPORT_CAPSULE = 0, TBR_TRANSPORT_DROPS16 = 1 };

/* Statistics of one hard render (host struct). */
typedef struct {
  int64_t band_steps;       /* pixel-stroke steps whose |sigma' - r| fell in the
                               FP64 band and were recomputed in FP64 */
  int64_t background_pixels;/* pixels that left every footprint */
  int64_t visited_steps;    /* pixel-stroke steps executed (early exit) */
} tbr_hard_stats;

/* Hard render (Sec. 3, Eq. chain and Eq. render with alpha = 1 on the closed
 * footprint K_i): each pixel is pulled back through psi_i (Eq. back) of the
 * strokes from n_prefix-1 down to 0 until it lands inside a footprint
 * (sigma' <= r, the tie counts as inside) and takes that stroke's colour, else
 * the background.  Steps with |sigma' - r| < 1e-4 decide membership and apply
 * psi in FP64 from the FP32 position.
 *   n_prefix   number of leading strokes to replay (-1 = all; Sec. 7 prefix
 *              replay)
 *   snap       0: softmax colour; 1: palette entry of the largest logit
 *   out_rgb    [H][W][3] output
 *   out_idx    [H][W] terminating stroke index or -1, or NULL
 *   stats      host pointer or NULL; when non-NULL the call synchronises the
 *              stream and reports device-side argument errors.
 * Scratch: the packed strokes (128 B per stroke) and counters are allocated
 * stream-ordered from the device's default memory pool and freed on return. */
TBR_API tbr_status tbr_render_hard(const tbr_program* prog, int32_t W, int32_t H, int32_t n_prefix,
                           int32_t snap, float* out_rgb, int32_t* out_idx,
                           tbr_hard_stats* stats, void* stream);

/* tbr_render_hard with a choice of transport (TBR_TRANSPORT_*): with
 * TBR_TRANSPORT_DROPS16 each pixel that is outside K_i is pulled back through
 * the sixteen drops instead of psi_i (membership in FP64 within the band, the
 * drops in FP32).  Otherwise identical to tbr_render_hard. */
TBR_API tbr_status tbr_render_hard_transport(const tbr_program* prog, int32_t W, int32_t H, int32_t n_prefix,
                                             int32_t snap, int32_t transport, float* out_rgb, int32_t* out_idx,
                                             tbr_hard_stats* stats, void* stream);

/* One-pass closed-form compensation (Sec. "Closed-form compensation
 * baseline"): returns a program whose hard render under the transport puts
 * each stroke where the given program's strokes would sit without transport.
 * From the last stroke to the first, the stroke's segment start (endpoint = 0,
 * the anchor variant: theta and length kept) or both segment ends
 * (endpoint = 1: centre, theta and length from the pre-imaged ends) are pulled
 * back through psi_j (Eq. back) of every later stroke j, already compensated,
 * last first.  A point inside K_j (sigma' <= r) has no pre-image: with
 * skip_blocked = 0 the step takes the ideal extension (sigma = 0: the point
 * goes onto the segment, a drop's disc onto its centre), with skip_blocked = 1
 * the step is skipped; either way the stroke is flagged as blocked.  Positions
 * are carried as float pairs; N (N - 1) / 2 point steps run on one CTA.
 *   out_cx, out_cy, out_theta, out_length  [n] device float32 outputs
 *   out_blocked                            [n] device int32, 1 = blocked
 *   n_blocked   host pointer or NULL; when non-NULL the call synchronises the
 *               stream, reports device-side value errors and returns the count.
 * half_width, logits and palette are unchanged and not returned. */
TBR_API tbr_status tbr_compensate(const tbr_program* prog, int32_t endpoint, int32_t skip_blocked,
                                  float* out_cx, float* out_cy, float* out_theta, float* out_length,
                                  int32_t* out_blocked, int64_t* n_blocked, void* stream);

/* Allocation-free hard render.  The paper has no counterpart: this entry
 * point exists for callers that may not allocate device memory at all (a
 * plugin hosted by another runtime that owns the device's memory budget, a
 * real-time loop that must never wait on an allocator, code that runs when
 * the memory pool is exhausted).  It renders exactly what tbr_render_hard
 * renders (same kernels, same arguments, no stats), but its scratch -- the
 * packed stroke records and the status words -- lives in one fixed device
 * array inside the library, sized for at most 8192 strokes (about 1 MiB,
 * held on every GPU that loads the library until the process exits).  The
 * caller still passes the program, out_rgb and out_idx.
 *   - Programs (or prefixes) longer than 8192 strokes are rejected with
 *     TBR_ERR_INVALID_ARG before anything is launched.
 *   - The first call on a device looks up the array's device address (once
 *     per device, with that device current); make that first call before any
 *     stream capture.
 *   - No cudaMalloc, cudaFree or other allocating routine is called.
 *   - Every call shares the one array, which keeps the last call's contents
 *     (the status words are cleared on each call).  Calls whose work overlaps
 *     on the GPU (for example on two streams at once) race on the array: run
 *     them one after another on a stream.
 *   - Parameter values that fail the device-side checks render NaN; there is
 *     no synchronising stats variant. */
TBR_API tbr_status tbr_render_hard_noalloc(const tbr_program* prog, int32_t W, int32_t H, int32_t n_prefix,
                                           int32_t snap, float* out_rgb, int32_t* out_idx, void* stream);

/* Options of the soft render / replay record. */
typedef struct {
  float tau;                /* relaxation width factor tau of Eq. relax */
  float tau_min;            /* floor tau_min of Eq. relax */
  int32_t checkpoint_every; /* k: store (x, log T) every k strokes (Sec. 5.2
                               conditioning); 0 = library default (32) */
  int32_t record_capacity;  /* side-table records per pixel; 0 = default (64) */
  int32_t inert;            /* 1: psi = id (inert-mark model, Definition 1) */
  float drift_tolerance;    /* FP32 regeneration drift at a checkpoint (canvas
                               units) above which the pixel's segment is
                               regenerated in FP64 by the adjoint (Sec. 5.2
                               conditioning); <= 0 = default (1e-5) */
  int32_t repair_capacity;  /* pixels the adjoint can repair per call, at most
                               1024; 0 = default (256).  Memory: 32 B x n per
                               pixel of capacity. */
  int32_t transport;        /* TBR_TRANSPORT_*; TBR_TRANSPORT_DROPS16 renders
                               forward only (no context, not inert) */
  float early_exit;         /* forward-only renders (no context): a pixel stops
                               once its transmittance T falls below this value
                               after compositing a stroke, and a CTA once all its
                               pixels have; the output is C + T c_0 with that T,
                               so the skipped strokes change each channel by at
                               most early_exit.  0 = off (every pixel visits all
                               N strokes); must be in [0, 1). */
} tbr_soft_opts;

typedef struct tbr_ctx tbr_ctx;

/* Soft render (Eq. relax coverage with alpha clamped at 1 - 1e-7, Eq. state
 * compositing, psi with the epsilon-floor C >= (1e-3 r)^2 of Sec. 5.2).
 *   out_rgb  [H][W][3]
 *   ctx      NULL: forward only.  Otherwise, if *ctx is NULL it receives a
 *            new handle that holds what the replay adjoint needs (Sec. 5.2):
 *            per pixel s_0 = (x_0, log T_0), position checkpoints every k
 *            strokes, and the side table of (i, x_i) for every sample the floor
 *            touched.  If *ctx is an existing handle of the same n, k, W, H,
 *            interval, capacity and inert flag, it is overwritten in place
 *            (no allocation).  The program arrays are packed into the handle,
 *            so the caller may change them once this call's work has run.
 * Memory: 16 B/pixel (s_0) + 16 B/pixel per checkpoint + 16 B/pixel per record
 * slot, allocated stream-ordered. */
TBR_API tbr_status tbr_render_soft(const tbr_program* prog, int32_t W, int32_t H,
                           const tbr_soft_opts* opts, float* out_rgb, tbr_ctx** ctx,
                           void* stream);

/* Replay adjoint (Sec. 5.2): for i = 1..N regenerate x_i = Phi_i(x_{i-1})
 * (Eq. rpos), or pop it from the side table, or reset it from a checkpoint;
 * regenerate log T_i (Eq. rT); take the adjoint step (Eq. adjstep) and
 * accumulate the parameter gradients (Eq. adjparam) of
 * J = sum_pixels dL_drgb . R.  A pixel whose FP32 regeneration drifts past the
 * drift tolerance at a checkpoint is replayed again from the start of that
 * segment with its positions regenerated in FP64, and its gradient
 * contributions from there on are replaced (counted in repaired_pixels).
 *   dL_drgb   [H][W][3] cotangent of the rendered image
 *   g_*       [n] gradients w.r.t. cx, cy, theta, length, half_width (written)
 *   g_logits  [n][k] (written)
 *   g_palette [k][3] or NULL (written)
 * The sums over pixels are reduced per CTA in fixed order and then across CTAs
 * in fixed order, so results are bitwise reproducible for a given size. */
TBR_API tbr_status tbr_render_backward(tbr_ctx* ctx, const float* dL_drgb, float* g_cx, float* g_cy,
                               float* g_theta, float* g_length, float* g_half_width,
                               float* g_logits, float* g_palette, void* stream);

/* Counters of a context (host struct). */
struct tbr_ctx_stats {
  int64_t records;          /* side-table records written */
  int64_t max_records;      /* largest per-pixel record count */
  int64_t overflow_pixels;  /* pixels whose records exceeded the capacity */
  int64_t drift_resets;     /* checkpoint resets where the regenerated position
                               differed from the stored one by more than the
                               drift tolerance */
  int64_t timeouts;         /* bounded waits that gave up */
  int64_t invalid_params;   /* strokes that failed the value checks */
  int64_t repaired_pixels;  /* pixels whose drifting segment (and the rest of
                               their replay) the adjoint regenerated in FP64 */
  int64_t repair_overflow;  /* drifting pixels when they outnumbered the repair
                               capacity (then none is repaired) */
};
typedef struct tbr_ctx_stats tbr_ctx_stats;

/* Synchronises the context's last stream and reads its counters.  Returns
 * TBR_ERR_OVERFLOW, TBR_ERR_TIMEOUT or TBR_ERR_INVALID_ARG if the matching
 * counter is non-zero (the gradients of such a context are NaN). */
TBR_API tbr_status tbr_ctx_status(tbr_ctx* ctx, tbr_ctx_stats* stats);

/* Device bytes held by a context. */
TBR_API size_t tbr_ctx_bytes(const tbr_ctx* ctx);

/* Releases a context (stream-ordered on the stream it was created on). */
TBR_API void tbr_ctx_destroy(tbr_ctx* ctx);

/* Pixel mean-squared error on sRGB values (Sec. 5.1 "Objective and
 * metrics"): loss = mean over the 3*H*W values of (rgb - target)^2, written to
 * loss_out[0] (device, fp32; the sum is carried in fp64), and
 * dL_drgb = 2 (rgb - target) / (3 H W) (device, may be NULL).  Scratch: one
 * fp64 partial per block, stream-ordered. */
TBR_API tbr_status tbr_loss_mse(const float* rgb, const float* target, int64_t n_pixels,
                        float* loss_out, float* dL_drgb, void* stream);

/* Loss-fused soft forward + replay adjoint for the pixel MSE (Sec. 5.1
 * objective; Sec. 5.2 adjoint): the seed lambda^C_0 = 2 (R - target) / (3HW) is
 * pixel-local, so each 32x8 tile runs its soft forward with the replay record
 * in per-CTA scratch (L2-resident), seeds, and runs the replay adjoint at once;
 * no full-image side table or checkpoint array is written.  Same gradients as
 * tbr_render_soft + tbr_loss_mse + tbr_render_backward (to rounding).
 *   target    [H][W][3]
 *   out_rgb   [H][W][3] soft render, or NULL
 *   loss_out  device scalar (MSE, FP64 sums) or NULL
 *   g_*       as tbr_render_backward (written)
 *   stats     host, or NULL; when non-NULL the call synchronises and reports
 *             overflow / invalid values / timeouts as errors.
 * opts->inert must be 0.  Scratch (packed strokes, per-CTA record, gradient
 * slices) is allocated stream-ordered and released on return. */
TBR_API tbr_status tbr_render_soft_adjoint_mse(const tbr_program* prog, int32_t W, int32_t H,
                                               const tbr_soft_opts* opts, const float* target, float* out_rgb,
                                               float* loss_out, float* g_cx, float* g_cy, float* g_theta,
                                               float* g_length, float* g_half_width, float* g_logits,
                                               float* g_palette, tbr_ctx_stats* stats, void* stream);

/* ------------------------------------------------------------------------
 * Fit (Sec. 5.1 "Parameterisation and relaxation", Eq. inverse, Table hyper):
 * Adam on (cx, cy, theta, length, half_width, logits [, palette]) against a
 * target image, loss = pixel MSE (Sec. 5.1 "Objective and metrics") +
 * length_weight * sum_i L_i.  Each step renders the soft image at the
 * annealed relaxation tau_t (geometric tau_start -> tau_end) and colour
 * temperature (geometric color_temp_start -> color_temp_end), runs the replay
 * adjoint, and applies Adam with cosine-decayed step sizes, then projects:
 * centres into [0,1]^2, 0 <= L <= length_max, r into [width_lo r0, width_hi r0]
 * with r0 the initial half-width of each stroke, palette into [0,1].
 * ------------------------------------------------------------------------ */
typedef struct {
  int32_t iterations;                   /* schedule length T (Table hyper: 240) */
  float tau_start, tau_end;             /* relaxation schedule (0.35 -> 0.02) */
  float tau_min;                        /* 0 = 0.7 / max(W, H) (Table hyper) */
  float color_temp_start, color_temp_end;  /* 1.0 -> 0.05 */
  float lr_center, lr_angle, lr_length, lr_width, lr_logits, lr_palette;
  float beta1, beta2, adam_eps;         /* Adam (0.9, 0.999, 1e-8) */
  float length_max;                     /* L_max (Table hyper: 0.30) */
  float width_lo, width_hi;             /* half-width window factors (0.6, 1.7) */
  float length_weight;                  /* lambda of the length regulariser (3e-4) */
  int32_t train_palette;                /* 1: the palette is optimised too */
  int32_t checkpoint_every;             /* replay checkpoint interval (0 = 32) */
  int32_t record_capacity;              /* initial side-table capacity (0 = 64);
                                           doubled and the step redone on overflow */
} tbr_fit_config;

typedef struct tbr_fit tbr_fit;

/* Fills the defaults listed above. */
TBR_API void tbr_fit_default_config(tbr_fit_config* cfg);

/* Creates a fit: copies the initial program and the [H][W][3] target into
 * library-owned device memory (stream-ordered).  cfg may be NULL (defaults). */
TBR_API tbr_status tbr_fit_create(const tbr_program* init, const float* target, int32_t W, int32_t H,
                                  const tbr_fit_config* cfg, tbr_fit** fit, void* stream);

/* One optimisation step (forward, loss, replay adjoint, update).  Synchronises
 * the stream once to read the loss and the context status; loss_out (host,
 * nullable) receives the loss of the parameters before the update. */
TBR_API tbr_status tbr_fit_step(tbr_fit* fit, float* loss_out, void* stream);

/* A view of the current program (device pointers into the fit; valid until the
 * next step or destroy).  color_temp is the current schedule value. */
TBR_API tbr_status tbr_fit_get_program(const tbr_fit* fit, tbr_program* view);

/* Number of completed steps. */
TBR_API int32_t tbr_fit_iteration(const tbr_fit* fit);

/* Releases the fit. */
TBR_API void tbr_fit_destroy(tbr_fit* fit);

/* ------------------------------------------------------------------------
 * Serving (continuous batching).  Programs are loaded once and stay resident
 * on the device.  Requests -- hard re-renders, soft render + adjoint against a
 * target, and edit re-renders (recolour, reorder, stroke insert; Sec. 7
 * "program edits", prefix replay via n_prefix) -- are admitted in arrival order
 * as request slots and the memory cap allow, and their work (32x8 hard tiles,
 * or groups of soft tiles fused with the MSE seed and the replay adjoint) is
 * claimed item by item by one persistent kernel, so requests that arrive while
 * others run are batched into the same launch.  Each result is bitwise the same
 * whether the request runs alone or in a mix (per-tile / per-group reductions
 * in a fixed order).  A library worker thread does admission and completion;
 * the persistent kernel exits after idle_exit_us without work and is relaunched
 * when work arrives.  Output buffers are caller-owned device memory and must
 * stay valid until the request is done.
 * ------------------------------------------------------------------------ */
typedef struct {
  size_t memory_cap_bytes;   /* admission cap on request working memory (80 GiB) */
  int32_t max_inflight;      /* admitted requests at a time (64, at most 1024) */
  int32_t max_strokes;       /* largest program + 1 (8192); sizes the per-CTA record */
  int32_t checkpoint_every;  /* soft requests: checkpoint interval (64) */
  int32_t record_capacity;   /* soft requests: side-table records per pixel (64) */
  int32_t idle_exit_us;      /* persistent kernel idle exit (2000 us) */
  int32_t ready_wait_us;     /* longest device wait for a request's ready word (1000000 us), see tbr_request */
} tbr_serve_config;

enum {
  TBR_REQ_HARD = 0,          /* hard render (n_prefix, snap apply) */
  TBR_REQ_SOFT_ADJOINT = 1,  /* soft render + MSE vs target + replay adjoint */
  TBR_REQ_RECOLOUR = 2,      /* swap palette entries edit_a, edit_b for strokes >= edit_start, hard render */
  TBR_REQ_REORDER = 3,       /* reverse strokes [edit_start, edit_start + edit_b), hard render */
  TBR_REQ_INSERT = 4         /* insert insert_stroke before index edit_start, hard render */
};

typedef struct {
  int32_t kind;              /* TBR_REQ_* */
  uint64_t program;          /* id from tbr_serve_load_program */
  int32_t W, H;
  int32_t n_prefix;          /* reserved (use -1) */
  int32_t snap;              /* hard kinds: palette snapping */
  float tau, tau_min;        /* soft: relaxation (Eq. relax) */
  const float* target;       /* soft: [H][W][3] */
  float* out_rgb;            /* [H][W][3] (soft: optional) */
  int32_t* out_idx;          /* hard kinds: [H][W] or NULL */
  float* out_loss;           /* soft: device scalar (MSE) or NULL */
  float* out_grad;           /* soft: [5n + n k]: cx, cy, theta, length, half_width (n each), logits */
  int32_t edit_a, edit_b;    /* recolour: palette entries; reorder: edit_b = window length */
  int32_t edit_start;        /* first stroke affected / insertion index */
  int32_t insert_palette;    /* insert: palette entry of the new stroke (logits 6 * onehot) */
  float insert_stroke[5];    /* insert: cx, cy, theta, length, half_width */
  /* Optional (NULL: none): a word in device or host-mapped memory that the
   * request's producer sets to nonzero once the inputs (target) and the output
   * buffers may be used, for producers outside the stream order of `stream`
   * (another process, a host thread, a copy engine the caller drives).  Each of
   * the request's work items waits for it on the device, at most
   * ready_wait_us; if the wait runs out the request completes without
   * rendering (a hard request leaves its outputs untouched, a soft request
   * writes NaN loss and gradients) and tbr_serve_poll / tbr_serve_wait report
   * TBR_ERR_TIMEOUT.  The server stays usable. */
  const volatile int32_t* ready;
} tbr_request;

typedef struct {
  int64_t admitted, completed, refused, queued, inflight, kernel_launches;
  int64_t bytes_in_use;      /* request working memory in use */
  int64_t fixed_bytes;       /* per-CTA replay scratch held by the server */
  int32_t persistent_ctas;
} tbr_serve_counters;

typedef struct tbr_server tbr_server;

TBR_API void tbr_serve_default_config(tbr_serve_config* cfg);
/* Creates a server on the current device (cfg may be NULL for the defaults). */
TBR_API tbr_status tbr_serve_create(const tbr_serve_config* cfg, tbr_server** server);
/* Copies a program into server memory (synchronous); *id names it in requests. */
TBR_API tbr_status tbr_serve_load_program(tbr_server* server, const tbr_program* prog, uint64_t* id);
/* Queues a request; returns at once.  `stream` is the caller's stream on which
 * the request's inputs (target, and anything written to the output buffers
 * before) were produced: the request's device work starts after everything
 * enqueued there so far.  After tbr_serve_wait / tbr_serve_poll report it
 * done, the outputs are visible to any work launched afterwards.
 * TBR_ERR_ADMISSION if the request could never fit the memory cap. */
TBR_API tbr_status tbr_serve_submit(tbr_server* server, const tbr_request* req, uint64_t* req_id, void* stream);
/* *done = 1 once the request's outputs are written; *result is its status. */
TBR_API tbr_status tbr_serve_poll(tbr_server* server, uint64_t req_id, int32_t* done, tbr_status* result);
/* Blocks until the request is done (timeout_ms < 0: no limit). */
TBR_API tbr_status tbr_serve_wait(tbr_server* server, uint64_t req_id, int32_t timeout_ms, tbr_status* result);
/* Host-clock times of a finished request: queueing (submit to admission) and
 * latency (submit to completion), in milliseconds. */
TBR_API tbr_status tbr_serve_request_times(tbr_server* server, uint64_t req_id, double* queue_ms,
                                           double* latency_ms);
/* Forgets a finished request. */
TBR_API tbr_status tbr_serve_release(tbr_server* server, uint64_t req_id);
TBR_API tbr_status tbr_serve_stats(tbr_server* server, tbr_serve_counters* stats);
/* Stops the worker and the persistent kernel and frees everything. */
TBR_API void tbr_serve_destroy(tbr_server* server);

/* ------------------------------------------------------------------------
 * Per-kernel timing without a profiler: while enabled, each launch of the
 * library's kernels is bracketed by CUDA events on its launch stream.
 * tbr_profile_read synchronises the pending events and returns the launch
 * count and summed device time of one kernel since the last reset.
 * ------------------------------------------------------------------------ */
enum {
  TBR_K_PACK = 0,        /* stroke packing */
  TBR_K_HARD = 1,        /* hard render */
  TBR_K_SOFT = 2,        /* soft forward (+ replay record) */
  TBR_K_BACKWARD = 3,    /* replay adjoint */
  TBR_K_EPILOGUE = 4,    /* gradient sums and colour chain rule */
  TBR_K_LOSS = 5,        /* MSE and adjoint seed */
  TBR_K_UPDATE = 6,      /* Adam update */
  TBR_K_SERVE = 7,       /* persistent serving kernel */
  TBR_K_COMPENSATE = 8,  /* one-pass closed-form compensation */
  TBR_K_COUNT = 9
};
typedef struct {
  int64_t launches;
  double total_ms;
} tbr_kernel_time;
TBR_API tbr_status tbr_profile_enable(int32_t on);
TBR_API tbr_status tbr_profile_read(int32_t kernel, tbr_kernel_time* out);
TBR_API void tbr_profile_reset(void);

/* ------------------------------------------------------------------------
 * Arithmetic peaks, measured (the denominators of the ALU roofline; no file
 * the driver writes gives an FP32 or MUFU rate).  Runs one warm-up and one
 * timed launch of a chain microbenchmark on every SM (4 CTAs of 256 threads
 * per SM, 8 independent chains per thread, iters iterations) on `stream` and
 * synchronises it.  *rate is in operations per second: FLOPs for the FMA kinds
 * (a fused multiply-add counts 2, per lane), results for the MUFU kinds;
 * *elapsed_ms (nullable) is the timed launch's duration.  TBR_ERR_INVALID_ARG
 * for an unknown kind, iters <= 0 or a NULL rate.
 * ------------------------------------------------------------------------ */
enum {
  TBR_PEAK_FFMA2 = 0,  /* packed FP32 fused multiply-add (FFMA2) */
  TBR_PEAK_FFMA = 1,   /* scalar FP32 fused multiply-add */
  TBR_PEAK_EX2 = 2,    /* MUFU ex2.approx */
  TBR_PEAK_RCP = 3     /* MUFU rcp.approx */
};
TBR_API tbr_status tbr_measure_peak(int32_t kind, int32_t iters, double* rate, double* elapsed_ms, void* stream);

/* Thread-local description of the last error (never NULL). */
TBR_API const char* tbr_last_error(void);

/* Library version string. */
TBR_API const char* tbr_version(void);

#ifdef __cplusplus
}
#endif

#endif  /* TBR_H_ */
