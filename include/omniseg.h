/*
 * omniseg.h -- C ABI of the GB300 (sm_103a) Omni-Seg slide-wise inference library.
 *
 * The method is the three-stage whole-slide pipeline of Leng, Deng et al.,
 * "An Accelerated Pipeline for Multi-label Renal Pathology Image Segmentation
 * at the Whole Slide Image Level":
 *   Sec. 2.1  tissue detection and tile extraction  -> omni_tile_slide
 *   Sec. 2.2  Omni-Seg segmentation of overlapping 40x/10x/5x tiles
 *   Sec. 2.3  slide-wise aggregation into per-class label maps
 *                                                    -> omni_segment_slide
 *             and the stained 40x product with its 10x resize -> omni_stain
 * plus a hand-written backward of the stitched soft-Dice + BCE loss through
 * the dynamic head, controller, pre-head and last decoder block
 * (omni_backward).
 *
 * Conventions (every entry point):
 *   - Returns an omni_status; 0 is success, negative values are errors.  No
 *     entry point aborts, asserts or traps; on error, omni_last_error(ctx)
 *     returns a one-line description and nothing has been launched unless the
 *     error is OMNI_ECUDA / OMNI_ETIMEOUT.
 *   - Pointers named *_dev are CUDA device pointers, *_host are host pointers.
 *     All inputs are borrowed (the caller keeps ownership, the library keeps
 *     no reference after the call returns).  All outputs are allocated by the
 *     caller, sized with omni_query.
 *   - Device work is enqueued on the caller's CUDA stream (`stream`, a
 *     cudaStream_t passed as void*, NULL = legacy default stream).  Calls that
 *     need a host-visible intermediate result (the foreground tile count)
 *     synchronise that stream once; this is stated per call.
 *   - Images are row-major interleaved RGB uint8 (HWC) with an explicit row
 *     stride in bytes.  Activations inside the library are NHWC.
 *   - A context is not thread safe; use one context per host thread/stream.
 */
#ifndef OMNISEG_H
#define OMNISEG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int omni_status;
#define OMNI_OK 0
#define OMNI_EINVAL (-1)    /* bad argument, shape or configuration          */
#define OMNI_ENOMEM (-2)    /* caller workspace smaller than omni_query says  */
#define OMNI_ECUDA (-3)     /* a CUDA runtime/driver call failed              */
#define OMNI_ETIMEOUT (-4)  /* a bounded device-side wait gave up             */
#define OMNI_EWEIGHTS (-5)  /* weights blob of the wrong size or non-finite   */
#define OMNI_ESTATE (-6)    /* call out of order (e.g. segment before weights) */

/* Arithmetic of the U-Net convolutions. */
#define OMNI_FP32 0  /* FP32 FFMA on the CUDA cores (plain path)                  */
#define OMNI_BF16 1  /* BF16 operands, FP32 accumulation in TMEM (tcgen05.mma)    */
#define OMNI_FP16 2  /* FP16 operands and activations, FP32 accumulation in TMEM;
                        same tensor-core rate as BF16, 3 more mantissa bits      */
#define OMNI_E4M3 3  /* omni_conv_layer only (experiment): E4M3 operands with one
                        activation scale and per-output-channel weight scales,
                        FP32 accumulation in TMEM, BF16 activations in and out */

/* Overlap aggregation (Sec. 2.2, Sec. 3.2). */
#define OMNI_STITCH_AVG 0   /* label = mean logit of covering tiles > 0            */
#define OMNI_STITCH_VOTE 1  /* label = at least half of covering tiles vote > 0    */

/* Weight of a tile's logit at a pixel in the overlap average (average mode;
 * votes are always counted with weight 1).  The weight is separable,
 * w(u, v) = t(u) t(v) at tile coordinates (u, v), 0 <= u, v < P:            */
#define OMNI_WINDOW_FLAT 0  /* t(u) = 1: the plain mean of Sec. 2.3                 */
#define OMNI_WINDOW_TENT 1  /* t(u) = min(u + 1, P - u)                              */
#define OMNI_WINDOW_HANN 2  /* t(u) = sin^2(pi (u + 1/2) / P)                         */

#define OMNI_MAX_SCALES 4
#define OMNI_MAX_CLASSES 16
#define OMNI_MAX_SLIDES 16   /* slides per omni_segment_slides call */

typedef struct omni_ctx omni_ctx;

/* Network and pipeline configuration (fixed for the life of a context). */
typedef struct omni_config {
  int32_t patch;        /* tile size P at every scale (Sec. 2.2: 512)                  */
  int32_t stride;       /* tile stride S (Sec. 3.2: 256 at 40x); P % S == 0; the stride
                           of every scale whose scale_stride entry is 0                  */
  int32_t levels;       /* U-Net levels L (2..6)                                        */
  int32_t base;         /* channels of level 0; level l has base << l (multiple of 8)   */
  int32_t n_scales;     /* number of magnifications (1..4)                              */
  int32_t factors[OMNI_MAX_SCALES];      /* downsample factor vs 40x: 1, 2, 4 or 8      */
  int32_t n_classes;    /* number of tissue classes / dynamic heads (1..16)             */
  int32_t class_scale[OMNI_MAX_CLASSES]; /* scale index each class is predicted at      */
  int32_t precision;    /* OMNI_FP32, OMNI_BF16 or OMNI_FP16                            */
  int32_t stitch_mode;  /* OMNI_STITCH_AVG or OMNI_STITCH_VOTE                          */
  int32_t tissue_filter;/* 1: segment only tiles touching tissue (Sec. 2.1)             */
  int32_t tissue_and;   /* 1: AND every label map with the tissue mask (Sec. 2.3)       */
  int32_t pad_lead;     /* border added on all sides before tiling (Sec. 2.1: 4096)     */
  int32_t median_k;     /* odd median-blur window on the 32x thumbnail (Sec. 3.2: 59)   */
  int32_t max_batch;    /* tiles per network batch (workspace scales with it)           */
  int32_t scale_stride[OMNI_MAX_SCALES]; /* per-scale tile stride S_s in that scale's
                           pixels; 0 = `stride`.  Sec. 3.2 uses 256 at 40x and 64 at 10x
                           and 5x.  Each S_s divides P, is a multiple of 4, and f_s * S_s
                           is a multiple of 32 (tile borders on thumbnail cells).  The
                           canvas is padded to a multiple of lcm_s(f_s * S_s).        */
  int32_t stitch_window;/* OMNI_WINDOW_*: overlap-average weight (omni_backward needs
                           OMNI_WINDOW_FLAT)                                             */
  int32_t min_tissue_area; /* Sec. 2.1 contour step: tissue regions (8-connected pixels of
                           the thumbnail mask) with fewer pixels than this are removed
                           before tiling and label masking; 0 = keep every region (the
                           paper gives no area).  Not supported by
                           omni_tile_slide_noalloc (OMNI_EINVAL when > 0).               */
} omni_config;

/* Sizes derived from a configuration and a slide size (omni_query). */
typedef struct omni_sizes {
  int32_t Hp, Wp;                         /* padded 40x canvas                            */
  int32_t thumb_h, thumb_w;               /* 32x32-box thumbnail / tissue mask            */
  int32_t grid_h[OMNI_MAX_SCALES];        /* tile rows per scale                          */
  int32_t grid_w[OMNI_MAX_SCALES];        /* tile columns per scale                       */
  int32_t n_tiles_max;                    /* sum over scales of grid_h * grid_w            */
  int32_t out_h[OMNI_MAX_SCALES];         /* label map rows at each scale = ceil(H / f)   */
  int32_t out_w[OMNI_MAX_SCALES];         /* label map cols at each scale = ceil(W / f)   */
  uint64_t tile_workspace_bytes;          /* device workspace for omni_tile_slide         */
  uint64_t workspace_bytes;               /* device workspace for omni_segment_slide      */
  uint64_t flops_per_tile;                /* algorithmic conv FLOPs of one tile (2 per MAC) */
} omni_sizes;

/* Result of tissue detection + tiling, in caller-allocated DEVICE buffers.
 * Any pointer except `tiles` and `counts` may be NULL. */
typedef struct omni_tile_list {
  int32_t* tiles;    /* [n_tiles_max][3] = (scale, y, x): foreground tile origins in
                        scale pixels, ordered by scale, then row, then column        */
  int32_t* counts;   /* [1 + n_scales]: total count, then count per scale          */
  uint8_t* flags;    /* per-scale tile grids concatenated (grid_h*grid_w each): 1 = fg */
  uint8_t* tissue;   /* [thumb_h][thumb_w] tissue mask, 1 = tissue                  */
  int32_t* otsu;     /* [1] Otsu threshold on the blurred thumbnail grey (-1: none)  */
} omni_tile_list;

/* Outputs of omni_segment_slide, caller-allocated DEVICE buffers (NULL = skip).
 * Class c lives at scale s = class_scale[c] and has out_h[s] x out_w[s] pixels,
 * row-major, cropped back to the slide (the padding is removed). */
typedef struct omni_outputs {
  uint8_t* labels[OMNI_MAX_CLASSES];    /* 0/1 label map per class                      */
  float* logits[OMNI_MAX_CLASSES];      /* stitched FP32 logit per class (0 if uncovered)*/
  uint16_t* coverage[OMNI_MAX_SCALES];  /* processed tiles covering each pixel           */
  uint8_t* argmax[OMNI_MAX_SCALES];     /* 0 = background, else 1 + class id of the
                                           largest positive logit (ties: lower id)       */
} omni_outputs;

/* Gradients of omni_backward, caller-allocated DEVICE FP32 buffers in the
 * weights-blob shapes.  Any may be NULL. */
typedef struct omni_grads {
  float* ctrl_w;   /* [153][C_{L-1} + n_classes + n_scales]  */
  float* ctrl_b;   /* [153]                                 */
  float* head_w;   /* [8][C_0]                              */
  float* head_b;   /* [8]                                   */
  float* dec0_w1;  /* [C_0][3 C_0][3][3]                    */
  float* dec0_g1;  /* [C_0]                                 */
  float* dec0_b1;  /* [C_0]                                 */
  float* dec0_w2;  /* [C_0][C_0][3][3]                      */
  float* dec0_g2;  /* [C_0]                                 */
  float* dec0_b2;  /* [C_0]                                 */
  float* dec0_wp;  /* [C_0][3 C_0]                          */
} omni_grads;

/* Create a context for `cfg` on the current CUDA device.  Validates the
 * configuration (OMNI_EINVAL with a message on failure).  Owns only the
 * device copy of the weights, a status word and timing events. */
omni_status omni_create(const omni_config* cfg, omni_ctx** out);
void omni_destroy(omni_ctx* ctx);
const char* omni_last_error(const omni_ctx* ctx);

/* Number of float32 values a weights blob for `cfg` must hold. The blob order
 * (C_l = base << l, conv weights [out][in][3][3]):
 *   encoder l = 0..L-1 (cin = 3 for l = 0 else C_{l-1}, cout = C_l):
 *       w1[cout][cin][3][3] g1[cout] b1[cout] w2[cout][cout][3][3] g2 b2 wp[cout][cin]
 *   decoder l = L-2..0 (cin = 3 C_l: upsampled C_{l+1} first, then skip C_l):
 *       same seven tensors
 *   pre-head wh[8][C_0] bh[8]; controller wc[153][C_{L-1}+n_classes+n_scales] bc[153]. */
int64_t omni_weights_count(const omni_config* cfg);

/* Weights of the Omni-Seg network of Sec. 2.2 (residual U-Net, pre-head,
 * class/scale-conditioned controller of the dynamic head).  The paper ships
 * no checkpoint, so the blob carries seeded random-init values in the order
 * given above.  Copies the host FP32 blob (borrowed; the caller keeps it) to
 * one device allocation owned by the context and builds the kernels' layouts
 * (FP32 K-major for the plain path, 16-bit K-major tiles for tcgen05).
 * Replaces any earlier weights and drops a captured CUDA graph, whose
 * arguments point at them.  Synchronous.  OMNI_EWEIGHTS if n_floats is wrong
 * or a value is not finite (nothing changed); OMNI_ECUDA if the copy fails. */
omni_status omni_load_weights(omni_ctx* ctx, const float* blob_host, int64_t n_floats);

/* Sizes for an H x W slide under `cfg` (pure host computation, no device
 * needed).  OMNI_EINVAL for an invalid configuration or slide size. */
omni_status omni_query(const omni_config* cfg, int32_t H, int32_t W, omni_sizes* out);

/* Sec. 2.1: pad (2x2-mean colour), 32x thumbnail, integer grey, median blur,
 * Otsu threshold, tissue mask, and the foreground tile list of every scale.
 * Bit-exact integer arithmetic.  `rgb_dev` is H x W x 3 uint8 with
 * `row_stride` bytes per row.  Asynchronous on `stream`. */
omni_status omni_tile_slide(omni_ctx* ctx, const uint8_t* rgb_dev, int32_t H, int32_t W,
                            int64_t row_stride, void* workspace_dev, uint64_t workspace_bytes,
                            const omni_tile_list* out, void* stream);

/* Whole path: tiling (as omni_tile_slide), the 40x/10x/5x pyramid, the U-Net
 * and dynamic heads on every foreground tile of every requested scale, and
 * the overlap stitch + label emission of every requested class.  Tiles run in
 * batches of max_batch in (scale, row, column) order; after each batch the
 * output rows whose covering tile rows are all done are stitched, so tile
 * logits are kept only for the P/S + 1 tile rows in flight (workspace_bytes
 * does not grow with the number of tiles).
 * `scale_mask` / `class_mask` select scales / classes (bit i = index i); a
 * class is computed only if its scale is selected.  Synchronises `stream`
 * once (after tiling) to size the batch loop.  The workspace must hold
 * omni_sizes.workspace_bytes. */
omni_status omni_segment_slide(omni_ctx* ctx, const uint8_t* rgb_dev, int32_t H, int32_t W,
                               int64_t row_stride, uint32_t scale_mask, uint32_t class_mask,
                               void* workspace_dev, uint64_t workspace_bytes,
                               const omni_outputs* out, void* stream);

/* Same as omni_segment_slide with a HOST slide and HOST label outputs
 * (`labels_host[c]` of out_h x out_w bytes, NULL = skip).  The slide is
 * uploaded on `stream`; the labels leave band by band: the stitch finalises
 * the output rows covered by finished tile rows after every network batch,
 * and each such band is copied to the host on a second stream owned by the
 * context while the next batches compute.  Pinned host memory gives full copy
 * bandwidth (pageable memory works, without the overlap).  Returns after
 * both streams have drained. */
omni_status omni_segment_slide_host(omni_ctx* ctx, const uint8_t* rgb_host, int32_t H,
                                    int32_t W, int64_t row_stride, uint32_t scale_mask,
                                    uint32_t class_mask, void* workspace_dev,
                                    uint64_t workspace_bytes, uint8_t* const* labels_host,
                                    void* stream);

/* Final products of the slide-wise aggregation (Sec. 2.3): every class's
 * merged label map stained onto the 40x slide in its own colour, and the
 * lower-magnification product resized directly from that stained image.
 *   rgb_dev      the H x W x 3 u8 slide, row_stride bytes per row.
 *   labels_dev   HOST array of n_maps (<= 16) DEVICE pointers, NULL = skip:
 *                map k is ceil(H / f_k) x ceil(W / f_k) u8, row-major, nonzero =
 *                on (the label maps omni_segment_slide writes).
 *   factors, colours, alpha   HOST arrays: f_k in {1, 2, 4, 8}; colour_k as
 *                n_maps x 3 u8; alpha_k in 0..256.
 *   Stained pixel: starting from the slide colour c, for k = 0 .. n_maps-1
 *   in order, where map k is on at (y / f_k, x / f_k):
 *     c = (c * (256 - alpha_k) + colour_k * alpha_k + 128) >> 8 per channel.
 *   out40_dev    H x W x 3 u8 (out40_stride bytes per row), or NULL.
 *   down, outd_dev   2, 4 or 8 (Sec. 2.3: 4, the 10x product) and a
 *                ceil(H/down) x ceil(W/down) x 3 u8 image (outd_stride), or NULL:
 *                pixel = rounded mean (sum + n/2) / n of the n stained 40x
 *                pixels of its down x down block (fewer at the right and
 *                bottom edges of a ragged slide).
 * At least one output must be given.  Asynchronous on `stream`; OMNI_EINVAL
 * for bad sizes, factors, alphas or strides, OMNI_ECUDA on a launch error. */
omni_status omni_stain(const uint8_t* rgb_dev, int32_t H, int32_t W, int64_t row_stride,
                       int32_t n_maps, const uint8_t* const* labels_dev, const int32_t* factors,
                       const uint8_t* colours, const int32_t* alpha, uint8_t* out40_dev,
                       int64_t out40_stride, int32_t down, uint8_t* outd_dev, int64_t outd_stride,
                       void* stream);

/* Several slides in one call: a batch of whole-slide images (the paper times
 * its pipeline over a batch of WSIs, Table 1).  Every slide is tiled as by
 * omni_tile_slide; then, scale by scale, the foreground tiles of ALL slides
 * form one list (slide order, then row, column) and go through the network in
 * shared batches of max_batch tiles -- a batch may hold tiles of several
 * slides, so small slides and the few tiles of the coarse scales still fill
 * whole batches -- and each slide's bands are stitched as its tile rows
 * complete.  With graphs enabled (omni_set_graphs) the whole post-tiling
 * chain of all slides is one captured CUDA graph.
 *   n          1..OMNI_MAX_SLIDES slides; rgb_dev[i], H[i], W[i], row_stride[i]
 *              as for omni_segment_slide (HOST arrays of device pointers/sizes)
 *   out        HOST array of n omni_outputs (caller-allocated device buffers,
 *              sized per slide by omni_query)
 *   workspace  omni_query_slides() bytes: every slide's tiling stage plus one
 *              network stage.
 * Labels, logits, coverage and argmax equal n omni_segment_slide calls bit for
 * bit (a tile's result does not depend on its batch).  Synchronises `stream`
 * once, after tiling every slide. */
omni_status omni_query_slides(const omni_config* cfg, int32_t n, const int32_t* H, const int32_t* W,
                              uint64_t* workspace_bytes);
omni_status omni_segment_slides(omni_ctx* ctx, int32_t n, const uint8_t* const* rgb_dev, const int32_t* H,
                                const int32_t* W, const int64_t* row_stride, uint32_t scale_mask,
                                uint32_t class_mask, void* workspace_dev, uint64_t workspace_bytes,
                                const omni_outputs* out, uint64_t* slide_ns_dev, void* stream);
/* slide_ns_dev (optional, NULL = none): caller-allocated DEVICE array of n + 1
 * uint64 that the chain fills, on `stream`, with the device clock in ns
 * (%globaltimer) at the start of the post-tiling chain and after each slide's
 * last stitch band (also when replayed from a graph): per-slide completion
 * time = slide_ns[1 + i] - slide_ns[0]. */

/* Seeded synthetic slide window (input generator, not part of the method):
 * pixel (y, x) of a slide_w-wide slide drawn from `n_ell` rotated ellipses
 * (int64 rows cy, cx, a, b, cos_q14, sin_q14) and SplitMix64 noise seeded
 * with `seed`; with `structures` != 0 the tissue also holds sharp-edged
 * discs on a 512-pixel cell grid (needle-biopsy cores); writes rows
 * y0..y0+h-1, cols x0..x0+w-1 to out_dev. */
omni_status omni_synth_slide(const int64_t* ellipses_host, int32_t n_ell, uint64_t seed,
                             int32_t structures, int32_t slide_w, int32_t y0, int32_t x0, int32_t h,
                             int32_t w, uint8_t* out_dev, int64_t row_stride, void* stream);

/* Building block for layer-level checks: one fused residual-U-Net convolution
 * y = ReLU(g * conv3x3(x) + b [+ wp . r]) on B images of R x R pixels, with the
 * same kernels omni_segment_slide uses.  x / r / y are NHWC with channel
 * stride *_cs and channel offset *_co (elements); dtype float32 for
 * OMNI_FP32, bfloat16 for OMNI_BF16, float16 for OMNI_FP16.  Weights are host FP32 ([cout][cin][3][3],
 * [cout], [cout], [cout][cr]); r may be NULL (no residual).  The layer is
 * launched `repeat` (>= 1) times back to back; if `ms_per_launch` is not NULL
 * it receives the mean device time of one launch (CUDA events on `stream`).
 * `config` (tensor-core precisions; NULL: the default choice for the shape)
 * selects one configuration as 4 int32 rows of omni_conv_candidates (the
 * stages entry may be lowered to 2 or more); a configuration not legal for
 * the shape returns OMNI_EINVAL.
 * OMNI_E4M3 (the 8-bit experiment of the network's convolutions): x and y are
 * bfloat16, x contiguous (x_cs = cin, x_co = 0), no residual, cin a multiple
 * of 128.  The call quantises x to E4M3 with one scale s_x = max|x| / 448 and
 * weight row o with s_w[o] = max_k |w[o][k]| / 448 (round to nearest even,
 * saturating), then runs the per-tap kernel on the E4M3 operands (kind::f8f6f4,
 * FP32 accumulation) with g[o] s_x s_w[o] as the epilogue scale; only those
 * launches are timed.  `config`: kind 0 or 8 (CTA pairs; R * R a multiple of
 * 256), N tile 128 or 256, chunk 128, stages 0; NULL picks kind 8 (kind 0
 * where R * R is not a multiple of 256) with the widest N tile that divides
 * cout.
 * Allocates and frees its own temporary weight buffers; synchronises `stream`. */
omni_status omni_conv_layer(int32_t precision, int32_t B, int32_t R, int32_t cin, int32_t cout,
                            const void* x_dev, int32_t x_cs, int32_t x_co,
                            const float* w_host, const float* g_host, const float* b_host,
                            const void* r_dev, int32_t r_cs, int32_t r_co, int32_t cr,
                            const float* wp_host, void* y_dev, int32_t y_cs, int32_t y_co,
                            const int32_t* config, int32_t repeat, float* ms_per_launch, void* stream);

/* Tensor-core configurations legal for a conv layer shape (R, cin, cout,
 * projection channels cr): writes 4 int32 per configuration (kind as in
 * omni_get_tuned, N tile, channel chunk, pipeline stages) to `rows` (host,
 * up to max_rows) and returns how many it wrote (0: the shape has none). */
int32_t omni_conv_candidates(int32_t R, int32_t cin, int32_t cout, int32_t cr, int32_t* rows,
                             int32_t max_rows);

/* Device timing of omni_segment_slide calls with CUDA events recorded on the
 * call's stream around every launch.  omni_set_timing(ctx, 1) enables it and
 * starts a new record (later calls append to it); omni_get_timing sums, for
 * one kind (0 = U-Net convolutions, 1 = stitch + labels, 2 = GAP + head,
 * 3 = everything else), the milliseconds and launch count of the record and
 * returns its algorithmic work (kind 0: conv FLOPs of the processed tiles;
 * kind 1: bytes the stitch must move).  Synchronises on the recorded events. */
omni_status omni_set_timing(omni_ctx* ctx, int32_t enabled);
omni_status omni_get_timing(omni_ctx* ctx, int32_t kind, double* ms, int64_t* launches,
                            double* flops_or_bytes);

/* Number of kernel launches enqueued by the last omni_segment_slide call. */
int64_t omni_last_launch_count(const omni_ctx* ctx);

/* Conv autotuner (BF16 contexts).  When enabled, the first time a layer
 * shape (R, cin, cout, residual channels, residual kind, batch) is met, every
 * legal tensor-core configuration (small-N variant with 32/64-channel chunks
 * and one or two 8x16 blocks per tile; dx-in-N variant; per-tap variant with
 * each legal N tile and channel chunk) is timed on the
 * real operands and the fastest is kept for the context's lifetime.  Tuning
 * synchronises the stream, so run one untimed call first.  omni_get_tuned
 * writes 10 int32 per tuned shape: R, cin, cout, cr, residual kind, batch,
 * kind (0 per-tap, 1 small-N, 2 dx-in-N, 3 small-N with two blocks per tile,
 * 4 dx-in-N with two blocks per tile, 6 kind 3 on pairs of CTAs whose
 * cta_group::2 MMAs cover 256 pixel rows, 7 kind 4 launched once per 32
 * output channels, 8 kind 0 on pairs of CTAs),
 * N tile, channel chunk, stages; returns the count. */
omni_status omni_set_autotune(omni_ctx* ctx, int32_t enabled);
int32_t omni_get_tuned(const omni_ctx* ctx, int32_t* rows, int32_t max_rows);

/* Kernel choice for checks (tensor-core contexts): kind >= 0 (as in
 * omni_get_tuned) makes every conv layer whose shape has a configuration of
 * that kind run the first such configuration of omni_conv_candidates,
 * overriding the autotuner; other layers keep the default choice.  -1
 * restores the default / autotuned choice.  omni_get_tuned then also lists the
 * configuration each layer shape ran with.  OMNI_EINVAL outside -1..8. */
omni_status omni_set_conv_kind(omni_ctx* ctx, int32_t kind);

/* E4M3 experiment of the network (BF16 contexts; off by default).  When
 * enabled, every conv without a residual projection, fused pool or fused head
 * whose cin and cout are multiples of 128 (the first conv of the deeper
 * encoder and decoder levels) runs as the E4M3 layer of omni_conv_layer: the
 * call's activation is quantised with its own scale max|x| / 448 (computed on
 * the device), the weights with the per-row scales prepared at
 * omni_load_weights, and the output stays BF16.  Everything else runs as in
 * BF16.  Graph capture is skipped while it is on.  OMNI_EINVAL on a context
 * that is not BF16. */
omni_status omni_set_e4m3(omni_ctx* ctx, int32_t enabled);

/* CUDA graphs.  When enabled, omni_segment_slide captures its post-tiling
 * launch chain (every network batch and the stitches) into a CUDA graph on
 * the second call that sees the same slide pointer, size, scale/class masks,
 * workspace, stream, output buffers and foreground tile counts, and replays
 * that graph on later such calls.  Tiling still runs eagerly each call (its
 * counts decide the key).  Ignored while timing is enabled and on the legacy
 * default stream (NULL), which cannot be captured: pass a created stream. */
omni_status omni_set_graphs(omni_ctx* ctx, int32_t enabled);

/* Epilogue fusion (tensor-core contexts; on by default).  When enabled, the
 * second conv of encoder levels 0..L-2 also writes the 2x2 max-pooled input
 * of the next level (the pooling step of the encoder, Sec. 2.2) from its
 * epilogue, and the last decoder conv runs the pre-head and the dynamic heads
 * of the tile's classes (Sec. 2.2; at most two classes per scale) in its
 * epilogue, writing the FP32 tile logits directly; its 16-bit output is then
 * not stored.  Pooling fuses into the small-N and dx-in-N variants (kinds
 * 1-4 and 6), the head into kinds 1-3 and 6 for 32 or 64 output channels and
 * kind 4 for 32 (the per-tap kinds 0 and 8 and the sliced kind 7 fuse
 * neither; the pool then runs as its own launch); the
 * autotuner then considers only variants that fuse the head, so the dynamic
 * head needs no launch of its own.  The GAP of the bottleneck and the
 * controller always run as one launch per batch.  With the head fused, the
 * pre-head reads the FP32 epilogue value instead of its 16-bit rounding, so
 * logits differ from the unfused path by that rounding only.  Disabling is
 * for testing and comparison. */
omni_status omni_set_fusion(omni_ctx* ctx, int32_t enabled);

/* Per-launch device times (ms) of the current timing record, with each
 * launch's kind (as above), tag and algorithmic
 * work (FLOPs for convolutions, else 0).  Tags: conv of encoder level l =
 * 10 l (first) / 10 l + 1 (second), decoder level l = 100 + 10 l (+1);
 * max-pool 200 + l, upsample 300 + l, GAP + controller 401, head 500, stitch 600 + scale,
 * pad 700, pyramid 701, tissue 702, tiles 703.  Writes at most `max`
 * entries into the caller's host arrays (any may be NULL) and returns the
 * count, or -1 on error.  Synchronises on the recorded events. */
int64_t omni_get_launch_times(omni_ctx* ctx, int64_t max, double* ms, int32_t* kinds,
                              int32_t* tags, double* work);

/* Loss and hand-written backward for one slide (FP32 contexts only).  The
 * paper trains nothing (Omni-Seg is used pre-trained, Sec. 2.2); this entry
 * differentiates its Sec. 2.2 head chain through the Sec. 2.3 overlap
 * average, for fine-tuning the class/scale-conditioned parts.
 * Forward: the whole path with stitched FP32 logits; loss = mean over the
 * classes of soft-Dice (smoothing 1) + mean BCE between the stitched logits of
 * the class (label-map pixels of its scale) and `gt_dev[c]` (uint8 0/1, same
 * size as the class's label map).  Backward through the overlap average, the
 * dynamic heads, the controller, the pre-head and the last decoder block;
 * the gradient stops at the GAP feature and at that block's input.  The last
 * block is recomputed batch by batch from its saved input, so memory is bounded
 * by one batch of tiles.  Writes the loss to `loss_dev[0]` and every non-NULL
 * gradient of `grads` (blob layouts).  Deterministic: every sum has a fixed
 * order.  The workspace must hold omni_backward_workspace() bytes; the call
 * synchronises `stream` once per batch.  OMNI_EINVAL for BF16 contexts or
 * max_batch > 64. */
uint64_t omni_backward_workspace(const omni_config* cfg, int32_t H, int32_t W);
omni_status omni_backward(omni_ctx* ctx, const uint8_t* rgb_dev, int32_t H, int32_t W,
                          int64_t row_stride, const uint8_t* const* gt_dev, void* workspace_dev,
                          uint64_t workspace_bytes, float* loss_dev, const omni_grads* grads,
                          void* stream);

/* Tissue detection and tiling (as omni_tile_slide) for callers that may not
 * allocate device memory while they run -- for instance a slide scanner's
 * acquisition loop that reserves its whole device-memory budget at start-up,
 * or a host process whose device memory is owned by another framework's pool,
 * where an extra cudaMalloc could fail or fragment that pool mid-run.  It
 * takes no workspace and calls no allocating routine: its scratch is a fixed
 * static device array of about 13 MiB (OMNI_NOALLOC_MAX_THUMB_PX thumbnail
 * pixels, OMNI_NOALLOC_MAX_TILES tile-grid cells, i.e. slides up to about
 * 4 Gpx at 40x), which every GPU that loads the library keeps until the
 * process exits.  Larger slides return OMNI_EINVAL with a message on stderr
 * and launch nothing.  The thumbnail is computed straight from `rgb_dev`
 * (padding is applied virtually), so no padded copy of the slide is made.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any
 * stream capture.  All calls share the one array and leave their scratch in
 * it (every call re-initialises what it needs), so calls that can overlap on
 * the GPU -- on different streams or host threads, on the same device --
 * race and must be serialised by the caller.  The outputs go to the caller's
 * `out` buffers exactly as for omni_tile_slide and are bit-identical to its.
 * The paper has no counterpart of this entry point. */
#define OMNI_NOALLOC_MAX_THUMB_PX (4 << 20)
#define OMNI_NOALLOC_MAX_TILES (1 << 16)
omni_status omni_tile_slide_noalloc(const omni_config* cfg, const uint8_t* rgb_dev, int32_t H,
                                    int32_t W, int64_t row_stride, const omni_tile_list* out,
                                    void* stream);

#ifdef __cplusplus
}
#endif
#endif /* OMNISEG_H */
