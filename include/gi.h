/*
 * gi.h -- C ABI of libgi, a GB300 (sm_103a) implementation of the
 * differentiable accumulated-summation rasterizer of GaussianImage
 * (arXiv 2403.08551): 2D Gaussians with 8 parameters each (mean mu, Cholesky
 * vector l = (l1, l2, l3), weighted colour c'), rendered as
 *     C_i = sum_n c'_n exp(-sigma_n),  sigma_n = 1/2 d^T Sigma_n^-1 d,
 * with Sigma = L L^T, d = pixel centre - mu, no alpha blending, no depth
 * order (Sec. 3.1 Eq. 1, Sec. 3.2 Eqs. 5 and 7).
 *
 * Conventions for every entry point:
 *  - Pointers named *_dev or documented "device" are CUDA device pointers
 *    owned by the caller; the library never frees them. Unless stated, a
 *    call allocates nothing (gi_fit_create and gi_alu_peaks are the
 *    exceptions).
 *  - Arrays are dense, row-major and 16-byte aligned; a misaligned or NULL
 *    required pointer returns GI_ERR_INVALID_ARG without launching.
 *  - Images are HWC float32 ([height][width][3]); pixel (x, y) has centre
 *    (x + 0.5, y + 0.5); means are in the same pixel frame.
 *  - Parameters are pixel-space values (no activation functions applied).
 *  - Every call is stream-ordered on `stream` (NULL = legacy default
 *    stream), does not synchronise the host and can be captured in a CUDA
 *    graph. Launch failures return GI_ERR_CUDA; faults during execution
 *    surface at a later synchronisation. Conditions detected on the device
 *    (pair capacity exceeded, a bounded wait that gave up) set bits in a
 *    per-device error word read by gi_device_errors().
 *  - On failure gi_last_error() returns a thread-local message.
 *
 * Support of a Gaussian (the paper leaves it unspecified): the tile-granular
 * rectangle of its 3-sigma ellipse, evaluated in FP32 with correctly rounded
 * operations only:
 *     rx = 3|l1|, ry = 3 sqrt(l2^2 + l3^2)
 *     tx0 = clamp(floor((mx - rx)/T), 0, tw), tx1 = clamp(floor((mx + rx)/T) + 1, 0, tw)
 * (y likewise), tw = ceil(W/T), th = ceil(H/T). A Gaussian whose parameters
 * are non-finite, whose det = (l1 l3)^2 is 0, whose FP32 inverse covariance
 * (Sigma^-1 = [[A, B], [B, C]]) is not finite, or whose rectangle is empty is
 * culled (count 0). (A finite FP32 Sigma^-1 implies a finite record factor,
 * GI_REC_FLOATS.) Pixel i receives Gaussian n iff i's tile lies in n's
 * rectangle.
 */
#ifndef GI_H_
#define GI_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GI_API __attribute__((visibility("default")))
#else
#define GI_API
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st* gi_stream;

typedef enum {
    GI_OK = 0,
    GI_ERR_INVALID_ARG = 1, /* bad pointer, size, alignment or tile edge */
    GI_ERR_CUDA = 2,        /* a CUDA runtime call or launch failed */
    GI_ERR_CAPACITY = 3,    /* more (tile, Gaussian) pairs than capacity */
    GI_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
    GI_ERR_UNSUPPORTED = 5, /* configuration not supported */
    GI_ERR_NO_MEMORY = 6    /* allocation failed (gi_fit_create only) */
} gi_status;

/* Device error bits reported by gi_device_errors(). */
#define GI_DEVERR_CAPACITY 1u /* K exceeded capacity: binned outputs incomplete */
#define GI_DEVERR_TIMEOUT 2u  /* a bounded spin/mbarrier wait gave up */
#define GI_DEVERR_BOUNDS 4u   /* an index check failed; the access was skipped */

/* An image and its tile edge T (8, 16 or 32). */
typedef struct {
    int32_t width, height, tile;
} gi_image;

/* Floats per projected record: (mx, my, m11, m21, m22, c'r, c'g, c'b) where
 * [[m11, 0], [m21, m22]] = k L^-1, k = sqrt(log2(e)/2), i.e. m11 = k/l1,
 * m21 = -k l2/(l1 l3), m22 = k/l3. With z1 = m11 dx, z2 = m21 dx + m22 dy:
 * sigma = 1/2 d^T Sigma^-1 d = (z1^2 + z2^2)/log2(e) and
 * exp(-sigma) = exp2(-(z1^2 + z2^2)) (Sec. 3.1 with Sigma^-1 = L^-T L^-1). */
#define GI_REC_FLOATS 8

/* ABI version: 8 (gi_fit_desc gained param_mode, optimizer, beta3, lr_halve_every in 2,
 * cov_mode in 3, the codec fine-tuning fields in 4, opacity_mode and opacity_logits in 5;
 * gi_fit_set_target_source in 6; gi_codec_decode in 7; gi_fit_count_pairs and the
 * GI_FIT_KEYS .. GI_FIT_MEANS16 pointers in 8). */
GI_API int32_t gi_abi_version(void);
GI_API const char* gi_last_error(void);
GI_API const char* gi_status_string(int32_t status);

/* Synchronises `stream`, returns the OR of GI_DEVERR_* bits raised on the
 * current device since the last clear, clearing them if `clear` != 0. */
GI_API gi_status gi_device_errors(uint32_t* bits, int32_t clear, gi_stream stream);

/* ------------------------------------------------------------------------
 * gi_project -- 2D Gaussian formation (Sec. 3.1, Eq. 1; Sec. 3.2, Eq. 5):
 * Sigma = L L^T, the scaled inverse Cholesky factor and the support
 * rectangle.
 *   means [n][2], chol [n][3] = (l1, l2, l3), color [n][3]: device, f32.
 *   rec [n][8] f32 (GI_REC_FLOATS), rect [n][4] i32 (tx0, ty0, tx1, ty1),
 *   cnt [n] i32 = (tx1 - tx0)(ty1 - ty0), 0 when culled (rect = 0).
 * n = 0 is allowed (nothing is written).
 * ---------------------------------------------------------------------- */
GI_API gi_status gi_project(const float* means, const float* chol, const float* color, int32_t n, gi_image img,
                     float* rec, int32_t* rect, int32_t* cnt, gi_stream stream);

/* ------------------------------------------------------------------------
 * gi_bin_tiles -- tile binning for the tile-based rasterization the paper
 * builds on (Sec. 4.1, implementation details) without any depth sort
 * (Sec. 3.2): for every tile t (row-major, t = ty*tw + tx) the list of
 * Gaussians n whose rect contains t, in ascending n.
 *   rect, cnt    from gi_project (device).
 *   rec          nullable; if given with rec_binned, rec_binned[k] = rec[ids[k]].
 *   capacity     number of pairs the outputs can hold (1 .. 2^30 - 1).
 *   ws, ws_bytes scratch of gi_bin_workspace_size() bytes (device, 256-byte
 *                aligned); contents are overwritten.
 *   keys [capacity] u32  sorted tile id of each pair;
 *   ids  [capacity] u32  Gaussian id of each pair (ascending within a tile);
 *   ranges [tw*th][2] i32  [begin, end) of each tile in keys/ids, [0,0) empty;
 *   rec_binned [capacity][8] f32, nullable;
 *   pair_off [n+1] i64  exclusive prefix sum of cnt (pair index of n's first
 *                tile in emission order); pair_off[n] = K;
 *   k_dev [1] i64        K, the total number of pairs.
 * If K > capacity only the first `capacity` emitted pairs are binned, the
 * outputs are incomplete, k_dev still holds K and GI_DEVERR_CAPACITY is
 * raised on the device (the call itself returns GI_OK: it does not wait).
 * Bit-exact: identical inputs give identical outputs on every run.
 * ---------------------------------------------------------------------- */
GI_API gi_status gi_bin_workspace_size(int32_t n, gi_image img, int64_t capacity, size_t* bytes);
GI_API gi_status gi_bin_tiles(const int32_t* rect, const int32_t* cnt, const float* rec, int32_t n, gi_image img,
                       int64_t capacity, void* ws, size_t ws_bytes, uint32_t* keys, uint32_t* ids,
                       int32_t* ranges, float* rec_binned, int64_t* pair_off, int64_t* k_dev,
                       gi_stream stream);

/* ------------------------------------------------------------------------
 * gi_bin_tiles_noalloc -- gi_bin_tiles for callers that cannot allocate
 * device memory. It has no counterpart in the paper: it exists because some
 * callers cannot provide gi_bin_tiles' scratch workspace -- code hosted in
 * another framework's memory pool that may not call cudaMalloc itself,
 * latency-critical loops that must avoid the device synchronisation an
 * allocation can cause, or fixed-budget deployments that reserve all memory
 * up front. Arguments and outputs are those of gi_bin_tiles without ws and
 * ws_bytes; results are identical (bit for bit).
 * Scratch: a fixed array of 6 MiB of this library's device memory, held by
 * every GPU that loads the library until the process exits. Sizes beyond
 * n <= GI_NOALLOC_MAX_GAUSSIANS or capacity <= GI_NOALLOC_MAX_PAIRS are
 * rejected with GI_ERR_INVALID_ARG before anything is launched. The call
 * allocates nothing (no cudaMalloc/cudaFree, no allocating library call).
 * Every call on a device shares the array, which keeps the previous call's
 * contents; the call clears what must start at zero itself. Calls whose
 * work overlaps on the GPU (e.g. on two unordered streams) race on the
 * array and must not be issued. The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current:
 * make this first call before any stream capture.
 * ---------------------------------------------------------------------- */
#define GI_NOALLOC_MAX_GAUSSIANS 262144
#define GI_NOALLOC_MAX_PAIRS 524288
GI_API gi_status gi_bin_tiles_noalloc(const int32_t* rect, const int32_t* cnt, const float* rec, int32_t n,
                                      gi_image img, int64_t capacity, uint32_t* keys, uint32_t* ids,
                                      int32_t* ranges, float* rec_binned, int64_t* pair_off, int64_t* k_dev,
                                      gi_stream stream);

/* ------------------------------------------------------------------------
 * gi_render -- accumulated-summation render (Sec. 3.2, Eq. 7) with an
 * optional fused L2 reconstruction loss (Sec. 3.4, read as the mean over the
 * 3*H*W values).
 *   rec_binned, ranges: from gi_bin_tiles (device).
 *   target [H][W][3] f32, nullable. out [H][W][3] f32 (written).
 *   dl_dout [H][W][3] f32, nullable: dL/dC = 2 (C - target) / (3HW).
 *   loss_sum [1] f64, nullable: sum of (C - target)^2 is ADDED to it
 *   (zero it first; the loss is loss_sum / (3HW)).
 * Summation per pixel runs over the tile's list in a fixed split order, so
 * the result is the same on every run. c' is not clamped (Sec. 3.2).
 * ---------------------------------------------------------------------- */
GI_API gi_status gi_render(const float* rec_binned, const int32_t* ranges, gi_image img, const float* target,
                    float* out, float* dl_dout, double* loss_sum, gi_stream stream);

/* ------------------------------------------------------------------------
 * gi_render_backward -- gradients of the render (App. A.1) chained through
 * Sigma = L L^T to the Cholesky vector (App. A.2; the printed dL/dl2 has a
 * typo: it is 2 g2 l1 + 2 g3 l2), recomputing exp(-sigma) per tile instead
 * of storing per-pixel state.
 *   rec_binned, keys, ids, ranges, pair_off, k_dev: from gi_bin_tiles;
 *   rect, cnt: from gi_project; chol [n][3]: the parameters.
 *   dl_dout [H][W][3] f32: upstream dL/dC.
 *   capacity: the value given to gi_bin_tiles.
 *   ws, ws_bytes: scratch of gi_backward_workspace_size() bytes.
 *   g_means [n][2], g_chol [n][3], g_color [n][3]: written (not added).
 *   g_conic [n][3], nullable: dL/dA, dL/dB, dL/dC of Sigma^-1 = [[A,B],[B,C]]
 *   (B counted once).
 * Deterministic: per-pair partial sums are reduced per Gaussian in emission
 * order; no floating-point atomics.
 * ---------------------------------------------------------------------- */
GI_API gi_status gi_backward_workspace_size(int32_t n, gi_image img, int64_t capacity, size_t* bytes);
GI_API gi_status gi_render_backward(const float* rec_binned, const uint32_t* keys, const uint32_t* ids,
                             const int32_t* ranges, const int32_t* rect, const int32_t* cnt,
                             const int64_t* pair_off, const int64_t* k_dev, const float* chol, int32_t n,
                             gi_image img, int64_t capacity, const float* dl_dout, void* ws, size_t ws_bytes,
                             float* g_means, float* g_chol, float* g_color, float* g_conic, gi_stream stream);

/* ------------------------------------------------------------------------
 * gi_vq_decode -- codec decode (Sec. 3.3): FP16 positions and residual
 * vector quantisation, hat c^M = sum_{k=1..M} C^k[i^k], for the Cholesky
 * vector (attribute 0) and the weighted colour (attribute 1).
 *   means16 [n][2] IEEE binary16 bits; idx [2][stages][n] u8;
 *   codebooks [2][stages][cb_size][3] f32 (cb_size <= 256);
 *   means [n][2], chol [n][3], color [n][3] f32 (written).
 * Bit-exact: each output is the exact stage sum rounded once to FP32.
 * ---------------------------------------------------------------------- */
GI_API gi_status gi_vq_decode(const uint16_t* means16, const uint8_t* idx, const float* codebooks, int32_t n,
                       int32_t stages, int32_t cb_size, float* means, float* chol, float* color,
                       gi_stream stream);

/* ------------------------------------------------------------------------
 * gi_codec_decode -- decode of the paper's codec (Sec. 3.3), the stream a
 * codec fine-tuning context produces: FP16 positions, b-bit Cholesky codes
 * with per-component scale and offset (Eq. 9: l_bar_i = code_i gamma_i +
 * beta_i, FP32 product then sum, each rounded once) and the greedy RVQ
 * colour (Eq. 10: the chosen entries summed in stage order in FP64, rounded
 * once).
 *   means16 [n][2] binary16 bits; codes [n][4] u8 (x, y, z used);
 *   gamma_beta HOST [6] f32 (gamma[3], beta[3]); idx [stages][n] u8;
 *   codebooks [stages][size][3] f32 (size <= 256);
 *   means [n][2], chol [n][3], color [n][3] f32 (written).
 * Bit-exact against the oracle; an index >= size raises GI_DEVERR_BOUNDS
 * and decodes as entry 0.
 * ---------------------------------------------------------------------- */
GI_API gi_status gi_codec_decode(const uint16_t* means16, const uint8_t* codes, const float* gamma_beta,
                          const uint8_t* idx, const float* codebooks, int32_t n, int32_t stages, int32_t size,
                          float* means, float* chol, float* color, gi_stream stream);

/* ------------------------------------------------------------------------
 * Fitting (Sec. 3.4: L2 loss, no adaptive density control, Gaussian count
 * fixed): one step = formation, binning, render + loss, backward and an
 * Adam update (the paper uses Adan; Adam with bias correction here) of all
 * 8 parameters. Several images of different sizes and Gaussian counts are
 * fitted together: their tiles share one launch per stage. The step can be
 * captured once into a CUDA graph and replayed.
 * ---------------------------------------------------------------------- */
typedef struct gi_fit gi_fit;

typedef struct {
    int32_t n_images;
    const int32_t* widths;  /* host [n_images] */
    const int32_t* heights; /* host [n_images] */
    const int32_t* counts;  /* host [n_images] Gaussians per image */
    const float* targets;   /* device, images concatenated, sum W*H*3 f32 */
    const float* params;    /* device [sum counts][8] f32 initial (mx,my,l1,l2,l3,c'r,c'g,c'b) */
    int32_t tile;           /* 8, 16 or 32 */
    float lr_means, lr_chol, lr_color;
    float beta1, beta2, eps;
    int64_t capacity; /* pair capacity (>= 1), fixed for the context */
    int32_t use_graph; /* 1: capture the step once and replay it */
    int32_t stage_events; /* 1: record CUDA events between the five stages */
    int32_t render_split; /* lane groups sharing one tile's list in the render: 0 = default;
                             tile 8: 2 or 4, tile 16: 4 or 8, tile 32: 1 or 2 */
    int32_t param_mode;   /* 0: params are pixel-space (mx, my, l1, l2, l3, c');
                             1: params are the raw parameters of App. C.1: positions
                             theta with mu = (tanh(theta) + 1) / 2 * (W, H), Cholesky
                             diagonal stored without its +0.5 (l1 + 0.5, l2, l3 + 0.5) */
    int32_t optimizer;    /* 0: Adam (beta1, beta2, eps); 1: Adan (Sec. 4.1; Xie et al. 2022):
                             beta1, beta2, beta3 decay the averages of the gradient, of its
                             change and of the squared extrapolated gradient
                             g + beta2 (g - g_prev) (Adan's 0.02, 0.08, 0.01 are 0.98, 0.92,
                             0.99 here), bias-corrected, no weight decay */
    float beta3;          /* Adan only */
    int32_t lr_halve_every; /* every learning rate halves every this many steps (the paper:
                               20000); 0 = constant */
    int32_t cov_mode;     /* 0: params slots 2..4 are the Cholesky vector (l1, l2, l3), Sec. 3.1;
                             1: the rotation-scaling form (theta, s1, s2), Sigma = (R S)(R S)^T
                             (Sec. 3.1, Eq. 2-3), mapped in FP64 to the Cholesky vector of the
                             same Sigma; with param_mode 1 the +0.5 goes on s1 and s2 instead of
                             the Cholesky diagonal */
    /* Attribute quantisation-aware fine-tuning (Sec. 3.3-3.4), one image only,
       Cholesky form only. Each step renders FP16 positions, the b-bit quantised
       Cholesky vector l_bar_i = round(clamp((l_i - beta_i)/gamma_i, 0, 2^b - 1))
       gamma_i + beta_i (half to even; l is the pixel-space vector, after App.
       C.1's +0.5 in param_mode 1) and the greedy M-stage RVQ colour (FP32
       distances, lowest index on ties); gradients pass straight through the
       FP16 rounding and the RVQ and through the quantiser inside its range;
       gamma, beta take the optimiser's step at lr_chol; the codebooks follow
       an exponential moving average of the residuals assigned to each entry
       (count and sum start at 1 and the initial entry). */
    int32_t codec_bits;       /* b in [1, 8]; 0 = off (the fields below are then ignored) */
    int32_t codec_stages;     /* M in [1, 4] */
    int32_t codec_size;       /* B in [1, 256], M x B <= 512 */
    const float* codebooks;   /* device [M][B][3] initial colour codebooks (copied) */
    float lsq_gamma[3];       /* initial gamma_i (> 0) */
    float lsq_beta[3];        /* initial beta_i */
    float ema_decay;          /* in [0, 1) */
    float ema_eps;            /* Laplace smoothing of the counts (>= 0) */
    /* Table 3's ablations: the basic 2D Gaussian of Sec. 3.1 with colour c and a
       separate opacity o = sigmoid(logit) (9 parameters, "w/o M"). params then
       hold c in slots 5..7 and the logits live beside them.
       1: accumulated summation of c o exp(-sigma) (Eq. 5);
       2: sorted alpha-blending (Eq. 3-4, "w/o AR"): per pixel, front to back in
          ascending Gaussian index, alpha = min(0.99, o exp(-sigma)) skipped below
          1/255, stopping before T (1 - alpha) < 1e-4 (3D GS's thresholds);
          tile 16 only. The logits take the optimiser's step at lr_color. */
    int32_t opacity_mode;     /* 0 (merged c', the paper's form), 1 or 2; codec needs 0 */
    const float* opacity_logits; /* device [sum counts] initial logits (copied); NULL = 0 */
    /* Render schedule (results are identical either way): 0 = one block per
       tile in tile order; 1 = a queue of all tiles of the batch ordered by
       descending list length (built on the device each step), served to one
       wave of persistent render blocks. The alpha-blending form ignores it. */
    int32_t tile_queue;
} gi_fit_desc;

/* Allocates the context and copies targets and params (the caller's buffers
 * are not referenced afterwards). */
GI_API gi_status gi_fit_create(const gi_fit_desc* desc, gi_stream stream, gi_fit** out);
/* Runs `steps` fit steps (graph replays when use_graph). Asynchronous. */
GI_API gi_status gi_fit_step(gi_fit* fit, int32_t steps, gi_stream stream);
/* Renders the current parameters into the context's output buffer
 * (formation, binning, Eq. 7; no loss, no dL/dC; GI_FIT_LOSS keeps the last
 * step's value). Replays a captured graph when use_graph. Asynchronous. */
GI_API gi_status gi_fit_render(gi_fit* fit, gi_stream stream);
/* Where the training steps read the target image(s) (Sec. 3.4's L2 loss):
 * src = NULL selects the context's own device copy (GI_FIT_TARGET, the
 * default); otherwise src is a buffer of the same layout (images
 * concatenated, HWC f32) that the device can address: device memory of this
 * device, managed memory, or pinned / registered host memory, which each
 * step's render then reads over the host link, overlapped with its
 * accumulation (no separate copy). The caller keeps src alive and unchanged
 * while steps that read it are in flight. Synchronises `stream` and, with
 * use_graph, recaptures the step graphs. GI_ERR_INVALID_ARG for pageable
 * host memory or another device's memory. */
GI_API gi_status gi_fit_set_target_source(gi_fit* fit, const float* src, gi_stream stream);

/* Device pointers into the context (valid until gi_fit_destroy):
 *   GI_FIT_PARAMS [N][8], GI_FIT_ADAM_M [N][8], GI_FIT_ADAM_V [N][8] (the
 *   optimiser's first two averages; Adan also GI_FIT_ADAN_N, GI_FIT_ADAN_GPREV),
 *   GI_FIT_GRADS [N][8] (gradients of the last step),
 *   GI_FIT_OUT (images concatenated, HWC f32, the last step's render),
 *   GI_FIT_LOSS [n_images] f64 sums of squared error of the last step,
 *   GI_FIT_STEP [1] i32 completed steps, GI_FIT_K [1] i64 pairs of the last
 *   step, GI_FIT_TARGET (images concatenated, HWC f32; may be overwritten
 *   between steps to change the targets). */
enum {
    GI_FIT_PARAMS = 0,
    GI_FIT_ADAM_M = 1,
    GI_FIT_ADAM_V = 2,
    GI_FIT_GRADS = 3,
    GI_FIT_OUT = 4,
    GI_FIT_LOSS = 5,
    GI_FIT_STEP = 6,
    GI_FIT_K = 7,
    GI_FIT_TARGET = 8,
    GI_FIT_ADAN_N = 9,     /* [N][8] Adan's third average (NULL pointer for Adam) */
    GI_FIT_ADAN_GPREV = 10, /* [N][8] Adan's previous gradient (NULL pointer for Adam) */
    /* codec fine-tuning (NULL pointers when codec_bits == 0): */
    GI_FIT_CODEC_GB = 11,    /* f32 [5][6]: gamma[3], beta[3]; then the optimiser's m, v, n, g_prev */
    GI_FIT_CODEBOOKS = 12,   /* f32 [M][B][3] current codebooks */
    GI_FIT_EMA_COUNT = 13,   /* f64 [M][B] EMA counts */
    GI_FIT_EMA_TOTAL = 14,   /* f64 [M][B][3] EMA residual sums */
    GI_FIT_CODES = 15,       /* u8 [N][4] quantiser codes of the last step (4th byte 0) */
    GI_FIT_RVQ_IDX = 16,     /* u8 [M][N] RVQ indices of the last step */
    GI_FIT_CODEC_OUT = 17,   /* f64 [7] last step: L_c, dL/dgamma[3], dL/dbeta[3] */
    /* separate opacity (NULL pointers when opacity_mode == 0): */
    GI_FIT_OPACITY = 18,     /* f32 [7][N]: logit, o of the last formation, optimiser m, v, n,
                                g_prev, dL/dlogit of the last step */
    GI_FIT_N_LAST = 19,      /* i32 [pixels] alpha-blending: list entries each pixel walked */
    /* the binning of the last step (or render), as gi_bin_tiles returns it for the
       batch: global tile id t = the image's first tile + ty tw + tx, global Gaussian
       id = the image's first Gaussian + its index (images in order): */
    GI_FIT_KEYS = 20,        /* u32 [capacity] sorted tile id of each pair (first GI_FIT_K valid) */
    GI_FIT_IDS = 21,         /* u32 [capacity] Gaussian id of each pair, ascending within a tile */
    GI_FIT_RANGES = 22,      /* i32 [tiles][2] [begin, end) of each tile, [0, 0) when empty */
    GI_FIT_PAIR_OFF = 23,    /* i64 [N + 1] exclusive prefix of the counts (emission order) */
    GI_FIT_RECT = 24,        /* i32 [N][4] support rectangle of each Gaussian (image tiles) */
    GI_FIT_CNT = 25,         /* i32 [N] tiles in the rectangle, 0 when culled */
    GI_FIT_MEANS16 = 26      /* u16 [N][2] codec fine-tuning: binary16 bits of the positions the
                                last step rendered (the stream's positions; NULL without codec) */
};
GI_API gi_status gi_fit_pointer(gi_fit* fit, int32_t what, void** ptr);

/* Number of (tile, Gaussian) pairs the first step of a context created from
 * `desc` would bin: the formation of that context (its param_mode, cov_mode
 * and codec quantiser, Sec. 3.1-3.3 and App. C.1) applied to desc->params,
 * then the sum of the support-rectangle tile counts (the opacity forms do
 * not move a rectangle and are not applied). For sizing desc->capacity;
 * desc->capacity itself is ignored. *pairs is a host int64. Allocates
 * temporary device memory (freed before returning) and synchronises
 * `stream`; GI_ERR_INVALID_ARG for a descriptor gi_fit_create would refuse. */
GI_API gi_status gi_fit_count_pairs(const gi_fit_desc* desc, gi_stream stream, int64_t* pairs);
GI_API gi_status gi_fit_destroy(gi_fit* fit);

/* With stage_events set: waits for the last step and writes the device time
 * in milliseconds of its five stages: ms[0] formation, ms[1] binning,
 * ms[2] render + loss, ms[3] backward, ms[4] reduction + Adam update. */
GI_API gi_status gi_fit_stage_times(gi_fit* fit, float* ms);

/* Measures FP32 FMA, packed f32x2 FMA and MUFU.EX2 throughput on the current
 * device (synchronous; allocates a few bytes). result[0..5] = FFMA lane-ops/s,
 * f32x2 FMA lane-ops/s, EX2/s, render-mix elements/s (6 FP32 + 1 EX2),
 * SM MHz during the FFMA run, SM count. */
GI_API gi_status gi_alu_peaks(double* result, gi_stream stream);

/* Self-test of the bounded waits (failure detection without a GPU fault; the
 * paper has no counterpart). Launches one kernel that waits on an mbarrier
 * nothing arrives at (the wait of the render's TMA staging) and one that
 * spins on a device flag nothing sets (the pattern of the look-back scans),
 * each with limit_ns (1 ns .. 2 s) of global time, and returns their private
 * status bits in *observed (host pointer): bit 0 = the mbarrier wait gave up,
 * bit 1 = the spin gave up; bits 2 and 3 would mean a wait ended without its
 * event (never expected). Synchronises `stream`; allocates nothing; leaves
 * gi_device_errors() untouched and the context usable. */
GI_API gi_status gi_selftest_bounded_waits(uint32_t* observed, int64_t limit_ns, gi_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* GI_H_ */
