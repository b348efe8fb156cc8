/*
 * bsf.h -- C ABI of the GB300 space-variant box-spline filter library (libbsf.so).
 *
 * The filter (Chaudhury & Sanyal, "Improvements on 'Fast space-variant
 * elliptical filtering using box splines'", Section 1.1, the BoxFilter
 * algorithm) runs in two steps:
 *
 *   1. pre-integration: n-fold running sums of the (extended, fixed-point)
 *      image along each of the N = 4 grid directions d1 = (1,0), d2 = (1,1),
 *      d3 = (0,1), d4 = (-1,1)  (x is the column, y the row);
 *   2. a per-pixel finite difference of order n along every direction, with
 *      integer steps L_k set by that pixel's covariance, so each output pixel
 *      combines (n+1)^4 samples of the running sum:
 *         out(p) = sum_t w_t S(p + sum_k (c_k - t_k L_k) d_k) / (2^q prod_k L_k^n),
 *         w_t = prod_k (-1)^t_k C(n, t_k),  c_k = n (L_k - 1) / 2.
 *
 * The steps come from the minimum-kurtosis scale vector of the pixel's
 * covariance (Section 1.1; kurtosis matrix of Section 2.3 read for the
 * Cartesian directions), solved in float32 with a fixed sequence of IEEE
 * operations, then L_k = admissible integer nearest to sqrt(1 + a_k^2/|d_k|^2).
 *
 * Arithmetic: the input is quantised once, Q(f) = round-half-even(f 2^q); the
 * running sums and the taps are exact two's-complement integers modulo 2^64
 * (BSF_FIX64) or 2^128 (BSF_FIX128); the wrap-around cancels in the
 * differences whenever |Q| max * prod L^n < 2^(b-1), which the library
 * checks.  The only rounding after Q is the final one:
 *    float32 out: RN32(RN32(acc) 2^-q) / RN32(D)   (IEEE float32 divide)
 *    float64 out: RN64(RN64(acc) 2^-q) / RN64(D)   (IEEE float64 divide)
 * with D = prod_k L_k^n and RNxx round-to-nearest-even of an exact integer.
 *
 * Conventions for every entry point
 *   - Pointers named "device" must point to device memory of the current
 *     device; the caller owns them.  Images are row-major [H][ld] (ld >= W
 *     elements).  Covariance fields are three contiguous float32 planes
 *     [3][H][W]: (C11, C12, C22) for BSF_COV_C, (log sigma, theta, log rho)
 *     for BSF_COV_LOGSIG_THETA_LOGRHO.
 *   - The context owns its workspace (running sums S, step field, scan
 *     carries, status word) and allocates it in bsf_create / bsf_plan only.
 *   - Every call is asynchronous on the context's stream unless stated;
 *     calls on one context must not run concurrently from several threads.
 *   - Return value: BSF_OK (0) or a negative BSF_E* code; no exception
 *     crosses the ABI.  bsf_last_error() gives a message for the last failure.
 *   - Errors found on the device (covariance beyond the elongation bound,
 *     taps beyond the padding, fixed-point overflow) are recorded in a device
 *     status word and reported by bsf_status().
 */
#ifndef BSF_H
#define BSF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define BSF_OK         0
#define BSF_EINVAL    (-1)  /* bad argument */
#define BSF_ENOMEM    (-2)  /* device allocation failed */
#define BSF_ECUDA     (-3)  /* a CUDA runtime call failed */
#define BSF_ERANGE    (-4)  /* a pixel's taps reach beyond the padding R */
#define BSF_ETIMEOUT  (-5)  /* a bounded device wait expired */
#define BSF_EOVERFLOW (-6)  /* max|Q(f)| * prod L^n does not fit the modulus */
#define BSF_ESTATE    (-7)  /* call order: e.g. filter before any pre-integration */
#define BSF_ECOV      (-8)  /* non-finite covariance entries (treated as zero) */

/* boundary extension of the image beyond its borders (the paper is silent) */
#define BSF_ZERO       0    /* f = 0 outside */
#define BSF_REPLICATE  1    /* nearest border sample */
#define BSF_SYMMETRIC  2    /* half-sample mirror: d c b a | a b c d */

/* element types of images */
#define BSF_U8   0
#define BSF_F32  1
#define BSF_F64  2

/* precision of the running sums */
#define BSF_FIX     0       /* modular fixed point of the narrowest of 32, 64, 128 bits that
                               holds the bound, chosen at each pre-integration (see
                               bsf_set_precision) */
#define BSF_FIX64   1       /* uint64 modular fixed point (8 B per element) */
#define BSF_FIX128  2       /* uint128 modular fixed point (16 B per element) */
#define BSF_F64ACC  3       /* precision study: float64 running sums (8 B) */
#define BSF_F32KAHAN 4      /* precision study: compensated float32 running sums, each
                               element an unevaluated sum hi + lo of two float32 added
                               with error-free transformations (8 B) */
#define BSF_FIX32   5       /* uint32 modular fixed point (4 B per element): forward
                               filtering with integer steps only (no backward, no
                               BSF_STEP_D2, no batches); the vertical sums always use the
                               three-phase scan */

/* covariance field encodings */
#define BSF_COV_C   0       /* (C11, C12, C22) in px^2 */
#define BSF_COV_LOGSIG_THETA_LOGRHO 1
                            /* (log sigma, theta, log rho): C has trace 2 sigma^2,
                               eigenvalue ratio rho (>= 1 for log rho >= 0) and its
                               major axis at angle theta from +x; built per pixel in
                               float64 (exp, sin, cos of the plane values, fixed
                               operation order) and rounded once to float32:
                               k = 2 e^(2 ls) / (1 + rho),
                               C11 = k (rho cos^2 + sin^2), C22 = k (rho sin^2 + cos^2),
                               C12 = k (rho - 1) sin cos */

/* step rules */
#define BSF_STEP_D1        0  /* L = admissible integer nearest sqrt(1 + a^2/|d|^2) */
#define BSF_STEP_D1_PAPER  1  /* L = admissible integer nearest a/|d| (paper's step scaling) */
#define BSF_STEP_D2        2  /* continuous steps with interpolated taps (n = 1, 2; fixed
                                 point only): see bsf_filter_jacobian */
#define BSF_STEP_SAMPLED   3  /* the paper's continuous box spline, sampled (Section 2.3, eq.
                                 "interpolation"): order n = 1 only, BSF_FIX64 / BSF_FIX128,
                                 forward only.  Cartesian set: lambda_k = a_k/|d_k| quantised
                                 to 2^-9, Lq_k = max(1, RNE(512 lambda_k)); the running sums are
                                 interpolated at the 16 continuous taps by the grid box spline
                                 of unit steps (nine samples per tap, integer weights over
                                 2^23), so out(p) = sum_m f(m) beta_a(p + tau - m) with
                                 out = RN(RN(acc) 2^(13-q)) / RN(prod Lq).  BSF_DIRS_SECOND
                                 (Algorithm 3 as printed): lambda_k = a_k/sqrt(5) quantised to
                                 2^-5, Lq_k = max(1, RNE(32 lambda_k)), beta'_b interpolation
                                 (6 x 6 samples per tap, integer weights over 491520),
                                 out = RN(RN(acc) 2^(5-q)) / RN(15 prod Lq).  BSF_DIRS_PAIR:
                                 either, per pixel by sector */

/* direction sets (BSF_OPT_DIRECTIONS), Section 2.3 of the paper */
#define BSF_DIRS_CARTESIAN 0  /* beta_a: d1 = (1,0), d2 = (1,1), d3 = (0,1), d4 = (-1,1) (default) */
#define BSF_DIRS_SECOND    1  /* beta'_a of Algorithm 3: e1 = (2,1), e2 = (1,2), e3 = (-1,2),
                                 e4 = (-2,1) (x the column), the mesh of Table 1 with integer
                                 steps; C = (n/60) sum_k A_k e_k e_k^T, feasible for
                                 4 C11 >= C22, 4 C22 >= C11, |C12| <= (2/5)(C11 + C22) (beyond:
                                 clamped and counted like BSF_DIRS_CARTESIAN's e(phi)) */
#define BSF_DIRS_PAIR      2  /* Algorithm 2: both sets of running sums; each pixel takes
                                 beta'_a where its elongation bound is the larger one, i.e.
                                 |C11 - C22| < 3|C12| < 6|C11 - C22| (|C11 - C22| rounded once
                                 to float64), else beta_a.  Twice the running-sum workspace.
   BSF_DIRS_SECOND and BSF_DIRS_PAIR: forward filtering only (bsf_filter, bsf_filter_rows,
   bsf_filter_host, bsf_filter_two_pass), step rules BSF_STEP_D1 / BSF_STEP_D1_PAPER,
   precisions BSF_FIX64 / BSF_FIX128; other calls return BSF_EINVAL.  The second set's
   vertical running sums always use the three-phase scan. */

/* phases timed by bsf_set_profiling / bsf_read_profile */
#define BSF_PHASE_STEPS    0  /* per-pixel step solve */
#define BSF_PHASE_ROWS     1  /* extension + quantisation + running sums along d1 */
#define BSF_PHASE_D3       2  /* running sums along d3 (two kernels; one with look-back) */
#define BSF_PHASE_D2       3  /* running sums along d2 (two kernels; one with look-back) */
#define BSF_PHASE_D4       4  /* running sums along d4 (two kernels; one with look-back) */
#define BSF_PHASE_STENCIL  5  /* finite differences + final rounding */
#define BSF_PHASE_BWD_SCATTER 6  /* backward: weight quantisation + tap scatter */
#define BSF_PHASE_BWD_SCANS   7  /* backward: suffix sums along d4, d2, d3, d1 */
#define BSF_PHASE_BWD_FOLD    8  /* backward: extension adjoint + output */
#define BSF_PHASE_SECOND      9  /* BSF_DIRS_SECOND / _PAIR: extension + quantisation, then the
                                    running sums along e1..e4 (nine kernels) */
#define BSF_PHASE_TILES      10  /* the fused tile filter (BSF_OPT_TILES): one kernel */
#define BSF_PHASE_VJP        11  /* continuous steps: the covariance gradient, from a stored
                                    Jacobian (bsf_jacobian_vjp) or recomputed (bsf_filter_backward) */
#define BSF_NUM_PHASES        12

/* options of bsf_set_option */
#define BSF_OPT_SCAN_MODE    1  /* value BSF_SCAN_THREE_PHASE (default) or BSF_SCAN_LOOKBACK */
#define BSF_OPT_WAIT_LIMIT   2  /* polls a block may spend waiting for a predecessor
                                   (default 1048576, >= 0); past it: BSF_ETIMEOUT */
#define BSF_OPT_SCAN_CHUNK   4  /* rows per chunk of the three-phase scan, 16..4096 (default 48) */
#define BSF_OPT_SCAN_SHORT_TILES 5  /* 1 = look-back tiles of half the rows (16 for uint64) */
#define BSF_OPT_TEST_UNPUBLISHED 3  /* failure injection for tests: 1 = the look-back
                                       scan's first chunk never marks its results
                                       ready, so every wait on it runs out */
#define BSF_OPT_PLAN_UNION   6  /* 1 = each bsf_plan widens the plan instead of replacing it:
                                   R and the mass bound become the largest over every plan
                                   since the option was set (one context for many fields) */
#define BSF_OPT_HOST_BANDS   7  /* row bands of bsf_filter_host's overlapped transfers, 1..32 (default 8) */
#define BSF_OPT_DIRECTIONS   8  /* direction set of the integer-step filter (BSF_DIRS_*); changing
                                   it drops the plan (the next call plans again) */
#define BSF_OPT_TILES        9  /* 1 (default): bsf_filter / bsf_filter_rows with an image run as one
                                   fused kernel of restarted tiles whenever a tile of at least
                                   64 x 64 outputs plus the padding R on each side fits in shared
                                   memory (BSF_STEP_D1 / _PAPER; the Cartesian set in every
                                   precision, the second set and the pair in fixed point, the
                                   pair with two windows per block): each block pre-integrates
                                   its own window in
                                   shared memory, and no running sums are kept (a later
                                   bsf_filter with img NULL, or bsf_copy_preintegrated, needs
                                   bsf_preintegrate); same results as the global passes in fixed
                                   point.  0: always the global passes */
#define BSF_SCAN_LOOKBACK     0 /* single pass, decoupled look-back between blocks */
#define BSF_SCAN_THREE_PHASE  1 /* reduce, then rescan with the carries folded in; no block waits on another
                                   (measured faster on GB300 for 2048^2, n = 2) */

/* device status flags reported through bsf_info_t.flags */
#define BSF_FLAG_CLAMPED  1u  /* some covariance exceeded e(phi) and was clamped */

typedef struct bsf_ctx* bsf_t;

/* Sizes and state of a context (bsf_get_info). */
typedef struct {
  int H, W;            /* image size */
  int N, n;            /* directions (4) and order (1..3) */
  int boundary;        /* BSF_ZERO / BSF_REPLICATE / BSF_SYMMETRIC */
  int R;               /* padding reach; -1 until planned */
  int Hp, Wp;          /* padded domain (H + 2R) x (W + 2R) */
  long long pitch;     /* elements per row of S */
  int elem_bytes;      /* bytes per element of S (4, 8 or 16) */
  int precision;       /* element type of S in use: BSF_FIX32 / _FIX64 / _FIX128 / _F64ACC / _F32KAHAN */
  int frac_bits;       /* q in use (-1 = not yet resolved) */
  int step_rule;       /* BSF_STEP_* */
  int max_reach;       /* largest tap reach of the last plan (-1 before any) */
  double max_mass;     /* largest prod_k L_k^n of the last plan */
  unsigned clamp_count;/* pixels clamped to the elongation bound, last call */
  unsigned flags;      /* BSF_FLAG_* */
  long long workspace_bytes;
  int grad_elem_bytes; /* bytes per element of the backward's adjoint sums: 16 for the
                          continuous steps and for 128-bit contexts, else 8 */
} bsf_info_t;

/* Create a context for H x W images, N = 4 directions, order n in 1..3
 * (Section 1.1: the four-directional box spline beta_a with directions
 * 0, pi/4, pi/2, 3pi/4; Section 2.1: its n-fold self-convolution, whose
 * finite-difference mesh has (n+1)^4 points).
 * boundary: BSF_ZERO / BSF_REPLICATE / BSF_SYMMETRIC.
 * max_reach: padding R >= 0 (fixes the workspace now), or -1 to size it from
 * the first covariance field seen (bsf_plan, or the first bsf_filter).
 * Defaults: precision BSF_FIX64 with automatic q, step rule BSF_STEP_D1,
 * stream 0.  Synchronous; allocates device memory.
 * Errors: BSF_EINVAL (sizes, N != 4, n outside 1..3, boundary), BSF_ENOMEM. */
int bsf_create(bsf_t* out, int H, int W, int N, int n, int boundary, int max_reach);

/* Free the context and its workspace (synchronises its stream). NULL is a no-op. */
void bsf_destroy(bsf_t h);

/* Issue all later work on this cudaStream_t (NULL = the legacy default stream). */
int bsf_set_stream(bsf_t h, void* stream);

/* Choose the arithmetic of the running sums and the number q of fractional
 * bits of the fixed-point input.  BSF_F64ACC / BSF_F32KAHAN keep the image
 * values as they are (q is ignored) and are not exact: the n-fold sums grow
 * like prod_k (extent^n / n!) and their rounding is not cancelled by the
 * differences (forward only).  frac_bits in [0, 30] (BSF_FIX32), [0, 62]
 * (BSF_FIX64 and BSF_FIX) or [0, 100] (BSF_FIX128) fixes q; -1 chooses the
 * largest q (at most 30 for 32 bits, b - 28 otherwise) with
 * (max|f| 2^q) * max prod L^n < 2^(b-2), from the value bound (see
 * bsf_set_value_bound; uint8 images use 255; float images without a declared
 * bound are reduced on the device, which synchronises) and the mass bound of
 * the last plan.
 * BSF_FIX chooses b at every pre-integration, from the same bounds: with a
 * fixed q, the narrowest b in {32, 64, 128} with (max|f| 2^q + 1/2) mass <
 * 2^(b-2); with automatic q, the narrowest b whose automatic q reaches
 * q_t = 0 for uint8 images (exact) and q_t = 25 - ceil(log2 max|f|)
 * otherwise (quantisation below half a float32 ulp of the largest value).
 * 32 bits only for the forward filter with integer steps; the continuous
 * steps choose between 64 and 128.  The backward reads no running sums; its
 * adjoint sums are 128-bit for 128-bit contexts and the continuous steps,
 * 64-bit otherwise (bsf_info_t.grad_elem_bytes).  bsf_get_info reports the
 * element size taken.  Errors: BSF_EINVAL. */
int bsf_set_precision(bsf_t h, int mode, int frac_bits);

/* Declare max |f| of the images to come (used by automatic q; no sync). */
int bsf_set_value_bound(bsf_t h, double max_abs);

/* BSF_STEP_D1 (default), BSF_STEP_D1_PAPER or BSF_STEP_D2 (n <= 2 only).
 * Errors: BSF_EINVAL. */
int bsf_set_step_rule(bsf_t h, int rule);

/* Set an execution option (BSF_OPT_*); it affects how, not what, the filter
 * computes.  BSF_OPT_SCAN_MODE picks the scheme of the running sums along
 * d3/d2/d4; BSF_OPT_WAIT_LIMIT bounds every wait of one block for another
 * (look-back scan): when it runs out the block records BSF_ETIMEOUT in the
 * status word and finishes without hanging (its results are then invalid).
 * Errors: BSF_EINVAL. */
int bsf_set_option(bsf_t h, int option, long long value);

/* Solve the steps of a covariance field (device, [3][H][W] float32), then
 * synchronise: if the context was created with max_reach = -1, set R to the
 * largest tap reach and allocate the running-sum workspace.  Also records the
 * largest kernel mass for automatic q.  Errors: BSF_EINVAL, BSF_ENOMEM,
 * BSF_ECUDA. */
int bsf_plan(bsf_t h, const float* cov, int cov_kind);

/* Pre-integration (step 1 of Section 1.1's BoxFilter: the running sums of
 * the image along each direction, one grid step apart on the axes and on the
 * diagonals; n-fold for order n, Algorithm 3's recursion form without its
 * step-length factor): extend the device image img ([H][ld], dtype
 * BSF_U8 / BSF_F32 / BSF_F64) by the boundary rule onto the padded domain,
 * quantise it, and run the n-fold running sums along d1, d3, d2, d4 into the
 * context's workspace.  Requires R (max_reach or a plan).
 * Errors: BSF_EINVAL, BSF_ESTATE (no R yet), BSF_ECUDA. */
int bsf_preintegrate(bsf_t h, const void* img, int dtype, long long ld);

/* Whole forward filter (Section 1.1's BoxFilter: pre-integration, then per
 * pixel the finite differences of the running sums on the 16-tap mesh of
 * eq. "geometry"'s scales, generalised to (n+1)^4 taps for order n, the
 * steps set by the pixel's covariance through the minimum-kurtosis choice,
 * normalised by the kernel mass).  img != NULL: pre-integrate it first (as
 * bsf_preintegrate; plans on the fly, synchronously, when R is not known);
 * img == NULL: reuse the last pre-integration.  cov: device [3][H][W] float32.
 * out: device [H][ldo] of out_dtype BSF_F32 or BSF_F64.
 * Errors: BSF_EINVAL, BSF_ESTATE, BSF_ECUDA; device-side problems go to bsf_status. */
int bsf_filter(bsf_t h, const void* img, int dtype, long long ld,
               const float* cov, int cov_kind, void* out, int out_dtype, long long ldo);

/* Whole forward filter on HOST buffers, overlapping the transfers with the
 * work: the image is uploaded first and pre-integrated as soon as it has
 * arrived, while the covariance planes follow in row bands (eight by default,
 * BSF_OPT_HOST_BANDS; the last band a quarter of the others' height, so that
 * little work remains after the last upload) on a second stream; the stencil
 * runs band by band as each band's field arrives, and each finished band of
 * the output goes back on a third stream while the next is computed.  img: host [H][ld] of dtype; cov: host [3][H][W] float32
 * of cov_kind; out: host [H][ldo] of out_dtype.  Use page-locked host memory
 * (cudaHostAlloc / torch pin_memory) for the copies to overlap; pageable
 * memory works but serialises them.  The library keeps device copies of the
 * inputs and output (allocated on first use, synchronously).  Synchronous:
 * returns when out holds the result.  The first call plans (waits for the
 * whole field).  Errors: as bsf_filter. */
int bsf_filter_host(bsf_t h, const void* img, int dtype, long long ld, const float* cov, int cov_kind,
                    void* out, int out_dtype, long long ldo);

/* Algorithm 1 of the paper (better Gaussian approximation): split each
 * covariance C = sigma^2 I + Delta C (eq. "SigmaIso"), filter the image with
 * the isotropic box spline of covariance sigma^2 I, then filter that result
 * with the space-variant box spline of the residual Delta C.  sigma^2 is
 * `frac` (the paper takes 1/2) times the smallest eq. "condition2" bound over
 * the field, floored at zero, which keeps every residual within the
 * elongation bound e(phi); the bound is evaluated without trigonometry in a
 * fixed float64 order ((e+1)/(e-1) = (1+t)/sqrt(1+t^2),
 * t = |tan(phi) - cot(phi)|/2 of the orientation phi of C), and
 * sigma^2 = RN32(frac * min).  Both passes run bsf_filter (integer steps,
 * the context's precision and q); the first pass's float32 output is the
 * second pass's input.  The library keeps the two fields and the
 * intermediate image (allocated on first use, synchronously).  The first
 * call plans both fields (synchronous).  sigma2: NULL, or host float that
 * receives sigma^2 (synchronises).  img / dtype / ld / cov / cov_kind / out /
 * out_dtype / ldo as in bsf_filter.  Errors: BSF_EINVAL (frac outside (0, 1),
 * BSF_STEP_D2), as bsf_filter. */
int bsf_filter_two_pass(bsf_t h, const void* img, int dtype, long long ld, const float* cov,
                        int cov_kind, double frac, void* out, int out_dtype, long long ldo,
                        float* sigma2);

/* Forward filter of the band of rows [y0, y1) only (0 <= y0 < y1 <= H).
 * img and cov are the whole image and field ([H][ld], [3][H][W]); out
 * receives the band's rows ([y1-y0][ldo], row 0 = image row y0).  The
 * running sums restart at zero R rows above the band and cover its padded
 * rows [y0 - R, y1 + R) only: every tap of a band pixel lies in that padded
 * band, and the running sums restricted to any rectangle that holds all taps
 * give the same finite differences (every line crosses a rectangle once), so
 * the result equals the whole-image filter bit for bit.  This is the
 * row-band decomposition of one image over several devices (each filters its
 * band; no exchange in the forward).  Requires R (max_reach or a plan).
 * Errors: as bsf_filter. */
int bsf_filter_rows(bsf_t h, const void* img, int dtype, long long ld, const float* cov,
                    int cov_kind, void* out, int out_dtype, long long ldo, int y0, int y1);

/* Backward pass with respect to the image (adjoint of Section 1.1's
 * BoxFilter; the paper has no backward, this is the exact transpose of the
 * forward operator): gimg(i) = sum over the padded positions r that extend
 * onto pixel i of sum_p gout(p) K_p(r - p) / D_p.  Runs as a scatter of
 * w_t gout(p)/D_p at the (n+1)^4 taps of every pixel (64-bit integer
 * reductions, order-independent), reversed n-fold running sums along d4, d2,
 * d3, d1, and the adjoint of the boundary extension.  Fixed point: each
 * gout(p)/D_p is quantised once, RNE(RN32(RN32(gout 2^qg) / RN32(D))), with
 * qg = 54 - ceil(log2 max|gout|) in [0, 100] (found on the device); the
 * result is RN32(acc) 2^-qg.
 *   gout  device [H][ldg] float32;  cov  device [3][H][W] float32 (the field
 *         of the forward call);  gimg device [H][ldgi] float32 (written);
 *   gcov  NULL or device [3][H][W] float32: the integer steps of D1 are
 *         piecewise constant in the covariance, so this gradient is zero
 *         almost everywhere and is written as zeros.
 * Requires a known R (plan or max_reach); any element type of the forward
 * (the backward reads no running sums).  Contexts with uint128 running sums
 * (masses too large for 64-bit weights) take the same pipeline in 128 bits:
 * qg = 118 - ceil(log2 max|gout|) in [0, 126], weights g(p) =
 * RNE(RN32(RN32(gout 2^qg) / RN32(D))), sums modulo 2^128 (128-bit additions
 * from two 64-bit atomics and the carry of the first), gimg = RN32(acc)
 * 2^-qg.  The first call allocates the backward workspace (synchronous).
 * With step rule BSF_STEP_D2: gcov (if not NULL) = gout * d out / d plane,
 * from the held running sums of the forward's image (see
 * bsf_filter_jacobian); gimg (if not NULL; any fixed-point context) is the image
 * gradient: each pixel scatters g(p) = RNE(RN32(RN32(gout 2^qg) / RN32(M)))
 * times the product of its four interpolation weights at its 5^4 (n = 2) or
 * 4^4 (n = 1) samples into uint128 adjoint sums (128-bit additions built from
 * two 64-bit atomics and the carry of the first), qg = 118 -
 * ceil(log2 max|gout|) in [0, 126]; reversed running sums and the extension
 * fold follow as above, then gimg = RN32(acc) 2^-qg.  At least one of gimg and
 * gcov must be given.
 * Errors: BSF_EINVAL, BSF_ESTATE, BSF_ENOMEM, BSF_ECUDA. */
int bsf_filter_backward(bsf_t h, const float* gout, long long ldg, const float* cov, int cov_kind,
                        float* gimg, long long ldgi, float* gcov);

/* Row-band backward (integer or continuous steps): the multi-device form of
 * bsf_filter_backward.  A device that filtered rows [y0, y1) computes the
 * adjoint of its band alone: the pixels of the band scatter into running
 * sums over the band's padded rows [y0 - R, y1 + R), which are summed in
 * reverse and folded by the boundary rule onto image rows
 * [a0, a1) = [max(0, y0 - R), min(H, y1 + R)).  The band's outputs equal the
 * whole image's on every input, so these adjoints add up to the whole-image
 * gradient: each device adds its neighbours' overlapping rows (the halo
 * add-exchange of R rows each way) to its own rows [y0, y1) and finalises.
 * The sums are exact integers modulo 2^64, or 2^128 where the context's
 * adjoint is 128-bit (bsf_info_t.grad_elem_bytes = 16: continuous steps,
 * 128-bit running sums), so the assembled gradient equals
 * bsf_filter_backward's bit for bit when every band uses the same grad_bits:
 * take bsf_grad_frac_bits_of of the maximum of |gout| over all bands
 * (bsf_grad_absmax_rows per band, then the maximum across devices).
 *   acc   device [a1 - a0][lda] elements of grad_elem_bytes (written): two's
 *         complement int64, or int128 as (low, high) int64 pairs; row 0 is
 *         image row a0.
 * Requires R <= H.  Errors: BSF_EINVAL, BSF_ESTATE, BSF_ENOMEM, BSF_ECUDA. */
int bsf_filter_backward_rows(bsf_t h, const float* gout, long long ldg, const float* cov,
                             int cov_kind, int y0, int y1, int grad_bits, long long* acc,
                             long long lda);

/* Fraction bits qg = 54 - ceil(log2 m) of the fixed-point gradient weights for
 * m = max |gout| (float32 value of m), clamped to [0, 100].  Pure function. */
int bsf_grad_frac_bits(double max_abs_gout);

/* The context's rule for qg: bsf_grad_frac_bits for 64-bit adjoint sums, and
 * 118 - ceil(log2 m) in [0, 126] for 128-bit ones (bsf_info_t.grad_elem_bytes).
 * Pure function of the context's configuration.  Errors: BSF_EINVAL. */
int bsf_grad_frac_bits_of(bsf_t h, double max_abs_gout);

/* max |gout| over rows [y0, y1) of device gout [H][ldg] into *result (host
 * float).  Synchronises.  Errors: BSF_EINVAL, BSF_ECUDA. */
int bsf_grad_absmax_rows(bsf_t h, const float* gout, long long ldg, int y0, int y1, float* result);

/* acc[r][x] += halo[r][x] modulo 2^64 (or 2^128: elements of the context's
 * grad_elem_bytes) for rows r < rows and x < W (device acc [rows][lda] and
 * halo [rows][ldh], in elements): the add step of the row-band
 * backward's exchange, where a band's adjoint sums receive the rows its
 * neighbours' adjoints reach into it (the transpose of Section 1.1's
 * BoxFilter spreads each band's contribution up to R rows beyond the band).
 * Exact in two's complement, so the order of the adds does not matter.
 * Asynchronous on the context's stream.  Errors: BSF_EINVAL, BSF_ECUDA. */
int bsf_grad_halo_add(bsf_t h, long long* acc, long long lda, const long long* halo, long long ldh,
                      int rows);

/* gimg[r][x] = RN32(acc[r][x]) 2^-grad_bits for rows r < rows (device acc
 * [rows][lda] of the context's grad_elem_bytes, two's complement; device
 * float32 gimg [rows][ldgi]): the final rounding of the backward.
 * Errors: BSF_EINVAL, BSF_ECUDA. */
int bsf_grad_finalize(bsf_t h, const long long* acc, long long lda, int rows, int grad_bits,
                      float* gimg, long long ldgi);

/* Continuous-step filter (step rule BSF_STEP_D2) and its Jacobian with
 * respect to the covariance field.
 *
 * The paper samples the running sums at off-grid taps by interpolation
 * (Section 2.3, eq. "interpolation").  Here each direction's step
 * lambda_k = sqrt(1 + a_k^2/|d_k|^2) is kept continuous, quantised to 2^-9 of
 * a grid step (Hq = RNE(512 lambda), lambda~ = Hq/512), and every tap
 * q_t = c - t lambda~ (c = n (lambda~ - 1)/2, t = 0..n) along d_k is the
 * linear interpolation of the running sum between its two neighbouring grid
 * points, with integer weights (multiples of 2^-10).  Per direction the 1-D
 * kernel is then exactly the triangle max(0, lambda~ - |j|) sampled at the
 * integers (n = 2) or the overlap of the unit cell at j with the box of
 * width lambda~ (n = 1), and the output is normalised by the exact mass
 * prod_k M_k of the four kernels (integers, times 2^40):
 *    out = RN(RN(acc) 2^-q) / RN(prod_k M_k)   (as in the header comment).
 * For lambda~ an admissible integer it equals BSF_STEP_D1.  The samples are
 * 5^4 = 625 per pixel for n = 2 (4^4 = 256 for n = 1).  The running sums
 * carry 40 more bits than with D1; BSF_FIX128 is the usual choice.
 *
 * jac (NULL, or device float32 [3][H][ldj]) receives d out(p) / d plane_c(p)
 * for the three planes of cov_kind (covariance entries or log sigma, theta,
 * log rho): the derivative of the interpolation weights at fixed brackets
 * (the right derivative in lambda), through the quantisation as the
 * identity, the scale solve (implicit derivative of its stationarity cubic)
 * and the covariance encoding.  Computed from exact integer derivative sums
 * (float64 combination, float32 chain).  Pixels out of reach (identity
 * steps) get zero.  Whole image only; requires BSF_STEP_D2, n <= 2 and a
 * fixed-point precision; automatic q keeps two more guard bits for the
 * derivative sums.  img / dtype / ld / cov / out / ldo as in bsf_filter;
 * out_dtype must be BSF_F32 here.  Errors: BSF_EINVAL, BSF_ESTATE, BSF_ECUDA. */
int bsf_filter_jacobian(bsf_t h, const void* img, int dtype, long long ld, const float* cov,
                        int cov_kind, void* out, int out_dtype, long long ldo, float* jac,
                        long long ldj);

/* Vector-Jacobian product of the continuous-step filter: gcov[c][p] =
 * gout[p] * jac[c][p] for the Jacobian planes of bsf_filter_jacobian.
 * gout device [H][ldg], jac device [3][H][ldj], gcov device [3][H][W]
 * (float32).  With step rule BSF_STEP_D2, bsf_filter_backward(gimg = NULL,
 * gcov) computes the same product without a stored Jacobian, from the
 * running sums of the last pre-integration (which must be the forward's).
 * Errors: BSF_EINVAL. */
int bsf_jacobian_vjp(bsf_t h, const float* gout, long long ldg, const float* jac, long long ldj,
                     float* gcov);

/* Synchronise the stream and return the first device-side error recorded
 * since the last call (BSF_ERANGE, BSF_EOVERFLOW, BSF_ECOV) or BSF_OK, then
 * clear it.  Refreshes the counters in bsf_get_info. */
int bsf_status(bsf_t h);

/* Message describing the last failure on this context (never NULL). */
const char* bsf_last_error(bsf_t h);

/* Fill *info (host pointer).  Does not synchronise. */
int bsf_get_info(bsf_t h, bsf_info_t* info);

/* Copy the integer step field of the last plan/filter into dst (device,
 * uint16 [4][H][W]: L1, L2, L3, L4 planes).  The filter solves the steps
 * inside its stencil kernel, so this solves the last covariance field passed
 * to bsf_filter again (that device buffer must still hold it).  For tests and
 * diagnostics. */
int bsf_copy_steps(bsf_t h, uint16_t* dst);

/* Copy the running sums S of the last pre-integration into dst (device,
 * [Hp][Wp] elements of elem_bytes each, row-major, no pitch padding; for a
 * band of bsf_filter_rows, its rows + 2R padded rows).  For tests and
 * diagnostics. */
int bsf_copy_preintegrated(bsf_t h, void* dst);

/* Time every kernel phase with CUDA events recorded on the context's stream
 * (on != 0), or stop (0).  Up to 4096 phase executions are kept between two
 * bsf_read_profile calls; later ones are counted as dropped.
 * Errors: BSF_ECUDA (event creation). */
int bsf_set_profiling(bsf_t h, int on);

/* Synchronise, then write per phase (BSF_PHASE_*) the summed device time in
 * milliseconds (ms[BSF_NUM_PHASES]) and the number of executions
 * (count[BSF_NUM_PHASES]) since the last read, and reset them.  Host arrays;
 * either may be NULL.  Returns the number of dropped executions (>= 0) or an
 * error code. */
int bsf_read_profile(bsf_t h, double* ms, int* count);

/* Forward filter that allocates nothing.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory while
 * they run, such as an application that gave its whole device-memory budget
 * to its own pool at start-up, or a latency-critical loop that cannot afford
 * the device-wide synchronisation cudaMalloc / cudaFree may cause.
 *
 * It runs the same kernels as bsf_filter (step solve, extension +
 * quantisation + running sums, finite differences; uint64 running sums,
 * BSF_STEP_D1) on scratch memory held in one static device array of 24 MiB
 * inside the library, which every GPU that loads the library keeps until the
 * process exits.  No context is needed; the caller passes inputs and outputs:
 *   img   device [H][ld] of dtype BSF_U8 / BSF_F32 / BSF_F64
 *   cov   device [3][H][W] float32 (C11, C12, C22)
 *   out   device [H][ldo] of out_dtype BSF_F32 / BSF_F64
 *   n     order 1..3; boundary BSF_ZERO / BSF_REPLICATE / BSF_SYMMETRIC
 *   reach padding R >= 3n (pixels whose taps exceed it fall back to identity
 *         steps and make the call return BSF_ERANGE)
 *   frac_bits  q in [0, 62]
 *   stream     cudaStream_t (NULL = legacy default stream)
 * Sizes whose workspace (running sums, chunk aggregates of the vertical sums) would not fit the
 * array -- at most 2^24 pixels and 2^24 padded elements, and 24 MiB in all --
 * are rejected with BSF_ERANGE before any device work.
 * Synchronous: returns BSF_OK, a host-side error (BSF_EINVAL, BSF_ERANGE,
 * BSF_ECUDA) or the device status of this call (BSF_ERANGE, BSF_EOVERFLOW,
 * BSF_ECOV).
 * The first call on each device looks up the array's device address with
 * cudaGetSymbolAddress (the device must be current); make that first call
 * before any stream capture.  With CUDA's lazy module loading (the default
 * since CUDA 12.2) that first call is also when the array's 24 MiB and the
 * library's code are reserved on the device, and it may synchronise the
 * device: a caller that hands all remaining device memory to its own pool
 * should make one small warm-up call on each device at start-up, before
 * reserving the pool (or set CUDA_MODULE_LOADING=EAGER).  All calls share the
 * array and it keeps the last call's contents, so calls that overlap on the
 * GPU race: serialise them.  A failing call returns only after the work it
 * queued has finished. */
int bsf_filter_noalloc(const void* img, int dtype, long long ld, int H, int W, int n,
                       int boundary, int reach, int frac_bits, const float* cov,
                       void* out, int out_dtype, long long ldo, void* stream);

/* ------------------------------------------------------------------------
 * Batches: many images of uneven sizes, each with its own covariance field
 * (the paper filters one image at a time; batching is this library's
 * serving form).  One batch object owns one device arena laid out for a
 * given list of images; every image keeps its own padding R and scan chunk
 * height, and all share one q.
 * ------------------------------------------------------------------------ */
typedef struct bsf_batch* bsf_batch_t;

/* One image of a batch (device pointers; the caller owns them). */
typedef struct {
  int H, W;              /* image size */
  const void* img;       /* [H][ld] of dtype */
  int dtype;             /* BSF_U8 / BSF_F32 / BSF_F64; the same for every image */
  long long ld;
  const float* cov;      /* [3][H][W] float32 (C11, C12, C22) */
  void* out;             /* [H][ldo] of out_dtype */
  int out_dtype;         /* BSF_F32 / BSF_F64; the same for every image */
  long long ldo;
} bsf_image_desc;

typedef struct {
  int B;                 /* images in the plan */
  int frac_bits;         /* common q */
  long long arena_bytes; /* running sums + scan states of all images */
  int scan_chunk[4];     /* scan chunk rows per padded-height class (<=384, <=768, <=1536, more) */
  int blocks[5];         /* blocks of the five batched phases (rows, d3, d2, d4, stencil) */
  long long pixels;      /* output pixels of the batch */
  int graph_ready;       /* a CUDA graph of the batched launches is instantiated */
  int persist_items;     /* work items of the persistent launch */
  int persist_grid;      /* its resident blocks (SMs x blocks per SM) */
  int rows_per_item;     /* padded rows of one row item */
  int stencil_tile_rows; /* rows of one finite-difference tile (32 pixels wide) */
  int persist_graph_ready; /* a CUDA graph of the persistent launch is instantiated */
  int persist_groups;    /* image groups of the persistent launch */
} bsf_batch_info_t;

#define BSF_BATCH_GRAPH      1  /* record the launches once in a CUDA graph, replay it */
#define BSF_BATCH_PER_IMAGE  2  /* baseline: the per-image kernels, image after image */
#define BSF_BATCH_AUTOTUNE   4  /* bsf_batch_plan: tune chunk heights, item shapes and blocks per SM */
#define BSF_BATCH_PERSISTENT 8  /* bsf_filter_batched: the whole batch as one persistent launch */

/* Options of a batch (bsf_batch_set_option). */
#define BSF_BATCH_OPT_WAIT_LIMIT    1  /* polls of one wait of the persistent launch before it
                                          records BSF_ETIMEOUT and goes on (default 2^22) */
#define BSF_BATCH_OPT_TEST_WITHHOLD 2  /* failure injection for tests: 1 = the row phase of image 0
                                          never signals completion, so every wait on it runs out */
#define BSF_BATCH_OPT_ROWS_PER_ITEM 3  /* padded rows per row item of the persistent launch (1..64) */
#define BSF_BATCH_OPT_STENCIL_ROWS  4  /* rows of a finite-difference tile: 8, 16, 32 or 64 */
#define BSF_BATCH_OPT_BLOCKS_PER_SM 5  /* resident blocks per SM of the persistent launch (0 = all that fit) */
#define BSF_BATCH_OPT_GROUP_MB      6  /* running-sum MiB of one image group of the persistent launch
                                          (0 = the whole batch is one group; default 48) */

/* Create a batch object for order n (1..3) and a boundary rule.  It uses
 * uint64 running sums and its own non-blocking stream.  Errors: BSF_EINVAL,
 * BSF_ENOMEM, BSF_ECUDA. */
int bsf_batch_create(bsf_batch_t* out, int n, int boundary);

/* Free the batch (synchronises its stream).  NULL is a no-op. */
void bsf_batch_destroy(bsf_batch_t b);

/* Use this cudaStream_t (must not be the legacy default stream: graph
 * capture needs a real stream).  Drops a recorded graph. */
int bsf_batch_set_stream(bsf_batch_t b, void* stream);

/* The batch's stream (its own unless set). */
void* bsf_batch_stream(bsf_batch_t b);

/* q for the batch: frac_bits in [0, 62], or -1 for automatic (the smallest
 * per-image choice from value_bound (max |f| over the batch; uint8 uses 255)
 * and each image's largest kernel mass). */
int bsf_batch_set_precision(bsf_batch_t b, int frac_bits, double value_bound);

/* Text file in which autotuned chunk heights are kept (read now, appended
 * after tuning); lines "gpu class n rows". */
int bsf_batch_set_tune_cache(bsf_batch_t b, const char* path);

/* Plan a batch of B images (host array of descriptors): solve each image's
 * steps to find its R (synchronous), choose q, allocate one arena, build the
 * per-phase block offsets and the work items of the persistent launch; with
 * BSF_BATCH_AUTOTUNE also time scan chunk heights of 32, 64 and 128 rows on
 * the largest image of each height class (running the filter on it), then
 * tune the persistent launch on the batch itself by coordinate descent (two
 * passes): the chunk height of each height class present (32..128 rows),
 * padded rows per row item (1, 2, 4, 8), rows of a finite-difference tile
 * (8, 16, 32), blocks per SM and the image-group budget (16..96 MiB, or one
 * group), each kept only when the timed launch gets
 * faster.  Tuning writes the outputs.  Values from the tune cache (or set
 * as options) are not tuned again.
 * Errors: BSF_EINVAL, BSF_ENOMEM, BSF_ECUDA. */
int bsf_batch_plan(bsf_batch_t b, int B, const bsf_image_desc* descs, int flags);

/* Filter every image of the planned batch (descs must equal the plan's).
 * Default: one launch per phase for the whole batch (row sums, the two
 * kernels of each vertical direction, finite differences: 8 launches);
 * BSF_BATCH_GRAPH records them in a CUDA graph on the first call and replays
 * it; BSF_BATCH_PER_IMAGE runs the single-image kernels image by image
 * (8 launches per image).  BSF_BATCH_PERSISTENT runs the batch as one
 * persistent launch (a memset of its counters, then one kernel): resident
 * blocks take work items -- padded rows, chunks of 256 lines of each vertical
 * direction's two passes, tiles of the finite differences -- from one ticket
 * counter, image group by image group (consecutive images whose running sums
 * fit BSF_BATCH_OPT_GROUP_MB, so that a group's sums stay in L2 across its
 * passes) and within a group phase by phase; an item waits until the phase before it has
 * finished on its image (a per-image counter; waits are bounded by
 * BSF_BATCH_OPT_WAIT_LIMIT and report BSF_ETIMEOUT); with BSF_BATCH_GRAPH
 * that launch is recorded in a CUDA graph and replayed.  The results equal
 * the other modes' bit for bit.  Asynchronous on the batch's stream.
 * Errors: BSF_EINVAL, BSF_ESTATE, BSF_ECUDA; device-side problems go to
 * bsf_batch_status. */
int bsf_filter_batched(bsf_batch_t b, int B, const bsf_image_desc* descs, int flags);

/* Synchronise and return the first device-side error since the last call
 * (as bsf_status), then clear it. */
int bsf_batch_status(bsf_batch_t b);

/* Set a batch option (BSF_BATCH_OPT_*).  The shape options re-lay the plan
 * (synchronous) and drop recorded graphs.  Errors: BSF_EINVAL. */
int bsf_batch_set_option(bsf_batch_t b, int option, long long value);

int bsf_batch_get_info(bsf_batch_t b, bsf_batch_info_t* info);
const char* bsf_batch_last_error(bsf_batch_t b);

#ifdef __cplusplus
}
#endif

#endif /* BSF_H */
