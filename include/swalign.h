/*
 * swalign.h -- C ABI of the GB300 library for rigid image alignment in
 * sliced 2-Wasserstein distance (arXiv 2503.13756, "Fast rigid alignment of
 * heterogeneous images in sliced Wasserstein distance").
 *
 * The library scores a reference image f against a moving image g at every
 * rotation on the grid alpha_l = 2 pi l / n (Eq. optimal_rotation, Sec. 1.1;
 * Eq. discrete_rot_sw2, Sec. 2.3) and, optionally, at the closed-form optimal
 * translation (derived from the shift lemma in the proof of Theorem 3.2,
 * App. B: a translation by s adds <s, theta_k> to every quantile of
 * projection k).  It returns the best rotation, the translation and the
 * squared distance d^2 = 1/(nM) ||U_I - T_l V_I||_F^2 (Eq. discrete_sw2).
 *
 * Conventions shared by every call
 *  - Images are L x L float32, row-major [row][column]; cell centres at
 *    x = -1 + (c + 1/2) h, y = -1 + (r + 1/2) h with h = 2/L (App. A.1.2),
 *    so y grows with the row index.  Rotations are counter-clockwise in
 *    (x, y).  Negative pixels are clipped to 0 (the g+ rule of Sec. 5.4);
 *    images need not be normalised (quantiles do not depend on the mass).
 *  - Projection angles theta_k = 2 pi k / n, k = 0..n-1; B bins of width h
 *    centred at s_b = (b - (B-1)/2) h; M quantile levels z_p = (p + 1/2)/M
 *    (or p/M with level_rule = 1).
 *  - Every pointer named d_* is DEVICE memory owned by the caller; the
 *    library never frees it.  Image, projection and quantile pointers must be
 *    16-byte aligned, sw_result pointers 8-byte aligned.  The library owns only its workspace, held in the
 *    context (grown on demand by cudaMalloc, or sized up front by
 *    sw_reserve).
 *  - Every call is asynchronous on the given stream (NULL = legacy default
 *    stream).  The return value reports argument validation and launch errors
 *    synchronously; sw_last_error() gives a message.  A call that returns an
 *    error has launched nothing.
 *  - Per-item failures (an image with no positive mass or a non-finite
 *    pixel) are reported in sw_result.status; such results hold NaN.
 *  - A context is used by one host thread at a time.  No C++ exception
 *    crosses this interface.
 */
#ifndef SWALIGN_H
#define SWALIGN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t, declared without the CUDA headers. */
typedef struct CUstream_st *sw_stream_t;

typedef enum {
    SW_OK = 0,
    SW_ERR_INVALID_ARG = 1, /* bad size, NULL or misaligned pointer       */
    SW_ERR_UNSUPPORTED = 2, /* valid but not built (e.g. precision)       */
    SW_ERR_OOM = 3,         /* workspace does not fit the memory limit    */
    SW_ERR_CUDA = 4,        /* a CUDA runtime call or launch failed       */
    SW_ERR_TIMEOUT = 5      /* a bounded device wait gave up              */
} sw_status;

typedef enum {
    SW_PREC_FP32 = 0,      /* FP32-accurate correlation: tcgen05 GEMM on a 3-term FP16 */
                           /* split, x = hi + lo, hi*hi + hi*lo + lo*hi, FP32 accumulate */
    SW_PREC_BF16 = 1,      /* correlation GEMM on tcgen05, BF16 in, FP32 accumulate    */
    SW_PREC_FP16 = 2,      /* correlation GEMM on tcgen05, FP16 in, FP32 accumulate    */
    SW_PREC_FP32_SIMT = 3  /* correlation in FP32 on the CUDA cores                    */
} sw_precision;

/* Distance between two images. */
typedef enum {
    SW_METRIC_SW2 = 0,   /* sliced 2-Wasserstein of the projections (Eq.          */
                         /* sliced_wasserstein_2, discrete Eq. discrete_sw2)       */
    SW_METRIC_RFSW2 = 1, /* ramp-filtered sliced 2-Wasserstein (Sec. 2.1 "High-    */
                         /* pass filter", Eq. signed_sliced_wasserstein, discrete  */
                         /* Eq. discrete_ssw2): each projection row is filtered by */
                         /* |xi| circularly on its bin grid, split into its        */
                         /* positive part and absolute negative part, each         */
                         /* normalised; the squared distance is the sum of the two */
                         /* parts' sliced W2^2 (1/(n M) with M levels per part).   */
                         /* One translation moves both parts: s* = (c+ + c-)/2.    */
    SW_METRIC_MSW2 = 2   /* max-sliced 2-Wasserstein (Eq. max_sliced_wasserstein): */
                         /* D(l) = max_k (1/M) sum_p (u_pk - v_p,(k-l))^2, direct  */
                         /* O(n^2 M) per pair in FP32 on the CUDA cores (the FFT   */
                         /* correlation does not apply to a maximum); with         */
                         /* translation = 1 the quantiles are centred first (the   */
                         /* sliced-W2 optimal shift, reported as the shift).  Not  */
                         /* for banks, translation grids or the allocation-free    */
                         /* call (SW_ERR_UNSUPPORTED / SW_ERR_INVALID_ARG).        */
} sw_metric;

/* Projection of the images (Sec. 2.1 Eq. radon_transform, Sec. 2.3). */
typedef enum {
    SW_PROJ_SPLAT = 0, /* pixel-driven linear splat: each cell's mass goes to    */
                       /* the two bins around s = <(x, y), theta_k>, split       */
                       /* linearly (exact mass and first moment)                 */
    SW_PROJ_SLICE = 1  /* the paper's Fourier-slice projection (Sec. 2.3,        */
                       /* Theorem proj_nufft): the slice samples of the cell     */
                       /* image at omega_j = 2 pi j / (B h), |j| <= B/2, by a     */
                       /* type-2 NUFFT, and the band-limited projection h g~(s_b) */
                       /* at the bin centres by an inverse FFT over the bin      */
                       /* period B h.  Rows are clipped at zero except for       */
                       /* RFSW2, which splits the signed rows.  The default bin  */
                       /* count is the smallest multiple of 32 >= the default B  */
                       /* and 1.5 L (it is also the grid length of the NUFFT);   */
                       /* an explicit n_bins must be such a count too.           */
                       /* L <= 256 (else SW_ERR_UNSUPPORTED); above L = 128 the  */
                       /* bins are 256, 320 or 384 and the grids and slice       */
                       /* samples use scratch memory owned by the context.  Not  */
                       /* for the allocation-free call.                          */
} sw_projector;

typedef struct {
    int32_t L;              /* image side, 2..512                                   */
    int32_t n_theta;        /* n: even, 4..1024, factors 2, 3, 5 only               */
    int32_t n_levels;       /* M: 1..1024                                           */
    int32_t n_bins;         /* 0 = default B = 2 ceil((L-1)/sqrt 2) + 2; else even, */
                            /* >= the default (fewer bins would lose mass)          */
    int32_t translation;    /* 1 = closed-form optimal translation, 0 = rotation    */
                            /* only (the paper's Eq. discrete_rot_sw2)              */
    int32_t level_rule;     /* 0 = midpoints (p+1/2)/M, 1 = p/M (App. A, Thm. E3)   */
    int32_t gemm_precision; /* sw_precision, used by sw_align_batch / sw_bank_align */
    int32_t metric;         /* sw_metric (0 = sliced W2).  RFSW2: the default bin   */
                            /* count is the smallest even 2/3/5-smooth count >= the */
                            /* default B (the filter's FFT length), an explicit     */
                            /* n_bins must be 2/3/5-smooth, n_levels <= 512         */
    int32_t shift_grid;     /* explicit translation sampling (Sec. 1, exhaustive    */
                            /* search over a translation grid; Sec. 7): with        */
                            /* translation = 1 and shift_grid = K > 0 the shift is  */
                            /* restricted to the grid (i, j) * step, |i|, |j| <= K; */
                            /* 0 = unbounded closed form.  The grid minimum is      */
                            /* exact: D(l, s) = D_T(l) + rho |s - c(l)|^2 (rho 0.5  */
                            /* sliced W2, 1 RFSW2), so it is the grid point nearest */
                            /* the closed-form optimum c(l), per rotation           */
    int32_t shift_step_q;   /* grid step in sixteenths of a pixel (step = q h / 16, */
                            /* h = 2/L); must be > 0 when shift_grid > 0            */
    int32_t projector;      /* sw_projector: how the Radon projections are formed   */
} sw_params;

typedef struct {
    int32_t best_l;   /* l*: g is turned by alpha* = 2 pi l* / n onto f         */
    int32_t status;   /* 0 ok, 1 reference/query unusable, 2 template unusable, */
                      /* 3 a bounded device wait gave up (results NaN)           */
    float angle_rad;  /* alpha* = 2 pi l* / n                                   */
    int32_t template_index; /* j, the template (moving image) this result is  */
                      /* for: the pair's j; in sw_align_batch / sw_bank_align   */
                      /* mode 1 the best template (-1 when none is usable); 0   */
                      /* for single-pair calls                                  */
    double shift[2];  /* s*: f ~ T_{s*} R_{alpha*} g; 0 when translation == 0   */
    double d2;        /* squared distance at (l*, s*), Eq. discrete_sw2         */
} sw_result;          /* 40 bytes */

typedef struct sw_ctx sw_ctx;
typedef struct sw_bank sw_bank;

/* Context on CUDA device `device`.  *out receives the context. */
sw_status sw_create(int device, sw_ctx **out);
/* Frees the workspace; waits for the device. NULL is ignored. */
void sw_destroy(sw_ctx *ctx);
/* Message for the last failing call on ctx ("" if none).  Owned by ctx. */
const char *sw_last_error(const sw_ctx *ctx);
/* Limit, in SM clock cycles, of every wait of one pipeline role on another
 * inside the tensor-core correlation kernel (not part of the method: it
 * bounds the kernel's producer / consumer waits so that a stalled pipeline
 * cannot hang the GPU).  0 = the default, about 4e9 cycles (~2 s).  A wait
 * that runs out stops the kernel's remaining work after letting every copy
 * and MMA already issued land; every result of that call then has status 3
 * and NaN values, and later calls are unaffected.  Applies to later calls on
 * ctx.  Negative values return SW_ERR_INVALID_ARG. */
sw_status sw_set_wait_limit(sw_ctx *ctx, int64_t cycles);
/* Test hook for that failure path (not part of the method): while enabled
 * (enable != 0), every tensor-core correlation on ctx issues no operand
 * copies, so its MMA role waits on a barrier that nothing completes, runs
 * out at the wait limit and the call's results get status 3.  No fault and
 * no hang: every wait stays bounded.  enable = 0 restores normal work. */
sw_status sw_set_correlation_stall(sw_ctx *ctx, int enable);
/* Measured FP32 FMA throughput of device `device` (not part of the method:
 * the denominator of the benchmark's ALU-bound rooflines).  Runs a probe
 * kernel of independent FFMA chains on every SM at the clocks the GPU runs at
 * (it changes no setting), timed with CUDA events: *tflops receives the best
 * of 10 timed launches (2 flops per FMA), *ms_per_launch (may be NULL) that
 * launch's time.  Synchronous; allocates a small output buffer. */
sw_status sw_measure_fp32_fma(int device, double *tflops, double *ms_per_launch);
/* Default bin count for side L: 2 ceil((L-1)/sqrt 2) + 2. */
int sw_default_bins(int L);
/* Caps the workspace (bytes; 0 = no cap).  A call whose workspace would
 * exceed the cap returns SW_ERR_OOM without launching anything. */
sw_status sw_set_workspace_limit(sw_ctx *ctx, size_t bytes);
/* Workspace bytes that sw_align_batch needs for Nq x Nt pairs; 0 when p is
 * NULL or fails the limits of sw_params, or when Nq or Nt is negative. */
size_t sw_batch_workspace_bytes(const sw_params *p, int Nq, int Nt);
/* Allocates the workspace for batches up to Nq x Nt now, so that later
 * calls of that size allocate nothing (and can be stream-captured). */
sw_status sw_reserve(sw_ctx *ctx, const sw_params *p, int Nq, int Nt);

/* Stages of the alignment, for sw_profile_read. */
typedef enum {
    SW_STAGE_PROJECT = 0,   /* Radon projection                         */
    SW_STAGE_QUANTILE = 1,  /* CDF + quantiles                          */
    SW_STAGE_SPECTRUM = 2,  /* centring + FFT over angle                */
    SW_STAGE_CORR = 3,      /* per-frequency correlation GEMM           */
    SW_STAGE_DECIDE = 4,    /* inverse FFT + argmin + FP64 distance     */
    SW_STAGE_BEST = 5,      /* best template per query                  */
    SW_STAGE_RAMP = 6,      /* ramp filter + split (RFSW2)              */
    SW_STAGE_COUNT = 8
} sw_stage;

/* Kernel timing (not part of the method; used by the benchmark).  With
 * enable = 1 every kernel launched through ctx is bracketed by CUDA events on
 * its stream; sw_profile_read waits for the recorded events, writes the
 * summed milliseconds and launch counts per stage (arrays of SW_STAGE_COUNT)
 * and clears the record.  enable = 0 stops recording. */
sw_status sw_profile(sw_ctx *ctx, int enable);
sw_status sw_profile_read(sw_ctx *ctx, double *ms, int64_t *launches);
/* Kernels launched through ctx since its creation. */
int64_t sw_launch_count(const sw_ctx *ctx);

/* Autotuning of launch shapes (no counterpart in the paper: it concerns this
 * implementation's kernels only).  For the parameter set p, times candidate
 * values of four launch choices on a trial batch of random images (up to
 * 1,024 x 64 pairs, ~64 MB of images, within the workspace limit) and keeps
 * the fastest for every later call on ctx with the same L, n_theta, n_levels,
 * bins and gemm_precision:
 *   choice[0] target CTA count of the projection's split over angles,
 *   choice[1] signals per FFT batch of the angle spectra (4, 8 or 16),
 *   choice[2] form of the decision's inverse FFT: 1 = one warp per pair of
 *             curves, in registers (n_theta = 64, 128, 256 or 512 on 32
 *             lanes; 60, 120, 180, 240, 360 or 480 on 30 lanes),
 *             4, 8 or 16 = that many signals per CTA in shared memory,
 *   choice[3] FFT plan, 0..7: bit 2 clear takes the power-of-two part of
 *             the length in radix-4 stages, set in radix-8 stages (with at
 *             most one radix-4 stage); bits 0-1 give the order (0: the
 *             power-of-two stages first, then 2, 3, 5; 1: 2, 3, 5 first;
 *             2: power-of-two first, then 5, 3, 2; 3: 5, 3, 2 first);
 *             a value of 0 in choice[0..2] means the built-in default;
 *   choice[4] output tile width of the tensor-core correlation (columns of
 *             the real-embedded product, two per template: 256 or 128) for
 *             batches of at most 64 templates, where a 256-wide tile would
 *             be half padding,
 *   choice[5] the same for batches of more templates (0 = 256; both timed
 *             on the trial images, for BF16 / FP16 / FP32 split only).
 * None of them changes what is computed; the FFT plan changes the
 * rounding only.  cache_path (may be NULL): a text file of lines
 * "swtune2 <device> L= n= M= B= prec= w s d r g1 g2"; a matching line is used
 * without timing, and a new result is appended.  Synchronous (waits for its
 * own work); allocates trial buffers for the duration of the call.  Banks
 * keep the choice in force when they were created.  Returns SW_ERR_OOM if the
 * trial buffers do not fit, SW_ERR_INVALID_ARG if the cache cannot be
 * written. */
sw_status sw_autotune(sw_ctx *ctx, const sw_params *p, const char *cache_path);
/* The choice in force for p on ctx (zeros before sw_autotune); choice holds
 * 6 ints. */
sw_status sw_autotune_get(const sw_ctx *ctx, const sw_params *p, int *choice);

/* Radon projections (Eq. radon_transform, Sec. 2.1; Sec. 2.3 "Computation")
 * of nb images by the projector p->projector: the linear splat (the mass of
 * each cell goes to the two bins around s = <(x, y), theta_k>, split
 * linearly) or the Fourier slice (the band-limited projection of the cell
 * image by a NUFFT, clipped at zero except for RFSW2; see sw_projector).
 * Negative pixels are clipped to 0 first (Sec. 5.4's g+ rule).
 *   d_img   [nb][L][L] float32 (input)
 *   d_proj  [nb][n][B] float32 (output); row k is the projection at theta_k,
 *           holding the clipped (not renormalised) mass of the image; rows
 *           k >= n/2 are the mirrors of rows k - n/2
 *   d_scale [nb] double (output, may be NULL; 8-byte aligned): 1 / m with
 *           m = sum max(pixel, 0) summed in FP64, the factor that makes the
 *           image a probability density (Sec. 1.1); NaN for an image with no
 *           positive mass or a non-finite pixel.  d_scale[i] * d_proj[i] is
 *           the projection of the normalised image. */
sw_status sw_project(sw_ctx *ctx, const sw_params *p, const float *d_img, int nb,
                     float *d_proj, double *d_scale, sw_stream_t stream);

/* Projections, as sw_project writes them for p, of nb images of side L/2
 * upsampled 2 x 2 to L x L (each pixel split into the four cells of a 2 x 2
 * block with a quarter of its value; the paper has no counterpart: it is the
 * projection that sw_bank_align applies to queries of side L/2).  L even.
 * With the Fourier slice above L = 128 the L/2 image's own grid is used
 * (T_L(t) = (1 + e^{-2 pi i t_1})(1 + e^{-2 pi i t_2}) / 4 T_{L/2}(2 t), Sec. 2.3
 * "Computation" applied to the L/2 image), so the rows equal those of the
 * upsampled image to the NUFFT's accuracy, not bitwise.
 *   d_img  [nb][L/2][L/2] float32 (input)
 *   d_proj [nb][n][B] float32 (output), layout of sw_project
 * Returns SW_ERR_INVALID_ARG for odd L. */
sw_status sw_project_upsampled(sw_ctx *ctx, const sw_params *p, const float *d_img, int nb,
                               float *d_proj, sw_stream_t stream);

/* Quantile functions of projections (Sec. 2.3: CDF by cumulative sum, ICDF
 * by linear interpolation; Eq. inv_cdf with the ">=" of App. A.1.1).
 *   d_proj   [nb][n][B] float32 (input, as written by sw_project)
 *   d_q      [nb][n][M] float32 (output): d_q[i][k][p] = Q_k(z_p), uncentred
 *   d_center [nb][2] double (output, may be NULL): a = (2/n) sum_k ubar_k theta_k,
 *            the centring vector (= the translation-optimal offset)
 *   d_norm   [nb] double (output, may be NULL): sum_k sum_p (Q_k(z_p) - <a, theta_k>)^2
 * With metric RFSW2 every row is first ramp-filtered and split (see sw_metric):
 * d_q is [nb][2][n][M] (positive part, then absolute negative part), d_center
 * [nb][2][2] and d_norm [nb][2], per part. */
sw_status sw_quantiles(sw_ctx *ctx, const sw_params *p, const float *d_proj, int nb,
                       float *d_q, double *d_center, double *d_norm, sw_stream_t stream);

/* One pair, every rotation (Eq. discrete_rot_sw2 with the FFT
 * cross-correlation of Sec. 2.3 "Fast computation over rotations").
 *   d_f, d_g [L][L] float32: reference f and moving image g
 *   d_D      [n] double (may be NULL): d^2 at every l (at s*(l) if translation)
 *   d_shift  [n][2] double (may be NULL): s*(l) (0 if translation == 0)
 *   d_best   [1] sw_result: the argmin (lowest l on ties) */
sw_status sw_align_all_rotations(sw_ctx *ctx, const sw_params *p, const float *d_f,
                                 const float *d_g, double *d_D, double *d_shift,
                                 sw_result *d_best, sw_stream_t stream);

/* Allocation-free variant of sw_align_all_rotations (the paper has no
 * counterpart; this is an interface for callers that cannot allocate device
 * memory while running -- a process that has given all device memory to its
 * own pool, a latency-critical loop that cannot accept the device-wide
 * synchronisation of cudaMalloc/cudaFree, or a plugin whose host forbids
 * device allocations after start-up).  Same arguments and results as
 * sw_align_all_rotations, minus the context, for the sliced-W2 metric with
 * the linear-splat projector only: metric RFSW2 or MSW2 and projector
 * SW_PROJ_SLICE return SW_ERR_UNSUPPORTED.  The pair is scored in the FP32
 * path (CUDA-core correlation) on the current device and the given stream.
 * It calls no cudaMalloc, cudaFree or allocating library routine, and copies
 * nothing from host memory: every intermediate buffer and the angle tables
 * (computed by a kernel) live in one fixed 4 MiB device array inside the
 * library, which every GPU that loads the library holds until the process
 * exits.
 *   Limit: the per-pair intermediates, about 8 (n/2) B + 16 n M + 20 n
 *   bytes, must fit in 4 MiB (e.g. L <= 512 with n <= 512 and M <= 256);
 *   larger sizes return SW_ERR_OOM and launch nothing.  Parameters that fail
 *   the limits of sw_params return the status sw_align_all_rotations would
 *   (SW_ERR_INVALID_ARG or SW_ERR_UNSUPPORTED); NULL or misaligned pointers
 *   return SW_ERR_INVALID_ARG.  No message is kept (there is no context).
 *   The first call on a device looks up the array's device address (make it
 *   before any stream capture).  All calls on a device share the array and
 *   leave their intermediates in it; calls that overlap on the GPU (e.g. on
 *   unordered streams) race and must be serialised by the caller. */
sw_status sw_align_all_rotations_noalloc(const sw_params *p, const float *d_f, const float *d_g,
                                         double *d_D, double *d_shift, sw_result *d_best,
                                         sw_stream_t stream);

/* Many pairs: every query i (reference f) against every template j (moving
 * image g).  The per-frequency correlation sum_p Qhat_i(k,p) conj(Qhat_j(k,p))
 * runs as a batched GEMM in the precision p->gemm_precision.
 *   d_q_img [Nq][L][L] float32, d_t_img [Nt][L][L] float32
 *   mode 0: d_out [Nq][Nt] sw_result, every pair
 *   mode 1: d_out [Nq] sw_result, the best template per query (least d^2,
 *           lowest index on ties); best_l etc. refer to that template, whose
 *           index is template_index. */
sw_status sw_align_batch(sw_ctx *ctx, const sw_params *p, const float *d_q_img, int Nq,
                         const float *d_t_img, int Nt, int mode, sw_result *d_out,
                         sw_stream_t stream);

/* Template bank for serving: the angle spectra, centring vectors and norms
 * of Nt templates, computed once and kept on the device (owned by the bank,
 * freed by sw_bank_destroy). */
sw_status sw_bank_create(sw_ctx *ctx, const sw_params *p, const float *d_t_img, int Nt,
                         sw_bank **out, sw_stream_t stream);
/* Queries against a bank.  q_L == p->L, or q_L == p->L / 2: the query is then
 * upsampled 2 x 2 (each cell split into four of a quarter of its value,
 * exact under the cell-average model).  mode as in sw_align_batch. */
sw_status sw_bank_align(sw_ctx *ctx, const sw_bank *bank, const float *d_q_img, int Nq,
                        int q_L, int mode, sw_result *d_out, sw_stream_t stream);
int sw_bank_size(const sw_bank *bank);
/* Context workspace bytes that sw_bank_align needs for Nq queries (the
 * basis of memory-based admission in a serving loop). */
size_t sw_bank_workspace_bytes(const sw_bank *bank, int Nq, int mode);
void sw_bank_destroy(sw_bank *bank);

#ifdef __cplusplus
}
#endif
#endif /* SWALIGN_H */
