/*
 * bf.h -- C ABI of the GB300 shiftable O(1) Gaussian bilateral filter.
 *
 * The filter is the one of Chaudhury, "Acceleration of the shiftable O(1)
 * algorithm for bilateral filtering and non-local means" (arXiv:1203.5128):
 *
 *   out(x) = sum_y g_s(x-y) phi(f(y)-f(x)) f(y) / sum_y g_s(x-y) phi(f(y)-f(x))
 *
 * (eq. (BF), Sec. 1) with the Gaussian range kernel replaced by the truncated
 * raised cosine phi_eps of eq. (approx) (Sec. 3), evaluated by SHIFTABLE-BF
 * (Sec. 1.2: modulate, Gaussian-filter, demodulate, normalise), with T from
 * the windowed max filter of Algorithm 1 (Sec. 2) and N, M from Algorithm 2.
 *
 * Conventions shared by every entry point
 *   - Images are float32, row-major, H rows by W columns; `pitch` is the row
 *     stride in ELEMENTS (>= W).  The caller owns every image buffer.
 *   - Pointers named *_dev are device pointers (cudaMalloc / torch tensors on
 *     the plan's device); pointers named *_host are host pointers.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All device work is enqueued on it and the call returns
 *     without synchronising, unless the comment says otherwise.  Results are
 *     valid once the stream has reached the work.
 *   - A plan owns its device workspace (parameter tables, T words, status
 *     word), allocated in bf_plan and freed in bf_destroy.  bf_execute
 *     allocates nothing; bf_execute_host and bf_backward allocate their own
 *     scratch on their first call on a plan.  One plan must not be used on
 *     two streams at the same time.
 *   - Errors are returned as bf_status codes, never as exceptions.  Argument
 *     errors are detected on the host before anything is enqueued.
 *     Data-dependent failures (order above the plan's cap, a bounded wait
 *     that ran out) are recorded in the plan's device status word and read
 *     with bf_get_device_status.
 *   - Borders: sums run over in-image pixels only (clipped windows), the
 *     window is the (2R+1)^2 square with R = ceil(3 sigma_s) (R = sigma_s
 *     for the box spatial filter, BF_SPATIAL_BOX).
 */
#ifndef BF_H
#define BF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bf_plan_s *bf_plan_t; /* opaque; owned by the library */

typedef enum bf_status {
    BF_OK = 0,
    BF_ERR_INVALID_ARG = 1,     /* bad size, sigma, eps, pointer or option   */
    BF_ERR_ORDER_TOO_LARGE = 2, /* N would exceed the plan's cap (n_max)     */
    BF_ERR_ALLOC = 3,           /* device or host allocation failed          */
    BF_ERR_CUDA = 4,            /* a CUDA runtime call failed                */
    BF_ERR_TIMEOUT = 5,         /* a bounded device wait ran out             */
    BF_ERR_NO_FORWARD = 6,      /* bf_backward before any bf_execute         */
    BF_ERR_NOT_SUPPORTED = 7,   /* option combination not built              */
    BF_ERR_DEVICE_STATUS = 8    /* the device status word holds an error     */
} bf_status;

/* How T (Sec. 2) is obtained. */
enum {
    BF_T_FIXED = 0,  /* T = t_fixed (the "global [0,T]" of the earlier method) */
    BF_T_GLOBAL = 1, /* exact T of eq. (bound) by Algorithm 1, one per image    */
    BF_T_TILE = 2    /* T per t_tile x t_tile block of outputs, own N and M      */
};

/* Which M (Sec. 3).  eq. (trunc) is the defining criterion: the smallest M
 * whose dropped tail mass stays within eps, so it keeps the fewest terms
 * for a given eps.  Algorithm 2 takes M = 0 above sigma_r = 40, eq. (trunc)
 * in (10, 40] and the Chernoff estimate of it at sigma_r <= 10, which the
 * paper prefers there to avoid summing the tail; the estimate keeps more
 * terms (at 4096^2, sigma_s = 8, sigma_r = 10, per 128 x 128 T-tile: 19.9
 * against 12.1 on average).  Every rule's weights and M are computed in
 * FP64 on the device. */
enum {
    BF_RULE_ALG2 = 0,    /* Algorithm 2 step 4: sigma_r bands (8-bit scale)   */
    BF_RULE_TRUNC = 1,   /* eq. (trunc)                                       */
    BF_RULE_CHERNOFF = 2 /* eq. (Chernoff), floored                           */
};

/* Spatial filter of the modulated planes (step 2 of SHIFTABLE-BF, Sec. 1.2).
 * FIR: the Gaussian truncated to the (2R+1)^2 window, clipped at the image
 * border.  YVV: the "recursive O(1)" filter that Sec. 1.2 admits, here the
 * third-order recursion of Young and van Vliet (1995), causal plus
 * anti-causal per row then per column, on the image extended by zeros
 * without limit; it approximates the Gaussian of scale sigma_s (a few per
 * cent) at a cost per pixel independent of sigma_s.  YVV needs sigma_s >=
 * 0.5, FP32 planes and t_mode FIXED or GLOBAL (else BF_ERR_NOT_SUPPORTED);
 * its plan holds 512 B per pixel of row-filtered planes (32 terms at a
 * time), 24 B per pixel of row states and 8 B per pixel per pass group of
 * num/den partials (2 or 4 groups): about 9.1 GB at 4096 x 4096.
 * bf_backward and bf_execute_batch take FIR plans only.  AUTO = FIR: the two
 * filters give different results, so the library never swaps one for the
 * other. */
enum { BF_FILTER_AUTO = 0, BF_FILTER_FIR = 1, BF_FILTER_YVV = 2 };

/* Spatial kernel g_s of eq. (BF).  GAUSS: exp(-k^2 / (2 sigma_s^2)) per
 * axis, R = ceil(3 sigma_s).  BOX: the constant filter that Sec. 4 uses to
 * compare SHIFTABLE-BF with BF2 (whose integral histograms work only for
 * box filters); there sigma_s is the radius of the box, so it must be an
 * integer >= 1 (else BF_ERR_INVALID_ARG), R = sigma_s, and every pixel of
 * the clipped (2R+1)^2 square weighs 1.  T (Algorithm 1) is taken over the
 * same square.  The box runs through the FIR, tensor-core, batch and
 * adjoint kernels with unit taps (cost per pixel as the Gaussian's of the
 * same R); BOX with filter = YVV is BF_ERR_NOT_SUPPORTED. */
enum { BF_SPATIAL_GAUSS = 0, BF_SPATIAL_BOX = 1 };

/* Range kernel phi of eq. (BF).  COSINE: the raised cosine of eq. (RCconv)
 * with its binomial expansion, truncation and T (Secs. 1.3, 2, 3, Algorithm
 * 2).  POLY: the raised polynomial of eq. (RPconv), phi(s) = (1 - s^2 /
 * (2 N sigma_r^2))^N with N = max(1, ceil(T^2 / (2 sigma_r^2))) (its
 * positivity threshold, Sec. 1.3) and no truncation (eps is ignored); it is
 * evaluated through an interpolating polynomial basis (Lagrange polynomials
 * of 2N + 1 Chebyshev points over the values of each parameter set's
 * region), so it takes 2N + 1 terms of two planes each.  For POLY, T is the
 * range (max - min) of f over the region a parameter set's expansion spans:
 * the image for BF_T_GLOBAL, each T-tile grown by R for BF_T_TILE, and
 * t_fixed for BF_T_FIXED (which must be >= value_range, the range the
 * expansion then spans; else BF_ERR_NOT_SUPPORTED).  POLY takes FP32 planes
 * and the FIR filter only, and no bf_backward or bf_execute_batch
 * (BF_ERR_NOT_SUPPORTED). */
enum { BF_RANGE_COSINE = 0, BF_RANGE_POLY = 1 };

/* Storage / multiply type of the modulated planes. */
enum { BF_PLANES_FP32 = 0, BF_PLANES_BF16 = 1, BF_PLANES_FP16 = 2 };

/* Device status bits (bf_get_device_status). */
enum {
    BF_DEV_ORDER_TOO_LARGE = 1u << 0, /* some T gave N > cap: those outputs = f */
    BF_DEV_TIMEOUT = 1u << 1,         /* a bounded wait ran out                  */
    BF_DEV_BAD_WORK = 1u << 2         /* a work item failed its range check      */
};

typedef struct bf_options {
    int t_mode;          /* BF_T_*; default BF_T_GLOBAL                           */
    float t_fixed;       /* T for BF_T_FIXED; <= 0 means value_range              */
    float value_range;   /* image range (255, 65535); default 255.  Sets the
                            centring constant and the 8-bit scale of the
                            Algorithm 2 bands (sigma_r * 255 / value_range).      */
    int trunc_rule;      /* BF_RULE_*; default BF_RULE_ALG2                       */
    int filter;          /* BF_FILTER_*; default AUTO (= FIR)                     */
    int plane_dtype;     /* BF_PLANES_*; default FP32                             */
    int n_max;           /* cap on N; default 4096                                */
    int t_tile;          /* T-tile side for BF_T_TILE; default 64 (multiple of 64).
                            16-bit planes need a multiple of 128 (the height of
                            the tensor-core tile, which must lie in one
                            T-tile), else bf_plan returns BF_ERR_INVALID_ARG;
                            FP32 planes use 128-row tiles for multiples of 128
                            and 64-row tiles otherwise.                           */
    long long spin_limit;/* iteration bound of the tensor-core kernel's hand-off
                            waits; default 1<<22, at least 1<<16 (smaller values
                            are raised).  The wait that lets issued MMAs drain
                            before a stopping CTA frees tensor memory has its
                            own fixed bound.                                     */
    int spatial;         /* BF_SPATIAL_*; default GAUSS                           */
    float lowp_recheck;  /* 16-bit planes only: an output whose denominator is
                            below lowp_recheck x its clipped spatial mass
                            (g * 1_Omega)(x) is recomputed in FP32 after the
                            tensor-core pass, by the direct sum of eq. (BF)
                            with phi_eps over its window (bf_info.n_rechecked
                            counts them).  At such pixels (unlike most of
                            their window) the 16-bit rounding of the planes
                            is amplified by mass / den.  Default 0.05; 0
                            turns the recheck off; must lie in [0, 1).     */
    int range_kernel;    /* BF_RANGE_*; default COSINE                            */
    int patch_mask;      /* 0: the bilateral filter.  Else the non-local means of
                            Sec. 6 (eqs. (NL1), (NL2)) with the patch pixels
                            u_i given by the set bits of a 3 x 3 mask, bit
                            3 (dy + 1) + (dx + 1); the centre (bit 4, 0x10)
                            must be set.  The range kernel is the product over
                            the p patch pixels of phi_eps with the N, M that T
                            (Algorithm 1) and Algorithm 2 give; its expansion
                            has (N - 2M + 1)^p terms (half of them run, as
                            conjugate pairs), which must be at most 2^22 for
                            the plan's largest N (else BF_ERR_NOT_SUPPORTED).
                            The spatial weight is sigma_s's Gaussian or, with
                            BF_SPATIAL_BOX, the equal weights of the paper's
                            sums over the window.  Patch values outside the
                            image are taken at the nearest in-image pixel.
                            Takes FP32 planes, the FIR filter, t_mode FIXED or
                            GLOBAL and the cosine kernel, and no bf_backward or
                            bf_execute_batch (else BF_ERR_NOT_SUPPORTED).     */
    float fp32_recheck;  /* FP32 planes with R > 24 (the two-pass FIR, the small
                            FIR tiles, the box's integer running sums): an
                            output whose denominator is below fp32_recheck x
                            its clipped spatial mass is recomputed by the same
                            FP32 direct sum as lowp_recheck's.  Over a large
                            window the terms of eqs. (f1), (f2) are of the
                            order of the window's mass and cancel down to den,
                            so at a pixel unlike most of its window the FP32
                            rounding of the planes is amplified by mass / den.
                            Default 0.05, which keeps every output within 1e-3
                            gray levels of the exact filter with the same T,
                            N, M; 0 turns the recheck off; must lie in [0, 1);
                            plans with R > 63 take no recheck.               */
    int reserved[3];     /* must be zero                                          */
} bf_options;

/* Fills *opt with the defaults listed above. */
void bf_options_init(bf_options *opt);

/* Creates a plan for H x W images (Algorithm 2 inputs: sigma_s, sigma_r,
 * tolerance eps in [0, 1)).  opt may be NULL (defaults).  Selects the
 * device current on the calling thread, allocates the plan's workspace and
 * uploads the spatial taps.  Synchronous.  On error *out is set to NULL. */
bf_status bf_plan(int H, int W, double sigma_s, double sigma_r, double eps,
                  const bf_options *opt, bf_plan_t *out);

/* Algorithm 2 on one image: T (Algorithm 1), N and M (steps 3-4), then
 * SHIFTABLE-BF with phi_eps (Sec. 1.2), writing out_dev.  f_dev and out_dev
 * are H x W float32 device images with row pitches f_pitch and out_pitch
 * (elements); they must not overlap.  Asynchronous on `stream`. */
bf_status bf_execute(bf_plan_t plan, const float *f_dev, size_t f_pitch,
                     float *out_dev, size_t out_pitch, void *stream);

/* bf_execute on host images (contiguous, pitch W): copies f_host to a
 * plan-owned device buffer, filters, copies the result to out_host and
 * synchronises `stream` before returning.  The device buffers are
 * allocated by the first call on a plan and reused.  Plans with exact T per
 * T-tile and 16-bit planes run in row bands (copy in, filter, copy out of
 * different bands overlap, on streams and events the plan creates on this
 * first call and owns: the compute streams at the device's highest stream
 * priority, the FP32 recheck's at its lowest); the result is the same, bit
 * for bit, as copying the whole image and calling bf_execute. */
bf_status bf_execute_host(bf_plan_t plan, const float *f_host, float *out_host,
                          void *stream);

/* Gradient of L = sum_x grad_out(x) out(x) with respect to f, with T, N, M
 * (and the denominator guard) held at the values the last bf_execute of this
 * plan produced on device (not in the paper; derived from eqs. (f1)-(f2)).
 * f_dev must be the image of that bf_execute.  All three images share
 * `pitch`.  The gradient is that of the FP32-plane filter whatever the
 * plan's plane_dtype: a forward pass with FP32 planes recomputes out and the
 * denominator, then the adjoint kernel runs.  The first call on a plan
 * allocates that pass's scratch (two H x W float images), later calls reuse
 * it.  Returns BF_ERR_NO_FORWARD if the plan has not been executed, and
 * BF_ERR_NOT_SUPPORTED if R is too large for the adjoint's tiles. */
bf_status bf_backward(bf_plan_t plan, const float *f_dev, const float *grad_out_dev,
                      float *grad_in_dev, size_t pitch, void *stream);

/* Algorithm 2 on n images, each with its own plan (sizes, sigmas, eps),
 * in one persistent launch fed by a tile work queue.  Images are contiguous
 * (pitch = W of their plan).  Each image needs a plan of its own (a plan
 * named twice is BF_ERR_INVALID_ARG: its workspace serves one image at a
 * time).  FIR plans with the cosine kernel and no patch (else
 * BF_ERR_NOT_SUPPORTED); 16-bit plans run the tensor-core kernel and its
 * FP32 recheck as launches of their own inside the graph.  The results
 * equal n bf_execute calls bit for bit. */
bf_status bf_execute_batch(int n, const bf_plan_t *plans, const float *const *f_dev,
                           float *const *out_dev, void *stream);

typedef struct bf_info {
    int H, W, R;            /* plan sizes; R = ceil(3 sigma_s)                 */
    int n_sets;             /* parameter sets: 1, or the number of T-tiles      */
    float T;                /* T of the last execute (max over T-tiles)         */
    int N, M, K;            /* N, M, K = N-2M+1 of the set with the largest N   */
    long long n_guarded;    /* outputs where the denominator guard fired        */
    long long terms_total;  /* sum over sets of K (work measure)                */
    unsigned device_status; /* BF_DEV_* bits (not cleared)                      */
    int filter, plane_dtype, t_mode;
    int tile_h, tile_w;     /* output tile of the forward kernel                */
    long long n_rechecked;  /* outputs recomputed in FP32 (lowp_recheck, fp32_recheck) */
} bf_info;

/* Synchronises the plan's last stream and reports the parameters the last
 * bf_execute produced. */
bf_status bf_get_info(bf_plan_t plan, bf_info *info);

/* Copies the per-set parameters of the last execute to host arrays of
 * n_sets entries each (any pointer may be NULL).  Synchronising. */
bf_status bf_get_sets(bf_plan_t plan, float *T, int *N, int *M, int n_sets);

/* Synchronises, returns BF_ERR_DEVICE_STATUS if the device status word has
 * any bit set (the bits go to *bits when bits != NULL) and clears it. */
bf_status bf_get_device_status(bf_plan_t plan, unsigned *bits);

/* Frees the plan and its workspace (synchronises its last stream). */
void bf_destroy(bf_plan_t plan);

/* Static text for a status code. */
const char *bf_status_string(bf_status s);

/* ---- device timing of the plan's own launches -------------------------- */

/* on != 0: every later bf_execute of this plan records CUDA events on its
 * stream around K1 (range/T), K2 (N, M, weights), K3 (fused filter) and
 * the FP32 recheck of 16-bit plans (lowp_recheck), up to 4096 executes.
 * Costs five event records per execute. */
bf_status bf_set_timing(bf_plan_t plan, int on);

/* Synchronises and returns, summed over the executes recorded since the
 * last call, the device milliseconds of ms[0] = K1, ms[1] = K2, ms[2] = K3,
 * ms[3] = the recheck (0 when none runs; ms must hold 4 doubles) and their
 * number in *count; then forgets them. */
bf_status bf_get_timing(bf_plan_t plan, double *ms, int *count);

/* ---- allocation-free variant ------------------------------------------- */

/* The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory while they run -- for example a
 * real-time imaging pipeline that reserves all of its GPU memory at start-up,
 * or an application that owns the device's memory budget and only lends
 * this library its image buffers -- and so cannot create a plan.
 *
 * It runs what bf_execute runs for a plan with t_mode = BF_T_GLOBAL,
 * trunc_rule = BF_RULE_ALG2 and FP32 planes: T by Algorithm 1, N and M by
 * Algorithm 2, then the fused filter, from f_dev into out_dev (device images,
 * row pitches in elements), asynchronously on `stream`.  It allocates
 * nothing: all scratch lives in one fixed-size static device array of the
 * library (under 32 KB per GPU, held until the process exits).  Limits:
 * R = ceil(3 sigma_s) <= 48 (else BF_ERR_NOT_SUPPORTED) and the order needed
 * for an image within [0, value_range], ceil(4 value_range^2 / (pi^2
 * sigma_r^2)), <= 1024 (else BF_ERR_ORDER_TOO_LARGE); pixels outside
 * [0, value_range] may push N past the table, and then the output is a copy
 * of the input and the call still returns BF_OK: the status bit that
 * records it is read with bf_noalloc_device_status.  Radii above 24 run on
 * the fused kernel's small tiles (there is no two-pass workspace), so they
 * cost far more per pixel than a plan's two-pass path.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  Every call reuses the same array and
 * clears what must start at zero, so calls whose work overlaps on the GPU
 * (two streams, or two host threads without ordering) race on it: the caller
 * must order them. */
bf_status bf_execute_noalloc(const float *f_dev, size_t f_pitch, float *out_dev,
                             size_t out_pitch, int H, int W, double sigma_s,
                             double sigma_r, double eps, float value_range, void *stream);

/* Device status of bf_execute_noalloc calls on the current device: waits
 * for `stream`, copies the static scratch's status word (BF_DEV_* bits) to
 * *bits (may be NULL), clears it on `stream` and returns
 * BF_ERR_DEVICE_STATUS if any bit was set.  BF_DEV_ORDER_TOO_LARGE means an
 * image had pixels outside [0, value_range] whose local range needed an
 * order above the table: that call's output was a copy of its input.
 * Allocates nothing. */
bf_status bf_noalloc_device_status(void *stream, unsigned *bits);

/* ---- single steps of the path (tests and profiling) ------------------- */

/* Test of the bounded-wait path of the tensor-core forward (16-bit plans):
 * with on != 0, every later bf_execute of the plan makes the tensor-core
 * kernel's MMA-issuing thread wait, first, for a barrier that nothing
 * arrives on.  The wait runs out after spin_limit polls, the CTA stops all
 * of its roles (no MMA has been issued), frees its tensor memory and
 * returns; the outputs of that execute are undefined and the device status
 * word holds BF_DEV_TIMEOUT.  on = 0 restores normal execution.  Not in the
 * paper; for tests of the failure path.  BF_ERR_NOT_SUPPORTED for plans
 * that do not use the tensor-core kernel. */
bf_status bf_test_stall(bf_plan_t plan, int on);

/* Windowed max and min of f over the clipped (2R+1)^2 square (Prop.
 * MAX-FILTER, Algorithm 1 steps 2-3, by the van Herk / Gil-Werman running
 * maxima of the Appendix).  Mx_dev and mn_dev are H x W with row pitch
 * `pitch` like f_dev.  Asynchronous. */
bf_status bf_maxmin(const float *f_dev, int H, int W, size_t pitch, int R,
                    float *Mx_dev, float *mn_dev, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* BF_H */
