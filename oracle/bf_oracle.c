/*
 * FP64 CPU oracle for the shiftable O(1) Gaussian bilateral filter and the
 * accelerations of Chaudhury, "Acceleration of the shiftable O(1) algorithm
 * for bilateral filtering and non-local means" (arXiv:1203.5128).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header, table or constant generator with the CUDA path.
 *
 * Every routine is the plain definition, written for a reader to check by
 * eye against the paper: no blocking, no fusion, no reordering beyond what
 * the cited passage states.  All arithmetic is IEEE double.  Compile with
 * -ffp-contract=off so that integer decisions (N, M) are the same on every
 * host.
 *
 * Conventions (readings of the paper where it is silent or garbled):
 *   - window: the (2R+1)x(2R+1) square, R = ceil(3 sigma_s) (Sec. 2: "say,
 *     R = 3 sigma_s"; the smallest rectangle containing the neighbourhood);
 *   - borders: clipped windows, i.e. sums run over in-image pixels only; the
 *     max filter pads with -inf and the min filter with +inf;
 *   - N = max(1, ceil(4 T^2 / (pi^2 sigma_r^2))), the positivity threshold
 *     N0 of Sec. 1.3 rounded up;
 *   - M: eq. (trunc) literally, eq. (Chernoff) floored, or the sigma_r bands
 *     of Algorithm 2;
 *   - denominator guard: where den <= 1e-6 * (g * 1_Omega)(x) the output is
 *     f(x) (the paper is silent; phi_eps may dip to -eps on its tails);
 *   - recursive mode: the Young-van Vliet recursion applied to the image
 *     extended by zeros without limit (a margin beyond double precision).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

static int imin(int a, int b) { return a < b ? a : b; }
static int imax(int a, int b) { return a > b ? a : b; }

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Spatial kernel (Sec. 1, eq. (BF); support R from Sec. 2).           */
/* ------------------------------------------------------------------ */

int orc_radius(double sigma_s) { return (int)ceil(3.0 * sigma_s); }

/* g[k + R] = exp(-k^2 / (2 sigma_s^2)), k = -R..R (unnormalised: the
 * filter output num/den does not depend on the scale of g). */
void orc_gauss_taps(double sigma_s, int R, double *g)
{
    for (int k = -R; k <= R; ++k)
        g[k + R] = exp(-(double)k * (double)k / (2.0 * sigma_s * sigma_s));
}

/* ------------------------------------------------------------------ */
/* Windowed max / min (Sec. 2, Prop. MAX-FILTER; Appendix).            */
/* ------------------------------------------------------------------ */

/* Brute force: Mx(x) = max of f over the clipped (2R+1)^2 window, mn the min. */
void orc_maxmin_brute(const double *f, int H, int W, int R, double *Mx, double *mn)
{
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double hi = -INFINITY, lo = INFINITY;
            for (int a = imax(0, i - R); a <= imin(H - 1, i + R); ++a)
                for (int b = imax(0, j - R); b <= imin(W - 1, j + R); ++b) {
                    double v = f[(size_t)a * W + b];
                    if (v > hi) hi = v;
                    if (v < lo) lo = v;
                }
            Mx[(size_t)i * W + j] = hi;
            mn[(size_t)i * W + j] = lo;
        }
}

/* One-dimensional MAX-FILTER of the Appendix (van Herk / Gil-Werman), on n
 * values read with stride `stride` from src and written with the same
 * stride to dst.  The sequence is padded by R values of `pad` on each side
 * and then up to a multiple of the window size Wn = 2R+1; l and r are the
 * running extrema from the left and from the right, restarted at every
 * partition boundary; the windowed extremum at i is extr(r[i], l[i+2R]) in
 * padded coordinates.  sign = +1 gives the max filter, -1 the min filter.
 * Returns the number of max (min) operations performed. */
static long vhgw_1d(const double *src, double *dst, int n, long stride, int R,
                    double sign, double *buf)
{
    const int Wn = 2 * R + 1;
    const int Lp = ((n + 2 * R + Wn - 1) / Wn) * Wn;
    double *p = buf, *l = buf + Lp, *r = buf + 2 * (size_t)Lp;
    long ops = 0;
    /* work on sign*f so that one max routine serves both filters; the
     * padding is -inf in that domain (+inf for the min filter) */
    for (int q = 0; q < Lp; ++q) {
        int s = q - R;
        p[q] = (s >= 0 && s < n) ? sign * src[(size_t)s * stride] : -INFINITY;
    }
    for (int k0 = 0; k0 < Lp; k0 += Wn) {
        l[k0] = p[k0];
        for (int q = k0 + 1; q < k0 + Wn; ++q) { l[q] = fmax(l[q - 1], p[q]); ++ops; }
        r[k0 + Wn - 1] = p[k0 + Wn - 1];
        for (int q = k0 + Wn - 2; q >= k0; --q) { r[q] = fmax(r[q + 1], p[q]); ++ops; }
    }
    for (int i = 0; i < n; ++i) {
        dst[(size_t)i * stride] = sign * fmax(r[i], l[i + 2 * R]);
        ++ops;
    }
    return ops;
}

/* Separable 2-D max and min filters (Algorithm 1, steps 2-3): rows, then
 * columns of the row result.  Returns the total operation count (both
 * filters) so that the O(1) cost per point can be checked. */
long orc_maxmin_vhgw(const double *f, int H, int W, int R, double *Mx, double *mn)
{
    long ops = 0;
    double *tmp = (double *)malloc(sizeof(double) * (size_t)H * W);
    for (int pass = 0; pass < 2; ++pass) {
        double sign = pass == 0 ? 1.0 : -1.0;
        double *out = pass == 0 ? Mx : mn;
        #pragma omp parallel reduction(+ : ops)
        {
            int L = imax(H, W) + 4 * R + 2;
            double *buf = (double *)malloc(sizeof(double) * 3 * (size_t)(L + 2 * R + 1));
            #pragma omp for schedule(static)
            for (int i = 0; i < H; ++i)
                ops += vhgw_1d(f + (size_t)i * W, tmp + (size_t)i * W, W, 1, R, sign, buf);
            #pragma omp for schedule(static)
            for (int j = 0; j < W; ++j)
                ops += vhgw_1d(tmp + j, out + j, H, W, R, sign, buf);
            free(buf);
        }
    }
    free(tmp);
    return ops;
}

/* ------------------------------------------------------------------ */
/* Dynamic range T (Sec. 2, eq. (bound), Prop. 2.1, Algorithm 1).      */
/* ------------------------------------------------------------------ */

/* Local range r(x) = max_{y in window} |f(y) - f(x)| = max(M(x)-f(x), f(x)-m(x)). */
void orc_local_range(const double *f, const double *Mx, const double *mn, int H, int W,
                     double *r)
{
    for (size_t k = 0; k < (size_t)H * W; ++k)
        r[k] = fmax(Mx[k] - f[k], f[k] - mn[k]);
}

/* Per-tile T: T[tile] = max of r over the pixels of each tile x tile block
 * of a grid anchored at (0,0), rounded to FP32 (the GPU receives T as a
 * float).  A single tile covering the image gives the global T of eq. (bound). */
void orc_t_tiles(const double *r, int H, int W, int tile_h, int tile_w, float *T)
{
    int ty = (H + tile_h - 1) / tile_h, tx = (W + tile_w - 1) / tile_w;
    for (int a = 0; a < ty; ++a)
        for (int b = 0; b < tx; ++b) {
            double m = 0.0;
            for (int i = a * tile_h; i < imin(H, (a + 1) * tile_h); ++i)
                for (int j = b * tile_w; j < imin(W, (b + 1) * tile_w); ++j)
                    m = fmax(m, r[(size_t)i * W + j]);
            T[a * tx + b] = (float)m;
        }
}

/* ------------------------------------------------------------------ */
/* Order N and truncation M (Sec. 1.3, Sec. 3, Algorithm 2).           */
/* ------------------------------------------------------------------ */

/* Real threshold N0 = 4 T^2 / (pi^2 sigma_r^2). */
double orc_n0(double T, double sigma_r)
{
    return (4.0 * T * T) / (ORC_PI * ORC_PI * sigma_r * sigma_r);
}

/* N = max(1, ceil(N0)). */
int orc_order(double T, double sigma_r)
{
    double n0 = orc_n0(T, sigma_r);
    int N = (int)ceil(n0);
    return N < 1 ? 1 : N;
}

/* log of the binomial weights of eq. (expansion): w_n = 2^-N C(N,n),
 * in the log domain so that 2^-N does not underflow for large N. */
void orc_log_weights(int N, double *lw)
{
    double c = lgamma((double)N + 1.0) - (double)N * log(2.0);
    for (int n = 0; n <= N; ++n)
        lw[n] = c - lgamma((double)n + 1.0) - lgamma((double)(N - n) + 1.0);
}

/* eq. (trunc): the smallest M with sum_{n=0}^{M+1} w_n > eps/2. */
int orc_trunc_m(int N, double eps)
{
    if (!(eps > 0.0)) return 0;
    double *lw = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    orc_log_weights(N, lw);
    int M = 0;
    double S = exp(lw[0]);                 /* S(0) */
    for (M = 0; M + 1 <= N; ++M) {
        S += exp(lw[M + 1]);               /* S(M+1) */
        if (S > eps / 2.0) break;
    }
    free(lw);
    if (M > N / 2) M = N / 2;
    return M;
}

/* eq. (Chernoff): M = (N - sqrt(4 N log(2/eps))) / 2, floored and clamped. */
int orc_chernoff_m(int N, double eps)
{
    if (!(eps > 0.0)) return 0;
    double m = 0.5 * ((double)N - sqrt(4.0 * (double)N * log(2.0 / eps)));
    int M = (int)floor(m);
    if (M < 0) M = 0;
    if (M > N / 2) M = N / 2;
    return M;
}

/* Algorithm 2, step 4.  The sigma_r bands are stated for 8-bit images;
 * sigma_r is compared on the 8-bit scale, sigma_r * 255 / value_range. */
int orc_alg2_m(int N, double sigma_r, double eps, double value_range)
{
    if (!(eps > 0.0)) return 0;
    double s8 = sigma_r * 255.0 / value_range;
    if (s8 > 40.0) return 0;
    if (s8 > 10.0) return orc_trunc_m(N, eps);
    return orc_chernoff_m(N, eps);
}

/* phi_eps(s) of eq. (approx) at each of ns points (M = 0 gives eq. (expansion)). */
void orc_phi_eval(const double *s, int ns, int N, int M, double sigma_r, double *out)
{
    double *lw = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    orc_log_weights(N, lw);
    double scale = sqrt((double)N) * sigma_r;
    for (int i = 0; i < ns; ++i) {
        double acc = 0.0;
        for (int n = M; n <= N - M; ++n)
            acc += exp(lw[n]) * cos((double)(2 * n - N) * s[i] / scale);
        out[i] = acc;
    }
    free(lw);
}

/* ------------------------------------------------------------------ */
/* SHIFTABLE-BF (Sec. 1.2, eqs. (GF), (f1), (f2); four-step procedure)  */
/* ------------------------------------------------------------------ */

/* (g * 1_Omega)(i, j): the clipped Gaussian mass at an output pixel. */
static double clipped_mass(const double *g, int R, int H, int W, int i, int j)
{
    double sy = 0.0, sx = 0.0;
    for (int a = imax(0, i - R); a <= imin(H - 1, i + R); ++a) sy += g[a - i + R];
    for (int b = imax(0, j - R); b <= imin(W - 1, j + R); ++b) sx += g[b - j + R];
    return sy * sx;
}

/* Outputs for the pixels of the block [y0,y1) x [x0,x1), computed with the
 * range kernel phi_eps(N, M) (one kernel for the whole block).  For each
 * kept n (no folding of n and N-n):
 *   1. planes F_n = f cos(w_n f), f sin(w_n f), G_n = cos(w_n f), sin(w_n f)
 *      over the block grown by R and clipped to the image;
 *   2. separable Gaussian on each plane (rows, then columns; clipped);
 *   3. num += w_n [cos(w_n f(x)) Fc + sin(w_n f(x)) Fs],
 *      den += w_n [cos(w_n f(x)) Gc + sin(w_n f(x)) Gs];
 * then out = num / den (guarded).  Output is written into out[H*W] at the
 * block's pixels; the number of guarded pixels is returned. */
long orc_shiftable_block(const double *f, int H, int W, const double *g, int R,
                         int N, int M, double sigma_r,
                         int y0, int y1, int x0, int x1,
                         double *out, double *num_out, double *den_out)
{
    const int ry0 = imax(0, y0 - R), ry1 = imin(H, y1 + R);
    const int rx0 = imax(0, x0 - R), rx1 = imin(W, x1 + R);
    const int rh = ry1 - ry0, rw = rx1 - rx0, oh = y1 - y0, ow = x1 - x0;
    double *P = (double *)malloc(sizeof(double) * 4 * (size_t)rh * rw);
    double *Hp = (double *)malloc(sizeof(double) * 4 * (size_t)rh * ow);
    double *num = (double *)calloc((size_t)oh * ow, sizeof(double));
    double *den = (double *)calloc((size_t)oh * ow, sizeof(double));
    double *lw = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    orc_log_weights(N, lw);
    const double scale = sqrt((double)N) * sigma_r;
    const size_t rsz = (size_t)rh * rw, hsz = (size_t)rh * ow;

    for (int n = M; n <= N - M; ++n) {
        const double wn = exp(lw[n]);
        const double om = (double)(2 * n - N) / scale;
        /* step 1: modulated planes */
        #pragma omp parallel for schedule(static)
        for (int a = 0; a < rh; ++a)
            for (int b = 0; b < rw; ++b) {
                double v = f[(size_t)(ry0 + a) * W + (rx0 + b)];
                double c = cos(om * v), s = sin(om * v);
                size_t k = (size_t)a * rw + b;
                P[k] = v * c; P[rsz + k] = v * s; P[2 * rsz + k] = c; P[3 * rsz + k] = s;
            }
        /* step 2a: rows */
        #pragma omp parallel for schedule(static)
        for (int a = 0; a < rh; ++a)
            for (int ox = 0; ox < ow; ++ox) {
                int x = x0 + ox;
                for (int q = 0; q < 4; ++q) {
                    double acc = 0.0;
                    for (int b = imax(rx0, x - R); b <= imin(rx1 - 1, x + R); ++b)
                        acc += g[b - x + R] * P[q * rsz + (size_t)a * rw + (b - rx0)];
                    Hp[q * hsz + (size_t)a * ow + ox] = acc;
                }
            }
        /* step 2b: columns, then step 3: demodulate and accumulate */
        #pragma omp parallel for schedule(static)
        for (int oy = 0; oy < oh; ++oy)
            for (int ox = 0; ox < ow; ++ox) {
                int y = y0 + oy;
                double fb[4];
                for (int q = 0; q < 4; ++q) {
                    double acc = 0.0;
                    for (int a = imax(ry0, y - R); a <= imin(ry1 - 1, y + R); ++a)
                        acc += g[a - y + R] * Hp[q * hsz + (size_t)(a - ry0) * ow + ox];
                    fb[q] = acc;
                }
                double v = f[(size_t)y * W + (x0 + ox)];
                double c = cos(om * v), s = sin(om * v);
                num[(size_t)oy * ow + ox] += wn * (c * fb[0] + s * fb[1]);
                den[(size_t)oy * ow + ox] += wn * (c * fb[2] + s * fb[3]);
            }
    }
    long nfb = 0;
    for (int oy = 0; oy < oh; ++oy)
        for (int ox = 0; ox < ow; ++ox) {
            int y = y0 + oy, x = x0 + ox;
            size_t k = (size_t)oy * ow + ox;
            double mass = clipped_mass(g, R, H, W, y, x);
            double v;
            if (den[k] > 1e-6 * mass) v = num[k] / den[k];
            else { v = f[(size_t)y * W + x]; ++nfb; }
            out[(size_t)y * W + x] = v;
            if (num_out) num_out[(size_t)y * W + x] = num[k];
            if (den_out) den_out[(size_t)y * W + x] = den[k];
        }
    free(P); free(Hp); free(num); free(den); free(lw);
    return nfb;
}

/* ------------------------------------------------------------------ */
/* Recursive Gaussian (Young and van Vliet, Signal Processing 44, 1995) */
/* as the "recursive O(1)" spatial filter that Sec. 1.2 allows in place */
/* of the truncated Gaussian.  The recursion is the published method;   */
/* the paper itself names no particular recursive filter.               */
/* ------------------------------------------------------------------ */

/* Coefficients of the third-order recursion for scale sigma (>= 0.5):
 *   q  = 0.98711 sigma - 0.96330                   for sigma >= 2.5,
 *   q  = 3.97156 - 4.14554 sqrt(1 - 0.26891 sigma) for 0.5 <= sigma < 2.5,
 *   b0 = 1.57825 + 2.44413 q + 1.4281 q^2 + 0.422205 q^3,
 *   b1 = 2.44413 q + 2.85619 q^2 + 1.26661 q^3,
 *   b2 = -(1.4281 q^2 + 1.26661 q^3),
 *   b3 = 0.422205 q^3,
 *   B  = 1 - (b1 + b2 + b3) / b0  (unit gain at zero frequency).
 * c[0] = B and c[k] = bk / b0 for k = 1, 2, 3. */
void orc_yvv_coeffs(double sigma, double *c)
{
    double q;
    if (sigma >= 2.5) q = 0.98711 * sigma - 0.96330;
    else q = 3.97156 - 4.14554 * sqrt(1.0 - 0.26891 * sigma);
    const double q2 = q * q, q3 = q2 * q;
    const double b0 = 1.57825 + 2.44413 * q + 1.4281 * q2 + 0.422205 * q3;
    const double b1 = 2.44413 * q + 2.85619 * q2 + 1.26661 * q3;
    const double b2 = -(1.4281 * q2 + 1.26661 * q3);
    const double b3 = 0.422205 * q3;
    c[0] = 1.0 - (b1 + b2 + b3) / b0;
    c[1] = b1 / b0;
    c[2] = b2 / b0;
    c[3] = b3 / b0;
}

/* Length of the zero extension that stands for an infinite one: the
 * recursion's impulse response decays like |pole|^d with 1 - |pole| of
 * order 1/sigma, so 60 sigma + 64 samples leave a tail far below double
 * precision for every sigma (the tests check that doubling it changes
 * nothing). */
int orc_yvv_margin(double sigma) { return (int)ceil(60.0 * sigma) + 64; }

/* The filter on one line of n samples x[0], x[stride], ... (in place),
 * the line extended by zeros on both sides:
 *   causal      w[i] = B x[i] + c1 w[i-1] + c2 w[i-2] + c3 w[i-3],
 *               zero state before i = 0, run on through L zeros past the end;
 *   anti-causal y[i] = B w[i] + c1 y[i+1] + c2 y[i+2] + c3 y[i+3],
 *               zero state after i = n - 1 + L, run back to i = 0.
 * (Zeros before the line leave the causal state at zero, so only the right
 * extension needs samples.)  w holds n + L doubles of scratch. */
static void yvv_line(double *x, int n, long stride, const double *c, int L, double *w)
{
    const double B = c[0];
    double w1 = 0.0, w2 = 0.0, w3 = 0.0;
    for (int i = 0; i < n + L; ++i) {
        const double xi = i < n ? x[(long)i * stride] : 0.0;
        const double wi = B * xi + c[1] * w1 + c[2] * w2 + c[3] * w3;
        w[i] = wi;
        w3 = w2; w2 = w1; w1 = wi;
    }
    double y1 = 0.0, y2 = 0.0, y3 = 0.0;
    for (int i = n + L - 1; i >= 0; --i) {
        const double yi = B * w[i] + c[1] * y1 + c[2] * y2 + c[3] * y3;
        if (i < n) x[(long)i * stride] = yi;
        y3 = y2; y2 = y1; y1 = yi;
    }
}

/* Two-dimensional filter: every row, then every column, of the H x W image
 * in (margin L; L < 0 takes orc_yvv_margin(sigma)), written to out. */
void orc_yvv_2d(const double *in, double *out, int H, int W, double sigma, int L)
{
    double c[4];
    orc_yvv_coeffs(sigma, c);
    if (L < 0) L = orc_yvv_margin(sigma);
    if (out != in) memcpy(out, in, sizeof(double) * (size_t)H * W);
    #pragma omp parallel
    {
        double *w = (double *)malloc(sizeof(double) * (size_t)((H > W ? H : W) + L));
        #pragma omp for schedule(static)
        for (int i = 0; i < H; ++i) yvv_line(out + (size_t)i * W, W, 1, c, L, w);
        #pragma omp for schedule(static)
        for (int j = 0; j < W; ++j) yvv_line(out + j, H, W, c, L, w);
        free(w);
    }
}

/* Impulse response h[d + half], d = -half..half: the filtered line of
 * 2 half + 1 samples with a unit sample in the middle. */
void orc_yvv_impulse(double sigma, int half, double *h)
{
    double c[4];
    orc_yvv_coeffs(sigma, c);
    const int n = 2 * half + 1, L = orc_yvv_margin(sigma);
    double *w = (double *)malloc(sizeof(double) * (size_t)(n + L));
    for (int i = 0; i < n; ++i) h[i] = 0.0;
    h[half] = 1.0;
    yvv_line(h, n, 1, c, L, w);
    free(w);
}

/* SHIFTABLE-BF with the recursive filter in step 2, one kernel (N, M) for
 * the whole image (every output depends on every pixel, so blocks do not
 * apply).  For each kept n (no folding): planes f c, f s, c, s over the
 * image; each filtered by orc_yvv_2d; num += w_n (c Fc + s Fs),
 * den += w_n (c Gc + s Gs).  Guard: den <= 1e-6 Y(1_Omega)(x) -> f(x),
 * Y(1_Omega) being the same filter applied to the indicator of the image.
 * Returns the number of guarded pixels. */
long orc_shiftable_yvv(const double *f, int H, int W, double sigma_s, int N, int M,
                       double sigma_r, double *out, double *num_out, double *den_out)
{
    const size_t n_px = (size_t)H * W;
    double *P = (double *)malloc(sizeof(double) * 4 * n_px);
    double *num = (double *)calloc(n_px, sizeof(double));
    double *den = (double *)calloc(n_px, sizeof(double));
    double *mass = (double *)malloc(sizeof(double) * n_px);
    double *lw = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    orc_log_weights(N, lw);
    const double scale = sqrt((double)N) * sigma_r;
    for (int n = M; n <= N - M; ++n) {
        const double wn = exp(lw[n]);
        const double om = (double)(2 * n - N) / scale;
        for (size_t k = 0; k < n_px; ++k) {
            const double v = f[k], c = cos(om * v), s = sin(om * v);
            P[k] = v * c; P[n_px + k] = v * s; P[2 * n_px + k] = c; P[3 * n_px + k] = s;
        }
        for (int q = 0; q < 4; ++q) orc_yvv_2d(P + q * n_px, P + q * n_px, H, W, sigma_s, -1);
        for (size_t k = 0; k < n_px; ++k) {
            const double v = f[k], c = cos(om * v), s = sin(om * v);
            num[k] += wn * (c * P[k] + s * P[n_px + k]);
            den[k] += wn * (c * P[2 * n_px + k] + s * P[3 * n_px + k]);
        }
    }
    for (size_t k = 0; k < n_px; ++k) mass[k] = 1.0;
    orc_yvv_2d(mass, mass, H, W, sigma_s, -1);
    long nfb = 0;
    for (size_t k = 0; k < n_px; ++k) {
        if (den[k] > 1e-6 * mass[k]) out[k] = num[k] / den[k];
        else { out[k] = f[k]; ++nfb; }
        if (num_out) num_out[k] = num[k];
        if (den_out) den_out[k] = den[k];
    }
    free(P); free(num); free(den); free(mass); free(lw);
    return nfb;
}

/* ------------------------------------------------------------------ */
/* Direct sums (eq. (BF) with the Gaussian or with phi_eps).           */
/* ------------------------------------------------------------------ */

/* Direct filter at npts pixels (ys[i], xs[i]) with the range kernel phi_eps
 * of (Ns[i], Ms[i]) (per point, so that per-tile parameters can be used):
 *   out = sum_y g(x-y) phi(f(y)-f(x)) f(y) / sum_y g(x-y) phi(f(y)-f(x)),
 * y over the clipped window, with the same denominator guard as above.
 * If gauss != 0 the range kernel is exp(-s^2/(2 sigma_r^2)) instead. */
long orc_direct_points(const double *f, int H, int W, const double *g, int R,
                       const int *Ns, const int *Ms, double sigma_r, int gauss,
                       const int *ys, const int *xs, int npts,
                       double *out, double *num_out, double *den_out)
{
    long nfb = 0;
    #pragma omp parallel reduction(+ : nfb)
    {
        double *lw = NULL; int lwN = -1;
        double *wk = NULL, *omk = NULL; int nk = 0;
        #pragma omp for schedule(dynamic, 4)
        for (int p = 0; p < npts; ++p) {
            const int i = ys[p], j = xs[p];
            const int N = Ns[p], M = Ms[p];
            if (!gauss && N != lwN) {
                free(lw); free(wk); free(omk);
                lw = (double *)malloc(sizeof(double) * (size_t)(N + 1));
                orc_log_weights(N, lw);
                nk = N - 2 * M + 1;
                wk = (double *)malloc(sizeof(double) * (size_t)nk);
                omk = (double *)malloc(sizeof(double) * (size_t)nk);
                for (int n = M; n <= N - M; ++n) {
                    wk[n - M] = exp(lw[n]);
                    omk[n - M] = (double)(2 * n - N) / (sqrt((double)N) * sigma_r);
                }
                lwN = N;
            }
            const double fx = f[(size_t)i * W + j];
            double num = 0.0, den = 0.0;
            for (int a = imax(0, i - R); a <= imin(H - 1, i + R); ++a)
                for (int b = imax(0, j - R); b <= imin(W - 1, j + R); ++b) {
                    const double fy = f[(size_t)a * W + b];
                    const double s = fy - fx;
                    double phi = 0.0;
                    if (gauss) phi = exp(-s * s / (2.0 * sigma_r * sigma_r));
                    else
                        for (int k = 0; k < nk; ++k) phi += wk[k] * cos(omk[k] * s);
                    const double wgt = g[a - i + R] * g[b - j + R] * phi;
                    num += wgt * fy;
                    den += wgt;
                }
            const double mass = clipped_mass(g, R, H, W, i, j);
            if (den > 1e-6 * mass) out[p] = num / den;
            else { out[p] = fx; ++nfb; }
            if (num_out) num_out[p] = num;
            if (den_out) den_out[p] = den;
        }
        free(lw); free(wk); free(omk);
    }
    return nfb;
}

/* ------------------------------------------------------------------ */
/* Gradient of L = sum_x u(x) out(x) with respect to f (not in the      */
/* paper; derived from eqs. (f1)-(f2), T, N, M held fixed).            */
/* ------------------------------------------------------------------ */

/* Shiftable form, one kernel (N, M) for the block [y0,y1)x[x0,x1) of
 * outputs.  Inputs: a = u/den and b = -a*out at the block's pixels (zero
 * where the guard fired; the caller adds u there).  Writes the gradient
 * contribution of this block into grad (accumulated, full image).
 * For each kept n, with c, s = cos, sin(w_n f) and G(h) = g * h (clipped):
 *   grad(z) += w_n [ c G(ac) + s G(as) - w f (s G(ac) - c G(as))
 *                    - w (s G(bc) - c G(bs))
 *                    + w a (c G(fs) - s G(fc)) + w b (c G(s) - s G(c)) ],
 * the last two terms only at z inside the block (centre terms). */
static void sep_filter(const double *in, double *tmp, double *outp, int H, int W,
                       const double *g, int R)
{
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double acc = 0.0;
            for (int b = imax(0, j - R); b <= imin(W - 1, j + R); ++b)
                acc += g[b - j + R] * in[(size_t)i * W + b];
            tmp[(size_t)i * W + j] = acc;
        }
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            double acc = 0.0;
            for (int a = imax(0, i - R); a <= imin(H - 1, i + R); ++a)
                acc += g[a - i + R] * tmp[(size_t)a * W + j];
            outp[(size_t)i * W + j] = acc;
        }
}

void orc_grad_shiftable_block(const double *f, int H, int W, const double *g, int R,
                              int N, int M, double sigma_r,
                              int y0, int y1, int x0, int x1,
                              const double *a_blk, const double *b_blk, double *grad)
{
    const size_t HW = (size_t)H * W;
    double *buf = (double *)malloc(sizeof(double) * HW * 13);
    double *ac = buf, *as = buf + HW, *bc = buf + 2 * HW, *bs = buf + 3 * HW;
    double *Gac = buf + 4 * HW, *Gas = buf + 5 * HW, *Gbc = buf + 6 * HW, *Gbs = buf + 7 * HW;
    double *fc = buf + 8 * HW, *fs = buf + 9 * HW, *cc = buf + 10 * HW, *ss = buf + 11 * HW;
    double *tmp = buf + 12 * HW;
    double *lw = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    orc_log_weights(N, lw);
    const double scale = sqrt((double)N) * sigma_r;
    for (int n = M; n <= N - M; ++n) {
        const double wn = exp(lw[n]);
        const double om = (double)(2 * n - N) / scale;
        memset(ac, 0, sizeof(double) * HW * 4);
        for (int i = y0; i < y1; ++i)
            for (int j = x0; j < x1; ++j) {
                size_t k = (size_t)i * W + j;
                double c = cos(om * f[k]), s = sin(om * f[k]);
                ac[k] = a_blk[k] * c; as[k] = a_blk[k] * s;
                bc[k] = b_blk[k] * c; bs[k] = b_blk[k] * s;
            }
        sep_filter(ac, tmp, Gac, H, W, g, R);
        sep_filter(as, tmp, Gas, H, W, g, R);
        sep_filter(bc, tmp, Gbc, H, W, g, R);
        sep_filter(bs, tmp, Gbs, H, W, g, R);
        #pragma omp parallel for schedule(static)
        for (size_t k = 0; k < HW; ++k) {
            double c = cos(om * f[k]), s = sin(om * f[k]);
            fc[k] = f[k] * c; fs[k] = f[k] * s; cc[k] = c; ss[k] = s;
        }
        /* forward planes filtered (needed only for the centre terms) */
        double *Gfc = (double *)malloc(sizeof(double) * HW * 4);
        double *Gfs = Gfc + HW, *Gc = Gfc + 2 * HW, *Gs = Gfc + 3 * HW;
        sep_filter(fc, tmp, Gfc, H, W, g, R);
        sep_filter(fs, tmp, Gfs, H, W, g, R);
        sep_filter(cc, tmp, Gc, H, W, g, R);
        sep_filter(ss, tmp, Gs, H, W, g, R);
        #pragma omp parallel for schedule(static)
        for (int i = 0; i < H; ++i)
            for (int j = 0; j < W; ++j) {
                size_t k = (size_t)i * W + j;
                double c = cc[k], s = ss[k], fz = f[k];
                double v = c * Gac[k] + s * Gas[k]
                         - om * fz * (s * Gac[k] - c * Gas[k])
                         - om * (s * Gbc[k] - c * Gbs[k]);
                if (i >= y0 && i < y1 && j >= x0 && j < x1)
                    v += om * a_blk[k] * (c * Gfs[k] - s * Gfc[k])
                       + om * b_blk[k] * (c * Gs[k] - s * Gc[k]);
                grad[k] += wn * v;
            }
        free(Gfc);
    }
    free(buf); free(lw);
}

/* Direct form of the same gradient, at npts pixels z, for a single kernel
 * (N, M) used at every output x (global parameters):
 *   grad(z) = sum_{x in win(z)} g(x-z) [ a(x) (phi(f_z-f_x) + f_z phi'(f_z-f_x))
 *                                       + b(x) phi'(f_z-f_x) ]
 *           - a(z) sum_y g(z-y) f_y phi'(f_y-f_z) - b(z) sum_y g(z-y) phi'(f_y-f_z),
 * phi' = -sum_n w_n w_n' sin(w_n s).  a, b full images (zero at guarded
 * pixels; the caller adds u there). */
void orc_grad_direct_points(const double *f, int H, int W, const double *g, int R,
                            int N, int M, double sigma_r, const double *a, const double *b,
                            const int *zs_y, const int *zs_x, int npts, double *out)
{
    double *lw = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    orc_log_weights(N, lw);
    const int nk = N - 2 * M + 1;
    double *wk = (double *)malloc(sizeof(double) * (size_t)nk);
    double *omk = (double *)malloc(sizeof(double) * (size_t)nk);
    for (int n = M; n <= N - M; ++n) {
        wk[n - M] = exp(lw[n]);
        omk[n - M] = (double)(2 * n - N) / (sqrt((double)N) * sigma_r);
    }
    #pragma omp parallel for schedule(dynamic, 4)
    for (int p = 0; p < npts; ++p) {
        const int zi = zs_y[p], zj = zs_x[p];
        const size_t zk = (size_t)zi * W + zj;
        const double fz = f[zk];
        double acc = 0.0;
        for (int i = imax(0, zi - R); i <= imin(H - 1, zi + R); ++i)
            for (int j = imax(0, zj - R); j <= imin(W - 1, zj + R); ++j) {
                const size_t k = (size_t)i * W + j;
                const double fy = f[k];
                const double gw = g[i - zi + R] * g[j - zj + R];
                double ph1 = 0.0, dph1 = 0.0, dph2 = 0.0;
                for (int q = 0; q < nk; ++q) {
                    ph1 += wk[q] * cos(omk[q] * (fz - fy));
                    dph1 += -wk[q] * omk[q] * sin(omk[q] * (fz - fy));
                    dph2 += -wk[q] * omk[q] * sin(omk[q] * (fy - fz));
                }
                /* neighbour part: x = (i,j) is an output whose window holds z */
                acc += gw * (a[k] * (ph1 + fz * dph1) + b[k] * dph1);
                /* centre part: y = (i,j) is a neighbour of the output z */
                acc -= gw * (a[zk] * fy * dph2 + b[zk] * dph2);
            }
        out[p] = acc;
    }
    free(lw); free(wk); free(omk);
}

/* ------------------------------------------------------------------ */
/* Raised-polynomial range kernel (Sec. 1.3, eqs. (RP) and (RPconv)):  */
/*   phi(s) = (1 - s^2 / (2 N sigma_r^2))^N,                          */
/* which tends to exp(-s^2 / (2 sigma_r^2)) as N grows and is positive */
/* and monotone on [-T, T] when N >= N0 = 0.5 (T / sigma_r)^2.         */
/* ------------------------------------------------------------------ */

/* N = max(1, ceil(N0)), N0 = T^2 / (2 sigma_r^2). */
int orc_poly_order(double T, double sigma_r)
{
    double n0 = (T * T) / (2.0 * sigma_r * sigma_r);
    int N = (int)ceil(n0);
    return N < 1 ? 1 : N;
}

/* phi(s) at ns points. */
void orc_poly_phi(const double *s, int ns, int N, double sigma_r, double *out)
{
    for (int i = 0; i < ns; ++i)
        out[i] = pow(1.0 - s[i] * s[i] / (2.0 * (double)N * sigma_r * sigma_r), (double)N);
}

/* T of the polynomial kernel per tile: the range (max - min) of f over the
 * tile grown by R on every side and clipped to the image, so that every
 * pair of values a pixel of the tile meets (and every pair the polynomial
 * expansion over that region represents) lies within [-T, T].  A single
 * tile covering the image gives the image's range.  Returned in double
 * (the difference of two image values is exact). */
void orc_range_tiles(const double *f, int H, int W, int R, int tile_h, int tile_w, double *T)
{
    int ty = (H + tile_h - 1) / tile_h, tx = (W + tile_w - 1) / tile_w;
    for (int a = 0; a < ty; ++a)
        for (int b = 0; b < tx; ++b) {
            int i0 = imax(0, a * tile_h - R), i1 = imin(H, (a + 1) * tile_h + R);
            int j0 = imax(0, b * tile_w - R), j1 = imin(W, (b + 1) * tile_w + R);
            double mx = -INFINITY, mn = INFINITY;
            for (int i = i0; i < i1; ++i)
                for (int j = j0; j < j1; ++j) {
                    mx = fmax(mx, f[(size_t)i * W + j]);
                    mn = fmin(mn, f[(size_t)i * W + j]);
                }
            T[a * tx + b] = mx - mn;
        }
}

/* Direct filter of eq. (BF) with the raised-polynomial range kernel of
 * order Ns[p] at the points (ys[p], xs[p]), clipped window, with the same
 * denominator guard as the cosine kernel.  Returns the guarded count. */
long orc_poly_direct_points(const double *f, int H, int W, const double *g, int R,
                            const int *Ns, double sigma_r, const int *ys, const int *xs, int npts,
                            double *out, double *num_out, double *den_out)
{
    long nfb = 0;
    #pragma omp parallel for schedule(dynamic, 4) reduction(+ : nfb)
    for (int p = 0; p < npts; ++p) {
        const int i = ys[p], j = xs[p], N = Ns[p];
        const double a = 2.0 * (double)N * sigma_r * sigma_r;
        const double fx = f[(size_t)i * W + j];
        double num = 0.0, den = 0.0;
        for (int y = imax(0, i - R); y <= imin(H - 1, i + R); ++y)
            for (int x = imax(0, j - R); x <= imin(W - 1, j + R); ++x) {
                const double fy = f[(size_t)y * W + x];
                const double s = fy - fx;
                const double phi = pow(1.0 - s * s / a, (double)N);
                const double wgt = g[y - i + R] * g[x - j + R] * phi;
                num += wgt * fy;
                den += wgt;
            }
        const double mass = clipped_mass(g, R, H, W, i, j);
        if (den > 1e-6 * mass) out[p] = num / den;
        else { out[p] = fx; ++nfb; }
        if (num_out) num_out[p] = num;
        if (den_out) den_out[p] = den;
    }
    return nfb;
}

/* ------------------------------------------------------------------ */
/* Non-local means with a small patch (Sec. 6, eqs. (NL1), (NL2)):     */
/*   NL1(x) = sum_y s(y) f(x-y) g(f(x+u_1) - f(x-y+u_1), ...,           */
/*                              f(x+u_p) - f(x-y+u_p)),                 */
/*   NL2(x) = the same without f(x-y),   out = NL1 / NL2,               */
/* g a product of one-dimensional Gaussians of width sigma_r, each      */
/* approximated by phi_eps (eq. (approx)) with the N, M of T (eq.       */
/* (bound)).  s is the spatial weight (the box of the paper's sums, or  */
/* the Gaussian), y over the clipped window.  Patch values f(z + u_i)   */
/* outside the image are taken at the nearest in-image pixel.           */
/* ------------------------------------------------------------------ */

static double f_clamped(const double *f, int H, int W, int y, int x)
{
    y = imin(imax(y, 0), H - 1);
    x = imin(imax(x, 0), W - 1);
    return f[(size_t)y * W + x];
}

/* Direct sums at npts points.  uy, ux: the p patch offsets (u_1 = 0 first).
 * gauss != 0: the range kernel is the product of exact Gaussians. */
long orc_nlm_direct_points(const double *f, int H, int W, const double *g, int R,
                           int N, int M, double sigma_r, int gauss,
                           const int *uy, const int *ux, int p,
                           const int *ys, const int *xs, int npts,
                           double *out, double *num_out, double *den_out)
{
    long nfb = 0;
    int nk = N - 2 * M + 1;
    double *lw = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    double *wk = (double *)malloc(sizeof(double) * (size_t)nk);
    double *omk = (double *)malloc(sizeof(double) * (size_t)nk);
    orc_log_weights(N, lw);
    for (int n = M; n <= N - M; ++n) {
        wk[n - M] = exp(lw[n]);
        omk[n - M] = (double)(2 * n - N) / (sqrt((double)N) * sigma_r);
    }
    #pragma omp parallel for schedule(dynamic, 4) reduction(+ : nfb)
    for (int q = 0; q < npts; ++q) {
        const int i = ys[q], j = xs[q];
        double num = 0.0, den = 0.0;
        for (int a = imax(0, i - R); a <= imin(H - 1, i + R); ++a)
            for (int b = imax(0, j - R); b <= imin(W - 1, j + R); ++b) {
                double kern = 1.0;
                for (int c = 0; c < p; ++c) {
                    const double s = f_clamped(f, H, W, i + uy[c], j + ux[c]) -
                                     f_clamped(f, H, W, a + uy[c], b + ux[c]);
                    double phi = 0.0;
                    if (gauss) phi = exp(-s * s / (2.0 * sigma_r * sigma_r));
                    else
                        for (int k = 0; k < nk; ++k) phi += wk[k] * cos(omk[k] * s);
                    kern *= phi;
                }
                const double wgt = g[a - i + R] * g[b - j + R] * kern;
                num += wgt * f[(size_t)a * W + b];
                den += wgt;
            }
        const double mass = clipped_mass(g, R, H, W, i, j);
        if (den > 1e-6 * mass) out[q] = num / den;
        else { out[q] = f[(size_t)i * W + j]; ++nfb; }
        if (num_out) num_out[q] = num;
        if (den_out) den_out[q] = den;
    }
    free(lw); free(wk); free(omk);
    return nfb;
}

/* The shiftable form of the same sums (the O(1) algorithm of the paper's
 * Sec. 6): expanding every phi_eps(s_i) = sum_n w_n exp(j omega_n s_i)
 * gives, for each multi-index nu = (n_1, ..., n_p) in [M, N-M]^p, the
 * weight w_nu = prod_i w_{n_i} and the phase image theta_nu(z) = sum_i
 * omega_{n_i} f(z + u_i); then
 *   NL2(x) = sum_nu w_nu [cos theta_nu(x) (s * cos theta_nu)(x)
 *                        + sin theta_nu(x) (s * sin theta_nu)(x)],
 * and NL1 likewise with the planes f cos theta_nu, f sin theta_nu (f at the
 * window pixel).  Every multi-index is visited (no folding). */
long orc_nlm_shiftable(const double *f, int H, int W, const double *g, int R,
                       int N, int M, double sigma_r, const int *uy, const int *ux, int p,
                       double *out, double *num_out, double *den_out)
{
    const size_t HW = (size_t)H * W;
    int nk = N - 2 * M + 1;
    double *lw = (double *)malloc(sizeof(double) * (size_t)(N + 1));
    orc_log_weights(N, lw);
    double *buf = (double *)malloc(sizeof(double) * HW * 11);
    double *th = buf, *P = buf + HW, *Q = buf + 5 * HW, *tmp = buf + 9 * HW;
    double *num = (double *)calloc(HW, sizeof(double)), *den = (double *)calloc(HW, sizeof(double));
    int *idx = (int *)calloc((size_t)p, sizeof(int));
    const double scale = sqrt((double)N) * sigma_r;
    long total = 1;
    for (int c = 0; c < p; ++c) total *= nk;
    for (long t = 0; t < total; ++t) {
        long r = t;
        double wnu = 1.0;
        for (int c = 0; c < p; ++c) {
            idx[c] = M + (int)(r % nk);
            r /= nk;
            wnu *= exp(lw[idx[c]]);
        }
        for (int i = 0; i < H; ++i)
            for (int j = 0; j < W; ++j) {
                double v = 0.0;
                for (int c = 0; c < p; ++c)
                    v += (double)(2 * idx[c] - N) / scale * f_clamped(f, H, W, i + uy[c], j + ux[c]);
                th[(size_t)i * W + j] = v;
            }
        for (size_t k = 0; k < HW; ++k) {
            const double c = cos(th[k]), s = sin(th[k]);
            P[k] = f[k] * c; P[HW + k] = f[k] * s; P[2 * HW + k] = c; P[3 * HW + k] = s;
        }
        for (int q = 0; q < 4; ++q) sep_filter(P + q * HW, tmp, Q + q * HW, H, W, g, R);
        for (size_t k = 0; k < HW; ++k) {
            const double c = cos(th[k]), s = sin(th[k]);
            num[k] += wnu * (c * Q[k] + s * Q[HW + k]);
            den[k] += wnu * (c * Q[2 * HW + k] + s * Q[3 * HW + k]);
        }
    }
    long nfb = 0;
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) {
            const size_t k = (size_t)i * W + j;
            const double mass = clipped_mass(g, R, H, W, i, j);
            if (den[k] > 1e-6 * mass) out[k] = num[k] / den[k];
            else { out[k] = f[k]; ++nfb; }
            if (num_out) num_out[k] = num[k];
            if (den_out) den_out[k] = den[k];
        }
    free(lw); free(buf); free(num); free(den); free(idx);
    return nfb;
}
