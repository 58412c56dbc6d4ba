// K3-yvv: SHIFTABLE-BF (Sec. 1.2) with a recursive Gaussian in step 2.
//
// Sec. 1.2 lets the Gaussian filtering of the modulated planes be done by an
// O(1) recursive filter.  This one is the third-order recursion of Young and
// van Vliet (Signal Processing 44, 1995): a causal pass and an anti-causal
// pass with the same poles, on the plane extended by zeros without limit,
// rows and then columns.  Its cost per sample does not depend on sigma_s.
//
// Form of the recursion.  The cascade (causal, then anti-causal) has the
// symmetric impulse response h[n] = sum_i c_i p_i^|n| over its three poles
// (one real, one complex pair), so the same filter is the sum of a causal
// part sum_{m>=0} h[m] x[n-m] and an anti-causal part sum_{m>=1} h[m] x[n+m],
// each a first-order section per pole:
//   causal       u_i[n] = p_i u_i[n-1] + x[n],   y+[n] = sum_i c_i u_i[n]
//   anti-causal  v_i[n] = p_i v_i[n+1] + x[n],   y-[n] = sum_i c_i p_i v_i[n+1]
// both starting from zero state at the ends of the line, which is exact for
// the zero extension (no margin).  First-order sections keep the FP32
// rounding small (the gain of one section is 1 / (1 - |p|)); the direct
// third-order form would amplify it by the whole filter's DC gain
// b0 / (b0 - b1 - b2 - b3), two orders of magnitude more at sigma_s = 8.
//
// Because the filtered planes are demodulated and summed linearly, the
// column pass never materialises its output: the down sweep adds the causal
// part's contribution to num and den, the up sweep the anti-causal part's.
//
// Kernels, per pass of C terms (C in {8, 16, 32}; lanes = 32 / C lines x C
// terms, term k = pass * C + lane % C, the zero frequency as term F with
// omega = 0 and weight w0):
//   k_yvv_rows  one warp per 32 / C rows: planes f'c, f's, c, s of each term
//               (f' = f - value_range / 2), causal sweep writing the row-
//               filtered planes to P[y][x][term][4], anti-causal sweep adding
//               into them;
//   k_yvv_cols  one warp per 32 / C columns: down and up sweeps over P,
//               demodulation with the term's cos, sin at the output pixel, a
//               shuffle sum over the C terms, accumulated into (num, den);
//   k_yvv_final num / den + value_range / 2, with the denominator guard
//               against 1e-6 times the filter of the image's indicator
//               (separable: mass_y[y] mass_x[x]).
// The number of passes follows the plan's cap on N (the host never reads
// the device's N); passes beyond the set's terms return at once.
#include <complex>
#include <math.h>

#include "bf_fir32.cuh"

namespace bf {

namespace {

constexpr int kWarpsPerCta = 4;

struct Sec {
    float a, re, im;      // real-pole state, complex-pole state
};

// u <- p u + x for the real pole and the complex pole.
__device__ __forceinline__ void sec_update(Sec& s, float x, const YvvCoef& k)
{
    s.a = fmaf(k.P0, s.a, x);
    const float re = fmaf(k.Pr, s.re, fmaf(-k.Pi, s.im, x));
    const float im = fmaf(k.Pr, s.im, k.Pi * s.re);
    s.re = re;
    s.im = im;
}

// c0 u_0 + 2 Re(c1 u_1): the causal output after the update.
__device__ __forceinline__ float sec_causal_out(const Sec& s, const YvvCoef& k)
{
    return fmaf(k.C0, s.a, fmaf(k.Cr, s.re, -k.Ci * s.im));
}

// c0 p0 v_0 + 2 Re(c1 p1 v_1): the anti-causal output, before the update.
__device__ __forceinline__ float sec_anti_out(const Sec& s, const YvvCoef& k)
{
    return fmaf(k.D0, s.a, fmaf(k.Dr, s.re, -k.Di * s.im));
}

__device__ __forceinline__ void term_of(const YvvArgs& a, const SetHdr& hd, int k, float& om_hi,
                                        float& om_lo, float& Wk)
{
    om_hi = om_lo = Wk = 0.f;
    if (k < hd.F) {
        const Pair p = a.pairs[k];
        om_hi = p.om_hi;
        om_lo = p.om_lo;
        Wk = p.W;
    } else if (k == hd.F && hd.z) {
        Wk = hd.w0;        // zero frequency: cos = 1, sin = 0
    }
}

__device__ __forceinline__ void planes_at(float v, float om_hi, float om_lo, float (&in)[4])
{
    float c, s;
    fir32::phase_cs(v, om_hi, om_lo, c, s);
    in[0] = v * c;
    in[1] = v * s;
    in[2] = c;
    in[3] = s;
}

template <int C>
__global__ void __launch_bounds__(32 * kWarpsPerCta)
k_yvv_rows(YvvArgs a, int pass)
{
    constexpr int LPW = 32 / C;                    // lines per warp
    const int lane = threadIdx.x & 31;
    const int slot = lane % C;
    const int y = (blockIdx.x * kWarpsPerCta + (threadIdx.x >> 5)) * LPW + lane / C;
    const SetHdr hd = a.hdr[0];
    const int nterms = hd.F < 0 ? 0 : hd.F + hd.z;
    if (pass * C >= nterms || y >= a.H) return;
    const int k = pass * C + slot;
    const bool act = k < nterms;
    float om_hi, om_lo, Wk;
    term_of(a, hd, k, om_hi, om_lo, Wk);
    const YvvCoef cf = a.coef;
    const float* frow = a.f + (size_t)y * a.f_pitch;
    float4* P = a.P + (size_t)y * a.W * C + slot;  // (y, x, slot) at P[x * C]
    const int W = a.W;

    Sec st[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) st[q] = Sec{0.f, 0.f, 0.f};
    // causal sweep: write y+
#pragma unroll 4
    for (int x = 0; x < W; ++x) {
        float in[4];
        planes_at(__ldg(frow + x) - a.c0, om_hi, om_lo, in);
        float o[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            sec_update(st[q], in[q], cf);
            o[q] = sec_causal_out(st[q], cf);
        }
        if (act) P[(size_t)x * C] = make_float4(o[0], o[1], o[2], o[3]);
    }
    // anti-causal sweep: add y-, in chunks whose loads are issued together
#pragma unroll
    for (int q = 0; q < 4; ++q) st[q] = Sec{0.f, 0.f, 0.f};
    constexpr int kChunk = 8;
    for (int x1 = W - 1; x1 >= 0; x1 -= kChunk) {
        float4 cur[kChunk];
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
            const int x = x1 - j;
            cur[j] = (act && x >= 0) ? P[(size_t)x * C] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
            const int x = x1 - j;
            if (x < 0) break;
            float4 t = cur[j];
            t.x += sec_anti_out(st[0], cf);
            t.y += sec_anti_out(st[1], cf);
            t.z += sec_anti_out(st[2], cf);
            t.w += sec_anti_out(st[3], cf);
            if (act) P[(size_t)x * C] = t;
            float in[4];
            planes_at(__ldg(frow + x) - a.c0, om_hi, om_lo, in);
#pragma unroll
            for (int q = 0; q < 4; ++q) sec_update(st[q], in[q], cf);
        }
    }
}

template <int C>
__device__ __forceinline__ void reduce_terms(float& nu, float& de)
{
#pragma unroll
    for (int o = C / 2; o >= 1; o >>= 1) {
        nu += __shfl_xor_sync(0xffffffffu, nu, o);
        de += __shfl_xor_sync(0xffffffffu, de, o);
    }
}

template <int C>
__global__ void __launch_bounds__(32 * kWarpsPerCta)
k_yvv_cols(YvvArgs a, int pass)
{
    constexpr int LPW = 32 / C;
    const int lane = threadIdx.x & 31;
    const int slot = lane % C;
    const int x = (blockIdx.x * kWarpsPerCta + (threadIdx.x >> 5)) * LPW + lane / C;
    const SetHdr hd = a.hdr[0];
    const int nterms = hd.F < 0 ? 0 : hd.F + hd.z;
    if (pass * C >= nterms) return;               // uniform over the grid
    // lanes past the last column stay for the shuffles
    if ((blockIdx.x * kWarpsPerCta + (threadIdx.x >> 5)) * LPW >= a.W) return;  // whole warp out
    const bool xin = x < a.W;
    const int k = pass * C + slot;
    const bool act = xin && k < nterms;
    float om_hi, om_lo, Wk;
    term_of(a, hd, k, om_hi, om_lo, Wk);
    if (!act) Wk = 0.f;
    const YvvCoef cf = a.coef;
    const int H = a.H, W = a.W;
    const int xc = xin ? x : 0;
    const float4* P = a.P + (size_t)xc * C + slot;   // (y, x, slot) at P[y * W * C]
    const size_t pstride = (size_t)W * C;
    const float* fcol = a.f + xc;
    float2* ND = a.nd + xc;
    const bool writer = xin && slot == 0;
    const bool first = pass == 0;
    constexpr int kChunk = 8;

    Sec st[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) st[q] = Sec{0.f, 0.f, 0.f};
    // down sweep: causal part
    for (int y0 = 0; y0 < H; y0 += kChunk) {
        float4 cur[kChunk];
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
            const int y = y0 + j;
            cur[j] = (act && y < H) ? P[(size_t)y * pstride] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
            const int y = y0 + j;
            if (y >= H) break;
            sec_update(st[0], cur[j].x, cf);
            sec_update(st[1], cur[j].y, cf);
            sec_update(st[2], cur[j].z, cf);
            sec_update(st[3], cur[j].w, cf);
            float c, s;
            fir32::phase_cs(__ldg(fcol + (size_t)y * a.f_pitch) - a.c0, om_hi, om_lo, c, s);
            float nu = Wk * fmaf(c, sec_causal_out(st[0], cf), s * sec_causal_out(st[1], cf));
            float de = Wk * fmaf(c, sec_causal_out(st[2], cf), s * sec_causal_out(st[3], cf));
            reduce_terms<C>(nu, de);
            if (writer) {
                float2* d = ND + (size_t)y * W;
                if (first) {
                    *d = make_float2(nu, de);
                } else {
                    float2 t = *d;
                    *d = make_float2(t.x + nu, t.y + de);
                }
            }
        }
    }
    // up sweep: anti-causal part
#pragma unroll
    for (int q = 0; q < 4; ++q) st[q] = Sec{0.f, 0.f, 0.f};
    for (int y1 = H - 1; y1 >= 0; y1 -= kChunk) {
        float4 cur[kChunk];
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
            const int y = y1 - j;
            cur[j] = (act && y >= 0) ? P[(size_t)y * pstride] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int j = 0; j < kChunk; ++j) {
            const int y = y1 - j;
            if (y < 0) break;
            const float oA = sec_anti_out(st[0], cf), oB = sec_anti_out(st[1], cf);
            const float oC = sec_anti_out(st[2], cf), oD = sec_anti_out(st[3], cf);
            sec_update(st[0], cur[j].x, cf);
            sec_update(st[1], cur[j].y, cf);
            sec_update(st[2], cur[j].z, cf);
            sec_update(st[3], cur[j].w, cf);
            float c, s;
            fir32::phase_cs(__ldg(fcol + (size_t)y * a.f_pitch) - a.c0, om_hi, om_lo, c, s);
            float nu = Wk * fmaf(c, oA, s * oB);
            float de = Wk * fmaf(c, oC, s * oD);
            reduce_terms<C>(nu, de);
            if (writer) {
                float2* d = ND + (size_t)y * W;
                const float2 t = *d;
                *d = make_float2(t.x + nu, t.y + de);
            }
        }
    }
}

__global__ void k_yvv_final(YvvArgs a)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= a.W) return;
    const SetHdr hd = a.hdr[0];
    for (int y = blockIdx.y; y < a.H; y += gridDim.y) {
        const float fv = a.f[(size_t)y * a.f_pitch + x];
        float v;
        if (hd.F < 0) {
            v = fv;                                  // order above the cap: pass through
        } else {
            const float2 nd = a.nd[(size_t)y * a.W + x];
            if (nd.y > kGuard * (a.mass_y[y] * a.mass_x[x])) {
                v = __fdiv_rn(nd.x, nd.y) + a.c0;
            } else {
                v = fv;
                atomicAdd(a.n_guarded, 1ull);
            }
        }
        a.out[(size_t)y * a.out_pitch + x] = v;
    }
}

}  // namespace

// ---- plan-time design (host, double) ---------------------------------------

bool yvv_design(double sigma, YvvCoef* out, double* poles_c /* [6]: p0, Re p1, Im p1, c0, Re c1, Im c1 */)
{
    if (!(sigma >= 0.5) || !isfinite(sigma)) return false;
    // published coefficients of the recursion (Young and van Vliet 1995)
    const double q = sigma >= 2.5 ? 0.98711 * sigma - 0.96330
                                  : 3.97156 - 4.14554 * sqrt(1.0 - 0.26891 * sigma);
    const double b0 = 1.57825 + q * (2.44413 + q * (1.4281 + q * 0.422205));
    const double b1 = q * (2.44413 + q * (2.85619 + q * 1.26661));
    const double b2 = -q * q * (1.4281 + q * 1.26661);
    const double b3 = 0.422205 * q * q * q;
    const double a1 = b1 / b0, a2 = b2 / b0, a3 = b3 / b0;
    const double B = 1.0 - (a1 + a2 + a3);
    // poles: roots of z^3 - a1 z^2 - a2 z - a3; P(0) = -a3 < 0 < P(1) = B,
    // so one real root lies in (0, 1) (bisection to the last bit); the other
    // two are the roots of the deflated quadratic z^2 + bq z + cq.
    auto P = [&](double z) { return ((z - a1) * z - a2) * z - a3; };
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        (P(mid) < 0.0 ? lo : hi) = mid;
    }
    const double r = 0.5 * (lo + hi);
    const double bq = r - a1, cq = a3 / r;
    const double disc = 4.0 * cq - bq * bq;
    if (!(disc > 0.0)) return false;          // the published design has a complex pair
    using cd = std::complex<double>;
    const cd p[3] = {cd(r, 0.0), cd(-0.5 * bq, 0.5 * sqrt(disc)), cd(-0.5 * bq, -0.5 * sqrt(disc))};
    // 1 / prod_j (1 - p_j / z) = sum_i al_i / (1 - p_i / z), al_i = p_i^2 / prod_{j != i} (p_i - p_j)
    cd al[3];
    for (int i = 0; i < 3; ++i) {
        cd d(1.0, 0.0);
        for (int j = 0; j < 3; ++j)
            if (j != i) d *= p[i] - p[j];
        al[i] = p[i] * p[i] / d;
    }
    // h[n] = B^2 sum_m g[m + n] g[m], g[m] = sum_i al_i p_i^m, gives
    // h[n] = sum_i c_i p_i^n with c_i = B^2 al_i sum_j al_j / (1 - p_i p_j)
    cd c[3];
    for (int i = 0; i < 3; ++i) {
        cd sacc(0.0, 0.0);
        for (int j = 0; j < 3; ++j) sacc += al[j] / (1.0 - p[i] * p[j]);
        c[i] = B * B * al[i] * sacc;
    }
    const cd d1 = c[1] * p[1];
    out->P0 = (float)r;
    out->Pr = (float)p[1].real();
    out->Pi = (float)p[1].imag();
    out->C0 = (float)c[0].real();
    out->Cr = (float)(2.0 * c[1].real());
    out->Ci = (float)(2.0 * c[1].imag());
    out->D0 = (float)(c[0].real() * r);
    out->Dr = (float)(2.0 * d1.real());
    out->Di = (float)(2.0 * d1.imag());
    if (poles_c) {
        poles_c[0] = r;
        poles_c[1] = p[1].real();
        poles_c[2] = p[1].imag();
        poles_c[3] = c[0].real();
        poles_c[4] = c[1].real();
        poles_c[5] = c[1].imag();
    }
    return true;
}

// Filter of the indicator of [0, n) at each of its n samples, in double:
// the causal and anti-causal first-order sections of yvv_design run on ones.
void yvv_line_mass(double sigma, int n, float* mass)
{
    double pc[6];
    YvvCoef k;
    if (!yvv_design(sigma, &k, pc)) return;
    using cd = std::complex<double>;
    const double p0 = pc[0];
    const cd p1(pc[1], pc[2]);
    const double c0 = pc[3];
    const cd c1(pc[4], pc[5]);
    double u0 = 0.0;
    cd u1(0.0, 0.0);
    for (int i = 0; i < n; ++i) {
        u0 = p0 * u0 + 1.0;
        u1 = p1 * u1 + 1.0;
        mass[i] = (float)(c0 * u0 + 2.0 * (c1 * u1).real());
    }
    double v0 = 0.0;
    cd v1(0.0, 0.0);
    for (int i = n - 1; i >= 0; --i) {
        mass[i] = (float)((double)mass[i] + c0 * p0 * v0 + 2.0 * (c1 * p1 * v1).real());
        v0 = p0 * v0 + 1.0;
        v1 = p1 * v1 + 1.0;
    }
}

int yvv_terms_per_pass(int n_terms_cap)
{
    if (n_terms_cap <= 8) return 8;
    if (n_terms_cap <= 16) return 16;
    return 32;
}

cudaError_t launch_yvv(const YvvArgs& a, int C, int n_passes, cudaStream_t s)
{
    const int lines_per_cta = kWarpsPerCta * (32 / C);
    const dim3 block(32 * kWarpsPerCta);
    const dim3 grow((a.H + lines_per_cta - 1) / lines_per_cta);
    const dim3 gcol((a.W + lines_per_cta - 1) / lines_per_cta);
    for (int pass = 0; pass < n_passes; ++pass) {
        switch (C) {
        case 8:
            k_yvv_rows<8><<<grow, block, 0, s>>>(a, pass);
            k_yvv_cols<8><<<gcol, block, 0, s>>>(a, pass);
            break;
        case 16:
            k_yvv_rows<16><<<grow, block, 0, s>>>(a, pass);
            k_yvv_cols<16><<<gcol, block, 0, s>>>(a, pass);
            break;
        case 32:
            k_yvv_rows<32><<<grow, block, 0, s>>>(a, pass);
            k_yvv_cols<32><<<gcol, block, 0, s>>>(a, pass);
            break;
        default:
            return cudaErrorInvalidValue;
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_yvv_final<<<dim3((a.W + 255) / 256, a.H < 65535 ? a.H : 65535), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace bf
